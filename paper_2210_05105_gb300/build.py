"""Build libcpd.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_2210_05105_gb300/libcpd.so (git-ignored).  Run ``python -m
paper_2210_05105_gb300.build`` or call :func:`build`.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
GENSRC = os.path.join(HERE, "gen")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcpd.so")
GENLIB = os.path.join(HERE, "libzipfgen.so")   # input generator, separate from the method's library
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources(d=CSRC):
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".cu"))


def _compile(nvcc, src, extra):
    obj = os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose=False, extra=()):
    """Compile every CUDA source and link libcpd.so; returns the library path."""
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = sources()
    gsrcs = sources(GENSRC)
    with cf.ThreadPoolExecutor(max_workers=min(12, len(srcs) + len(gsrcs))) as ex:
        results = list(ex.map(lambda s: _compile(nvcc, s, list(extra)), srcs + gsrcs))
    objs = [o for o, _ in results[:len(srcs)]]
    gobjs = [o for o, _ in results[len(srcs):]]
    if verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    for lib, ob in ((LIB, objs), (GENLIB, gobjs)):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *ob]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
