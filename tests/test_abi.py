"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/cpd.h declares, the options struct has the same
layout in C and in the binding, and argument errors are returned before any
CUDA work."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.gpu_common import lib_or_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cpd.h")


@pytest.fixture(scope="module")
def cpd():
    return lib_or_build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cpd_[a-z_0-9]+)\s*\(", text)))


def test_header_functions_are_exported(cpd):
    L = cpd.lib()
    names = declared_functions()
    assert "cpd_create" in names and "cpd_sampled_mttkrp" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(cpd.EXPORTS)


def test_options_layout_matches_c(tmp_path, cpd):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cpd.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cpd_options), offsetof(cpd_options, samples),'
                   'offsetof(cpd_options, seed), offsetof(cpd_options, leaf_rows),'
                   'offsetof(cpd_options, input_on_host), offsetof(cpd_options, reserved_i64),'
                   'offsetof(cpd_options, nnz_sel_capacity), offsetof(cpd_options, deterministic),'
                   'offsetof(cpd_options, duplicate_policy));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    O = cpd.cpd_options
    assert got == [ctypes.sizeof(O), O.samples.offset, O.seed.offset, O.leaf_rows.offset,
                   O.input_on_host.offset, O.reserved_i64.offset, O.nnz_sel_capacity.offset,
                   O.deterministic.offset, O.duplicate_policy.offset]


def test_default_options_and_argument_errors(cpd):
    L = cpd.lib()
    opt = cpd.cpd_options()
    assert L.cpd_default_options(ctypes.byref(opt)) == 0
    assert opt.method == cpd.CPD_ARLS_LEV and opt.rank == 8 and opt.samples == 2000
    assert L.cpd_default_options(None) == 1
    out = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    # N = 0, rank out of range, nonzeros without indices: rejected before
    # touching CUDA (a NULL init_factors is valid: the library draws them)
    assert L.cpd_create(0, ctypes.cast(dims, ctypes.c_void_p), 0, None, None, None, ctypes.byref(opt), None,
                        ctypes.byref(out)) == 1
    bad = cpd.cpd_options()
    L.cpd_default_options(ctypes.byref(bad))
    bad.rank = 129
    assert L.cpd_create(3, ctypes.cast(dims, ctypes.c_void_p), 0, None, None, None, ctypes.byref(bad), None,
                        ctypes.byref(out)) == 1
    assert L.cpd_create(3, ctypes.cast(dims, ctypes.c_void_p), 5, None, None, None, ctypes.byref(opt), None,
                        ctypes.byref(out)) == 1
    assert out.value is None
    assert L.cpd_als_sweep(None, 1) == 1
    assert L.cpd_synchronize(None) == 1
    L.cpd_destroy(None)
