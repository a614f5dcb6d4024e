"""Benchmark: randomized CP-ALS sweeps per second on one GB300 (or N replicas).

Workload (default, the largest single-GPU configuration): 3-mode tensor
8,200,000 x 177,000 x 8,100,000 (the Reddit tensor's dims) with 1e9 distinct
nonzeros, mode indices Zipf(s = 1.3), values log(1 + Poisson(3)), R = 100,
J = 2^17, CP-ARLS-LEV (or STS-CP with --method sts), float32 factors with
float64-accurate Grams, leverage scores and R x R algebra; the coordinates are
drawn on the device.  --workload zipf_1e5cube_50M runs the 1e5^3, 5e7-nonzero
Zipf(1.1), R = 32, J = 65,536 workload.  Data is synthetic and seeded.

A step is one ALS round (Algorithm 1: every mode sampled, MTTKRP'd, solved),
replayed from a captured CUDA graph with inputs resident in HBM.  Between
timed steps L2 is flushed (a 256 MB write), outside the events.

Also reported on the same JSON line: end-to-end sweeps/s through the C ABI
from host buffers (cpd_create from pinned host COO, the sweeps, fit, factors
back to the host), the roofline of the dominant kernel, the FP64 oracle timed
on the host (cpu_baseline), a per-phase breakdown, clocks during the timed
region and the kernel-launch count.

--impl reference times the FP64 oracle on the host cores instead (each step
one mode update of the same workload).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2210_05105_gb300 import synth

METRIC = "ALS sweeps/s"
ORACLE_MAX_NNZ = 60_000_000
FALLBACK_HBM = 6800.0
# float32 lane operations per second (an FMA counts as one): 152 SMs x 128
# FP32 lanes x 2070 MHz; the bound of the df64 and float32 dense kernels
FP32_LANE_TOPS = 152 * 128 * 2.07e9 / 1e12
# float32 operations of one double-float multiply-add term (exact TwoProduct
# 2, TwoSum 6, low-word corrections 2): the Gram and leverage-score terms
DF64_TERM_OPS = 10


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--method", default="arls", choices=["arls", "sts", "exact"])
    p.add_argument("--sketched", action="store_true", help="solve with the Gram of the draws (Fig. 3, bottom)")
    p.add_argument("--fast", action="store_true", help="float32 Grams / leverage scores (precision option 1)")
    p.add_argument("--samples", type=int, default=0, help="override J of the workload")
    p.add_argument("--study-J", default="", help="comma-separated J values: print one line per J (runtime breakdown "
                   "and fit after --steps sweeps), the sample-count study of the paper's Figs. 12-13")
    p.add_argument("--workload", default="zipf_reddit_1B",
                   choices=sorted(synth.WORKLOADS) + sorted(synth.BATCH_WORKLOADS))
    p.add_argument("--branches", type=int, default=16, help="concurrent branches of the batched graph")
    p.add_argument("--leaf-rows", type=int, default=0,
                   help="STS-CP rows per tree leaf F (0: the library's default, the smallest of 8, 16, 32 below R "
                        "whose trees fit in 8 GB, else R)")
    p.add_argument("--autotune", action="store_true", help="run cpd_autotune on the handle before timing")
    p.add_argument("--no-autotune", action="store_true", help="batched workloads: keep the default launch shapes")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-parity", action="store_true", help="skip the oracle parity block of the JSON line")
    p.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    p.add_argument("--cpu-large", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampling every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def allreduce_max(x, world):
    """Max of x over the replicas (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as tdist
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, local_ms):
    """Whole-job sweeps/s of `world` independent replicas that each ran
    `steps` sweeps in local_ms: all sweeps / the slowest replica's time."""
    slowest = allreduce_max(local_ms, world)
    return world * steps / (slowest / 1e3), slowest


def barrier(world):
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()


# ---------------------------------------------------------------- CPU oracle
def cpu_worker(path):
    """Time the FP64 oracle: one ALS round (N mode updates) of the workload."""
    from oracle import cpals as oc
    d = np.load(path, allow_pickle=True)
    meta = json.loads(str(d["meta"]))
    idx, vals = d["idx"], d["vals"]
    init = [d["init%d" % k] for k in range(len(meta["dims"]))]
    modes = meta.get("modes", list(range(len(meta["dims"]))))
    state = oc.als_init(idx, vals, meta["dims"], [u.astype(np.float64) for u in init], meta["method"])
    t0 = time.perf_counter()
    for n in modes:
        oc.als_mode_update(state, n, meta["method"], meta["J"], meta["seed"], 0)
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "mode_updates": len(modes)}))


def parity_check(cpd, h, w, method, idx_np, vals_np, sweep_id, leaf_rows=0, sts_draws=8192):
    """Step-wise parity of the GPU against the FP64 oracle after the timed
    sweeps, from the GPU's current model: the fit formula (Sec. 5.1) on the
    GPU's factors, one mode update's draws (index matches, oracle near-ties
    at 1e-12), the downsampled MTTKRP on the GPU's draws (Eq. 7, relative
    Frobenius error and selected-nonzero count) and the solve (Eq. 4)."""
    import torch
    from oracle import cpals as oc
    dims, R, J = w["dims"], w["R"], w["J"]
    N = len(dims)
    mode = 1 % N
    t0 = time.perf_counter()
    fs = [cpd.cpd_get_factors(h, k).double().cpu().numpy() for k in range(N)]
    sigma = cpd.cpd_get_sigma(h).cpu().numpy()
    fit_gpu = cpd.cpd_fit(h)
    fit_or = oc.fit(idx_np, vals_np, fs, sigma)
    out = {"kind": "one mode update of the oracle from the GPU's factors after the timed sweeps", "mode": mode,
           "fit_gpu": fit_gpu, "fit_oracle": fit_or, "fit_gap": abs(fit_gpu - fit_or)}
    if method == "exact":
        Y = cpd.cpd_exact_mttkrp(h, mode)
        Yo = oc.exact_mttkrp(idx_np, vals_np, dims, fs, mode)
        out["mttkrp_rel_err"] = float(np.linalg.norm(Y.double().cpu().numpy() - Yo) / np.linalg.norm(Yo))
    else:
        Jd = J if method == "arls" else min(J, sts_draws)
        gi, gp = cpd.cpd_leverage_sample(h, mode, Jd, sweep_id)
        if method == "arls":
            oi, op, near = oc.arls_draw([oc.arls_build(U) for U in fs], mode, Jd, w["sample_seed"], sweep_id)
        else:
            oi, op, near = oc.sts_draw([oc.sts_build(U, leaf_rows or R) for U in fs], fs, [oc.gram(U) for U in fs],
                                       mode, Jd, w["sample_seed"], sweep_id)
        gi_np = gi.cpu().numpy()
        mism = np.any(gi_np != oi, axis=0)
        ok = ~mism
        gp_np = gp.cpu().numpy()
        wts = 1.0 / (Jd * gp)
        Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, gi, wts)
        Yg = Y.double().cpu().numpy()
        Yo = oc.sampled_mttkrp(idx_np, vals_np, dims, fs, mode, gi_np, wts.cpu().numpy())
        out.update({"draws": Jd, "index_match": int(ok.sum()), "ties": int(near.sum()),
                    "differ_away_from_tie": int((mism & ~near).sum()),
                    "prob_max_rel_err": float(np.max(np.abs(gp_np[ok] - op[ok]) / op[ok])) if ok.any() else None,
                    "mttkrp_rel_err": float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo)),
                    "nnz_sel_gpu": nsel, "nnz_sel_oracle": oc.selected_nnz(idx_np, dims, mode, gi_np)})
    G = oc.hadamard_of_grams([oc.gram(U) for U in fs], mode)
    Un, _ = oc.solve_and_renorm(Y.double().cpu().numpy(), oc.pinv_sym(G))
    cpd.cpd_gram_solve(h, mode, Y)
    Ug = cpd.cpd_get_factors(h, mode).double().cpu().numpy()
    out["solve_rel_err"] = float(np.linalg.norm(Ug - Un) / np.linalg.norm(Un))
    out["seconds"] = time.perf_counter() - t0
    torch.cuda.synchronize()
    return out


def parity_check_large(cpd, h, w, method, idx, vals, sweep_id, nrows=512):
    """Parity of one mode update at a size where the oracle cannot take the
    whole tensor (the billion-scale workload): the oracle's CP-ARLS-LEV draws
    from the GPU's factors (all J; Algorithm 3), and the downsampled MTTKRP
    (Eq. 7) and the solve (Eq. 4) on `nrows` random output rows, whose
    nonzeros are picked out of the device COO with torch.  STS-CP draws and
    the fit are not compared here: the oracle's tree of 2^18 node Grams of
    R x R float64 and its dense per-nonzero model matrix do not fit a bounded
    sample."""
    import torch
    from oracle import cpals as oc
    dims, R, J = w["dims"], w["R"], w["J"]
    N = len(dims)
    mode = 1 % N
    t0 = time.perf_counter()
    fs = [cpd.cpd_get_factors(h, k).double().cpu().numpy() for k in range(N)]
    out = {"kind": "one mode update of the oracle from the GPU's factors after the timed sweeps; MTTKRP and solve "
                   "on %d random output rows" % nrows, "mode": mode, "fit_gpu": cpd.cpd_fit(h), "fit_oracle": None}
    if method == "arls":
        gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep_id)
        smp = [oc.arls_build(U) if k != mode else None for k, U in enumerate(fs)]
        oi, op, near = oc.arls_draw(smp, mode, J, w["sample_seed"], sweep_id, tie_tol="conditioned")
        out["tie_window"] = "max(1e-12, 8 cond(G_k) 2^-53) C_k; cond(G_k) = %s" % (
            ["%.3g" % oc.gram_condition(x["G"]) for x in smp if x is not None])
        gi_np = gi.cpu().numpy()
        mism = np.any(gi_np != oi, axis=0)
        ok = ~mism
        gp_np = gp.cpu().numpy()
        out.update({"draws": J, "index_match": int(ok.sum()), "ties": int(near.sum()),
                    "differ_away_from_tie": int((mism & ~near).sum()),
                    "prob_max_rel_err": float(np.max(np.abs(gp_np[ok] - op[ok]) / op[ok])) if ok.any() else None})
    else:
        gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep_id)
        gi_np = gi.cpu().numpy()
    wts = 1.0 / (J * gp)
    Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, gi, wts)
    rng = np.random.default_rng(99)
    rows = np.sort(rng.choice(dims[mode], size=min(nrows, dims[mode]), replace=False))
    rows_t = torch.from_numpy(rows).to(idx.device)
    sel = torch.isin(idx[mode].long(), rows_t)
    sub_idx = idx[:, sel].cpu().numpy()
    sub_vals = vals[sel].cpu().numpy()
    Yo = oc.sampled_mttkrp(sub_idx, sub_vals, dims, fs, mode, gi_np, wts.cpu().numpy())[rows]
    Yg = Y.double().cpu().numpy()
    out.update({"mttkrp_rows": int(rows.size), "mttkrp_rows_nonzeros": int(sub_vals.size),
                "mttkrp_rel_err": float(np.linalg.norm(Yg[rows] - Yo) / np.linalg.norm(Yo)) if np.any(Yo) else 0.0,
                "nnz_sel_gpu": nsel})
    G = oc.hadamard_of_grams([oc.gram(U) for U in fs], mode)
    Un, _ = oc.solve_and_renorm(Yg, oc.pinv_sym(G))
    cpd.cpd_gram_solve(h, mode, Y)
    Ug = cpd.cpd_get_factors(h, mode).double().cpu().numpy()
    out["solve_rel_err"] = float(np.linalg.norm(Ug[rows] - Un[rows]) / np.linalg.norm(Un[rows]))
    out["seconds"] = time.perf_counter() - t0
    return out


def cpu_worker_large(path):
    """Time pieces of one oracle ALS round on bounded samples of a workload too
    large for the oracle as a whole, and extrapolate linearly: the downsampled
    MTTKRP of mode 0 on the first S nonzeros (x nnz / S, x N modes), the
    CP-ARLS-LEV sampler build and the solve on the first m rows of the largest
    factor (x the total rows of all factors)."""
    from oracle import cpals as oc
    d = np.load(path, allow_pickle=True)
    meta = json.loads(str(d["meta"]))
    dims, R, nnz = meta["dims"], meta["R"], meta["nnz"]
    N = len(dims)
    idx, vals = d["idx"], d["vals"]
    m = int(meta["rows"])
    if "samp_idx" in d:
        # the GPU's draws and factors
        factors = [np.load(path + ".f%d.npy" % k) if k != 0 else np.zeros((1, R)) for k in range(N)]
        factors = [np.asarray(f, dtype=np.float64) for f in factors]
        samp_idx, wts, t_draw = d["samp_idx"], d["w"], 0.0
        U = np.asarray(np.load(path + ".big.npy"), dtype=np.float64)
    else:
        # the oracle's own samplers and draws over the first m rows of each
        # factor (N(0, 1) rows), a bounded stand-in for full-height factors
        rng = np.random.default_rng(int(meta["seed"]))
        factors = [rng.standard_normal((min(m, dims[k]), R)) for k in range(N)]
        samplers = [oc.arls_build(U) for U in factors]
        t0 = time.perf_counter()
        samp_idx, p, _ = oc.arls_draw(samplers, 0, int(meta["J"]), int(meta["seed"]), 0)
        t_draw = time.perf_counter() - t0
        wts = oc.sample_weights(p, int(meta["J"]))
        U = factors[int(np.argmax(dims))]
    t0 = time.perf_counter()
    oc.sampled_mttkrp(idx, vals, dims, factors, 0, samp_idx, wts)
    t_mttkrp = time.perf_counter() - t0
    m = U.shape[0]
    t0 = time.perf_counter()
    st = oc.arls_build(U)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    oc.solve_and_renorm(U, st["Gpinv"])
    t_solve = time.perf_counter() - t0
    S = idx.shape[1]
    round_s = N * (t_mttkrp * (nnz / S) + t_draw) + (t_build + t_solve) * (sum(dims) / m)
    print(json.dumps({"seconds": round_s, "t_mttkrp_sample": t_mttkrp, "nnz_sample": S, "t_build": t_build,
                      "t_solve": t_solve, "t_draw": t_draw, "rows_sample": m}))


def run_oracle_large(idx_h, vals_h, samp, w, threads, S=20_000_000, rows=400_000):
    """samp = (GPU draws, weights, GPU factors), or None: the oracle draws from
    its own samplers on the first `rows` rows of N(0, 1) factors."""
    dims = w["dims"]
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "case.npz")
        meta = {"dims": list(dims), "R": w["R"], "nnz": w["nnz"], "rows": rows, "J": w["J"],
                "seed": w["sample_seed"]}
        if samp is not None:
            samp_idx, wts, fs = samp
            np.savez(path, idx=idx_h[:, :S].numpy(), vals=vals_h[:S].numpy(), samp_idx=samp_idx, w=wts,
                     meta=json.dumps(meta))
            for k, f in enumerate(fs):
                if k != 0:
                    np.save(path + ".f%d.npy" % k, f)       # factors read by mode 0's MTTKRP
            np.save(path + ".big.npy", fs[int(np.argmax(dims))][:rows])
        else:
            np.savez(path, idx=idx_h[:, :S].numpy(), vals=vals_h[:S].numpy(), meta=json.dumps(meta))
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
        env["CUDA_VISIBLE_DEVICES"] = ""
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", path, "--cpu-large"], env=env,
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        res = json.loads(r.stdout.strip().splitlines()[-1])
    draws = ("the GPU's %d draws" % w["J"]) if samp is not None else \
        ("%d draws of its own samplers over the first %d rows of each factor (%.2f s each)" % (w["J"], rows,
                                                                                             res["t_draw"]))
    return {"value": 1.0 / res["seconds"], "unit": "sweeps/s", "cores": threads, "kind": "oracle",
            "extrapolated": True, "seconds": res["seconds"],
            "sample": "extrapolated ALS round: the oracle's downsampled MTTKRP of mode 0 on the first %d nonzeros "
                      "with %s (%.2f s, x nnz / %d x %d modes) plus its CP-ARLS-LEV sampler build and "
                      "solve on %d rows of the largest factor (x all rows); FP64 numpy, %d BLAS threads"
                      % (S, draws, res["t_mttkrp_sample"], S, len(dims), rows, threads)}


def small_fit_parity(method):
    """Whole-run parity on the 200 x 150 x 100 workload (2e4 nonzeros, R = 8,
    J = 2000): 5 ALS rounds on the GPU and in the FP64 oracle from the same
    inputs and uniforms, final fits compared."""
    import torch
    from oracle import cpals as oc
    from paper_2210_05105_gb300 import cpd
    w = synth.WORKLOADS["small_uniform_200x150x100"]
    dims, R, J, S = w["dims"], w["R"], w["J"], w["sweeps"]
    idx, vals = synth.make_tensor(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"])
    init = synth.init_factors(dims, R, w["init_seed"])
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method=method, rank=R, samples=J,
                       seed=w["sample_seed"])
    cpd.cpd_als_sweep(h, S)
    f_gpu = cpd.cpd_fit(h)
    h.close()
    _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], method, S, J=J, seed=w["sample_seed"])
    return {"workload": "small_uniform_200x150x100", "sweeps": S, "fit_gpu": f_gpu, "fit_oracle": fits[-1],
            "fit_gap": abs(f_gpu - fits[-1])}


def run_oracle(idx, vals, init, w, method, modes, threads=1):
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "case.npz")
        meta = {"dims": list(w["dims"]), "J": w["J"], "seed": w["sample_seed"], "method": method, "modes": modes}
        np.savez(path, idx=idx, vals=vals, meta=json.dumps(meta), **{"init%d" % k: u for k, u in enumerate(init)})
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
        env["CUDA_VISIBLE_DEVICES"] = ""
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", path], env=env,
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------ byte models
def algorithmic(phase, w, stats, fast=False):
    """Algorithmic bytes (or float32 lane operations) per launch of a phase's
    kernel.  fast: precision option 1, whose Gram and leverage terms are float32
    (one FMA a Gram term; a multiply and an FMA a leverage term)."""
    N, R, J = len(w["dims"]), w["R"], w["J"]
    Rp = (R + 3) // 4 * 4
    if phase == "spmm":
        # selected (row, value) pairs, weight + offsets per distinct column,
        # its KRP row, one write of every touched output row
        return "hbm", stats["nnz_sel"] * 8 + stats["J_u"] * (R * 4 + 16) + stats["rows"] * R * 4
    if phase == "probe":
        return "hbm", J * (N - 1) * 4 + J * 8 + stats["J_u"] * ((N - 1) * R * 4 + R * 4) + J * 16
    if phase in ("sampler", "gram"):
        # df64 terms of the quadratic forms (leverage scores) or Gram pairs,
        # R(R+1)/2 per row, as float32 lane operations
        ops = (2 if phase == "sampler" else 1) if fast else DF64_TERM_OPS
        return "alu", stats["I_mean"] * R * (R + 1) / 2 * ops
    if phase == "solve":
        # Y G+ with G+ rounded to float32: R^2 FMAs a row
        return "alu", stats["I_mean"] * R * R
    if phase == "exact":
        # every nonzero: N indices + value, N - 1 factor rows, one output row update
        nnz = w["nnz"]
        return "hbm", nnz * (N * 4 + 4) + nnz * (N - 1) * R * 4 + stats["I_mean"] * R * 4
    return "hbm", 0


# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernel (`dram__bytes_read.sum + dram__bytes_write.sum`, mean over the mode updates of a timed round of
# the same command line), keyed by (workload, method, phase).
TRAFFIC_BYTES = {("zipf_1e5cube_50M", "arls", "spmm"): 67.45e6}


def profile_round(cpd, h, w, method, sweep_id):
    """One ALS round through the step-wise entry points with the phase timers
    on: -> ({phase: (ms, launches)}, per-mode MTTKRP statistics)."""
    import torch
    dims, J = w["dims"], w["J"]
    N = len(dims)
    cpd.cpd_profile(h, True)
    stats = {"nnz_sel": 0, "J_u": 0, "rows": 0, "I_mean": sum(dims) / N}
    per_mode = []
    for n in range(N):
        if method == "exact":
            Y = cpd.cpd_exact_mttkrp(h, n)
            cpd.cpd_gram_solve(h, n, Y)
            per_mode.append(cpd.cpd_profile_read(h))
            continue
        gi, gp = cpd.cpd_leverage_sample(h, n, J, sweep_id)
        wts = 1.0 / (J * gp)
        Y, nsel = cpd.cpd_sampled_mttkrp(h, n, gi, wts)
        cpd.cpd_gram_solve(h, n, Y)
        per_mode.append(cpd.cpd_profile_read(h))
        keys = torch.zeros(J, dtype=torch.int64, device="cuda")
        mult = 1
        for k in range(N):
            if k != n:
                keys += gi[k].long() * mult
                mult *= dims[k]
        stats["nnz_sel"] += nsel
        stats["J_u"] += int(torch.unique(keys).numel())
        stats["rows"] += int((Y != 0).any(dim=1).sum())
    cpd.cpd_profile(h, False)
    phases = {}
    for ph in per_mode:
        for k, (ms, n_) in ph.items():
            a, b = phases.get(k, (0.0, 0))
            phases[k] = (a + ms, b + n_)
    for k in ("nnz_sel", "J_u", "rows"):
        stats[k] = stats[k] / N          # per mode update
    return phases, stats


def workload(args):
    w = dict(synth.WORKLOADS[args.workload])
    if args.samples:
        w["J"] = args.samples
    return w


def study_J(args):
    """Runtime breakdown and fit against the sample count J (Figs. 12-13)."""
    import torch
    from paper_2210_05105_gb300 import cpd
    w = workload(args)
    dims, R = w["dims"], w["R"]
    N = len(dims)
    idx, vals = synth.make_tensor_torch(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"], device="cuda")
    init = [torch.from_numpy(u).cuda() for u in synth.init_factors(dims, R, w["init_seed"])]
    for J in [int(x) for x in args.study_J.split(",")]:
        h = cpd.cpd_create(dims, idx, vals, init, method=args.method, rank=R, samples=J, seed=w["sample_seed"],
                           sketched_gram=args.sketched, fast=args.fast)
        cpd.cpd_als_sweep(h, args.warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        cpd.cpd_als_sweep(h, args.steps, sync=False)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        fit = cpd.cpd_fit(h)
        cpd.cpd_profile(h, True)
        nsel = 0
        for n in range(N):
            gi, gp = cpd.cpd_leverage_sample(h, n, J, args.warmup + args.steps)
            Y, ns = cpd.cpd_sampled_mttkrp(h, n, gi, 1.0 / (J * gp))
            nsel += ns
            cpd.cpd_gram_solve(h, n, Y)
        ph = cpd.cpd_profile_read(h)
        h.close()
        groups = {"sampling": ["draw", "pinv"], "mttkrp": ["clear", "probe", "scan", "spmm"],
                  "post-processing": ["solve", "gram", "sampler"]}
        print(json.dumps({"study": "sample count", "workload": args.workload, "method": args.method,
                          "sketched_gram": args.sketched, "J": J, "ms_per_sweep": ms,
                          "fit_after_%d_sweeps" % (args.warmup + args.steps): fit,
                          "nnz_sel_per_mode": nsel / N,
                          "phase_ms_per_sweep": {g: round(sum(ph[k][0] for k in ks), 4) for g, ks in groups.items()}}))


def ours(args, world, rank, local):
    import torch
    from paper_2210_05105_gb300 import cpd
    torch.cuda.set_device(local)
    if args.study_J:
        study_J(args)
        return
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    w = workload(args)
    dims, R, J = w["dims"], w["R"], w["J"]
    N = len(dims)
    gen_s = draws_used = None
    t0 = time.perf_counter()
    if w.get("generator") == "device":
        # billion-scale: coordinates drawn on the device, N(0, 1) initial
        # factors drawn by the library from the seed (init_factors = NULL)
        idx, vals, draws_used = synth.make_tensor_device(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"])
        init_np, init = None, None
    else:
        idx, vals = synth.make_tensor_torch(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"], device="cuda")
        init_np = synth.init_factors(dims, R, w["init_seed"])
        init = [torch.from_numpy(u).cuda() for u in init_np]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    large = w["nnz"] > ORACLE_MAX_NNZ
    t0 = time.perf_counter()
    h = cpd.cpd_create(dims, idx, vals, init, method=args.method, rank=R, samples=J, seed=w["sample_seed"],
                       sketched_gram=args.sketched, fast=args.fast, leaf_rows=args.leaf_rows)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    tuned = cpd.cpd_autotune(h) if args.autotune else None

    cpd.cpd_als_sweep(h, args.warmup)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = Clocks(local)
    clk.start()
    barrier(world)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        cpd.cpd_als_sweep(h, 1, sync=False)
        stops[i].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    value, total_ms = replica_throughput(world, args.steps, sum(step_ms))
    launches_per_step = cpd.cpd_sweep_kernel_count(h)
    fit = cpd.cpd_fit(h)

    # per-phase breakdown of one round, step-wise entry points (same kernels)
    phases, stats = profile_round(cpd, h, w, args.method, args.warmup + args.steps)
    dominant = max((k for k in phases if phases[k][1] > 0), key=lambda k: phases[k][0])
    hbm_peak, peak_kind = peaks()

    def roof(phase):
        ms, n_ = phases[phase]
        per_launch_ms = ms / max(n_, 1)
        bound, amount = algorithmic(phase, w, stats, fast=args.fast)
        if bound == "alu":
            ach = amount / (per_launch_ms / 1e3) / 1e12
            return {"phase": phase, "bound": "alu", "achieved": ach, "peak": FP32_LANE_TOPS,
                    "unit": "Tops/s (float32 lane operations)", "frac": ach / FP32_LANE_TOPS, "traffic": None,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz", "ms_per_launch": per_launch_ms}
        ach = amount / (per_launch_ms / 1e3) / 1e9
        t = None if (args.fast or args.sketched) else TRAFFIC_BYTES.get((args.workload, args.method, phase))
        return {"phase": phase, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": t, "peak_source": peak_kind, "ms_per_launch": per_launch_ms}

    modelled = [k for k in ("spmm", "exact", "sampler", "gram", "solve") if phases.get(k, (0, 0))[1] > 0]
    roofline_phases = {k: roof(k) for k in modelled}
    # the roofline of the line is the kernel class with the most device time
    top = max(modelled, key=lambda k: phases[k][0])
    roofline = roofline_phases[top]
    roofline_spmm = roofline_phases.get("exact" if args.method == "exact" else "spmm")

    # parity against the FP64 oracle from the GPU's model after the timed sweeps
    parity = None
    idx_np = vals_np = None
    if not args.no_parity and rank == 0:
        if large:
            parity = parity_check_large(cpd, h, w, args.method, idx, vals, args.warmup + args.steps + 1)
        else:
            idx_np, vals_np = idx.cpu().numpy(), vals.cpu().numpy()
            parity = parity_check(cpd, h, w, args.method, idx_np, vals_np, args.warmup + args.steps + 1,
                                  leaf_rows=args.leaf_rows)
            if args.workload != "small_uniform_200x150x100":
                parity["small_workload_run"] = small_fit_parity(args.method)
    samp_for_cpu = None
    if large and not args.no_cpu and rank == 0:
        gi, gp = cpd.cpd_leverage_sample(h, 0, J, args.warmup + args.steps + 2)
        samp_for_cpu = (gi.cpu().numpy(), (1.0 / (J * gp)).cpu().numpy(),
                        [cpd.cpd_get_factors(h, k).cpu().numpy() for k in range(N)])
    h.close()
    torch.cuda.synchronize()

    # end-to-end through the C ABI from pinned host buffers
    e2e = None
    idx_h = vals_h = None
    if not args.no_e2e or (large and not args.no_cpu and rank == 0):
        idx_h = idx.cpu().pin_memory() if not args.no_e2e else idx.cpu()
        vals_h = vals.cpu().pin_memory() if not args.no_e2e else vals.cpu()
    if not args.no_e2e:
        init_h = None if init is None else [u.cpu().pin_memory() for u in init]
        if large:
            del idx, vals
            idx = vals = None
            torch.cuda.empty_cache()
        # pinned destinations of the factors, like the pinned inputs, are the
        # caller's buffers: allocated before the timed job
        outs_h = [torch.empty((dims[k], R), dtype=torch.float32).pin_memory() for k in range(N)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = cpd.cpd_create(dims, idx_h, vals_h, init_h, method=args.method, rank=R, samples=J, seed=w["sample_seed"],
                            sketched_gram=args.sketched, fast=args.fast)
        cpd.cpd_als_sweep(h2, args.steps, sync=False)
        f2 = cpd.cpd_fit(h2)
        outs = [cpd.cpd_get_factors(h2, k, out=outs_h[k]) for k in range(N)]
        e2e_s = time.perf_counter() - t0
        h2.close()
        h2d = idx_h.numel() * 4 + vals_h.numel() * 4 + (0 if init_h is None else sum(u.numel() * 4 for u in init_h))
        d2h = sum(o.numel() * 4 for o in outs) + 8
        e2e_s = allreduce_max(e2e_s, world)
        e2e = {"value": world * args.steps / e2e_s, "unit": "sweeps/s", "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps, "job": "cpd_create(host COO) + %d sweeps + fit + factors to host"
               % args.steps, "job_seconds": e2e_s, "fit": f2}
        del outs

    cpu = cpu1 = None
    if not args.no_cpu and rank == 0 and large:
        cpu = run_oracle_large(idx_h, vals_h, samp_for_cpu, w, threads=os.cpu_count() or 1)
    elif not args.no_cpu and rank == 0:
        if idx_np is None:
            idx_np, vals_np = idx.cpu().numpy(), vals.cpu().numpy()
        ncpu = os.cpu_count() or 1
        res = run_oracle(idx_np, vals_np, init_np, w, args.method, list(range(N)), threads=ncpu)
        res1 = run_oracle(idx_np, vals_np, init_np, w, args.method, list(range(N)), threads=1)
        cpu = {"value": (res["mode_updates"] / N) / res["seconds"], "unit": "sweeps/s", "cores": ncpu,
               "kind": "oracle", "sample": "one ALS round (all %d mode updates) of the full workload, FP64 numpy "
                                          "with %d BLAS threads (numpy's elementwise steps stay on one core), "
                                          "from the initial factors" % (N, ncpu), "seconds": res["seconds"]}
        cpu1 = {"value": (res1["mode_updates"] / N) / res1["seconds"], "unit": "sweeps/s", "cores": 1,
                "kind": "oracle", "sample": "the same ALS round, 1 thread", "seconds": res1["seconds"]}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": args.workload, "dims": list(dims), "nnz": w["nnz"], "zipf_s": w["zipf"],
                           "values": w["values"], "R": R, "J": J, "method": args.method,
                           "sketched_gram": args.sketched, "precision": "fast" if args.fast else "exact-draws",
                           "leaf_rows": args.leaf_rows or "library default", "autotuned": tuned,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed between steps (256 MB write, outside the events)",
                           "generate_seconds": gen_s, "generator_draws": draws_used,
                           "init": "library-drawn N(0,1) from the seed" if init is None else "host N(0,1)",
                           "create_seconds": create_s},
                "roofline": roofline, "roofline_spmm": roofline_spmm, "roofline_phases": roofline_phases,
                "cpu_baseline": cpu,
                "cpu_baseline_1core": cpu1, "parity": parity, "e2e": e2e,
                "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
                "phases_ms_per_sweep": {k: round(v[0], 4) for k, v in phases.items() if v[1]},
                "mttkrp_stats_per_mode": {k: stats[k] for k in ("nnz_sel", "J_u", "rows")},
                "fit": fit, "step_ms_median": statistics.median(step_ms)}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def batch_bench(args, world, rank, local):
    """Many uneven tensors: one graph replays an ALS round of all of them on
    concurrent branches.  value = tensor sweeps per second (T per step); the
    same handles swept one graph after another give sequential_value."""
    import torch
    from paper_2210_05105_gb300 import cpd
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    specs = synth.batch_specs(**synth.BATCH_WORKLOADS[args.workload])
    T = len(specs)
    handles, inputs = [], []
    t0 = time.perf_counter()
    for s in specs:
        idx, vals = synth.make_tensor_torch(s["dims"], s["nnz"], s["data_seed"], s["zipf"], s["values"], device="cuda")
        init = [torch.from_numpy(u).cuda() for u in synth.init_factors(s["dims"], s["R"], s["init_seed"])]
        inputs.append((idx, vals, init))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for s, (idx, vals, init) in zip(specs, inputs):
        handles.append(cpd.cpd_create(s["dims"], idx, vals, init, method=args.method, rank=s["R"], samples=s["J"],
                                      seed=s["sample_seed"], fast=args.fast))
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    choices = [cpd.cpd_autotune(h) for h in handles] if not args.no_autotune else None
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(step_fn):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for _ in range(args.warmup):
            step_fn()
        barrier(world)
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step_fn()
            stops[i].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return [a.elapsed_time(b) for a, b in zip(starts, stops)]

    def seq_step():
        for h in handles:
            cpd.cpd_als_sweep(h, 1, sync=False)

    seq_ms = timed(seq_step)
    b = cpd.cpd_batch_create(handles, branches=args.branches)
    clk = Clocks(local)
    clk.start()
    torch.cuda.nvtx.range_push("timed")
    bat_ms = timed(lambda: cpd.cpd_batch_sweep(b, 1, sync=False))
    torch.cuda.nvtx.range_pop()
    clocks = clk.stop()
    value, total_ms = replica_throughput(world, args.steps * T, sum(bat_ms))
    seq_value, _ = replica_throughput(world, args.steps * T, sum(seq_ms))
    launches = sum(cpd.cpd_sweep_kernel_count(h) for h in handles)
    fits = [cpd.cpd_fit(h) for h in handles]

    # SpMM roofline over one step-wise round of every tensor
    hbm_peak, peak_kind = peaks()
    spmm_ms = spmm_bytes = 0.0
    phases = {}
    for s, h in zip(specs, handles):
        ph, st = profile_round(cpd, h, s, args.method, 1 << 40)
        for k, (ms, n_) in ph.items():
            a_, b_ = phases.get(k, (0.0, 0))
            phases[k] = (a_ + ms, b_ + n_)
        if args.method != "exact":
            spmm_ms += ph["spmm"][0]
            spmm_bytes += algorithmic("spmm", s, st)[1] * len(s["dims"])
    ach = spmm_bytes / (spmm_ms / 1e3) / 1e9 if spmm_ms else 0.0
    roofline = {"phase": "spmm", "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": None, "peak_source": peak_kind,
                "note": "algorithmic bytes of all %d tensors' SpMM launches / their summed time" % T}

    e2e = None
    if not args.no_e2e:
        host = [(i.cpu().pin_memory(), v.cpu().pin_memory(), [u.cpu().pin_memory() for u in ini])
                for i, v, ini in inputs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs2 = [cpd.cpd_create(s["dims"], i, v, ini, method=args.method, rank=s["R"], samples=s["J"],
                              seed=s["sample_seed"], fast=args.fast) for s, (i, v, ini) in zip(specs, host)]
        if choices is not None:
            for hh in hs2:
                cpd.cpd_autotune(hh)
        b2 = cpd.cpd_batch_create(hs2, branches=args.branches)
        cpd.cpd_batch_sweep(b2, args.steps, sync=False)
        f2 = [cpd.cpd_fit(hh) for hh in hs2]
        outs = [[cpd.cpd_get_factors(hh, k, out=torch.empty((s["dims"][k], s["R"]), dtype=torch.float32).pin_memory())
                 for k in range(len(s["dims"]))] for s, hh in zip(specs, hs2)]
        e2e_s = allreduce_max(time.perf_counter() - t0, world)
        b2.close()
        for hh in hs2:
            hh.close()
        h2d = sum(i.numel() * 4 + v.numel() * 4 + sum(u.numel() * 4 for u in ini) for i, v, ini in host)
        d2h = sum(o.numel() * 4 for os_ in outs for o in os_) + 8 * T
        e2e = {"value": world * T * args.steps / e2e_s, "unit": "tensor sweeps/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "job": "%d x cpd_create(host COO) + autotune + batched graph + %d rounds + fits + factors to host"
               % (T, args.steps), "job_seconds": e2e_s, "fit_mean": float(np.mean(f2))}

    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = batch_oracle(specs, inputs, args.method, budget_s=12.0)
    b.close()
    for h in handles:
        h.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "tensor sweeps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": args.workload, "tensors": T, "nnz_total": sum(s["nnz"] for s in specs),
                           "orders": "3 and 4 alternating", "R": "16/32/64", "J": "4096-65536 log-uniform",
                           "method": args.method, "precision": "fast" if args.fast else "exact-draws",
                           "branches": args.branches, "autotuned": choices is not None,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed between steps (256 MB write, outside the events)",
                           "generate_seconds": gen_s, "create_seconds": create_s, "autotune_seconds": tune_s},
                "sequential_value": seq_value, "batched_over_sequential": value / seq_value,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches * args.steps,
                "phases_ms_per_round": {k: round(v[0], 4) for k, v in phases.items() if v[1]},
                "fit_mean": float(np.mean(fits)), "fit_min": float(np.min(fits)),
                "autotune_choices": {"spmm_blocks_per_sm": sorted(set(c[0] for c in choices)) if choices else None,
                                     "sts_lanes_per_draw": sorted(set(c[1] for c in choices)) if choices else None},
                "step_ms_median": statistics.median(bat_ms), "sequential_step_ms_median": statistics.median(seq_ms)}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def batch_oracle(specs, inputs, method, budget_s):
    """The FP64 oracle on a bounded sample of a batched workload: one ALS
    round of each tensor, smallest first, until budget_s of oracle time."""
    order = sorted(range(len(specs)), key=lambda t: specs[t]["nnz"])
    secs, done, nnz = 0.0, 0, 0
    for t in order:
        s = specs[t]
        if inputs is not None:
            idx, vals = inputs[t][0].cpu().numpy(), inputs[t][1].cpu().numpy()
        else:
            idx, vals = synth.make_tensor(s["dims"], s["nnz"], s["data_seed"], s["zipf"], s["values"])
        init = synth.init_factors(s["dims"], s["R"], s["init_seed"])
        res = run_oracle(idx, vals, init, s, method, list(range(len(s["dims"]))))
        secs += res["seconds"]
        done += 1
        nnz += s["nnz"]
        if secs >= budget_s:
            break
    return {"value": done / secs, "unit": "tensor sweeps/s", "cores": 1, "kind": "oracle", "seconds": secs,
            "sample": "one ALS round of the %d smallest of the %d tensors (%d nonzeros), FP64 numpy, 1 thread"
                      % (done, len(specs), nnz)}


def reference(args, world, rank, local):
    """FP64 oracle on the host cores, each step one mode update."""
    if rank != 0:
        return
    import torch
    w = synth.WORKLOADS[args.workload]
    dims = w["dims"]
    N = len(dims)
    if w.get("generator") == "device":
        # billion-scale: each step one bounded, extrapolated ALS round of the
        # oracle (the whole tensor does not fit the oracle's per-nonzero arrays)
        idx_d, vals_d, _ = synth.make_tensor_device(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"])
        S = 5_000_000
        idx_h, vals_h = idx_d[:, :S].cpu(), vals_d[:S].cpu()
        del idx_d, vals_d
        torch.cuda.empty_cache()
        ncpu = os.cpu_count() or 1
        for _ in range(args.warmup):
            run_oracle_large(idx_h, vals_h, None, w, ncpu, S=S, rows=100_000)
        res = [run_oracle_large(idx_h, vals_h, None, w, ncpu, S=S, rows=100_000) for _ in range(args.steps)]
        sec = float(np.mean([r["seconds"] for r in res]))
        value = 1.0 / sec
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "dims": list(dims), "nnz": w["nnz"], "R": w["R"], "J": w["J"],
                           "method": args.method, "step": "one extrapolated ALS round of the FP64 oracle"},
                "cpu_baseline": {"kind": "oracle", "cores": ncpu, "value": value, "extrapolated": True,
                                 "sample": res[-1]["sample"]},
                "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if torch.cuda.is_available():
        idx, vals = synth.make_tensor_torch(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"], device="cuda")
        idx, vals = idx.cpu().numpy(), vals.cpu().numpy()
    else:
        idx, vals = synth.make_tensor(dims, w["nnz"], w["data_seed"], w["zipf"], w["values"])
    init = synth.init_factors(dims, w["R"], w["init_seed"])
    modes_w = [k % N for k in range(args.warmup)]
    modes_t = [k % N for k in range(args.steps)]
    if modes_w:
        run_oracle(idx, vals, init, w, args.method, modes_w)
    res = run_oracle(idx, vals, init, w, args.method, modes_t)
    value = (len(modes_t) / N) / res["seconds"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["seconds"] * 1e3 / max(len(modes_t), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(dims), "nnz": w["nnz"], "R": w["R"], "J": w["J"],
                       "method": args.method, "step": "one mode update of the FP64 oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value,
                             "sample": "%d mode updates of the full workload, FP64 numpy, 1 thread" % len(modes_t)},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batch_reference(args, world, rank, local):
    """Reference arm of a batched workload: the FP64 oracle, each step one ALS
    round of a bounded sample of the tensors (smallest first)."""
    if rank != 0:
        return
    specs = synth.batch_specs(**synth.BATCH_WORKLOADS[args.workload])
    for _ in range(args.warmup):
        batch_oracle(specs, None, args.method, budget_s=2.0)
    vals = [batch_oracle(specs, None, args.method, budget_s=8.0) for _ in range(args.steps)]
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tensor sweeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "tensors": len(specs), "method": args.method,
                       "step": "one ALS round of the smallest tensors of the batch, FP64 oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": "tensor sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.cpu_worker:
        (cpu_worker_large if args.cpu_large else cpu_worker)(args.cpu_worker)
        return
    world, rank, local = dist()
    batched = args.workload in synth.BATCH_WORKLOADS
    if args.impl == "reference":
        (batch_reference if batched else reference)(args, world, rank, local)
    else:
        (batch_bench if batched else ours)(args, world, rank, local)


if __name__ == "__main__":
    main()
