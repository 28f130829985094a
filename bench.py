#!/usr/bin/env python3
"""Throughput of the extra-component apply (forward + adjoint) on one node.

One step = for every plan of the workload: y = A x (xc_apply) and x = A^T y
(xc_apply_adjoint) over the workload's right-hand sides, inputs resident in
HBM.  Default workload: Chebyshev T_k at 4096 Chebyshev-Gauss points and
Laguerre functions at 4096 Gauss-Laguerre nodes, eps = 1e-12, FP64, 64
standard-normal right-hand sides.

Prints one JSON line (rank 0).  `value` counts vector applies (one right-hand
side through one direction of one plan) per second over all ranks; ranks are
independent replicas (weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import math
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_11610_gb300 import inputs  # noqa: E402

METRIC = "vectors/s and HBM GB/s (fraction of peak) vs GPU direct dense GEMM at stated rel-l2 error"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x FP64 FMA/clk/SM x 2 flops x max SM clock
# band products of XC_FP64_PAIR plans: 12 FP32 instructions per pair multiply-add (2 algorithmic flops)
PAIR_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 6 / 1e12
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("xc", "reference"), default="xc")
    ap.add_argument("--workload", default="cheb_lag4096_fp64", choices=sorted(inputs.WORKLOADS) + ["batch1000"])
    ap.add_argument("--nplans", type=int, default=1000, help="plans of the batch workload")
    ap.add_argument("--batch-schedule", default="",
                    help="rpw_f,rpw_a,lockstep_f,lockstep_a: a fixed batch schedule instead of the tuner (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the precision variant (XC_FP64_PAIR of FP64 workloads, XC_FP64 of FP32 ones)")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the FP32 configurations and the 1000-plan batch")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------- workload
def plan_specs(wl):
    out = []
    for i, (fam, N, params) in enumerate(wl["plans"]):
        out.append(dict(family=fam, N=N, params=params, index=i))
    return out


def plan_label(fam, N, params):
    return f"{fam} N={N}" + "".join(f" {k}={v}" for k, v in sorted(params.items()))


def laguerre_transform_nodes(N, eta):
    """The Laguerre transform's points x_i = eta t_i, t_i = 12 (i + 1) / (N - 1)
    (Section 5.3's t_i = 12 i / (N - 1), i = 1..N)."""
    h = 12.0 * eta / (N - 1)
    return h * (1.0 + np.arange(N))


def make_xc_plan(xc, fam, N, params, eps, precision):
    if params.get("scheme") == "2d":
        nodes = laguerre_transform_nodes(N, params["eta"]) if fam in ("laguerre", "hermite") else None
        return xc.Plan(fam, N, eps, precision=precision, nodes=nodes, scheme="2d")
    return xc.Plan(fam, N, eps, precision=precision, alpha=params.get("alpha", 0.0), beta=params.get("beta", 0.0))


def oracle_apply_pair(fam, N, params, eps, precision):
    """(forward, adjoint) of the oracle's plan for one plan of a workload, with
    the library's schedule (eps2 default of the precision)."""
    from oracle import families as F
    from oracle import method as M
    prec = "fp64" if precision == "fp64pair" else precision
    if params.get("scheme") == "2d":
        from oracle import method2d as M2
        h = 12.0 * params["eta"] / (N - 1)
        P = M2.build(M2.Spec2D(fam, N, h, h), eps, eps2=M.default_eps2(prec))
        return (lambda X: M2.apply(P, X)), (lambda Y: M2.apply_adjoint(P, Y))
    sp = F.make_spec(fam, N, params.get("alpha", 0.0), params.get("beta", 0.0))
    P = M.build(sp, eps, precision=prec)
    return (lambda X: M.apply(P, X)), (lambda Y: M.apply_adjoint(P, Y))


def workload_config(name, wl):
    return {
        "workload": name,
        "plans": [plan_label(fam, N, p) for fam, N, p in wl["plans"]],
        "nodes": ("angles: arc midpoints (2n+1-N) pi/N (exp), psi_j = 2 arctan(2 k_j/eta) - pi "
                  "(spectral Laguerre)" if any(f in ("exp", "lagspec") for f, _, _ in wl["plans"])
                  else "Gauss nodes of each family (Chebyshev-Gauss for Chebyshev)"),
        "eps": wl["eps"], "precision": wl["precision"], "nrhs": wl["nrhs"], "input": wl["dist"],
        "step": "forward + adjoint apply of every plan",
        "l2": "flushed before every timed step (256 MiB write)",
    }


COMPLEX_FAMILY_IDS = (7, 8)   # exp, spectral Laguerre
SCHEME_2D = 3


def algorithmic_work(info, nrhs, precision, chunked=False):
    """Per kernel: algorithmic flops and bytes of one launch.  Bytes: the
    kept band values read once per launch (the 2-D CSR also its index words),
    the vectors and spectra read and written once per right-hand side.  Flops
    per right-hand side: 4 per kept element of a real plan (complex value times
    complex spectrum, real part kept), 8 for complex plans and the 2-D CSR,
    2.5 L log2 L per real FFT of length L (5 L log2 L complex), 2 per element
    of a dense tail or rectangle.  A chunked forward product (plans with long bands) leaves the dense tail
    and the output to the reduction kernel; its partial sums are scratch, not
    algorithmic traffic."""
    eb = 8 if precision in ("fp64", "fp64pair") else 4
    nnz = sum(info["nnz"])
    N, mt = info["N"], info["m_tail"]
    if info.get("scheme") == SCHEME_2D:
        # per direction: input transforms, CSR product (2 complex values and an
        # index per entry, 8 real flops per entry and RHS), output transforms,
        # combine (dense rectangles: 2 flops per element and RHS)
        nnz2, de = info["nnz2d"], info["dense_elems2d"]
        return {
            "fft_in_2d": (0.0, nrhs * N * eb),
            "sparse_2d": (8.0 * nnz2 * nrhs, nnz2 * (4 * eb + 4)),
            "fft_out_2d": (0.0, nrhs * N * eb),
            "combine_2d": (2.0 * de * nrhs, de * eb + 2 * nrhs * N * eb),
        }
    if info.get("family") in COMPLEX_FAMILY_IDS:
        # complex vectors and values (2 eb per element), full spectrum of L
        # bins, 8 real flops per complex multiply-add, 5 L log2 L per FFT
        ce, L = 2 * eb, info["L"][0]
        cfft = 5.0 * L * math.log2(L) * nrhs
        return {
            "fwd_fft": (cfft, nrhs * (N + L) * ce),
            "fwd_sparse": (8.0 * nnz * nrhs, nnz * ce + nrhs * (L + N) * ce),
            "row_scale": (6.0 * N * nrhs, N * ce + 2 * nrhs * N * ce),
            "adj_sparse": (8.0 * nnz * nrhs, nnz * ce + nrhs * (N + L) * ce),
            "adj_fft": (cfft, nrhs * (L + N) * ce),
        }
    fft_flops = sum(2.5 * L * math.log2(L) for L in info["L"]) * nrhs
    H = sum(L // 2 + 1 for L in info["L"])
    if chunked:
        fwd_sparse = (nrhs * 4.0 * nnz, nnz * 2 * eb + nrhs * H * 2 * eb)
    else:
        fwd_sparse = (nrhs * (4.0 * nnz + 2.0 * N * mt), nnz * 2 * eb + nrhs * (H * 2 * eb + N * eb + mt * eb))
    return {
        "fwd_fft": (fft_flops, nrhs * (N * eb + H * 2 * eb)),
        "fwd_sparse": fwd_sparse,
        "fwd_reduce": (nrhs * 2.0 * N * mt, N * mt * eb + nrhs * (N * eb + mt * eb)),
        "adj_sparse": (nrhs * 4.0 * nnz, nnz * 2 * eb + nrhs * (N * eb + H * 2 * eb)),
        "adj_fft": (fft_flops, nrhs * (H * 2 * eb + N * eb)),
        "adj_tail": (nrhs * 2.0 * N * mt, N * mt * eb + nrhs * N * eb),
        # layout change only (y -> its transpose, RHS padded to 8): no flops
        "adj_transpose": (0.0, N * eb * (nrhs + (nrhs + 7) // 8 * 8)),
        # per-RHS scaling of FP64 pair plans: read the vector (adjoint: write its pairs)
        "pair_scale": (0.0, 2.0 * N * eb * nrhs),
        # row factors of the complex spectral Laguerre matrix (not run by real plans)
        "row_scale": (0.0, 0.0),
        # kernels of the 2-D block scheme (not run by 1-D plans)
        "fft_in_2d": (0.0, 0.0), "sparse_2d": (0.0, 0.0), "fft_out_2d": (0.0, 0.0), "combine_2d": (0.0, 0.0),
    }


def step_bytes(info, nrhs, precision):
    """Algorithmic HBM bytes of one forward + adjoint apply of one plan."""
    eb = 8 if precision in ("fp64", "fp64pair") else 4
    if info.get("family") in COMPLEX_FAMILY_IDS:   # complex vectors, full spectrum
        ce, L = 2 * eb, info["L"][0]
        return info["matrix_bytes"] + info["adjoint_bytes"] + 4 * nrhs * info["N"] * ce + 2 * 2 * nrhs * L * ce
    H = sum(L // 2 + 1 for L in info["L"])
    vec = 4 * nrhs * info["N"] * eb                    # x in, y out, y in, x out
    spec = 2 * 2 * nrhs * H * 2 * eb                   # spectra written + read, both directions
    return info["matrix_bytes"] + info["adjoint_bytes"] + vec + spec


# ------------------------------------------------------------------ ranks
def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank number over all ranks (the slowest replica sets
    the job's time).  Works with any torch.distributed backend."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_per_step: float, steps: int, max_ms: float, world: int) -> float:
    """Whole-job units per second: every rank processes its own units
    (replicas, weak scaling), the job takes the slowest rank's time."""
    return world * units_per_rank_per_step * steps / (max_ms / 1e3)


# ------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [c.strip() for c in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- cpu oracle
def _ref_step(args):
    """Worker of the reference arm: one step's share (forward + adjoint of
    every plan on its own right-hand side), started together by the barrier."""
    _POOL_STATE["barrier"].wait(timeout=900)
    t0 = time.perf_counter()
    for fwd, adj, X in _POOL_STATE["plans"]:
        adj(fwd(X))
    return time.perf_counter() - t0


def run_reference(args, rank, world):
    """The FP64 oracle as it stands, timed on the host cores: one
    single-threaded process per core, each applying forward + adjoint of every
    plan of the workload to one right-hand side of its own per step; a step
    ends when every process has finished its share."""
    if rank != 0:
        return
    if args.workload == "batch1000":
        # bounded sample: the first plans of the batch with N <= 1024
        sample = [w for w in inputs.batch_workload(args.nplans) if w[1] <= 1024][:4]
        wl = {"plans": [(f, N, p) for f, N, p, _ in sample], "eps": 1e-7, "precision": "fp32", "nrhs": 1,
              "dist": "normal"}
    else:
        wl = inputs.WORKLOADS[args.workload]
    n = host_cores()
    with oracle_pool(n, wl["plans"], wl["eps"], wl["precision"], wl["dist"], 1) as pool:
        for _ in range(args.warmup):
            pool.map(_ref_step, [None] * n, chunksize=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_ref_step, [None] * n, chunksize=1)
        el = time.perf_counter() - t0
    vectors = args.steps * len(wl["plans"]) * 2 * n
    value = vectors / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": (workload_config(args.workload, wl) if args.workload != "batch1000" else {"workload": "batch1000"})
        | {"sample": f"1 right-hand side per plan, direction and process per step, {n} processes"
           + ("" if args.workload != "batch1000" else "; 4 plans of the batch with N <= 1024")},
        "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": n, "kind": "oracle",
                         "sample": f"1 RHS per plan and process per step, forward + adjoint, {n} single-threaded "
                                   "numpy/scipy processes"},
        "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU path
KERNEL_SOURCES = ("xc_items.cuh", "xc_apply.cu", "xc_batch.cu", "xc_fft.cuh", "xc_complex.cu", "xc_2d.cu",
                  "xc_lock.cuh", "xc_dense.cu", "xc_tc.cuh", "xc_window.cuh")


def kernel_source_hash(files=KERNEL_SOURCES):
    """sha256 over the code of the given kernel sources (changes whenever a
    kernel in them does; '//' comments and blank lines are left out, so a
    comment edit does not orphan the profiles)."""
    h = hashlib.sha256()
    for f in files:
        text = open(os.path.join(ROOT, "paper_2004_11610_gb300", "csrc", f), encoding="utf-8").read()
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


def traffic_from_profiles(kernel, workload, plan=None):
    """dram bytes of one launch from the committed ncu summary of this kernel
    and workload (line `traffic: <kernel> plan=<i> dram_bytes=<B>`), provided
    the sources its kernels are compiled from (line `sources:`, else all
    kernel sources) have not changed since the capture (`source_sha256:`)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}__{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"source_sha256:\s*([0-9a-f]{16,64})", text)
    src = re.search(r"^sources:\s*(.+)$", text, re.M)
    files = tuple(src.group(1).split()) if src else KERNEL_SOURCES
    if not h or not kernel_source_hash(files).startswith(h.group(1)):
        return None
    for m in re.finditer(r"traffic:\s*(\S+)\s+plan=(\S+)\s+dram_bytes=([0-9.eE+]+)", text):
        if m.group(1) == kernel and (plan is None or m.group(2) == str(plan)):
            return float(m.group(3))
    return None


def sample_rows(N, k=64, seed=0):
    """Rows of a plan on which forward outputs are checked against the oracle."""
    g = np.random.default_rng([N, seed])
    return np.unique(np.concatenate([[0, N // 2, N - 1], g.integers(0, N, k)]))


def oracle_spec(fam, N, params, nodes):
    """The oracle's matrix at exactly the plan's nodes (Chebyshev: its exact
    Chebyshev-Gauss angles, which the library uses as well)."""
    from oracle import families as F
    if fam == "chebyshev":
        return F.make_spec("chebyshev", N)
    return F.make_spec(fam, N, params.get("alpha", 0.0), params.get("beta", 0.0), x=nodes)


def oracle_accuracy(torch, plans, specs, X, rhs_fwd=16, rhs_adj=4, adj_max_n=16384):
    """Relative l2 error of each plan's forward apply (sampled rows, the first
    rhs_fwd right-hand sides) and adjoint apply (every output, rhs_adj seeded
    right-hand sides, plans up to adj_max_n) against the FP64 oracle's plain
    dense product at the plan's nodes.  Part of the bench's CPU (oracle) leg."""
    from oracle import method as M
    out = []
    for p, s, x in zip(plans, specs, X):
        if p.is_complex or s["params"].get("scheme") == "2d":
            out.append(None)
            continue
        sp = oracle_spec(s["family"], s["N"], s["params"], p.nodes())
        rows = sample_rows(s["N"])
        xs = x[:rhs_fwd]
        y = p.apply(xs).double().cpu().numpy()[:, rows]
        e = {"plan": f"{s['family']} N={s['N']}",
             "forward": M.rel_l2(y, M.dense_apply(sp, xs.double().cpu().numpy(), rows=rows)),
             "forward_sample": f"{len(rows)} rows x {xs.shape[0]} RHS"}
        if s["N"] <= adj_max_n:
            Yh = inputs.normal(s["N"], rhs_adj, 96, s["index"])
            ya = p.apply_adjoint(torch.from_numpy(Yh).to(x.device, p.torch_dtype)).double().cpu().numpy()
            e["adjoint"] = M.rel_l2(ya, M.dense_apply_adjoint(sp, Yh))
            e["adjoint_sample"] = f"all outputs x {rhs_adj} RHS"
        out.append(e)
    return out


# ------------------------------------------------------------ CPU (oracle) leg
_POOL_STATE = {}


def _pool_init(barrier, counter, plans_desc, eps, precision, dist, rhs):
    """Worker start: take a worker index, build the oracle plans of the
    sample (the precompute, not timed) with inputs of its own, warm them."""
    with counter.get_lock():
        w = counter.value
        counter.value += 1
    _POOL_STATE["barrier"] = barrier
    plans = []
    for i, (fam, N, params) in enumerate(plans_desc):
        fwd, adj = oracle_apply_pair(fam, N, params, eps, precision)
        plans.append((fwd, adj, inputs.draw(dist, N, rhs, 90, i, w)))
    for fwd, adj, X in plans:
        adj(fwd(X))
    _POOL_STATE["plans"] = plans


def _pool_run(args):
    """Worker: after every worker has reached the barrier (so each of the n
    tasks runs on its own worker), forward + adjoint applies of the sample
    until `seconds` have passed; returns (vectors, seconds)."""
    seconds, = args
    _POOL_STATE["barrier"].wait(timeout=900)
    plans = _POOL_STATE["plans"]
    reps, t0 = 0, time.perf_counter()
    while True:
        for fwd, adj, X in plans:
            adj(fwd(X))
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * sum(2 * X.shape[0] for _, _, X in plans), el


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(n, plans_desc, eps, precision, dist, rhs):
    """n single-threaded oracle processes (spawned, so no GPU state is
    forked), each holding the sample's plans."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    return ctx.Pool(n, initializer=_pool_init,
                    initargs=(ctx.Barrier(n), ctx.Value("i", 0), plans_desc, eps, precision, dist, rhs))


def time_oracle_parallel(plans_desc, eps, precision, dist, rhs, seconds, cores=None):
    """The FP64 oracle as it stands on every host core: each process applies
    forward + adjoint of every plan of the sample to `rhs` right-hand sides of
    its own for `seconds`.  Returns (vectors/s summed over the processes,
    processes, seconds)."""
    n = cores or host_cores()
    with oracle_pool(n, plans_desc, eps, precision, dist, rhs) as pool:
        res = pool.map(_pool_run, [(seconds,)] * n, chunksize=1)
    vectors = sum(v for v, _ in res)
    el = max(e for _, e in res)
    return vectors / el, n, el


# ---------------------------------------------------------------- GPU path
def measure_gemm_peaks(torch, dev):
    """Measured FP64 and FP32 (no TF32) pipe rates: cuBLAS DGEMM and SGEMM on
    4096^3, best of 5 after a warm-up, CUDA events -- the same kind of
    denominator as the driver's cuBLAS bf16 peak."""
    out = {}
    torch.backends.cuda.matmul.allow_tf32 = False
    n = 4096
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        c = torch.empty(n, n, device=dev, dtype=dt)
        for _ in range(2):
            torch.matmul(a, b, out=c)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        del a, b, c
    return out


def make_plans(xc, torch, wl, dev, rank, precision=None, eps2=None, seed=1):
    precision = precision or wl["precision"]
    plans, specs, X, Y, XA = [], plan_specs(wl), [], [], []
    for s in specs:
        if eps2 is None:
            p = make_xc_plan(xc, s["family"], s["N"], s["params"], wl["eps"], precision)
        else:
            p = xc.Plan(s["family"], s["N"], wl["eps"], precision=precision, eps2=eps2,
                        alpha=s["params"].get("alpha", 0.0), beta=s["params"].get("beta", 0.0))
        p.reserve(wl["nrhs"])
        plans.append(p)
        x = torch.from_numpy(inputs.draw(wl["dist"], s["N"], wl["nrhs"], seed, s["index"], rank)).to(dev, p.torch_dtype)
        X.append(x)
        Y.append(torch.empty_like(x))
        XA.append(torch.empty_like(x))
    return plans, specs, X, Y, XA


def timed_steps(torch, step, steps, stream, flush):
    """Device ms of `steps` calls of step(), L2 flushed before each, events on
    the launching stream."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        stops[k].record(stream)
    stops[-1].synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts, stops))


def measure_variant(xc, torch, wl, dev, steps, warmup, world, precision, eps2=None, label=None):
    """The workload's plans built in another precision (same eps; eps2 as
    given, else that precision's default): vector applies per second over
    `steps` flushed steps."""
    R = wl["nrhs"]
    plans, specs, X, Y, XA = make_plans(xc, torch, wl, dev, 0, precision=precision, eps2=eps2)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        for p, x, y, xa in zip(plans, X, Y, XA):
            p.apply(x, out=y, stream=stream)
            p.apply_adjoint(y, out=xa, stream=stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    total = reduce_max(timed_steps(torch, step, steps, stream, flush), world, dev)
    out = {"precision": label or precision, "value": job_throughput(2 * R * len(plans), steps, total, world),
           "unit": "vectors/s", "ms_per_step": total / steps, "eps2": plans[0].info()["eps2"]}
    return out, plans, specs


def dense_comparators(xc, torch, plans, X, Y, XA, dev, stream, flush, steps, prec, cplx):
    """The direct dense product the method replaces, per plan y = A x and
    x = A^T y, on the matrix from xc_dense_matrix: cuBLAS (torch.matmul,
    TF32 off) in the plan's precision and, for FP32 plans, the library's own
    tensor-core product (tcgen05, 3xTF32).  Times and the relative l2 gap
    between the method and each comparator."""
    torch.backends.cuda.matmul.allow_tf32 = False
    R = X[0].shape[0]
    vectors = 2 * R * len(plans)
    mats = [p.dense_matrix() for p in plans]
    torch.cuda.synchronize(dev)

    def timed(step):
        for _ in range(3):
            step()
        torch.cuda.synchronize(dev)
        return timed_steps(torch, step, steps, stream, flush) / steps

    def cublas_step():
        for A, x, y, xa in zip(mats, X, Y, XA):
            torch.matmul(x, A.T, out=y)
            torch.matmul(y, A, out=xa)

    ms = timed(cublas_step)
    gaps = []
    for p, A, x in zip(plans, mats, X):
        y_d = x @ A.T
        gaps.append(float(torch.linalg.norm(p.apply(x) - y_d) / torch.linalg.norm(y_d)))
        xa_d = y_d @ A
        gaps.append(float(torch.linalg.norm(p.apply_adjoint(y_d) - xa_d) / torch.linalg.norm(xa_d)))
    fp64 = prec in ("fp64", "fp64pair")
    out = {"cublas": {"library": "cuBLAS via torch.matmul (TF32 off)", "ms_per_step": ms,
                      "vectors_per_s": vectors / (ms / 1e3),
                      "dtype": ("c128" if fp64 else "c64") if cplx else ("f64" if fp64 else "f32"),
                      "method_rel_l2_vs_it": max(gaps)}}
    if not fp64 and not cplx:
        dens = [xc.Dense(A) for A in mats]
        gaps_tc = []
        for d, p, A, x in zip(dens, plans, mats, X):
            y_t = d.apply(x)
            gaps_tc.append(float(torch.linalg.norm(p.apply(x) - y_t) / torch.linalg.norm(y_t)))
            xa_t = d.apply(y_t, transpose=True)
            gaps_tc.append(float(torch.linalg.norm(p.apply_adjoint(y_t) - xa_t) / torch.linalg.norm(xa_t)))
            y_c = x @ A.T
            gaps_tc.append(float(torch.linalg.norm(y_t - y_c) / torch.linalg.norm(y_c)))   # vs cuBLAS
        del mats

        def tc_step():
            for d, x, y, xa in zip(dens, X, Y, XA):
                d.apply(x, out=y, stream=stream)
                d.apply(y, transpose=True, out=xa, stream=stream)

        ms_tc = timed(tc_step)
        # per-launch time of the GEMM kernel alone (the split of the right-hand
        # sides excluded): the forward product of the first plan
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        gemm_ms = []
        for _ in range(5):
            flush.zero_()
            ev[0].record(stream)
            dens[0].apply(X[0], out=Y[0], stream=stream)
            ev[1].record(stream)
            ev[1].synchronize()
            gemm_ms.append(ev[0].elapsed_time(ev[1]))
        assert all(d.status() == xc.XC_OK for d in dens)
        N0 = plans[0].N
        out["tensor_core"] = {
            "library": "own tcgen05 kernel (TMA, TMEM accumulators), 3xTF32 split (FP32 accuracy)",
            "ms_per_step": ms_tc, "vectors_per_s": vectors / (ms_tc / 1e3), "dtype": "f32 (3xTF32)",
            "method_rel_l2_vs_it": max(gaps_tc[0::3] + gaps_tc[1::3]),
            "rel_l2_vs_cublas_sgemm": max(gaps_tc[2::3]),
            "forward_launch_ms": min(gemm_ms),
            "forward_tf32_mma_tflops": 3 * 2.0 * N0 * N0 * R / (min(gemm_ms) / 1e3) / 1e12}
        for d in dens:
            d.close()
    else:
        del mats
    best = min(v["vectors_per_s"] for v in out.values())
    out["best_vectors_per_s"] = max(v["vectors_per_s"] for v in out.values())
    return out


def cufft_ms(torch, lengths, nrhs, dtype, dev, flush, stream, reps=5):
    """cuFFT (torch.fft.rfft) on nrhs real vectors of each block length, the
    transforms the forward FFT stage computes: summed over the blocks, best of
    `reps` with L2 flushed, CUDA events on `stream`."""
    total = 0.0
    for L in lengths:
        x = torch.randn(nrhs, L, dtype=dtype, device=dev)
        for _ in range(2):
            torch.fft.rfft(x)
        best = 1e30
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            torch.fft.rfft(x)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        total += best
        del x
    return total


def measure_workload(xc, torch, name, dev, rank, world, steps, warmup, opts, wl=None):
    """One named workload: timed steps, per-kernel roofline, e2e through
    xc_apply_host, dense comparators, precision variants, and (rank 0 of a
    single-rank run) the FP64 oracle's accuracy figures.  Returns the bench
    line's fields."""
    wl = wl or inputs.WORKLOADS[name]
    prec = wl["precision"]
    R = wl["nrhs"]
    plans, specs, X, Y, XA = make_plans(xc, torch, wl, dev, rank)
    infos = [p.info() for p in plans]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def step():
        for p, x, y, xa in zip(plans, X, Y, XA):
            p.apply(x, out=y, stream=stream)
            p.apply_adjoint(y, out=xa, stream=stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(warmup):
        step()
    barrier()
    launches0 = xc.xc_launch_count()
    total_ms = timed_steps(torch, step, steps, stream, flush)
    barrier()
    launches = xc.xc_launch_count() - launches0

    # per-kernel device time, same steps again with every launch bracketed by events
    for p in plans:
        p.timing_enable(True)
        p.timing_read()
    for k in range(steps):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    per_kernel, per_pair = {}, {}
    for pi, (p, info) in enumerate(zip(plans, infos)):
        timing = p.timing_read()
        work = algorithmic_work(info, R, prec, chunked="fwd_reduce" in timing)
        for kname, (n, ms) in timing.items():
            for key, table in ((kname, per_kernel), ((pi, kname), per_pair)):
                e = table.setdefault(key, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
                e["launches"] += n
                e["ms"] += ms
                e["flops"] += work[kname][0] * n
                e["bytes"] += work[kname][1] * n
        p.timing_enable(False)

    max_ms = reduce_max(total_ms, world, dev)
    vectors_per_step = 2 * R * len(plans)
    value = job_throughput(vectors_per_step, steps, max_ms, world)
    ms_per_step = max_ms / steps

    # roofline of the dominant kernel: the (plan, kernel) pair with the largest summed device time
    (dom_plan, kname), e = max(per_pair.items(), key=lambda kv: kv[1]["ms"])
    avg_ms = e["ms"] / e["launches"]
    achieved = e["flops"] / e["launches"] / (avg_ms / 1e3) / 1e12
    peaks = opts["peaks"]
    if prec == "fp64" or (prec == "fp64pair" and kname not in ("fwd_sparse", "adj_sparse")):
        peak = peaks.get("fp64") or FP64_PEAK_TFLOPS
        src = ("measured: cuBLAS DGEMM 4096^3, best of 5, in this run" if peaks.get("fp64")
               else "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz")
    elif prec == "fp64pair":
        peak = PAIR_PEAK_TFLOPS
        src = ("derived: 152 SMs x 128 FP32 instr/clk x 2070 MHz / 6 FP32 instructions per algorithmic "
               "flop (one pair multiply-add = 2 flops = 12 instructions)")
    else:
        peak = peaks.get("fp32") or 152 * 128 * 2 * 2.070e9 / 1e12
        src = ("measured: cuBLAS SGEMM (TF32 off) 4096^3, best of 5, in this run" if peaks.get("fp32")
               else "derived: 152 SMs x 128 FP32 FMA/clk x 2 flops x 2070 MHz")
    roofline = {"kernel": kname, "plan": f"{specs[dom_plan]['family']} N={specs[dom_plan]['N']}",
                "bound": "alu", "achieved": achieved, "unit": "TFLOP/s", "peak": peak, "peak_source": src,
                "frac": achieved / peak, "peak_derived": FP64_PEAK_TFLOPS if prec == "fp64" else None,
                "traffic": traffic_from_profiles(kname, name, dom_plan),
                "algorithmic_bytes_per_launch": e["bytes"] / e["launches"], "avg_launch_ms": avg_ms,
                "nnz_per_row": sum(infos[dom_plan]["nnz"]) / infos[dom_plan]["N"]}
    kernel_table = {k: {"launches": v["launches"], "avg_ms": v["ms"] / v["launches"],
                        "share": v["ms"] / sum(w["ms"] for w in per_kernel.values()),
                        "tflops": v["flops"] / v["ms"] / 1e9 if v["ms"] > 0 else None}
                    for k, v in per_kernel.items()}
    hbm_peak, hbm_src = measured_peaks()
    sb = sum(step_bytes(i, R, prec) for i in infos)
    hbm_gbs = sb / (ms_per_step / 1e3) / 1e9

    # the FFT stage against cuFFT, a timed cross-check only: the library's
    # forward FFT launch (extension, window division, real FFT, half
    # spectrum out, every block) against torch.fft.rfft of the same lengths
    fft_cmp = []
    for pi, (p, info) in enumerate(zip(plans, infos)):
        ours = per_pair.get((pi, "fwd_fft"))
        if p.is_complex or info.get("scheme") == SCHEME_2D or not ours or not info["L"]:
            continue
        ours_ms = ours["ms"] / ours["launches"]
        ms = cufft_ms(torch, info["L"], R, torch.float64 if prec in ("fp64", "fp64pair") else torch.float32, dev,
                      flush, stream)
        fft_cmp.append({"plan": f"{specs[pi]['family']} N={specs[pi]['N']}", "blocks_L": info["L"],
                        "own_fwd_fft_ms": ours_ms, "cufft_rfft_ms": ms, "cufft_over_own": ms / ours_ms})

    out = {"value": value, "ms_per_step": ms_per_step, "steps": steps, "warmup": warmup,
           "config": workload_config(name, wl) | {"parallelism": f"replicas x{world}"},
           "roofline": roofline,
           "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                   "peak_source": hbm_src, "note": "algorithmic bytes of the whole step / step time"},
           "kernels": kernel_table, "gpu_launches": int(launches), "fft_vs_cufft": fft_cmp,
           "plans": [{k: i[k] for k in ("L", "nnz", "stored", "m_tail", "zeta", "matrix_bytes")}
                     | {"nnz_per_row": sum(i["nnz"]) / i["N"],
                        "nnz_per_row_per_block": [round(v / i["N"], 2) for v in i["nnz"]]} for i in infos]}

    if opts.get("e2e", True):
        e2e_steps = max(3, min(steps, 50))
        hx = [torch.from_numpy(inputs.draw(wl["dist"], s["N"], R, 2, s["index"], rank)).to(p.torch_dtype).pin_memory()
              for s, p in zip(specs, plans)]
        hy = [torch.empty_like(h).pin_memory() for h in hx]
        hz = [torch.empty_like(h).pin_memory() for h in hx]
        import ctypes
        st = ctypes.c_void_p(stream.cuda_stream)

        def e2e_step():
            for p, a, b, c in zip(plans, hx, hy, hz):
                xc._check(xc._lib.xc_apply_host(p.handle, 0, ctypes.c_void_p(a.data_ptr()),
                                                ctypes.c_void_p(b.data_ptr()), R, p.N, st), "xc_apply_host")
                xc._check(xc._lib.xc_apply_host(p.handle, 1, ctypes.c_void_p(b.data_ptr()),
                                                ctypes.c_void_p(c.data_ptr()), R, p.N, st), "xc_apply_host")

        for _ in range(2):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        barrier()
        e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
        eb = 8 if prec in ("fp64", "fp64pair") else 4
        io_bytes = sum(2 * R * s["N"] * eb * (2 if p.is_complex else 1) for s, p in zip(specs, plans))
        out["e2e"] = {"value": job_throughput(vectors_per_step, e2e_steps, 1e3 * e2e_s, world), "unit": "vectors/s",
                      "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes}
    cplx = any(p.is_complex for p in plans)
    two_d = any(sp["params"].get("scheme") == "2d" for sp in specs)
    if not opts.get("no_dense"):
        ds = max(3, min(steps, 20))
        dense = dense_comparators(xc, torch, plans, X, Y, XA, dev, stream, flush, ds, prec, cplx)
        dense["speedup_of_method"] = (value / world) / dense["best_vectors_per_s"]
        out["dense_gemm"] = dense
    if opts.get("oracle") and rank == 0 and world == 1:
        out["rel_l2_vs_fp64_oracle"] = oracle_accuracy(torch, plans, specs, X)
    for p in plans:
        p.close()
    del X, Y, XA
    torch.cuda.empty_cache()
    # precision variants of the same plans
    if not opts.get("no_variant") and not cplx and not two_d:
        vs = max(3, min(steps, 50))
        if prec == "fp64":
            v, vplans, vspecs = measure_variant(xc, torch, wl, dev, vs, 3, world, "fp64pair",
                                                label="fp64pair (FP64 vectors, FFTs and tail; band values, spectra "
                                                      "and band products in FP32 pairs, TwoProduct/TwoSum)")
            out["fp64_pair_variant"] = v
        elif prec in ("fp32", "fp32c"):
            # the same compressed matrices (same eps and eps2) applied in FP64
            v, vplans, vspecs = measure_variant(xc, torch, wl, dev, vs, 3, world, "fp64", eps2=infos[0]["eps2"],
                                                label="fp64 (same eps and eps2: the same compressed matrices)")
            v["method_speedup_over_it"] = (value / world) / v["value"]
            out["fp64_apply"] = v
        else:
            vplans = []
        if opts.get("oracle") and rank == 0 and world == 1 and vplans:
            Xv = [torch.from_numpy(inputs.draw(wl["dist"], s["N"], 16, 1, s["index"], 0)).to(dev, p.torch_dtype)
                  for s, p in zip(vspecs, vplans)]
            key = "fp64_pair_variant" if prec == "fp64" else "fp64_apply"
            out[key]["rel_l2_vs_fp64_oracle"] = oracle_accuracy(torch, vplans, vspecs, Xv)
        for p in vplans:
            p.close()
        torch.cuda.empty_cache()
    return out


def run_xc(args, rank, world, local_rank):
    import torch
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = inputs.WORKLOADS[args.workload]
    prec = wl["precision"]
    cplx = any(f in ("exp", "lagspec") for f, _, _ in wl["plans"])
    clocks = ClockSampler(local_rank)
    clocks.start()
    peaks = measure_gemm_peaks(torch, dev) if not args.no_dense else {}
    opts = {"peaks": peaks, "no_dense": args.no_dense, "no_variant": args.no_variant,
            "oracle": not args.no_cpu_baseline}
    res = measure_workload(xc, torch, args.workload, dev, rank, world, args.steps, args.warmup, opts)
    # the other configurations, measured in the same process (shorter runs)
    extra = {}
    if not args.no_extra and args.workload == "cheb_lag4096_fp64":
        sub_steps = max(3, min(args.steps, 20))
        for name in ("leg_jac16384_fp32c", "legendre32768_fp32"):
            r = measure_workload(xc, torch, name, dev, rank, world, sub_steps, 3, opts | {"e2e": True})
            extra[name] = {k: r[k] for k in ("value", "ms_per_step", "roofline", "e2e", "dense_gemm",
                                             "rel_l2_vs_fp64_oracle", "fp64_apply", "plans", "fft_vs_cufft")
                           if k in r}
            extra[name]["unit"] = "vectors/s"
            extra[name]["config"] = r["config"]
        b = measure_batch(xc, torch, 1000, dev, rank, world, sub_steps, 3, tune=True)
        extra["batch1000"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "roofline", "launch_ms", "e2e",
                                                "config", "plan_create_s", "gpu_launches")}
    clock_info = clocks.stop()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample_rhs = 2
        v, cores, el = time_oracle_parallel(wl["plans"], wl["eps"], prec, wl["dist"], sample_rhs, 10.0)
        cpu = {"value": v, "unit": "vectors/s", "cores": cores, "kind": "oracle",
               "sample": f"{sample_rhs} RHS per plan and process, forward + adjoint, {cores} single-threaded "
                         f"processes for {el:.1f} s (numpy/scipy FP64 oracle as it stands)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": res["value"], "unit": "vectors/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp64pair": "f64 (band products in f32 pairs)", "fp32": "f32"}.get(
                prec, "f32-compensated") + (" complex" if cplx else ""),
            "data": "synthetic", "config": res["config"],
            "roofline": res["roofline"], "hbm": res["hbm"], "kernels": res["kernels"],
            "fft_vs_cufft": res.get("fft_vs_cufft"),
            "dense_gemm": res.get("dense_gemm"), "fp64_pair_variant": res.get("fp64_pair_variant"),
            "fp64_apply": res.get("fp64_apply"), "rel_l2_vs_fp64_oracle": res.get("rel_l2_vs_fp64_oracle"),
            "measured_peaks_tflops": peaks or None,
            "cpu_baseline": cpu, "e2e": res.get("e2e"), "gpu_launches": res["gpu_launches"],
            "clocks": clock_info, "plans": res["plans"], "other_configs": extra or None,
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batch path
def measure_batch(xc, torch, nplans, dev, rank, world, steps, warmup, tune=True, schedule=None):
    """The many-plan workload (N log-uniform in [256, 8192], families uniform
    over Chebyshev / Legendre / Jacobi(1/2,-1/2) / Hermite, 1..32 right-hand
    sides), FP32, eps = 1e-7: forward + adjoint as two persistent launches
    (and, forward, the tensor-core window launches) replayed from one CUDA
    graph.  `schedule` (rpw_f, rpw_a, lockstep_f, lockstep_a) replaces the
    tuner's choice (fixed launch counts, for profiling).  Returns the bench
    line's fields."""
    wl = inputs.batch_workload(nplans)
    t_create = time.perf_counter()
    plans, xs, ys, xa = [], [], [], []
    for i, (fam, N, params, R) in enumerate(wl):
        p = xc.Plan(fam, N, 1e-7, precision="fp32", alpha=params.get("alpha", 0.0), beta=params.get("beta", 0.0))
        plans.append(p)
        x = torch.from_numpy(inputs.normal(N, R, 4, i, rank)).to(dev, torch.float32)
        xs.append(x)
        ys.append(torch.empty_like(x))
        xa.append(torch.empty_like(x))
    t_create = time.perf_counter() - t_create
    stream = torch.cuda.current_stream(dev)
    fwd, adj = xc.Batch(plans), xc.Batch(plans)
    fwd.bind(xs, ys)          # forward: x -> y
    adj.bind(xa, ys)          # adjoint: y -> xa (keeps x)
    if schedule is not None:
        fwd.schedule(*schedule)
        adj.schedule(*schedule)
    elif tune:
        fwd.tune(stream)
        adj.tune(stream)
    infos = [p.info() for p in plans]
    R_tot = sum(x.shape[0] for x in xs)
    vectors_per_step = 2 * R_tot
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        fwd.apply(False, stream)
        adj.apply(True, stream)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream(dev)
    with torch.cuda.stream(gs):
        with torch.cuda.graph(graph, stream=gs):
            fwd.apply(False, gs)
            adj.apply(True, gs)
    torch.cuda.synchronize(dev)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize(dev)
    assert fwd.status() == xc.XC_OK and adj.status() == xc.XC_OK

    launches0 = xc.xc_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    total_ms = timed_steps(torch, graph.replay, steps, stream, flush)
    torch.cuda.synchronize(dev)
    # graph replays launch the library's kernels without passing through its
    # launch counter: two persistent launches per step
    launches = 2 * steps + (xc.xc_launch_count() - launches0)

    # each direction timed on its own (events around single launches)
    dir_ms = [0.0, 0.0]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    nrep = max(3, min(steps, 20))
    for _ in range(nrep):
        flush.zero_()
        ev[0].record(stream)
        fwd.apply(False, stream)
        ev[1].record(stream)
        flush.zero_()
        ev[2].record(stream)
        adj.apply(True, stream)
        ev[3].record(stream)
        ev[3].synchronize()
        dir_ms[0] += ev[0].elapsed_time(ev[1])
        dir_ms[1] += ev[2].elapsed_time(ev[3])
    dir_ms = [d / nrep for d in dir_ms]
    max_ms = reduce_max(total_ms, world, dev)
    value = job_throughput(vectors_per_step, steps, max_ms, world)
    ms_per_step = max_ms / steps

    # algorithmic bytes of one launch per direction: every plan's stored band
    # values once, its vectors in and out, its spectra (forward) or chunk
    # partials (adjoint) written and read once
    eb = 4
    fwd_bytes = adj_bytes = 0
    for info, x in zip(infos, xs):
        R = x.shape[0]
        H = sum(L // 2 + 1 for L in info["L"])
        fwd_bytes += info["matrix_bytes"] + R * (2 * info["N"] * eb + 2 * H * 2 * eb)
        adj_bytes += info["adjoint_bytes"] + R * (2 * info["N"] * eb + 2 * H * 2 * eb)
    hbm_peak, hbm_src = measured_peaks()
    dom = 0 if dir_ms[0] >= dir_ms[1] else 1
    achieved = (fwd_bytes, adj_bytes)[dom] / (dir_ms[dom] / 1e3) / 1e9
    roofline = {"kernel": ("batch_kernel (forward)", "batch_kernel (adjoint)")[dom], "bound": "hbm",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": hbm_src,
                "traffic": traffic_from_profiles("batch_kernel", "batch1000", ("forward", "adjoint")[dom]),
                "algorithmic_bytes_per_launch": (fwd_bytes, adj_bytes)[dom], "avg_launch_ms": dir_ms[dom],
                "other_direction": {"kernel": ("batch_kernel (forward)", "batch_kernel (adjoint)")[1 - dom],
                                    "achieved": (fwd_bytes, adj_bytes)[1 - dom] / (dir_ms[1 - dom] / 1e3) / 1e9,
                                    "avg_launch_ms": dir_ms[1 - dom],
                                    "traffic": traffic_from_profiles("batch_kernel", "batch1000",
                                                                     ("forward", "adjoint")[1 - dom])}}
    roofline["other_direction"]["frac"] = roofline["other_direction"]["achieved"] / hbm_peak

    # end to end: pinned host inputs copied in, both launches, results copied out
    hx = [x.cpu().pin_memory() for x in xs]
    hy = [torch.empty(y.shape, dtype=y.dtype).pin_memory() for y in ys]
    hz = [torch.empty(y.shape, dtype=y.dtype).pin_memory() for y in ys]

    def e2e_step():
        for a, x in zip(hx, xs):
            x.copy_(a, non_blocking=True)
        graph.replay()
        for b, y in zip(hy, ys):
            b.copy_(y, non_blocking=True)
        for c, z in zip(hz, xa):
            c.copy_(z, non_blocking=True)
        torch.cuda.synchronize(dev)

    e2e_step()
    e2e_steps = max(3, min(steps, 20))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
    io_in = sum(x.numel() * 4 for x in xs)
    out = {
        "value": value, "unit": "vectors/s", "ms_per_step": ms_per_step, "roofline": roofline,
        "launch_ms": {"forward": dir_ms[0], "adjoint": dir_ms[1]},
        "e2e": {"value": job_throughput(vectors_per_step, e2e_steps, 1e3 * e2e_s, world), "unit": "vectors/s",
                "h2d_bytes_per_step": io_in, "d2h_bytes_per_step": 2 * io_in},
        "gpu_launches": int(launches), "plan_create_s": t_create,
        "config": {"workload": "batch1000", "plans": len(plans), "rhs_total": R_tot, "eps": 1e-7,
                   "precision": "fp32", "step": "forward + adjoint of every plan, one CUDA-graph replay "
                   "of two persistent launches", "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}",
                   "tuned_rhs_per_item": [fwd.info()["rhs_per_item"], adj.info()["rhs_per_item_adjoint"]],
                   "tuned_lockstep": [fwd.info()["lockstep_forward"], adj.info()["lockstep_adjoint"]],
                   "tensor_window_plans": [fwd.info()["tensor_plans"], adj.info()["tensor_plans_adjoint"]],
                   "tune_ms": {"forward": _tune_table(fwd.info()["tune_ms_forward"]),
                               "adjoint": _tune_table(adj.info()["tune_ms_adjoint"])}},
        "matrix_bytes": sum(i["matrix_bytes"] for i in infos),
        "adjoint_bytes": sum(i["adjoint_bytes"] for i in infos),
    }
    del graph
    fwd.close()
    adj.close()
    for p in plans:
        p.close()
    del xs, ys, xa
    torch.cuda.empty_cache()
    return out


def _tune_table(ms):
    """The tuner's summed timings keyed "lockstep<l>_rpw<r>" (tried candidates only)."""
    return {f"lockstep{k // 4}_rpw{1 << (k % 4)}": round(v, 4) for k, v in enumerate(ms) if v >= 0}


def run_batch(args, rank, world, local_rank):
    import torch
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    sched = tuple(int(v) for v in args.batch_schedule.split(",")) if args.batch_schedule else None
    b = measure_batch(xc, torch, args.nplans, dev, rank, world, args.steps, args.warmup, schedule=sched)
    clock_info = clocks.stop()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = [w for w in inputs.batch_workload(args.nplans) if w[1] <= 1024][:6]
        v, cores, el = time_oracle_parallel([(f, N, p) for f, N, p, _ in sample], 1e-7, "fp32", "normal", 2, 10.0)
        cpu = {"value": v, "unit": "vectors/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(sample)} plans of the batch with N <= 1024, 2 RHS each per process, forward + "
                         f"adjoint, {cores} single-threaded processes for {el:.1f} s (FP64 oracle)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": b["value"], "unit": "vectors/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": b["config"],
            "roofline": b["roofline"], "launch_ms": b["launch_ms"], "cpu_baseline": cpu, "e2e": b["e2e"],
            "gpu_launches": b["gpu_launches"], "clocks": clock_info, "plan_create_s": b["plan_create_s"],
            "matrix_bytes": b["matrix_bytes"], "adjoint_bytes": b["adjoint_bytes"],
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "batch1000":
            run_batch(args, rank, world, local_rank)
        else:
            run_xc(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
