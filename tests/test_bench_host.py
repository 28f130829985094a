"""Host-side logic of bench.py: the cross-rank reduction under a real
two-rank torch.distributed group (gloo on CPU), the replica throughput
formula, and the reference arm's rank handling."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow replica
        m = bench.reduce_max(local_ms, world)
        v = bench.job_throughput(100, 4, m, world)
        out.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_reduce_max_and_throughput_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 15.0                       # every rank sees the slowest time
        assert v == pytest.approx(2 * 100 * 4 / 0.015)


def test_job_throughput_single_rank():
    import bench
    assert bench.job_throughput(64, 10, 5.0, 1) == pytest.approx(64 * 10 / 0.005)
    assert bench.reduce_max(3.5, 1) == 3.5


def test_reference_arm_non_zero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_work_model_covers_every_kernel_the_library_times():
    """Every kernel name the library reports in its timings has an entry in
    bench.py's algorithmic work model (otherwise the bench stops at a KeyError)."""
    import pathlib
    import re
    root = pathlib.Path(__file__).resolve().parents[1]
    src = (root / "paper_2004_11610_gb300" / "csrc" / "xc_abi.cpp").read_text()
    m = re.search(r"names\[K_COUNT\]\s*=\s*\{([^}]*)\}", src)
    assert m
    names = re.findall(r'"([a-z_]+)"', m.group(1))
    import bench
    info = {"nnz": [100, 50], "N": 64, "m_tail": 3, "L": [80, 24]}
    for chunked in (False, True):
        work = bench.algorithmic_work(info, 4, "fp32", chunked)
        assert set(names) <= set(work), set(names) - set(work)
    # complex families run the FFT, band and row-scale kernels
    cinfo = {"nnz": [900], "N": 64, "m_tail": 0, "L": [80], "family": 8}
    work = bench.algorithmic_work(cinfo, 4, "fp64")
    assert {"fwd_fft", "fwd_sparse", "adj_sparse", "adj_fft", "row_scale"} <= set(work)
    assert work["fwd_sparse"][0] == 8.0 * 900 * 4


def test_workload_plumbing_for_the_complex_and_2d_workloads():
    """Every named workload has a label and a config; the 2-D workload's nodes
    are the Laguerre transform's points; the oracle arms build the right kind
    of plan (1-D, complex, 2-D) and give outputs of the input's shape."""
    import numpy as np
    import bench
    from paper_2004_11610_gb300 import inputs
    for name, wl in inputs.WORKLOADS.items():
        cfg = bench.workload_config(name, wl)
        assert cfg["workload"] == name and len(cfg["plans"]) == len(wl["plans"])
    x = bench.laguerre_transform_nodes(4096, 100.0)
    assert np.allclose(np.diff(x), 12.0 * 100.0 / 4095) and x[0] == pytest.approx(12.0 * 100.0 / 4095)
    for fam, N, params, dist in (("laguerre", 60, {"scheme": "2d", "eta": 10.0}, "normal"),
                                 ("lagspec", 40, {"alpha": 30.0, "beta": 2.0}, "complex_normal"),
                                 ("legendre", 50, {}, "uniform_pm1")):
        fwd, adj = bench.oracle_apply_pair(fam, N, params, 1e-8, "fp64")
        X = inputs.draw(dist, N, 2, 5)
        assert fwd(X).shape == X.shape and adj(X).shape == X.shape
        assert np.iscomplexobj(fwd(X)) == (fam == "lagspec")


def test_work_model_of_2d_plans():
    import bench
    info = {"nnz": [], "N": 100, "m_tail": 0, "L": [], "scheme": 3, "nnz2d": 5000, "dense_elems2d": 700}
    work = bench.algorithmic_work(info, 8, "fp64")
    assert work["sparse_2d"][0] == 8.0 * 5000 * 8
    assert work["combine_2d"][0] == 2.0 * 700 * 8
    assert bench.step_bytes(dict(info, matrix_bytes=10, adjoint_bytes=20), 8, "fp64") > 30


def test_profile_summaries_are_current_and_name_their_kernels_sources():
    """Every committed ncu summary names the sources its kernels are compiled
    from (the translation unit and everything it includes among the kernel
    sources).  Its hash matches them and each `traffic:` line is found by the
    bench's lookup, or the summary says `stale:` and the lookup gives None.
    The default workload's summaries are current."""
    import pathlib
    import re
    import bench
    csrc = pathlib.Path(ROOT) / "paper_2004_11610_gb300" / "csrc"

    def closure(f, seen):
        if f in seen or f not in bench.KERNEL_SOURCES:
            return seen
        seen.add(f)
        for inc in re.findall(r'#include "([^"]+)"', (csrc / f).read_text()):
            closure(inc, seen)
        return seen

    profiles = sorted((pathlib.Path(ROOT) / "profiles").glob("*__*.md"))
    assert profiles
    for path in profiles:
        text = path.read_text()
        files = re.search(r"^sources:\s*(.+)$", text, re.M).group(1).split()
        tu = [f for f in files if f.endswith(".cu")]
        assert len(tu) == 1, path.name
        assert set(files) == closure(tu[0], set()), path.name
        h = re.search(r"source_sha256:\s*([0-9a-f]+)", text).group(1)
        current = bench.kernel_source_hash(tuple(files)).startswith(h)
        stale = re.search(r"^stale:", text, re.M) is not None
        assert current != stale, path.name
        kernel, workload = path.stem.split("__", 1)
        assert not (stale and workload == "cheb_lag4096_fp64"), path.name
        for k, plan, b in re.findall(r"traffic:\s*(\S+)\s+plan=(\S+)\s+dram_bytes=([0-9.eE+]+)", text):
            if k == kernel:
                assert bench.traffic_from_profiles(k, workload, plan) == (None if stale else float(b))


def test_tune_table_names_every_tried_schedule():
    """The batch tuner's timings (entry 4 * lockstep + log2(rhs per item),
    lockstep 0/1/2 = row per lane / lockstep items / tensor windows) become
    named bench fields; untried candidates (-1) are left out."""
    import bench
    ms = [float(k) for k in range(12)]
    ms[5] = -1.0
    t = bench._tune_table(ms)
    assert len(t) == 11 and "lockstep1_rpw2" not in t
    assert t["lockstep0_rpw1"] == 0.0 and t["lockstep0_rpw8"] == 3.0
    assert t["lockstep2_rpw1"] == 8.0 and t["lockstep2_rpw8"] == 11.0
