"""The many-plan persistent launch (xc_batch_*): results equal the single-plan
applies (FP64 batches bit for bit; FP32 batches to rounding, since lockstep
items of plans with long bands group their sums by window pieces), the
launch replays from a CUDA graph, the autotuner keeps results unchanged, and
an injected missing dependency ends in XC_ERR_TIMEOUT (a bounded device
wait) rather than a hang."""
import numpy as np
import pytest

from paper_2004_11610_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_11610_gb300 import build
    build.build()
    from paper_2004_11610_gb300 import xc as mod
    return mod


def make_batch(xc, nplans, precision, seed, nmax=3000):
    """Mixed families, log-uniform N, 1..32 right-hand sides (a small copy of
    the 1000-plan workload)."""
    g = np.random.default_rng(seed)
    fams = ("chebyshev", "legendre", "jacobi", "hermite")
    plans, xs, ys = [], [], []
    for i in range(nplans):
        N = int(round(np.exp(g.uniform(np.log(40), np.log(nmax)))))
        fam = fams[i % 4]
        R = int(g.integers(1, 33))
        p = xc.Plan(fam, N, 1e-7, precision=precision, alpha=0.5, beta=-0.5)
        plans.append(p)
        x = torch.from_numpy(inputs.normal(N, R, 80, i)).to("cuda", p.torch_dtype)
        xs.append(x)
        ys.append(torch.empty_like(x))
    return plans, xs, ys


def close_all(plans):
    for p in plans:
        p.close()


def rel(a, b):
    return float((a.double() - b.double()).abs().max() / b.double().abs().max().clamp_min(1e-300))


def tol_for(precision):
    """Batch against single-plan applies: FP64 bit for bit; FP32 to rounding
    (the single-plan adjoint of small plans, and the batch's lockstep items
    of long-band plans, group their partial sums differently)."""
    return 1e-12 if precision == "fp64" else 2e-6


@pytest.mark.parametrize("precision,nplans", [("fp32", 24), ("fp64", 9), ("fp32c", 8)])
def test_batch_matches_single_plan_applies(xc, precision, nplans):
    plans, xs, ys = make_batch(xc, nplans, precision, 1)
    try:
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            b.apply(adjoint=False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            for p, x, y in zip(plans, xs, ys):
                assert rel(y, p.apply(x)) <= tol_for(precision)
            y_saved = [y.clone() for y in ys]
            b.apply(adjoint=True)          # reads y, writes x
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            # single-plan adjoints of small plans cut their bands into shorter
            # chunks than the batch (more warps per right-hand side), which
            # changes the summation order: equal to rounding, not bit for bit
            tol = tol_for(precision)
            for p, x, y in zip(plans, xs, y_saved):
                assert rel(x, p.apply_adjoint(y)) <= tol
    finally:
        close_all(plans)


def test_batch_graph_capture_and_replay(xc):
    plans, xs, ys = make_batch(xc, 16, "fp32", 2)
    try:
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            b.apply(False)                 # warm-up outside the capture
            b.apply(True)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                with torch.cuda.graph(graph, stream=stream):
                    b.apply(False, stream=stream)
            for rep in range(2):
                for i, (p, x) in enumerate(zip(plans, xs)):
                    x.copy_(torch.from_numpy(inputs.normal(p.N, x.shape[0], 81 + rep, i)).to(x.dtype))
                graph.replay()
                torch.cuda.synchronize()
                assert b.status() == xc.XC_OK
                for p, x, y in zip(plans, xs, ys):
                    assert rel(y, p.apply(x)) <= tol_for("fp32")
    finally:
        close_all(plans)


def test_batch_autotune_keeps_results(xc):
    plans, xs, ys = make_batch(xc, 12, "fp32", 3)
    try:
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            x0 = [x.clone() for x in xs]
            b.tune()
            assert all(torch.equal(a, c) for a, c in zip(xs, x0))   # inputs restored
            info = b.info()
            assert info["tuned"] == 1 and info["rhs_per_item"] in (1, 2, 4, 8)
            assert info["rhs_per_item_adjoint"] in (1, 2, 4, 8)
            b.apply(False)
            torch.cuda.synchronize()
            for p, x, y in zip(plans, xs, ys):
                assert rel(y, p.apply(x)) <= tol_for("fp32")
    finally:
        close_all(plans)


def test_batch_missing_dependency_times_out_without_hanging(xc):
    plans, xs, ys = make_batch(xc, 6, "fp32", 4)
    try:
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            b.debug_set(3, 1, 2000)        # plan 3 waits for one FFT that never comes
            b.apply(False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_ERR_TIMEOUT
            assert b.status() == xc.XC_OK   # cleared on read
            b.debug_set(3, 0, 1 << 22)
            b.apply(False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            for p, x, y in zip(plans, xs, ys):
                assert rel(y, p.apply(x)) <= tol_for("fp32")
    finally:
        close_all(plans)


def test_batch_rejects_mixed_precision(xc):
    a = xc.Plan("legendre", 100, 1e-8, precision="fp64")
    c = xc.Plan("legendre", 100, 1e-8, precision="fp32")
    try:
        with pytest.raises(xc.XcError):
            xc.Batch([a, c])
    finally:
        a.close()
        c.close()


def test_batch_binding_survives_larger_single_applies_and_refused_binds(xc):
    """A single-plan apply with more right-hand sides than the batch bound
    grows the plan's scratch: the plan keeps the buffer the batch points at,
    so the batch's results stay right.  A refused bind leaves the previous
    binding in force; a plan listed twice is refused."""
    import ctypes
    plans, xs, ys = make_batch(xc, 6, "fp32", 5)
    try:
        with pytest.raises(xc.XcError) as e:
            xc.Batch([plans[0], plans[1], plans[0]])
        assert e.value.code == xc.XC_ERR_ARG
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            b.apply(False)
            torch.cuda.synchronize()
            ref = [y.clone() for y in ys]
            for i, p in enumerate(plans):        # 40 > 32 right-hand sides: every scratch grows
                big = torch.from_numpy(inputs.normal(p.N, 40, 82, i)).to("cuda", p.torch_dtype)
                p.apply(big)
                p.apply_adjoint(big)
            n = len(plans)
            xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
            yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
            yp[2] = None                          # refused: plan 2 has no output
            nr = (ctypes.c_int64 * n)(*[x.shape[0] for x in xs])
            ld = (ctypes.c_int64 * n)(*[p.N for p in plans])
            assert xc._lib.xc_batch_bind(b._h, xp, yp, nr, ld) == xc.XC_ERR_ARG
            for y in ys:
                y.zero_()
            b.apply(False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            for y, r in zip(ys, ref):
                assert rel(y, r) <= 1e-12
            b.bind(xs, ys)                        # a new bind takes the grown scratch
            b.apply(False)
            torch.cuda.synchronize()
            for p, x, y in zip(plans, xs, ys):
                assert rel(y, p.apply(x)) <= tol_for("fp32")
    finally:
        close_all(plans)


# Plans of the 1000-plan workload (inputs.batch_workload) chosen so that the
# slice holds its largest N (Legendre, 8157), its two largest Hermite plans
# (8039 and 7818), plans with 1 and with 32 right-hand sides, and every family.
CONFIG4_SLICE = (452, 754, 432, 196, 85, 78, 153, 0, 1, 2)


def test_batch_matches_the_oracle_on_a_slice_of_the_1000_plan_workload(xc):
    """Each plan's forward and adjoint output of the persistent launches
    (tuned, as the benchmark runs them) against the FP64 oracle: its method
    (Algorithms 1-4 on the same nodes) and the plain dense product (forward
    on sampled rows).  Tolerance: relative l2 <= max(10 eps, 1e-5)."""
    from oracle import families as F
    from oracle import method as M
    eps = 1e-7
    tol = max(10 * eps, 1e-5)
    wl = inputs.batch_workload(1000)
    plans, xs, ys, xa, specs, X, Yin = [], [], [], [], [], [], []
    try:
        for i in CONFIG4_SLICE:
            fam, N, params, R = wl[i]
            sp = F.make_spec(fam, N, params.get("alpha", 0.0), params.get("beta", 0.0))
            specs.append(sp)
            p = xc.Plan(fam, N, eps, precision="fp32", alpha=params.get("alpha", 0.0),
                        beta=params.get("beta", 0.0), nodes=None if fam == "chebyshev" else sp.x)
            plans.append(p)
            X.append(inputs.normal(N, R, 4, i, 0))
            Yin.append(inputs.normal(N, R, 5, i, 0))
            xs.append(torch.from_numpy(X[-1]).to("cuda", torch.float32))
            ys.append(torch.empty_like(xs[-1]))
            xa.append(torch.empty_like(xs[-1]))
        assert max(p.N for p in plans) >= 8000
        assert sum(1 for i in CONFIG4_SLICE if wl[i][0] == "hermite") >= 2
        assert {wl[i][3] for i in CONFIG4_SLICE} >= {1, 32}
        with xc.Batch(plans) as fwd, xc.Batch(plans) as adj:
            fwd.bind(xs, ys)
            adj.bind(xa, ys)
            fwd.tune()
            adj.tune()
            fwd.apply(False)
            torch.cuda.synchronize()
            assert fwd.status() == xc.XC_OK
            Y = [y.double().cpu().numpy() for y in ys]
            for y, v in zip(ys, Yin):          # independent adjoint inputs
                y.copy_(torch.from_numpy(v).to(torch.float32))
            adj.apply(True)
            torch.cuda.synchronize()
            assert adj.status() == xc.XC_OK
            XA = [x.double().cpu().numpy() for x in xa]
        for i, sp, y, x_in, xa_g, y_in in zip(CONFIG4_SLICE, specs, Y, X, XA, Yin):
            ora = M.build(sp, eps, precision="fp32")
            rows = np.unique(np.concatenate([[0, sp.N - 1], np.random.default_rng(i).integers(0, sp.N, 96)]))
            e = {"fwd_method": M.rel_l2(y, M.apply(ora, x_in)),
                 "fwd_dense": M.rel_l2(y[:, rows], M.dense_apply(sp, x_in, rows=rows)),
                 "adj_method": M.rel_l2(xa_g, M.apply_adjoint(ora, y_in))}
            print(f"batch plan {i} {sp.family} N={sp.N} R={x_in.shape[0]}: "
                  + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
            assert max(e.values()) <= tol, (i, e)
    finally:
        close_all(plans)


@pytest.mark.parametrize("lock,rpw", [(1, 8), (1, 4), (0, 4)])
def test_batch_lockstep_items_against_the_oracle(xc, lock, rpw):
    """Hermite plans (tight windows: lockstep items) and Legendre plans (not),
    short and long bands, 1 to 40 right-hand sides (1, 2 and 4 rows per lane
    in the lockstep forward items, a ragged second group of 32 right-hand
    sides), both directions with lockstep items on
    and off, in the kernels built for 4 and for 8 right-hand sides per
    classic item (80 and 128 registers per thread), against the FP64
    oracle's method on the same nodes: relative l2 <= max(10 eps, 1e-5)."""
    from oracle import families as F
    from oracle import method as M
    eps = 1e-7
    cases = [("hermite", 1500, 7), ("hermite", 600, 32), ("hermite", 3100, 1), ("hermite", 2200, 13),
             ("hermite", 900, 20), ("hermite", 1200, 40), ("legendre", 900, 5), ("chebyshev", 700, 4)]
    plans, specs, xs, ys, xa, X, Yin = [], [], [], [], [], [], []
    try:
        for i, (fam, N, R) in enumerate(cases):
            sp = F.make_spec(fam, N)
            specs.append(sp)
            plans.append(xc.Plan(fam, N, eps, precision="fp32", nodes=None if fam == "chebyshev" else sp.x))
            X.append(inputs.normal(N, R, 40, i))
            Yin.append(inputs.normal(N, R, 41, i))
            xs.append(torch.from_numpy(X[-1]).to("cuda", torch.float32))
            ys.append(torch.empty_like(xs[-1]))
            xa.append(torch.empty_like(xs[-1]))
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            # lockstep on or off for both directions (the tuner's switch)
            b.schedule(rpw, rpw, lock, lock)
            assert b.info()["lockstep_plans"] == (6 if lock else 0)
            b.apply(False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            Y = [y.double().cpu().numpy() for y in ys]
            for y, v in zip(ys, Yin):
                y.copy_(torch.from_numpy(v).to(torch.float32))
            b2 = xc.Batch(plans)
            b2.bind(xa, ys)
            b2.schedule(rpw, rpw, lock, lock)
            b2.apply(True)
            torch.cuda.synchronize()
            assert b2.status() == xc.XC_OK
            XA = [x.double().cpu().numpy() for x in xa]
            b2.close()
        for sp, y, xi, xg, yi in zip(specs, Y, X, XA, Yin):
            ora = M.build(sp, eps, precision="fp32")
            ef = M.rel_l2(y, M.apply(ora, xi))
            ea = M.rel_l2(xg, M.apply_adjoint(ora, yi))
            print(f"lockstep={lock} {sp.family} N={sp.N} R={xi.shape[0]}: fwd {ef:.2e} adj {ea:.2e}")
            assert ef <= max(10 * eps, 1e-5) and ea <= max(10 * eps, 1e-5)
    finally:
        close_all(plans)


@pytest.mark.parametrize("rpw", [4, 8])
def test_batch_tensor_windows_against_the_oracle(xc, rpw):
    """Band products on the tensor cores (schedule lockstep 2), forward and
    adjoint: Hermite plans with ragged row and bin groups (N not a multiple
    of 128), 1 to 64 right-hand sides (the three launch classes rp <= 16, 32,
    64, with rp above nrhs), against the FP64 oracle's method on the same
    nodes (relative l2 <= max(10 eps, 1e-5)) and against the batch's
    lockstep items on the same inputs (FP32 rounding); a Legendre plan in
    the same batch keeps its row-per-lane items."""
    from oracle import families as F
    from oracle import method as M
    eps = 1e-7
    cases = [("hermite", 300, 1), ("hermite", 1000, 9), ("hermite", 2500, 16), ("hermite", 777, 17),
             ("hermite", 4100, 24), ("hermite", 1300, 33), ("hermite", 2000, 64), ("legendre", 900, 5)]
    plans, specs, xs, ys, X, xa, Yin = [], [], [], [], [], [], []
    try:
        for i, (fam, N, R) in enumerate(cases):
            sp = F.make_spec(fam, N)
            specs.append(sp)
            plans.append(xc.Plan(fam, N, eps, precision="fp32", nodes=sp.x))
            X.append(inputs.normal(N, R, 42, i))
            Yin.append(inputs.normal(N, R, 43, i))
            xs.append(torch.from_numpy(X[-1]).to("cuda", torch.float32))
            ys.append(torch.empty_like(xs[-1]))
            xa.append(torch.empty_like(xs[-1]))
        with xc.Batch(plans) as b:
            b.bind(xs, ys)
            b.schedule(rpw, rpw, 1, 1)
            b.apply(False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            Y_lock = [y.double().cpu().numpy() for y in ys]
            b.schedule(rpw, rpw, 2, 1)
            info = b.info()
            print(f"tensor plans {info['tensor_plans']} of {len(cases)}, lockstep plans {info['lockstep_plans']}")
            assert info["tensor_plans"] >= 5 and info["lockstep_forward"] == 2
            for y in ys:
                y.fill_(float("nan"))
            b.apply(False)
            torch.cuda.synchronize()
            assert b.status() == xc.XC_OK
            Y = [y.double().cpu().numpy() for y in ys]
        for y, v in zip(ys, Yin):
            y.copy_(torch.from_numpy(v).to(torch.float32))
        with xc.Batch(plans) as b2:
            b2.bind(xa, ys)
            b2.schedule(rpw, rpw, 1, 1)
            b2.apply(True)
            torch.cuda.synchronize()
            assert b2.status() == xc.XC_OK
            XA_lock = [x.double().cpu().numpy() for x in xa]
            b2.schedule(rpw, rpw, 2, 2)
            info = b2.info()
            print(f"adjoint tensor plans {info['tensor_plans_adjoint']} of {len(cases)}")
            assert info["tensor_plans_adjoint"] >= 5 and info["lockstep_adjoint"] == 2
            for x in xa:
                x.fill_(float("nan"))
            b2.apply(True)
            torch.cuda.synchronize()
            assert b2.status() == xc.XC_OK
            XA = [x.double().cpu().numpy() for x in xa]
        for sp, y, yl, xi, xg, xl, yi in zip(specs, Y, Y_lock, X, XA, XA_lock, Yin):
            ora = M.build(sp, eps, precision="fp32")
            ef = M.rel_l2(y, M.apply(ora, xi))
            el = M.rel_l2(y, yl)
            ea = M.rel_l2(xg, M.apply_adjoint(ora, yi))
            eal = M.rel_l2(xg, xl)
            print(f"tensor windows {sp.family} N={sp.N} R={xi.shape[0]}: fwd vs oracle {ef:.2e}, vs lockstep "
                  f"{el:.2e}; adj vs oracle {ea:.2e}, vs lockstep {eal:.2e}")
            assert np.isfinite(y).all() and np.isfinite(xg).all()
            assert ef <= max(10 * eps, 1e-5) and el <= 2e-6
            assert ea <= max(10 * eps, 1e-5) and eal <= 2e-6
    finally:
        close_all(plans)
