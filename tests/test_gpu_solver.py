"""GPU YAND-MVSK solves (C ABI) against the CPU oracle.

FP64 path: under the convexity certificate the minimiser over Delta(tau) is
unique, so the GPU and oracle solutions must agree to ||w - w*||_inf <= 1e-9
when the reduced Hessian on the optimal face is well conditioned (its
smallest eigenvalue is reported by the test on failure).  Mixed precision
(BF16/FP32 direction passes, FP64 gradient/line search): the same KKT
tolerance is met in FP64, hence the same minimiser to the same bound.
"""
import math

import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu


def _problem(n, T, seed, lam, panel="sector"):
    if panel == "sector":
        R = panels.sector_factor_panel(n, T, seed)
    elif panel == "garch":
        R = panels.garch_sector_panel(n, T, seed)
    else:
        R = panels.single_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    c = O.scale_preferences(lam, A, "standardised")
    return R, mu, A, c


def _ctx(R, prec, lam, target=math.nan):
    import paper_2604_25378_gb300 as m
    ctx = m.MVSK(R, prec)
    ctx.set_prefs(np.asarray(lam, float), target)
    return ctx


def _face_lmin(A, c, x):
    sup = np.nonzero(x > 1e-8 + 1e-12)[0]
    if sup.size < 2:
        return math.inf
    U = O.tangent_basis(sup.size)
    G = O.gram(A, c, x)[np.ix_(sup, sup)]
    return float(np.min(np.linalg.eigvalsh(U.T @ G @ U)))


@pytest.mark.parametrize("n,T,seed,lam", [(20, 500, 0, (1, 1, 1, 1)), (60, 800, 42, (1, 1, 0.5, 2)),
                                          (200, 2000, 1, (1, 1, 1, 1)), (7, 64, 3, (3, 1, 1, 1))])
def test_pcg_fp64_matches_oracle(n, T, seed, lam):
    R, mu, A, c = _problem(n, T, seed, lam, "single" if n == 20 else "sector")
    x_ref, inf_ref = O.solve(A, mu, c, "pcg", 1e-10)
    assert inf_ref.status == "converged"
    ctx = _ctx(R, "fp64", lam)
    w, info = ctx.solve(1, 1e-10)
    assert info["status"] == "ok", info
    assert info["kkt_rel"] <= 1e-10
    assert abs(w.sum() - 1.0) <= 1e-12 and w.min() >= 1e-8
    g = O.gradient(A, mu, c, w)
    assert O.kkt_residual(w, g, 1e-8) <= 1e-10 * inf_ref.kkt0 * 1.0001
    lmin = _face_lmin(A, c, x_ref)
    assert np.max(np.abs(w - x_ref)) <= 1e-9, (np.max(np.abs(w - x_ref)), lmin)
    assert info["f"] == pytest.approx(inf_ref.f, rel=1e-12, abs=1e-15)


def test_pcg_direction_matches_oracle_step():
    """One affine-normal direction (PCG, Hutchinson probes of the same
    counter-based stream) at an interior point.  Finite-precision CG amplifies
    rounding differences with the condition number of the preconditioned
    system, so per-iteration parity is checked on the paper's stylised panel
    (U[-0.1, 0.4], raw profile [1,10,1,10]), whose reduced Hessian is well
    conditioned (Table ec-hessian-conditioning)."""
    R = panels.uniform_panel(40, 252, 5)
    mu, A = O.centre(R)
    lam = (1.0, 10.0, 1.0, 10.0)
    c = np.asarray(lam)
    x = np.random.default_rng(2).dirichlet(np.ones(40) * 5)
    import paper_2604_25378_gb300 as m
    ctx = m.MVSK(R, "fp64")
    ctx.set_option("pref_scaling", 0)
    ctx.set_prefs(np.asarray(lam))
    for it in (0, 3):
        d_gpu = ctx.direction(x, 1, it)
        F = np.ones(40, dtype=bool)
        d_ref, _ = O.direction_pcg(A, c, A @ x, O.gradient(A, mu, c, x), F, 1e-4, O.Options(), it)
        np.testing.assert_allclose(d_gpu, d_ref, rtol=0, atol=1e-8 * np.max(np.abs(d_ref)))


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_mixed_precision_reaches_fp64_minimiser(prec):
    R, mu, A, c = _problem(300, 3000, 7, (1, 1, 0.5, 2), "garch")
    x_ref, inf_ref = O.solve(A, mu, c, "pcg", 1e-10)
    ctx = _ctx(R, prec, (1, 1, 0.5, 2))
    w, info = ctx.solve(1, 1e-10)
    assert info["status"] == "ok", info
    g = O.gradient(A, mu, c, w)
    assert O.kkt_residual(w, g, 1e-8) <= 1e-10 * inf_ref.kkt0 * 1.0001
    assert np.max(np.abs(w - x_ref)) <= 1e-9


def test_nonconvex_preferences_reach_kkt_point():
    """(1,1,2,0.5) lies outside the certificate: compare KKT and objective."""
    R, mu, A, c = _problem(100, 1500, 11, (1, 1, 2, 0.5))
    x_ref, inf_ref = O.solve(A, mu, c, "pcg", 1e-9)
    ctx = _ctx(R, "fp64", (1, 1, 2, 0.5))
    w, info = ctx.solve(1, 1e-9)
    assert info["status"] == "ok"
    g = O.gradient(A, mu, c, w)
    assert O.kkt_residual(w, g, 1e-8) <= 1e-9 * inf_ref.kkt0 * 1.0001
    if np.max(np.abs(w - x_ref)) > 1e-9:
        assert O.objective(A, mu, c, w) == pytest.approx(inf_ref.f, rel=1e-6)


def test_target_calibration_matches_oracle():
    R, mu, A, c = _problem(80, 1200, 13, (1, 1, 1, 1))
    target = panels.quantile_targets(R, [0.7])[0]
    cc, x_ref, inf_ref, ev = O.calibrate_target(A, mu, c, target, "pcg", 1e-10)
    ctx = _ctx(R, "fp64", (1, 1, 1, 1), target)
    w, info = ctx.solve(1, 1e-10)
    assert info["status"] == "ok"
    assert abs(info["achieved_mean"] - target) <= 1e-9 * np.max(np.abs(mu))
    assert info["c"][0] == pytest.approx(cc[0], rel=1e-6)
    assert np.max(np.abs(w - x_ref)) <= 1e-7


def test_warm_start_and_errors():
    import paper_2604_25378_gb300 as m
    R, mu, A, c = _problem(30, 400, 17, (1, 1, 1, 1))
    ctx = m.MVSK(R, "fp64")
    with pytest.raises(m.MvskError) as e:
        ctx.solve(1, 1e-8)
    assert e.value.status == 6  # ESTATE: prefs first
    ctx.set_prefs(np.array([1.0, 1, 1, 1]))
    w, info = ctx.solve(1, 1e-10)
    w2, info2 = ctx.solve(1, 1e-10, w0=w)
    assert info2["iters"] <= 1 and np.max(np.abs(w2 - w)) <= 1e-12
    with pytest.raises(m.MvskError):
        ctx.solve(1, 1e-8, w0=np.full(30, 0.5))
    with pytest.raises(m.MvskError):
        ctx.set_prefs(np.array([1.0, -1, 1, 1]))
    with pytest.raises(m.MvskError):
        ctx.set_option("no_such_option", 1.0)
    ctx.set_option("pcg_max_iter", 2)
    ctx.set_option("restart_iter", 1)
    w3, info3 = ctx.solve(1, 1e-14)
    assert info3["status"] == "not_converged"
    bad = R.copy()
    bad[3, 4] = np.nan
    with pytest.raises(m.MvskError):
        m.MVSK(bad, "fp64")


def test_pcg_direction_bf16_tensor_cores():
    """PCG direction whose Hessian-vector and third-order products run on the
    tensor cores (BF16 A, FP32 accumulate) against the FP64 oracle direction on
    a well-conditioned panel: BF16 operator error (~2^-8) propagates through
    15 CG iterations, so the bound is 5e-2 of ||d||."""
    R = panels.uniform_panel(200, 1000, 8)
    mu, A = O.centre(R)
    lam = (1.0, 10.0, 1.0, 10.0)
    c = np.asarray(lam)
    x = np.random.default_rng(3).dirichlet(np.ones(200) * 5)
    import paper_2604_25378_gb300 as m
    ctx = m.MVSK(R, "bf16")
    ctx.set_option("pref_scaling", 0)
    ctx.set_prefs(np.asarray(lam))
    d_gpu = ctx.direction(x, 1, 2)
    d_ref, _ = O.direction_pcg(A, c, A @ x, O.gradient(A, mu, c, x), np.ones(200, dtype=bool), 1e-4, O.Options(), 2)
    assert np.linalg.norm(d_gpu - d_ref) <= 5e-2 * np.linalg.norm(d_ref)
    assert abs(d_gpu.sum()) <= 1e-12 * np.max(np.abs(d_gpu))


@pytest.mark.parametrize("split_products", [1, 0])
def test_batched_lockstep_matches_oracle(split_products):
    """mvsk_solve_batch (PCG, BF16 direction products shared by all instances on
    the tensor cores) against the oracle, instance by instance: preference
    vectors inside and outside the certificate, with and without targets.
    split_products = 1: value, gradient and line-search products as split
    tensor-core products; 0: FP64 streaming passes."""
    import paper_2604_25378_gb300 as m
    R = panels.garch_sector_panel(200, 2000, 9)
    mu, A = O.centre(R)
    lams = np.array([(1, 1, 0.5, 2), (1, 1, 2, 0.5), (1, 1, 1, 1), (0.5, 1, 0.5, 2)], dtype=float)
    tg = panels.quantile_targets(R, [0.6, 0.7])
    targets = np.array([np.nan, np.nan, tg[0], tg[1]])
    ctx = m.MVSK(R, "bf16")
    ctx.set_option("split_products", split_products)
    W, infos = ctx.solve_batch(lams, targets, m.PCG, 1e-10)
    for b in range(4):
        c = O.scale_preferences(lams[b], A, "standardised")
        if np.isnan(targets[b]):
            x_ref, inf_ref = O.solve(A, mu, c, "pcg", 1e-10)
            tol_w = 1e-9
        else:
            c, x_ref, inf_ref, ev = O.calibrate_target(A, mu, c, targets[b], "pcg", 1e-10)
            tol_w = 1e-7
            assert abs(infos[b]["achieved_mean"] - targets[b]) <= 1e-9 * np.max(np.abs(mu))
        assert infos[b]["status"] == "ok", (b, infos[b])
        # judged by the oracle alone, for the coefficients the GPU solved with
        cg = np.asarray(infos[b]["c"])
        x0 = np.full(A.shape[1], 1.0 / A.shape[1])
        k0 = O.kkt_residual(x0, O.gradient(A, mu, cg, x0), 1e-8)
        assert O.kkt_residual(W[b], O.gradient(A, mu, cg, W[b]), 1e-8) <= 1.5e-10 * k0
        if O.convexity_certificate(c):
            assert np.max(np.abs(W[b] - x_ref)) <= tol_w, (b, np.max(np.abs(W[b] - x_ref)))
        else:
            assert O.objective(A, mu, c, W[b]) <= inf_ref.f + 1e-9 * abs(inf_ref.f) or np.max(np.abs(W[b] - x_ref)) <= tol_w
    # a single-instance solve of the same problem gives the same point
    ctx.set_prefs(lams[0])
    w0, inf0 = ctx.solve(m.PCG, 1e-10)
    assert np.max(np.abs(w0 - W[0])) <= 1e-9


def test_batched_more_than_64_instances():
    """70 instances: the split products run in groups of 64 and 6 vectors."""
    import paper_2604_25378_gb300 as m
    R = panels.sector_factor_panel(30, 400, 4)
    mu, A = O.centre(R)
    rng = np.random.default_rng(5)
    lams = np.column_stack([np.ones(70), np.ones(70), rng.uniform(0.3, 2.5, 70), rng.uniform(0.3, 2.5, 70)])
    ctx = m.MVSK(R, "bf16")
    W, infos = ctx.solve_batch(lams, np.full(70, np.nan), m.PCG, 1e-10)
    assert all(i["status"] == "ok" for i in infos), [i["status"] for i in infos]
    for b in (0, 31, 63, 64, 69):
        c = O.scale_preferences(lams[b], A, "standardised")
        x_ref, inf_ref = O.solve(A, mu, c, "pcg", 1e-10)
        g = O.gradient(A, mu, c, W[b])
        assert O.kkt_residual(W[b], g, 1e-8) <= 1e-9 * inf_ref.kkt0
        if O.convexity_certificate(c):
            assert np.max(np.abs(W[b] - x_ref)) <= 1e-9, (b, np.max(np.abs(W[b] - x_ref)))


def test_profile_stride_samples_launches():
    """mvsk_profile_stride(k) brackets every k-th launch of the selected kinds:
    the same batched solve (deterministic; the iteration graph is captured per
    solve, and the correction-column PCG step runs 15 times in it) profiled
    with stride 1 and 3 records a third as many launches of that kind, over the
    same kernel launches; a stride below 1 is EINVAL."""
    import paper_2604_25378_gb300 as m
    R = panels.sector_factor_panel(40, 600, 3)
    lams = np.array([(1, 1, 1, 1), (1, 1, 0.5, 2)], dtype=float)
    ctx = m.MVSK(R, "bf16")
    ctx.set_option("face_small", 0)  # the per-step products and steps in every iteration
    ctx.solve_batch(lams, np.full(2, np.nan), m.PCG, 1e-10)  # buffers built
    counts = {}
    for k in (1, 3):
        ctx.profile_only("k_pcg_step_a")
        ctx.profile_stride(k)
        ctx.profile_enable(True)
        ctx.solve_batch(lams, np.full(2, np.nan), m.PCG, 1e-10)
        prof, launches = ctx.profile_read()
        ctx.profile_enable(False)
        counts[k] = (prof["k_pcg_step_a"]["launches"], launches)
    ctx.profile_stride(1)
    ctx.profile_only(None)
    assert counts[1][1] == counts[3][1] and counts[1][0] >= 15
    assert counts[3][0] * 3 == counts[1][0], counts
    with pytest.raises(Exception):
        ctx.profile_stride(0)


def test_batch_lanes_queue_matches_all_at_once():
    """batch_lanes = 8 for 40 requests (continuous batching: a lane whose
    request has finished takes the next) gives the requests the same
    solutions as advancing all 40 together; warm starts at those solutions
    reach each request in its lane (a few iterations each)."""
    import paper_2604_25378_gb300 as m
    R = panels.sector_factor_panel(30, 400, 21)
    mu, A = O.centre(R)
    rng = np.random.default_rng(22)
    k = 40
    lams = np.column_stack([np.ones(k), np.ones(k), rng.uniform(0.4, 2.5, k), rng.uniform(0.4, 2.5, k)])
    tg = np.where(rng.uniform(size=k) < 0.3, np.quantile(R.mean(0), 0.7), np.nan)
    ctx = m.MVSK(R, "bf16")
    W_all, inf_all = ctx.solve_batch(lams, tg, m.PCG, 1e-10)
    ctx.set_option("batch_lanes", 8)
    W_q, inf_q = ctx.solve_batch(lams, tg, m.PCG, 1e-10)
    assert all(i["status"] == "ok" for i in inf_all + inf_q)
    for b in range(k):
        c = np.asarray(inf_q[b]["c"])
        if O.convexity_certificate(c):
            assert np.max(np.abs(W_q[b] - W_all[b])) <= 1e-8, (b, np.max(np.abs(W_q[b] - W_all[b])))
        g = O.gradient(A, mu, c, W_q[b])
        assert O.kkt_residual(W_q[b], g, 1e-8) <= 1e-9 * inf_q[b]["kkt0"]
    free = np.isnan(tg)
    W_w, inf_w = ctx.solve_batch(lams, tg, m.PCG, 1e-10, W0=W_q)
    its_w = np.array([i["iters"] for i in inf_w])
    its_c = np.array([i["iters"] for i in inf_q])
    assert np.all(its_w[free] <= 3), its_w[free]
    assert np.all(its_w[free] < its_c[free])
    ctx.set_option("batch_lanes", 0)


def test_group_calibration_matches_per_request():
    """Requests that share (c2, c3, c4) and carry targets start their mean-
    coefficient calibration on a shared c1 grid (option group_calibration, on
    by default): each request must reach the same calibrated c1 and weights as
    when every request runs its own sequence from c1 = 0.  The targets include
    one met at c1 = 0 (below the minimum-risk portfolio's mean), ones inside
    the grid and one beyond its top (growth), on two preference vectors; a
    request without a target shares the batch."""
    import paper_2604_25378_gb300 as m
    R = panels.garch_sector_panel(300, 3000, 31)
    mu, A = O.centre(R)
    qs = panels.quantile_targets(R, [0.5, 0.7, 0.8, 0.9, 0.97, 0.995])
    lams, tgs = [], []
    for lam in [(1.0, 1.0, 0.5, 2.0), (1.0, 1.0, 2.0, 2.0)]:
        c = O.scale_preferences(lam, A, "standardised")
        c0 = c.copy()
        c0[0] = 0.0
        x0, _ = O.solve(A, mu, c0, "pcg", 1e-10)
        low = float(mu @ x0) - 0.1 * float(np.std(mu))       # met at c1 = 0
        for t in [low, *qs]:
            lams.append(lam)
            tgs.append(t)
    lams.append((1.0, 1.0, 0.5, 2.0))
    tgs.append(np.nan)
    lams, tgs = np.asarray(lams), np.asarray(tgs)
    ctx = m.MVSK(R, "bf16")
    W1, inf1 = ctx.solve_batch(lams, tgs, m.PCG, 1e-10)
    ctx.set_option("group_calibration", 0)
    W0, inf0 = ctx.solve_batch(lams, tgs, m.PCG, 1e-10)
    ctx.set_option("group_calibration", 1)
    assert all(i["status"] == "ok" for i in inf1 + inf0)
    scale = np.max(np.abs(mu))
    for b in range(len(tgs)):
        c1g, c10 = inf1[b]["c"][0], inf0[b]["c"][0]
        if not np.isnan(tgs[b]):
            assert abs(inf1[b]["achieved_mean"] - tgs[b]) <= 1e-9 * scale or c1g == 0.0, b
        assert abs(c1g - c10) <= 1e-6 * max(c10, 1e-300) or (c1g == 0.0 and c10 == 0.0), (b, c1g, c10)
        assert np.max(np.abs(W1[b] - W0[b])) <= 1e-8, (b, np.max(np.abs(W1[b] - W0[b])))
        cg = np.asarray(inf1[b]["c"])
        x0 = np.full(A.shape[1], 1.0 / A.shape[1])
        k0 = O.kkt_residual(x0, O.gradient(A, mu, cg, x0), 1e-8)
        assert O.kkt_residual(W1[b], O.gradient(A, mu, cg, W1[b]), 1e-8) <= 1.5e-10 * k0, b
        assert inf1[b]["kkt0"] == pytest.approx(k0, rel=1e-9), b
    assert inf1[0]["c"][0] == 0.0 and inf1[7]["c"][0] == 0.0   # the low targets
    # the oracle's calibration of one grid request
    b = 3
    c = O.scale_preferences(lams[b], A, "standardised")
    cc, x_ref, _, _ = O.calibrate_target(A, mu, c, tgs[b], "pcg", 1e-12, rel_tol=1e-12)
    assert np.max(np.abs(W1[b] - x_ref)) <= 1e-7


def test_small_face_direction_matches_products():
    """Once every working face of a batch has at most 320 coordinates, the
    direction block forms each face's Gram matrix and runs both PCG rounds
    on it (option face_small, on by default; in the narrow launch shape while
    every face has at most 128, option value 2 keeps the wide one) instead of
    the tensor-core products on the union of the faces: every form must reach
    the same minimisers (judged by the oracle's KKT residual), and the
    products-only form must agree with the oracle's own minimiser under the
    certificate."""
    import paper_2604_25378_gb300 as m
    R = panels.garch_sector_panel(600, 6000, 41)
    mu, A = O.centre(R)
    lams = np.array([(1, 1, 0.5, 2), (1, 1, 2, 0.5), (1, 1, 1, 1), (0.5, 1, 0.5, 2), (1, 1, 2, 2)], dtype=float)
    tg = np.array([np.nan, np.nan, np.nan, panels.quantile_targets(R, [0.7])[0], np.nan])
    ctx = m.MVSK(R, "bf16")
    W1, inf1 = ctx.solve_batch(lams, tg, m.PCG, 1e-10)
    ctx.set_option("face_small", 0)
    W0, inf0 = ctx.solve_batch(lams, tg, m.PCG, 1e-10)
    ctx.set_option("face_small", 2)
    W2, inf2 = ctx.solve_batch(lams, tg, m.PCG, 1e-10)
    ctx.set_option("face_small", 1)
    x0 = np.full(600, 1.0 / 600)
    for b in range(len(lams)):
        assert inf1[b]["status"] == "ok" and inf0[b]["status"] == "ok", (b, inf1[b], inf0[b])
        assert inf2[b]["status"] == "ok", (b, inf2[b])
        cg = np.asarray(inf1[b]["c"])
        k0 = O.kkt_residual(x0, O.gradient(A, mu, cg, x0), 1e-8)
        assert O.kkt_residual(W1[b], O.gradient(A, mu, cg, W1[b]), 1e-8) <= 1.5e-10 * k0, b
        cg2 = np.asarray(inf2[b]["c"])
        assert O.kkt_residual(W2[b], O.gradient(A, mu, cg2, W2[b]), 1e-8) <= 1.5e-10 * k0, b
        if O.convexity_certificate(cg):
            assert np.max(np.abs(W1[b] - W0[b])) <= 1e-8, (b, np.max(np.abs(W1[b] - W0[b])))
            assert np.max(np.abs(W1[b] - W2[b])) <= 1e-8, (b, np.max(np.abs(W1[b] - W2[b])))
    c = O.scale_preferences(lams[0], A, "standardised")
    x_ref, _ = O.solve(A, mu, c, "pcg", 1e-12)
    assert np.max(np.abs(W1[0] - x_ref)) <= 1e-9
