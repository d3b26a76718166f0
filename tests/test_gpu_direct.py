"""Direct configuration on the GPU against the CPU oracle (C ABI).

The weighted Gram is held to the FP64 summation bound 1e-12 * (|A|^T |D| |A| / T).
The direct direction involves no Krylov iteration, so it must match the
oracle's exact-trace direction to rounding amplified by the reduced
Hessian's condition number.  Solves match the oracle's minimiser.
"""
import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu


def _ctx(R, prec, lam, target=np.nan):
    import paper_2604_25378_gb300 as m
    ctx = m.MVSK(R, prec)
    ctx.set_prefs(np.asarray(lam, float), target)
    return ctx


@pytest.mark.parametrize("n,T", [(20, 500), (300, 3001), (70, 64), (3, 40)])
def test_gram_fp64(n, T):
    R = panels.sector_factor_panel(n, T, 5) if n >= 5 else panels.single_factor_panel(n, T, 5)
    mu, A = O.centre(R)
    lam = (1.0, 1.0, 0.5, 2.0)
    c = O.scale_preferences(lam, A, "standardised")
    x = np.random.default_rng(1).dirichlet(np.ones(n))
    G = _ctx(R, "fp64", lam).gram(x)
    D = O.d2psi(c, A @ x)
    scale = np.abs(A).T @ (np.abs(D)[:, None] * np.abs(A)) / T
    np.testing.assert_array_less(np.abs(G - O.gram(A, c, x)), 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("n,T,seed", [(40, 600, 5), (150, 2000, 6)])
def test_direct_direction_matches_oracle(n, T, seed):
    R = panels.sector_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    lam = (1.0, 1.0, 1.0, 1.0)
    c = O.scale_preferences(lam, A, "standardised")
    x = np.random.default_rng(seed).dirichlet(np.ones(n) * 4)
    ctx = _ctx(R, "fp64", lam)
    d_gpu = ctx.direction(x, 0, 0)
    d_ref, info = O.direction_direct(A, c, A @ x, O.gradient(A, mu, c, x), np.ones(n, dtype=bool), 0.0)
    np.testing.assert_allclose(d_gpu, d_ref, rtol=0, atol=1e-9 * np.max(np.abs(d_ref)))


@pytest.mark.parametrize("n,T,seed,lam,panel", [(20, 500, 0, (1, 1, 1, 1), "single"),
                                                (100, 1500, 11, (1, 1, 2, 0.5), "sector"),
                                                (500, 5000, 1, (1, 1, 1, 1), "sector")])
def test_direct_fp64_matches_oracle(n, T, seed, lam, panel):
    R = panels.single_factor_panel(n, T, seed) if panel == "single" else panels.sector_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    c = O.scale_preferences(lam, A, "standardised")
    x_ref, inf_ref = O.solve(A, mu, c, "direct", 1e-10)
    assert inf_ref.status == "converged"
    ctx = _ctx(R, "fp64", lam)
    w, info = ctx.solve(0, 1e-10)
    assert info["status"] == "ok", info
    g = O.gradient(A, mu, c, w)
    assert O.kkt_residual(w, g, 1e-8) <= 1e-10 * inf_ref.kkt0 * 1.0001
    if O.convexity_certificate(c):
        assert np.max(np.abs(w - x_ref)) <= 1e-9
    else:
        assert O.objective(A, mu, c, w) <= inf_ref.f + 1e-9 * abs(inf_ref.f) or np.max(np.abs(w - x_ref)) <= 1e-9


def test_direct_target_sweep_c2():
    """C2: n = 500, T = 5000, 2 of the 8 return targets, direct configuration."""
    R, lams, tg = panels.workload("c2_direct_n500_T5000")
    mu, A = O.centre(R)
    c = O.scale_preferences(lams[0], A, "standardised")
    for target in tg[[1, 6]]:
        cc, x_ref, inf_ref, ev = O.calibrate_target(A, mu, c, target, "direct", 1e-9)
        ctx = _ctx(R, "fp64", lams[0], target)
        w, info = ctx.solve(0, 1e-9)
        assert info["status"] == "ok"
        assert abs(info["achieved_mean"] - target) <= 1e-9 * np.max(np.abs(mu))
        assert np.max(np.abs(w - x_ref)) <= 1e-7


@pytest.mark.parametrize("n,T", [(300, 3001), (20, 500), (3, 40), (129, 64)])
def test_gram_bf16_tensor_cores(n, T):
    """tcgen05 BF16 x BF16 -> FP32 Gram against the FP64 oracle: the operands A
    and Diag(psi'')A are rounded to BF16 (2^-9 relative), so the bound is
    2e-2 * (|A|^T |D| |A| / T)."""
    R = panels.sector_factor_panel(n, T, 5) if n >= 5 else panels.single_factor_panel(n, T, 5)
    mu, A = O.centre(R)
    lam = (1.0, 1.0, 0.5, 2.0)
    c = O.scale_preferences(lam, A, "standardised")
    x = np.random.default_rng(1).dirichlet(np.ones(n))
    ctx = _ctx(R, "bf16", lam)
    ctx.set_option("oracle_prec", 1)
    G = ctx.gram(x)
    D = O.d2psi(c, A @ x)
    scale = np.abs(A).T @ (np.abs(D)[:, None] * np.abs(A)) / T
    Gr = O.gram(A, c, x)
    np.testing.assert_array_less(np.abs(G - Gr), 2e-2 * scale + 1e-300)
    # and it is not trivially small: the relative Frobenius error is at BF16 level
    assert np.linalg.norm(G - Gr) <= 1e-2 * np.linalg.norm(Gr)
