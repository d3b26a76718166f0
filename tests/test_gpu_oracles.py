"""GPU parity of the sample-oracle kernels against the CPU oracle (C ABI).

FP64 results must agree to rounding: the bound scales with sum |terms| of
each reduction (the same quantity that bounds floating-point summation
error), times 1e-12.  BF16/FP32 copies of A are held to 1e-2 / 1e-5 of the
same scale (storage rounding of A is 2^-9 / 2^-24 relative).
"""
import math

import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu

SHAPES = [(20, 500), (300, 3001), (64, 152), (3, 1), (2, 97), (1, 40), (1000, 2500)]


def _ctx(R, prec="fp64", lam=(1.0, 1.0, 0.5, 2.0)):
    import paper_2604_25378_gb300 as m
    ctx = m.MVSK(R, prec)
    ctx.set_prefs(np.asarray(lam))
    return ctx


def _setup(n, T, seed=0, lam=(1.0, 1.0, 0.5, 2.0)):
    R = panels.sector_factor_panel(n, T, seed) if n >= 5 else panels.single_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    c = O.scale_preferences(lam, A, "standardised")
    rng = np.random.default_rng(seed + 7)
    x = rng.dirichlet(np.ones(n))
    return R, mu, A, c, x, rng


@pytest.mark.parametrize("n,T", SHAPES)
def test_eval_value_gradient_kkt(n, T):
    R, mu, A, c, x, rng = _setup(n, T)
    ctx = _ctx(R)
    f, g, kkt = ctx.eval(x)
    z = A @ x
    scale = np.abs(A).T @ np.abs(O.dpsi(c, z)) / T + abs(c[0]) * np.abs(mu)
    np.testing.assert_array_less(np.abs(g - O.gradient(A, mu, c, x)), 1e-12 * scale + 1e-300)
    fs = abs(c[0] * (mu @ x)) + np.sum(np.abs(O.psi(c, z))) / T
    assert abs(f - O.objective(A, mu, c, x)) <= 1e-12 * fs
    assert kkt == pytest.approx(O.kkt_residual(x, O.gradient(A, mu, c, x), 1e-8), rel=1e-9, abs=1e-14)


@pytest.mark.parametrize("n,T", SHAPES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("bf16", 2e-2)])
def test_hvp_and_third(n, T, prec, tol):
    R, mu, A, c, x, rng = _setup(n, T, seed=1)
    ctx = _ctx(R, prec)
    ctx.set_option("oracle_prec", {"fp64": 0, "bf16": 1, "fp32": 2}[prec])
    v, u = rng.standard_normal((2, n))
    z = A @ x
    hv = ctx.hvp(x, v)
    scale = np.abs(A).T @ (np.abs(O.d2psi(c, z)) * (np.abs(A) @ np.abs(v))) / T
    np.testing.assert_array_less(np.abs(hv - O.hvp(A, c, x, v)), tol * scale + 1e-300)
    t3 = ctx.third(x, u, v)
    scale3 = np.abs(A).T @ (np.abs(O.d3psi(c, z)) * (np.abs(A) @ np.abs(u)) * (np.abs(A) @ np.abs(v))) / T
    np.testing.assert_array_less(np.abs(t3 - O.third(A, c, x, u, v)), tol * scale3 + 1e-300)


@pytest.mark.parametrize("n,T", SHAPES)
def test_line_search_coefficients_and_cap(n, T):
    R, mu, A, c, x, rng = _setup(n, T, seed=2)
    ctx = _ctx(R)
    d = rng.standard_normal(n)
    d -= d.mean()
    coef, am = ctx.line_search(x, d)
    ref = O.quartic_coefficients(c, mu, x, d, O.power_sums(A @ x, A @ d))
    z, w = np.abs(A @ x), np.abs(A @ d)
    sc = np.array([abs(c[0] * (mu @ x)) + np.sum(c[1] * z**2 + c[2] * z**3 + c[3] * z**4) / T,
                   abs(c[0] * (mu @ d)) + np.sum(2 * c[1] * z * w + 3 * c[2] * z**2 * w + 4 * c[3] * z**3 * w) / T,
                   np.sum(c[1] * w**2 + 3 * c[2] * z * w**2 + 6 * c[3] * z**2 * w**2) / T,
                   np.sum(c[2] * w**3 + 4 * c[3] * z * w**3) / T,
                   np.sum(c[3] * w**4) / T])
    np.testing.assert_array_less(np.abs(coef - ref), 1e-12 * sc + 1e-300)
    ref_am = O.alpha_max(x, d, 1e-8)
    if n == 1:
        assert am == math.inf or am == pytest.approx(ref_am)
    else:
        assert am == pytest.approx(ref_am, rel=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 300, 6144])
def test_projection(n):
    rng = np.random.default_rng(n)
    R = panels.single_factor_panel(n, 8, 0)
    ctx = _ctx(R)
    for tau in (1e-8, 0.1 / n):
        v = rng.standard_normal(n) * (3.0 / n)
        p = ctx.project_slice(v, tau)
        np.testing.assert_allclose(p, O.project_slice(v, tau), rtol=0, atol=1e-15)


# Inputs that stress the two-stage threshold search (FP32 estimate, FP64
# finish): cancellation between large values, a few huge entries among tiny
# ones, ties, constant and subnormal-scale vectors, and a C4-sized x - g.
def _hard_vectors(n, rng):
    big = rng.choice([-1.0, 1.0], n) * 1e6 + rng.standard_normal(n)
    spiky = rng.standard_normal(n) * 1e-9
    spiky[rng.choice(n, size=min(n, 3), replace=False)] = [5e3, -7e3, 2e3][: min(n, 3)]
    ties = np.repeat(rng.standard_normal(max(1, n // 50)), 50)[:n]
    ties = np.concatenate([ties, np.zeros(n - len(ties))])
    const = np.full(n, 0.25)
    tiny = rng.standard_normal(n) * 1e-310
    xg = np.full(n, 1.0 / n) - rng.standard_normal(n) * 0.05 - 0.2 * (rng.random(n) < 0.01)
    return {"big": big, "spiky": spiky, "ties": ties, "const": const, "tiny": tiny, "xg": xg}


@pytest.mark.parametrize("n", [5, 1000, 5440, 6144])
def test_projection_hard_cases(n):
    rng = np.random.default_rng(100 + n)
    R = panels.single_factor_panel(n, 8, 0)
    ctx = _ctx(R)
    for name, v in _hard_vectors(n, rng).items():
        for tau in (1e-8, 0.0):
            p = ctx.project_slice(v, tau)
            ref = O.project_slice(v, tau)
            # theta = (sum_S u - b) / |S| is summed in another order on each
            # side (the oracle by a running sum): each differs from the exact
            # value by at most about eps (sum_S |u| + |b|) (the running sum's
            # bound |S| eps sum_S |u|, over |S|), so the projections agree to
            # a few times that
            S = ref > tau
            scale = 1.0 + np.sum(np.abs(v[S])) + np.max(np.abs(v))
            np.testing.assert_allclose(p, ref, rtol=0, atol=8 * 2.0**-52 * scale, err_msg=name)
            assert np.all(p >= tau), name
            assert abs(np.sum(p) - 1.0) <= 1e-12 * scale * max(1, np.sum(p > tau)), name


def test_quartic_argmin_matches_oracle_routine():
    R = panels.single_factor_panel(3, 8, 0)
    ctx = _ctx(R)
    rng = np.random.default_rng(5)
    cases = [([0, -1.0, 0, 0, 0], 2.0), ([0, -1.0, 2.0, 0, 0], 2.0), ([0, -3.0, 0, 1.0, 0], 5.0),
             ([0, 1.0, 1.0, 0, 0], 1.0), ([0, -1.0, 0, 0, 0], 0.0), ([0, -1.29e-8, 2.3, 0.066, 3.1], 0.09)]
    for _ in range(200):
        coef = rng.standard_normal(5) * 10.0 ** rng.uniform(-6, 3, 5)
        cases.append((coef, float(rng.uniform(0.01, 5))))
    for coef, am in cases:
        a_gpu = ctx.quartic_argmin(coef, am)
        a_ref = O.quartic_argmin(np.asarray(coef, float), am)
        dg = O._decrease(np.asarray(coef, float), a_gpu)
        dr = O._decrease(np.asarray(coef, float), a_ref)
        assert a_gpu == a_ref or abs(dg - dr) <= 1e-14 * (abs(dr) + 1e-300)


@pytest.mark.slow
def test_full_size_eval_sampled():
    """n = 5440, T = 12000 (the batched-sweep panel shape): gradient, f and KKT
    in the launch configuration the solver uses."""
    R = panels.garch_sector_panel(5440, 12000, 3)
    mu, A = O.centre(R)
    c = O.scale_preferences((1, 1, 0.5, 2), A, "standardised")
    x = np.random.default_rng(0).dirichlet(np.ones(5440))
    ctx = _ctx(R, "bf16", (1, 1, 0.5, 2))
    f, g, kkt = ctx.eval(x)
    z = A @ x
    scale = np.abs(A).T @ np.abs(O.dpsi(c, z)) / 12000 + abs(c[0]) * np.abs(mu)
    np.testing.assert_array_less(np.abs(g - O.gradient(A, mu, c, x)), 1e-12 * scale)
    assert f == pytest.approx(O.objective(A, mu, c, x), rel=1e-11)
    ctx.set_option("oracle_prec", 1)
    v = np.random.default_rng(1).standard_normal(5440)
    hv = ctx.hvp(x, v)
    sc = np.abs(A).T @ (np.abs(O.d2psi(c, z)) * (np.abs(A) @ np.abs(v))) / 12000
    np.testing.assert_array_less(np.abs(hv - O.hvp(A, c, x, v)), 2e-2 * sc)
