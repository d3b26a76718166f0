"""Solver-level pins of the oracle (Alg. 1 with the boundary block).

The minimiser over Delta(tau) is checked against methods that share nothing
with Alg. 1: a one-variable quartic for n = 2, brute-force support
enumeration with Newton on each face, the textbook minimum-variance portfolio,
and accelerated projected gradient.
"""
import math

import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

TAU = 1e-8


def _problem(n, T, seed, lam, mode="standardised", panel="single"):
    R = panels.single_factor_panel(n, T, seed) if panel == "single" else panels.sector_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    return mu, A, O.scale_preferences(lam, A, mode)


@pytest.mark.parametrize("cfg", ["direct", "pcg"])
def test_n2_closed_form(cfg):
    mu, A, c = _problem(2, 300, 21, (0.3, 1.0, 1.0, 1.0))
    # f(t, 1-t) as a quartic in t from the explicit comoment tensors
    Sig, S, K = O.comoment_tensors(A)
    ts = np.linspace(0, 1, 9)
    vals = [(-c[0] * m1 + c[1] * m2 - c[2] * m3 + c[3] * m4)
            for m1, m2, m3, m4 in (O.moments_tensor(mu, Sig, S, K, np.array([t, 1 - t])) for t in ts)]
    poly = np.polyfit(ts, vals, 4)
    cands = [TAU, 1 - TAU] + [r.real for r in np.roots(np.polyder(poly))
                             if abs(r.imag) < 1e-12 and TAU < r.real < 1 - TAU]
    t_best = min(cands, key=lambda t: np.polyval(poly, t))
    x, info = O.solve(A, mu, c, cfg, 1e-12)
    assert info.status == "converged"
    assert x[0] == pytest.approx(t_best, abs=1e-9)


@pytest.mark.parametrize("seed,lam", [(31, (1, 1, 1, 1)), (32, (0.2, 1, 0.5, 2)), (33, (1, 1, 2, 0.5)),
                                      (34, (3, 1, 1, 1))])
def test_support_enumeration_small_n(seed, lam):
    mu, A, c = _problem(5, 200, seed, lam)
    x_bf = O.support_enumeration(A, mu, c, TAU)
    for cfg in ("direct", "pcg"):
        x, info = O.solve(A, mu, c, cfg, 1e-12)
        assert info.status == "converged", (cfg, info.status, info.kkt_rel)
        assert O.objective(A, mu, c, x) <= O.objective(A, mu, c, x_bf) + 1e-12 * abs(O.objective(A, mu, c, x_bf))
        if O.convexity_certificate(c):
            np.testing.assert_allclose(x, x_bf, atol=1e-9)


def test_minimum_variance_closed_form():
    """c1 = c3 = c4 = 0: the minimiser is Sigma^-1 1 / (1^T Sigma^-1 1) when interior."""
    rng = np.random.default_rng(40)
    n, T = 12, 3000
    R = rng.standard_normal((T, n)) * np.linspace(0.8, 1.2, n) * 1e-2
    mu, A = O.centre(R)
    Sig = A.T @ A / T
    w = np.linalg.solve(Sig, np.ones(n))
    w /= w.sum()
    assert w.min() > 0.01
    c = np.array([0.0, 1.0, 0.0, 0.0]) / np.array([1, 1e-4, 1, 1])
    for cfg in ("direct", "pcg"):
        x, info = O.solve(A, mu, c, cfg, 1e-12)
        assert info.status == "converged"
        np.testing.assert_allclose(x, w, atol=1e-10)


def test_agrees_with_projected_gradient():
    mu, A, c = _problem(15, 600, 41, (1, 1, 0.5, 2), panel="sector")
    x_pg = O.projected_gradient(A, mu, c, TAU, iters=20000)
    for cfg in ("direct", "pcg"):
        x, info = O.solve(A, mu, c, cfg, 1e-12)
        assert info.status == "converged"
        f, f_pg = O.objective(A, mu, c, x), O.objective(A, mu, c, x_pg)
        assert f <= f_pg + 1e-12 * abs(f_pg)
        np.testing.assert_allclose(x, x_pg, atol=1e-6)


@pytest.mark.parametrize("cfg", ["direct", "pcg"])
def test_kkt_and_budget_at_termination(cfg):
    mu, A, c = _problem(60, 800, 42, (1, 1, 1, 1), panel="sector")
    x, info = O.solve(A, mu, c, cfg, 1e-10)
    assert info.status == "converged"
    assert abs(x.sum() - 1.0) <= 1e-12
    assert x.min() >= TAU
    g = O.gradient(A, mu, c, x)
    assert O.kkt_residual(x, g, TAU) <= 1e-10 * info.kkt0 * (1 + 1e-9)
    # complementary slackness on the support: g constant on x > tau
    sup = x > TAU + 1e-12
    lam_ = g[sup].mean()
    assert np.max(np.abs(g[sup] - lam_)) <= 1e-8 * np.max(np.abs(g))
    assert np.min(g[~sup] - lam_) >= -1e-8 * np.max(np.abs(g))


def test_degenerate_sizes():
    mu, A, c = _problem(1, 50, 43, (1, 1, 1, 1))
    x, info = O.solve(A, mu, c, "direct", 1e-8)
    assert x.tolist() == [1.0]
    assert info.status == "converged"


def test_calibration_is_monotone_and_meets_target():
    mu, A, c = _problem(40, 1000, 44, (1, 1, 1, 1), panel="sector")
    means = []
    for c1 in np.geomspace(c[1] * 1e-5, c[1] * 1e-1, 7):
        cc = c.copy()
        cc[0] = c1
        x, info = O.solve(A, mu, cc, "direct", 1e-10)
        assert info.status == "converged"
        means.append(mu @ x)
    assert all(b >= a - 1e-12 * np.max(np.abs(mu)) for a, b in zip(means, means[1:]))
    target = 0.5 * (means[2] + means[4])
    cc, x, info, evals = O.calibrate_target(A, mu, c, target, "direct", 1e-10)
    assert abs(mu @ x - target) <= 1e-9 * np.max(np.abs(mu))
    assert info.status == "converged"
    assert evals <= 25
