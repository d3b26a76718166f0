"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
explicit comoment tensors (Sec. 2), finite-difference stencils that are exact
for polynomials, Vandermonde interpolation and dense grids for the quartic
line search (Prop. quartic exact line search), closed forms, brute force,
and a published reference sequence for the probe generator.
"""
import json
import math
import os

import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(n=5, T=40, seed=0, c=(0.3, 1.0, 0.7, 2.0)):
    R = panels.single_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    rng = np.random.default_rng(seed + 100)
    x = rng.dirichlet(np.ones(n))
    return mu, A, np.asarray(c, dtype=np.float64), x, rng


# --------------------------------------------------------------- Sec. 2 / Prop. 1


def test_centring_definition():
    R = panels.single_factor_panel(7, 33, 3)
    mu, A = O.centre(R)
    for j in range(7):
        assert abs(mu[j] - math.fsum(R[:, j]) / 33) <= 1e-17
    assert np.max(np.abs(A.sum(axis=0))) <= 1e-15  # 1_T^T A = 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_operators_match_explicit_comoment_tensors(seed):
    mu, A, c, x, rng = small_problem(seed=seed)
    Sig, S, K = O.comoment_tensors(A)
    m1, m2, m3, m4 = O.moments_tensor(mu, Sig, S, K, x)
    f_tensor = -c[0] * m1 + c[1] * m2 - c[2] * m3 + c[3] * m4
    assert O.objective(A, mu, c, x) == pytest.approx(f_tensor, rel=1e-13)
    # gradient of the tensor polynomial, written out from the multilinear forms
    g_tensor = (-c[0] * mu + 2 * c[1] * Sig @ x - 3 * c[2] * np.einsum("ijk,j,k->i", S, x, x)
                + 4 * c[3] * np.einsum("ijkl,j,k,l->i", K, x, x, x))
    np.testing.assert_allclose(O.gradient(A, mu, c, x), g_tensor, rtol=1e-12, atol=1e-15)
    H_tensor = (2 * c[1] * Sig - 6 * c[2] * np.einsum("ijk,k->ij", S, x)
                + 12 * c[3] * np.einsum("ijkl,k,l->ij", K, x, x))
    v = rng.standard_normal(x.size)
    u = rng.standard_normal(x.size)
    np.testing.assert_allclose(O.hvp(A, c, x, v), H_tensor @ v, rtol=1e-11, atol=1e-16)
    np.testing.assert_allclose(O.gram(A, c, x), H_tensor, rtol=1e-11, atol=1e-16)
    T_tensor = -6 * c[2] * np.einsum("ijk,j,k->i", S, u, v) + 24 * c[3] * np.einsum("ijkl,j,k,l->i", K, u, v, x)
    np.testing.assert_allclose(O.third(A, c, x, u, v), T_tensor, rtol=1e-11, atol=1e-16)


def test_finite_differences_exact_for_polynomials():
    """f is quartic, grad f cubic, Hv quadratic: the stencils below are exact."""
    mu, A, c, x, rng = small_problem(n=6, T=50, seed=4)
    v = rng.standard_normal(6)
    u = rng.standard_normal(6)
    h = 0.5
    f = lambda y: O.objective(A, mu, c, y)
    five = (f(x - 2 * h * v) - 8 * f(x - h * v) + 8 * f(x + h * v) - f(x + 2 * h * v)) / (12 * h)
    assert five == pytest.approx(O.gradient(A, mu, c, x) @ v, rel=1e-9)
    g = lambda y: O.gradient(A, mu, c, y)
    five_g = (g(x - 2 * h * v) - 8 * g(x - h * v) + 8 * g(x + h * v) - g(x + 2 * h * v)) / (12 * h)
    np.testing.assert_allclose(five_g, O.hvp(A, c, x, v), rtol=1e-8, atol=1e-14)
    Hv = lambda y: O.hvp(A, c, y, v)
    three = (Hv(x + h * u) - Hv(x - h * u)) / (2 * h)
    np.testing.assert_allclose(three, O.third(A, c, x, u, v), rtol=1e-8, atol=1e-14)


def test_symmetries():
    mu, A, c, x, rng = small_problem(n=6, T=60, seed=5)
    G = O.gram(A, c, x)
    assert np.max(np.abs(G - G.T)) <= 1e-16 * np.max(np.abs(G)) * 10
    u, v, w = rng.standard_normal((3, 6))
    t_uv = O.third(A, c, x, u, v)
    np.testing.assert_allclose(t_uv, O.third(A, c, x, v, u), rtol=1e-14, atol=1e-18)
    a = w @ t_uv
    assert a == pytest.approx(u @ O.third(A, c, x, w, v), rel=1e-12)
    assert a == pytest.approx(v @ O.third(A, c, x, u, w), rel=1e-12)


def test_crra_identity_and_certificate():
    for gamma in (0.5, 1.0, 3.0, 6.0, 10.0):
        c = O.crra_coefficients(gamma)
        lhs = 8 * c[1] * c[3] - 3 * c[2] ** 2
        rhs = gamma**2 * (gamma + 1) * (gamma + 3) / 12
        assert lhs == pytest.approx(rhs, rel=1e-13)
        assert O.convexity_certificate(c)
    assert np.allclose(O.crra_coefficients(6.0), [1, 3, 7, 14])
    assert not O.convexity_certificate([1, 1, 2, 0.5])
    # certificate => psi'' >= 2 c2 - 3 c3^2 / (4 c4) > 0 on a dense grid
    c = np.array([1.0, 1.0, 0.5, 2.0])
    s = np.linspace(-5, 5, 100001)
    assert np.min(O.d2psi(c, s)) >= 2 * c[1] - 3 * c[2] ** 2 / (4 * c[3]) - 1e-12


def test_standardised_scaling_keeps_certificate_ratio():
    R = panels.sector_factor_panel(30, 400, 1)
    _, A = O.centre(R)
    lam = np.array([1.0, 1.0, 0.5, 2.0])
    c = O.scale_preferences(lam, A, "standardised")
    assert c[1] * c[3] / c[2] ** 2 == pytest.approx(lam[1] * lam[3] / lam[2] ** 2, rel=1e-13)
    z = A @ np.full(30, 1 / 30)
    s = math.sqrt(z @ z / 400)
    assert c[1] * s**2 == pytest.approx(1.0, rel=1e-13)


# ------------------------------------------------- Prop. quartic exact line search


def test_quartic_coefficients_vandermonde_and_A0():
    mu, A, c, x, rng = small_problem(n=6, T=80, seed=6)
    d = rng.standard_normal(6)
    d -= d.mean()
    coef = O.quartic_coefficients(c, mu, x, d, O.power_sums(A @ x, A @ d))
    assert coef[0] == pytest.approx(O.objective(A, mu, c, x), rel=1e-13)
    al = np.array([-0.4, -0.1, 0.2, 0.5, 0.9])
    V = np.vander(al, 5, increasing=True)
    vals = np.array([O.objective(A, mu, c, x + a * d) for a in al])
    np.testing.assert_allclose(np.linalg.solve(V, vals), coef, rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_quartic_argmin_against_dense_grid(seed):
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal(5)
    coef[4] = abs(coef[4]) if seed % 2 == 0 else coef[4]
    amax = float(rng.uniform(0.5, 3.0))
    a_star = O.quartic_argmin(coef, amax)
    grid = np.linspace(0.0, amax, 2_000_001)
    dec = grid * (coef[1] + grid * (coef[2] + grid * (coef[3] + grid * coef[4])))
    best = float(np.min(dec))
    got = a_star * (coef[1] + a_star * (coef[2] + a_star * (coef[3] + a_star * coef[4])))
    assert got <= best + 1e-12
    assert 0.0 <= a_star <= amax


def test_quartic_argmin_degenerate_degrees():
    # linear: decreasing -> endpoint
    assert O.quartic_argmin([0, -1.0, 0, 0, 0], 2.0) == 2.0
    # quadratic minimum at 0.25
    assert O.quartic_argmin([0, -1.0, 2.0, 0, 0], 2.0) == pytest.approx(0.25, rel=1e-15)
    # cubic with interior minimum at 1: phi' = 3a^2 - 3 -> roots +-1
    assert O.quartic_argmin([0, -3.0, 0.0, 1.0, 0], 5.0) == pytest.approx(1.0, rel=1e-15)
    # increasing function: stay at 0
    assert O.quartic_argmin([0, 1.0, 1.0, 0, 0], 1.0) == 0.0
    # empty interval
    assert O.quartic_argmin([0, -1.0, 0, 0, 0], 0.0) == 0.0


def test_alpha_max_feasibility_lemma():
    rng = np.random.default_rng(7)
    tau = 1e-8
    for _ in range(20):
        n = 12
        x = O.project_slice(rng.dirichlet(np.ones(n)), tau)
        d = rng.standard_normal(n)
        d -= d.mean()
        am = O.alpha_max(x, d, tau)
        assert math.isfinite(am) and am >= 0
        for a in np.linspace(0, am, 11):
            y = x + a * d
            assert abs(y.sum() - 1.0) <= 1e-14
            assert y.min() >= tau - 1e-16
        # and it is the largest such step: any longer one leaves Delta(tau)
        # (the coordinate that attains the minimum crosses tau)
        y = x + (1.0 + 1e-9) * am * d
        assert y.min() < tau


def test_alpha_max_is_tight_and_infinite_without_decrease():
    """alpha_max is the largest feasible step, not just a feasible one: on
    drawn cases (interior points, points with coordinates at tau, directions
    with a single negative coordinate) a step 1e-9 longer leaves Delta(tau),
    brute-force over the coordinates gives the same value, and a direction with
    no negative coordinate has alpha_max = +inf."""
    rng = np.random.default_rng(17)
    tau = 1e-8
    for k in range(200):
        n = int(rng.integers(2, 40))
        x = O.project_slice(rng.dirichlet(np.ones(n) * rng.uniform(0.1, 3)), tau)
        if k % 3 == 1:
            x[rng.integers(0, n, size=max(1, n // 4))] = tau
            x = O.project_slice(x, tau)
        d = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 1)
        if k % 5 == 2:
            d = np.abs(d)
            d[int(rng.integers(0, n))] = -float(np.sum(d))
        d -= d.mean()
        am = O.alpha_max(x, d, tau)
        brute = min(((x[i] - tau) / -d[i] for i in range(n) if d[i] < 0), default=math.inf)
        assert am == brute
        if math.isfinite(am):
            longer = (1.0 + 1e-9) * am if am > 0 else 1e-12   # am = 0: a coordinate at tau with d_i < 0
            assert np.min(x + longer * d) < tau
            if am > 0:
                assert np.min(x + am * d) >= tau - 4 * np.finfo(float).eps
    d = np.zeros(5)
    assert O.alpha_max(np.full(5, 0.2), d, tau) == math.inf


# ---------------------------------------------------- projection and KKT residual


def _project_bisection(v, tau):
    """Independent projection: bisection on the threshold theta."""
    n = v.size
    b = 1.0 - n * tau
    lo, hi = float(np.min(v - tau)) - b, float(np.max(v - tau))
    for _ in range(300):
        th = 0.5 * (lo + hi)
        if np.sum(np.maximum(v - tau - th, 0.0)) > b:
            lo = th
        else:
            hi = th
    return tau + np.maximum(v - tau - 0.5 * (lo + hi), 0.0)


def test_projection_against_bisection_and_variational_inequality():
    rng = np.random.default_rng(8)
    tau = 1e-3
    for _ in range(20):
        v = rng.standard_normal(15) * 0.3
        p = O.project_slice(v, tau)
        np.testing.assert_allclose(p, _project_bisection(v, tau), atol=1e-13)
        assert abs(p.sum() - 1) <= 1e-13 and p.min() >= tau
        for _ in range(5):
            y = O.project_slice(rng.dirichlet(np.ones(15)), tau)
            assert (v - p) @ (y - p) <= 1e-13
        np.testing.assert_allclose(O.project_slice(p, tau), p, atol=1e-15)


# ------------------------------------------------------------ frames and bases


def test_householder_frames_orthonormal():
    rng = np.random.default_rng(9)
    for m in (2, 3, 10):
        U = O.tangent_basis(m)
        assert np.allclose(U.T @ U, np.eye(m - 1), atol=1e-14)
        assert np.allclose(U.T @ np.ones(m), 0, atol=1e-14)
        nu = rng.standard_normal(m)
        nu /= np.linalg.norm(nu)
        Q = O.householder_frame(nu)
        assert np.allclose(Q.T @ Q, np.eye(m - 1), atol=1e-14)
        assert np.allclose(Q.T @ nu, 0, atol=1e-14)


# --------------------------------------------------------- affine-normal direction


def _direction_problem(n=3, T=60, seed=11, lam=(0.0, 1.0, 0.6, 1.5)):
    R = panels.single_factor_panel(n, T, seed)
    mu, A = O.centre(R)
    c = O.scale_preferences(lam, A, "standardised")
    x = np.array([0.5, 0.3, 0.2]) if n == 3 else np.full(n, 1.0 / n)
    return mu, A, c, x


def test_direction_is_the_affine_normal_chord_midpoint_limit():
    """The affine normal is tangent to the locus of midpoints of chords parallel
    to the tangent line (classical characterisation for a convex curve).  With
    n = 3 the reduced level set is a plane curve; the chord midpoints at depth h
    converge to the direction Q u - nu of Sec. 3.2 as h -> 0."""
    from scipy.optimize import brentq

    mu, A, c, x = _direction_problem()
    assert O.convexity_certificate(c)
    U = O.tangent_basis(3)
    phi = lambda y: O.objective(A, mu, c, x + U @ y)
    gb = U.T @ O.gradient(A, mu, c, x)
    G = np.linalg.norm(gb)
    nu = gb / G
    q = O.householder_frame(nu)[:, 0]
    f0 = phi(np.zeros(2))
    lmax = float(np.max(np.linalg.eigvalsh(U.T @ O.gram(A, c, x) @ U)))
    scale = G / lmax                  # curvature radius of the level set

    def offset(h):
        base = -h * nu
        fun = lambda s: phi(base + s * q) - f0
        span = 1e-3
        while fun(span) < 0 or fun(-span) < 0:
            span *= 2
        sp = brentq(fun, 0.0, span, xtol=1e-18, rtol=1e-15)
        sm = brentq(fun, -span, 0.0, xtol=1e-18, rtol=1e-15)
        return 0.5 * (sp + sm) / h

    hs = [scale * 1e-3 * 2.0**-k for k in range(4)]
    vals = [offset(h) for h in hs]
    # Richardson extrapolation of the O(h) error
    lim = 2 * vals[-1] - vals[-2]
    z = A @ x
    d, _ = O.direction_direct(A, c, z, O.gradient(A, mu, c, x), np.ones(3, dtype=bool), 0.0, basis=U)
    dy = U.T @ d                      # = Q u - nu in reduced coordinates
    u = dy @ q
    assert dy @ nu == pytest.approx(-1.0, abs=1e-12)
    assert u == pytest.approx(lim, rel=1e-6)
    # the 1/n-weighted correction is what makes it match: the Newton part alone
    # (correction dropped) misses the limit by tens of percent here
    Gr = U.T @ O.gram(A, c, x) @ U
    Q = O.householder_frame(nu)
    u_newton = np.linalg.solve(Q.T @ Gr @ Q, Q.T @ Gr @ nu)[0]
    assert abs(u_newton - lim) > 0.1 * abs(lim)


def test_direction_basis_invariance_and_descent_identity():
    R = panels.single_factor_panel(7, 120, 12)
    mu, A = O.centre(R)
    c = np.array([0.2, 1.0, 0.8, 2.0]) / np.array([1e-2, 1e-4, 1e-6, 1e-8])
    x = np.random.default_rng(1).dirichlet(np.ones(7))
    g = O.gradient(A, mu, c, x)
    z = A @ x
    F = np.ones(7, dtype=bool)
    d1, _ = O.direction_direct(A, c, z, g, F, 0.0)
    Qr, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((6, 6)))
    U2 = O.tangent_basis(7) @ Qr
    d2, _ = O.direction_direct(A, c, z, g, F, 0.0, basis=U2)
    np.testing.assert_allclose(d1, d2, rtol=1e-10, atol=1e-12 * np.max(np.abs(d1)))
    gbar = g - g.mean()
    assert g @ d1 == pytest.approx(-np.linalg.norm(gbar), rel=1e-10)
    assert abs(d1.sum()) <= 1e-12 * np.max(np.abs(d1))


def test_direction_quadratic_case_is_normalised_newton():
    """c3 = c4 = 0: a = 0 and d = -H^-1 nu / (nu^T H^-1 nu) on the tangent space,
    with H the reduced Hessian built from the explicit covariance (Sec. 2)."""
    R = panels.single_factor_panel(6, 90, 13)
    mu, A = O.centre(R)
    c = np.array([0.01, 3.0, 0.0, 0.0])
    x = np.full(6, 1 / 6)
    g = O.gradient(A, mu, c, x)
    d, _ = O.direction_direct(A, c, A @ x, g, np.ones(6, dtype=bool), 0.0)
    U = O.tangent_basis(6)
    Sig = A.T @ A / A.shape[0]
    H = U.T @ (2 * c[1] * Sig) @ U
    gb = U.T @ g
    nu = gb / np.linalg.norm(gb)
    w = np.linalg.solve(H, nu)
    np.testing.assert_allclose(U.T @ d, -w / (nu @ w), rtol=1e-10, atol=1e-14)


def test_pcg_direction_reduces_to_direct_without_trace_noise():
    """With no third-order term (c3 = c4 = 0, a = 0), tight Krylov tolerance and no
    regularisation, the PCG direction equals the direct one."""
    R = panels.sector_factor_panel(12, 200, 14)
    mu, A = O.centre(R)
    c = np.array([0.05, 2.0, 0.0, 0.0]) / np.array([1e-2, 1e-4, 1, 1])
    x = np.full(12, 1 / 12)
    g = O.gradient(A, mu, c, x)
    F = np.ones(12, dtype=bool)
    d1, _ = O.direction_direct(A, c, A @ x, g, F, 0.0)
    opts = O.Options(krylov_tol=1e-14, krylov_maxit=200, probes=3)
    d2, _ = O.direction_pcg(A, c, A @ x, g, F, 0.0, opts, 0)
    np.testing.assert_allclose(d2, d1, rtol=1e-8, atol=1e-10 * np.max(np.abs(d1)))


def test_hutchinson_trace_converges_to_exact_trace():
    """Statistical pin of the PCG reading: with many probes and exact solves, the
    Hutchinson correction direction approaches the exact-trace direction."""
    R = panels.sector_factor_panel(8, 150, 15)
    mu, A = O.centre(R)
    c = np.array([0.0, 1.0, 0.8, 2.0]) / np.array([1, 1e-4, 1e-6, 1e-8])
    x = np.full(8, 1 / 8)
    g = O.gradient(A, mu, c, x)
    F = np.ones(8, dtype=bool)
    d_exact, _ = O.direction_direct(A, c, A @ x, g, F, 0.0)
    d_none, _ = O.direction_pcg(A, c, A @ x, g, F, 0.0,
                                O.Options(krylov_tol=1e-14, krylov_maxit=200, probes=0), 0)
    d_hut, _ = O.direction_pcg(A, c, A @ x, g, F, 0.0,
                               O.Options(krylov_tol=1e-14, krylov_maxit=200, probes=4000), 0)
    err_hut = np.linalg.norm(d_hut - d_exact)
    err_none = np.linalg.norm(d_none - d_exact)
    assert err_none > 0
    assert err_hut < 0.15 * err_none


def test_probe_generator_reference_values_and_distribution():
    ref = json.load(open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")))
    got = [int(O.splitmix64(np.uint64(ref["seed"]), np.uint64(i))) for i in range(5)]
    assert got == [int(s) for s in ref["outputs"]]
    from scipy import stats

    z = O.probe_vector(7, 3, 2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert not np.array_equal(z[:100], O.probe_vector(7, 3, 1, 100))


def test_reduced_hessian_spectra_match_paper_table_statistically():
    """Table ec-hessian-conditioning: same design (U[-0.1,0.4], T=252, raw
    profiles), other seeds; medians within a loose band."""
    table = json.load(open(os.path.join(GOLDEN, "ec_hessian_conditioning.json")))
    profiles = [(10, 1, 10, 1), (1, 10, 1, 10), (10, 10, 10, 10)]
    for row in table["rows"]:
        n = row["n"]
        lmins, lmaxs, kap = [], [], []
        for k, prof in enumerate(profiles):
            R = panels.uniform_panel(n, 252, seed=1000 + 10 * n + k)
            _, A = O.centre(R)
            x = np.full(n, 1.0 / n)
            U = O.tangent_basis(n)
            ev = np.linalg.eigvalsh(U.T @ O.gram(A, np.asarray(prof, float), x) @ U)
            assert ev.min() > 0
            lmins.append(ev.min())
            lmaxs.append(ev.max())
            kap.append(ev.max() / ev.min())
        assert 0.6 * row["lmin"] <= np.median(lmins) <= 1.6 * row["lmin"]
        assert 0.75 * row["lmax"] <= np.median(lmaxs) <= 1.35 * row["lmax"]
        assert 0.5 * row["kappa"] <= np.median(kap) <= 2.0 * row["kappa"]


# --------------------------------------------------------------- Armijo rule
def test_armijo_step_is_the_largest_accepted_halving():
    """Armijo backtracking on the quartic (Table yand-line-search diagnostic):
    brute force over alpha = amax 2^-j with the polynomial evaluated by
    numpy.polyval (not the oracle's nested form)."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        coef = rng.standard_normal(5) * np.array([1.0, 1.0, 3.0, 10.0, 30.0])
        coef[1] = -abs(coef[1])
        amax = float(rng.uniform(1e-3, 2.0))
        a = O.armijo_step(coef, amax)
        phi = lambda t: np.polyval(coef[::-1], t) - coef[0]
        acc = [amax * 0.5 ** j for j in range(60) if phi(amax * 0.5 ** j) <= 1e-4 * amax * 0.5 ** j * coef[1]]
        assert a == (acc[0] if acc else 0.0)
    assert O.armijo_step(np.array([0.0, 1.0, 1.0, 0.0, 1.0]), 1.0) == 0.0   # phi'(0) > 0: no step
    assert O.armijo_step(np.array([0.0, -1.0, 0.0, 0.0, 0.0]), 0.0) == 0.0  # empty interval


def test_armijo_solve_reaches_the_exact_rule_minimiser():
    """Under the certificate the minimiser is unique, so both step rules must end
    at the same point (Table yand-line-search compares their iterations)."""
    R = panels.uniform_panel(12, 252, 3)
    mu, A = O.centre(R)
    c = np.array([1.0, 10.0, 1.0, 10.0])
    x_e, inf_e = O.solve(A, mu, c, "direct", 1e-10)
    x_a, inf_a = O.solve(A, mu, c, "direct", 1e-10, opts=O.Options(line_search="armijo", max_iter=120))
    assert inf_e.status == "converged" and inf_a.status == "converged"
    assert np.max(np.abs(x_a - x_e)) <= 1e-8


@pytest.mark.parametrize("n,T,kappa", [(40, 80, 10.0), (60, 30, 100.0), (30, 200, 1.0)])
def test_crra_conditioning_construction(n, T, kappa):
    """Table crra-conditioning construction: A = Q diag(s) W^T with W = U V and
    A 1/n = 0 gives kappa_+(A U) = kappa and, since z = A x0 = 0 makes
    psi'' constant, kappa_+(H_0) = kappa^2 for the reduced Hessian at 1/n
    (checked by SVD and by eigenvalues of the oracle's Gram)."""
    R = panels.crra_conditioning_panel(n, T, kappa, 1)
    mu, A = O.centre(R)
    x0 = np.full(n, 1.0 / n)
    assert np.max(np.abs(A @ x0)) <= 1e-15
    U = O.tangent_basis(n)
    sv = np.linalg.svd(A @ U, compute_uv=False)
    sv = sv[sv > 1e-10 * sv[0]]
    assert sv[0] / sv[-1] == pytest.approx(kappa, rel=1e-9)
    ev = np.linalg.eigvalsh(U.T @ O.gram(A, np.array(panels.CRRA_GAMMA6), x0) @ U)
    ev = ev[ev > 1e-10 * ev.max()]
    assert ev.max() / ev.min() == pytest.approx(kappa ** 2, rel=1e-8)
