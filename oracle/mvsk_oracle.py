"""Plain FP64 CPU oracle of YAND-MVSK (arXiv 2604.25378).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this module.  The CUDA path shares
no code with it and never calls it.

Every function states the passage it follows.  Numbers are numpy float64;
library primitives (matmul, sort, eigh/cholesky) serve as single steps, with
no blocking, fusion or reordering beyond the formula written beside them.

Notation (the paper's): R (T x n) raw returns, mu = R^T 1 / T, A = R - 1 mu^T,
z = A x, psi(s) = c2 s^2 - c3 s^3 + c4 s^4, x in the simplex slice Delta(tau),
reduced coordinates x = x_ref + U y, Householder frame Q, tangent Hessian
H_{T,lambda}, correction vector a, direction d = U (Q u - nu).

Readings taken where the paper is silent (each is listed with its reason in
the design notes of the repository):
  * a(y): exact trace a_k = sum_ij (H^-1)_ij T3phi(Qe_i, Qe_j)_k, which the
    Blaschke affine-normal formula for a graph yields with the paper's 1/n
    coefficient; in the PCG configuration the trace is Hutchinson-estimated
    with K Gaussian probes drawn from a counter-based SplitMix64 stream.
  * lambda = reg * tr(H_QQ) / dim;  reg = 0 (direct, with 1e-4 / 1e-2
    fall-backs when the Cholesky factorisation fails) or 1e-4 (PCG).
  * PCG: zero start, Jacobi preconditioner diag(G) restricted to the face
    tangent space, stop at relative residual krylov_tol or krylov_maxit
    iterations, or on non-positive curvature (return current iterate).
  * KKT residual: ||x - Pi_{Delta(tau)}(x - grad f)||_2, relative to its
    value at x0 = 1/n.
  * Face continuation: the coordinates at tau form the active face, except
    every one whose violation nu_F - g_i (nu_F the mean of g over the
    coordinates above tau) is positive and at least 2 ||gbar_F||_2 (release
    ratio 0.5): those are released together.
  * Stall (PCG): max_iter reached or kkt not reduced by 1% over 10
    iterations; restarts at projected step 0.045 then 0.02 (120 its each).
    The 1% test only triggers restarts: the last phase runs to the
    tolerance or its 120 iterations.
  * Preference scaling RAW (c = lambda) or STANDARDISED (c_p = lambda_p/s^p,
    s = sqrt(m2(1/n))); a return target calibrates c1 >= 0 by a safeguarded
    secant/bisection root-find on mu^T x*(c1) = target.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Sec. 2: data, moments, coefficients
# ---------------------------------------------------------------------------


def centre(R):
    """mu = T^-1 R^T 1 and A = R - 1 mu^T (Sec. 2; Alg. 1 set-up)."""
    R = np.asarray(R, dtype=np.float64)
    T = R.shape[0]
    mu = R.sum(axis=0) / T
    A = R - mu[None, :]
    return mu, A


def psi(c, s):
    """psi(s) = c2 s^2 - c3 s^3 + c4 s^4 (Prop. 2, lifted separability)."""
    return c[1] * s**2 - c[2] * s**3 + c[3] * s**4


def dpsi(c, s):
    """psi'(s) = 2 c2 s - 3 c3 s^2 + 4 c4 s^3 (gradient weights, Eq. operator-grad)."""
    return 2.0 * c[1] * s - 3.0 * c[2] * s**2 + 4.0 * c[3] * s**3


def d2psi(c, s):
    """psi''(s) = 2 c2 - 6 c3 s + 12 c4 s^2 (Prop. 2)."""
    return 2.0 * c[1] - 6.0 * c[2] * s + 12.0 * c[3] * s**2


def d3psi(c, s):
    """psi'''(s) = -6 c3 + 24 c4 s (Eq. operator-third)."""
    return -6.0 * c[2] + 24.0 * c[3] * s


def comoment_tensors(A):
    """Explicit Sigma, S, K of Sec. 2 (only for tiny n: n^4 storage)."""
    T = A.shape[0]
    Sig = A.T @ A / T
    S = np.einsum("ti,tj,tk->ijk", A, A, A) / T
    K = np.einsum("ti,tj,tk,tl->ijkl", A, A, A, A) / T
    return Sig, S, K


def moments_tensor(mu, Sig, S, K, x):
    """(m1, m2, m3, m4) through the comoment tensors (Sec. 2)."""
    m1 = mu @ x
    m2 = x @ Sig @ x
    m3 = np.einsum("ijk,i,j,k->", S, x, x, x)
    m4 = np.einsum("ijkl,i,j,k,l->", K, x, x, x, x)
    return m1, m2, m3, m4


def crra_coefficients(gamma):
    """CRRA calibration (Remark 'Standard CRRA calibration')."""
    g = float(gamma)
    return np.array([1.0, g / 2.0, g * (g + 1.0) / 6.0, g * (g + 1.0) * (g + 2.0) / 24.0])


def convexity_certificate(c):
    """Cor. (coefficient-only convexity): c4 > 0 and 8 c2 c4 > 3 c3^2."""
    return bool(c[3] > 0.0 and 8.0 * c[1] * c[3] > 3.0 * c[2] ** 2)


def scale_preferences(lam, A, mode="raw"):
    """Map preferences lambda to coefficients c (Sec. 6 normalisation).

    raw: c = lambda.  standardised: with s = sqrt(m2(1/n)) of the equal-weight
    portfolio, c_p = lambda_p / s^p for p = 1..4 (raw when s = 0, e.g. T = 1).
    """
    lam = np.asarray(lam, dtype=np.float64)
    if mode == "raw":
        return lam.copy()
    n = A.shape[1]
    z = A @ np.full(n, 1.0 / n)
    s = math.sqrt(float(z @ z) / A.shape[0])
    if not s > 0.0:
        return lam.copy()
    return lam / np.array([s, s**2, s**3, s**4])


# ---------------------------------------------------------------------------
# Prop. 1 (exact operator representation) and Prop. 2
# ---------------------------------------------------------------------------


def objective(A, mu, c, x):
    """Eq. operator-f: f = -c1 mu^T x + c2/T ||z||^2 - c3/T sum z^3 + c4/T sum z^4."""
    T = A.shape[0]
    z = A @ x
    return -c[0] * (mu @ x) + (c[1] * (z @ z) - c[2] * np.sum(z**3) + c[3] * np.sum(z**4)) / T


def gradient(A, mu, c, x):
    """Eq. operator-grad: grad f = -c1 mu + T^-1 A^T psi'(z)."""
    T = A.shape[0]
    z = A @ x
    return -c[0] * mu + A.T @ dpsi(c, z) / T


def hvp(A, c, x, v):
    """Eq. operator-hvp: grad^2 f v = T^-1 A^T (psi''(z) o Av)."""
    T = A.shape[0]
    z = A @ x
    return A.T @ (d2psi(c, z) * (A @ v)) / T


def third(A, c, x, u, v):
    """Eq. operator-third: T3(u, v) = T^-1 A^T (psi'''(z) o Au o Av)."""
    T = A.shape[0]
    z = A @ x
    return A.T @ (d3psi(c, z) * (A @ u) * (A @ v)) / T


def gram(A, c, x):
    """Prop. 2: grad^2 f = T^-1 A^T D(x) A with D = Diag(psi''(z))."""
    T = A.shape[0]
    z = A @ x
    return A.T @ (d2psi(c, z)[:, None] * A) / T


# ---------------------------------------------------------------------------
# Prop. quartic exact line search; Lemma feasibility cap
# ---------------------------------------------------------------------------

POWER_SUM_KEYS = ("s20", "s30", "s40", "s11", "s21", "s31", "s02", "s12", "s22", "s03", "s13", "s04")


def power_sums(z, w):
    """s_rs = T^-1 sum_t z_t^r w_t^s for the pairs used by A0..A4 (Prop. quartic)."""
    T = z.shape[0]
    out = {}
    for key in POWER_SUM_KEYS:
        r, s = int(key[1]), int(key[2])
        out[key] = float(np.sum(z**r * w**s)) / T
    return out


def quartic_coefficients(c, mu, x, d, sums):
    """A0..A4 of phi(alpha) = f(x + alpha d) (Prop. quartic exact line search)."""
    A0 = -c[0] * (mu @ x) + c[1] * sums["s20"] - c[2] * sums["s30"] + c[3] * sums["s40"]
    A1 = -c[0] * (mu @ d) + 2 * c[1] * sums["s11"] - 3 * c[2] * sums["s21"] + 4 * c[3] * sums["s31"]
    A2 = c[1] * sums["s02"] - 3 * c[2] * sums["s12"] + 6 * c[3] * sums["s22"]
    A3 = -c[2] * sums["s03"] + 4 * c[3] * sums["s13"]
    A4 = c[3] * sums["s04"]
    return np.array([A0, A1, A2, A3, A4])


def alpha_max(x, d, tau):
    """alpha_max(x, d; tau) = min_{d_i < 0} (x_i - tau)/(-d_i) (Sec. 3.3, Lemma cap)."""
    neg = d < 0.0
    if not np.any(neg):
        return math.inf
    return float(np.min((x[neg] - tau) / (-d[neg])))


def _quad_roots(a, b, c):
    """Real roots of a t^2 + b t + c, cancellation-free (Numerical Recipes form)."""
    if a == 0.0:
        if b == 0.0:
            return []
        return [-c / b]
    disc = b * b - 4.0 * a * c
    if disc < 0.0:
        return []
    q = -0.5 * (b + math.copysign(math.sqrt(disc), b))
    roots = [q / a]
    if q != 0.0:
        roots.append(c / q)
    else:
        roots.append(0.0)
    return roots


def _decrease(coef, a):
    """phi(a) - phi(0) = a (A1 + a (A2 + a (A3 + a A4))), without forming A0 + ..."""
    return a * (coef[1] + a * (coef[2] + a * (coef[3] + a * coef[4])))


def _dpoly(coef, a):
    return ((4.0 * coef[4] * a + 3.0 * coef[3]) * a + 2.0 * coef[2]) * a + coef[1]


def quartic_argmin(coef, amax):
    """Exact minimiser of the quartic on [0, amax] (Prop. quartic exact line search).

    Candidates are 0, amax and the real roots of phi' in (0, amax).  phi'' is a
    quadratic; its real roots split (0, amax) into intervals on which phi' is
    monotone, and a sign change of phi' on such an interval brackets exactly
    one root, found by bisection to adjacent floating-point numbers.  Ties in
    phi take the smallest alpha.
    """
    if not (amax > 0.0):
        return 0.0
    brk = [0.0]
    for r in sorted(_quad_roots(12.0 * coef[4], 6.0 * coef[3], 2.0 * coef[2])):
        if 0.0 < r < amax:
            brk.append(r)
    brk.append(amax)
    cands = [0.0, amax]
    for lo, hi in zip(brk[:-1], brk[1:]):
        flo, fhi = _dpoly(coef, lo), _dpoly(coef, hi)
        if flo == 0.0:
            cands.append(lo)
            continue
        if fhi == 0.0:
            cands.append(hi)
            continue
        if (flo < 0.0) == (fhi < 0.0):
            continue
        a, b = lo, hi
        for _ in range(200):
            m = 0.5 * (a + b)
            if m <= a or m >= b:
                break
            fm = _dpoly(coef, m)
            if fm == 0.0:
                a = b = m
                break
            if (fm < 0.0) == (flo < 0.0):
                a = m
            else:
                b = m
        cands.append(0.5 * (a + b) if a != b else a)
    best_a, best_v = 0.0, 0.0
    for a in sorted(set(cands)):
        if not (0.0 <= a <= amax):
            continue
        v = _decrease(coef, a)
        if v < best_v:
            best_a, best_v = a, v
    return best_a


ARMIJO_SIGMA = 1e-4
ARMIJO_HALVINGS = 60


def armijo_step(coef, amax):
    """Armijo backtracking on the exact quartic along d (the paper's Armijo
    diagnostic, Table yand-line-search; constants are a
    reading; App. C.1 names Armijo backtracking as the rule of the
    convergence theory): the largest alpha = amax 2^-j, j < 60, with
    phi(alpha) - phi(0) <= sigma alpha phi'(0), sigma = 1e-4, phi'(0) = A1;
    0 when amax <= 0, phi'(0) >= 0 or no halving is accepted."""
    if not (amax > 0.0) or not (coef[1] < 0.0):
        return 0.0
    a = amax
    for _ in range(ARMIJO_HALVINGS):
        if _decrease(coef, a) <= ARMIJO_SIGMA * a * coef[1]:
            return a
        a *= 0.5
    return 0.0


def line_step(coef, amax, rule):
    """Step along a direction on [0, amax]: the exact quartic minimiser
    (rule "exact", Prop. quartic exact line search) or Armijo backtracking."""
    return quartic_argmin(coef, amax) if rule == "exact" else armijo_step(coef, amax)


# ---------------------------------------------------------------------------
# Simplex slice projection and the projected-simplex KKT residual
# ---------------------------------------------------------------------------


def project_slice(v, tau):
    """Euclidean projection onto Delta(tau) = {x : 1^T x = 1, x_i >= tau}.

    Pi(v) = tau + max(v - tau - theta, 0) with theta from the sorted
    threshold rule (Held, Wolfe & Crowder 1974).
    """
    v = np.asarray(v, dtype=np.float64)
    n = v.shape[0]
    b = 1.0 - n * tau
    u = v - tau
    s = np.sort(u)[::-1]
    css = np.cumsum(s)
    k = np.arange(1, n + 1)
    cond = s - (css - b) / k > 0.0
    rho = int(np.nonzero(cond)[0][-1])
    theta = (css[rho] - b) / (rho + 1)
    return tau + np.maximum(u - theta, 0.0)


def kkt_residual(x, g, tau):
    """Projected-simplex KKT residual ||x - Pi_{Delta(tau)}(x - g)||_2 (Sec. 5)."""
    return float(np.linalg.norm(x - project_slice(x - g, tau)))


# ---------------------------------------------------------------------------
# Reduced coordinates (Prop. affine-subspace reduction) and Householder frames
# ---------------------------------------------------------------------------


def householder_complement(v):
    """Orthonormal columns spanning v^perp (v a unit vector of R^m).

    The Householder reflector P = I - 2 w w^T / w^T w with w = v - s e_1
    (s = -sign(v_1)) maps e_1 to a multiple of v; its columns 2..m are
    orthonormal and orthogonal to v.
    """
    v = np.asarray(v, dtype=np.float64)
    m = v.shape[0]
    s = -1.0 if v[0] >= 0.0 else 1.0
    w = v.copy()
    w[0] -= s
    P = np.eye(m) - 2.0 * np.outer(w, w) / (w @ w)
    return P[:, 1:]


def tangent_basis(m):
    """Orthonormal basis U (m x (m-1)) of the tangent space {1^T v = 0} (Sec. 3.2)."""
    return householder_complement(np.full(m, 1.0 / math.sqrt(m)))


def householder_frame(nu):
    """Q_y with Q^T Q = I and Q^T nu = 0 (Sec. 3.2, Householder frame)."""
    return householder_complement(nu)


# ---------------------------------------------------------------------------
# Counter-based normal probes for the Hutchinson trace (PCG configuration)
# ---------------------------------------------------------------------------

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, index):
    """Output number `index` (0-based) of the SplitMix64 stream seeded with `seed`.

    SplitMix64 (Steele, Lea & Flood 2014): state_i = seed + (i+1) gamma, and the
    output is the mix of state_i.  Works elementwise on uint64 arrays.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def probe_vector(seed, iteration, k, n):
    """Standard normal probe zeta_k (length n) for one iteration.

    The probe's own stream seed is output (iteration*256 + k) of the stream
    `seed`; coordinate i uses outputs 2i and 2i+1 as 53-bit uniforms in (0, 1]
    and the cosine branch of the Box-Muller transform.
    """
    ps = splitmix64(np.uint64(seed), np.uint64(iteration) * np.uint64(256) + np.uint64(k))
    i = np.arange(n, dtype=np.uint64)
    u1 = ((splitmix64(ps, np.uint64(2) * i) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = ((splitmix64(ps, np.uint64(2) * i + np.uint64(1)) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# Affine-normal (YAND) direction on a face (Sec. 3.2, Sec. 3.4 formulas)
# ---------------------------------------------------------------------------


@dataclass
class Options:
    """Parameters of Table 'YAND-MVSK parameter settings' plus the readings."""
    tau: float = 1e-8
    eta: float = 0.05
    max_iter: int = 300
    reg: float | None = None          # None: 0 for direct, 1e-4 for pcg
    krylov_tol: float = 1e-3
    krylov_maxit: int = 15
    probes: int = 8
    probe_seed: int = 0x5EED
    restarts: tuple = ((0.045, 120), (0.02, 120))
    pcg_max_iter: int = 40
    stall_window: int = 10
    stall_factor: float = 0.99
    eps_act: float = 1e-15
    release_ratio: float = 0.5
    descent_eps: float = 1e-10
    arc_halvings: int = 40
    max_elapsed: float = math.inf
    line_search: str = "exact"        # "exact" quartic, or "armijo" backtracking on the quartic


def _face_tangent(A, c, z, F):
    """Quantities shared by both configurations on the free set F."""
    T = A.shape[0]
    AF = A[:, F]
    D2 = d2psi(c, z)
    return AF, D2, T


def direction_direct(A, c, z, g, F, reg, basis=None):
    """Exact-trace YAND direction, direct reduced solve (Sec. 3.2, 3.4).

    On the free set F (m = |F| coordinates) with U an orthonormal tangent
    basis: gbar = U^T g_F, nu = gbar/||gbar||, Q the Householder frame,
    H_{T,lambda} = Q^T (U^T G_FF U) Q + lambda I, h = Q^T U^T G_FF U nu,
    a_k = tr(H^-1 Q^T D^3phi[., ., Qe_k] Q) evaluated as
    a = Q^T U^T T^-1 A_F^T (psi'''(z) o r) with r_t = a_t^T M H^-1 M^T a_t,
    u = H^-1 (h - ||gbar||/m a), d_y = Q u - nu, d_F = U d_y.

    Returns (d, info) with d zero off F.
    """
    n = A.shape[1]
    idx = np.nonzero(F)[0]
    m = idx.size
    d = np.zeros(n)
    info = {"lambda": 0.0, "chol_fallbacks": 0}
    if m <= 1:
        return d, info
    U = tangent_basis(m) if basis is None else basis
    gb = U.T @ g[idx]
    G = float(np.linalg.norm(gb))
    if G == 0.0:
        return d, info
    nu = gb / G
    if m == 2:
        d[idx] = U @ (-nu)
        return d, info
    AF, D2, T = _face_tangent(A, c, z, idx)
    GFF = AF.T @ (D2[:, None] * AF) / T
    Hred = U.T @ GFF @ U                        # grad^2 phi (Prop. simplex reduction)
    Q = householder_frame(nu)
    HQQ = Q.T @ Hred @ Q
    h = Q.T @ Hred @ nu
    trace = abs(float(np.trace(HQQ))) / (m - 2)
    regs = [0.0 if reg is None else reg]
    regs += [r for r in (1e-4, 1e-2) if r > regs[0]]
    L = None
    for k, rg in enumerate(regs):
        lam = rg * trace
        H = HQQ + lam * np.eye(m - 2)
        try:
            L = np.linalg.cholesky(H)
            info["lambda"] = lam
            info["chol_fallbacks"] = k
            break
        except np.linalg.LinAlgError:
            continue
    if L is None:
        info["chol_fallbacks"] = len(regs)
        d[idx] = U @ (-nu)
        return d, info
    Hinv = np.linalg.inv(H)
    AM = AF @ (U @ Q)                            # rows a_t^T M
    r = np.sum((AM @ Hinv) * AM, axis=1)         # r_t = a_t^T M H^-1 M^T a_t
    a = Q.T @ (U.T @ (AF.T @ (d3psi(c, z) * r) / T))
    u = np.linalg.solve(H, h - (G / m) * a)
    d[idx] = U @ (Q @ u - nu)
    return d, info


def pcg(apply_H, apply_P, rhs, tol, maxit):
    """Preconditioned CG on one right-hand side (reading of 'pcg reduced solve').

    Zero start; stops when ||r|| <= tol ||rhs||, after maxit iterations, or
    when p^T H p <= 0 (the current iterate is returned).  Returns (sol, its).
    """
    x = np.zeros_like(rhs)
    r = rhs.copy()
    nb = float(np.linalg.norm(rhs))
    if nb == 0.0:
        return x, 0
    zz = apply_P(r)
    p = zz.copy()
    rz = float(r @ zz)
    its = 0
    for _ in range(maxit):
        q = apply_H(p)
        pq = float(p @ q)
        if not (pq > 0.0):
            break
        al = rz / pq
        x = x + al * p
        r = r - al * q
        its += 1
        if float(np.linalg.norm(r)) <= tol * nb:
            break
        zz = apply_P(r)
        rz_new = float(r @ zz)
        p = zz + (rz_new / rz) * p
        rz = rz_new
    return x, its


def direction_pcg(A, c, z, g, F, reg, opts: Options, iteration, basis=None):
    """YAND direction with PCG reduced solves and a Hutchinson trace (Sec. 3.2).

    Same quantities as `direction_direct`, but H_{T,lambda} is applied matrix-
    free through Hessian-vector oracles and inverted by PCG.  The trace in
    a(y) is estimated with K probes: p_k = M^T zeta_k (zeta_k standard normal
    in R^n restricted to F), s_k = H^-1 p_k by PCG,
    r = K^-1 sum_k (A_F M s_k) o (A_F M p_k), a = M^T T^-1 A_F^T (psi''' o r);
    then u = H^-1 h - (||gbar||/m) H^-1 a.
    """
    n = A.shape[1]
    idx = np.nonzero(F)[0]
    m = idx.size
    d = np.zeros(n)
    info = {"lambda": 0.0, "krylov_its": 0, "hvps": 0}
    if m <= 1:
        return d, info
    U = tangent_basis(m) if basis is None else basis
    gb = U.T @ g[idx]
    G = float(np.linalg.norm(gb))
    if G == 0.0:
        return d, info
    nu = gb / G
    if m == 2:
        d[idx] = U @ (-nu)
        return d, info
    AF, D2, T = _face_tangent(A, c, z, idx)
    Q = householder_frame(nu)
    M = U @ Q                                     # m x (m-2), orthonormal basis of V_F
    nu_amb = U @ nu
    Dg = np.sum(D2[:, None] * AF * AF, axis=0) / T   # diag(G_FF), Jacobi
    dabs = np.abs(Dg)
    dabs = np.maximum(dabs, 1e-300 + 1e-12 * float(np.mean(dabs)))

    def Gmul(p):
        return AF.T @ (D2 * (AF @ p)) / T

    ones = np.ones(m)
    trG = float(np.sum(Dg)) - float(ones @ Gmul(ones)) / m - float(nu_amb @ Gmul(nu_amb))
    lam = (0.0 if reg is None else reg) * abs(trG) / (m - 2)
    info["lambda"] = lam

    def apply_H(eta_):
        return M.T @ Gmul(M @ eta_) + lam * eta_

    def apply_P(r_):
        return M.T @ ((M @ r_) / dabs)

    h = M.T @ Gmul(nu_amb)
    uh, its = pcg(apply_H, apply_P, h, opts.krylov_tol, opts.krylov_maxit)
    info["krylov_its"] += its
    a = np.zeros(m - 2)
    if opts.probes > 0:
        r = np.zeros(T)
        for k in range(opts.probes):
            zeta = probe_vector(opts.probe_seed, iteration, k, n)[idx]
            pk = M.T @ zeta
            sk, its = pcg(apply_H, apply_P, pk, opts.krylov_tol, opts.krylov_maxit)
            info["krylov_its"] += its
            r += (AF @ (M @ sk)) * (AF @ (M @ pk))
        r /= opts.probes
        a = M.T @ (AF.T @ (d3psi(c, z) * r) / T)
    ua, its = pcg(apply_H, apply_P, a, opts.krylov_tol, opts.krylov_maxit)
    info["krylov_its"] += its
    u = uh - (G / m) * ua
    d[idx] = M @ u - nu_amb
    return d, info


# ---------------------------------------------------------------------------
# Alg. 1 with the boundary block (App. C.3) and face continuation
# ---------------------------------------------------------------------------


@dataclass
class SolveInfo:
    status: str = "running"
    iters: int = 0
    restarts: int = 0
    f: float = math.nan
    kkt: float = math.nan
    kkt0: float = math.nan
    kkt_rel: float = math.nan
    free_count: int = 0
    krylov_its: int = 0
    branches: dict = field(default_factory=lambda: {"raw": 0, "segment": 0, "capped": 0, "face": 0, "release": 0})
    history: list = field(default_factory=list)
    seconds: float = 0.0


def _ls_step(A, mu, c, x, z, d, amax, rule="exact"):
    w = A @ d
    coef = quartic_coefficients(c, mu, x, d, power_sums(z, w))
    return line_step(coef, amax, rule)


def working_set(x, g, opts: Options, counts=None):
    """Active face of the boundary block (face continuation reading).

    Every coordinate at tau is held at tau, except those whose violation
    nu_F - g_i (nu_F the mean of g over the coordinates above tau) is
    positive and at least ||gbar_F||_2 / release_ratio: they are released
    together.  Returns the boolean mask of held coordinates.
    """
    bound = x - opts.tau <= opts.eps_act
    F = ~bound
    nuF = float(np.mean(g[F]))
    gn = float(np.linalg.norm(g[F] - nuF))
    viol = np.where(bound, nuF - g, -math.inf)
    rel = bound & (viol > 0.0) & (gn <= opts.release_ratio * viol)
    if np.any(rel):
        bound = bound.copy()
        bound[rel] = False
        if counts is not None:
            counts["release"] += int(np.sum(rel))
    return bound


def boundary_step(A, mu, c, x, z, g, d, opts: Options, counts):
    """Quartic step + boundary block of Alg. 1 (App. C.3 projected active-set step).

    The nominal projected step is eta_k = min(eta, alpha_1), alpha_1 the exact
    quartic minimiser along d on [0, eta] (the damped step, never longer than
    the unconstrained line minimiser).  If alpha_max >= eta_k: exact quartic on
    [0, alpha_max] along d.  Otherwise the projected trial
    xbar = Pi(x + eta_k d) and segment dbar = xbar - x, with eta_k halved
    while dbar is not a descent direction and eta_k/2 > alpha_max (at most 40
    halvings); if g^T dbar < -1e-10 ||P g|| ||dbar|| (P the tangent
    projector), exact quartic on alpha in [0, 1] along dbar; else the capped
    raw step when alpha_max > 0; else the face hand-off: the projected-gradient
    segment Pi(x - s g) - x with s = eta ||d|| / ||P g||, exact quartic on
    [0, 1].  Coordinates within eps_act of tau are set to tau exactly.
    With opts.line_search = "armijo" the four steps along d or the segment
    use Armijo backtracking on the same quartic instead (eta_k keeps its exact
    definition: it sets the projected trial, not the step rule).
    """
    tau = opts.tau
    rule = opts.line_search
    amax = alpha_max(x, d, tau)
    coef = quartic_coefficients(c, mu, x, d, power_sums(z, A @ d))
    eta_k = min(opts.eta, quartic_argmin(coef, opts.eta))
    if amax >= eta_k:
        al = line_step(coef, amax, rule)
        x_new = x + al * d
        counts["raw"] += 1
    else:
        # Halve the nominal step along the projection arc until the projected
        # segment is a descent direction (or the arc reaches alpha_max).
        gt = float(np.linalg.norm(g - np.mean(g)))
        for _ in range(opts.arc_halvings + 1):
            xbar = project_slice(x + eta_k * d, tau)
            dbar = xbar - x
            descent = float(g @ dbar) < -opts.descent_eps * gt * float(np.linalg.norm(dbar))
            if descent or 0.5 * eta_k <= amax:
                break
            eta_k *= 0.5
        if descent:
            al = _ls_step(A, mu, c, x, z, dbar, 1.0, rule)
            x_new = xbar.copy() if al == 1.0 else x + al * dbar
            counts["segment"] += 1
        elif amax > 0.0:
            al = line_step(coef, amax, rule)
            x_new = x + al * d
            counts["capped"] += 1
        else:
            # Face hand-off: the projected-gradient segment, scaled to the
            # length of the YAND trial, is a descent direction at any non-KKT x.
            s = opts.eta * float(np.linalg.norm(d)) / max(gt, 1e-300)
            xbar = project_slice(x - s * g, tau)
            dbar = xbar - x
            counts["face"] += 1
            if not float(g @ dbar) < 0.0:
                return x.copy()
            w = A @ dbar
            al = line_step(quartic_coefficients(c, mu, x, dbar, power_sums(z, w)), 1.0, rule)
            x_new = xbar.copy() if al == 1.0 else x + al * dbar
    x_new = x_new.copy()
    x_new[x_new - tau <= opts.eps_act] = tau
    return x_new


def solve(A, mu, c, config="direct", tol=1e-8, w0=None, opts: Options | None = None,
          callback=None):
    """YAND-MVSK, Alg. 1: oracle block, affine-normal block, quartic step, boundary block.

    Returns (x, SolveInfo).  The best iterate (smallest KKT residual) is
    returned when the iteration budget ends first.
    """
    opts = Options() if opts is None else opts
    t0 = time.perf_counter()
    T, n = A.shape
    tau = opts.tau
    reg = opts.reg if opts.reg is not None else (1e-4 if config == "pcg" else 0.0)
    info = SolveInfo()
    if n == 1:                      # Delta(tau) = {1}
        info.status = "converged"
        return _finish(A, mu, c, np.ones(1), info, 0.0, 0.0, opts, t0)
    x0 = np.full(n, 1.0 / n)
    info.kkt0 = kkt_residual(x0, gradient(A, mu, c, x0), tau)
    x = x0.copy() if w0 is None else np.asarray(w0, dtype=np.float64).copy()
    if config == "pcg":
        phases = [(opts.eta, opts.pcg_max_iter)] + list(opts.restarts)
    else:
        phases = [(opts.eta, opts.max_iter)]
    best = (math.inf, x.copy())
    it_global = 0
    for ph, (eta, max_iter) in enumerate(phases):
        if ph > 0:
            info.restarts += 1
        popts = Options(**{**opts.__dict__, "eta": eta})
        hist = []
        for _k in range(max_iter):
            z = A @ x
            g = -c[0] * mu + A.T @ dpsi(c, z) / T
            kkt = kkt_residual(x, g, tau)
            rel = kkt / max(info.kkt0, 1e-300)
            hist.append(rel)
            info.history.append(rel)
            if rel < best[0]:
                best = (rel, x.copy())
            if callback is not None:
                callback(it_global, x, rel)
            if rel <= tol:
                info.status = "converged"
                return _finish(A, mu, c, x, info, kkt, rel, opts, t0)
            if time.perf_counter() - t0 > opts.max_elapsed:
                info.status = "timeout"
                break
            # the stall test ends a phase to restart it; the last phase has no
            # restart after it and runs to the tolerance or its budget
            if (config == "pcg" and ph + 1 < len(phases) and len(hist) > opts.stall_window
                    and hist[-1] > opts.stall_factor * hist[-1 - opts.stall_window]):
                break
            active = working_set(x, g, opts, info.branches)
            F = ~active
            if config == "pcg":
                d, dinfo = direction_pcg(A, c, z, g, F, reg, popts, it_global)
                info.krylov_its += dinfo["krylov_its"]
            else:
                d, _ = direction_direct(A, c, z, g, F, reg)
            x = boundary_step(A, mu, c, x, z, g, d, popts, info.branches)
            it_global += 1
            info.iters = it_global
        if info.status == "timeout":
            break
    x = best[1]
    g = gradient(A, mu, c, x)
    kkt = kkt_residual(x, g, tau)
    if info.status != "timeout":
        info.status = "not_converged"
    return _finish(A, mu, c, x, info, kkt, kkt / max(info.kkt0, 1e-300), opts, t0)


def _finish(A, mu, c, x, info, kkt, rel, opts, t0):
    info.f = float(objective(A, mu, c, x))
    info.kkt = kkt
    info.kkt_rel = rel
    info.free_count = int(np.sum(x - opts.tau > opts.eps_act))
    info.seconds = time.perf_counter() - t0
    return x, info


# ---------------------------------------------------------------------------
# Return-target calibration (Sec. 6: calibrate the mean coefficient)
# ---------------------------------------------------------------------------


def calibrate_target(A, mu, c, target, config="direct", tol=1e-8, opts=None,
                     rel_tol=1e-9, bracket_tol=1e-12, max_evals=40, c1_max=None, callback=None):
    """Find c1 >= 0 with mu^T x*(c1) = target (Illinois regula falsi).

    mu^T x*(c1) is non-decreasing in c1.  If x*(0) already meets the target,
    c1 = 0.  The upper end starts at c[0] (or c2 s^2 / max|mu| with s^2 = m2(1/n)
    when c[0] = 0) and grows x8 until the target is bracketed or c1_max =
    1e6 c2 s^2 / max|mu| is reached (then c1 = c1_max).  Each solve is warm-
    started from the nearest bracket end.  Illinois stops at |gap| <= rel_tol
    max|mu|, at a relative bracket width of bracket_tol, or at an inner solve
    that needs no iteration from its warm start with |gap| within ten gap
    tolerances (the inner tolerance then resolves the mean no finer).  `callback` is handed to every
    inner solve.  Returns (c, x, info, evals).
    """
    c = np.asarray(c, dtype=np.float64).copy()
    scale = float(np.max(np.abs(mu)))
    gap_tol = rel_tol * scale
    n = A.shape[1]
    z = A @ np.full(n, 1.0 / n)
    s2 = float(z @ z) / A.shape[0]
    c1_ref = max(c[1], 1e-300) * s2 / max(scale, 1e-300)   # c1 at which mean and variance trade evenly
    if c1_max is None:
        c1_max = 1e6 * c1_ref

    def run(c1, w0):
        cc = c.copy()
        cc[0] = c1
        x, inf = solve(A, mu, cc, config, tol, w0=w0, opts=opts, callback=callback)
        return x, inf, float(mu @ x) - target

    evals = 0
    x_lo, inf_lo, h_lo = run(0.0, None)
    evals += 1
    if h_lo >= -gap_tol:
        c[0] = 0.0
        return c, x_lo, inf_lo, evals
    c_lo = 0.0
    c_hi = c[0] if c[0] > 0.0 else c1_ref
    x_hi, inf_hi, h_hi = run(c_hi, x_lo)
    evals += 1
    while h_hi < 0.0 and c_hi < c1_max:
        c_lo, x_lo, inf_lo, h_lo = c_hi, x_hi, inf_hi, h_hi
        c_hi = min(8.0 * c_hi, c1_max)
        x_hi, inf_hi, h_hi = run(c_hi, x_lo)
        evals += 1
    if h_hi < 0.0:
        c[0] = c_hi
        return c, x_hi, inf_hi, evals
    if abs(h_hi) <= gap_tol:
        c[0] = c_hi
        return c, x_hi, inf_hi, evals
    # Illinois regula falsi (Dowell & Jarratt 1971): the retained end's h is
    # halved whenever the same end survives twice in a row.
    side = 0
    while evals < max_evals:
        cm = c_hi - h_hi * (c_hi - c_lo) / (h_hi - h_lo)
        if not (c_lo < cm < c_hi):
            cm = 0.5 * (c_lo + c_hi)
        w0 = x_lo if (cm - c_lo) <= (c_hi - cm) else x_hi
        xm, infm, hm = run(cm, w0)
        evals += 1
        # an inner solve that needs no iteration from its warm start cannot
        # resolve mu^T x*(c1) any finer: its point ends the calibration when
        # its gap is within ten gap tolerances
        if (abs(hm) <= gap_tol or (infm.iters == 0 and abs(hm) <= 10.0 * gap_tol)
                or (c_hi - c_lo) <= bracket_tol * c_hi):
            c[0] = cm
            return c, xm, infm, evals
        if hm < 0.0:
            c_lo, x_lo, inf_lo, h_lo = cm, xm, infm, hm
            if side == -1:
                h_hi *= 0.5
            side = -1
        else:
            c_hi, x_hi, inf_hi, h_hi = cm, xm, infm, hm
            if side == 1:
                h_lo *= 0.5
            side = 1
    c[0] = c_hi
    return c, x_hi, inf_hi, evals


# ---------------------------------------------------------------------------
# Independent cross-check solvers (used by the oracle's own tests)
# ---------------------------------------------------------------------------


def projected_gradient(A, mu, c, tau=1e-8, iters=20000, x0=None):
    """Accelerated projected gradient (FISTA with restarts) on Delta(tau).

    A different method from Alg. 1, used only to cross-check the oracle's
    minimiser on small convex instances.  Step 1/L with L an upper bound on
    the Hessian norm over the iterates (backtracking on the quadratic bound).
    """
    n = A.shape[1]
    x = np.full(n, 1.0 / n) if x0 is None else x0.copy()
    y = x.copy()
    t = 1.0
    L = float(np.linalg.norm(gram(A, c, x), 2)) + 1e-300
    fx = objective(A, mu, c, x)
    for _ in range(iters):
        gy = gradient(A, mu, c, y)
        fy = objective(A, mu, c, y)
        while True:
            xn = project_slice(y - gy / L, tau)
            dx = xn - y
            if objective(A, mu, c, xn) <= fy + gy @ dx + 0.5 * L * (dx @ dx) + 1e-18 * abs(fy):
                break
            L *= 2.0
        fn = objective(A, mu, c, xn)
        if fn > fx:
            y = x.copy()
            t = 1.0
            continue
        tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        y = xn + ((t - 1.0) / tn) * (xn - x)
        x, fx, t = xn, fn, tn
    return x


def support_enumeration(A, mu, c, tau=1e-8, newton_its=100):
    """Brute-force minimiser over Delta(tau) for tiny n (n <= 10).

    For every support S, Newton's method on the face {x_i = tau off S,
    1^T x = 1} (dense reduced Hessian from the explicit Gram) finds the face
    stationary point; feasible points that satisfy the simplex KKT sign
    conditions are kept and the one with the smallest objective is returned.
    """
    import itertools

    T, n = A.shape
    best = (math.inf, None)
    for size in range(1, n + 1):
        for S in itertools.combinations(range(n), size):
            S = list(S)
            x = np.full(n, tau)
            x[S] = (1.0 - (n - size) * tau) / size
            if size > 1:
                U = tangent_basis(size)
                ok = True
                for _ in range(newton_its):
                    g = gradient(A, mu, c, x)
                    gr = U.T @ g[S]
                    H = U.T @ gram(A, c, x)[np.ix_(S, S)] @ U
                    try:
                        step = np.linalg.solve(H, -gr)
                    except np.linalg.LinAlgError:
                        ok = False
                        break
                    x[S] = x[S] + U @ step
                    if np.linalg.norm(step) <= 1e-15 * max(1.0, np.linalg.norm(x[S])):
                        break
                if not ok:
                    continue
            if np.any(x < tau - 1e-14):
                continue
            g = gradient(A, mu, c, x)
            lam_ = float(np.mean(g[S]))
            if np.max(np.abs(g[S] - lam_)) > 1e-9 * max(1.0, np.max(np.abs(g))):
                continue
            off = [i for i in range(n) if i not in S]
            if off and np.min(g[off] - lam_) < -1e-9 * max(1.0, np.max(np.abs(g))):
                continue
            f = objective(A, mu, c, x)
            if f < best[0]:
                best = (f, x.copy())
    return best[1]
