"""Seeded synthetic return panels shared by the oracle side and the CUDA side.

This module only draws raw returns R (T x n, row-major float64) and the
preference/target grids of each workload.  It holds none of the method's
arithmetic: no centring, no moments, no derivatives.  Every draw comes from
numpy's PCG64 bit generator seeded explicitly, so the same call returns the
same bytes on every run of a given numpy version.

The licensed 5-minute A-share panel of the paper's real-data study (Sec. 6)
is not available; the factor / GARCH(1,1) / Student-t panels below stand in
for it with the same n and the 48-bars-per-day layout.  The paper's own
synthetic benchmark (Sec. 5, R ~ U[-0.1, 0.4], T = 252) is `uniform_panel`.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "student_t_unit",
    "garch_t_series",
    "single_factor_panel",
    "sector_factor_panel",
    "garch_sector_panel",
    "uniform_panel",
    "workload",
    "WORKLOADS",
    "PAPER_SYNTHETIC",
    "CRRA_GAMMA6",
    "crra_conditioning_panel",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def student_t_unit(rng: np.random.Generator, nu: float, size) -> np.ndarray:
    """Student-t draws with nu degrees of freedom rescaled to unit variance."""
    return rng.standard_t(nu, size=size) * np.sqrt((nu - 2.0) / nu)


def garch_t_series(rng, T: int, sigma, alpha=0.05, beta=0.9, nu=4.0, burn=1000):
    """GARCH(1,1) series with unit-variance t_nu innovations.

    sigma is the unconditional standard deviation (scalar or per-series array);
    omega = sigma^2 (1 - alpha - beta).  Returns a (T, k) array.
    """
    sigma = np.atleast_1d(np.asarray(sigma, dtype=np.float64))
    k = sigma.shape[0]
    omega = sigma * sigma * (1.0 - alpha - beta)
    eta = student_t_unit(rng, nu, (T + burn, k))
    out = np.empty((T + burn, k))
    h = sigma * sigma
    prev = np.zeros(k)
    for t in range(T + burn):
        h = omega + alpha * prev * prev + beta * h
        prev = np.sqrt(h) * eta[t]
        out[t] = prev
    return out[burn:]


def single_factor_panel(n=20, T=500, seed=0, nu=5.0, sigma_f=1e-2, eps_loc=1e-2, eps_disp=0.3):
    """One-factor Student-t panel: R[t,i] = beta_i f_t + sigma_i eps_{t,i}."""
    rng = _rng(seed)
    beta = rng.uniform(0.5, 1.5, size=n)
    sig = np.exp(rng.normal(np.log(eps_loc), eps_disp, size=n))
    f = sigma_f * student_t_unit(rng, nu, T)
    eps = student_t_unit(rng, nu, (T, n)) * sig
    return np.ascontiguousarray(np.outer(f, beta) + eps)


def sector_factor_panel(n=500, T=5000, seed=1, nu=4.0, n_sectors=5, sigma_m=1e-2,
                        sigma_s=5e-3, eps_loc=2e-3, eps_disp=0.3):
    """Market + sector Student-t panel; asset i belongs to sector i mod n_sectors."""
    rng = _rng(seed)
    beta = rng.uniform(0.5, 1.5, size=n)
    load = rng.uniform(0.0, 1.0, size=n)
    sig = np.exp(rng.normal(np.log(eps_loc), eps_disp, size=n))
    m = sigma_m * student_t_unit(rng, nu, T)
    s = sigma_s * student_t_unit(rng, nu, (T, n_sectors))
    eps = student_t_unit(rng, nu, (T, n)) * sig
    sec = np.arange(n) % n_sectors
    return np.ascontiguousarray(np.outer(m, beta) + s[:, sec] * load + eps)


def garch_sector_panel(n=2000, T=12000, seed=2, n_sectors=10, sigma_m=1e-3, sigma_s=5e-4,
                       eps_loc=1e-3, eps_disp=0.3, alpha=0.05, beta_g=0.9, nu=4.0):
    """Intraday-scale panel: 48 bars/day x 250 days when T = 12000.

    Market, sector and idiosyncratic series are each GARCH(1,1) with t_nu
    innovations; asset i loads on the market (U(0.5,1.5)) and on sector
    i mod n_sectors (U(0,1)).
    """
    rng = _rng(seed)
    beta = rng.uniform(0.5, 1.5, size=n)
    load = rng.uniform(0.0, 1.0, size=n)
    sig = np.exp(rng.normal(np.log(eps_loc), eps_disp, size=n))
    m = garch_t_series(rng, T, sigma_m, alpha, beta_g, nu)[:, 0]
    s = garch_t_series(rng, T, np.full(n_sectors, sigma_s), alpha, beta_g, nu)
    e = garch_t_series(rng, T, sig, alpha, beta_g, nu)
    sec = np.arange(n) % n_sectors
    R = np.outer(m, beta)
    R += s[:, sec] * load
    R += e
    return np.ascontiguousarray(R)


def uniform_panel(n=20, T=252, seed=0, lo=-0.1, hi=0.4):
    """The paper's stylised benchmark panel (Sec. 5): R i.i.d. U[lo, hi]."""
    return np.ascontiguousarray(_rng(seed).uniform(lo, hi, size=(T, n)))


def quantile_targets(R: np.ndarray, qs) -> np.ndarray:
    """Return floors at quantiles q of the per-asset sample means (Sec. 6).

    The per-asset mean is the same column average every user of R computes; it
    is taken here only to place the floors, not as part of the method.
    """
    col = R.sum(axis=0) / R.shape[0]
    return np.quantile(col, np.asarray(qs, dtype=np.float64))


# Named workloads: sizes, panel recipe, preference grid and targets.
WORKLOADS = {
    "c1_direct_n20_T500": dict(panel="single", n=20, T=500, seed=0,
                               lambdas=[(1.0, 1.0, 1.0, 1.0)], qs=None, config="direct"),
    "c2_direct_n500_T5000": dict(panel="sector", n=500, T=5000, seed=1,
                                 lambdas=[(1.0, 1.0, 1.0, 1.0)],
                                 qs=list(np.round(np.arange(0.40, 0.751, 0.05), 2)), config="direct"),
    "c3_pcg_n2000_T12000": dict(panel="garch", n=2000, T=12000, seed=2,
                                lambdas=[(1.0, 1.0, 1.0, 1.0)], qs=None, config="pcg"),
    "c4_batch_n5440_T12000": dict(panel="garch", n=5440, T=12000, seed=3,
                                  lambdas=[(1.0, 1.0, l3, l4) for l3 in (0.5, 2.0) for l4 in (0.5, 2.0)],
                                  qs=list(np.linspace(0.40, 0.85, 16)), config="pcg"),
}


def crra_conditioning_panel(n: int, T: int, kappa: float, seed: int, vol: float = 2e-2, mean_hi: float = 1e-3):
    """Controlled-conditioning panel of the CRRA benchmark (Sec. 5.2, Tables
    crra-conditioning and crra-conditioning-stress): A = Q diag(s) W^T with
    W = U V, U an orthonormal basis of the simplex tangent space (columns
    orthogonal to 1_n), V an (n-1) x r matrix with orthonormal columns, Q a
    T x r matrix with orthonormal columns orthogonal to 1_T, r = min(n-1, T-1),
    and s log-spaced from vol sqrt(T) down to vol sqrt(T) / kappa.  Then
    A 1/n = 0, 1^T A = 0 (A is centred) and the positive singular values of A U
    are s, so kappa_+(A U) = kappa.  R = A + 1 mu^T with mu_i ~ U[0, mean_hi].
    vol and mean_hi are readings (the paper fixes only kappa, n, T)."""
    rng = _rng(seed)
    r = min(n - 1, T - 1)
    # U: orthonormal complement of 1_n (QR of [1, Gaussian])
    M = rng.standard_normal((n, n - 1))
    U = np.linalg.qr(np.column_stack([np.ones(n), M]))[0][:, 1:]
    V = np.linalg.qr(rng.standard_normal((n - 1, r)))[0]
    Qm = np.linalg.qr(np.column_stack([np.ones(T), rng.standard_normal((T, r))]))[0][:, 1:]
    s = vol * math.sqrt(T) * np.logspace(0.0, -math.log10(kappa), r) if r > 1 else np.array([vol * math.sqrt(T)])
    W = U @ V
    A = (Qm * s) @ W.T
    mu = rng.uniform(0.0, mean_hi, n)
    return A + mu[None, :]


# CRRA calibration gamma = 6 of the conditioning benchmark (Sec. 5.2).
CRRA_GAMMA6 = (1.0, 3.0, 7.0, 14.0)

# The paper's synthetic coefficient-stress benchmark (Sec. 5.3, Table
# synthetic-summary): T = 252, R i.i.d. U[-0.1, 0.4], the three raw profiles,
# the direct configuration for n <= 100 and PCG with stall recovery beyond.
# The paper names only some dimensions (4..100 in 54 runs, 120..5000 in 48
# runs); the two grids below have 18 and 16 dimensions (3 profiles each) and
# contain every dimension it names.  One return matrix per dimension, seed n.
PAPER_SYNTHETIC = dict(
    T=252,
    profiles=[(10.0, 1.0, 10.0, 1.0), (1.0, 10.0, 1.0, 10.0), (10.0, 10.0, 10.0, 10.0)],
    small_n=[4, 8, 12, 16, 20, 25, 30, 35, 40, 45, 50, 60, 70, 75, 80, 90, 95, 100],
    large_n=[120, 150, 200, 250, 300, 400, 500, 600, 800, 1000, 1200, 1500, 2000, 2500, 3000, 5000],
)


def workload(name: str, n: int | None = None, T: int | None = None):
    """Build (R, lambdas, targets) for a named workload, optionally resized."""
    w = dict(WORKLOADS[name])
    n = w["n"] if n is None else n
    T = w["T"] if T is None else T
    if w["panel"] == "single":
        R = single_factor_panel(n, T, w["seed"])
    elif w["panel"] == "sector":
        R = sector_factor_panel(n, T, w["seed"])
    else:
        R = garch_sector_panel(n, T, w["seed"])
    lam = np.asarray(w["lambdas"], dtype=np.float64)
    if w["qs"] is None:
        tg = np.full(1, np.nan)
    else:
        tg = quantile_targets(R, w["qs"])
    return R, lam, tg
