"""GPU parity of the batched direction products (the lockstep iteration of
mvsk_solve_batch) against the plain FP64 products, at the full size of the
n = 5440, T = 12000 frontier sweep and at small ragged sizes.

mvsk_batch_hvp runs the same launches as the solver's Krylov steps: A P16
with the psi'' weighting (fused into the GEMM epilogue when the product
needs no split-K, otherwise split-K partials and a weighting pass), then
A^T S split-K; plus the Gram-diagonal block (G nuhat, diag G).
mvsk_batch_third runs the Hutchinson correction (rhat and A^T (psi''' o rhat)).
Both run, as the solver does by default, on the union of the instances'
working faces (A's columns gathered), and on all columns with the option
face_products = 0.
The reference is numpy FP64 on the centred panel: Eq. operator-hvp
T^-1 A^T (psi''(z) o A v), Prop. 2 for diag G, Eq. operator-third for the
correction.  Bound: A, the columns and the weighted rows are rounded to BF16
(2^-9 relative each) with FP32 accumulation, so every element is held to
2e-2 of the same products on |A| and the absolute operands (the scale of the
summation), the BF16 bound of the single-instance oracle tests.
"""
import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu

C4 = (5440, 12000)
LAMS = [(1.0, 1.0, 0.5, 0.5), (1.0, 1.0, 0.5, 2.0), (1.0, 1.0, 2.0, 0.5), (1.0, 1.0, 2.0, 2.0)]


def _panel(n, T):
    if (n, T) == C4:
        return panels.garch_sector_panel(n, T, 3)
    return panels.sector_factor_panel(n, T, n + T)


def _inputs(n, T, B, seed):
    R = _panel(n, T)
    mu, A = O.centre(R)
    rng = np.random.default_rng(seed)
    C = np.array([O.scale_preferences(LAMS[b % 4], A, "standardised") for b in range(B)])
    X = rng.dirichlet(np.ones(n) * 0.5, size=B)
    return R, A, C, X, rng


def _ctx(R):
    import paper_2604_25378_gb300 as m
    return m.MVSK(R, "bf16")


def _faces(n, B, rng, sparse, sizes=(40, 81), pool=400):
    """Working faces (B x n of 0/1): every coordinate free, or faces of 40-80
    coordinates drawn from a shared pool of 400 (the overlapping supports of a
    frontier sweep), so that their union U is a few hundred coordinates."""
    if not sparse:
        return None
    pool = rng.choice(n, size=min(n, pool), replace=False)
    M = np.zeros((B, n))
    for b in range(B):
        M[b, rng.choice(pool, size=min(len(pool), int(rng.integers(*sizes))), replace=False)] = 1.0
    return M


# (n, T, B, nc, fused, sparse faces, face_products): the full sweep shape (64
# instances x 9 PCG columns = 576 columns, the fused-epilogue form) with all
# coordinates free and with sparse faces, on the face-restricted path and on
# the all-column path; small shapes (split-K form), ragged in T, n and the
# column count.
HVP_CASES = [(5440, 12000, 64, 9, 1, True, 1), (5440, 12000, 64, 9, 1, False, 1), (5440, 12000, 64, 9, 1, False, 0),
             (300, 3001, 4, 9, 0, True, 1), (300, 3001, 4, 9, 0, False, 0), (130, 1000, 3, 5, 0, True, 1),
             (1000, 2500, 7, 1, 0, True, 1)]


@pytest.mark.parametrize("n,T,B,nc,fused,sparse,fp", HVP_CASES)
def test_batch_hvp_matches_plain_products(n, T, B, nc, fused, sparse, fp):
    R, A, C, X, rng = _inputs(n, T, B, 11)
    M = _faces(n, B, rng, sparse)
    V = rng.standard_normal((B, nc, n))
    NU = rng.standard_normal((B, n))
    if M is not None:
        V *= M[:, None, :]
        NU *= M
    NU /= np.linalg.norm(NU, axis=1, keepdims=True)
    ctx = _ctx(R)
    ctx.set_option("face_products", fp)
    HV, Gn, Dg, path = ctx.batch_hvp(C, X, NU, V, M)
    assert path[0] == fused, path  # which form of the weighted product ran
    # coordinates the products are defined on: the union of the faces on the
    # face-restricted path, every coordinate otherwise (zero outside)
    Umask = np.ones(n, dtype=bool) if (fp == 0 or M is None) else M.any(axis=0)
    Z = A @ X.T                                   # T x B
    H = np.column_stack([O.d2psi(C[b], Z[:, b]) for b in range(B)])
    Aa = np.abs(A)
    # all columns at once: (A V)_t, weighted by the instance's psi''
    AV = A @ V.reshape(B * nc, n).T               # T x (B nc)
    AVa = Aa @ np.abs(V).reshape(B * nc, n).T
    Hc = np.repeat(H, nc, axis=1)
    ref = (A.T @ (Hc * AV)).T / T
    scale = (Aa.T @ (np.abs(Hc) * AVa)).T / T
    got = HV.reshape(B * nc, n)
    err = np.abs(got[:, Umask] - ref[:, Umask])
    assert np.all(err <= 2e-2 * scale[:, Umask] + 1e-300), float(np.max(err / (scale[:, Umask] + 1e-300)))
    assert np.all(got[:, ~Umask] == 0.0)
    # the Gram-diagonal block: G nuhat and diag G (Prop. 2)
    refg = (A.T @ (H * (A @ NU.T))).T / T
    scg = (Aa.T @ (np.abs(H) * (Aa @ np.abs(NU).T))).T / T
    assert np.all(np.abs(Gn - refg)[:, Umask] <= 2e-2 * scg[:, Umask] + 1e-300)
    refd = ((A * A).T @ H).T / T
    scd = ((A * A).T @ np.abs(H)).T / T
    assert np.all(np.abs(Dg - refd)[:, Umask] <= 2e-2 * scd[:, Umask] + 1e-300)
    assert np.all(Gn[:, ~Umask] == 0.0) and np.all(Dg[:, ~Umask] == 0.0)
    # the same call again gives the same bits (fixed reduction orders)
    HV2, _, _, _ = ctx.batch_hvp(C, X, NU, V, M)
    assert np.array_equal(HV, HV2)


# (n, T, B, K, sparse faces, face_products, face_small): the full sweep (64
# instances x 8 probe pairs) and small shapes; with sparse faces on the
# union products (face_small = 0) and on the small-face block's tensor-core
# kernel in its narrow (faces <= 128) and wide (<= 320) launch shapes.
THIRD_CASES = [(5440, 12000, 64, 8, True, 1, 0), (5440, 12000, 64, 8, False, 0, 0), (300, 3001, 4, 8, True, 1, 0),
               (130, 1000, 3, 3, False, 1, 0), (5440, 12000, 64, 8, True, 1, 1), (5440, 12000, 64, 8, True, 1, 2),
               (300, 3001, 4, 8, True, 1, 1), (700, 2999, 5, 5, True, 1, 2), (130, 1000, 3, 3, True, 1, 1)]


@pytest.mark.parametrize("n,T,B,K,sparse,fp,fs", THIRD_CASES)
def test_batch_third_matches_plain_products(n, T, B, K, sparse, fp, fs):
    R, A, C, X, rng = _inputs(n, T, B, 12)
    # the wide small-face shape on faces of 130-320 coordinates (all three of its M tiles)
    M = _faces(n, B, rng, sparse, (130, 321), 600) if fs == 2 else _faces(n, B, rng, sparse)
    U = rng.standard_normal((B, K, n))
    P = rng.standard_normal((B, K, n))
    if M is not None:
        U *= M[:, None, :]
        P *= M[:, None, :]
    ctx = _ctx(R)
    ctx.set_option("face_products", fp)
    ctx.set_option("face_small", fs)
    at = ctx.batch_third(C, X, U, P, M)
    # the union products give the correction on the union of the faces, the
    # small-face block on each instance's own face
    if fp == 0 or M is None:
        keep = np.ones((B, n), dtype=bool)
    elif fs == 0:
        keep = np.broadcast_to(M.any(axis=0), (B, n))
    else:
        keep = M > 0
    Z = A @ X.T
    Aa = np.abs(A)
    AU = (A @ U.reshape(B * K, n).T).reshape(T, B, K)
    AP = (A @ P.reshape(B * K, n).T).reshape(T, B, K)
    AUa = (Aa @ np.abs(U).reshape(B * K, n).T).reshape(T, B, K)
    APa = (Aa @ np.abs(P).reshape(B * K, n).T).reshape(T, B, K)
    rhat = np.mean(AU * AP, axis=2)               # T x B (Hutchinson pair products)
    rhat_a = np.mean(AUa * APa, axis=2)
    W3 = np.column_stack([O.d3psi(C[b], Z[:, b]) for b in range(B)])
    ref = (A.T @ (W3 * rhat)).T / T
    scale = (Aa.T @ (np.abs(W3) * rhat_a)).T / T
    err = np.abs(at - ref)[keep]
    assert np.all(err <= 2e-2 * scale[keep] + 1e-300), float(np.max(err / (scale[keep] + 1e-300)))
    assert np.all(at[~keep] == 0.0)
