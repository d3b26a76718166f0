"""Emulated-FP64 tensor-core products A V and A^T V against FP64 (C ABI).

The split product is exact for operands that fit 49 bits relative to their
row / vector maximum, so integer-valued panels must match bit for bit (this
also checks that the tensor cores accumulate the digit products exactly).
For general data the error is bounded by the rounding of both operands to 49
bits plus the dropped digit levels:
    |err_m| <= 40 K 2^-49 max_k |A_mk| max_k |v_k|   (bound used: 1e-13 K max max).
"""
import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu


def _ctx(R):
    import paper_2604_25378_gb300 as m
    return m.MVSK(R, "bf16")


def _check_bound(got, A, V, transpose):
    # rows of the left operand: A (forward) or A^T (transpose)
    L = A.T if transpose else A
    ref = V @ L.T
    K = L.shape[1]
    bound = 1e-13 * K * np.abs(L).max(axis=1)[None, :] * np.abs(V).max(axis=1)[:, None]
    err = np.abs(got - ref)
    assert np.all(err <= bound + 1e-300), float((err / (bound + 1e-300)).max())
    # typical error: far below the bound (rounding of 49-bit operands)
    scale = (np.abs(V) @ np.abs(L).T) + 1e-300
    assert np.median(err / scale) < 1e-14


@pytest.mark.parametrize("n,T,nvec", [(20, 500, 3), (300, 3001, 16), (1000, 1537, 17), (70, 64, 64), (3, 40, 1),
                                      (129, 1025, 48)])
@pytest.mark.parametrize("transpose", [False, True])
def test_product_random(n, T, nvec, transpose):
    import torch
    R = panels.sector_factor_panel(n, T, 11) if n >= 5 else panels.single_factor_panel(n, T, 11)
    mu, A = O.centre(R)
    rng = np.random.default_rng(n + T + nvec)
    V = rng.standard_normal((nvec, T if transpose else n)) * np.exp(rng.uniform(-3, 3, (nvec, 1)))
    ctx = _ctx(R)
    got = ctx.product(torch.from_numpy(V).cuda(), transpose=transpose).cpu().numpy()
    _check_bound(got, A, V, transpose)


# (n, half of T, entry bits): K <= 4096 (one integer slot), and T = 10000
# for A^T V (20 chunks of 512: two slots of 16 chunks)
@pytest.mark.parametrize("n,half,bits", [(600, 1100, 20), (300, 5000, 18)])
@pytest.mark.parametrize("transpose", [False, True])
def test_product_integer_panel_is_exact(transpose, n, half, bits):
    """Columns of R with exactly zero mean (rows +R0 and -R0): A = R exactly.
    Entries below 2^bits with 2 bits + log2 K <= 53 keep every FP64 partial
    sum of the reference exact."""
    import torch
    rng = np.random.default_rng(7)
    R0 = rng.integers(-(1 << bits), 1 << bits, size=(half, n)).astype(np.float64)
    # left-operand rows (rows of A, or columns for A^T) of very different
    # magnitude; each row keeps bits + 1 significant bits, so it fits 49 bits
    # relative to its own maximum
    if transpose:
        R0 *= 2.0 ** -rng.integers(0, 12, size=(1, n))
    else:
        R0 *= 2.0 ** -rng.integers(0, 12, size=(half, 1))
    R = np.vstack([R0, -R0])
    mu, A = O.centre(R)
    assert np.all(mu == 0.0) and np.array_equal(A, R)
    T = R.shape[0]
    nvec = 64
    V = rng.integers(-(1 << bits), 1 << bits, size=(nvec, T if transpose else n)).astype(np.float64)
    V *= 2.0 ** -rng.integers(0, 12, size=(nvec, 1))
    ctx = _ctx(R)
    got = ctx.product(torch.from_numpy(V).cuda(), transpose=transpose).cpu().numpy()
    ref = V @ (A if transpose else A.T)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("transpose", [False, True])
def test_product_full_size(transpose):
    """n = 5440 assets, T = 12000 days, 64 vectors (one lockstep batch)."""
    import torch
    R, _, _ = panels.workload("c4_batch_n5440_T12000")
    mu, A = O.centre(R)
    rng = np.random.default_rng(3)
    V = rng.dirichlet(np.ones(A.shape[0] if transpose else A.shape[1]), size=64)
    ctx = _ctx(R)
    got = ctx.product(torch.from_numpy(V).cuda(), transpose=transpose).cpu().numpy()
    _check_bound(got, A, V, transpose)


def test_product_rejects_bad_counts():
    import torch

    import paper_2604_25378_gb300 as m
    R = panels.single_factor_panel(8, 50, 1)
    ctx = _ctx(R)
    for nv in (0, 65):
        with pytest.raises(m.MvskError):
            ctx.product(torch.zeros((nv, 8), dtype=torch.float64, device="cuda"))
