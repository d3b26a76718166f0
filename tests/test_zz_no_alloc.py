"""mvsk_eval_noalloc: value and gradient for callers that cannot allocate GPU memory.

Some callers cannot call cudaMalloc (a fixed memory budget, or a steady-state
loop inside a framework that owns the allocator).  This entry point takes the
caller's buffers only and keeps its scratch in a static device array.  The test
calls it through the C ABI twice in a row (different points, so stale scratch
from the first call would show) and compares f and grad f with mvsk_eval and
with the CPU oracle (Eqs. operator-f and operator-grad), and z with A x, within
the FP64 bound the other parity tests use (1e-12 of the sum of |terms| of each
reduction).
"""
import numpy as np
import pytest

import panels
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu


def test_noalloc_matches_eval_twice():
    import torch

    import paper_2604_25378_gb300 as m

    n, T = 300, 3001
    R = panels.sector_factor_panel(n, T, 21)
    lam = np.array([0.7, 900.0, 4.0e4, 2.0e6])          # raw coefficients c = lambda
    ctx = m.MVSK(R, "fp64")
    ctx.set_option("pref_scaling", 0)
    ctx.set_prefs(lam)
    mu, A = O.centre(R)
    ld = 320
    Ap = np.zeros((T, ld))
    Ap[:, :n] = A
    A_d = torch.from_numpy(Ap).cuda()
    mu_d = torch.from_numpy(mu.copy()).cuda()
    z_d = torch.empty(T, dtype=torch.float64, device="cuda")
    g_d = torch.empty(n, dtype=torch.float64, device="cuda")
    f_d = torch.empty(1, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3)
    for call in range(2):
        x = rng.dirichlet(np.ones(n) * (1.0 + call))
        x_d = torch.from_numpy(x).cuda()
        m.eval_noalloc(A_d, mu_d, lam, x_d, z_d, g_d, f_d)
        torch.cuda.synchronize()
        f_ref, g_ref, _ = ctx.eval(x)
        z = A @ x
        scale = np.abs(A).T @ np.abs(O.dpsi(lam, z)) / T + abs(lam[0]) * np.abs(mu)
        np.testing.assert_array_less(np.abs(g_d.cpu().numpy() - g_ref), 1e-12 * scale + 1e-300)
        np.testing.assert_array_less(np.abs(g_d.cpu().numpy() - O.gradient(A, mu, lam, x)), 1e-12 * scale + 1e-300)
        fs = abs(lam[0] * (mu @ x)) + np.sum(np.abs(O.psi(lam, z))) / T
        assert abs(float(f_d.item()) - f_ref) <= 1e-12 * fs
        assert abs(float(f_d.item()) - O.objective(A, mu, lam, x)) <= 1e-12 * fs
        zs = np.abs(A) @ np.abs(x)
        np.testing.assert_array_less(np.abs(z_d.cpu().numpy() - z), 1e-12 * zs + 1e-300)


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch

    import paper_2604_25378_gb300 as m

    A_d = torch.zeros((4, 6400), dtype=torch.float64, device="cuda")
    mu_d = torch.zeros(6200, dtype=torch.float64, device="cuda")
    x_d = torch.zeros(6200, dtype=torch.float64, device="cuda")
    z_d = torch.empty(4, dtype=torch.float64, device="cuda")
    g_d = torch.empty(6200, dtype=torch.float64, device="cuda")
    f_d = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MvskError) as e:
        m.eval_noalloc(A_d, mu_d, [1, 1, 1, 1], x_d, z_d, g_d, f_d)
    assert e.value.status == 1 and "6144" in str(e.value)
