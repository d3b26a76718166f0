"""The learned warm start on the GPU (include/mvsk_mlp.h) against its oracle
(oracle/mlp_oracle.py): panel statistics and request features, the forward
pass and the gradients under the oracle's model of the BF16 storage points
(tolerances: FP32 accumulation in another order, plus isolated one-ulp BF16
rounding flips of intermediates, bound the relative error of each layer's
output and gradient norms by 5e-3), Adam's first step in closed form, and the
warm start itself: fewer YAND iterations to the same minimiser."""
import math

import numpy as np
import pytest

import panels
from oracle import mlp_oracle as M
from oracle import mvsk_oracle as O

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_column_stats_and_features_match_oracle():
    torch = _torch()
    import paper_2604_25378_gb300 as m
    R = panels.sector_factor_panel(200, 1500, 11)
    ctx = m.MVSK(torch.from_numpy(R).cuda(), "bf16")
    mu, sg = ctx.column_stats()
    assert np.allclose(mu.cpu().numpy(), R.mean(axis=0), rtol=1e-12, atol=1e-17)
    assert np.allclose(sg.cpu().numpy(), R.std(axis=0), rtol=1e-10, atol=0)
    lam = np.array([(1, 1, 1, 1), (1, 1, 0.5, 2), (0.5, 1, 2, 0.5)], dtype=float)
    tg = np.array([np.nan, float(np.quantile(R.mean(0), 0.6)), float(np.quantile(R.mean(0), 0.8))])
    X = m.MLP.features(mu, sg, lam, tg, 21).cpu().numpy()
    Xo = M.features(R.mean(axis=0), R.std(axis=0), lam, tg, 21)
    assert X.shape == Xo.shape == (3, m.MLP_D_IN)
    assert np.max(np.abs(X - Xo)) <= 1e-6 * max(1.0, np.max(np.abs(Xo)))


@pytest.mark.parametrize("B", [16, 13])
def test_forward_and_gradients_match_oracle(B):
    torch = _torch()
    import paper_2604_25378_gb300 as m
    net = m.MLP(d_in=128, d_hidden=64, n_hidden=2, d_out=192, max_batch=16, seed=3)
    rng = np.random.default_rng(4)
    params = []
    for l in range(3):
        W, _ = net.params(l)
        b = (rng.standard_normal(W.shape[0]) * 0.05).astype(np.float32)
        net.set_params(l, W, b)
        params.append((W.astype(np.float64), b.astype(np.float64)))
    X = rng.standard_normal((B, 128)).astype(np.float32)
    Yt = rng.standard_normal((B, 192)).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Yt).cuda()
    y = net.forward(Xd).cpu().numpy()
    yo, _, _ = M.forward(params, X.astype(np.float64), rounding=True)
    assert _rel(y, yo) <= 5e-3
    loss = net.train_step(Xd, Yd, 0.0)  # step size 0: the parameters stay
    lo, go = M.loss_and_grads(params, X.astype(np.float64), Yt.astype(np.float64), rounding=True)
    assert math.isclose(loss, lo, rel_tol=1e-4)
    for l in range(3):
        gW, gb = net.params(l, grads=True)
        assert _rel(gW, go[l][0]) <= 5e-3, (l, _rel(gW, go[l][0]))
        assert _rel(gb, go[l][1]) <= 5e-3, (l, _rel(gb, go[l][1]))
        W, b = net.params(l)
        assert np.array_equal(W, params[l][0].astype(np.float32))


def test_adam_first_step_closed_form():
    """A fresh network's first step: W1 = W0 - lr g / (|g| + eps) (FP32)."""
    torch = _torch()
    import paper_2604_25378_gb300 as m
    net = m.MLP(d_in=128, d_hidden=32, n_hidden=1, d_out=40, max_batch=8, seed=5)
    rng = np.random.default_rng(6)
    W0 = [net.params(l) for l in range(2)]
    X = torch.from_numpy(rng.standard_normal((8, 128)).astype(np.float32)).cuda()
    Yt = torch.from_numpy(rng.standard_normal((8, 40)).astype(np.float32)).cuda()
    net.train_step(X, Yt, 1e-3)
    for l in range(2):
        gW, gb = net.params(l, grads=True)
        W1, b1 = net.params(l)
        for p0, g, p1 in ((W0[l][0], gW, W1), (W0[l][1], gb, b1)):
            want = p0.astype(np.float64) - 1e-3 * g / (np.abs(g) + M.ADAM_EPS)
            assert np.max(np.abs(p1 - want)) <= 1e-6 * max(1.0, np.max(np.abs(p0)))


def test_warm_start_cuts_iterations_to_the_same_minimiser():
    """Train on solver outputs of requests on one panel; held-out requests
    solved from the network's projected output take fewer YAND iterations than
    from 1/n, and reach the same minimiser (under the certificate)."""
    torch = _torch()
    import paper_2604_25378_gb300 as m
    n, T = 200, 2000
    R = panels.garch_sector_panel(n, T, 12)
    Rd = torch.from_numpy(R).cuda()
    ctx = m.MVSK(Rd, "bf16")
    mu, sg = ctx.column_stats()
    rng = np.random.default_rng(13)

    def requests(k):
        lam = np.column_stack([np.ones(k), np.ones(k), rng.uniform(0.5, 2.0, k), rng.uniform(0.5, 2.0, k)])
        return lam, np.full(k, np.nan)

    lam_tr, tg_tr = requests(256)
    Wtr, infos = ctx.solve_batch(lam_tr, tg_tr, m.PCG, 1e-10, out=torch.empty((256, n), dtype=torch.float64,
                                                                                device="cuda"))
    assert all(i["status"] == "ok" for i in infos)
    Xtr = m.MLP.features(mu, sg, lam_tr, tg_tr, 31)
    Ytr = (Wtr * n).float().contiguous()
    net = m.MLP(d_in=m.MLP_D_IN, d_hidden=512, n_hidden=4, d_out=n, max_batch=64, seed=7)
    first = None
    for ep in range(150):
        perm = torch.randperm(256, device="cuda")
        for k in range(4):
            idx = perm[k * 64:(k + 1) * 64]
            loss = net.train_step(Xtr[idx].contiguous(), Ytr[idx].contiguous(), 1e-3 if ep < 100 else 3e-4)
            first = loss if first is None else first
    assert loss < 0.1 * first, (first, loss)
    lam_te, tg_te = requests(32)
    Xte = m.MLP.features(mu, sg, lam_te, tg_te, 31)
    W0 = net.warm_start(Xte, n, 1e-8)
    out = torch.empty((32, n), dtype=torch.float64, device="cuda")
    Wc, ic = ctx.solve_batch(lam_te, tg_te, m.PCG, 1e-10, out=out.clone())
    Ww, iw = ctx.solve_batch(lam_te, tg_te, m.PCG, 1e-10, W0=W0, out=out.clone())
    assert all(i["status"] == "ok" for i in ic + iw)
    cold = np.mean([i["iters"] for i in ic])
    warm = np.mean([i["iters"] for i in iw])
    assert warm < cold, (cold, warm)
    A = O.centre(R)[1]
    for b in range(32):
        c = O.scale_preferences(lam_te[b], A, "standardised")
        if O.convexity_certificate(c):
            assert np.max(np.abs((Ww[b] - Wc[b]).cpu().numpy())) <= 1e-7
