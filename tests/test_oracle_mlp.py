"""Pins of the warm-start oracle (oracle/mlp_oracle.py) against facts other
than itself: central finite differences of the loss, Adam's first step in
closed form, BF16 rounding against a brute-force nearest-neighbour search, and
invariances of the feature sketch."""
import math

import numpy as np

from oracle import mlp_oracle as M
from oracle import mvsk_oracle as O


def _loss(params, X, T):
    y, _, _ = M.forward(params, X)
    return float(np.sum((y - T) ** 2)) / y.size


def test_gradients_match_central_differences():
    dims = [6, 5, 4, 3]
    params = M.init_params(dims, 1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((3, 6))
    T = rng.standard_normal((3, 3))
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    loss, grads = M.loss_and_grads(params, X, T)
    assert abs(loss - _loss(params, X, T)) <= 1e-15 * max(1.0, loss)
    h = 1e-6
    for l in range(len(params)):
        for q in (0, 1):
            p = params[l][q]
            fd = np.zeros_like(p)
            for idx in np.ndindex(p.shape):
                old = p[idx]
                p[idx] = old + h
                lp = _loss(params, X, T)
                p[idx] = old - h
                lm = _loss(params, X, T)
                p[idx] = old
                fd[idx] = (lp - lm) / (2 * h)
            g = grads[l][q]
            assert np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd))), (l, q)


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2: p - lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    W = rng.standard_normal((4, 3))
    b = rng.standard_normal(4)
    gW = rng.standard_normal((4, 3))
    gb = rng.standard_normal(4)
    state = [((np.zeros_like(W), np.zeros_like(W)), (np.zeros_like(b), np.zeros_like(b)))]
    (W1, b1), = M.adam_step([(W, b)], [(gW, gb)], state, 1e-3, 1)
    assert np.allclose(W1, W - 1e-3 * gW / (np.abs(gW) + M.ADAM_EPS), rtol=0, atol=1e-15)
    assert np.allclose(b1, b - 1e-3 * gb / (np.abs(gb) + M.ADAM_EPS), rtol=0, atol=1e-15)


def test_bf16_rounding():
    one = 1.0
    u = 2.0 ** -7  # BF16 spacing at 1
    assert M.bf16(one) == one
    assert M.bf16(one + u / 2) == one                  # tie, even neighbour
    assert M.bf16(one + 3 * u / 2) == one + 2 * u      # tie, even neighbour
    assert M.bf16(one + u / 2 + 2.0 ** -20) == one + u  # above the tie
    assert M.bf16(-(one + 3 * u / 2)) == -(one + 2 * u)
    # brute force: the nearest of the two BF16 neighbours, ties to the even one
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(2000) * np.exp(rng.uniform(-20, 20, 2000))).astype(np.float32)
    bits = x.view(np.uint32)
    lo = (bits & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi_bits = (bits & np.uint32(0xFFFF0000)) + np.uint32(0x10000)
    hi = hi_bits.view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    got = M.bf16(xd)
    for k in range(x.size):
        dl, dh = abs(xd[k] - lo[k]), abs(hi[k] - xd[k])
        if dl < dh:
            want = lo[k]
        elif dh < dl:
            want = hi[k]
        else:
            want = lo[k] if ((int(bits[k]) >> 16) & 1) == 0 else hi[k]
        assert got[k] == want, (x[k], got[k], want)


def test_feature_sketch_invariances():
    rng = np.random.default_rng(5)
    n = 300
    mu = rng.normal(1e-3, 2e-3, n)
    sigma = np.exp(rng.normal(np.log(1e-2), 0.3, n))
    lam = np.array([[1, 1, 0.5, 2], [1, 1, 2, 0.5]], dtype=float)
    tg = np.array([np.nan, 2e-3])
    X = M.features(mu, sigma, lam, tg, 7)
    assert X.shape == (2, M.D_IN)
    assert np.all(X[:, M.D_FEAT:] == 0.0)
    assert np.array_equal(X[:, :4], lam)
    assert X[0, 4] == 0.0 and X[0, 5] == 0.0 and X[1, 5] == 1.0
    assert math.isclose(X[1, 4], (2e-3 - mu.mean()) / mu.std(), rel_tol=1e-12)
    # the sketch depends on the statistics only through their standardised shape
    X2 = M.features(3.0 * mu + 5e-3, 0.5 * sigma + 1e-3, lam, tg, 7)
    assert np.allclose(X2[:, 6:M.D_FEAT], X[:, 6:M.D_FEAT], rtol=0, atol=1e-12)
    # entry r is the projection of the unit-norm standardised statistic on the
    # r-th normal vector of the seed's stream
    um = (mu - mu.mean()) / (mu.std() * math.sqrt(n))
    assert math.isclose(float(np.linalg.norm(um)), 1.0, rel_tol=1e-12)
    p3 = O.probe_vector(7, 0, 3, n)
    assert math.isclose(X[0, 6 + 3], float(p3 @ um), rel_tol=1e-12, abs_tol=1e-15)
    # another seed gives other projections
    assert not np.allclose(M.features(mu, sigma, lam, tg, 8)[:, 6:M.D_FEAT], X[:, 6:M.D_FEAT])


def test_warm_start_lies_on_the_slice():
    dims = [M.D_IN, 16, 16, 40]
    params = M.init_params(dims, 6)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((3, M.D_IN))
    W0 = M.warm_start(params, X, 40, 1e-8)
    assert W0.shape == (3, 40)
    assert np.allclose(W0.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    assert np.all(W0 >= 1e-8 - 1e-18)
