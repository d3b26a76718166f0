"""CPU oracle of the learned warm start (test infrastructure, not product code).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import this
module.  The warm start is not a method of the paper: it is the optional
learned initialiser of the batched solver (a 4 x 512 multilayer perceptron
whose output, projected onto Delta(tau), is the x^0 of a YAND-MVSK solve that
then runs to its own tolerance).  The paper's starting point is x^0 = 1/n
(Sec. 5); the solver judges any other start by the same KKT test.

What is written here, in plain NumPy, is:
  * the request features (the preference vector, the target, and a 64-entry
    sketch of the panel's column means and scales through fixed Gaussian
    projections drawn from the SplitMix64 / Box-Muller stream of
    mvsk_oracle.probe_vector);
  * the network: affine layers with ReLU between them, y = z_L, and the
    mean-squared-error loss against n w* (the scaled solver output);
  * its gradients by the chain rule, and Adam (Kingma & Ba 2015);
  * a model of the GPU's storage rounding (activations, weights and the
    back-propagated error stored in BF16 between layers; FP32 accumulation)
    used to compare the GPU's gradients element by element.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss in
FP64, Adam's first step in closed form, the BF16 rounding of known values,
and the feature sketch against its definition written out by loops.
"""
import math

import numpy as np

from . import mvsk_oracle as O

SKETCH = 32          # projections per column statistic (means, scales)
D_FEAT = 4 + 2 + 2 * SKETCH   # lambda (4), target and its flag (2), sketch (64)
D_IN = 128           # the input width of the network (features zero-padded)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


# ---------------------------------------------------------------- features
def features(mu, sigma, lam, target, seed):
    """Feature rows (B x D_IN) of B requests on one panel.

    mu, sigma: the panel's column means and scales (length n).  Each is
    standardised to mean 0 and norm 1 (u = (s - mean s) / (std s sqrt n)), and
    projected on SKETCH fixed normal vectors P_r = probe_vector(seed, 0, r, n)
    (r < SKETCH for mu, SKETCH <= r < 2 SKETCH for sigma).  A request
    contributes lambda (4 values as given), (target - mean mu) / std mu with
    a flag 1 (0 and 0 without a target).  Zero padding to D_IN.
    """
    mu = np.asarray(mu, np.float64)
    sigma = np.asarray(sigma, np.float64)
    n = mu.shape[0]

    def unit(s):
        sd = float(np.std(s))
        return (s - np.mean(s)) / (sd * math.sqrt(n)) if sd > 0.0 else np.zeros_like(s)

    um, us = unit(mu), unit(sigma)
    sk = np.empty(2 * SKETCH)
    for r in range(2 * SKETCH):
        p = O.probe_vector(seed, 0, r, n)
        sk[r] = float(p @ (um if r < SKETCH else us))
    lam = np.atleast_2d(np.asarray(lam, np.float64))
    target = np.atleast_1d(np.asarray(target, np.float64))
    B = lam.shape[0]
    X = np.zeros((B, D_IN))
    m0, s0 = float(np.mean(mu)), float(np.std(mu))
    for b in range(B):
        X[b, 0:4] = lam[b]
        if np.isfinite(target[b]):
            X[b, 4] = (target[b] - m0) / s0 if s0 > 0.0 else 0.0
            X[b, 5] = 1.0
        X[b, 6:6 + 2 * SKETCH] = sk
    return X


# --------------------------------------------------------------- rounding
def bf16(x):
    """Round to BF16 (nearest, ties to even) and return as float64.

    FP32 value first (the GPU rounds FP32 values), then the top 16 bits of
    its pattern after adding 0x7FFF plus the lowest kept bit.  NaN/Inf are
    not expected here.
    """
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------- network
def init_params(dims, seed):
    """He-normal weights W_l (dims[l+1] x dims[l]) and zero biases (a plain
    initialiser for the oracle's own tests; the GPU draws its own)."""
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((dims[l + 1], dims[l])) * math.sqrt(2.0 / dims[l]), np.zeros(dims[l + 1]))
            for l in range(len(dims) - 1)]


def forward(params, X, rounding=False):
    """Activations a_0 = X, z_l = a_{l-1} W_l^T + b_l, a_l = relu(z_l) (l < L),
    y = z_L.  With rounding, the operands of every product (a_{l-1}, W_l) are
    BF16 as on the GPU.  Returns (y, zs, as_) for the backward pass."""
    r = bf16 if rounding else (lambda v: v)
    a = np.asarray(X, np.float64)
    zs, as_ = [], [r(a)]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = as_[-1] @ r(W).T + b
        zs.append(z)
        if l < L - 1:
            as_.append(r(np.maximum(z, 0.0)))
    return z, zs, as_


def loss_and_grads(params, X, Tt, rounding=False):
    """MSE loss (1/(B n)) sum (y - t)^2 and its gradients by the chain rule:
    dz_L = 2 (y - t)/(B n); dW_l = dz_l^T a_{l-1}; db_l = sum_rows dz_l;
    da_{l-1} = dz_l W_l; dz_{l-1} = da_{l-1} o [z_{l-1} > 0].  With rounding,
    dz_l is BF16 where it enters a product, as on the GPU."""
    r = bf16 if rounding else (lambda v: v)
    y, zs, as_ = forward(params, X, rounding)
    B, n = y.shape
    d = y - Tt
    loss = float(np.sum(d * d)) / (B * n)
    dz = 2.0 * d / (B * n)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dzr = r(dz)
        grads[l] = (dzr.T @ as_[l], np.sum(dz, axis=0))
        if l > 0:
            da = dzr @ r(W)
            dz = da * (zs[l - 1] > 0.0)
    return loss, grads


def adam_step(params, grads, state, lr, t):
    """One Adam step (t >= 1): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  state: list of
    ((mW, vW), (mb, vb)) per layer, updated in place; returns new params."""
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for q, (p, g) in enumerate(((W, gW), (b, gb))):
            m, v = state[l][q]
            m[...] = ADAM_B1 * m + (1.0 - ADAM_B1) * g
            v[...] = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
            mh = m / (1.0 - ADAM_B1 ** t)
            vh = v / (1.0 - ADAM_B2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + ADAM_EPS))
        out.append(tuple(new))
    return out


def warm_start(params, X, n, tau):
    """x^0 of each request: Pi_Delta(tau)(y / n) of the network output."""
    y, _, _ = forward(params, X, rounding=True)
    return np.stack([O.project_slice(y[b] / n, tau) for b in range(y.shape[0])])
