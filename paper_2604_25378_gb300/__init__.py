"""GB300 (sm_103a) YAND-MVSK sample-oracle library: Python binding.

Argument marshalling only.  Every step of the method runs in libmvsk's CUDA
kernels behind the C ABI of include/mvsk.h; this module never computes any
part of the method itself.  Arrays may be numpy float64 (host) or torch
float64 tensors (host or CUDA); outputs follow the input kind of `R` or of
the `out` argument.

If libmvsk.so has not been built, `load()` raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

__all__ = ["load", "MVSK", "MLP", "MvskError", "DIRECT", "PCG", "PREC", "lib_path", "eval_noalloc", "MLP_D_IN"]

MLP_D_IN = 128  # width of the warm-start request features (include/mvsk_mlp.h)

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "lib", "libmvsk.so")

DIRECT, PCG = 0, 1
PREC = {"fp64": 0, "bf16": 1, "fp32": 2}
STATUS = {0: "ok", 1: "einval", 2: "enomem", 3: "ecuda", 4: "not_converged", 5: "timeout", 6: "estate",
          7: "enumeric"}

_lib = None


class MvskError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("hvps", ctypes.c_int32), ("third_calls", ctypes.c_int32), ("krylov_iters", ctypes.c_int32),
                ("free_count", ctypes.c_int32), ("evals", ctypes.c_int32), ("f", ctypes.c_double),
                ("kkt_residual", ctypes.c_double), ("kkt0", ctypes.c_double), ("kkt_rel", ctypes.c_double),
                ("c", ctypes.c_double * 4), ("achieved_mean", ctypes.c_double), ("seconds", ctypes.c_double),
                ("status", ctypes.c_int32), ("batch_iters", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "c"}
        d["c"] = list(self.c)
        d["status"] = STATUS.get(self.status, self.status)
        return d


class ProfEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 56), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGS = {
    "mvsk_create": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.POINTER(_P)]),
    "mvsk_set_stream": (ctypes.c_int, [_P, _P]),
    "mvsk_set_prefs": (ctypes.c_int, [_P, _P, ctypes.c_double]),
    "mvsk_set_option": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_double]),
    "mvsk_solve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _P, _P, _P]),
    "mvsk_solve_batch": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int32, _P, _P, ctypes.c_double, _P, _P, _P]),
    "mvsk_eval": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mvsk_oracle_hvp": (ctypes.c_int, [_P, _P, _P, _P]),
    "mvsk_oracle_third": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mvsk_oracle_gram": (ctypes.c_int, [_P, _P, _P]),
    "mvsk_product": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int64]),
    "mvsk_oracle_ls": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mvsk_batch_hvp": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P, _P, _P, _P, _P]),
    "mvsk_batch_third": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P, _P, _P]),
    "mvsk_oracle_direction": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int32, _P]),
    "mvsk_project_slice": (ctypes.c_int, [_P, _P, ctypes.c_double, _P]),
    "mvsk_quartic_argmin": (ctypes.c_int, [_P, _P, ctypes.c_double, _P]),
    "mvsk_eval_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P,
                                         _P, _P]),
    "mvsk_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "mvsk_profile_only": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "mvsk_profile_stride": (ctypes.c_int, [_P, ctypes.c_int32]),
    "mvsk_profile_read": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "mvsk_column_stats": (ctypes.c_int, [_P, _P, _P]),
    "mvsk_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "mvsk_mlp_destroy": (ctypes.c_int, [_P]),
    "mvsk_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "mvsk_mlp_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_float, _P]),
    "mvsk_mlp_access": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "mvsk_mlp_features": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, ctypes.c_uint64, _P]),
    "mvsk_mlp_warm_start": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, _P]),
    "mvsk_last_error": (ctypes.c_char_p, [_P]),
    "mvsk_destroy": (None, [_P]),
}


def load(path: str | None = None):
    """Load libmvsk.so (raises if it is missing: the library has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or lib_path
    if not os.path.exists(p):
        raise ImportError(f"libmvsk.so not built at {p}; run paper_2604_25378_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """(pointer, keep-alive) of a float64 array: numpy (host) or torch (host/CUDA)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise TypeError("torch tensors must be contiguous float64")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data_as(ctypes.c_void_p), arr


def _like(x, n_or_shape):
    shape = (n_or_shape,) if isinstance(n_or_shape, int) else tuple(n_or_shape)
    if hasattr(x, "data_ptr"):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=x.device)
    return np.empty(shape, dtype=np.float64)


def eval_noalloc(A, mu, c, x, z, g, f, stream=0):
    """f, grad f and z = A x into caller buffers (torch CUDA float64 tensors),
    through mvsk_eval_noalloc: the library allocates no GPU memory for it."""
    lib = load()
    T, ld = A.shape
    n = mu.shape[0]
    cc = np.ascontiguousarray(c, dtype=np.float64)
    st = lib.mvsk_eval_noalloc(_ptr(A)[0], _ptr(mu)[0], T, n, ld, cc.ctypes.data_as(ctypes.c_void_p), _ptr(x)[0],
                               _ptr(z)[0], _ptr(g)[0], _ptr(f)[0], ctypes.c_void_p(stream))
    if st != 0:
        raise MvskError(st, (lib.mvsk_last_error(None) or b"").decode())


class MVSK:
    """One context: a centred copy of the returns on the GPU plus solver state."""

    def __init__(self, R, precision: str = "fp64"):
        self._lib = load()
        T, n = R.shape
        self.T, self.n = int(T), int(n)
        self.precision = precision
        self._ref = R
        p, keep = _ptr(R)
        h = ctypes.c_void_p()
        self._check(self._lib.mvsk_create(p, T, n, n, PREC[precision], ctypes.byref(h)), None)
        self._h = h
        del keep

    def _check(self, st, h=None):
        if st != 0:
            msg = self._lib.mvsk_last_error(h if h is not None else getattr(self, "_h", None))
            raise MvskError(st, (msg or b"").decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mvsk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int):
        self._check(self._lib.mvsk_set_stream(self._h, ctypes.c_void_p(stream_handle)))

    def set_prefs(self, lam, target=math.nan):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self._check(self._lib.mvsk_set_prefs(self._h, lam.ctypes.data_as(ctypes.c_void_p), float(target)))

    def set_option(self, key: str, value: float):
        self._check(self._lib.mvsk_set_option(self._h, key.encode(), float(value)))

    def solve(self, config: int = PCG, tol: float = 1e-8, w0=None, out=None):
        """Returns (w, info dict); raises MvskError on hard failures.  A solve
        that ends on its iteration budget returns with info['status'] set."""
        out = _like(self._ref, self.n) if out is None else out
        po, ko = _ptr(out)
        pw, kw = (None, None) if w0 is None else _ptr(w0)
        info = Info()
        st = self._lib.mvsk_solve(self._h, int(config), float(tol), pw, po, ctypes.byref(info))
        if st not in (0, 4, 5):
            self._check(st)
        return (ko if ko is not out else out), info.as_dict()

    def solve_batch(self, lambdas, targets=None, config: int = PCG, tol: float = 1e-8, W0=None, out=None):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(-1, 4)
        B = lam.shape[0]
        tg = np.full(B, np.nan) if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
        out = _like(self._ref, (B, self.n)) if out is None else out
        po, ko = _ptr(out)
        pw, kw = (None, None) if W0 is None else _ptr(W0)
        infos = (Info * B)()
        st = self._lib.mvsk_solve_batch(self._h, int(config), B, lam.ctypes.data_as(ctypes.c_void_p),
                                        tg.ctypes.data_as(ctypes.c_void_p), float(tol), pw, po, infos)
        if st not in (0, 4, 5):
            self._check(st)
        return (ko if ko is not out else out), [i.as_dict() for i in infos]

    def eval(self, w):
        pw, kw = _ptr(w)
        g = np.empty(self.n)
        f = ctypes.c_double()
        k = ctypes.c_double()
        self._check(self._lib.mvsk_eval(self._h, pw, ctypes.byref(f), g.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(k)))
        return f.value, g, k.value

    def hvp(self, w, v):
        pw, kw = _ptr(w)
        pv, kv = _ptr(v)
        out = np.empty(self.n)
        self._check(self._lib.mvsk_oracle_hvp(self._h, pw, pv, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def third(self, w, u, v):
        pw, kw = _ptr(w)
        pu, ku = _ptr(u)
        pv, kv = _ptr(v)
        out = np.empty(self.n)
        self._check(self._lib.mvsk_oracle_third(self._h, pw, pu, pv, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def gram(self, w):
        pw, kw = _ptr(w)
        out = np.empty((self.n, self.n))
        self._check(self._lib.mvsk_oracle_gram(self._h, pw, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def product(self, V, transpose=False):
        """A V (transpose=False; V: nvec x n CUDA float64 tensor -> nvec x T) or
        A^T V (V: nvec x T -> nvec x n), emulated FP64 on the tensor cores."""
        import torch
        if not (hasattr(V, "is_cuda") and V.is_cuda and V.dtype == torch.float64 and V.dim() == 2
                and V.is_contiguous()):
            raise TypeError("V must be a contiguous 2-D float64 CUDA tensor")
        m = self.n if transpose else self.T
        out = torch.empty((V.shape[0], m), dtype=torch.float64, device=V.device)
        self._check(self._lib.mvsk_product(self._h, 1 if transpose else 0, V.shape[0], ctypes.c_void_p(V.data_ptr()),
                                           V.shape[1], ctypes.c_void_p(out.data_ptr()), m))
        return out

    def batch_hvp(self, C, X, nuhat, V, mask=None):
        """Direction products of a lockstep batch iteration (mvsk_batch_hvp):
        C (B x 4), X (B x n), nuhat (B x n), V (B x nc x n), optional working
        faces mask (B x n of 0/1) -> (HV (B x nc x n), Gnu (B x n), diagG (B x n),
        (fused first product, split count of the second))."""
        C = np.ascontiguousarray(C, dtype=np.float64)
        X = np.ascontiguousarray(X, dtype=np.float64)
        NU = np.ascontiguousarray(nuhat, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        MK = None if mask is None else np.ascontiguousarray(mask, dtype=np.float64)
        B, nc = V.shape[0], V.shape[1]
        HV = np.empty((B, nc, self.n))
        Gn = np.empty((B, self.n))
        Dg = np.empty((B, self.n))
        path = (ctypes.c_int32 * 2)()
        vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        self._check(self._lib.mvsk_batch_hvp(self._h, B, vp(C), vp(X), vp(NU), vp(MK), nc, vp(V), vp(HV), vp(Gn),
                                             vp(Dg), path))
        return HV, Gn, Dg, (int(path[0]), int(path[1]))

    def batch_third(self, C, X, U, P, mask=None):
        """Hutchinson correction of a lockstep batch (mvsk_batch_third): C (B x 4),
        X (B x n), probe pairs U, P (B x K x n), optional working faces mask
        (B x n of 0/1) -> at (B x n)."""
        C = np.ascontiguousarray(C, dtype=np.float64)
        X = np.ascontiguousarray(X, dtype=np.float64)
        U = np.ascontiguousarray(U, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        MK = None if mask is None else np.ascontiguousarray(mask, dtype=np.float64)
        B, K = U.shape[0], U.shape[1]
        at = np.empty((B, self.n))
        vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        self._check(self._lib.mvsk_batch_third(self._h, B, vp(C), vp(X), vp(MK), K, vp(U), vp(P), vp(at)))
        return at

    def line_search(self, w, d):
        pw, kw = _ptr(w)
        pd, kd = _ptr(d)
        coef = np.empty(5)
        am = ctypes.c_double()
        self._check(self._lib.mvsk_oracle_ls(self._h, pw, pd, coef.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.byref(am)))
        return coef, am.value

    def direction(self, w, config: int = PCG, iteration: int = 0):
        pw, kw = _ptr(w)
        out = np.empty(self.n)
        self._check(self._lib.mvsk_oracle_direction(self._h, int(config), pw, int(iteration),
                                                    out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def column_stats(self):
        """(mu, sigma): the panel's column means and population standard deviations."""
        mu = _like(self._ref, self.n)
        sg = _like(self._ref, self.n)
        self._check(self._lib.mvsk_column_stats(self._h, _ptr(mu)[0], _ptr(sg)[0]))
        return mu, sg

    def project_slice(self, v, tau=1e-8):
        pv, kv = _ptr(v)
        out = np.empty(self.n)
        self._check(self._lib.mvsk_project_slice(self._h, pv, float(tau), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def profile_enable(self, on: bool = True):
        self._check(self._lib.mvsk_profile_enable(self._h, 1 if on else 0))

    def profile_only(self, prefix=None):
        """Record only kinds whose label starts with `prefix` (None: all)."""
        self._check(self._lib.mvsk_profile_only(self._h, None if prefix is None else prefix.encode()))

    def profile_stride(self, k: int = 1):
        """Bracket only every k-th launch of the selected kinds (k >= 1)."""
        self._check(self._lib.mvsk_profile_stride(self._h, int(k)))

    def profile_read(self):
        """({kind: {launches, total_ms, bytes_per_launch}}, kernel launches since enabling)."""
        buf = (ProfEntry * 64)()
        cnt = ctypes.c_int32()
        nl = ctypes.c_int64()
        self._check(self._lib.mvsk_profile_read(self._h, buf, 64, ctypes.byref(cnt), ctypes.byref(nl)))
        out = {}
        for e in buf[:cnt.value]:
            out[e.name.decode()] = {"launches": e.launches, "total_ms": e.total_ms,
                                    "bytes_per_launch": e.bytes_per_launch}
        return out, nl.value

    def quartic_argmin(self, coef, amax):
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        a = ctypes.c_double()
        self._check(self._lib.mvsk_quartic_argmin(self._h, coef.ctypes.data_as(ctypes.c_void_p), float(amax),
                                                  ctypes.byref(a)))
        return a.value


def _dptr(t, dtype):
    """Device pointer of a contiguous CUDA torch tensor of the given dtype."""
    if not hasattr(t, "data_ptr") or not t.is_cuda or not t.is_contiguous() or str(t.dtype) != dtype:
        raise TypeError(f"expected a contiguous CUDA tensor of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


class MLP:
    """The learned warm start (include/mvsk_mlp.h): d_in -> n_hidden x d_hidden
    (ReLU) -> d_out, trained by Adam on the mean-squared error.  Data arrays are
    CUDA torch tensors (features and outputs float32, W0 float64)."""

    def __init__(self, d_in=MLP_D_IN, d_hidden=512, n_hidden=4, d_out=8, max_batch=256, seed=1):
        self._lib = load()
        h = _P()
        st = self._lib.mvsk_mlp_create(int(d_in), int(d_hidden), int(n_hidden), int(d_out), int(max_batch),
                                       int(seed), ctypes.byref(h))
        if st != 0:
            raise MvskError(st, (self._lib.mvsk_last_error(None) or b"").decode())
        self._h = h
        self.dims = [int(d_in)] + [int(d_hidden)] * int(n_hidden) + [int(d_out)]

    def _check(self, st):
        if st != 0:
            raise MvskError(st, (self._lib.mvsk_last_error(None) or b"").decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mvsk_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, X):
        import torch
        B = X.shape[0]
        Y = torch.empty((B, self.dims[-1]), dtype=torch.float32, device=X.device)
        self._check(self._lib.mvsk_mlp_forward(self._h, _dptr(X, "torch.float32"), B, _dptr(Y, "torch.float32")))
        return Y

    def train_step(self, X, Yt, lr):
        loss = ctypes.c_double()
        self._check(self._lib.mvsk_mlp_train_step(self._h, _dptr(X, "torch.float32"), _dptr(Yt, "torch.float32"),
                                                  X.shape[0], float(lr), ctypes.byref(loss)))
        return loss.value

    def _access(self, layer, what, W=None, b=None):
        pw = None if W is None else W.ctypes.data_as(ctypes.c_void_p)
        pb = None if b is None else b.ctypes.data_as(ctypes.c_void_p)
        self._check(self._lib.mvsk_mlp_access(self._h, int(layer), int(what), pw, pb))

    def params(self, layer, grads=False):
        """(W, b) of a layer (or its last gradients) as float32 numpy arrays."""
        W = np.empty((self.dims[layer + 1], self.dims[layer]), dtype=np.float32)
        b = np.empty(self.dims[layer + 1], dtype=np.float32)
        self._access(layer, 2 if grads else 0, W, b)
        return W, b

    def set_params(self, layer, W, b):
        self._access(layer, 1, np.ascontiguousarray(W, dtype=np.float32), np.ascontiguousarray(b, dtype=np.float32))

    @staticmethod
    def features(mu, sigma, lambdas, targets, seed):
        """Request features (B x MLP_D_IN float32, CUDA) from the panel statistics
        (CUDA float64) and the requests' lambda (B x 4) and targets (B)."""
        import torch
        lam = torch.as_tensor(np.ascontiguousarray(lambdas, dtype=np.float64).reshape(-1, 4), device=mu.device)
        tg = torch.as_tensor(np.ascontiguousarray(targets, dtype=np.float64).reshape(-1), device=mu.device)
        B = lam.shape[0]
        X = torch.empty((B, MLP_D_IN), dtype=torch.float32, device=mu.device)
        lib = load()
        st = lib.mvsk_mlp_features(_dptr(mu, "torch.float64"), _dptr(sigma, "torch.float64"), mu.shape[0], B,
                                   _dptr(lam, "torch.float64"), _dptr(tg, "torch.float64"), int(seed),
                                   _dptr(X, "torch.float32"))
        if st != 0:
            raise MvskError(st, (lib.mvsk_last_error(None) or b"").decode())
        return X

    def warm_start(self, X, n, tau=1e-8):
        import torch
        W0 = torch.empty((X.shape[0], int(n)), dtype=torch.float64, device=X.device)
        self._check(self._lib.mvsk_mlp_warm_start(self._h, _dptr(X, "torch.float32"), X.shape[0], int(n), float(tau),
                                                  _dptr(W0, "torch.float64")))
        return W0
