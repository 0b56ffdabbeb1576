"""ctypes binding of the surrogate's device kernels (include/egn_mlp.h).

Argument marshalling only: every function takes torch CUDA tensors (for their
device memory) and launches the library's kernels on the given stream.
"""
import ctypes as C
from typing import Optional

from . import egn as E

EPI_BIAS_RELU, EPI_BIAS, EPI_F32, EPI_RELU_GRAD, EPI_BIAS_GELU, EPI_GELU_GRAD = 0, 1, 2, 3, 4, 5

_bound = False


def _lib():
    global _bound
    L = E.lib()
    if not _bound:
        vp, i, ll, f = C.c_void_p, C.c_int, C.c_longlong, C.c_float
        L.egn_mlp_gemm.argtypes = [i, i, i, i, vp, vp, i, vp, vp, vp, vp, vp]
        L.egn_mlp_reduce_splits.argtypes = [vp, i, ll, vp, vp]
        L.egn_mlp_transpose.argtypes = [vp, i, i, i, vp, vp]
        L.egn_mlp_colsum.argtypes = [vp, i, i, vp, vp]
        L.egn_mlp_head.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.egn_mlp_adam.argtypes = [vp, vp, vp, vp, ll, f, f, f, f, i, vp, vp, i, i, vp]
        L.egn_mlp_cast.argtypes = [vp, ll, vp, vp]
        L.egn_mlp_outputs.argtypes = [vp, i, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp]
        for fn in ("egn_mlp_gemm", "egn_mlp_reduce_splits", "egn_mlp_transpose", "egn_mlp_colsum", "egn_mlp_head",
                   "egn_mlp_adam", "egn_mlp_cast", "egn_mlp_outputs"):
            getattr(L, fn).restype = C.c_int
        _bound = True
    return L


def _p(t) -> Optional[int]:
    return None if t is None else C.c_void_p(t.data_ptr())


def _s(stream) -> Optional[int]:
    return C.c_void_p(stream) if stream else None


def gemm(a, b, out, epilogue, bias=None, aux=None, splits=1, err=None, stream=None):
    """out = epilogue(a @ b.T): a BF16 [m][k], b BF16 [n][k]."""
    m, k = a.shape
    n = b.shape[0]
    E._check(_lib().egn_mlp_gemm(m, n, k, splits, _p(a), _p(b), epilogue, _p(bias), _p(aux), _p(out), _p(err),
                                 _s(stream)))


def reduce_splits(part, splits, out, stream=None):
    E._check(_lib().egn_mlp_reduce_splits(_p(part), splits, out.numel(), _p(out), _s(stream)))


def transpose(x, rows_pad, out, stream=None):
    rows, cols = x.shape
    E._check(_lib().egn_mlp_transpose(_p(x), rows, cols, rows_pad, _p(out), _s(stream)))


def colsum(x, out, stream=None):
    rows, cols = x.shape
    E._check(_lib().egn_mlp_colsum(_p(x), rows, cols, _p(out), _s(stream)))


def head(h, w, b, y, target=None, mask=None, loss=None, g=None, dh=None, dw=None, db=None, stream=None):
    rows, hid = h.shape
    E._check(_lib().egn_mlp_head(_p(h), rows, hid, _p(w), _p(b), _p(y), _p(target), _p(mask), _p(loss), _p(g),
                                 _p(dh), _p(dw), _p(db), _s(stream)))


def adam(w, g, m, v, lr, t, w_bf16=None, wt_bf16=None, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    rows, cols = (w.shape if w.dim() == 2 else (1, w.numel()))
    E._check(_lib().egn_mlp_adam(_p(w), _p(g), _p(m), _p(v), w.numel(), lr, beta1, beta2, eps, t, _p(w_bf16),
                                 _p(wt_bf16), rows, cols, _s(stream)))


def cast(x, out, stream=None):
    E._check(_lib().egn_mlp_cast(_p(x), x.numel(), _p(out), _s(stream)))


def outputs(acc, rows, rows_pad, n_out, b, y, target=None, mask=None, loss=None, g=None, db=None, stream=None):
    """Multi-output layer (and loss): y [rows][n_out] = acc [rows][n_pad] + b; with a target
    also the loss, g = dloss/dy (BF16 [rows_pad][n_pad]) and db."""
    n_pad = acc.shape[-1]
    E._check(_lib().egn_mlp_outputs(_p(acc), rows, rows_pad, n_out, n_pad, _p(b), _p(y), _p(target), _p(mask),
                                    _p(loss), _p(g), _p(db), _s(stream)))
