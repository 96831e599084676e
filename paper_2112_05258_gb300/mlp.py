"""Python binding of the warm-start network entry points (include/lbm_mlp.h).

Argument marshalling only: the forward pass, backpropagation, loss and Adam
run in the CUDA kernels of liblbm.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .lbm import LBMError, load

EXPORTS = ["lbm_mlp_create", "lbm_mlp_num_params", "lbm_mlp_set_params", "lbm_mlp_get_params",
           "lbm_mlp_forward", "lbm_mlp_grad", "lbm_mlp_set_data", "lbm_mlp_train", "lbm_mlp_destroy"]

_fp = ctypes.POINTER(ctypes.c_float)
_ready = False


def _lib():
    global _ready
    L = load()
    if not _ready:
        H = ctypes.c_void_p
        L.lbm_mlp_create.argtypes = [ctypes.c_int] * 6 + [ctypes.c_void_p, ctypes.POINTER(H)]
        L.lbm_mlp_create.restype = ctypes.c_int
        L.lbm_mlp_num_params.argtypes = [H]
        L.lbm_mlp_num_params.restype = ctypes.c_int64
        for n in ("lbm_mlp_set_params", "lbm_mlp_get_params"):
            getattr(L, n).argtypes = [H, _fp, ctypes.c_int64]
            getattr(L, n).restype = ctypes.c_int
        L.lbm_mlp_forward.argtypes = [H, _fp, ctypes.c_int, _fp]
        L.lbm_mlp_forward.restype = ctypes.c_int
        L.lbm_mlp_grad.argtypes = [H, _fp, _fp, ctypes.c_int, _fp]
        L.lbm_mlp_grad.restype = ctypes.c_int
        L.lbm_mlp_set_data.argtypes = [H, _fp, _fp, ctypes.c_int]
        L.lbm_mlp_set_data.restype = ctypes.c_int
        L.lbm_mlp_train.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_int, ctypes.c_float, _fp]
        L.lbm_mlp_train.restype = ctypes.c_int
        L.lbm_mlp_destroy.argtypes = [H]
        L.lbm_mlp_destroy.restype = None
        _ready = True
    return L


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class MLP:
    """n_in -> hidden (x n_hidden, SiLU) -> n_out network on the GPU."""

    def __init__(self, n_in: int, hidden: int, n_hidden: int, n_out: int, max_batch: int, device: int = 0):
        L = _lib()
        h = ctypes.c_void_p()
        st = L.lbm_mlp_create(n_in, hidden, n_hidden, n_out, max_batch, device, None, ctypes.byref(h))
        if st != 0:
            raise LBMError(st, "lbm_mlp_create failed (see stderr)")
        self._h = h
        self.n_in, self.n_out = n_in, n_out
        self.n_params = int(L.lbm_mlp_num_params(h))

    def _ck(self, st, what):
        if st != 0:
            raise LBMError(st, what)

    def close(self):
        if getattr(self, "_h", None):
            _lib().lbm_mlp_destroy(self._h)
            self._h = None

    __del__ = close

    def set_params(self, theta):
        t = _f32(theta)
        self._ck(_lib().lbm_mlp_set_params(self._h, t.ctypes.data_as(_fp), t.size), "set_params")

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        self._ck(_lib().lbm_mlp_get_params(self._h, out.ctypes.data_as(_fp), out.size), "get_params")
        return out

    def forward(self, x) -> np.ndarray:
        x = _f32(x)
        y = np.empty((x.shape[0], self.n_out), dtype=np.float32)
        self._ck(_lib().lbm_mlp_forward(self._h, x.ctypes.data_as(_fp), x.shape[0], y.ctypes.data_as(_fp)),
                 "forward")
        return y

    def grad(self, x, dy) -> np.ndarray:
        x, dy = _f32(x), _f32(dy)
        g = np.empty(self.n_params, dtype=np.float32)
        self._ck(_lib().lbm_mlp_grad(self._h, x.ctypes.data_as(_fp), dy.ctypes.data_as(_fp), x.shape[0],
                                     g.ctypes.data_as(_fp)), "grad")
        return g

    def set_data(self, x, t):
        x, t = _f32(x), _f32(t)
        self._ck(_lib().lbm_mlp_set_data(self._h, x.ctypes.data_as(_fp), t.ctypes.data_as(_fp), x.shape[0]),
                 "set_data")

    def train(self, order, batch: int, lr: float) -> np.ndarray:
        order = np.ascontiguousarray(order, dtype=np.int32)
        steps = order.size // batch
        losses = np.empty(steps, dtype=np.float32)
        self._ck(_lib().lbm_mlp_train(self._h, order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), steps, batch,
                                      float(lr), losses.ctypes.data_as(_fp)), "train")
        return losses
