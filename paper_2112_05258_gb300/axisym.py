"""Thin ctypes binding of the axisymmetric lattice (include/lbm_axi.h).

Argument marshalling only: every step runs in the CUDA library.  Inputs are
:class:`workloads.axisym.AxiInstance` objects (node array ``(nr, nx)``,
``tau``, ``boundaries`` with axis 0, ``q_scale``).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from .lbm import PRECISIONS, BoundaryDesc, LBMError, _dp, _p, _u8p, load as _load_lib

EXPORTS = ["lbm_axi_create", "lbm_axi_step", "lbm_axi_sync", "lbm_axi_read_fields",
           "lbm_axi_read_populations", "lbm_axi_init_populations", "lbm_axi_read_0d_state",
           "lbm_axi_read_waveforms", "lbm_axi_last_error", "lbm_axi_destroy"]


class AxiConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nr", ctypes.c_int), ("node", _u8p), ("tau", ctypes.c_double),
                ("q_scale", ctypes.c_int), ("n_bc", ctypes.c_int), ("bc", ctypes.POINTER(BoundaryDesc)),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("wave_capacity", ctypes.c_int)]


_ready = False


def load():
    global _ready
    L = _load_lib()
    if not _ready:
        H = ctypes.c_void_p
        L.lbm_axi_create.argtypes = [ctypes.POINTER(AxiConfig), ctypes.POINTER(H)]
        L.lbm_axi_step.argtypes = [H, ctypes.c_int64]
        L.lbm_axi_sync.argtypes = [H]
        L.lbm_axi_read_fields.argtypes = [H, _dp, _dp, _dp]
        L.lbm_axi_read_populations.argtypes = [H, _dp]
        L.lbm_axi_init_populations.argtypes = [H, _dp]
        L.lbm_axi_read_0d_state.argtypes = [H, ctypes.c_int, _dp]
        L.lbm_axi_read_waveforms.argtypes = [H, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_axi_last_error.argtypes = [H]
        L.lbm_axi_last_error.restype = ctypes.c_char_p
        L.lbm_axi_destroy.argtypes = [H]
        L.lbm_axi_destroy.restype = None
        for name in EXPORTS:
            if name not in ("lbm_axi_last_error", "lbm_axi_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _ready = True
    return L


class AxiLattice:
    """One axisymmetric instance advanced on one GPU (FP32 or FP64)."""

    def __init__(self, inst, precision="f32", device: int = 0, stream: Optional[int] = None,
                 graph_steps: int = 0, wave_capacity: int = 0):
        L = load()
        if isinstance(precision, str):
            precision = PRECISIONS[precision.lower()]
        nr, nx = inst.node.shape
        node = np.ascontiguousarray(inst.node, dtype=np.uint8).reshape(-1)
        keep = [node]
        bcs = (BoundaryDesc * max(1, len(inst.boundaries)))()
        for k, b in enumerate(inst.boundaries):
            par = np.ascontiguousarray(b.params, dtype=np.float64)
            keep.append(par)
            bcs[k].kind, bcs[k].axis, bcs[k].sign = int(b.kind), int(b.axis), int(b.sign)
            bcs[k].n_params, bcs[k].params = par.size, _p(par)
            if b.profile is not None:
                prof = np.ascontiguousarray(b.profile, dtype=np.float64)
                keep.append(prof)
                bcs[k].n_profile, bcs[k].profile = prof.shape[0], _p(prof)
            if b.elastance is not None:
                et = np.ascontiguousarray(b.elastance, dtype=np.float64)
                keep.append(et)
                bcs[k].period, bcs[k].elastance = et.shape[0], _p(et)
        cfg = AxiConfig(nx=nx, nr=nr, node=node.ctypes.data_as(_u8p), tau=float(inst.tau),
                        q_scale=int(getattr(inst, "q_scale", 1)), n_bc=len(inst.boundaries),
                        bc=ctypes.cast(bcs, ctypes.POINTER(BoundaryDesc)), precision=int(precision),
                        stream=ctypes.c_void_p(stream or 0), device=device, graph_steps=graph_steps,
                        wave_capacity=wave_capacity)
        h = ctypes.c_void_p()
        st = L.lbm_axi_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise LBMError(st, "lbm_axi_create failed (see stderr)")
        self._h = h
        self.nx, self.nr = nx, nr
        self.nbc = len(inst.boundaries)

    def _ck(self, st):
        if st != 0:
            raise LBMError(st, load().lbm_axi_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().lbm_axi_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1):
        self._ck(load().lbm_axi_step(self._h, int(n)))

    def sync(self):
        self._ck(load().lbm_axi_sync(self._h))

    def fields(self):
        """P, u_x, u_r as (nr, nx) arrays."""
        out = [np.empty(self.nr * self.nx) for _ in range(3)]
        self._ck(load().lbm_axi_read_fields(self._h, *[_p(a) for a in out]))
        return tuple(a.reshape(self.nr, self.nx) for a in out)

    def populations(self) -> np.ndarray:
        out = np.empty(9 * self.nr * self.nx)
        self._ck(load().lbm_axi_read_populations(self._h, _p(out)))
        return out.reshape(9, self.nr, self.nx)

    def init_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        self._ck(load().lbm_axi_init_populations(self._h, _p(f)))

    def state_0d(self, bc: int) -> np.ndarray:
        out = np.empty(8)
        self._ck(load().lbm_axi_read_0d_state(self._h, bc, _p(out)))
        return out

    def waves(self, max_rows: int = 1 << 30) -> np.ndarray:
        width = 1 + 4 * self.nbc
        rows_cap = min(max_rows, 1 << 20)
        out = np.empty((max(rows_cap, 1), width))
        rows = ctypes.c_int64()
        self._ck(load().lbm_axi_read_waveforms(self._h, _p(out), rows_cap, ctypes.byref(rows)))
        return out[:rows.value]
