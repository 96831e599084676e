"""Python binding of liblbm (argument marshalling only).

Every step of the method runs in the CUDA kernels behind ``include/lbm.h``;
this module converts numpy arrays and instance descriptions into the C
structures, calls the entry points of the same names, and raises on a
non-zero status.  There is no fallback: if ``liblbm.so`` is missing or no
GPU is present, creating a :class:`Lattice` fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "liblbm.so")

F32, F16, BF16, F64 = 0, 1, 2, 3
PRECISIONS = {"f32": F32, "fp32": F32, "f16": F16, "fp16": F16, "bf16": BF16, "f64": F64, "fp64": F64}
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
          -4: "LBM_ERR_UNSTABLE", -5: "LBM_ERR_STATE"}

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class BoundaryDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("axis", ctypes.c_int), ("sign", ctypes.c_int),
                ("n_params", ctypes.c_int), ("params", _dp),
                ("n_profile", ctypes.c_int64), ("profile", _dp),
                ("period", ctypes.c_int), ("elastance", _dp)]


class InstanceDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("node", _u8p), ("tau", ctypes.c_double), ("q_scale", ctypes.c_int),
                ("n_bc", ctypes.c_int), ("bc", ctypes.POINTER(BoundaryDesc)),
                ("n_ib", ctypes.c_int64), ("ib_X0", _dp), ("ib_dA", _dp), ("ib_ks", _dp),
                ("ib_pinned", _u8p), ("ib_alpha", ctypes.c_double), ("ib_beta", ctypes.c_double),
                ("ib_ms", ctypes.c_double), ("ib_n_fil", ctypes.c_int64),
                ("ib_fil_count", ctypes.POINTER(ctypes.c_int64)),
                ("ib_fil_nodes", ctypes.POINTER(ctypes.c_int64)), ("ib_fil_par", _dp)]


class Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("n_instances", ctypes.c_int),
                ("inst", ctypes.POINTER(InstanceDesc)), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("graph_steps", ctypes.c_int),
                ("wave_capacity", ctypes.c_int), ("block_size", ctypes.c_int),
                ("ib_threads_per_node", ctypes.c_int), ("ib_slabs", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("fluid_cells", ctypes.c_int64), ("stored_cells", ctypes.c_int64),
                ("box_cells", ctypes.c_int64), ("band_cells", ctypes.c_int64),
                ("ib_nodes", ctypes.c_int64), ("links", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("precision", ctypes.c_int),
                ("bytes_per_population", ctypes.c_int), ("slabs", ctypes.c_int),
                ("launches_per_step", ctypes.c_int), ("launches_first_step", ctypes.c_int),
                ("graph_steps", ctypes.c_int)]


class LayoutStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "fluid_cells", "stored_cells", "box_cells", "band_cells", "links", "ib_nodes", "filaments", "slabs")]


EXPORTS = ["lbm_create", "lbm_set_0d_params", "lbm_init_populations", "lbm_step", "lbm_sync",
           "lbm_read_fields", "lbm_read_populations", "lbm_read_0d_state", "lbm_read_waveforms",
           "lbm_read_ib", "lbm_set_ib_state", "lbm_set_kernel_timing", "lbm_get_kernel_time",
           "lbm_get_info", "lbm_last_error", "lbm_destroy", "lbm_boundary_flux_noalloc", "lbm_step_io",
           "lbm_init_equilibrium", "lbm_set_0d_state", "lbm_cycle_change", "lbm_autotune",
           "lbm_wall_shear", "lbm_check_config", "lbm_checkpoint_size", "lbm_checkpoint_save",
           "lbm_checkpoint_load", "lbm_read_fields_device", "lbm_set_stream_collide_shape",
           "lbm_read_0d_state_async"]

_lib = None


def load(path: Optional[str] = None):
    """Loads liblbm.so (builds nothing; call ``build()`` first).  The
    environment variable LBM_LIBRARY overrides the in-tree path."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("LBM_LIBRARY") or SO_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"liblbm.so not built at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    L.lbm_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(H)]
    L.lbm_set_0d_params.argtypes = [H, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int]
    L.lbm_init_populations.argtypes = [H, ctypes.c_int, _dp]
    L.lbm_step.argtypes = [H, ctypes.c_int64]
    L.lbm_sync.argtypes = [H]
    L.lbm_read_fields.argtypes = [H, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.lbm_read_populations.argtypes = [H, ctypes.c_int, _dp]
    L.lbm_read_0d_state.argtypes = [H, ctypes.c_int, ctypes.c_int, _dp]
    L.lbm_read_waveforms.argtypes = [H, ctypes.c_int, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.lbm_read_ib.argtypes = [H, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.lbm_set_ib_state.argtypes = [H, ctypes.c_int, _dp, _dp]
    L.lbm_set_kernel_timing.argtypes = [H, ctypes.c_int]
    L.lbm_get_kernel_time.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    L.lbm_get_info.argtypes = [H, ctypes.POINTER(Info)]
    L.lbm_last_error.argtypes = [H]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_destroy.argtypes = [H]
    L.lbm_destroy.restype = None
    L.lbm_init_equilibrium.argtypes = [H, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.lbm_wall_shear.argtypes = [H, ctypes.c_int, _dp]
    L.lbm_checkpoint_size.argtypes = [H, ctypes.POINTER(ctypes.c_int64)]
    L.lbm_set_stream_collide_shape.argtypes = [H, ctypes.c_int, ctypes.c_int]
    L.lbm_read_0d_state_async.argtypes = [H, ctypes.c_int, ctypes.c_void_p]
    L.lbm_step_io.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                              ctypes.c_void_p]
    L.lbm_read_fields_device.argtypes = [H, ctypes.c_int] + [ctypes.c_void_p] * 4
    L.lbm_checkpoint_save.argtypes = [H, ctypes.c_void_p, ctypes.c_int64]
    L.lbm_checkpoint_load.argtypes = [H, ctypes.c_void_p, ctypes.c_int64]
    L.lbm_check_config.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(LayoutStats), ctypes.c_char_p,
                                   ctypes.c_int]
    L.lbm_set_0d_state.argtypes = [H, ctypes.c_int, ctypes.c_int, _dp]
    L.lbm_cycle_change.argtypes = [H, ctypes.POINTER(ctypes.c_int64), _dp]
    L.lbm_autotune.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), _dp]
    L.lbm_boundary_flux_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    for name in EXPORTS:
        if name not in ("lbm_last_error", "lbm_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _config(instances, precision, device=0, stream=None, graph_steps=0, wave_capacity=0, block_size=0,
            ib_threads_per_node=0, ib_slabs=0):
    """lbm_config for the instances and the host arrays it points to (to be
    kept alive while the library copies them)."""
    keep = []
    n = len(instances)
    descs = (InstanceDesc * n)()
    for q, inst in enumerate(instances):
        nz, ny, nx = inst.node.shape
        node = np.ascontiguousarray(inst.node, dtype=np.uint8).reshape(-1)
        keep.append(node)
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
        keep.append(bcs)
        d = descs[q]
        d.nx, d.ny, d.nz = nx, ny, nz
        d.node = node.ctypes.data_as(_u8p)
        d.tau = float(inst.tau)
        d.q_scale = int(getattr(inst, "q_scale", 1))
        d.n_bc = len(inst.boundaries)
        d.bc = ctypes.cast(bcs, ctypes.POINTER(BoundaryDesc))
        ib = getattr(inst, "ib", None)
        if ib is not None and ib.n > 0:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (ib.X0, ib.dA, ib.ks)]
            pin = np.ascontiguousarray(ib.pinned, dtype=np.uint8)
            keep += arrs + [pin]
            d.n_ib = ib.n
            d.ib_X0, d.ib_dA, d.ib_ks = (_p(a) for a in arrs)
            d.ib_pinned = pin.ctypes.data_as(_u8p)
            d.ib_alpha, d.ib_beta, d.ib_ms = float(ib.alpha), float(ib.beta), float(ib.ms)
            fils = getattr(ib, "filaments", None)
            if fils:
                cnt = np.array([len(f) for f in fils], dtype=np.int64)
                nodes = np.ascontiguousarray(np.concatenate(fils), dtype=np.int64)
                fpar = np.ascontiguousarray(ib.fil_par, dtype=np.float64).reshape(-1)
                keep += [cnt, nodes, fpar]
                d.ib_n_fil = cnt.size
                d.ib_fil_count = cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
                d.ib_fil_nodes = nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
                d.ib_fil_par = _p(fpar)
    cfg = Config(precision=int(precision), n_instances=n,
                 inst=ctypes.cast(descs, ctypes.POINTER(InstanceDesc)),
                 stream=ctypes.c_void_p(stream or 0), device=device, graph_steps=graph_steps,
                 wave_capacity=wave_capacity, block_size=block_size,
                 ib_threads_per_node=ib_threads_per_node, ib_slabs=ib_slabs)
    keep.append(descs)
    return cfg, keep


def check_config(instances, precision="f32", ib_threads_per_node: int = 0, ib_slabs: int = 0) -> dict:
    """Host-only validation and layout sizes of a batch (no GPU needed):
    raises LBMError with the reason if lbm_create would reject it."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision.lower()]
    cfg, keep = _config(instances, precision, ib_threads_per_node=ib_threads_per_node, ib_slabs=ib_slabs)
    st = LayoutStats()
    why = ctypes.create_string_buffer(512)
    rc = load().lbm_check_config(ctypes.byref(cfg), ctypes.byref(st), why, len(why))
    if rc != 0:
        raise LBMError(rc, why.value.decode())
    return {n: getattr(st, n) for n, _ in LayoutStats._fields_}


class Lattice:
    """A batch of lattice instances advanced together on one GPU.

    ``instances``: objects with the attributes of :class:`workloads.Instance`
    (``node``, ``tau``, ``boundaries``, ``ib``, ``q_scale``).
    """

    def __init__(self, instances: Sequence, precision="f32", device: int = 0,
                 stream: Optional[int] = None, graph_steps: int = 0, wave_capacity: int = 0,
                 block_size: int = 0, ib_threads_per_node: int = 0, ib_slabs: int = 0):
        L = load()
        if isinstance(precision, str):
            precision = PRECISIONS[precision.lower()]
        cfg, self._keep = _config(instances, precision, device, stream, graph_steps, wave_capacity,
                                  block_size, ib_threads_per_node, ib_slabs)
        self.shapes = [(inst.node.shape[2], inst.node.shape[1], inst.node.shape[0]) for inst in instances]
        self.nbc = [len(inst.boundaries) for inst in instances]
        n = len(instances)
        h = ctypes.c_void_p()
        st = L.lbm_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            msg = "lbm_create failed (see stderr)"
            if st == -1:
                why = ctypes.create_string_buffer(512)
                if L.lbm_check_config(ctypes.byref(cfg), None, why, len(why)) != 0:
                    msg = why.value.decode()
            raise LBMError(st, msg)
        self._keep = None
        self._h = h
        self.precision = int(precision)
        self.n_instances = n

    def _ck(self, st):
        if st != 0:
            raise LBMError(st, load().lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().lbm_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- entry points ---------------------------------------------------
    def set_0d_params(self, inst: int, bc: int, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        self._ck(load().lbm_set_0d_params(self._h, inst, bc, _p(p), p.size))

    def init_populations(self, inst: int, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        nx, ny, nz = self.shapes[inst]
        if f.size != 19 * nx * ny * nz:
            raise ValueError("populations must be 19 x nx*ny*nz")
        self._ck(load().lbm_init_populations(self._h, inst, _p(f)))

    def step(self, n: int = 1):
        self._ck(load().lbm_step(self._h, int(n)))

    def sync(self):
        self._ck(load().lbm_sync(self._h))

    def fields(self, inst: int = 0):
        nx, ny, nz = self.shapes[inst]
        out = [np.empty(nx * ny * nz) for _ in range(4)]
        self._ck(load().lbm_read_fields(self._h, inst, *[_p(a) for a in out]))
        return out

    def populations(self, inst: int = 0) -> np.ndarray:
        nx, ny, nz = self.shapes[inst]
        out = np.empty((19, nx * ny * nz))
        self._ck(load().lbm_read_populations(self._h, inst, _p(out)))
        return out

    def state_0d(self, inst: int, bc: int) -> np.ndarray:
        out = np.empty(8)
        self._ck(load().lbm_read_0d_state(self._h, inst, bc, _p(out)))
        return out

    def waves(self, inst: int = 0, max_rows: int = 1 << 30) -> np.ndarray:
        info = self.info()
        rows_cap = int(min(max_rows, info.steps, 1 << 24))
        width = 1 + 4 * self.nbc[inst]
        out = np.empty((max(rows_cap, 1), width))
        rows = ctypes.c_int64()
        self._ck(load().lbm_read_waveforms(self._h, inst, _p(out), rows_cap, ctypes.byref(rows)))
        return out[:rows.value]

    def ib_state(self, inst: int, n: int):
        out = [np.empty((n, 3)) for _ in range(4)]
        self._ck(load().lbm_read_ib(self._h, inst, *[_p(a) for a in out]))
        return out  # X, Vs, F, Vf

    def set_ib_state(self, inst: int, X, Vs):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Vs = np.ascontiguousarray(Vs, dtype=np.float64)
        self._ck(load().lbm_set_ib_state(self._h, inst, _p(X), _p(Vs)))

    def set_kernel_timing(self, enable: bool):
        self._ck(load().lbm_set_kernel_timing(self._h, int(bool(enable))))

    def kernel_time(self):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        self._ck(load().lbm_get_kernel_time(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def wall_shear(self, inst: int = 0) -> np.ndarray:
        """(nx*ny*nz, 3) tangential wall traction next to rigid walls (box order)."""
        nx, ny, nz = self.shapes[inst]
        out = np.empty((nx * ny * nz, 3))
        self._ck(load().lbm_wall_shear(self._h, inst, _p(out)))
        return out

    def fields_device(self, inst: int, P: int, jx: int, jy: int, jz: int):
        """Writes P and j of f(t_n) as FP32 into caller-owned device arrays of
        nx*ny*nz floats (raw device pointers, e.g. tensor.data_ptr()),
        ordered on the lattice's stream."""
        self._ck(load().lbm_read_fields_device(self._h, inst, *(ctypes.c_void_p(int(a)) for a in (P, jx, jy, jz))))

    def checkpoint(self) -> np.ndarray:
        """The whole device state as a byte array (exact resume with restore)."""
        n = ctypes.c_int64()
        self._ck(load().lbm_checkpoint_size(self._h, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._ck(load().lbm_checkpoint_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value))
        return buf

    def restore(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._ck(load().lbm_checkpoint_load(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size))

    def init_equilibrium(self, inst: int, P, vx, vy, vz):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (P, vx, vy, vz)]
        nx, ny, nz = self.shapes[inst]
        if any(a.size != nx * ny * nz for a in arrs):
            raise ValueError("fields must have nx*ny*nz entries")
        self._ck(load().lbm_init_equilibrium(self._h, inst, *[_p(a) for a in arrs]))

    def set_0d_state(self, inst: int, bc: int, state, valve_open: float = 0.0, Td: float = -1e300):
        s = np.array([float(state), float(valve_open), float(Td)])
        self._ck(load().lbm_set_0d_state(self._h, inst, bc, _p(s)))

    def cycle_change(self, periods) -> np.ndarray:
        per = np.ascontiguousarray(periods, dtype=np.int64)
        if per.size != self.n_instances:
            raise ValueError("one period per instance")
        out = np.empty(self.n_instances)
        self._ck(load().lbm_cycle_change(self._h, per.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(out)))
        return out

    def state_0d_async(self, inst: int, out_ptr: int):
        """Enqueues the 8-value 0D state rows of every boundary of instance
        inst into page-locked host memory at out_ptr (8 * n_bc doubles),
        filled when the lattice's stream reaches the call."""
        self._ck(load().lbm_read_0d_state_async(self._h, inst, ctypes.c_void_p(int(out_ptr))))

    def step_io(self, inst: int, bc: int, n: int, params_ptr: int, n_params: int, states_ptr: int):
        """n steps with per-step params of boundary bc of instance inst read from
        page-locked host memory at params_ptr (n x n_params doubles) and the
        0D state rows of every boundary of inst written to page-locked host
        memory at states_ptr (n x 8 * n_bc doubles) after each step, all in
        stream order on the device (lbm_step_io)."""
        self._ck(load().lbm_step_io(self._h, int(inst), int(bc), int(n), ctypes.c_void_p(int(params_ptr)),
                                    int(n_params), ctypes.c_void_p(int(states_ptr))))

    def set_stream_collide_shape(self, block: int, variant: int):
        """Fixes the stream-collide block size and variant (0..4)."""
        self._ck(load().lbm_set_stream_collide_shape(self._h, int(block), int(variant)))

    def autotune(self, iters: int = 20, return_times: bool = False):
        """Picks the fastest stream-collide launch shape; returns (block,
        min_blocks_per_sm, cells_per_thread) and, optionally, the (5, 4) table
        of mean launch times in ms (variants x block sizes 64, 128, 192, 256)."""
        b, m, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        times = np.zeros(20)
        self._ck(load().lbm_autotune(self._h, int(iters), ctypes.byref(b), ctypes.byref(m), ctypes.byref(c),
                                     _p(times)))
        out = (b.value, m.value, c.value)
        return (out, times.reshape(5, 4)) if return_times else out

    def info(self) -> Info:
        i = Info()
        self._ck(load().lbm_get_info(self._h, ctypes.byref(i)))
        return i
