"""Plain FP64 CPU oracle of the 0D-3D lattice Boltzmann step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library under
``paper_2112_05258_gb300`` never imports it, and it imports nothing from
there.  The C source ``lbm_oracle.c`` follows Algorithm 1 of the paper
step by step; see the comments there for the passage each function follows.

Parity pins: every function of the C file is pinned by a test under
``tests/test_oracle_*.py`` against closed forms, conservation laws,
invariants or brute force (no pin re-types a formula of the oracle).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (IEEE FP64, no fast-math, no FMA
    contraction), with OpenMP for the per-cell loops where gcc has it (the
    results do not depend on the thread count; one thread by default)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int]
            L.orc_add_boundary.restype = ctypes.c_int
            L.orc_add_boundary.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, _dp, ctypes.c_int, _dp,
                                           ctypes.c_long, _dp, ctypes.c_int]
            L.orc_set_ib.argtypes = [ctypes.c_void_p, ctypes.c_long, _dp, _dp, _dp, _u8p,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_set_ib_state.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_lv_step_ord.argtypes = [_dp, _dp, _dp, ctypes.c_long] + [ctypes.c_double] * 4 + \
                [ctypes.c_int] + [ctypes.c_double] * 3 + [ctypes.POINTER(ctypes.c_int)]
            L.orc_set_filaments.argtypes = [ctypes.c_void_p, ctypes.c_long, _lp, _lp, _lp, _dp]
            L.orc_filament_force.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, _dp]
            L.orc_set_body_force.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 3
            L.orc_set_populations.argtypes = [ctypes.c_void_p, _dp]
            L.orc_get_populations.argtypes = [ctypes.c_void_p, _dp]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            L.orc_get_macros.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_get_force.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            L.orc_get_0d.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
            L.orc_wall_shear.argtypes = [ctypes.c_void_p, _dp]
            L.orc_wave_rows.restype = ctypes.c_long
            L.orc_wave_rows.argtypes = [ctypes.c_void_p]
            L.orc_get_waves.argtypes = [ctypes.c_void_p, _dp]
            L.orc_get_ib.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_n_xf.restype = ctypes.c_long
            L.orc_n_xf.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_n_links.restype = ctypes.c_long
            L.orc_n_links.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_feq.argtypes = [ctypes.c_double, _dp, _dp]
            L.orc_forcing.argtypes = [ctypes.c_double, _dp, _dp, _dp]
            L.orc_smooth.restype = ctypes.c_double
            L.orc_smooth.argtypes = [ctypes.c_double] * 3
            L.orc_rcr_step.restype = ctypes.c_double
            L.orc_rcr_step.argtypes = [_dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double]
            L.orc_lv_ode.restype = ctypes.c_double
            L.orc_lv_ode.argtypes = [ctypes.c_double] * 4
            L.orc_lv_step.argtypes = [_dp, _dp, _dp, ctypes.c_long, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
            L.orc_rcr_step_ord.restype = ctypes.c_double
            L.orc_rcr_step_ord.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int]
            L.orc_lv_ode_ord.restype = ctypes.c_double
            L.orc_lv_ode_ord.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int]
            L.orc_phi.restype = ctypes.c_double
            L.orc_phi.argtypes = [ctypes.c_double]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_openmp.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


# ---- small pure functions (for pins) -------------------------------------

def feq(P: float, v) -> np.ndarray:
    out = np.zeros(19)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    lib().orc_feq(P, _p(vv), _p(out))
    return out


def forcing(tau: float, v, b) -> np.ndarray:
    out = np.zeros(19)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    lib().orc_forcing(tau, _p(vv), _p(bb), _p(out))
    return out


def smooth(t: float, t0: float, LS: float) -> float:
    return lib().orc_smooth(t, t0, LS)


def rcr_step(Pw: float, Qout: float, Rp: float, C: float, Rd: float):
    """Returns (P_w(t_{n+1}), boundary gauge pressure P(t_{n+1}))."""
    s = np.array([Pw], dtype=np.float64)
    P = lib().orc_rcr_step(_p(s), Qout, Rp, C, Rd)
    return float(s[0]), P


def lv_ode(Pv: float, E: float, Edot: float, Qin: float) -> float:
    return lib().orc_lv_ode(Pv, E, Edot, Qin)


def rcr_step_ord(Pw: float, Qout: float, Rp: float, C: float, Rd: float, order: int):
    s = np.array([Pw], dtype=np.float64)
    P = lib().orc_rcr_step_ord(_p(s), Qout, Rp, C, Rd, int(order))
    return float(s[0]), P


def lv_ode_ord(Pv, E0, D0, E1, D1, Qin, order):
    return lib().orc_lv_ode_ord(Pv, E0, D0, E1, D1, Qin, int(order))


def lv_step(Pv, valve_open, Td, n, E, Edot, Qu, Pbar_gauge, P_la):
    """Returns (P_v, valve_open, T_d, closed_now) after one hybrid LV step."""
    a = np.array([Pv]); b = np.array([valve_open]); c = np.array([Td])
    closed = ctypes.c_int(0)
    lib().orc_lv_step(_p(a), _p(b), _p(c), n, E, Edot, Qu, Pbar_gauge, P_la,
                      ctypes.byref(closed))
    return float(a[0]), float(b[0]), float(c[0]), int(closed.value)


def lv_step_ord(Pv, valve_open, Td, n, E, Edot, E1, Edot1, order, Qu, Pbar_gauge, P_la):
    """lv_step marched at the given order with the elastance table values at
    t_n (E, Edot) and t_{n+1} (E1, Edot1)."""
    a = np.array([Pv]); b = np.array([valve_open]); c = np.array([Td])
    closed = ctypes.c_int(0)
    lib().orc_lv_step_ord(_p(a), _p(b), _p(c), n, E, Edot, E1, Edot1, int(order), Qu, Pbar_gauge, P_la,
                          ctypes.byref(closed))
    return float(a[0]), float(b[0]), float(c[0]), int(closed.value)


def filament_force(X, gl, gr, ds: float, Eh: float, EI: float) -> np.ndarray:
    """SGFD internal force per unit length at the interior nodes of one
    filament (zero at its two ends); ``gl``/``gr`` the ghost nodes beyond them."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(X)
    gl = np.ascontiguousarray(gl, dtype=np.float64)
    gr = np.ascontiguousarray(gr, dtype=np.float64)
    lib().orc_filament_force(X.shape[0], _p(X), _p(gl), _p(gr), float(ds), float(Eh), float(EI), _p(out))
    return out


def phi(r: float) -> float:
    return lib().orc_phi(r)


def set_threads(n: int) -> int:
    """Threads of the oracle's per-cell loops (process-wide); returns the
    count in effect (1 when the oracle was built without OpenMP)."""
    L = lib()
    n = max(1, int(n)) if L.orc_openmp() else 1
    L.orc_set_threads(n)
    return n


# ---- the lattice ---------------------------------------------------------

class Oracle:
    """One instance run by the CPU oracle.

    ``inst`` is a :class:`workloads.Instance`.  ``periodic`` is a bitmask of
    periodic axes (x = 1, y = 2, z = 4; oracle-only, for pins).
    """

    def __init__(self, inst, periodic: int = 0):
        L = lib()
        self.inst = inst
        nx, ny, nz = inst.shape
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        node = np.ascontiguousarray(inst.node, dtype=np.uint8).reshape(-1)
        self._h = L.orc_create(nx, ny, nz, node.ctypes.data_as(_u8p), float(inst.tau),
                               int(periodic), int(inst.q_scale))
        for b in inst.boundaries:
            par = np.ascontiguousarray(b.params, dtype=np.float64)
            prof = (np.ascontiguousarray(b.profile, dtype=np.float64)
                    if b.profile is not None else np.zeros((1, 3)))
            etab = (np.ascontiguousarray(b.elastance, dtype=np.float64)
                    if b.elastance is not None else np.zeros((1, 2)))
            nprof = prof.shape[0] if b.profile is not None else 0
            period = etab.shape[0] if b.elastance is not None else 0
            k = L.orc_add_boundary(self._h, int(b.kind), int(b.axis), int(b.sign), _p(par),
                                   par.size, _p(prof), nprof, _p(etab), period)
            if k < 0:
                raise ValueError(f"oracle rejected boundary ({k})")
        if inst.ib is not None:
            ib = inst.ib
            self._ib_args = (np.ascontiguousarray(ib.X0, dtype=np.float64),
                             np.ascontiguousarray(ib.dA, dtype=np.float64),
                             np.ascontiguousarray(ib.ks, dtype=np.float64),
                             np.ascontiguousarray(ib.pinned, dtype=np.uint8))
            X0, dA, ks, pin = self._ib_args
            L.orc_set_ib(self._h, ib.n, _p(X0), _p(dA), _p(ks), pin.ctypes.data_as(_u8p),
                         float(ib.alpha), float(ib.beta), float(ib.ms))
            if getattr(ib, "filaments", None):
                cnt = np.array([len(f) for f in ib.filaments], dtype=np.int64)
                st = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
                nodes = np.ascontiguousarray(np.concatenate(ib.filaments), dtype=np.int64)
                par = np.ascontiguousarray(ib.fil_par, dtype=np.float64).reshape(-1)
                self._fil_args = (cnt, st, nodes, par)
                L.orc_set_filaments(self._h, cnt.size, st.ctypes.data_as(_lp), cnt.ctypes.data_as(_lp),
                                    nodes.ctypes.data_as(_lp), _p(par))
        self.nbc = len(inst.boundaries)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_ib_state(self, X, Vs):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Vs = np.ascontiguousarray(Vs, dtype=np.float64)
        lib().orc_set_ib_state(self._h, _p(X), _p(Vs))

    def set_body_force(self, g):
        lib().orc_set_body_force(self._h, float(g[0]), float(g[1]), float(g[2]))

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
        lib().orc_set_populations(self._h, _p(f))

    def populations(self) -> np.ndarray:
        f = np.empty((19, self.N))
        lib().orc_get_populations(self._h, _p(f))
        return f

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def macros(self):
        """(P, jx, jy, jz) of the current f(t_n), each flat (N,)."""
        out = [np.empty(self.N) for _ in range(4)]
        lib().orc_get_macros(self._h, *[_p(a) for a in out])
        return out

    def force(self):
        out = [np.empty(self.N) for _ in range(3)]
        lib().orc_get_force(self._h, *[_p(a) for a in out])
        return out

    def wall_shear(self) -> np.ndarray:
        """(N, 3) tangential wall traction at the fluid cells next to a wall."""
        out = np.empty((self.N, 3))
        lib().orc_wall_shear(self._h, _p(out))
        return out

    def state_0d(self, k: int) -> np.ndarray:
        out = np.empty(8)
        lib().orc_get_0d(self._h, int(k), _p(out))
        return out

    def waves(self) -> np.ndarray:
        rows = lib().orc_wave_rows(self._h)
        out = np.empty((rows, 1 + 4 * self.nbc))
        if rows:
            lib().orc_get_waves(self._h, _p(out))
        return out

    def ib_state(self):
        ns = self.inst.ib.n
        out = [np.empty((ns, 3)) for _ in range(4)]
        lib().orc_get_ib(self._h, *[_p(a) for a in out])
        return out  # X, Vs, F, Vf

    def n_xf(self, k: int) -> int:
        return lib().orc_n_xf(self._h, int(k))

    def n_links(self, k: int) -> int:
        return lib().orc_n_links(self._h, int(k))


from .periodic import cycle_change  # noqa: E402,F401  (periodic-state criterion)
