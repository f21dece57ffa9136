"""FP64 CPU oracle of the hybrid LB / Beris-Edwards colloid step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``lclb_oracle.c`` (plain C,
FP64, no code shared with the CUDA library) through ctypes.  The C source
cites, function by function, the passage of Lintuvuori et al. (Sec. 2,
Eqs. 1-8) it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lclb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liblclb_oracle.so")
_lock = threading.Lock()
_lib = None

NQ = 19


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
            L.oracle_create.restype = vp
            L.oracle_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_int, C.c_int]
            L.oracle_destroy.argtypes = [vp]
            L.oracle_set_threads.argtypes = [vp, C.c_int]
            L.oracle_S0.restype = C.c_double
            L.oracle_S0.argtypes = [vp]
            L.oracle_step_count.restype = C.c_long
            L.oracle_step_count.argtypes = [vp]
            L.oracle_init_uniaxial.argtypes = [vp, dp, C.c_double, C.c_uint64]
            L.oracle_init_helix.argtypes = [vp, C.c_int, C.c_double, C.c_uint64]
            for n in ("oracle_set_Q", "oracle_get_Q", "oracle_set_f", "oracle_get_f"):
                getattr(L, n).argtypes = [vp, dp]
            L.oracle_get_solid.argtypes = [vp, C.POINTER(C.c_int16)]
            L.oracle_get_rho_u.argtypes = [vp, dp, dp]
            L.oracle_lc_fields.argtypes = [vp, dp, dp, dp, dp]
            L.oracle_add_colloid.restype = C.c_int
            L.oracle_add_colloid.argtypes = [vp, dp, C.c_double, C.c_int, C.c_double, C.c_int, dp]
            L.oracle_set_colloid_velocity.argtypes = [vp, C.c_int, dp, dp]
            L.oracle_set_colloid_torque.argtypes = [vp, C.c_int, dp]
            L.oracle_get_colloid.argtypes = [vp, C.c_int, dp]
            L.oracle_step.argtypes = [vp, C.c_int]
            L.oracle_contact.restype = C.c_int
            L.oracle_contact.argtypes = [vp, C.POINTER(C.c_long)]
            L.oracle_links.restype = C.c_long
            L.oracle_links.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int8), C.POINTER(C.c_int16),
                                       C.c_long]
            L.oracle_diag.argtypes = [vp, dp]
            L.oracle_feq.argtypes = [C.c_double, dp, dp]
            L.oracle_lattice.argtypes = [ip, dp]
            L.oracle_eig3.argtypes = [dp, dp, dp]
            L.oracle_bulk_q.restype = C.c_double
            L.oracle_bulk_q.argtypes = [C.c_double]
            L.oracle_noise.restype = C.c_double
            L.oracle_noise.argtypes = [C.c_uint64, C.c_long, C.c_int, C.c_double]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(v, n=3) -> np.ndarray:
    a = np.zeros(n, dtype=np.float64)
    if v is not None:
        a[:] = np.asarray(v, dtype=np.float64)
    return a


NORMAL, PLANAR = 0, 1


class Oracle:
    """One periodic (or z-walled) box stepped by the FP64 C oracle.

    Fields use the SoA layout ``[comp][z][y][x]``; Q stores
    ``(xx, xy, xz, yy, yz)`` with ``zz = -xx - yy``.
    """

    def __init__(self, nx, ny, nz, *, wall_z=False, rho0=1.0, tau=2.5, A0=0.01, gamma=3.0, K=0.01, q0=0.0,
                 xi=0.7, Gamma=0.5, S0=0.0, body_force=(0.0, 0.0, 0.0), lc=True, flow=True, threads=None):
        self.L = lib()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        p = np.array([rho0, tau, A0, gamma, K, q0, xi, Gamma, S0, *body_force], dtype=np.float64)
        self.h = self.L.oracle_create(nx, ny, nz, int(bool(wall_z)), _dp(p), int(bool(lc)), int(bool(flow)))
        if not self.h:
            raise ValueError("oracle_create failed")
        self.params = dict(rho0=rho0, tau=tau, A0=A0, gamma=gamma, K=K, q0=q0, xi=xi, Gamma=Gamma)
        self.set_threads(threads if threads else 1)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.oracle_destroy(h)
            self.h = None

    def set_threads(self, n: int):
        self.L.oracle_set_threads(self.h, int(n))

    @property
    def S0(self) -> float:
        return self.L.oracle_S0(self.h)

    def init_uniaxial(self, n=(0, 0, 1), amp=0.0, seed=0):
        self.L.oracle_init_uniaxial(self.h, _dp(_vec(n)), float(amp), int(seed) & (2**64 - 1))

    def init_helix(self, axis=2, amp=0.0, seed=0):
        self.L.oracle_init_helix(self.h, int(axis), float(amp), int(seed) & (2**64 - 1))

    def set_Q(self, Q):
        a = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).reshape(5, self.N))
        self.L.oracle_set_Q(self.h, _dp(a))

    def get_Q(self) -> np.ndarray:
        a = np.empty((5, self.N))
        self.L.oracle_get_Q(self.h, _dp(a))
        return a.reshape(5, *self.shape)

    def set_f(self, f):
        a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(NQ, self.N))
        self.L.oracle_set_f(self.h, _dp(a))

    def get_f(self) -> np.ndarray:
        a = np.empty((NQ, self.N))
        self.L.oracle_get_f(self.h, _dp(a))
        return a.reshape(NQ, *self.shape)

    def get_solid(self) -> np.ndarray:
        a = np.empty(self.N, dtype=np.int16)
        self.L.oracle_get_solid(self.h, a.ctypes.data_as(C.POINTER(C.c_int16)))
        return a.reshape(self.shape)

    def get_rho_u(self):
        rho = np.empty(self.N)
        u = np.empty((3, self.N))
        self.L.oracle_get_rho_u(self.h, _dp(rho), _dp(u))
        return rho.reshape(self.shape), u.reshape(3, *self.shape)

    def lc_fields(self):
        H = np.empty((5, self.N))
        P = np.empty((9, self.N))
        F = np.empty((3, self.N))
        fe = np.empty(self.N)
        self.L.oracle_lc_fields(self.h, _dp(H), _dp(P), _dp(F), _dp(fe))
        s = self.shape
        return H.reshape(5, *s), P.reshape(9, *s), F.reshape(3, *s), fe.reshape(s)

    def add_colloid(self, X, a0, anchoring=NORMAL, w=float("inf"), mobile=False, F_ext=None) -> int:
        r = self.L.oracle_add_colloid(self.h, _dp(_vec(X)), float(a0), int(anchoring), float(w), int(bool(mobile)),
                                      _dp(_vec(F_ext)))
        if r < 0:
            raise ValueError(f"oracle_add_colloid failed ({r})")
        return r

    def set_colloid_velocity(self, cid, V, W=(0, 0, 0)):
        self.L.oracle_set_colloid_velocity(self.h, int(cid), _dp(_vec(V)), _dp(_vec(W)))

    def set_colloid_torque(self, cid, T):
        self.L.oracle_set_colloid_torque(self.h, int(cid), _dp(_vec(T)))

    def colloid(self, cid) -> dict:
        a = np.empty(27)
        self.L.oracle_get_colloid(self.h, int(cid), _dp(a))
        keys = ("X", "V", "W", "F_hyd", "T_hyd", "F_lc", "T_lc", "impulse", "ang_impulse")
        return {k: a[3 * i:3 * i + 3].copy() for i, k in enumerate(keys)}

    def step(self, n=1):
        self.L.oracle_step(self.h, int(n))

    def contact(self):
        """First contact since the last call, as ``(step, colloid, partner)``
        (partner -1: a z wall), or None.  A mobile colloid whose move would
        touch a wall or another colloid keeps its position (the oracle's
        reading; the paper treats no contact)."""
        a = (C.c_long * 3)()
        if self.L.oracle_contact(self.h, a) == 0:
            return None
        return int(a[0]), int(a[1]), int(a[2])

    @property
    def step_count(self) -> int:
        return self.L.oracle_step_count(self.h)

    def links(self):
        n = self.L.oracle_links(self.h, None, None, None, 0)
        node = np.empty(n, dtype=np.int32)
        d = np.empty(n, dtype=np.int8)
        c = np.empty(n, dtype=np.int16)
        self.L.oracle_links(self.h, node.ctypes.data_as(C.POINTER(C.c_int32)), d.ctypes.data_as(C.POINTER(C.c_int8)),
                            c.ctypes.data_as(C.POINTER(C.c_int16)), n)
        return node, d, c

    def diag(self) -> dict:
        a = np.empty(9)
        self.L.oracle_diag(self.h, _dp(a))
        return dict(mass=a[0], momentum=a[1:4].copy(), free_energy=a[4], resid_rms=a[5], resid_max=a[6],
                    n_fluid=int(a[7]), n_defect=int(a[8]))


def feq(rho: float, u) -> np.ndarray:
    out = np.empty(NQ)
    lib().oracle_feq(float(rho), _dp(_vec(u)), _dp(out))
    return out


def lattice():
    c = np.empty(3 * NQ, dtype=np.int32)
    w = np.empty(NQ)
    lib().oracle_lattice(c.ctypes.data_as(C.POINTER(C.c_int)), _dp(w))
    return c.reshape(NQ, 3), w


def eig3(A):
    a = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
    ev = np.empty(3)
    V = np.empty(9)
    lib().oracle_eig3(_dp(a), _dp(ev), _dp(V))
    return ev, V.reshape(3, 3)


def bulk_q(gamma: float) -> float:
    return lib().oracle_bulk_q(float(gamma))


def noise(seed: int, i: int, k: int, amp: float) -> float:
    return lib().oracle_noise(int(seed) & (2**64 - 1), int(i), int(k), float(amp))
