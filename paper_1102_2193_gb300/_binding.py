"""ctypes binding of ``liblclb.so`` (argument marshalling only).

Names follow the C ABI of ``include/lc_lb.h``.  Every step of the solver runs
in the CUDA library; nothing here computes.  The library must have been
built (``python -c "import __graft_entry__ as g; g.build()"``); loading fails
loudly otherwise.  PyTorch is used, when importable, only to hand the
library its caching allocator and current stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

LC_OK, LC_ERR_ARG, LC_ERR_CUDA, LC_ERR_OOM, LC_ERR_OVERLAP, LC_ERR_NONFINITE, LC_ERR_TIMEOUT, LC_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
LC_FP32, LC_FP64 = 0, 1
LC_NORMAL, LC_PLANAR = 0, 1
LC_Q, LC_U, LC_RHO, LC_F_PRE, LC_FORCE, LC_SOLID = 0, 1, 2, 3, 4, 5
PHASES = ("flb", "lc", "links", "colloid", "step")  # "flb": the force + LB part, whatever its variant

VARIANTS = ("fused", "split", "stored", "dataflow")
VARIANT_KERNELS = (("k_flb",), ("k_force", "k_lb"), ("k_stress", "k_lbp"), ("k_stress", "k_lbp"))


def _profile_dict(ms) -> dict:
    """Mean ms per step: the force + LB part, the Q update, the link exchange
    and the colloid update run as separate kernels (a breakdown), and the whole
    step as it runs ("step": for the dataflow variant the one persistent
    launch k_step)."""
    out = dict(zip(PHASES, ms[:5].tolist()))
    v = int(round(ms[5]))
    out["variant"] = VARIANTS[v]
    out["kernels"] = dict(zip(VARIANT_KERNELS[v], ms[6:8].tolist()))
    if VARIANTS[v] == "dataflow":
        out["kernels"]["k_step"] = out["step"]
    return out


_NCOMP = {LC_Q: 5, LC_U: 3, LC_RHO: 1, LC_F_PRE: 19, LC_FORCE: 3, LC_SOLID: 1}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")


def library_path() -> str:
    return os.path.join(_LIBDIR, "liblclb.so")


class LcLbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lc_lb error {code}: {msg}")
        self.code = code


class lc_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("wall_z", C.c_int)]


class lc_params(C.Structure):
    _fields_ = [("rho0", C.c_double), ("tau", C.c_double), ("A0", C.c_double), ("gamma", C.c_double),
                ("K", C.c_double), ("q0", C.c_double), ("xi", C.c_double), ("Gamma", C.c_double),
                ("S0", C.c_double), ("body_force", C.c_double * 3), ("precision", C.c_int),
                ("lc_enabled", C.c_int), ("flow_enabled", C.c_int), ("reserved", C.c_int)]


class lc_diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("momentum", C.c_double * 3), ("free_energy", C.c_double),
                ("resid_rms", C.c_double), ("resid_max", C.c_double), ("n_fluid", C.c_longlong),
                ("n_defect", C.c_longlong), ("step", C.c_longlong)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_lock = threading.Lock()
_lib = None
_keep = []


def _torch_allocator(L):
    """Route the library's device allocations through PyTorch's caching allocator."""
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except Exception:
        return

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0) or torch.cuda.current_stream().cuda_stream)
        except Exception:
            return None

    def free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a, f = _ALLOC(alloc), _FREE(free)
    _keep.extend([a, f])
    L.lc_lb_set_allocator(a, f, None)


def lib(use_torch_allocator: bool = True):
    """Load ``liblclb.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        L = C.CDLL(path)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.lc_lb_set_allocator.argtypes = [_ALLOC, _FREE, vp]
        L.lc_lb_create.argtypes = [C.POINTER(lc_grid), C.POINTER(lc_params), vp, C.POINTER(vp)]
        L.lc_lb_destroy.argtypes = [vp]
        L.lc_lb_destroy.restype = None
        L.lc_lb_init_uniaxial.argtypes = [vp, dp, C.c_double, C.c_uint64]
        L.lc_lb_init_helix.argtypes = [vp, C.c_int, C.c_double, C.c_uint64]
        L.lc_lb_set_fields.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
        L.lc_lb_add_colloid.argtypes = [vp, dp, C.c_double, C.c_int, C.c_double, C.c_int, dp, ip]
        L.lc_lb_set_colloid_velocity.argtypes = [vp, C.c_int, dp, dp]
        L.lc_lb_set_colloid_force.argtypes = [vp, C.c_int, dp]
        L.lc_lb_set_colloid_torque.argtypes = [vp, C.c_int, dp]
        L.lc_lb_step.argtypes = [vp, C.c_int]
        L.lc_lb_relax.argtypes = [vp, C.c_double, C.c_longlong, C.c_int, C.POINTER(C.c_longlong), dp]
        L.lc_lb_get_fields.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
        L.lc_lb_get_forces.argtypes = [vp, C.c_int, dp, dp, dp, dp, dp]
        L.lc_lb_get_colloid.argtypes = [vp, C.c_int, dp]
        L.lc_lb_get_links.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int8), C.POINTER(C.c_int16),
                                      C.c_size_t, C.POINTER(C.c_size_t)]
        lp = C.POINTER(C.c_longlong)
        L.lc_lb_defects.argtypes = [vp, C.c_double, C.c_size_t, lp, lp, lp, lp, dp, dp]
        L.lc_lb_defect_labels.argtypes = [vp, C.c_double, vp, C.c_size_t, C.c_int]
        L.lc_lb_diagnostics.argtypes = [vp, C.POINTER(lc_diag)]
        L.lc_lb_diagnostics_noalloc.argtypes = [vp, C.POINTER(lc_diag)]
        L.lc_lb_profile.argtypes = [vp, C.c_int, dp]
        L.lc_lb_batch_profile.argtypes = [vp, C.c_int, dp]
        L.lc_lb_profile_detail.argtypes = [vp, C.c_int, dp]
        L.lc_lb_batch_profile_detail.argtypes = [vp, C.c_int, dp]
        L.lc_lb_step_launches.argtypes = [vp, ip]
        L.lc_lb_batch_step_launches.argtypes = [vp, ip]
        L.lc_lb_synchronize.argtypes = [vp]
        L.lc_lb_last_error.argtypes = [vp]
        L.lc_lb_last_error.restype = C.c_char_p
        L.lc_lb_version.argtypes = []
        L.lc_lb_version.restype = C.c_char_p
        L.lc_lb_batch_create.argtypes = [C.c_int, C.POINTER(lc_grid), C.POINTER(lc_params), vp, C.POINTER(vp)]
        L.lc_lb_batch_destroy.argtypes = [vp]
        L.lc_lb_batch_destroy.restype = None
        L.lc_lb_batch_box.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.lc_lb_batch_step.argtypes = [vp, C.c_int]
        L.lc_lb_batch_relax.argtypes = [vp, C.c_double, C.c_longlong, C.c_int, C.POINTER(C.c_longlong), dp]
        L.lc_lb_batch_last_error.argtypes = [vp]
        L.lc_lb_batch_last_error.restype = C.c_char_p
        L.lc_lb_autotune.argtypes = [C.POINTER(lc_grid), C.c_int, vp, C.c_char_p, C.c_size_t]
        # learned warm start (include/lc_nn.h)
        L.lc_nn_conv3d_fwd.argtypes = [vp, vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_int, vp]
        L.lc_nn_conv3d_dgrad.argtypes = [vp, vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]
        L.lc_nn_conv3d_wgrad.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]
        L.lc_nn_wgrad_partial_floats.argtypes = [C.c_int] * 6
        L.lc_nn_wgrad_partial_floats.restype = C.c_size_t
        L.lc_nn_bias_grad.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.lc_nn_relu_bwd.argtypes = [vp, vp, vp, vp, C.c_size_t, vp]
        L.lc_nn_cast_bf16.argtypes = [vp, vp, C.c_size_t, vp]
        L.lc_nn_pool2.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.lc_nn_pool2_bwd.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.lc_nn_up2_concat.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, vp]
        L.lc_nn_up2_concat_bwd.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, vp]
        L.lc_nn_mse.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int, C.c_int, C.c_double, vp]
        L.lc_nn_mse_coarse.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_double, vp]
        L.lc_nn_adam.argtypes = [vp, vp, vp, vp, vp, C.c_size_t, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                                 vp]
        L.lc_nn_pack_input.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, vp, vp, vp, vp, C.c_int, C.c_int,
                                       vp]
        L.lc_nn_from_soa.argtypes = [vp, vp, C.c_int, vp]
        L.lc_nn_to_soa.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
        L.lc_nn_trilinear2.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        if use_torch_allocator:
            _torch_allocator(L)
        _lib = L
        return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _v3(v):
    a = np.zeros(3)
    if v is not None:
        a[:] = np.asarray(v, dtype=np.float64)
    return a


def make_params(rho0=1.0, tau=2.5, A0=0.01, gamma=3.0, K=0.01, q0=0.0, xi=0.7, Gamma=0.5, S0=0.0,
                body_force=(0.0, 0.0, 0.0), precision=LC_FP32, lc=True, flow=True) -> lc_params:
    p = lc_params()
    p.rho0, p.tau, p.A0, p.gamma, p.K, p.q0, p.xi, p.Gamma, p.S0 = rho0, tau, A0, gamma, K, q0, xi, Gamma, S0
    for k in range(3):
        p.body_force[k] = float(body_force[k])
    p.precision = {"f32": LC_FP32, "f64": LC_FP64}.get(precision, precision)
    p.lc_enabled, p.flow_enabled = int(bool(lc)), int(bool(flow))
    return p


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Solver:
    """One box (``lc_lb*``).  Keyword arguments as :func:`make_params`."""

    def __init__(self, nx, ny, nz, wall_z=False, stream=None, _borrowed=None, _owner=None, **params):
        self.L = lib()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self._owner = _owner
        if _borrowed is not None:
            self.h = _borrowed
            self._own = False
            return
        g = lc_grid(nx, ny, nz, int(bool(wall_z)))
        p = make_params(**params)
        h = C.c_void_p()
        self._check(self.L.lc_lb_create(C.byref(g), C.byref(p), _stream_ptr(stream), C.byref(h)), None)
        self.h = h
        self._own = True

    def _check(self, rc, h="self"):
        if rc != LC_OK:
            hh = self.h if h == "self" else h
            msg = self.L.lc_lb_last_error(hh)
            raise LcLbError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_own", False) and self.h:
            self.L.lc_lb_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ---------------------------------------------------------
    def init_uniaxial(self, n=(0, 0, 1), amp=0.0, seed=0):
        self._check(self.L.lc_lb_init_uniaxial(self.h, _dp(_v3(n)), float(amp), int(seed) & (2**64 - 1)))

    def init_helix(self, axis=2, amp=0.0, seed=0):
        self._check(self.L.lc_lb_init_helix(self.h, int(axis), float(amp), int(seed) & (2**64 - 1)))

    def set_fields(self, which, arr):
        if hasattr(arr, "data_ptr"):  # device tensor (FP64, contiguous)
            self._check(self.L.lc_lb_set_fields(self.h, which, C.c_void_p(arr.data_ptr()), arr.numel() * 8, 1))
            return
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
        self._check(self.L.lc_lb_set_fields(self.h, which, a.ctypes.data_as(C.c_void_p), a.nbytes, 0))

    def set_Q(self, Q):
        self.set_fields(LC_Q, Q)

    def set_f(self, f):
        self.set_fields(LC_F_PRE, f)

    def get_fields(self, which, out=None):
        n = _NCOMP[which]
        if out is not None and hasattr(out, "data_ptr"):
            self._check(self.L.lc_lb_get_fields(self.h, which, C.c_void_p(out.data_ptr()), out.numel() * 8, 1))
            return out
        a = np.empty((n, *self.shape)) if out is None else out
        self._check(self.L.lc_lb_get_fields(self.h, which, a.ctypes.data_as(C.c_void_p), a.nbytes, 0))
        return a

    def get_Q(self):
        return self.get_fields(LC_Q)

    def get_f(self):
        return self.get_fields(LC_F_PRE)

    def get_rho_u(self):
        return self.get_fields(LC_RHO)[0], self.get_fields(LC_U)

    def get_force_field(self):
        return self.get_fields(LC_FORCE)

    def get_solid(self):
        return self.get_fields(LC_SOLID)[0].astype(np.int16)

    # -- colloids --------------------------------------------------------
    def add_colloid(self, X, a0, anchoring=LC_NORMAL, w=float("inf"), mobile=False, F_ext=None) -> int:
        cid = C.c_int()
        self._check(self.L.lc_lb_add_colloid(self.h, _dp(_v3(X)), float(a0), int(anchoring), float(w),
                                             int(bool(mobile)), _dp(_v3(F_ext)), C.byref(cid)))
        return cid.value

    def set_colloid_velocity(self, cid, V, W=(0, 0, 0)):
        self._check(self.L.lc_lb_set_colloid_velocity(self.h, int(cid), _dp(_v3(V)), _dp(_v3(W))))

    def set_colloid_force(self, cid, F_ext):
        self._check(self.L.lc_lb_set_colloid_force(self.h, int(cid), _dp(_v3(F_ext))))

    def set_colloid_torque(self, cid, T_ext):
        self._check(self.L.lc_lb_set_colloid_torque(self.h, int(cid), _dp(_v3(T_ext))))

    def colloid(self, cid) -> dict:
        a = np.empty(27)
        self._check(self.L.lc_lb_get_colloid(self.h, int(cid), _dp(a)))
        keys = ("X", "V", "W", "F_hyd", "T_hyd", "F_lc", "T_lc", "impulse", "ang_impulse")
        return {k: a[3 * i:3 * i + 3].copy() for i, k in enumerate(keys)}

    def forces(self, cid):
        F, T, V, W, X = (np.empty(3) for _ in range(5))
        self._check(self.L.lc_lb_get_forces(self.h, int(cid), _dp(F), _dp(T), _dp(V), _dp(W), _dp(X)))
        return dict(F=F, T=T, V=V, W=W, X=X)

    def links(self):
        n = C.c_size_t()
        self._check(self.L.lc_lb_get_links(self.h, None, None, None, 0, C.byref(n)))
        k = n.value
        node = np.empty(k, np.int32)
        d = np.empty(k, np.int8)
        c = np.empty(k, np.int16)
        self._check(self.L.lc_lb_get_links(self.h, node.ctypes.data_as(C.POINTER(C.c_int32)),
                                           d.ctypes.data_as(C.POINTER(C.c_int8)),
                                           c.ctypes.data_as(C.POINTER(C.c_int16)), k, C.byref(n)))
        return node, d, c

    def defects(self, thr=0.435) -> dict:
        """Components of the defect nodes (lc_lb_defects): counts, roots,
        sizes, centroids [n, 3] and gyration tensors [n, 6]."""
        nd, nc = C.c_longlong(), C.c_longlong()
        self._check(self.L.lc_lb_defects(self.h, float(thr), 0, C.byref(nd), C.byref(nc), None, None, None, None))
        k = nc.value
        root = np.empty(k, np.int64)
        size = np.empty(k, np.int64)
        cen = np.empty((k, 3))
        gyr = np.empty((k, 6))
        lp = C.POINTER(C.c_longlong)
        self._check(self.L.lc_lb_defects(self.h, float(thr), k, C.byref(nd), C.byref(nc), root.ctypes.data_as(lp),
                                         size.ctypes.data_as(lp), _dp(cen), _dp(gyr)))
        return dict(n_defect=nd.value, n_comp=nc.value, root=root, size=size, centroid=cen, gyration=gyr)

    def defect_labels(self, thr=0.435, out=None):
        """Per-node root of the node's defect component, -1 elsewhere
        (lc_lb_defect_labels); into a device int32 tensor when given."""
        if out is not None and hasattr(out, "data_ptr"):
            self._check(self.L.lc_lb_defect_labels(self.h, float(thr), C.c_void_p(out.data_ptr()), out.numel(), 1))
            return out
        a = np.empty(self.shape, np.int32)
        self._check(self.L.lc_lb_defect_labels(self.h, float(thr), a.ctypes.data_as(C.c_void_p), a.size, 0))
        return a

    # -- dynamics --------------------------------------------------------
    def step(self, n=1):
        self._check(self.L.lc_lb_step(self.h, int(n)))

    def relax(self, tol=1e-8, max_steps=10**6, check_every=500):
        s = C.c_longlong()
        r = C.c_double()
        self._check(self.L.lc_lb_relax(self.h, float(tol), int(max_steps), int(check_every), C.byref(s), C.byref(r)))
        return s.value, r.value

    def synchronize(self):
        self._check(self.L.lc_lb_synchronize(self.h))

    def step_launches(self) -> int:
        """Kernel launches in one captured step."""
        n = C.c_int()
        self._check(self.L.lc_lb_step_launches(self.h, C.byref(n)))
        return n.value

    def profile(self, n=10) -> dict:
        """Mean ms per step of each phase over n non-graph steps (advances the
        state), the step variant and its force + LB kernels."""
        ms = np.empty(8)
        self._check(self.L.lc_lb_profile_detail(self.h, int(n), _dp(ms)))
        return _profile_dict(ms)

    def diag(self) -> dict:
        d = lc_diag()
        self._check(self.L.lc_lb_diagnostics(self.h, C.byref(d)))
        return dict(mass=d.mass, momentum=np.array(d.momentum[:]), free_energy=d.free_energy,
                    resid_rms=d.resid_rms, resid_max=d.resid_max, n_fluid=d.n_fluid, n_defect=d.n_defect,
                    step=d.step)


class Batch:
    """Many independent boxes advanced together (``lc_lb_batch*``).

    ``boxes`` is a list of dicts with ``grid=(nx,ny,nz)``, optional
    ``wall_z`` and ``params`` (keyword arguments of :func:`make_params`).
    """

    def __init__(self, boxes, precision=LC_FP32, stream=None):
        self.L = lib()
        n = len(boxes)
        G = (lc_grid * n)()
        P = (lc_params * n)()
        for i, b in enumerate(boxes):
            nx, ny, nz = b["grid"]
            G[i] = lc_grid(nx, ny, nz, int(bool(b.get("wall_z", False))))
            P[i] = make_params(precision=precision, **b.get("params", {}))
        h = C.c_void_p()
        rc = self.L.lc_lb_batch_create(n, G, P, _stream_ptr(stream), C.byref(h))
        if rc != LC_OK:
            msg = self.L.lc_lb_batch_last_error(None)
            raise LcLbError(rc, msg.decode() if msg else "")
        self.h = h
        self.n = n
        self.boxes = []
        for i, b in enumerate(boxes):
            bh = C.c_void_p()
            self._check(self.L.lc_lb_batch_box(self.h, i, C.byref(bh)))
            nx, ny, nz = b["grid"]
            self.boxes.append(Solver(nx, ny, nz, _borrowed=bh, _owner=self))

    def _check(self, rc):
        if rc != LC_OK:
            msg = self.L.lc_lb_batch_last_error(self.h)
            raise LcLbError(rc, msg.decode() if msg else "")

    def step(self, n=1):
        self._check(self.L.lc_lb_batch_step(self.h, int(n)))

    def relax(self, tol=1e-8, max_steps=10**6, check_every=500):
        s = C.c_longlong()
        r = np.empty(self.n)
        self._check(self.L.lc_lb_batch_relax(self.h, float(tol), int(max_steps), int(check_every), C.byref(s),
                                             _dp(r)))
        return s.value, r

    def step_launches(self) -> int:
        n = C.c_int()
        self._check(self.L.lc_lb_batch_step_launches(self.h, C.byref(n)))
        return n.value

    def profile(self, n=10) -> dict:
        ms = np.empty(8)
        self._check(self.L.lc_lb_batch_profile_detail(self.h, int(n), _dp(ms)))
        return _profile_dict(ms)

    def close(self):
        if getattr(self, "h", None):
            for b in self.boxes:
                b.h = None
            self.L.lc_lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
