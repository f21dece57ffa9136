"""Learned warm start: a small 3D U-Net proposing the relaxed Q around a colloid.

The network maps a periodic S^3 box (S divisible by 4) with input channels
[solid indicator, the 5 components of the initial Q, R/32, pitch/64, 20 w] to
a correction of Q, pred = Q_init + net(...), and is trained with a masked
mean-square error on fluid nodes against fields that the lattice relaxation
of ``lc_lb`` produced (Sec. 3.2: the relaxed defect structure around a
colloid in a cholesteric).  Every arithmetic step runs in the CUDA kernels of
``include/lc_nn.h`` (BF16 convolutions with FP32 accumulation on the tensor
cores, FP32 Adam masters); this module only sequences the calls and holds the
buffers, which are PyTorch device tensors used as plain device memory.

Architecture (3x3x3 convolutions, ReLU, periodic): 16 -> 16, 16 (S) | pool |
16 -> 32, 32 (S/2) | pool | 32 -> 48, 48 (S/4) | up + skip | 80 -> 32 (S/2) |
up + skip | 48 -> 16 (S) | 1x1 16 -> 16 (5 used); 249,744 parameters.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from ._binding import LC_Q, LC_SOLID, lib

CPAD = 16  # input channels (9 used, padded for the tensor-core K dimension)

# (name, cin, cout, taps, relu, level): level 0 = S, 1 = S/2, 2 = S/4
LAYERS = [("c0a", CPAD, 16, 27, 1, 0), ("c0b", 16, 16, 27, 1, 0), ("c1a", 16, 32, 27, 1, 1), ("c1b", 32, 32, 27, 1, 1),
          ("c2a", 32, 48, 27, 1, 2), ("c2b", 48, 48, 27, 1, 2), ("c3", 80, 32, 27, 1, 1), ("c4", 48, 16, 27, 1, 0),
          ("head", 16, 16, 1, 0, 0)]


def _p(t):
    return C.c_void_p(t.data_ptr())


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc})")


class UNet:
    """Parameters, optimiser state and activation buffers for one box size S."""

    def __init__(self, S: int = 64, seed: int = 0, device="cuda", stream=None):
        import torch
        assert S % 4 == 0
        self.torch = torch
        self.L = lib()
        self.S = S
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.sp = C.c_void_p(self.stream.cuda_stream)
        g = np.random.default_rng(seed)
        self.params = {}
        for name, cin, cout, taps, relu, lvl in LAYERS:
            fan_in = cin * taps
            scale = math.sqrt(2.0 / fan_in) if relu else 0.0  # the head starts at zero: pred = Q_init
            w = (g.standard_normal((cout, taps, cin)) * scale).astype(np.float32)
            if name == "c0a":
                w[:, :, 9:] = 0.0
            P = {"w": torch.tensor(w, device=self.dev), "b": torch.zeros(cout, device=self.dev)}
            for k in ("w", "b"):
                P["g" + k] = torch.zeros_like(P[k])
                P["m" + k] = torch.zeros_like(P[k])
                P["v" + k] = torch.zeros_like(P[k])
            P["w16"] = torch.empty(P["w"].shape, dtype=torch.bfloat16, device=self.dev)
            P["wt"] = torch.empty(P["w"].numel(), dtype=torch.bfloat16, device=self.dev)
            self.params[name] = P
            self._cast(P["w"], P["w16"])
        self.step_count = 0
        self._alloc()

    # -- buffers ---------------------------------------------------------------
    def _alloc(self):
        t, S = self.torch, self.S
        n = [S**3, (S // 2)**3, (S // 4)**3]
        bf = lambda k, c: t.empty((n[k], c), dtype=t.bfloat16, device=self.dev)  # noqa: E731
        f32 = lambda k, c: t.empty((n[k], c), dtype=t.float32, device=self.dev)  # noqa: E731
        self.a = {"x": bf(0, CPAD), "c0a": bf(0, 16), "c0b": bf(0, 16), "p0": bf(1, 16), "c1a": bf(1, 32),
                  "c1b": bf(1, 32), "p1": bf(2, 32), "c2a": bf(2, 48), "c2b": bf(2, 48), "u1": bf(1, 80),
                  "c3": bf(1, 32), "u0": bf(0, 48), "c4": bf(0, 16)}
        self.y = f32(0, 16)
        self.base = f32(0, 5)
        self.target = f32(0, 5)
        self.fluid = t.empty(n[0], dtype=t.float32, device=self.dev)
        self.loss = t.zeros(1, dtype=t.float64, device=self.dev)
        self.nfluid = t.zeros(1, dtype=t.float64, device=self.dev)
        self.nf = 0.0
        self.dy = f32(0, 16)  # gradient of the loss w.r.t. the head output
        self.dskip = {"c0b": f32(0, 16), "c1b": f32(1, 32)}
        # partial sums of the weight gradients (deterministic, summed in chunk order)
        nwp = max(self.L.lc_nn_wgrad_partial_floats(S >> lvl, S >> lvl, S >> lvl, cin, cout, taps)
                  for _, cin, cout, taps, _, lvl in LAYERS)
        self.wpart = t.empty(nwp, dtype=t.float32, device=self.dev)

    def _cast(self, a, b):
        _ok(self.L.lc_nn_cast_bf16(_p(a), _p(b), a.numel(), self.sp), "cast")

    def _dims(self, lvl):
        s = self.S >> lvl
        return s, s, s

    def n_params(self) -> int:
        return sum(P["w"].numel() + P["b"].numel() for P in self.params.values())

    # -- forward ---------------------------------------------------------------
    def _conv(self, name, src):
        _, cin, cout, taps, relu, lvl = next(x for x in LAYERS if x[0] == name)
        P = self.params[name]
        W, H, D = self._dims(lvl)
        out16 = self.a[name] if name != "head" else None
        out32 = self.y if name == "head" else None
        _ok(self.L.lc_nn_conv3d_fwd(_p(src), _p(P["w16"]), _p(P["b"]), _p(out32) if out32 is not None else None,
                                    _p(out16) if out16 is not None else None, W, H, D, cin, cout, taps, relu, self.sp),
            f"conv {name}")

    def set_input(self, solid, q, R, pitch, w):
        """solid ([S^3] FP64, -1 fluid) and q ([5][S^3] FP64): device tensors."""
        self.nfluid.zero_()
        _ok(self.L.lc_nn_pack_input(_p(solid), _p(q), float(R), float(pitch), float(w), _p(self.a["x"]),
                                    _p(self.base), _p(self.fluid), _p(self.nfluid), self.S**3, CPAD, self.sp), "pack")
        self.nf = float(self.nfluid.item())

    def forward(self):
        S, a, L, sp = self.S, self.a, self.L, self.sp
        self._conv("c0a", a["x"])
        self._conv("c0b", a["c0a"])
        _ok(L.lc_nn_pool2(_p(a["c0b"]), _p(a["p0"]), S, 16, sp), "pool")
        self._conv("c1a", a["p0"])
        self._conv("c1b", a["c1a"])
        _ok(L.lc_nn_pool2(_p(a["c1b"]), _p(a["p1"]), S // 2, 32, sp), "pool")
        self._conv("c2a", a["p1"])
        self._conv("c2b", a["c2a"])
        _ok(L.lc_nn_up2_concat(_p(a["c2b"]), _p(a["c1b"]), _p(a["u1"]), S // 2, 48, 32, sp), "up")
        self._conv("c3", a["u1"])
        _ok(L.lc_nn_up2_concat(_p(a["c3"]), _p(a["c0b"]), _p(a["u0"]), S, 32, 16, sp), "up")
        self._conv("c4", a["u0"])
        self._conv("head", a["c4"])

    def loss_and_grad(self, target_q=None, grad=True, coarse=None) -> float:
        """Masked MSE of Q_init + y[:, :5] against the target (set with set_target).
        ``coarse = (b, weight)`` adds weight x the same error averaged over cubes
        of b^3 nodes (lc_nn_mse_coarse), which weights the long-wavelength part
        of the error by up to b^3 relative to node-scale noise."""
        nf = self.nf
        self.loss.zero_()
        inv = 1.0 / max(nf * 5.0, 1.0)
        _ok(self.L.lc_nn_mse(_p(self.y), _p(self.base), _p(self.target), _p(self.fluid),
                             _p(self.dy) if grad else None, _p(self.loss), self.S**3, 16, inv, self.sp), "mse")
        if coarse is not None:
            b, wgt = coarse
            blk = self.torch.empty(((self.S // b)**3 * 5,), dtype=self.torch.float32, device=self.dev)
            _ok(self.L.lc_nn_mse_coarse(_p(self.y), _p(self.base), _p(self.target), _p(self.fluid),
                                        _p(self.dy) if grad else None, _p(self.loss), _p(blk), self.S, int(b), 16,
                                        inv * float(wgt), self.sp), "mse_coarse")
        return float(self.loss.item())

    def set_target(self, q_soa):
        """Target Q as a [5][S^3] FP64 device tensor."""
        _ok(self.L.lc_nn_from_soa(_p(q_soa), _p(self.target), self.S**3, self.sp), "from_soa")

    # -- backward --------------------------------------------------------------
    def _layer_bwd(self, name, src, dout32, need_din, din32=None):
        """dout32: FP32 gradient w.r.t. the layer's output (n x cout, post-activation)."""
        _, cin, cout, taps, relu, lvl = next(x for x in LAYERS if x[0] == name)
        P, L, sp, t = self.params[name], self.L, self.sp, self.torch
        W, H, D = self._dims(lvl)
        n = W * H * D
        dz16 = t.empty((n, cout), dtype=t.bfloat16, device=self.dev)
        if relu:
            dz32 = t.empty((n, cout), dtype=t.float32, device=self.dev)
            _ok(L.lc_nn_relu_bwd(_p(dout32), _p(self.a[name]), _p(dz32), _p(dz16), n * cout, sp), "relu_bwd")
        else:
            dz32 = dout32
            self._cast(dout32, dz16)
        _ok(L.lc_nn_conv3d_wgrad(_p(dz16), _p(src), _p(P["gw"]), _p(self.wpart), W, H, D, cin, cout, taps, sp),
            "wgrad")
        _ok(L.lc_nn_bias_grad(_p(dz32), _p(P["gb"]), n, cout, sp), "bias_grad")
        if need_din:
            _ok(L.lc_nn_conv3d_dgrad(_p(dz16), _p(P["w16"]), _p(P["wt"]), _p(din32), None, W, H, D, cin, cout, taps,
                                     sp), "dgrad")

    def backward(self):
        t, S, a, L, sp = self.torch, self.S, self.a, self.L, self.sp
        for P in self.params.values():
            P["gw"].zero_()
            P["gb"].zero_()
        n0, n1, n2 = S**3, (S // 2)**3, (S // 4)**3
        new = lambda n, c: t.empty((n, c), dtype=t.float32, device=self.dev)  # noqa: E731
        d_c4 = new(n0, 16)
        self._layer_bwd("head", a["c4"], self.dy, True, d_c4)
        d_u0 = new(n0, 48)
        self._layer_bwd("c4", a["u0"], d_c4, True, d_u0)
        d_c3 = new(n1, 32)
        d_c0b = self.dskip["c0b"]
        d_c0b.zero_()
        _ok(L.lc_nn_up2_concat_bwd(_p(d_u0), _p(d_c3), _p(d_c0b), S, 32, 16, sp), "up_bwd")
        d_u1 = new(n1, 80)
        self._layer_bwd("c3", a["u1"], d_c3, True, d_u1)
        d_c2b = new(n2, 48)
        d_c1b = self.dskip["c1b"]
        d_c1b.zero_()
        _ok(L.lc_nn_up2_concat_bwd(_p(d_u1), _p(d_c2b), _p(d_c1b), S // 2, 48, 32, sp), "up_bwd")
        d_c2a = new(n2, 48)
        self._layer_bwd("c2b", a["c2a"], d_c2b, True, d_c2a)
        d_p1 = new(n2, 32)
        self._layer_bwd("c2a", a["p1"], d_c2a, True, d_p1)
        _ok(L.lc_nn_pool2_bwd(_p(d_p1), _p(d_c1b), S // 2, 32, sp), "pool_bwd")
        d_c1a = new(n1, 32)
        self._layer_bwd("c1b", a["c1a"], d_c1b, True, d_c1a)
        d_p0 = new(n1, 16)
        self._layer_bwd("c1a", a["p0"], d_c1a, True, d_p0)
        _ok(L.lc_nn_pool2_bwd(_p(d_p0), _p(d_c0b), S, 16, sp), "pool_bwd")
        d_c0a = new(n0, 16)
        self._layer_bwd("c0b", a["c0a"], d_c0b, True, d_c0a)
        self._layer_bwd("c0a", a["x"], d_c0a, False)

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for P in self.params.values():
            for k in ("w", "b"):
                _ok(self.L.lc_nn_adam(_p(P[k]), _p(P["g" + k]), _p(P["m" + k]), _p(P["v" + k]),
                                      _p(P["w16"]) if k == "w" else None, P[k].numel(), lr, b1, b2, eps,
                                      self.step_count, self.sp), "adam")

    def predict_soa(self):
        """Q = Q_init + y[:, :5] as a [5][S^3] FP64 device tensor."""
        q = self.torch.empty((5, self.S**3), dtype=self.torch.float64, device=self.dev)
        _ok(self.L.lc_nn_to_soa(_p(self.y), _p(self.base), _p(q), self.S**3, 16, self.sp), "to_soa")
        return q

    # -- persistence -------------------------------------------------------------
    def state(self) -> dict:
        return {n: {"w": P["w"].cpu().numpy(), "b": P["b"].cpu().numpy()} for n, P in self.params.items()}

    def load(self, st: dict):
        for n, P in self.params.items():
            P["w"].copy_(self.torch.tensor(st[n]["w"]))
            P["b"].copy_(self.torch.tensor(st[n]["b"]))
            self._cast(P["w"], P["w16"])


def solver_fields(solver, torch):
    """Solid map and Q of a solver as FP64 device tensors (through lc_lb_get_fields)."""
    nz, ny, nx = solver.shape
    solid = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    q = torch.empty((5, nx * ny * nz), dtype=torch.float64, device="cuda")
    solver.get_fields(LC_SOLID, solid)
    solver.get_fields(LC_Q, q)
    return solid, q


def upsample2(q_soa, S, torch, stream=None):
    """Trilinear x2 of a [5][S^3] FP64 device field to [5][(2S)^3]."""
    L = lib()
    out = torch.empty((5, 8 * S**3), dtype=torch.float64, device=q_soa.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    _ok(L.lc_nn_trilinear2(_p(q_soa), _p(out), S, 5, C.c_void_p(s.cuda_stream)), "trilinear2")
    return out
