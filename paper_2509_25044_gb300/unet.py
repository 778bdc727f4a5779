"""Learned initialiser: a small 3-D U-Net that maps a downsampled (F, M) pair
to a half-resolution initial displacement for the registration.

Network (channels 16-32-64-64, two 3x3x3 convolutions per level, LeakyReLU
0.2, 2x average pooling down, 2x trilinear upsampling + channel concat up):

    128^3 x 16 (F, M, zeros) --c0a,c0b--> e0 16 --pool--> 64^3
      --c1a,c1b--> e1 32 --pool--> 32^3 --c2a,c2b--> e2 64 --pool--> 16^3
      --c3a,c3b--> b3 64 --up--> 32^3 [64 | e2 64] --d2a,d2b--> d2 64
      --up--> 64^3 [64 | e1 32] --d1a,d1b--> d1 32 --head--> u 3 @ 64^3

Every operator is a library kernel through the C ABI (reg_nn_*): the
convolutions (forward, data and weight gradients) run on the tcgen05 tensor
cores; torch only holds the buffers.  Training pairs are made with the
library's own warp: F = M o (id + v_true) for a random smooth v_true, so the
target is v_true itself (pooled to 64^3, in 64^3 voxel units).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import capi, synth

SLOPE = 0.2
BF = torch.bfloat16

# (name, Cin, Cout, grid level)  level 0 = 128^3 ... 3 = 16^3
LAYERS = [
    ("c0a", 16, 16, 0), ("c0b", 16, 16, 0),
    ("c1a", 16, 32, 1), ("c1b", 32, 32, 1),
    ("c2a", 32, 64, 2), ("c2b", 64, 64, 2),
    ("c3a", 64, 64, 3), ("c3b", 64, 64, 3),
    ("d2a", 128, 64, 2), ("d2b", 64, 64, 2),
    ("d1a", 96, 32, 1), ("d1b", 32, 32, 1),
    ("head", 32, 3, 1),
]


def _dims(n):
    return capi.RegDims(n, n, n)


@dataclass
class Param:
    cin: int
    cout: int
    rows: int
    kpad: int
    w: torch.Tensor       # FP32 master [rows][kpad]
    wb: torch.Tensor      # BF16 copy used by the kernels
    b: torch.Tensor       # FP32 bias [rows]
    gw: torch.Tensor
    gb: torch.Tensor
    mw: torch.Tensor
    vw: torch.Tensor
    mb: torch.Tensor
    vb: torch.Tensor


class UNet:
    def __init__(self, n_in: int = 128, seed: int = 0, device="cuda"):
        self.L = capi.nn()
        self.dev = torch.device(device)
        self.n = [n_in, n_in // 2, n_in // 4, n_in // 8]
        self.V = [k ** 3 for k in self.n]
        rng = np.random.default_rng(seed)
        self.p = {}
        for name, cin, cout, _ in LAYERS:
            kpad = int(self.L.reg_nn_conv_kpad(cin))
            rows = (cout + 15) // 16 * 16
            w = np.zeros((rows, kpad), dtype=np.float32)
            real_cin = 2 if name == "c0a" else cin  # the input has 2 real channels (F, M)
            std = math.sqrt(2.0 / (1.0 + SLOPE ** 2) / (27 * real_cin))
            if name == "head":
                std *= 0.1  # start near the zero displacement
            blk = rng.standard_normal((cout, 27, real_cin)).astype(np.float32) * std
            wv = w[:cout, :27 * cin].reshape(cout, 27, cin)
            wv[:, :, :real_cin] = blk
            t = torch.from_numpy(w).to(self.dev)
            z = lambda shape: torch.zeros(shape, dtype=torch.float32, device=self.dev)
            self.p[name] = Param(cin, cout, rows, kpad, t, t.to(BF).contiguous(), z(rows), z((rows, kpad)), z(rows),
                                 z((rows, kpad)), z((rows, kpad)), z(rows), z(rows))
        self.t = 0
        self._alloc()

    # ---- buffers -------------------------------------------------------------
    def _act(self, level, C):
        return torch.empty((self.V[level], C), dtype=BF, device=self.dev)

    def _alloc(self):
        a = {}
        a["x0"] = self._act(0, 16)
        a["c0a"], a["e0"] = self._act(0, 16), self._act(0, 16)
        a["p0"] = self._act(1, 16)
        a["c1a"], a["e1"] = self._act(1, 32), self._act(1, 32)
        a["p1"] = self._act(2, 32)
        a["c2a"], a["e2"] = self._act(2, 64), self._act(2, 64)
        a["p2"] = self._act(3, 64)
        a["c3a"], a["b3"] = self._act(3, 64), self._act(3, 64)
        a["cat2"] = self._act(2, 128)
        a["d2a"], a["d2"] = self._act(2, 64), self._act(2, 64)
        a["cat1"] = self._act(1, 96)
        a["d1a"], a["d1"] = self._act(1, 32), self._act(1, 32)
        a["u"] = torch.empty((3, self.V[1]), dtype=torch.float32, device=self.dev)
        self.a = a
        g = {}
        for k, t in a.items():
            if k not in ("x0", "u"):
                g[k] = torch.empty_like(t)
        g["pre"] = torch.empty((self.V[0], 128), dtype=BF, device=self.dev).view(-1)  # leaky-backward scratch
        g["dpred"] = torch.empty((self.V[1], 16), dtype=BF, device=self.dev)
        g["up"] = torch.empty((self.V[2], 64), dtype=BF, device=self.dev)  # upsample-backward outputs
        self.g = g
        cs = max(int(self.L.reg_nn_conv_scratch_bytes(cin, cout)) for _, cin, cout, _ in LAYERS)
        self.cs = torch.empty(max(cs, 16), dtype=torch.uint8, device=self.dev)
        wd = max(int(self.L.reg_nn_dgrad_scratch_bytes(cin, cout)) for _, cin, cout, _ in LAYERS)
        self.wd = torch.empty(wd, dtype=torch.uint8, device=self.dev)
        wg = max(int(self.L.reg_nn_wgrad_scratch_bytes(_dims(self.n[lv]), cin, (cout + 15) // 16 * 16))
                 for _, cin, cout, lv in LAYERS)
        self.wg = torch.empty(wg, dtype=torch.uint8, device=self.dev)
        self.bg = torch.empty(int(self.L.reg_nn_bias_grad_scratch_bytes(64)), dtype=torch.uint8, device=self.dev)
        self.ms = torch.empty(int(self.L.reg_nn_mse_scratch_bytes()), dtype=torch.uint8, device=self.dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)

    # ---- helpers --------------------------------------------------------------
    def _s(self):
        return capi.stream_of(self.a["x0"])

    def _conv(self, name, src, dst, level, epi=0):
        P = self.p[name]
        capi.nn_check(self.L.reg_nn_conv3d_fwd(capi.ptr(src), P.cin, capi.ptr(P.wb), capi.ptr(P.b), P.cout,
                                               _dims(self.n[level]), epi, SLOPE, capi.ptr(self.cs), self.cs.numel(),
                                               capi.ptr(dst), self._s()),
                      f"conv {name}")

    def _pool(self, src, C, level, dst, backward=0):
        capi.nn_check(self.L.reg_nn_avgpool2(capi.ptr(src), C, _dims(self.n[level]), capi.ptr(dst), backward,
                                             self._s()), "avgpool2")

    def _up(self, src, C, level_coarse, dst, backward=0):
        capi.nn_check(self.L.reg_nn_upsample2(capi.ptr(src), C, _dims(self.n[level_coarse]), capi.ptr(dst), backward,
                                              self._s()), "upsample2")

    def _put(self, src, Cs, V, dst, Cd, c0, acc=0):
        capi.nn_check(self.L.reg_nn_put_channels(capi.ptr(src), Cs, V, capi.ptr(dst), Cd, c0, acc, self._s()), "put")

    def _take(self, src, Cs, c0, V, dst, Cd, acc=0):
        capi.nn_check(self.L.reg_nn_take_channels(capi.ptr(src), Cs, c0, V, capi.ptr(dst), Cd, acc, self._s()),
                      "take")

    # ---- forward --------------------------------------------------------------
    def pack(self, F, M, factor: int, f_range, m_range):
        d = capi.dims_of(F)
        capi.nn_check(self.L.reg_nn_pack_pair(capi.ptr(F), capi.ptr(M), capi._img_dtype(F), d, factor,
                                              float(f_range[0]), float(f_range[1]), float(m_range[0]),
                                              float(m_range[1]), capi.ptr(self.a["x0"]), self._s()), "pack_pair")

    def forward(self) -> torch.Tensor:
        a, V = self.a, self.V
        self._conv("c0a", a["x0"], a["c0a"], 0)
        self._conv("c0b", a["c0a"], a["e0"], 0)
        self._pool(a["e0"], 16, 0, a["p0"])
        self._conv("c1a", a["p0"], a["c1a"], 1)
        self._conv("c1b", a["c1a"], a["e1"], 1)
        self._pool(a["e1"], 32, 1, a["p1"])
        self._conv("c2a", a["p1"], a["c2a"], 2)
        self._conv("c2b", a["c2a"], a["e2"], 2)
        self._pool(a["e2"], 64, 2, a["p2"])
        self._conv("c3a", a["p2"], a["c3a"], 3)
        self._conv("c3b", a["c3a"], a["b3"], 3)
        up2 = self.g["up"][:V[2]]
        self._up(a["b3"], 64, 3, up2)
        self._put(up2, 64, V[2], a["cat2"], 128, 0)
        self._put(a["e2"], 64, V[2], a["cat2"], 128, 64)
        self._conv("d2a", a["cat2"], a["d2a"], 2)
        self._conv("d2b", a["d2a"], a["d2"], 2)
        up1 = torch.empty((V[1], 64), dtype=BF, device=self.dev) if not hasattr(self, "_up1") else self._up1
        self._up1 = up1
        self._up(a["d2"], 64, 2, up1)
        self._put(up1, 64, V[1], a["cat1"], 96, 0)
        self._put(a["e1"], 32, V[1], a["cat1"], 96, 64)
        self._conv("d1a", a["cat1"], a["d1a"], 1)
        self._conv("d1b", a["d1a"], a["d1"], 1)
        self._conv("head", a["d1"], a["u"], 1, epi=2)
        return a["u"]

    # ---- backward -------------------------------------------------------------
    def _layer_bwd(self, name, x, out, dout, level, dx=None):
        """dout: gradient of the layer output (post-activation for leaky layers,
        FP32-head gradient already as dpre for the head); fills P.gw, P.gb and
        (optionally) dx."""
        P = self.p[name]
        V = self.V[level]
        if name == "head":
            dpre, cpre = dout, 16
        else:
            dpre = self.g["pre"][:V * P.cout].view(V, P.cout)
            capi.nn_check(self.L.reg_nn_leaky_bwd(capi.ptr(out), capi.ptr(dout), V * P.cout, SLOPE, capi.ptr(dpre),
                                                  self._s()), "leaky_bwd")
            cpre = P.cout
        capi.nn_check(self.L.reg_nn_conv3d_wgrad(capi.ptr(x), P.cin, capi.ptr(dpre), cpre, _dims(self.n[level]),
                                                 capi.ptr(self.wg), self.wg.numel(), capi.ptr(P.gw), self._s()),
                      f"wgrad {name}")
        capi.nn_check(self.L.reg_nn_bias_grad(capi.ptr(dpre), V, cpre, capi.ptr(self.bg), capi.ptr(P.gb),
                                              self._s()), f"bias grad {name}")
        if dx is not None:
            capi.nn_check(self.L.reg_nn_conv3d_dgrad(capi.ptr(dpre), cpre, capi.ptr(P.wb), P.cin,
                                                     _dims(self.n[level]), capi.ptr(self.wd), capi.ptr(dx),
                                                     self._s()), f"dgrad {name}")

    def loss_and_backward(self, target: torch.Tensor) -> torch.Tensor:
        """MSE to the target field (SoA FP32 [3][64^3]) and all parameter gradients."""
        a, g, V = self.a, self.g, self.V
        capi.nn_check(self.L.reg_nn_mse(capi.ptr(a["u"]), capi.ptr(target), V[1], 16, capi.ptr(g["dpred"]),
                                        capi.ptr(self.ms), capi.ptr(self.loss), self._s()), "mse")
        self._layer_bwd("head", a["d1"], None, g["dpred"], 1, dx=g["d1"])
        self._layer_bwd("d1b", a["d1a"], a["d1"], g["d1"], 1, dx=g["d1a"])
        self._layer_bwd("d1a", a["cat1"], a["d1a"], g["d1a"], 1, dx=g["cat1"])
        up1 = self._up1
        self._take(g["cat1"], 96, 0, V[1], up1, 64)
        self._take(g["cat1"], 96, 64, V[1], g["e1"], 32)          # skip part of de1
        self._up(up1, 64, 2, g["d2"], backward=1)
        self._layer_bwd("d2b", a["d2a"], a["d2"], g["d2"], 2, dx=g["d2a"])
        self._layer_bwd("d2a", a["cat2"], a["d2a"], g["d2a"], 2, dx=g["cat2"])
        up2 = g["up"][:V[2]]
        self._take(g["cat2"], 128, 0, V[2], up2, 64)
        self._take(g["cat2"], 128, 64, V[2], g["e2"], 64)          # skip part of de2
        self._up(up2, 64, 3, g["b3"], backward=1)
        self._layer_bwd("c3b", a["c3a"], a["b3"], g["b3"], 3, dx=g["c3a"])
        self._layer_bwd("c3a", a["p2"], a["c3a"], g["c3a"], 3, dx=g["p2"])
        tmp2 = g["cat2"].view(-1)[:V[2] * 64].view(V[2], 64)       # cat2 gradient no longer needed
        self._pool(g["p2"], 64, 2, tmp2, backward=1)
        self._put(tmp2, 64, V[2], g["e2"], 64, 0, acc=1)
        self._layer_bwd("c2b", a["c2a"], a["e2"], g["e2"], 2, dx=g["c2a"])
        self._layer_bwd("c2a", a["p1"], a["c2a"], g["c2a"], 2, dx=g["p1"])
        tmp1 = g["cat1"].view(-1)[:V[1] * 32].view(V[1], 32)
        self._pool(g["p1"], 32, 1, tmp1, backward=1)
        self._put(tmp1, 32, V[1], g["e1"], 32, 0, acc=1)
        self._layer_bwd("c1b", a["c1a"], a["e1"], g["e1"], 1, dx=g["c1a"])
        self._layer_bwd("c1a", a["p0"], a["c1a"], g["c1a"], 1, dx=g["p0"])
        self._pool(g["p0"], 16, 0, g["e0"], backward=1)
        self._layer_bwd("c0b", a["c0a"], a["e0"], g["e0"], 0, dx=g["c0a"])
        self._layer_bwd("c0a", a["x0"], a["c0a"], g["c0a"], 0, dx=None)
        return self.loss

    def step(self, lr: float = 1e-3):
        self.t += 1
        ad = capi.adam_desc(lr, 0.9, 0.999, 1e-8)
        for P in self.p.values():
            capi.nn_check(self.L.reg_nn_adam(capi.ptr(P.w), capi.ptr(P.mw), capi.ptr(P.vw), capi.ptr(P.gw),
                                             P.w.numel(), capi.ctypes.byref(ad), self.t, capi.ptr(P.wb), self._s()),
                          "adam w")
            capi.nn_check(self.L.reg_nn_adam(capi.ptr(P.b), capi.ptr(P.mb), capi.ptr(P.vb), capi.ptr(P.gb),
                                             P.b.numel(), capi.ctypes.byref(ad), self.t, None, self._s()), "adam b")

    # ---- inference: initial field at the registration grid ---------------------
    def predict_init(self, F, M, f_range, m_range) -> torch.Tensor:
        """u0 for a pair of size n (n a multiple of the network input size):
        average-pool to the input grid, scale each image by its range on that
        grid (f_range, m_range are the ranges at n^3), run the network,
        upsample the 64^3 output to n^3 and rescale it to n^3 voxel units."""
        n = F.shape[0]
        factor = n // self.n[0]
        self.pack(F, M, factor, f_range, m_range)
        if factor > 1:
            # the network learned on images scaled by the range of the grid it
            # sees; pooling narrows that range (the noise averages out), so
            # measure it on the pooled grid (channels in units of the given
            # ranges) and pack again
            lo, hi = torch.aminmax(self.a["x0"][:, :2].float(), dim=0)
            lo, hi = lo.tolist(), hi.tolist()
            fw, mw = f_range[1] - f_range[0], m_range[1] - m_range[0]
            self.pack(F, M, factor, (f_range[0] + lo[0] * fw, f_range[0] + hi[0] * fw),
                      (m_range[0] + lo[1] * mw, m_range[0] + hi[1] * mw))
        u_half = self.forward()
        up = n // self.n[1]
        out = torch.empty((3,) + tuple(F.shape), dtype=torch.float32, device=self.dev)
        capi.nn_check(self.L.reg_nn_field_upsample(capi.ptr(u_half), _dims(self.n[1]), up, capi.ptr(out), self._s()),
                      "field_upsample")
        return out


def multimodal_training_pair(n: int, seed: int, device, noise: float = 0.03, smooth: float = 1.0) -> dict:
    """One multi-modal training pair at n^3 (the MI workloads' phantoms): a
    6-label ellipsoid map painted twice, through two intensity tables that
    are not monotone in each other, each with N(0, noise^2) and Gaussian
    smoothing at `smooth` (synth.label_images); a random smooth field v_true
    (sigma ~ U[4,12], max |v| ~ U(0,10]); F = F0 o (id + v_true) with the
    library's warp and M the second painting, aligned with F0, so that
    registering M onto F recovers v_true itself.  Random numbers come from
    torch's Philox generator on the device, seeded with `seed`."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    F0, M = synth.label_images((n, n, n), 6, noise, smooth, gen=gen, device=device)
    u01 = torch.rand(2, generator=gen, device=device, dtype=torch.float64).cpu().numpy()
    sigma = 4.0 + 8.0 * float(u01[0])
    mx = 10.0 * (1.0 - float(u01[1]))  # in (0, 10]
    v = synth.smooth_field((n, n, n), sigma, mx, gen=gen, device=device)
    F = capi.reg_warp(F0.contiguous(), v)
    return dict(F=F, M=M.contiguous(), v=v)


def training_pair(n: int, seed: int, device, noise: float = 0.02) -> dict:
    """One training pair at n^3 made with the library's own warp: a blob
    image B (sigma scaled to the grid) with N(0, noise^2) noise as M, a random
    smooth field v_true (sigma ~ U[4,12], max |v| ~ U(0,10]) and F = M o (id +
    v_true), so that v_true is the displacement the registration of M onto F
    recovers (the noise is part of the texture and moves with it, as in the
    mono-modal workloads).  noise = 0.02 is the workloads' acquisition noise
    at the grid itself; a pair that the network sees after 4^3 average
    pooling (the 512^3 workload at 128^3) carries 0.02 / 8.  Random numbers
    come from torch's Philox generator on the device, seeded with `seed`."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    s = n / 64.0
    B = synth.blobs((n, n, n), 40, (2.0 * s, 8.0 * s), noise_std=0.0, gen=gen, device=device)
    u01 = torch.rand(2, generator=gen, device=device, dtype=torch.float64).cpu().numpy()
    sigma = 4.0 + 8.0 * float(u01[0])
    mx = 10.0 * (1.0 - float(u01[1]))  # in (0, 10]
    v = synth.smooth_field((n, n, n), sigma, mx, gen=gen, device=device)
    M = B.add_(torch.randn((n, n, n), generator=gen, device=device, dtype=torch.float32), alpha=noise)
    F = capi.reg_warp(M, v)
    return dict(F=F, M=M, v=v)
