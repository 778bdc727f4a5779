"""Registration driver: runs the fused iteration (reg_iterate) for a pair.

Everything here is orchestration: buffers are torch tensors on the device, each
iteration is one C-ABI call (two sweeps of sm_103a kernels), the objective of
every iteration is written by the kernels into a device array and read once at
the end, so the loop never synchronises with the host.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import capi


@dataclass
class RegConfig:
    loss: str = "lncc"          # "lncc" or "mi"
    window: int = 7             # LNCC window side
    eps: float = 1e-9           # LNCC epsilon, added to B C (count-normalised moments)
    ants: bool = False          # LNCC gradient with the ANTs approximation (no second box sum)
    mi_hard: bool = False       # MI with the hard-binned approximate histogram estimator
    bins: int = 32              # MI bins
    f_range: tuple | None = None  # MI intensity ranges; default: each image's own (min, max)
    m_range: tuple | None = None
    lam: float = 0.1            # diffusion weight
    lr: float = 0.1             # Adam step size (voxels)
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    moments: str = "f32"        # "f32" or "bf16"
    sigma_grad: float = 0.0     # > 0: Gaussian smoothing of the gradient before each Adam step
    sigma_warp: float = 0.0     # > 0: Gaussian smoothing of the field after each step
    pad: int = capi.REG_PAD_BORDER

    def loss_desc(self, F, M=None):
        if self.loss == "lncc":
            return capi.lncc_desc(self.window, self.eps, ants=self.ants)
        fr = self.f_range if self.f_range is not None else (float(F.min()), float(F.max()))
        if self.m_range is not None:
            mr = self.m_range
        else:
            mr = (float(M.min()), float(M.max())) if M is not None else (0.0, 1.0)
        return capi.mi_desc(fr, mr, self.bins, hard=self.mi_hard)


@dataclass
class RegResult:
    u: torch.Tensor
    sim: np.ndarray           # similarity per iteration (at the iterate before the step)
    R: np.ndarray             # R(u) per iteration
    objective: np.ndarray     # C + lam R per iteration
    ms_per_iter: float
    extra: dict = field(default_factory=dict)


class Registration:
    """Holds the device state of one registration (u ping-pong, Adam moments,
    workspace) so that runs can be continued and timed without reallocation."""

    def __init__(self, F: torch.Tensor, M: torch.Tensor, cfg: RegConfig, u0: torch.Tensor | None = None,
                 affine=None):
        """affine: an optional capi.RegAffine; the deformable field is then
        optimised under the composite transform phi = A p + t + S u (the fused
        iteration of reg_run; with the smoothing regulariser the composite
        loss gradient, the smoothing and Adam run as separate launches)."""
        self._require_device(F)
        self.F, self.M, self.cfg = F.contiguous(), M.contiguous(), cfg
        self.shape = tuple(F.shape)
        self.N = F.numel()
        dev = F.device
        self.loss = cfg.loss_desc(self.F, self.M)
        mt = torch.bfloat16 if cfg.moments == "bf16" else torch.float32
        self.u = [torch.zeros((3,) + self.shape, device=dev), torch.zeros((3,) + self.shape, device=dev)]
        if u0 is not None:
            self.u[0].copy_(u0)
        self.m = torch.zeros((3,) + self.shape, dtype=mt, device=dev)
        self.v = torch.zeros((3,) + self.shape, dtype=mt, device=dev)
        self.ws = capi.workspace(self.loss, self.F)
        self.adam = capi.adam_desc(cfg.lr, cfg.beta1, cfg.beta2, cfg.adam_eps,
                                   capi.REG_BF16 if cfg.moments == "bf16" else capi.REG_F32, float(self.N))
        self.t = 0
        self.affine = affine
        self.smoothing = cfg.sigma_grad > 0.0 or cfg.sigma_warp > 0.0
        self.unfused = self.smoothing
        if self.unfused:
            self.g = torch.empty_like(self.u[0])
            self.tmp = torch.empty_like(self.u[0])
            self.tmp2 = torch.empty_like(self.u[0])
            self.sim1 = torch.zeros(2, dtype=torch.float64, device=dev)  # 16-byte aligned outputs
            self.r1 = torch.zeros(2, dtype=torch.float64, device=dev)

    @staticmethod
    def _require_device(F):
        if F.device.type != "cuda":
            raise ValueError("F and M must be CUDA tensors")

    @property
    def current(self) -> torch.Tensor:
        return self.u[self.t % 2]

    def run(self, iters: int) -> RegResult:
        hist = torch.zeros((iters, 2), dtype=torch.float64, device=self.F.device)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        if not self.unfused and iters > 0:
            # one native call runs all iterations (no host work between them)
            a, b = self.u[self.t % 2], self.u[(self.t + 1) % 2]
            capi.reg_run(self.loss, self.F, self.M, a, b, self.m, self.v, self.cfg.lam, self.adam, self.t, iters,
                         self.ws, pad=self.cfg.pad, obj_hist=hist, affine=self.affine)
            self.t += iters
        for k in range(iters if self.unfused else 0):
            a, b = self.u[self.t % 2], self.u[(self.t + 1) % 2]
            self.t += 1
            # gradient (composite or plain) -> [smooth(sigma_grad)] -> Adam -> [smooth(sigma_warp)]
            if self.affine is not None:
                capi.reg_loss_grad_composite(self.loss, self.F, self.M, self.affine, a, self.ws, pad=self.cfg.pad,
                                             need_affine=False, sim=self.sim1, grad_u=self.g)
            else:
                capi.reg_loss_grad(self.loss, self.F, self.M, a, self.ws, pad=self.cfg.pad, sim=self.sim1,
                                   grad=self.g)
            capi.reg_regularize(a, self.cfg.lam, self.ws, r=self.r1, grad=self.g)
            hist[k, 0] = self.sim1[0]
            hist[k, 1] = self.r1[0]
            g = self.g
            if self.cfg.sigma_grad > 0.0:
                g = capi.reg_smooth_field(self.g, self.cfg.sigma_grad, out=self.tmp2, tmp=self.tmp)
            capi.reg_step(a, b, self.m, self.v, g, self.adam, self.t)
            if self.cfg.sigma_warp > 0.0:
                capi.reg_smooth_field(b, self.cfg.sigma_warp, out=self.tmp2, tmp=self.tmp)
                b.copy_(self.tmp2)
        end.record()
        torch.cuda.synchronize()
        h = hist.cpu().numpy()
        sim, R = h[:, 0], h[:, 1]
        loss = 1.0 - sim if self.cfg.loss == "lncc" else -sim
        return RegResult(u=self.current, sim=sim, R=R, objective=loss + self.cfg.lam * R,
                         ms_per_iter=start.elapsed_time(end) / max(iters, 1))

    def objective(self, u: torch.Tensor | None = None, F=None, M=None) -> dict:
        """Similarity, R and objective at u (default: the current iterate),
        optionally on other images (for example the FP32 pair of a BF16 run)."""
        u = self.current if u is None else u
        F = self.F if F is None else F
        M = self.M if M is None else M
        ws = self.ws if F.dtype == self.F.dtype else capi.workspace(self.loss, F)
        if self.affine is not None:
            sim = capi.reg_loss_grad_composite(self.loss, F, M, self.affine, u, ws, pad=self.cfg.pad, need_u=False,
                                               need_affine=False)[0][:1]
        else:
            sim = capi.reg_loss(self.loss, F, M, u, ws, pad=self.cfg.pad)
        R = capi.reg_regularize(u, 0.0, ws)
        s, r = float(sim.item()), float(R.item())
        c = 1.0 - s if self.cfg.loss == "lncc" else -s
        return dict(sim=s, R=r, objective=c + self.cfg.lam * r)

    def fold_check(self, u: torch.Tensor | None = None) -> dict:
        u = self.current if u is None else u
        mn, nf = capi.reg_jacdet_min(u)
        return dict(min_det=float(mn.item()), n_fold=int(nf.item()))


def register(F, M, cfg: RegConfig, iters: int, u0=None) -> RegResult:
    """Run `iters` fused iterations from u0 (zero by default)."""
    reg = Registration(F, M, cfg, u0)
    t0 = time.perf_counter()
    res = reg.run(iters)
    res.extra.update(reg.fold_check())
    res.extra["wall_s"] = time.perf_counter() - t0
    return res


def register_multiscale(F, M, cfg: RegConfig, scales=(4, 2, 1), iters=(100, 100, 100), u0=None) -> dict:
    """Coarse-to-fine registration (the multi-scale schedules the paper runs
    with): the level of scale s registers the images averaged down by s (2x
    block means, reg_downsample2, repeated), starting from the previous
    level's field upsampled trilinearly with its displacements scaled
    (reg_nn_field_upsample); Adam restarts at every level.  Scales must be
    decreasing powers of two ending at 1 and divide the image size; u0
    (optional) is the initial field on the coarsest level's grid, in its
    voxels.  Returns the full-resolution field, every level's RegResult and
    the device time of the whole schedule (pyramid and upsampling included)."""
    if list(scales)[-1] != 1 or any(a <= b for a, b in zip(scales, scales[1:])):
        raise ValueError("scales must decrease to 1")
    if len(iters) != len(scales):
        raise ValueError("one iteration count per scale")
    coarse = (3,) + tuple(n // scales[0] for n in F.shape)
    if u0 is not None and tuple(u0.shape) != coarse:
        raise ValueError(f"u0 must be the coarsest level's field, shape {coarse}")
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    pyr = {1: (F.contiguous(), M.contiguous())}
    s = 1
    while s < scales[0]:
        f, m = pyr[s]
        pyr[2 * s] = (capi.reg_downsample2(f), capi.reg_downsample2(m))
        s *= 2
    L = capi.nn()
    u, prev, levels = u0, None, []
    for s, it in zip(scales, iters):
        f, m = pyr[s]
        init = None
        if u is not None and prev is not None:
            factor = prev // s
            cz, cy, cx = u.shape[1:]
            init = torch.empty((3,) + tuple(f.shape), dtype=torch.float32, device=f.device)
            capi.nn_check(L.reg_nn_field_upsample(capi.ptr(u), capi.RegDims(cx, cy, cz), factor, capi.ptr(init),
                                                  capi.stream_of(init)), "field_upsample")
        elif u is not None:
            init = u
        r = Registration(f, m, cfg, u0=init)
        res = r.run(it)
        levels.append({"scale": s, "result": res, "shape": tuple(f.shape)})
        u, prev = r.current.clone(), s
    end.record()
    torch.cuda.synchronize()
    return {"u": u, "levels": levels, "ms": start.elapsed_time(end)}


def _centre(shape):
    nz, ny, nx = shape
    return np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])


def affine_about_centre(A, tc, shape):
    """(A, t) of phi(p) = A p + t for the map A (p - c) + c + tc about the
    volume centre c (tc in voxels)."""
    c = _centre(shape)
    A = np.asarray(A, dtype=np.float64)
    return A, c - A @ c + np.asarray(tc, dtype=np.float64)


def centred_affine_grads(gA, gt, c, s):
    """Gradients in the centred parameters of phi(p) = A (p - c) + c + tc / s
    (c the volume centre of the level, s its scale, tc in full-resolution
    voxels) from those in phi(p) = A p + t: since t = c - A c + tc / s,
    dC/dA at fixed tc = dC/dA - (dC/dt) c^T and dC/dtc = (dC/dt) / s."""
    gA = np.asarray(gA, dtype=np.float64).reshape(3, 3)
    gt = np.asarray(gt, dtype=np.float64).reshape(3)
    return gA - np.outer(gt, c), gt / s


def register_affine(F, M, cfg: RegConfig, scales=(4, 2, 1), iters=(100, 60, 40), lr_A: float = 0.01,
                    lr_t: float = 0.3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                    final_lr: float = 0.1, on_device: bool = True) -> dict:
    """Affine stage of the paper's pipeline: phi(p) = A (p - c) + c + tc about
    the volume centre, optimised by Adam over the 12 parameters at each scale
    of a 2x block-mean pyramid, with the similarity and dC/dA, dC/dt from the
    composite sampler (u = 0).  tc is kept in voxels of the full-resolution
    grid; at scale s it is tc / s.  The step sizes decay linearly to final_lr
    of their value over each level: a constant Adam step leaves A jittering by
    about lr_A, a motion of lr_A times the radius at the volume's edge.

    on_device (default): each iteration is two launches -- the composite
    similarity and gradients with the transform read from device memory
    (reg_loss_grad_composite_dev) and the 12-parameter Adam step on the
    device (reg_affine_adam_step), which writes the next transform; the host
    reads the state once per level.  on_device=False runs the same Adam on
    the host (one 112-byte read per iteration).  Returns A, t of the
    full-resolution map (phi = A p + t), tc, and the objective history per
    level."""
    if on_device:
        return _register_affine_device(F, M, cfg, scales, iters, lr_A, lr_t, beta1, beta2, eps, final_lr)
    pyr = {1: (F.contiguous(), M.contiguous())}
    s = 1
    while s < scales[0]:
        f, m = pyr[s]
        pyr[2 * s] = (capi.reg_downsample2(f), capi.reg_downsample2(m))
        s *= 2
    loss = cfg.loss_desc(F, M)
    A = np.eye(3)
    tc = np.zeros(3)
    levels = []
    for s, it in zip(scales, iters):
        f, m = pyr[s]
        shape = tuple(f.shape)
        c = _centre(shape)
        ws = capi.workspace(loss, f)
        buf = torch.zeros(14, dtype=torch.float64, device=f.device)  # sim (2), dC/dA (9), dC/dt (3)
        mA, vA, mt, vt = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros(3), np.zeros(3)
        hist = []
        for k in range(it):
            t = c - A @ c + tc / s
            capi.reg_loss_grad_composite(loss, f, m, capi.affine_desc(A, t), None, ws, pad=cfg.pad, need_u=False,
                                         sim=buf[0:2], grad_affine=buf[2:14])
            h = buf.cpu().numpy()
            sim, gA, gt = h[0], h[2:11].reshape(3, 3), h[11:14]
            hist.append(1.0 - sim if cfg.loss == "lncc" else -sim)
            gA, gtc = centred_affine_grads(gA, gt, c, s)
            b1, b2 = 1.0 - beta1 ** (k + 1), 1.0 - beta2 ** (k + 1)
            decay = 1.0 - (1.0 - final_lr) * k / max(it - 1, 1)
            mA = beta1 * mA + (1 - beta1) * gA
            vA = beta2 * vA + (1 - beta2) * gA * gA
            mt = beta1 * mt + (1 - beta1) * gtc
            vt = beta2 * vt + (1 - beta2) * gtc * gtc
            A = A - decay * lr_A * (mA / b1) / (np.sqrt(vA / b2) + eps)
            tc = tc - decay * lr_t * s * (mt / b1) / (np.sqrt(vt / b2) + eps)
        levels.append({"scale": s, "objective": np.asarray(hist)})
    A_full, t_full = affine_about_centre(A, tc, tuple(F.shape))
    return {"A": A_full, "t": t_full, "tc": tc, "levels": levels}


def _register_affine_device(F, M, cfg, scales, iters, lr_A, lr_t, beta1, beta2, eps, final_lr) -> dict:
    pyr = {1: (F.contiguous(), M.contiguous())}
    s = 1
    while s < scales[0]:
        f, m = pyr[s]
        pyr[2 * s] = (capi.reg_downsample2(f), capi.reg_downsample2(m))
        s *= 2
    loss = cfg.loss_desc(F, M)
    dev = F.device
    state = torch.zeros(36, dtype=torch.float64, device=dev)  # A, tc, m_A, v_A, m_t, v_t
    state[0:9] = torch.eye(3, dtype=torch.float64, device=dev).reshape(9)
    T = torch.zeros(15, dtype=torch.float32, device=dev)
    buf = torch.zeros(14, dtype=torch.float64, device=dev)  # sim (2), dC/dA (9), dC/dt (3)
    kind = capi.REG_LOSS_LNCC if cfg.loss == "lncc" else capi.REG_LOSS_MI
    levels = []
    for s, it in zip(scales, iters):
        f, m = pyr[s]
        shape = tuple(f.shape)
        c = _centre(shape)
        ws = capi.workspace(loss, f)
        st = state.cpu().numpy()  # A and tc carried over from the previous level (one read per level)
        A, tc = st[0:9].reshape(3, 3), st[9:12]
        state[12:36] = 0.0  # fresh moments for the level
        t0 = c - A @ c + tc / s
        T.copy_(torch.tensor(np.concatenate([A.reshape(9), t0, np.ones(3)]), dtype=torch.float32))
        desc = capi.affine_adam_desc(lr_A, lr_t, it, s, c, kind, beta1, beta2, eps, final_lr)
        hist = torch.zeros((it, 2), dtype=torch.float64, device=dev)  # 16-byte rows: every entry aligned
        for k in range(it):
            capi.reg_loss_grad_composite_dev(loss, f, m, T, None, ws, pad=cfg.pad, need_u=False, sim=buf[0:2],
                                             grad_affine=buf[2:14])
            capi.reg_affine_adam_step(buf[2:14], buf[0:1], state, T, desc, k, obj=hist[k])
        levels.append({"scale": s, "objective": hist[:, 0].cpu().numpy()})
    st = state.cpu().numpy()
    A, tc = st[0:9].reshape(3, 3), st[9:12]
    A_full, t_full = affine_about_centre(A, tc, tuple(F.shape))
    return {"A": A_full, "t": t_full, "tc": tc, "levels": levels}


def register_svf(F, M, cfg: RegConfig, iters: int, steps: int = 6, v0=None) -> dict:
    """Diffeomorphic registration on a stationary velocity field v: each
    iteration forms u = exp(v) by scaling and squaring on the fused sampler
    (reg_exp_field, keeping the intermediate fields), takes the similarity
    gradient dC/du (reg_loss_grad), pulls it back through every squaring step
    (reg_exp_field_backward), adds lam * dR/dv of the diffusion term on v
    (reg_regularize) and steps v with Adam (reg_step).  Returns v, u = exp(v),
    the objective history (C(u) + lam R(v)) and the device time per
    iteration."""
    F, M = F.contiguous(), M.contiguous()
    shape = tuple(F.shape)
    dev = F.device
    loss = cfg.loss_desc(F, M)
    ws = capi.workspace(loss, F)
    v = [torch.zeros((3,) + shape, device=dev), torch.zeros((3,) + shape, device=dev)]
    if v0 is not None:
        v[0].copy_(v0)
    m = torch.zeros_like(v[0])
    s2 = torch.zeros_like(v[0])
    u = torch.empty_like(v[0])
    gu = torch.empty_like(v[0])
    gv = torch.empty_like(v[0])
    tmp = torch.empty_like(v[0])
    saved = torch.empty((max(steps - 1, 1), 3) + shape, device=dev)
    adam = capi.adam_desc(cfg.lr, cfg.beta1, cfg.beta2, cfg.adam_eps, capi.REG_F32, float(F.numel()))
    sim = torch.zeros((iters, 2), dtype=torch.float64, device=dev)
    r = torch.zeros((iters, 2), dtype=torch.float64, device=dev)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for k in range(iters):
        a, b = v[k % 2], v[(k + 1) % 2]
        capi.reg_exp_field(a, steps, cfg.pad, out=u, saved=saved)
        capi.reg_loss_grad(loss, F, M, u, ws, pad=cfg.pad, sim=sim[k], grad=gu)
        capi.reg_exp_field_backward(a, steps, gu, saved=saved, pad=cfg.pad, gv=gv, tmp=tmp)
        capi.reg_regularize(a, cfg.lam, ws, r=r[k], grad=gv)
        capi.reg_step(a, b, m, s2, gv, adam, k + 1)
    end.record()
    torch.cuda.synchronize()
    vf = v[iters % 2]
    capi.reg_exp_field(vf, steps, cfg.pad, out=u, saved=saved)
    h, hr = sim.cpu().numpy()[:, 0], r.cpu().numpy()[:, 0]
    c = 1.0 - h if cfg.loss == "lncc" else -h
    return {"v": vf, "u": u, "objective": c + cfg.lam * hr, "sim": h,
            "ms_per_iter": start.elapsed_time(end) / max(iters, 1)}
