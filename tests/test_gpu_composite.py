"""GPU parity of the composite implicit grid sampler phi(p) = A p + t + S u(p)
(Sec. 2.1; Algorithm gridsampler, forward and backward) and of the losses
and their A, t, u gradients under it, against the FP64 oracle on the same
seeded inputs."""
import numpy as np
import pytest
import torch

import oracle as O
from _util import GRAD_RTOL, LOSS_RTOL, WARP_TOL, assert_rel, bf16_values, field, mono_images, \
    multimodal_images, rel_l2, to64

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def _affine(shape, seed, angle=0.05, shift=(1.2, -0.7, 0.4), s=(1.0, 1.0, 1.0)):
    """A small rotation about z, anisotropic scale and shear about the volume
    centre, plus a shift; returned as the FP32 values the descriptor holds."""
    rng = np.random.default_rng(seed)
    c, sn = np.cos(angle), np.sin(angle)
    R = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
    A = R @ (np.diag([1.03, 0.98, 1.01]) + 0.01 * rng.standard_normal((3, 3)))
    ctr = np.array([(shape[2] - 1) / 2, (shape[1] - 1) / 2, (shape[0] - 1) / 2])
    t = ctr - A @ ctr + np.asarray(shift)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return f32(A), f32(t), f32(s)


def _desc(capi, A, t, s):
    return capi.affine_desc(A, t, s)


def _img(t, dtype):
    return t.to(DEV).to(dtype).contiguous()


def _oimg(t, dtype):
    return to64(bf16_values(t) if dtype == torch.bfloat16 else t)


@pytest.mark.parametrize("shape", [(20, 18, 40), (1, 7, 50), (9, 33, 31)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("pad", [0, 1])
@pytest.mark.parametrize("with_u", [False, True])
def test_warp_composite_matches_oracle(capi, shape, dtype, pad, with_u):
    F, M = mono_images(shape, 3)
    u = field(shape, 3.0, 1.5, 4) if with_u else None
    A, t, s = _affine(shape, 5, s=(1.2, 0.9, 1.0))
    T = _desc(capi, A, t, s)
    J, dJ = capi.reg_warp_composite(_img(M, dtype), T, None if u is None else u.to(DEV), pad=pad, with_slope=True)
    torch.cuda.synchronize()
    Jr, dJr = O.warp_composite(_oimg(M, dtype), A, t, s, None if u is None else to64(u), pad, with_grad=True)
    rng = float(M.max() - M.min())
    assert np.abs(to64(J) - Jr).max() <= WARP_TOL * rng
    assert rel_l2(to64(dJ), dJr) <= GRAD_RTOL


def test_identity_composite_is_plain_warp(capi):
    shape = (12, 10, 36)
    _, M = mono_images(shape, 7)
    u = field(shape, 3.0, 2.0, 8).to(DEV)
    I = capi.affine_desc()
    J0, d0 = capi.reg_warp(M.to(DEV), u, with_slope=True)
    J1, d1 = capi.reg_warp_composite(M.to(DEV), I, u, with_slope=True)
    torch.cuda.synchronize()
    assert torch.equal(J0, J1) and torch.equal(d0, d1)


@pytest.mark.parametrize("shape", [(20, 18, 40), (5, 40, 33)])
@pytest.mark.parametrize("pad", [0, 1])
def test_composite_backward_matches_oracle(capi, shape, pad):
    _, M = mono_images(shape, 11)
    u = field(shape, 3.0, 1.5, 12)
    g = torch.from_numpy(np.random.default_rng(13).standard_normal(shape).astype(np.float32))
    A, t, s = _affine(shape, 14, s=(0.8, 1.1, 1.3))
    T = _desc(capi, A, t, s)
    g_u, ga = capi.reg_warp_composite_backward(M.to(DEV), T, g.to(DEV), u.to(DEV), pad=pad)
    torch.cuda.synchronize()
    gur, gAr, gtr = O.sampler_backward_composite(to64(M), A, t, s, to64(u), to64(g), pad)
    assert rel_l2(to64(g_u), gur) <= GRAD_RTOL
    ga = to64(ga)
    assert rel_l2(ga[:9], gAr.ravel()) <= GRAD_RTOL
    assert rel_l2(ga[9:], gtr) <= GRAD_RTOL
    # the affine part alone (u omitted) and without g_u
    _, ga0 = capi.reg_warp_composite_backward(M.to(DEV), T, g.to(DEV), None, pad=pad, need_u=False)
    torch.cuda.synchronize()
    _, gA0, gt0 = O.sampler_backward_composite(to64(M), A, t, s, None, to64(g), pad)
    assert rel_l2(to64(ga0), np.concatenate([gA0.ravel(), gt0])) <= GRAD_RTOL


def _loss(capi, kind, F, M):
    if kind.startswith("lncc"):
        ants = kind == "lncc_ants"
        return (capi.lncc_desc(5, 1e-4, ants=ants),
                O.LossSpec(kind=O.LOSS_LNCC, window=5, eps=1e-4, lncc_grad=1 if ants else 0))
    fr = (float(F.min()), float(F.max()))
    mr = (float(M.min()), float(M.max()))
    hard = kind == "mi_hard"
    # as in the plain MI parity tests: 16 bins below 4096 voxels, where a
    # sparsely filled 32 x 32 histogram makes the FP32 adjoint table rough
    # (the FP32 rounding of phi itself moves the oracle's gradient by ~1e-6)
    bins = 32 if F.numel() >= 4096 else 16
    return (capi.mi_desc(fr, mr, bins, hard=hard),
            O.LossSpec(kind=O.LOSS_MI, bins=bins, f_range=fr, m_range=mr, mi_estimator=1 if hard else 0))


@pytest.mark.parametrize("kind", ["lncc", "lncc_ants", "mi", "mi_hard"])
@pytest.mark.parametrize("shape", [(18, 20, 40), (3, 9, 70)])
@pytest.mark.parametrize("pad", [0, 1])
@pytest.mark.parametrize("with_u", [False, True])
def test_loss_grad_composite_matches_oracle(capi, kind, shape, pad, with_u):
    F, M = (mono_images if kind.startswith("lncc") else multimodal_images)(shape, 21)
    u = field(shape, 3.0, 1.5, 22) if with_u else None
    A, t, s = _affine(shape, 23, s=(1.0, 1.1, 0.9))
    T = _desc(capi, A, t, s)
    loss, spec = _loss(capi, kind, F, M)
    sim, gu, ga = capi.reg_loss_grad_composite(loss, F.to(DEV), M.to(DEV), T, None if u is None else u.to(DEV),
                                               pad=pad)
    torch.cuda.synchronize()
    Sr, gur, gAr, gtr = O.similarity_and_grad_composite(to64(F), to64(M), A, t, s, None if u is None else to64(u),
                                                        spec, pad)
    assert_rel(sim[0].item(), Sr, LOSS_RTOL, "similarity")
    assert rel_l2(to64(gu), gur) <= GRAD_RTOL
    ga = to64(ga)
    assert rel_l2(ga[:9], gAr.ravel()) <= GRAD_RTOL, (ga[:9], gAr.ravel())
    assert rel_l2(ga[9:], gtr) <= GRAD_RTOL, (ga[9:], gtr)
    # similarity alone
    sim0, _, _ = capi.reg_loss_grad_composite(loss, F.to(DEV), M.to(DEV), T, None if u is None else u.to(DEV),
                                              pad=pad, need_u=False, need_affine=False)
    torch.cuda.synchronize()
    assert_rel(sim0[0].item(), Sr, LOSS_RTOL, "similarity alone")
    assert capi.reg_get_device_error() == 0


@pytest.mark.parametrize("kind", ["lncc", "lncc_ants", "mi", "mi_hard"])
def test_identity_composite_loss_is_plain_loss(capi, kind):
    """With A = I, t = 0, s = 1 the composite kernels sample at the same
    points as the plain ones: the streaming sweeps give the same bits; the
    exact LNCC sweep may march other chunks (other rounding of the box sums)."""
    shape = (16, 24, 40)
    F, M = (mono_images if kind.startswith("lncc") else multimodal_images)(shape, 31)
    u = field(shape, 3.0, 2.0, 32).to(DEV)
    loss, _ = _loss(capi, kind, F, M)
    ws = capi.workspace(loss, F.to(DEV))
    s0, g0 = capi.reg_loss_grad(loss, F.to(DEV), M.to(DEV), u, ws)
    s1, g1, ga = capi.reg_loss_grad_composite(loss, F.to(DEV), M.to(DEV), capi.affine_desc(), u, ws=ws)
    torch.cuda.synchronize()
    assert s0[0].item() == s1[0].item()
    if kind == "lncc":
        assert rel_l2(to64(g1), to64(g0)) <= 1e-6
    else:
        assert torch.equal(g0, g1)
    # dC/dt is the sum of the per-voxel gradient
    assert rel_l2(to64(ga)[9:], to64(g0).reshape(3, -1).sum(axis=1)) <= 1e-5


def test_composite_rejects_bad_affine(capi):
    M = torch.zeros((4, 4, 4), device=DEV)
    T = capi.affine_desc(t=(float("nan"), 0.0, 0.0))
    with pytest.raises(RuntimeError):
        capi.reg_warp_composite(M, T)


# ---------------------------------------------------------------------------
# field composition and scaling-and-squaring on the fused sampler
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(16, 18, 40), (1, 9, 70), (7, 33, 5)])
@pytest.mark.parametrize("pad", [0, 1])
def test_compose_fields_matches_oracle(capi, shape, pad):
    a = field(shape, 3.0, 2.0, 51)
    b = field(shape, 2.0, 1.5, 52)
    w = capi.reg_compose_fields(a.to(DEV), b.to(DEV), pad)
    torch.cuda.synchronize()
    ref = O.compose_fields(to64(a), to64(b), pad)
    assert np.abs(to64(w) - ref).max() <= 1e-5 * np.abs(ref).max()


def test_compose_with_zero_is_exact(capi):
    shape = (9, 10, 33)
    a = field(shape, 3.0, 2.0, 54).to(DEV)
    z = torch.zeros_like(a)
    assert torch.equal(capi.reg_compose_fields(z, a), a)
    assert torch.equal(capi.reg_compose_fields(a, z), a)
    assert torch.equal(capi.reg_exp_field(z, 5), z)


@pytest.mark.parametrize("steps", [0, 1, 4, 7])
@pytest.mark.parametrize("pad", [0, 1])
def test_exp_field_matches_oracle(capi, steps, pad):
    shape = (20, 24, 36)
    v = field(shape, 4.0, 6.0, 53)
    u = capi.reg_exp_field(v.to(DEV), steps, pad)
    torch.cuda.synchronize()
    ref = O.exp_field(to64(v), steps, pad)
    assert np.abs(to64(u) - ref).max() <= 2e-5 * np.abs(ref).max()
    assert capi.reg_get_device_error() == 0


def test_exp_field_rejects_aliasing(capi):
    v = torch.zeros((3, 4, 4, 4), device=DEV)
    t = torch.empty_like(v)
    with pytest.raises(RuntimeError):
        capi.reg_exp_field(v, 3, out=v, tmp=t)
    with pytest.raises(RuntimeError):
        capi.reg_exp_field(v, 31)
    with pytest.raises(RuntimeError):
        capi.reg_compose_fields(v, t, out=v)


@pytest.mark.parametrize("shape", [(12, 18, 40), (1, 9, 70), (7, 33, 5)])
@pytest.mark.parametrize("pad", [0, 1])
def test_compose_backward_matches_oracle(capi, shape, pad):
    a = field(shape, 3.0, 2.5, 61)
    b = field(shape, 2.0, 1.5, 62)
    gw = torch.from_numpy(np.random.default_rng(63).standard_normal((3,) + shape).astype(np.float32))
    ga, gb = capi.reg_compose_fields_backward(a.to(DEV), b.to(DEV), gw.to(DEV), pad)
    torch.cuda.synchronize()
    gar, gbr = O.compose_fields_backward(to64(a), to64(b), to64(gw), pad)
    assert rel_l2(to64(ga), gar) <= GRAD_RTOL
    assert rel_l2(to64(gb), gbr) <= GRAD_RTOL
    # a and b one field: the whole gradient in one buffer
    ad = a.to(DEV)
    _, gs = capi.reg_compose_fields_backward(ad, ad, gw.to(DEV), pad, same=True)
    torch.cuda.synchronize()
    g1, g2 = O.compose_fields_backward(to64(a), to64(a), to64(gw), pad)
    assert rel_l2(to64(gs), g1 + g2) <= GRAD_RTOL


@pytest.mark.parametrize("steps", [0, 1, 3, 6])
@pytest.mark.parametrize("pad", [0, 1])
def test_exp_backward_matches_oracle(capi, steps, pad):
    shape = (16, 20, 36)
    v = field(shape, 4.0, 5.0, 64)
    gout = torch.from_numpy(np.random.default_rng(65).standard_normal((3,) + shape).astype(np.float32))
    vd = v.to(DEV)
    saved = torch.empty((max(steps - 1, 1), 3) + shape, device=DEV)
    out = capi.reg_exp_field(vd, steps, pad, saved=saved)
    gv = capi.reg_exp_field_backward(vd, steps, gout.to(DEV), saved=saved, pad=pad)
    torch.cuda.synchronize()
    assert np.abs(to64(out) - O.exp_field(to64(v), steps, pad)).max() <= 2e-5 * np.abs(to64(v)).max()
    ref = O.exp_field_backward(to64(v), steps, to64(gout), pad)
    assert rel_l2(to64(gv), ref) <= 1e-4
    assert capi.reg_get_device_error() == 0


@pytest.mark.parametrize("kind", ["lncc", "lncc_ants", "mi", "mi_hard"])
def test_run_under_composite_transform_matches_oracle(capi, kind):
    """reg_run with a composite transform (the fused iteration optimising u
    under phi = A p + t + S u): the objective history is the oracle's
    composite similarity and R(u), and the step is Adam on the oracle's
    gradient S dC/dphi + lam dR/du."""
    shape = (16, 18, 40)
    F, M = (mono_images if kind.startswith("lncc") else multimodal_images)(shape, 71)
    u = field(shape, 3.0, 1.0, 72)
    A, t, s = _affine(shape, 73, s=(1.0, 1.1, 0.9))
    loss, spec = _loss(capi, kind, F, M)
    N = F.numel()
    gen = torch.Generator().manual_seed(74)
    m0 = torch.randn((3,) + shape, generator=gen) * 1e-2
    v0 = m0 ** 2 + torch.rand((3,) + shape, generator=gen) * 1e-4
    lam, lr = 0.5, 0.1
    ud, m, v = u.to(DEV), m0.to(DEV), v0.to(DEV)
    ub = torch.empty_like(ud)
    adam = capi.adam_desc(lr, grad_scale=float(N))
    ws = capi.workspace(loss, F.to(DEV))
    hist = capi.reg_run(loss, F.to(DEV), M.to(DEV), ud, ub, m, v, lam, adam, 2, 1, ws,
                        affine=_desc(capi, A, t, s)).cpu().numpy()
    Sr, gur, _, _ = O.similarity_and_grad_composite(to64(F), to64(M), A, t, s, to64(u), spec)
    R, gR = O.diffusion(to64(u))
    assert_rel(hist[0, 0], Sr, LOSS_RTOL, "similarity")
    assert_rel(hist[0, 1], R, 1e-6, "R")
    ur, _, _ = O.adam(to64(u), to64(m0), to64(v0), gur + lam * gR, 3, lr, grad_scale=N)
    assert rel_l2(to64(ub) - to64(u), ur - to64(u)) <= 1e-3
    # the identity transform is the plain fused iteration
    u1, u2 = torch.empty_like(ud), torch.empty_like(ud)
    for T, out in ((capi.affine_desc(), u1), (None, u2)):
        mm, vv = m0.to(DEV), v0.to(DEV)
        capi.reg_run(loss, F.to(DEV), M.to(DEV), ud, out, mm, vv, lam, adam, 2, 1, ws, affine=T)
    torch.cuda.synchronize()
    if kind == "lncc":
        assert rel_l2(to64(u1) - to64(u), to64(u2) - to64(u)) <= 1e-5
    else:
        assert torch.equal(u1, u2)
    assert capi.reg_get_device_error() == 0
