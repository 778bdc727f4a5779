"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs (element by element where the oracle computes every
output, sampled at full size otherwise)."""
import numpy as np
import pytest
import torch

import oracle as O
from _util import (GRAD_RTOL, LOSS_RTOL, LOSS_RTOL_BF16, WARP_TOL, assert_bf16_drift, assert_rel, bf16_values,
                   field, mono_images, multimodal_images, rel_l2, to64)

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def _img(t, dtype):
    return t.to(DEV).to(dtype).contiguous()


def _oracle_img(t, dtype):
    return to64(bf16_values(t) if dtype == torch.bfloat16 else t)


# ---------------------------------------------------------------------------
# warp
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(17, 20, 33), (1, 6, 9), (24, 1, 7), (64, 64, 64)])
@pytest.mark.parametrize("pad", [0, 1])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_warp_matches_oracle(capi, shape, pad, dtype):
    F, M = mono_images(shape, 3)
    u = field(shape, 2.0, 4.0, 5)
    u[0, :, :, :2] += 6.0  # push some samples across the x border
    J, dJ = capi.reg_warp(_img(M, dtype), u.to(DEV), pad=pad, with_slope=True)
    torch.cuda.synchronize()
    Jr, dJr = O.warp(_oracle_img(M, dtype), to64(u), pad, with_grad=True)
    rng = float(M.max() - M.min())
    assert np.abs(to64(J) - Jr).max() <= WARP_TOL * rng
    assert np.abs(to64(dJ) - dJr).max() <= 2 * WARP_TOL * rng


def test_warp_zero_displacement_is_exact(capi):
    _, M = mono_images((19, 21, 23), 4)
    J = capi.reg_warp(M.to(DEV), torch.zeros((3,) + tuple(M.shape), device=DEV))
    assert torch.equal(J.cpu(), M)


# ---------------------------------------------------------------------------
# LNCC
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,window", [((16, 16, 16), 7), ((21, 35, 40), 5), ((20, 17, 44), 9),
                                          ((12, 13, 14), 15), ((1, 9, 40), 3), ((30, 30, 30), 3)])
@pytest.mark.parametrize("pad", [0, 1])
def test_lncc_matches_oracle(capi, shape, window, pad):
    F, M = mono_images(shape, 7)
    u = field(shape, 3.0, 2.5, 8)
    loss = capi.lncc_desc(window, 1e-4)
    ws = capi.workspace(loss, F.to(DEV))
    Fd, Md, ud = F.to(DEV), M.to(DEV), u.to(DEV)
    sim1 = capi.reg_loss(loss, Fd, Md, ud, ws, pad=pad)
    sim, g = capi.reg_loss_grad(loss, Fd, Md, ud, ws, pad=pad)
    torch.cuda.synchronize()
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=window, eps=1e-4)
    Sr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec, pad)
    assert_rel(sim1.item(), Sr, LOSS_RTOL, "S (reg_loss)")
    assert_rel(sim.item(), Sr, LOSS_RTOL, "S (reg_loss_grad)")
    assert rel_l2(to64(g), gr) <= GRAD_RTOL


# the ANTs gradient approximation (App. fused LNCC): the same similarity, the
# gradient without the second box sum; ragged volumes, borders, both pads
@pytest.mark.parametrize("shape,window", [((16, 16, 16), 7), ((21, 35, 40), 5), ((12, 13, 14), 15),
                                          ((1, 9, 40), 3)])
@pytest.mark.parametrize("pad", [0, 1])
def test_lncc_ants_gradient_matches_oracle(capi, shape, window, pad):
    F, M = mono_images(shape, 9)
    u = field(shape, 3.0, 2.5, 10)
    loss = capi.lncc_desc(window, 1e-4, ants=True)
    ws = capi.workspace(loss, F.to(DEV))
    Fd, Md, ud = F.to(DEV), M.to(DEV), u.to(DEV)
    sim, g = capi.reg_loss_grad(loss, Fd, Md, ud, ws, pad=pad)
    torch.cuda.synchronize()
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=window, eps=1e-4, lncc_grad=1)
    Sr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec, pad)
    assert_rel(sim.item(), Sr, LOSS_RTOL, "S")
    assert rel_l2(to64(g), gr) <= GRAD_RTOL
    # the exact adjoint differs: the flag is honoured
    spec0 = O.LossSpec(kind=O.LOSS_LNCC, window=window, eps=1e-4)
    _, g0 = O.similarity_and_grad(to64(F), to64(M), to64(u), spec0, pad)
    assert rel_l2(to64(g), g0) > 10 * GRAD_RTOL


def test_lncc_bf16_storage(capi):
    shape = (32, 40, 48)
    F, M = mono_images(shape, 11)
    u = field(shape, 3.0, 2.0, 12)
    loss = capi.lncc_desc(9, 1e-4)
    Fb, Mb = _img(F, torch.bfloat16), _img(M, torch.bfloat16)
    ws = capi.workspace(loss, Fb)
    sim, g = capi.reg_loss_grad(loss, Fb, Mb, u.to(DEV), ws)
    torch.cuda.synchronize()
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=9, eps=1e-4)
    # same stored values: FP32 arithmetic bars
    Sb, gb = O.similarity_and_grad(_oracle_img(F, torch.bfloat16), _oracle_img(M, torch.bfloat16), to64(u), spec)
    assert_rel(sim.item(), Sb, LOSS_RTOL, "S bf16 values")
    assert rel_l2(to64(g), gb) <= GRAD_RTOL
    # against the FP32 images: the BF16 storage bars
    Sr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec)
    assert_rel(sim.item(), Sr, LOSS_RTOL_BF16, "S bf16 vs f32")
    # the gradient against the FP32 images moves by the BF16 rounding of the
    # inputs themselves: no further than the oracle's own drift
    assert_bf16_drift(to64(g), gb, gr, "BF16 storage")


# ---------------------------------------------------------------------------
# MI
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,bins", [((16, 16, 16), 32), ((33, 29, 40), 32), ((24, 26, 28), 8),
                                        ((20, 22, 36), 64), ((1, 30, 41), 16)])
@pytest.mark.parametrize("pad", [0, 1])
def test_mi_matches_oracle(capi, shape, bins, pad):
    F, M = multimodal_images(shape, 21)
    u = field(shape, 3.0, 3.0, 22)
    fr = (float(F.min()), float(F.max()))
    mr = (float(M.min()), float(M.max()))
    loss = capi.mi_desc(fr, mr, bins)
    ws = capi.workspace(loss, F.to(DEV))
    Fd, Md, ud = F.to(DEV), M.to(DEV), u.to(DEV)
    sim1 = capi.reg_loss(loss, Fd, Md, ud, ws, pad=pad)
    sim, g = capi.reg_loss_grad(loss, Fd, Md, ud, ws, pad=pad)
    torch.cuda.synchronize()
    spec = O.LossSpec(kind=O.LOSS_MI, bins=bins, f_range=fr, m_range=mr)
    vr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec, pad)
    assert_rel(sim1.item(), vr, LOSS_RTOL, "MI (reg_loss)")
    assert_rel(sim.item(), vr, LOSS_RTOL, "MI (reg_loss_grad)")
    assert rel_l2(to64(g), gr) <= GRAD_RTOL


# the hard-binned approximate estimator (App. fused MI): nearest-bin counts
# convolved with the kernel in the finalisation, the Parzen adjoint with
# the approximate table
@pytest.mark.parametrize("shape,bins", [((16, 16, 16), 32), ((33, 29, 40), 32), ((24, 26, 28), 8),
                                        ((1, 7, 50), 16)])
@pytest.mark.parametrize("pad", [0, 1])
def test_mi_hard_binned_matches_oracle(capi, shape, bins, pad):
    F, M = multimodal_images(shape, 13)
    u = field(shape, 3.0, 2.0, 14)
    fr = (float(F.min()), float(F.max()))
    mr = (float(M.min()), float(M.max()))
    loss = capi.mi_desc(fr, mr, bins, hard=True)
    ws = capi.workspace(loss, F.to(DEV))
    Fd, Md, ud = F.to(DEV), M.to(DEV), u.to(DEV)
    sim1 = capi.reg_loss(loss, Fd, Md, ud, ws, pad=pad)
    sim, g = capi.reg_loss_grad(loss, Fd, Md, ud, ws, pad=pad)
    torch.cuda.synchronize()
    spec = O.LossSpec(kind=O.LOSS_MI, bins=bins, f_range=fr, m_range=mr, mi_estimator=1)
    Sr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec, pad)
    assert_rel(sim1.item(), Sr, LOSS_RTOL, "MI (reg_loss)")
    assert_rel(sim.item(), Sr, LOSS_RTOL, "MI (reg_loss_grad)")
    assert rel_l2(to64(g), gr) <= GRAD_RTOL
    # a different estimate from the Parzen one: the flag is honoured
    spec0 = O.LossSpec(kind=O.LOSS_MI, bins=bins, f_range=fr, m_range=mr)
    assert abs(O.similarity_and_grad(to64(F), to64(M), to64(u), spec0, pad, need_grad=False)[0] - Sr) > 1e-4 * Sr


def test_mi_bf16_storage(capi):
    shape = (40, 36, 44)
    F, M = multimodal_images(shape, 31)
    u = field(shape, 3.0, 3.0, 32)
    Fb, Mb = _img(F, torch.bfloat16), _img(M, torch.bfloat16)
    fr = (float(Fb.min()), float(Fb.max()))
    mr = (float(Mb.min()), float(Mb.max()))
    loss = capi.mi_desc(fr, mr, 32)
    ws = capi.workspace(loss, Fb)
    sim, g = capi.reg_loss_grad(loss, Fb, Mb, u.to(DEV), ws)
    torch.cuda.synchronize()
    spec = O.LossSpec(kind=O.LOSS_MI, bins=32, f_range=fr, m_range=mr)
    vb, gb = O.similarity_and_grad(_oracle_img(F, torch.bfloat16), _oracle_img(M, torch.bfloat16), to64(u), spec)
    assert_rel(sim.item(), vb, LOSS_RTOL, "MI bf16 values")
    assert rel_l2(to64(g), gb) <= GRAD_RTOL
    vr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec)
    assert_rel(sim.item(), vr, LOSS_RTOL_BF16, "MI bf16 vs f32")
    # the gradient against the FP32 images moves by the BF16 rounding of the
    # inputs themselves: no further than the oracle's own drift
    assert_bf16_drift(to64(g), gb, gr, "BF16 storage")


# ---------------------------------------------------------------------------
# regulariser, Adam, det J
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(9, 10, 37), (1, 5, 6), (40, 40, 40)])
def test_regularizer_matches_oracle(capi, shape):
    u = field(shape, 2.0, 3.0, 41)
    ud = u.to(DEV)
    ws = capi.workspace(None, ud[0])
    base = torch.randn(ud.shape, device=DEV) * 1e-6  # same scale as lambda dR/du
    g = base.clone()
    r = capi.reg_regularize(ud, 0.37, ws, grad=g)
    torch.cuda.synchronize()
    Rr, gr = O.diffusion(to64(u))
    assert_rel(r.item(), Rr, 1e-6, "R")
    assert rel_l2(to64(g - base), 0.37 * gr) <= 1e-5


@pytest.mark.parametrize("mdt", [0, 1])
@pytest.mark.parametrize("t", [1, 7])
def test_adam_matches_oracle(capi, mdt, t):
    n = (6, 7, 33)
    gen = torch.Generator().manual_seed(5 + t)
    u = torch.randn((3,) + n, generator=gen)
    g = torch.randn((3,) + n, generator=gen) * 1e-3
    m0 = torch.randn((3,) + n, generator=gen) * 0.5
    v0 = m0 ** 2 + torch.rand((3,) + n, generator=gen) * 0.3  # v >= m^2, as Adam keeps it
    mt = torch.bfloat16 if mdt else torch.float32
    m, v = m0.to(mt).to(DEV), v0.to(mt).to(DEV)
    adam = capi.adam_desc(0.05, moment_dtype=mdt, grad_scale=1000.0)
    uo = torch.empty_like(u, device=DEV)
    capi.reg_step(u.to(DEV), uo, m, v, g.to(DEV), adam, t)
    torch.cuda.synchronize()
    ur, mr, vr = O.adam(to64(u), to64(m0.to(mt)), to64(v0.to(mt)), to64(g), t, 0.05, grad_scale=1000.0,
                        bf16_moments=bool(mdt))
    np.testing.assert_allclose(to64(uo) - to64(u), ur - to64(u), atol=2e-6 * 0.05 * 10, rtol=1e-5)
    if mdt:  # one bf16 ulp where FP32 and FP64 land on opposite sides of a rounding boundary
        np.testing.assert_allclose(to64(m), mr, rtol=2 ** -7, atol=1e-30)
        np.testing.assert_allclose(to64(v), vr, rtol=2 ** -7, atol=1e-30)
    else:
        # FP32 rounding of b1 m + (1 - b1) g: relative to the terms, not the result
        np.testing.assert_allclose(to64(m), mr, rtol=1e-6, atol=2e-7)
        np.testing.assert_allclose(to64(v), vr, rtol=1e-6, atol=2e-7)


def test_jacdet_matches_oracle(capi):
    shape = (20, 24, 28)
    u = field(shape, 2.0, 4.0, 51)
    mn, nf = capi.reg_jacdet_min(u.to(DEV))
    torch.cuda.synchronize()
    d = O.jacdet(to64(u))
    assert abs(mn.item() - d.min()) <= 1e-5 * max(1.0, abs(d.min()))
    near = np.abs(d) < 1e-5
    assert abs(int(nf.item()) - int((d <= 0).sum())) <= int(near.sum())
    u0 = torch.zeros((3,) + shape, device=DEV)
    mn0, nf0 = capi.reg_jacdet_min(u0)
    assert mn0.item() == 1.0 and nf0.item() == 0


# ---------------------------------------------------------------------------
# fused iteration
# ---------------------------------------------------------------------------
def _iterate_case(capi, kind, shape, dtype=torch.float32, mdt=0, t=1, seed=61, bins=32):
    if kind in ("lncc", "lncc_ants"):
        F, M = mono_images(shape, seed)
        ants = kind == "lncc_ants"
        loss = capi.lncc_desc(7, 1e-4, ants=ants)
        spec = O.LossSpec(kind=O.LOSS_LNCC, window=7, eps=1e-4, lncc_grad=int(ants))
    else:
        F, M = multimodal_images(shape, seed)
        fr = (float(F.min()), float(F.max()))
        mr = (float(M.min()), float(M.max()))
        hard = kind == "mi_hard"
        loss = capi.mi_desc(fr, mr, bins, hard=hard)
        spec = O.LossSpec(kind=O.LOSS_MI, bins=bins, f_range=fr, m_range=mr, mi_estimator=int(hard))
    u = field(shape, 3.0, 2.0, seed + 1)
    N = int(np.prod(shape))
    gen = torch.Generator().manual_seed(seed)
    m0 = torch.randn((3,) + shape, generator=gen) * 1e-2
    v0 = m0 ** 2 + torch.rand((3,) + shape, generator=gen) * 1e-4  # v >= m^2, as Adam keeps it
    mt = torch.bfloat16 if mdt else torch.float32
    Fd, Md = _img(F, dtype), _img(M, dtype)
    m, v = m0.to(mt).to(DEV), v0.to(mt).to(DEV)
    adam = capi.adam_desc(0.1, moment_dtype=mdt, grad_scale=float(N))
    ws = capi.workspace(loss, Fd)
    ud = u.to(DEV)
    uo = torch.empty_like(ud)
    g = torch.empty_like(ud)
    obj = capi.reg_iterate(loss, Fd, Md, ud, uo, m, v, 0.1, adam, t, ws, grad=g)
    torch.cuda.synchronize()
    return dict(F=F, M=M, u=u, m0=m0.to(mt), v0=v0.to(mt), spec=spec, uo=uo, m=m, v=v, g=g, obj=obj, N=N,
                dtype=dtype)


@pytest.mark.parametrize("kind", ["lncc", "mi", "lncc_ants", "mi_hard"])
@pytest.mark.parametrize("shape", [(24, 20, 35), (48, 48, 48)])
def test_iterate_matches_oracle(capi, kind, shape):
    c = _iterate_case(capi, kind, shape, t=3)
    ref = O.objective(to64(c["F"]), to64(c["M"]), to64(c["u"]), c["spec"], 0.1)
    assert_rel(c["obj"][0].item(), ref["sim"], LOSS_RTOL, "similarity")
    assert_rel(c["obj"][1].item(), ref["R"], 1e-6, "R")
    assert rel_l2(to64(c["g"]), ref["grad"]) <= GRAD_RTOL
    # Adam on the GPU's own gradient must agree elementwise with the oracle's Adam
    ur, mr, vr = O.adam(to64(c["u"]), to64(c["m0"]), to64(c["v0"]), to64(c["g"]), 3, 0.1, grad_scale=c["N"])
    np.testing.assert_allclose(to64(c["uo"]), ur, atol=1e-5, rtol=0)
    np.testing.assert_allclose(to64(c["m"]), mr, rtol=1e-5, atol=1e-7)


# Rows with nx % 8 == 0 take the TMA-staged MI sweep (an x pair per lane, the
# diffusion halo from the staged box; 64 x 31 tiles with BF16 moments, whose
# rings fit beside FP32 images, 64 x 20 with FP32 moments): rows that span
# several tiles with a partial last one, ragged y and z, both moment types;
# rows with nx % 8 != 0 the plain sweep.
@pytest.mark.parametrize("kind", ["mi", "mi_hard"])
@pytest.mark.parametrize("shape,mdt", [((9, 11, 264), 0), ((6, 70, 136), 1), ((5, 3, 8), 0), ((7, 9, 132), 1)])
def test_iterate_tile_rows_match_oracle(capi, kind, shape, mdt):
    c = _iterate_case(capi, kind, shape, mdt=mdt, t=2, seed=91)
    ref = O.objective(to64(c["F"]), to64(c["M"]), to64(c["u"]), c["spec"], 0.1)
    assert_rel(c["obj"][0].item(), ref["sim"], LOSS_RTOL, "similarity")
    assert_rel(c["obj"][1].item(), ref["R"], 1e-6, "R")
    assert rel_l2(to64(c["g"]), ref["grad"]) <= GRAD_RTOL
    ur, mr, vr = O.adam(to64(c["u"]), to64(c["m0"]), to64(c["v0"]), to64(c["g"]), 2, 0.1, grad_scale=c["N"],
                        bf16_moments=bool(mdt))
    np.testing.assert_allclose(to64(c["uo"]), ur, atol=1e-5, rtol=0)
    if mdt:  # BF16 moments: one BF16 ulp of the oracle's RNE-rounded moments, plus the FP32 rounding
        # of b1 m + (1 - b1) g where the two terms (|m| < 0.05) cancel: 2 * 2^-24 * 0.05 < 1e-8
        np.testing.assert_allclose(to64(c["m"]), mr, rtol=2 ** -7, atol=1e-8)
    else:
        np.testing.assert_allclose(to64(c["m"]), mr, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("kind", ["lncc", "mi"])
def test_iterate_is_deterministic(capi, kind):
    a = _iterate_case(capi, kind, (40, 33, 37), seed=71)
    b = _iterate_case(capi, kind, (40, 33, 37), seed=71)
    for k in ("uo", "m", "v", "g", "obj"):
        assert torch.equal(a[k], b[k]), k


# ---------------------------------------------------------------------------
# failure detection (host-visible device error word; no GPU fault)
# ---------------------------------------------------------------------------
def test_nonfinite_input_is_reported(capi):
    shape = (16, 16, 16)
    F, M = mono_images(shape, 81)
    F[3, 4, 5] = float("nan")
    loss = capi.lncc_desc(5, 1e-4)
    Fd = F.to(DEV)
    ws = capi.workspace(loss, Fd)
    assert capi.reg_get_device_error() == 0
    capi.reg_loss(loss, Fd, M.to(DEV), torch.zeros((3,) + shape, device=DEV), ws)
    assert capi.reg_get_device_error() == 6  # REG_ERR_NONFINITE
    assert capi.reg_get_device_error() == 0  # cleared


def test_bounded_wait_times_out_and_context_survives(capi):
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    capi.reg_debug_wait_flag(flag, 1, 2_000_000)  # nothing sets it: 2 ms limit
    assert capi.reg_get_device_error() == 7  # REG_ERR_TIMEOUT
    flag[0] = 1
    capi.reg_debug_wait_flag(flag, 1, 2_000_000)
    assert capi.reg_get_device_error() == 0
    assert torch.ones(3, device=DEV).sum().item() == 3.0


# ---------------------------------------------------------------------------
# Gaussian smoothing of fields (sigma_grad / sigma_warp regularisation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,sigma", [((9, 10, 37), 1.0), ((1, 5, 6), 0.5), ((40, 33, 20), 2.3), ((3, 70, 4), 7.9)])
def test_smooth_field_matches_oracle(capi, shape, sigma):
    u = field(shape, 2.0, 3.0, 5) + torch.randn((3,) + shape, generator=torch.Generator().manual_seed(5))
    out = capi.reg_smooth_field(u.to(DEV), sigma)
    torch.cuda.synchronize()
    ref = O.gaussian_smooth(to64(u), sigma)
    np.testing.assert_allclose(to64(out), ref, rtol=0, atol=2e-6 * np.abs(ref).max())


def test_smoothing_regularised_registration(capi):
    """The registration driver's smoothing path (gradient -> smooth -> Adam -> smooth, no
    diffusion term) decreases the objective and regularises the field: far
    fewer folded voxels than the same run without smoothing."""
    from paper_2509_25044_gb300 import synth
    from paper_2509_25044_gb300.register import RegConfig, Registration
    d = synth.make("c0", device=DEV)
    folds = {}
    for sg, sw in ((0.0, 0.0), (1.0, 1.0)):
        cfg = RegConfig(loss="lncc", window=7, eps=1e-9, lam=0.0, lr=0.1, sigma_grad=sg, sigma_warp=sw)
        r = Registration(d["F"], d["M"], cfg)
        res = r.run(50)
        assert np.all(np.isfinite(res.objective))
        assert res.objective[-1] < res.objective[0]
        folds[sg] = r.fold_check()["n_fold"]
    assert folds[1.0] * 10 <= max(folds[0.0], 1), folds
    assert capi.reg_get_device_error() == 0


@pytest.mark.parametrize("shape", [(8, 6, 10), (34, 18, 66), (2, 2, 2)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_downsample2_matches_oracle(capi, shape, dtype):
    img = torch.rand(shape, generator=torch.Generator().manual_seed(7)) * 3.0 - 1.0
    out = capi.reg_downsample2(_img(img, dtype))
    torch.cuda.synchronize()
    assert out.dtype == dtype and tuple(out.shape) == tuple(s // 2 for s in shape)
    ref = O.downsample2(_oracle_img(img, dtype))
    got = to64(out.float().cpu())
    if dtype == torch.float32:  # an FP32 sum of 8 terms
        np.testing.assert_allclose(got, ref, rtol=0, atol=4e-7 * np.abs(ref).max())
    else:  # the FP32 mean rounded once to BF16 (8 significant bits)
        np.testing.assert_allclose(got, ref, rtol=2.0 ** -8, atol=1e-6)


def test_downsample2_rejects_odd_and_aliasing(capi):
    img = torch.zeros((8, 8, 9), device=DEV)
    with pytest.raises(RuntimeError):
        capi.reg_downsample2(img)
    a = torch.zeros((8, 8, 8), device=DEV)
    st = capi._lib().reg_downsample2(capi._ptr(a), 0, capi.dims_of(a), capi._ptr(a), capi._stream(a))
    assert st != 0


@pytest.mark.parametrize("kind", ["lncc", "lncc_ants", "mi"])
@pytest.mark.parametrize("iters", [1, 4, 5])
def test_run_matches_repeated_iterate(capi, kind, iters):
    """reg_run (all iterations in one native call) gives the iterates and
    objective history of as many reg_iterate calls -- bit for bit for MI; for
    LNCC it forms F's window mean and variance once per call, which changes
    the last bits only -- and leaves the last iterate in u_a / u_b by the
    parity of the count."""
    shape = (12, 10, 20)
    gen = torch.Generator().manual_seed(11)
    F = torch.rand(shape, generator=gen).to(DEV)
    M = torch.rand(shape, generator=gen).to(DEV)
    loss = (capi.lncc_desc(5, 1e-9, ants=kind == "lncc_ants") if kind.startswith("lncc")
            else capi.mi_desc((0.0, 1.0), (0.0, 1.0), 32))
    adam = capi.adam_desc(0.05)
    ws = capi.workspace(loss, F)
    outs = []
    for native in (False, True):
        u = [torch.zeros((3,) + shape, device=DEV) for _ in range(2)]
        u[0].copy_(0.3 * torch.randn((3,) + shape, generator=torch.Generator().manual_seed(3)))
        m = torch.zeros((3,) + shape, device=DEV)
        v = torch.zeros((3,) + shape, device=DEV)
        hist = torch.zeros((iters, 2), dtype=torch.float64, device=DEV)
        t0 = 2  # continue a run: the step numbers are t0 + 1 ..
        if native:
            capi.reg_run(loss, F, M, u[0], u[1], m, v, 0.5, adam, t0, iters, ws, obj_hist=hist)
        else:
            for k in range(iters):
                capi.reg_iterate(loss, F, M, u[k % 2], u[(k + 1) % 2], m, v, 0.5, adam, t0 + k + 1, ws, obj=hist[k])
        torch.cuda.synchronize()
        outs.append((u[iters % 2].cpu(), m.cpu(), v.cpu(), hist.cpu()))
    if kind == "mi":
        for a, b in zip(*outs):
            assert torch.equal(a, b)
    else:
        u0 = 0.3 * torch.randn((3,) + shape, generator=torch.Generator().manual_seed(3))
        (ua, ma, _, ha), (ub, mb, _, hb) = outs
        np.testing.assert_allclose(hb.numpy(), ha.numpy(), rtol=1e-6, atol=0)
        assert rel_l2(to64(ub) - to64(u0), to64(ua) - to64(u0)) <= 1e-4
        assert rel_l2(to64(mb), to64(ma)) <= 1e-4
    assert capi.reg_get_device_error() == 0


@pytest.mark.parametrize("shape,img,bins,hard,pad", [
    ((37, 45, 72), torch.bfloat16, 32, False, 0),   # ragged columns in x and y (32 x 24 and 32 x 32)
    ((37, 45, 72), torch.float32, 32, True, 1),     # hard-binned, zero padding
    ((9, 7, 8), torch.float32, 16, False, 1),       # one column, 16 copies
    ((400, 310, 256), torch.bfloat16, 32, False, 0),  # copies flushed every 170 / 256 planes, many times per CTA
    ((400, 310, 256), torch.bfloat16, 64, False, 0),  # 8 copies
])
def test_identity_composite_histogram_equals_plain_histogram(capi, shape, img, bins, hard, pad):
    """The composite form with the identity transform (phi = I p + 0 + 1 u =
    p + u exactly, 64-bit offsets) forms the same fixed-point joint histogram,
    bit for bit, as the plain form, over ragged tiles, both estimators and
    pads, and volumes whose persistent CTAs flush their 32-bit copies many
    times.  With 32 bins on BF16 images the two forms also run different CTA
    shapes (the plain one two 768-thread CTAs per SM with 24 copies, the
    composite one 1024-thread CTA with 32), so this also checks that the
    shape leaves the integer sums alone."""
    gen = torch.Generator(device=DEV).manual_seed(bins + shape[0])
    F = torch.rand(shape, generator=gen, device=DEV).to(img)
    M = torch.rand(shape, generator=gen, device=DEV).to(img)
    u = 1.5 * torch.randn((3,) + shape, generator=gen, device=DEV)
    loss = capi.mi_desc((0.0, 1.0), (0.0, 1.0), bins, hard=hard)
    ws_plain, ws_comp = capi.workspace(loss, F), capi.workspace(loss, F)
    s_plain = capi.reg_loss(loss, F, M, u, ws_plain, pad=pad)
    s_comp, _, _ = capi.reg_loss_grad_composite(loss, F, M, capi.affine_desc(), u=u, ws=ws_comp, pad=pad,
                                                need_u=False, need_affine=False)
    torch.cuda.synchronize()
    n = bins * bins * 8  # the workspace starts with the u64 joint histogram
    h_plain, h_comp = ws_plain[:n].view(torch.int64), ws_comp[:n].view(torch.int64)
    assert int(h_plain.sum()) > 0
    assert torch.equal(h_plain, h_comp)
    assert float(s_plain[0]) == float(s_comp[0])
    assert capi.reg_get_device_error() == 0


# 64 bins on rows the TMA sweep takes: its 64 x 31 tile's rings and table do
# not fit a CTA's shared memory, so the 64 x 20 tile runs (BF16 moments) or,
# with FP32 images and moments, neither fits and the plain sweep runs.
@pytest.mark.parametrize("dtype,mdt", [(torch.float32, 0), (torch.float32, 1), (torch.bfloat16, 1)])
def test_iterate_64_bins_on_tma_rows_matches_oracle(capi, dtype, mdt):
    shape = (6, 45, 136)
    c = _iterate_case(capi, "mi", shape, dtype=dtype, mdt=mdt, t=2, seed=93, bins=64)
    if dtype == torch.bfloat16:
        F, M = bf16_values(c["F"]), bf16_values(c["M"])
    else:
        F, M = c["F"], c["M"]
    ref = O.objective(to64(F), to64(M), to64(c["u"]), c["spec"], 0.1)
    assert_rel(c["obj"][0].item(), ref["sim"], LOSS_RTOL, "similarity")
    assert_rel(c["obj"][1].item(), ref["R"], 1e-6, "R")
    assert rel_l2(to64(c["g"]), ref["grad"]) <= GRAD_RTOL
    ur, mr, vr = O.adam(to64(c["u"]), to64(c["m0"]), to64(c["v0"]), to64(c["g"]), 2, 0.1, grad_scale=c["N"],
                        bf16_moments=bool(mdt))
    np.testing.assert_allclose(to64(c["uo"]), ur, atol=1e-5, rtol=0)
    assert capi.reg_get_device_error() == 0


@pytest.mark.parametrize("shape,img,bf16_moments,hard", [
    ((20, 24, 64), torch.bfloat16, True, False),   # the TMA step with BF16 images and moments
    ((7, 9, 136), torch.bfloat16, True, False),    # ragged rows and tiles
    ((20, 24, 64), torch.float32, False, False),   # the TMA step in FP32
    ((20, 24, 64), torch.bfloat16, True, True),    # hard-binned histogram
    ((256, 256, 256), torch.bfloat16, True, False),  # chunks of 128 planes
])
def test_run_matches_repeated_iterate_mi_forms(capi, shape, img, bf16_moments, hard):
    """reg_run gives the objectives, iterates and moments of as many
    reg_iterate calls bit for bit in every MI form the bench times: BF16 and
    FP32 images and moments on the TMA step, the hard-binned estimator, and a
    volume whose CTAs take long chunks (the histogram is exact fixed point,
    so nothing depends on the order of its additions)."""
    iters = 3
    gen = torch.Generator(device=DEV).manual_seed(23)
    F = torch.rand(shape, generator=gen, device=DEV).to(img)
    M = torch.rand(shape, generator=gen, device=DEV).to(img)
    u0 = 0.4 * torch.randn((3,) + shape, generator=gen, device=DEV)
    loss = capi.mi_desc((0.0, 1.0), (0.0, 1.0), 32, hard=hard)
    mt = torch.bfloat16 if bf16_moments else torch.float32
    adam = capi.adam_desc(0.05, moment_dtype=capi.REG_BF16 if bf16_moments else capi.REG_F32,
                          grad_scale=float(F.numel()))
    ws = capi.workspace(loss, F)
    outs = []
    for native in (False, True):
        u = [u0.clone(), torch.zeros_like(u0)]
        m = torch.zeros((3,) + shape, dtype=mt, device=DEV)
        v = torch.zeros((3,) + shape, dtype=mt, device=DEV)
        hist = torch.zeros((iters, 2), dtype=torch.float64, device=DEV)
        if native:
            capi.reg_run(loss, F, M, u[0], u[1], m, v, 0.5, adam, 0, iters, ws, obj_hist=hist)
        else:
            for k in range(iters):
                capi.reg_iterate(loss, F, M, u[k % 2], u[(k + 1) % 2], m, v, 0.5, adam, k + 1, ws, obj=hist[k])
        torch.cuda.synchronize()
        outs.append((u[iters % 2], m, v, hist))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    assert not torch.equal(outs[0][0], u0)  # the iterations moved u
    assert capi.reg_get_device_error() == 0


# ---------------------------------------------------------------------------
# degenerate inputs the method has: constant images (zero window variances,
# a single-bin histogram) and one-voxel volumes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["lncc", "lncc_eps0", "mi"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3), (9, 10, 37)])
def test_constant_and_tiny_volumes_match_oracle(capi, kind, shape):
    gen = torch.Generator().manual_seed(81)
    F = torch.full(shape, 0.7)
    M = torch.rand(shape, generator=gen)
    u = 0.6 * torch.randn((3,) + shape, generator=gen)
    if kind == "mi":
        loss = capi.mi_desc((0.0, 1.0), (0.0, 1.0), 16)
        spec = O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=(0.0, 1.0), m_range=(0.0, 1.0))
    else:
        eps = 0.0 if kind == "lncc_eps0" else 1e-9
        loss = capi.lncc_desc(3, eps)
        spec = O.LossSpec(kind=O.LOSS_LNCC, window=3, eps=eps)
    ws = capi.workspace(loss, F.to(DEV))
    sim, g = capi.reg_loss_grad(loss, F.to(DEV), M.to(DEV), u.to(DEV), ws)
    torch.cuda.synchronize()
    Sr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec)
    # F constant: every window variance of F is 0, so each n_i is 0 (LNCC), and
    # the joint histogram has one fixed-image bin, so MI = 0
    assert abs(Sr) <= 1e-12
    assert abs(sim.item()) <= 1e-6
    assert np.all(np.isfinite(to64(g)))
    np.testing.assert_allclose(to64(g), gr, rtol=0, atol=1e-6 * max(1.0, np.abs(gr).max()))
    assert capi.reg_get_device_error() == 0
