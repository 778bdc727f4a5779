"""The learned initialiser's non-convolution operators on the GPU, through the
C ABI, against the FP64 oracle on the same BF16 / FP32 values: 2x average
pooling and 2x trilinear upsampling (forward and backward), the LeakyReLU
backward, channel concat / slicing, the network input, the training loss and
the bias gradient, and the displacement resampling between the network's
grid and the registration grid (field_down2, field_upsample).

Bars.  An operator that stores BF16 rounds its FP32 result once to nearest
even: |bf16(y) - y| <= 2^-8 |y|.  Its FP32 arithmetic adds at most
gamma_k = k u / (1 - k u), u = 2^-24, times the sum of the absolute terms
for a k-term sum (Higham, Accuracy and Stability of Numerical Algorithms,
Eq. 3.5).  So an output y of k terms must satisfy
|got - y| <= 2^-8 |y| + (1 + 2^-8) gamma_k S, S the sum of |terms|, which the
tests form with the oracle itself applied to absolute values."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
BF = 2.0 ** -8
U32 = 2.0 ** -24


def gamma(k):
    return k * U32 / (1.0 - k * U32)


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def _bf16(rng, shape, scale=1.0):
    return torch.from_numpy((rng.standard_normal(shape) * scale).astype(np.float32)).to(torch.bfloat16)


def _np(t):
    return t.detach().double().cpu().numpy()


def _within(got, ref, bound, what):
    err = np.abs(got - ref)
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} outside the bar; worst excess "
                           f"{float((err - bound).max()):.3e}, max |ref| {float(np.abs(ref).max()):.3e}")


def _dims(capi, shape):
    return capi.RegDims(shape[2], shape[1], shape[0])


# ---------------------------------------------------------------------------
# pooling and upsampling (channels-last BF16)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,C", [((6, 10, 14), 8), ((2, 4, 36), 24), ((8, 2, 6), 64)])
def test_avgpool2_forward_and_backward(capi, shape, C):
    L = capi.nn()
    rng = np.random.default_rng(C)
    x = _bf16(rng, shape + (C,))
    xd = x.to(DEV)
    cs = tuple(s // 2 for s in shape)
    out = torch.empty(cs + (C,), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_avgpool2(capi.ptr(xd), C, _dims(capi, shape), capi.ptr(out), 0, capi.stream_of(xd)),
                  "pool")
    g = _bf16(rng, cs + (C,)).to(DEV)
    gin = torch.empty(shape + (C,), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_avgpool2(capi.ptr(g), C, _dims(capi, shape), capi.ptr(gin), 1, capi.stream_of(g)),
                  "pool bwd")
    torch.cuda.synchronize()
    ref = O.avgpool2(_np(x))
    S = O.avgpool2(np.abs(_np(x)))
    _within(_np(out), ref, BF * np.abs(ref) + (1 + BF) * gamma(8) * S, "avgpool2")
    gref = O.avgpool2_adjoint(_np(g), shape)
    _within(_np(gin), gref, BF * np.abs(gref), "avgpool2 backward")


@pytest.mark.parametrize("cshape,C", [((3, 5, 7), 8), ((1, 2, 3), 16), ((4, 4, 20), 64)])
def test_upsample2_forward_and_backward(capi, cshape, C):
    L = capi.nn()
    rng = np.random.default_rng(10 + C)
    x = _bf16(rng, cshape + (C,))
    xd = x.to(DEV)
    fshape = tuple(2 * s for s in cshape)
    out = torch.empty(fshape + (C,), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_upsample2(capi.ptr(xd), C, _dims(capi, cshape), capi.ptr(out), 0, capi.stream_of(xd)),
                  "up")
    g = _bf16(rng, fshape + (C,)).to(DEV)
    gin = torch.empty(cshape + (C,), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_upsample2(capi.ptr(g), C, _dims(capi, cshape), capi.ptr(gin), 1, capi.stream_of(g)),
                  "up bwd")
    torch.cuda.synchronize()
    ref = O.upsample(_np(x), 2)
    S = O.upsample(np.abs(_np(x)), 2)
    _within(_np(out), ref, BF * np.abs(ref) + (1 + BF) * gamma(16) * S, "upsample2")
    gref = O.upsample_adjoint(_np(g), 2)
    Sg = O.upsample_adjoint(np.abs(_np(g)), 2)
    _within(_np(gin), gref, BF * np.abs(gref) + (1 + BF) * gamma(128) * Sg, "upsample2 backward")


# ---------------------------------------------------------------------------
# LeakyReLU backward, concat / slice, bias gradient
# ---------------------------------------------------------------------------
def test_leaky_backward(capi):
    L = capi.nn()
    rng = np.random.default_rng(20)
    n = 3 * 1000 + 5
    x = _bf16(rng, (n,))
    x[7] = 0.0  # the kink takes the slope
    out = torch.from_numpy(O.leaky(_np(x), 0.2)).to(torch.bfloat16)
    dout = _bf16(rng, (n,))
    outd, doutd = out.to(DEV), dout.to(DEV)
    dpre = torch.empty_like(doutd)
    capi.nn_check(L.reg_nn_leaky_bwd(capi.ptr(outd), capi.ptr(doutd), n, 0.2, capi.ptr(dpre),
                                     capi.stream_of(outd)), "leaky bwd")
    torch.cuda.synchronize()
    ref = O.leaky_bwd(_np(x), _np(dout), 0.2)  # the output's sign is the input's
    _within(_np(dpre), ref, (BF + U32) * np.abs(ref), "leaky backward")


def test_concat_and_slice_are_exact(capi):
    L = capi.nn()
    rng = np.random.default_rng(21)
    V = 4 * 5 * 6
    a, b = _bf16(rng, (V, 64)), _bf16(rng, (V, 32))
    ad, bd = a.to(DEV), b.to(DEV)
    cat = torch.empty((V, 96), dtype=torch.bfloat16, device=DEV)
    s = capi.stream_of(ad)
    capi.nn_check(L.reg_nn_put_channels(capi.ptr(ad), 64, V, capi.ptr(cat), 96, 0, 0, s), "put a")
    capi.nn_check(L.reg_nn_put_channels(capi.ptr(bd), 32, V, capi.ptr(cat), 96, 64, 0, s), "put b")
    back = torch.empty((V, 32), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_take_channels(capi.ptr(cat), 96, 64, V, capi.ptr(back), 32, 0, s), "take")
    torch.cuda.synchronize()
    ref = O.concat(_np(a), _np(b))
    np.testing.assert_array_equal(_np(cat), ref)
    np.testing.assert_array_equal(_np(back), ref[:, 64:])


def test_bias_gradient(capi):
    L = capi.nn()
    rng = np.random.default_rng(22)
    V, C = 7 * 9 * 11, 48
    d = _bf16(rng, (V, C)).to(DEV)
    scratch = torch.empty(int(L.reg_nn_bias_grad_scratch_bytes(C)), dtype=torch.uint8, device=DEV)
    out = torch.empty(C, device=DEV)
    capi.nn_check(L.reg_nn_bias_grad(capi.ptr(d), V, C, capi.ptr(scratch), capi.ptr(out), capi.stream_of(d)),
                  "bias grad")
    torch.cuda.synchronize()
    ref = _np(d).sum(axis=0)
    # FP64 partial sums (unit roundoff 2^-53), one FP32 rounding at the end
    _within(_np(out), ref, U32 * np.abs(ref) + V * 2.0 ** -53 * np.abs(_np(d)).sum(axis=0), "bias gradient")


# ---------------------------------------------------------------------------
# network input and training loss
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,factor", [(torch.float32, 2), (torch.bfloat16, 4)])
def test_pack_pair(capi, dtype, factor):
    L = capi.nn()
    rng = np.random.default_rng(23)
    shape = (4 * factor, 3 * factor, 5 * factor)
    F = torch.from_numpy(rng.uniform(1.0, 3.0, shape).astype(np.float32)).to(dtype)
    M = torch.from_numpy(rng.uniform(-2.0, 2.0, shape).astype(np.float32)).to(dtype)
    Fd, Md = F.to(DEV), M.to(DEV)
    cs = tuple(s // factor for s in shape)
    out = torch.empty(cs + (16,), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_pack_pair(capi.ptr(Fd), capi.ptr(Md), capi._img_dtype(Fd), _dims(capi, shape), factor,
                                     1.0, 3.0, -2.0, 2.0, capi.ptr(out), capi.stream_of(Fd)), "pack")
    torch.cuda.synchronize()
    ref = O.pack_pair(_np(F), _np(M), factor, (1.0, 3.0), (-2.0, 2.0))
    got = _np(out)
    k = factor ** 3
    # block sum (k terms) of values up to 3 in magnitude, then the range map
    bound = BF * np.abs(ref) + (1 + BF) * (gamma(k + 3) * (3.0 / 2.0 + 1.0))
    _within(got[..., :2], ref, bound, "pack_pair")
    assert not got[..., 2:].any()


def test_training_loss_and_its_gradient(capi):
    L = capi.nn()
    rng = np.random.default_rng(24)
    V = 6 * 7 * 8
    pred = torch.from_numpy(rng.standard_normal((3, V)).astype(np.float32)).to(DEV)
    tgt = torch.from_numpy(rng.standard_normal((3, V)).astype(np.float32)).to(DEV)
    dpred = torch.empty((V, 16), dtype=torch.bfloat16, device=DEV)
    scratch = torch.empty(int(L.reg_nn_mse_scratch_bytes()), dtype=torch.uint8, device=DEV)
    loss = torch.empty(1, dtype=torch.float64, device=DEV)
    capi.nn_check(L.reg_nn_mse(capi.ptr(pred), capi.ptr(tgt), V, 16, capi.ptr(dpred), capi.ptr(scratch),
                               capi.ptr(loss), capi.stream_of(pred)), "mse")
    torch.cuda.synchronize()
    lref, gref = O.mse(_np(pred), _np(tgt))
    assert abs(loss.item() - lref) <= 1e-6 * lref
    got = _np(dpred)
    _within(got[:, :3].T, gref, (BF + 4 * U32) * np.abs(gref), "mse gradient")
    assert not got[:, 3:].any()


# ---------------------------------------------------------------------------
# displacement resampling (FP32 SoA)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(6, 8, 10), (2, 14, 4)])
def test_field_down2(capi, shape):
    L = capi.nn()
    u = torch.from_numpy(np.random.default_rng(25).standard_normal((3,) + shape).astype(np.float32)).to(DEV)
    out = torch.empty((3,) + tuple(s // 2 for s in shape), device=DEV)
    capi.nn_check(L.reg_nn_field_down2(capi.ptr(u), _dims(capi, shape), capi.ptr(out), capi.stream_of(u)), "down2")
    torch.cuda.synchronize()
    ref = O.field_down2(_np(u))
    S = O.field_down2(np.abs(_np(u)))
    _within(_np(out), ref, gamma(10) * S, "field_down2")


@pytest.mark.parametrize("cshape,s", [((3, 4, 5), 2), ((2, 3, 2), 4), ((4, 1, 3), 8)])
def test_field_upsample(capi, cshape, s):
    L = capi.nn()
    u = torch.from_numpy(np.random.default_rng(26 + s).standard_normal((3,) + cshape).astype(np.float32)).to(DEV)
    out = torch.empty((3,) + tuple(s * k for k in cshape), device=DEV)
    capi.nn_check(L.reg_nn_field_upsample(capi.ptr(u), _dims(capi, cshape), s, capi.ptr(out), capi.stream_of(u)),
                  "field_upsample")
    torch.cuda.synchronize()
    ref = O.field_upsample(_np(u), s)
    S = O.field_upsample(np.abs(_np(u)), s)
    _within(_np(out), ref, gamma(16) * S, "field_upsample")
