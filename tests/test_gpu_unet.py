"""Learned initialiser on the GPU: the tcgen05 implicit-GEMM convolutions
against the FP64 oracle (forward, data and weight gradients), the whole
U-Net forward/backward against the oracle's composition of the same
operators with the same weights (layer by layer, and end to end), and a
short training run."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def _pack_w(w, rows, kpad):
    """[Cout][27][Cin] float -> packed [rows][kpad] (bf16 values)."""
    cout, _, cin = w.shape
    out = np.zeros((rows, kpad), dtype=np.float32)
    out[:cout, :27 * cin] = w.reshape(cout, 27 * cin)
    return torch.from_numpy(out).to(DEV).to(torch.bfloat16)


def _bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


# shapes: the gather kernel only (Cin 8), the TMA-fed kernel on ragged
# volumes spanning several tiles and M-tiles, several 16-channel chunks,
# N below 16 (the displacement head), nx above 128 (brick pitch 132)
@pytest.mark.parametrize("shape,cin,cout", [((9, 10, 11), 8, 16), ((6, 7, 8), 32, 64), ((5, 6, 4), 96, 32),
                                            ((13, 9, 20), 16, 16), ((7, 33, 64), 32, 32), ((5, 12, 17), 32, 3),
                                            ((3, 6, 130), 16, 16), ((4, 5, 16), 128, 64)])
@pytest.mark.parametrize("tma", [False, True])
def test_conv_forward_matches_oracle(capi, shape, cin, cout, tma):
    L = capi.nn()
    rng = np.random.default_rng(cin + cout)
    x = _bf(rng.standard_normal(shape + (cin,)))
    w = _bf(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin)).float().numpy()
    b = rng.standard_normal(cout).astype(np.float32)
    kpad = int(L.reg_nn_conv_kpad(cin))
    rows = (cout + 15) // 16 * 16
    W = _pack_w(w, rows, kpad)
    bias = torch.zeros(rows, device=DEV)
    bias[:cout] = torch.from_numpy(b)
    xd = x.to(DEV).contiguous()
    V = int(np.prod(shape))
    d = capi.RegDims(shape[2], shape[1], shape[0])
    nws = int(L.reg_nn_conv_scratch_bytes(cin, cout)) if tma else 0
    if tma and cin % 16 == 0:
        assert nws > 0
    ws = torch.empty(max(nws, 16), dtype=torch.uint8, device=DEV)
    wsp = capi.ptr(ws) if nws else None
    out32 = torch.empty((cout, V), device=DEV)
    capi.nn_check(L.reg_nn_conv3d_fwd(capi.ptr(xd), cin, capi.ptr(W), capi.ptr(bias), cout, d, 2, 0.2, wsp, nws,
                                      capi.ptr(out32), capi.stream_of(xd)), "fwd f32")
    torch.cuda.synchronize()
    ref = O.conv3d(x.float().numpy(), w, b).reshape(V, cout)
    got = out32.cpu().numpy().T
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    if cout % 8 == 0:
        outb = torch.empty((V, cout), dtype=torch.bfloat16, device=DEV)
        capi.nn_check(L.reg_nn_conv3d_fwd(capi.ptr(xd), cin, capi.ptr(W), capi.ptr(bias), cout, d, 0, 0.2, wsp, nws,
                                          capi.ptr(outb), capi.stream_of(xd)), "fwd leaky")
        torch.cuda.synchronize()
        leaky = np.where(ref > 0, ref, 0.2 * ref)
        assert np.abs(outb.float().cpu().numpy() - leaky).max() <= 2 ** -7 * np.abs(leaky).max()
    assert capi.reg_get_device_error() == 0


# small volumes take the gather weight-gradient kernel; volumes with at
# least 76 tiles (here 77-80 planes) the persistent TMA-fed tensor-core one
# (one chunk, six chunks, 8 output channel groups)
@pytest.mark.parametrize("shape,cin,cout", [((9, 10, 11), 16, 16), ((6, 8, 7), 96, 32), ((4, 5, 6), 128, 64),
                                            ((5, 9, 12), 8, 16), ((80, 5, 24), 16, 16), ((78, 3, 10), 96, 32),
                                            ((77, 3, 8), 128, 64)])
def test_conv_gradients_match_oracle(capi, shape, cin, cout):
    L = capi.nn()
    rng = np.random.default_rng(3 * cin + cout)
    x = _bf(rng.standard_normal(shape + (cin,)))
    w = _bf(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin)).float().numpy()
    g = _bf(rng.standard_normal(shape + (cout,)))
    kpad = int(L.reg_nn_conv_kpad(cin))
    W = _pack_w(w, (cout + 15) // 16 * 16, kpad)
    d = capi.RegDims(shape[2], shape[1], shape[0])
    V = int(np.prod(shape))
    xd, gd = x.to(DEV).contiguous(), g.to(DEV).contiguous()
    wd = torch.empty(int(L.reg_nn_dgrad_scratch_bytes(cin, cout)), dtype=torch.uint8, device=DEV)
    din = torch.empty((V, cin), dtype=torch.bfloat16, device=DEV)
    capi.nn_check(L.reg_nn_conv3d_dgrad(capi.ptr(gd), cout, capi.ptr(W), cin, d, capi.ptr(wd), capi.ptr(din),
                                        capi.stream_of(gd)), "dgrad")
    ws = torch.empty(int(L.reg_nn_wgrad_scratch_bytes(d, cin, cout)), dtype=torch.uint8, device=DEV)
    dW = torch.empty((cout, kpad), dtype=torch.float32, device=DEV)
    capi.nn_check(L.reg_nn_conv3d_wgrad(capi.ptr(xd), cin, capi.ptr(gd), cout, d, capi.ptr(ws), ws.numel(),
                                        capi.ptr(dW), capi.stream_of(gd)), "wgrad")
    torch.cuda.synchronize()
    ref_din = O.conv3d_dgrad(g.float().numpy(), w).reshape(V, cin)
    assert np.abs(din.float().cpu().numpy() - ref_din).max() <= 2 ** -7 * np.abs(ref_din).max()
    ref_dw = O.conv3d_wgrad(x.float().numpy(), g.float().numpy()).reshape(cout, 27 * cin)
    got = dW.cpu().numpy()
    assert np.abs(got[:, :27 * cin] - ref_dw).max() <= 1e-4 * np.abs(ref_dw).max()
    assert not got[:, 27 * cin:].any()


# ---------------------------------------------------------------------------
# the whole network against the oracle's composition
# ---------------------------------------------------------------------------
BFR = 2.0 ** -8          # one round-to-nearest-even to BF16: |bf16(y) - y| <= 2^-8 |y|
U_TC = 2.0 ** -23        # unit roundoff of the tensor cores' FP32 accumulation (one bit
                         # looser than IEEE round-to-nearest: the adder need not round to nearest)


def _gamma(k, u=U_TC):
    return k * u / (1.0 - k * u)


def _w(net, name):
    """The layer's BF16 weights as the oracle's [Cout][27][Cin] and its bias."""
    P = net.p[name]
    w = P.wb.double().cpu().numpy()[:P.cout, :27 * P.cin].reshape(P.cout, 27, P.cin)
    return w, P.b.double().cpu().numpy()[:P.cout]


def _act(net, key, n):
    t = net.a[key]
    return t.double().cpu().numpy().reshape(n, n, n, -1)


def _within(got, ref, bound, what):
    err = np.abs(got - ref)
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} outside the bar; worst excess "
                           f"{float((err - bound).max()):.3e} (max |ref| {float(np.abs(ref).max()):.3e})")


def _oracle_forward(net, x0, n, round_bf16):
    """The U-Net forward composed from the oracle's operators in FP64, fed the
    network's BF16 weights; with round_bf16 every stored activation is rounded
    to BF16 as the GPU stores it (the head's output stays unrounded)."""
    from paper_2509_25044_gb300.unet import SLOPE
    r = O.bf16_round if round_bf16 else (lambda a: a)

    def conv(name, x, act=True):
        w, b = _w(net, name)
        y = O.conv3d(x, w, b)
        return r(O.leaky(y, SLOPE)) if act else y

    e0 = conv("c0b", conv("c0a", x0))
    e1 = conv("c1b", conv("c1a", r(O.avgpool2(e0))))
    e2 = conv("c2b", conv("c2a", r(O.avgpool2(e1))))
    b3 = conv("c3b", conv("c3a", r(O.avgpool2(e2))))
    d2 = conv("d2b", conv("d2a", O.concat(r(O.upsample(b3, 2)), e2)))
    d1 = conv("d1b", conv("d1a", O.concat(r(O.upsample(d2, 2)), e1)))
    return conv("head", d1, act=False)


def test_unet_matches_oracle_layer_by_layer_and_end_to_end(capi):
    """Every layer of the forward and backward pass against the oracle fed the
    network's own BF16 inputs of that layer, with bars derived from one BF16
    rounding of the output and the FP32 accumulation of its k terms:
    |got - ref| <= 2^-8 |ref| + (1 + 2^-8) gamma_k S, S the oracle's result on
    absolute values (Higham, Eq. 3.5); gradients that consumed a BF16-stored
    LeakyReLU derivative add 2^-8 S for that rounding.  Then the whole forward
    from the input alone: the GPU's output may differ from the FP64 oracle by
    at most twice the drift of an oracle that rounds every stored activation
    to BF16 (two pipelines with rounding errors of the same size)."""
    from paper_2509_25044_gb300.unet import LAYERS, SLOPE, UNet, training_pair
    n = 32
    h, q, e = n // 2, n // 4, n // 8
    net = UNet(n_in=n, seed=3, device=DEV)
    pair = training_pair(n, 5, DEV)
    net.pack(pair["F"], pair["M"], 1, (float(pair["F"].min()), float(pair["F"].max())),
             (float(pair["M"].min()), float(pair["M"].max())))
    u = net.forward().clone()
    torch.cuda.synchronize()
    A = {k: _act(net, k, m) for k, m in [("x0", n), ("c0a", n), ("e0", n), ("p0", h), ("c1a", h), ("e1", h),
                                         ("p1", q), ("c2a", q), ("e2", q), ("p2", e), ("c3a", e), ("b3", e),
                                         ("cat2", q), ("d2a", q), ("d2", q), ("cat1", h), ("d1a", h), ("d1", h)]}
    up2 = net.g["up"][:net.V[2]].double().cpu().numpy().reshape(q, q, q, 64)
    up1 = net._up1.double().cpu().numpy().reshape(h, h, h, 64)

    # ---- forward, layer by layer ----
    src = {"c0a": "x0", "c0b": "c0a", "c1a": "p0", "c1b": "c1a", "c2a": "p1", "c2b": "c2a", "c3a": "p2",
           "c3b": "c3a", "d2a": "cat2", "d2b": "d2a", "d1a": "cat1", "d1b": "d1a", "head": "d1"}
    dst = {"c0a": "c0a", "c0b": "e0", "c1a": "c1a", "c1b": "e1", "c2a": "c2a", "c2b": "e2", "c3a": "c3a",
           "c3b": "b3", "d2a": "d2a", "d2b": "d2", "d1a": "d1a", "d1b": "d1"}
    for name, cin, cout, _ in LAYERS:
        w, b = _w(net, name)
        x = A[src[name]]
        pre = O.conv3d(x, w, b)
        S = O.conv3d(np.abs(x), np.abs(w), np.abs(b))
        acc = _gamma(27 * cin + 1) * S
        if name == "head":
            _within(u.double().cpu().numpy().T.reshape(pre.shape), pre, acc, "head")
        else:
            ref = O.leaky(pre, SLOPE)
            _within(A[dst[name]], ref, BFR * np.abs(ref) + (1 + BFR) * acc, f"forward {name}")
    for coarse, fine in (("e0", "p0"), ("e1", "p1"), ("e2", "p2")):
        ref = O.avgpool2(A[coarse])
        _within(A[fine], ref, BFR * np.abs(ref) + (1 + BFR) * _gamma(8, 2.0 ** -24) * O.avgpool2(np.abs(A[coarse])),
                f"pool {coarse}")
    for low, upv, skip, cat in (("b3", up2, "e2", "cat2"), ("d2", up1, "e1", "cat1")):
        ref = O.upsample(A[low], 2)
        _within(upv, ref, BFR * np.abs(ref) + (1 + BFR) * _gamma(16, 2.0 ** -24) * O.upsample(np.abs(A[low]), 2),
                f"upsample {low}")
        np.testing.assert_array_equal(A[cat], O.concat(upv, A[skip]))

    # ---- forward from the input alone ----
    o64 = _oracle_forward(net, A["x0"], n, False)
    obf = _oracle_forward(net, A["x0"], n, True)
    ug = u.double().cpu().numpy().T.reshape(o64.shape)
    drift = float(np.linalg.norm(obf - o64) / np.linalg.norm(o64))
    err = float(np.linalg.norm(ug - o64) / np.linalg.norm(o64))
    print(f"U-Net output vs FP64 oracle: GPU {err:.3e}, BF16-storing oracle {drift:.3e}")
    assert err <= 2.0 * drift + 1e-6

    # ---- backward, layer by layer ----
    target = torch.randn((3, h ** 3), device=DEV) * 0.1
    loss = net.loss_and_backward(target)
    torch.cuda.synchronize()
    lref, dpred = O.mse(u.double().cpu().numpy(), target.double().cpu().numpy())
    assert abs(loss.item() - lref) <= 1e-6 * lref
    G = {k: net.g[k].double().cpu().numpy() for k in ("d1", "d1a", "d2", "d2a", "b3", "c3a", "p2", "e2", "c2a",
                                                       "p1", "e1", "c1a", "p0", "e0", "c0a")}
    grid = {0: n, 1: h, 2: q, 3: e}
    outgrad = {"d1b": "d1", "d1a": "d1a", "d2b": "d2", "d2a": "d2a", "c3b": "b3", "c3a": "c3a", "c2b": "e2",
               "c2a": "c2a", "c1b": "e1", "c1a": "c1a", "c0b": "e0", "c0a": "c0a"}
    dxname = {"head": "d1", "d1b": "d1a", "d2b": "d2a", "c3b": "c3a", "c3a": "p2", "c2b": "c2a", "c2a": "p1",
              "c1b": "c1a", "c1a": "p0", "c0b": "c0a"}
    dcat = {}
    for name, cin, cout, lv in LAYERS:
        m = grid[lv]
        w, _ = _w(net, name)
        x = A[src[name]]
        V = m ** 3
        if name == "head":
            dpre = dpred.T.reshape(m, m, m, 3)
            store = BFR + 4 * 2.0 ** -24  # 2 (pred - target) / (3V) in FP32, stored in BF16
        else:
            dout = G[outgrad[name]].reshape(m, m, m, cout)
            dpre = O.leaky_bwd(A[dst[name]], dout, SLOPE)
            store = BFR + 2.0 ** -24  # FP32 product, BF16 store
        P = net.p[name]
        gw = P.gw.double().cpu().numpy()[:cout, :27 * cin].reshape(cout, 27, cin)
        ref = O.conv3d_wgrad(x, dpre)
        S = O.conv3d_wgrad(np.abs(x), np.abs(dpre))
        _within(gw, ref, (_gamma(V) + store) * S, f"weight gradient {name}")
        gb = P.gb.double().cpu().numpy()[:cout]
        _within(gb, dpre.reshape(V, cout).sum(0), (V * 2.0 ** -53 + store) * np.abs(dpre).reshape(V, cout).sum(0),
                f"bias gradient {name}")
        if name == "c0a":
            continue
        ref = O.conv3d_dgrad(dpre, w)
        S = O.conv3d_dgrad(np.abs(dpre), np.abs(w))
        bound = BFR * np.abs(ref) + (1 + BFR) * (_gamma(27 * cout) + store) * S
        if name in ("d1a", "d2a"):  # their input gradient is split and consumed below
            dcat[name] = (ref, bound)
            continue
        _within(G[dxname[name]].reshape(ref.shape), ref, bound, f"data gradient {name}")
    # split of the concat gradients, upsampling and pooling adjoints
    for conv_name, low, skip, pool_src in (("d1a", "d2", "e1", "p1"), ("d2a", "b3", "e2", "p2")):
        ref, bound = dcat[conv_name]
        up_ref = O.upsample_adjoint(ref[..., :64], 2)
        up_bound = O.upsample_adjoint(bound[..., :64], 2) + _gamma(128, 2.0 ** -24) * \
            O.upsample_adjoint(np.abs(ref[..., :64]) + bound[..., :64], 2)
        _within(G[low].reshape(up_ref.shape), up_ref, BFR * np.abs(up_ref) + (1 + BFR) * up_bound,
                f"upsample adjoint into {low}")
        m = ref.shape[0]
        pg = G[pool_src].reshape(m // 2, m // 2, m // 2, -1)
        pool_adj = O.avgpool2_adjoint(pg, (m, m, m))  # exact on the GPU too: a power-of-two scale
        skip_ref = ref[..., 64:] + pool_adj
        # the stored skip part of the concat gradient plus the pooling adjoint, one FP32 add
        skip_bound = bound[..., 64:] + 2.0 ** -24 * (np.abs(ref[..., 64:]) + np.abs(pool_adj))
        _within(G[skip].reshape(skip_ref.shape), skip_ref, BFR * np.abs(skip_ref) + (1 + BFR) * skip_bound,
                f"skip gradient {skip}")
    ref = O.avgpool2_adjoint(G["p0"].reshape(h, h, h, 16), (n, n, n))
    _within(G["e0"].reshape(ref.shape), ref, BFR * np.abs(ref), "pool adjoint into e0")
    assert capi.reg_get_device_error() == 0


def test_unet_training_reduces_loss(capi):
    from paper_2509_25044_gb300.unet import UNet, training_pair
    n = 32
    net = UNet(n_in=n, seed=1, device=DEV)
    pairs = [training_pair(n, 100 + i, DEV) for i in range(4)]
    tgts = []
    for p in pairs:
        t = torch.empty((3, (n // 2) ** 3), device=DEV)
        capi.nn_check(net.L.reg_nn_field_down2(capi.ptr(p["v"]), capi.RegDims(n, n, n), capi.ptr(t),
                                               capi.stream_of(t)), "down2")
        tgts.append(t)
    losses = []
    for epoch in range(80):
        tot = 0.0
        for p, t in zip(pairs, tgts):
            net.pack(p["F"], p["M"], 1, (float(p["F"].min()), float(p["F"].max())),
                     (float(p["M"].min()), float(p["M"].max())))
            net.forward()
            tot += net.loss_and_backward(t).item()
            net.step(2e-4)
        losses.append(tot / len(pairs))
    # memorising 4 pairs (Adam at 2e-4 is stable here; 1e-3 diverges): the
    # loss roughly halves within 80 epochs
    assert losses[-1] < 0.6 * losses[0], [round(v, 4) for v in losses]
    assert np.mean(losses[-5:]) < 0.7 * np.mean(losses[:5]), [round(v, 4) for v in losses]


def test_predict_init_scales_each_image_by_its_pooled_range(capi):
    """A pair larger than the network input is pooled first; the network then
    sees each image scaled by the range of the pooled grid (the scaling it was
    trained with), not by the range of the full-resolution image, whose noise
    tails pooling removes.  The packed input must equal the oracle's pack of
    the same pair with the pooled ranges the oracle computes."""
    from paper_2509_25044_gb300.unet import UNet
    rng = np.random.default_rng(29)
    n_in, factor = 32, 2
    shape = (n_in * factor,) * 3
    # a smooth ramp under heavy noise: pooling narrows the range markedly
    ramp = np.linspace(0.0, 1.0, shape[2])[None, None, :]
    F = (ramp + rng.normal(0.0, 0.3, shape)).astype(np.float32)
    M = (1.0 - ramp + rng.normal(0.0, 0.2, shape)).astype(np.float32)
    fr, mr = (float(F.min()), float(F.max())), (float(M.min()), float(M.max()))
    net = UNet(n_in=n_in, seed=0, device=DEV)
    net.predict_init(torch.from_numpy(F).to(DEV), torch.from_numpy(M).to(DEV), fr, mr)
    torch.cuda.synchronize()
    got = net.a["x0"].double().cpu().numpy().reshape((n_in,) * 3 + (16,))[..., :2]

    pF = O.avgpool2(F[..., None])[..., 0]
    pM = O.avgpool2(M[..., None])[..., 0]
    pr = [(float(pF.min()), float(pF.max())), (float(pM.min()), float(pM.max()))]
    assert pr[0][1] - pr[0][0] < 0.8 * (fr[1] - fr[0])  # the case exercises a narrower pooled range
    ref = O.pack_pair(F, M, factor, pr[0], pr[1])
    # The pooled range is read back from the first (full-range) pack, whose
    # values are BF16: its ends carry 2^-9 |e| of the full width, e in units of
    # it.  A packed value y moves by at most that over the pooled width.  Then
    # the pack's own bar: one BF16 rounding, and an FP32 8-term block mean.
    bars = []
    for c, (full, pooled) in enumerate(zip((fr, mr), pr)):
        fw, pw = full[1] - full[0], pooled[1] - pooled[0]
        ends = max(abs(pooled[0] - full[0]), abs(pooled[1] - full[0])) / fw
        bars.append(2.0 ** -9 * ends * fw / pw * (1 + 2.0 ** -8) + 2.0 ** -8 * np.abs(ref[..., c])
                    + 16 * 2.0 ** -24 * (np.abs(ref[..., c]) + 2.0 * max(abs(full[0]), abs(full[1])) / pw))
    for c in range(2):
        err = np.abs(got[..., c] - ref[..., c])
        assert (err <= bars[c]).all(), (c, float((err - bars[c]).max()))
