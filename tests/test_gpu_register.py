"""The registration driver on the small mono-modal and multimodal workloads:
the objective decreases, the field does not fold, and a replay is bitwise
identical."""
import numpy as np
import pytest
import torch

from paper_2509_25044_gb300 import synth
from paper_2509_25044_gb300.register import RegConfig, Registration, register

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_c0_lncc_converges_without_folding():
    d = synth.make("c0", device=DEV)
    # lam = 2: with the noise texture shared by F and M, lam = 1 folds a voxel or two
    cfg = RegConfig(loss="lncc", window=7, eps=1e-9, lam=2.0, lr=0.1)
    res = register(d["F"], d["M"], cfg, 50)
    assert np.all(np.isfinite(res.objective))
    assert res.objective[-1] < res.objective[0]
    assert res.extra["min_det"] > 0 and res.extra["n_fold"] == 0
    again = register(d["F"], d["M"], cfg, 50)
    assert torch.equal(res.u, again.u)


def test_c1_mi_small_converges():
    d = synth.make("c1", device=DEV, n=64)
    # lam = 2: at lam = 1 the MI run folds a few voxels of the 64^3 grid
    cfg = RegConfig(loss="mi", bins=32, f_range=d["f_range"], m_range=d["m_range"], lam=2.0, lr=0.1)
    reg = Registration(d["F"], d["M"], cfg)
    res = reg.run(60)
    assert res.objective[-1] < res.objective[0]  # MI increases: -MI + lam R decreases
    assert res.sim[-1] > res.sim[0]
    assert reg.fold_check()["n_fold"] == 0


def test_multiscale_schedule():
    """Coarse-to-fine (scales 4, 2, 1): every level decreases its objective,
    the returned field is full size, and its full-resolution objective is
    below the objective at zero displacement."""
    from paper_2509_25044_gb300.register import register_multiscale
    d = synth.make("c0", device=DEV)
    cfg = RegConfig(loss="lncc", window=7, eps=1e-9, lam=2.0, lr=0.1)
    out = register_multiscale(d["F"], d["M"], cfg, scales=(4, 2, 1), iters=(30, 30, 30))
    assert [lv["scale"] for lv in out["levels"]] == [4, 2, 1]
    n = tuple(d["F"].shape)
    assert [lv["shape"] for lv in out["levels"]] == [tuple(s // 4 for s in n), tuple(s // 2 for s in n), n]
    for lv in out["levels"]:
        obj = lv["result"].objective
        assert np.all(np.isfinite(obj)) and obj[-1] < obj[0]
    assert tuple(out["u"].shape) == (3,) + n
    r = Registration(d["F"], d["M"], cfg)
    zero = r.objective()["objective"]
    fin = Registration(d["F"], d["M"], cfg, u0=out["u"]).objective()["objective"]
    assert fin < zero
    assert out["ms"] > 0
    with pytest.raises(ValueError):
        register_multiscale(d["F"], d["M"], cfg, scales=(2, 4, 1), iters=(1, 1, 1))


def test_affine_stage_recovers_known_map():
    """Multi-modal pair related by a known affine map (rotation about two
    axes, anisotropic scale, shift): the multi-scale MI affine stage on the
    composite sampler recovers the map to well under a voxel."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _util import multimodal_images
    from paper_2509_25044_gb300 import capi
    from paper_2509_25044_gb300.register import affine_about_centre, register_affine
    shape = (64, 64, 64)
    F, Mbase = multimodal_images(shape, 41)
    a, b = 0.07, 0.035
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    A_true, t_true = affine_about_centre(Rz @ Rx @ np.diag([1.04, 0.97, 1.02]), (2.5, -1.5, 1.0), shape)
    Ai = np.linalg.inv(A_true)
    M = capi.reg_warp_composite(Mbase.to(DEV), capi.affine_desc(Ai, -Ai @ t_true))
    cfg = RegConfig(loss="mi", bins=32, m_range=(float(M.min()), float(M.max())))
    out = register_affine(F.to(DEV), M, cfg, scales=(4, 2, 1), iters=(100, 60, 40))
    for lv in out["levels"]:
        assert np.all(np.isfinite(lv["objective"])) and lv["objective"][-1] < lv["objective"][0]
    from oracle import identity_grid
    X = identity_grid(shape).reshape(3, -1)
    err = np.linalg.norm((out["A"] - A_true) @ X + (out["t"] - t_true)[:, None], axis=0)
    err0 = np.linalg.norm((np.eye(3) - A_true) @ X - t_true[:, None], axis=0)
    assert err0.mean() > 2.0
    # the map is recovered to a fraction of the initial misalignment, and the
    # optimiser reaches the MI optimum: the objective there is no worse than
    # at the generating map (double trilinear resampling and independent
    # noise leave the optimum a few tenths of a voxel from that map)
    assert err.mean() < 0.6 and err.mean() < 0.2 * err0.mean(), (err.mean(), err.max())
    loss = cfg.loss_desc(F)

    def C(A, t):
        sim = capi.reg_loss_grad_composite(loss, F.to(DEV), M, capi.affine_desc(A, t), None, need_u=False,
                                           need_affine=False)[0]
        return -float(sim[0].item())

    assert C(out["A"], out["t"]) <= C(A_true, t_true) + 1e-3, (C(out["A"], out["t"]), C(A_true, t_true))


def test_svf_registration_folds_far_less():
    """Stationary velocity field registration (u = exp(v) by scaling and
    squaring, the gradient pulled back through every squaring step): with no
    regulariser, where the plain displacement run folds over 10 % of the
    voxels, the exponential folds at least 10x fewer (the continuous map is
    invertible; the discrete squaring of an unregularised, rough v keeps a
    few folds) while the objective decreases."""
    from paper_2509_25044_gb300 import capi
    from paper_2509_25044_gb300.register import register_svf
    d = synth.make("c0", device=DEV)
    cfg = RegConfig(loss="lncc", window=7, eps=1e-9, lam=0.0, lr=0.1)
    plain = Registration(d["F"], d["M"], cfg)
    plain.run(50)
    out = register_svf(d["F"], d["M"], cfg, 50, steps=6)
    obj = out["objective"]
    assert np.all(np.isfinite(obj)) and obj[-1] < obj[0] - 0.05
    _, nf = capi.reg_jacdet_min(out["u"])
    folds_plain = plain.fold_check()["n_fold"]
    assert folds_plain > 0.1 * d["F"].numel()
    assert 10 * int(nf.item()) <= folds_plain, (int(nf.item()), folds_plain)
    assert capi.reg_get_device_error() == 0


@pytest.mark.parametrize("kind", ["lncc", "mi"])
def test_composite_gradient_with_the_transform_in_device_memory(kind):
    """reg_loss_grad_composite_dev (transform read by the kernels from device
    memory) gives the same bits as reg_loss_grad_composite (transform passed by
    value) for the same map."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _util import mono_images, multimodal_images
    from paper_2509_25044_gb300 import capi
    shape = (20, 24, 28)
    F, M = (mono_images if kind == "lncc" else multimodal_images)(shape, 7)
    Fd, Md = F.to(DEV), M.to(DEV)
    A = np.array([[1.02, 0.03, -0.01], [-0.02, 0.98, 0.04], [0.01, -0.03, 1.01]], dtype=np.float32)
    t = np.array([0.7, -1.2, 0.4], dtype=np.float32)
    if kind == "lncc":
        loss = capi.lncc_desc(5, 1e-5)
    else:
        loss = capi.mi_desc((float(F.min()), float(F.max())), (float(M.min()), float(M.max())), 32)
    u = torch.randn((3,) + shape, device=DEV) * 0.5
    s1, gu1, ga1 = capi.reg_loss_grad_composite(loss, Fd, Md, capi.affine_desc(A, t), u)
    T = torch.tensor(np.concatenate([A.reshape(9), t, np.ones(3, dtype=np.float32)]), device=DEV)
    s2, gu2, ga2 = capi.reg_loss_grad_composite_dev(loss, Fd, Md, T, u)
    torch.cuda.synchronize()
    assert torch.equal(s1[:1], s2[:1]) and torch.equal(gu1, gu2) and torch.equal(ga1, ga2)


def test_affine_stage_on_the_device_matches_the_host_optimiser():
    """The affine stage with its 12-parameter Adam on the device (two launches
    per iteration, no host round trip) follows the host optimiser: the same
    transforms within FP64 rounding, the same objective histories, and it
    runs faster."""
    import sys, os, time
    sys.path.insert(0, os.path.dirname(__file__))
    from _util import multimodal_images
    from paper_2509_25044_gb300 import capi
    from paper_2509_25044_gb300.register import affine_about_centre, register_affine
    shape = (48, 48, 48)
    F, Mbase = multimodal_images(shape, 43)
    A_true, t_true = affine_about_centre(np.diag([1.03, 0.98, 1.01]), (1.5, -1.0, 0.5), shape)
    Ai = np.linalg.inv(A_true)
    M = capi.reg_warp_composite(Mbase.to(DEV), capi.affine_desc(Ai, -Ai @ t_true))
    cfg = RegConfig(loss="mi", bins=32, m_range=(float(M.min()), float(M.max())))
    Fd = F.to(DEV)
    kw = dict(scales=(4, 2, 1), iters=(40, 30, 20))
    register_affine(Fd, M, cfg, on_device=True, **kw)  # warm-up (first launches, workspaces)
    times = {}
    outs = {}
    for dev_path in (False, True):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs[dev_path] = register_affine(Fd, M, cfg, on_device=dev_path, **kw)
        torch.cuda.synchronize()
        times[dev_path] = time.perf_counter() - t0
    print(f"affine stage, 90 iterations: host optimiser {1e3 * times[False]:.1f} ms, "
          f"device optimiser {1e3 * times[True]:.1f} ms")
    h, d = outs[False], outs[True]
    np.testing.assert_allclose(d["A"], h["A"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(d["t"], h["t"], rtol=0, atol=1e-4)
    for lh, ld in zip(h["levels"], d["levels"]):
        np.testing.assert_allclose(ld["objective"], lh["objective"], rtol=1e-6, atol=1e-9)
    assert times[True] < times[False]


def test_run_records_three_events_per_iteration():
    """The timing hook armed with three events per iteration is taken by a
    reg_run call of that many iterations: each iteration's events are recorded
    in order (first sweep, second sweep), the spans add up to no more than the
    whole call, and the hook is spent afterwards (a second call records
    nothing new)."""
    from paper_2509_25044_gb300 import capi
    capi.load()
    n, iters = 48, 4
    gen = torch.Generator(device=DEV).manual_seed(2)
    F = torch.rand((n, n, n), generator=gen, device=DEV)
    M = torch.rand((n, n, n), generator=gen, device=DEV)
    loss = capi.mi_desc((0.0, 1.0), (0.0, 1.0), 32)
    adam = capi.adam_desc(0.05, grad_scale=float(F.numel()))
    ws = capi.workspace(loss, F)
    u = [torch.zeros((3, n, n, n), device=DEV) for _ in range(2)]
    m, v = torch.zeros_like(u[0]), torch.zeros_like(u[0])
    s = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3 * iters)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    capi.reg_set_timing_events(evs)  # creates the events (a first record) and arms the hook
    start.record(s)
    capi.reg_run(loss, F, M, u[0], u[1], m, v, 0.5, adam, 0, iters, ws)
    end.record(s)
    torch.cuda.synchronize()
    # every event was recorded by the call (after `start`), in stream order
    assert all(start.elapsed_time(e) >= 0.0 for e in evs)
    spans = [evs[k].elapsed_time(evs[k + 1]) for k in range(3 * iters - 1)]
    assert all(t >= 0.0 for t in spans)
    assert sum(spans) <= start.elapsed_time(end) + 1e-3
    assert evs[0].elapsed_time(evs[-1]) > 0.0
    # spent: a further call does not re-record the events
    last = evs[-1].elapsed_time(end)
    capi.reg_run(loss, F, M, u[0], u[1], m, v, 0.5, adam, iters, iters, ws)
    torch.cuda.synchronize()
    assert evs[-1].elapsed_time(end) == last
    assert capi.reg_get_device_error() == 0
