"""Host-side arithmetic of the registration drivers, checked on the CPU with
the oracle's similarity: the affine stage's centred parametrisation (the
volume centre c, phi(p) = A (p - c) + c + tc / s at pyramid scale s) and its
conversion back to phi(p) = A p + t."""
import numpy as np
import pytest

import oracle as O
from paper_2509_25044_gb300.register import _centre, affine_about_centre, centred_affine_grads


@pytest.mark.parametrize("s", [1, 2])
def test_centred_affine_gradients_match_central_differences(rng, s):
    from scipy.ndimage import gaussian_filter
    shape = (10, 11, 12)
    F = gaussian_filter(rng.standard_normal(shape), 1.5)
    M = gaussian_filter(rng.standard_normal(shape), 1.5)
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=3, eps=1e-3)
    c = _centre(shape)
    A0 = np.eye(3) + 0.03 * rng.standard_normal((3, 3))
    tc0 = rng.uniform(-1.0, 1.0, 3)

    def cost(A, tc):
        S = O.similarity_and_grad_composite(F, M, A, c - A @ c + tc / s, spec=spec)[0]
        return 1.0 - S

    _, _, gA, gt = O.similarity_and_grad_composite(F, M, A0, c - A0 @ c + tc0 / s, spec=spec)
    gAc, gtc = centred_affine_grads(gA, gt, c, s)
    h = 1e-7
    fd_A = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            fd_A[i, j] = (cost(A0 + E, tc0) - cost(A0 - E, tc0)) / (2 * h)
    fd_t = np.array([(cost(A0, tc0 + h * e) - cost(A0, tc0 - h * e)) / (2 * h) for e in np.eye(3)])
    scale = max(np.abs(fd_A).max(), np.abs(fd_t).max())
    np.testing.assert_allclose(gAc, fd_A, rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(gtc, fd_t, rtol=0, atol=1e-5 * scale)
    # the uncentred gradient differs: the centring is not a no-op here
    assert np.abs(gA - fd_A).max() > 1e-3 * scale


def test_affine_about_centre_is_the_same_map(rng):
    shape = (9, 14, 20)
    c = _centre(shape)
    assert np.allclose(c, [9.5, 6.5, 4.0])  # (x, y, z) centre of [nz][ny][nx]
    A = np.eye(3) + 0.1 * rng.standard_normal((3, 3))
    tc = rng.uniform(-3.0, 3.0, 3)
    A2, t = affine_about_centre(A, tc, shape)
    p = rng.uniform(0.0, 20.0, (3, 50))
    np.testing.assert_allclose(A2 @ p + t[:, None], A @ (p - c[:, None]) + c[:, None] + tc[:, None], atol=1e-12)


def test_multiscale_schedule_is_validated_before_any_launch():
    """Scales must decrease to 1, one iteration count per scale, and u0 lives
    on the coarsest level's grid: each is rejected on the host."""
    import torch
    from paper_2509_25044_gb300.register import RegConfig, register_multiscale
    F = M = torch.zeros(16, 16, 16)
    cfg = RegConfig(loss="lncc")
    with pytest.raises(ValueError, match="decrease"):
        register_multiscale(F, M, cfg, scales=(2, 4, 1), iters=(1, 1, 1))
    with pytest.raises(ValueError, match="decrease"):
        register_multiscale(F, M, cfg, scales=(4, 2), iters=(1, 1))
    with pytest.raises(ValueError, match="one iteration count"):
        register_multiscale(F, M, cfg, scales=(4, 2, 1), iters=(1, 1))
    with pytest.raises(ValueError, match="coarsest"):
        register_multiscale(F, M, cfg, scales=(4, 2, 1), iters=(1, 1, 1), u0=torch.zeros(3, 16, 16, 16))


def test_mi_ranges_default_to_each_images_own():
    import torch
    from paper_2509_25044_gb300.register import RegConfig
    F = torch.linspace(-2.0, 3.0, 64).reshape(4, 4, 4)
    M = torch.linspace(10.0, 50.0, 64).reshape(4, 4, 4)
    d = RegConfig(loss="mi", bins=16).loss_desc(F, M)
    assert (d.f_lo, d.f_hi, d.m_lo, d.m_hi, d.bins) == (-2.0, 3.0, 10.0, 50.0, 16)
    d = RegConfig(loss="mi", m_range=(0.0, 60.0)).loss_desc(F, M)
    assert (d.m_lo, d.m_hi) == (0.0, 60.0)


def test_experiment_helpers():
    """Time-to-target takes the first iterate within tol of the target; the
    workload configurations map to the registration settings they state."""
    from paper_2509_25044_gb300 import synth
    from paper_2509_25044_gb300.experiments import LNCC_EPS, _cfg, _first_within
    assert _first_within([5.0, 3.0, 2.05, 1.0], 2.0, 0.1) == 2
    assert _first_within([5.0, 3.0], 2.0, 0.1) is None
    c0 = _cfg(synth.CONFIGS["c0"], {}, "f32", lam_scale=2.0)
    assert (c0.loss, c0.window, c0.eps, c0.lam, c0.moments) == ("lncc", 7, LNCC_EPS, 0.2, "f32")
    c1 = _cfg(synth.CONFIGS["c1"], {"f_range": (0.0, 1.0), "m_range": (0.1, 0.9)}, "bf16")
    assert (c1.loss, c1.bins, c1.m_range, c1.lam, c1.moments) == ("mi", 32, (0.1, 0.9), 0.05, "bf16")
