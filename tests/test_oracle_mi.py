"""Pins for the oracle's Parzen mutual information (Sec. 2.2 Eq. mi; App.
fused MI, Eq. gradientmi-threadn).  CPU only."""
import math

import numpy as np
import pytest

import oracle as O

B = 32


def _bin_value(s, bins=B):
    """Intensity whose bin coordinate is s (the kernel of bin m is centred at s = m)."""
    return (s - 1.0) / (bins - 3)


def test_kernel_equals_scipy_cardinal_cubic_bspline():
    from scipy.interpolate import BSpline
    ref = BSpline.basis_element([0, 1, 2, 3, 4], extrapolate=False)
    for t in np.linspace(-2.5, 2.5, 101):
        expect = ref(t + 2.0)
        expect = 0.0 if np.isnan(expect) else float(expect)
        assert abs(O.bspline3(t) - expect) < 1e-14
        d = ref.derivative()(t + 2.0)
        d = 0.0 if np.isnan(d) else float(d)
        assert abs(O.bspline3_deriv(t) - d) < 1e-12


def test_kernel_is_partition_of_unity():
    for s in np.linspace(1.0, B - 2.0, 77):
        tot = sum(O.bspline3(s - m) for m in range(B))
        dtot = sum(O.bspline3_deriv(s - m) for m in range(B))
        assert abs(tot - 1.0) < 1e-14 and abs(dtot) < 1e-13


def test_joint_histogram_sums_to_one(rng):
    Fh = rng.random(5000)
    Jh = rng.random(5000)
    Fh[:3] = [0.0, 1.0, 0.5]
    Jh[:3] = [1.0, 0.0, 0.0]
    v, p = O.mi(Fh, Jh, B, with_hist=True)
    assert abs(p.sum() - 1.0) < 1e-12
    assert (p >= 0).all()


def test_constant_moving_image_has_zero_mi(rng):
    Fh = rng.random(4000)
    assert abs(O.mi(Fh, np.full(4000, 0.37), B)) < 1e-14


def test_symmetry_and_entropy_bound(rng):
    Fh = rng.random(6000)
    Jh = np.clip(Fh ** 2 + 0.1 * rng.standard_normal(6000), 0, 1)
    v1, p = O.mi(Fh, Jh, B, with_hist=True)
    v2 = O.mi(Jh, Fh, B)
    assert abs(v1 - v2) < 1e-13
    pI, pJ = p.sum(1), p.sum(0)
    H = lambda q: -sum(x * math.log(x) for x in q if x > 0)
    assert 0.0 <= v1 <= min(H(pI), H(pJ)) + 1e-13


def test_closed_form_two_separated_modes_identical():
    """F = J taking two values whose kernels do not overlap, half the voxels
    each: p_IJ is 0.5 w w^T around each mode and p_I = p_J = 0.5 w there, so
    p_IJ / (p_I p_J) = 2 on the support and MI = log 2 exactly."""
    a, b = _bin_value(5.0), _bin_value(20.0)
    Fh = np.array([a, b] * 500)
    assert abs(O.mi(Fh, Fh, B) - math.log(2.0)) < 1e-13


def test_closed_form_independent_modes():
    """Four equally frequent combinations of two separated F modes and two
    separated J modes: p_IJ = p_I p_J, so MI = 0."""
    a, b = _bin_value(4.3), _bin_value(17.6)
    c, d = _bin_value(8.2), _bin_value(24.9)
    Fh = np.array([a, a, b, b] * 300)
    Jh = np.array([c, d, c, d] * 300)
    assert abs(O.mi(Fh, Jh, B)) < 1e-14


def test_streaming_equals_materialised_parzen_block(rng):
    """The O(1)-memory accumulation equals the vanilla form p = Psi_I Psi_J^T / N
    with the Parzen blocks Psi(m, k) = kappa(s_k - m) materialised (Sec. 2.2)."""
    N = 300
    Fh, Jh = rng.random(N), rng.random(N)
    sF, sJ = Fh * (B - 3) + 1, Jh * (B - 3) + 1
    PF = np.array([[O.bspline3(sF[k] - m) for k in range(N)] for m in range(B)])
    PJ = np.array([[O.bspline3(sJ[k] - m) for k in range(N)] for m in range(B)])
    ref = PF @ PJ.T / N
    _, p = O.mi(Fh, Jh, B, with_hist=True)
    np.testing.assert_allclose(p, ref, atol=1e-15)


def test_gradient_wrt_Jh_matches_central_differences(rng):
    N = 2000
    Fh = rng.uniform(0.02, 0.98, N)
    Jh = np.clip(0.6 * Fh + 0.3 * rng.random(N), 0.01, 0.99)
    v, g = O.mi_grad(Fh, Jh, B)
    # the kernel is a cubic inside each knot interval, so the central
    # difference has no truncation error there; h only trades rounding noise.
    h = 1e-5
    for k in rng.integers(0, N, 25):
        Jp = Jh.copy()
        Jp[k] += h
        Jm = Jh.copy()
        Jm[k] -= h
        fd = -(O.mi(Fh, Jp, B) - O.mi(Fh, Jm, B)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-12, (k, g[k], fd)


def test_full_chain_gradient_wrt_u_matches_central_differences(rng):
    """dC/du through warp + normalisation + MI at 16^3, FP64, rel 1e-6."""
    from scipy.ndimage import gaussian_filter
    n = 16
    F = gaussian_filter(rng.random((n, n, n)), 1.0)
    M = np.cos(3 * F) + 0.05 * rng.random((n, n, n))
    u = rng.integers(-1, 2, (3, n, n, n)) + rng.uniform(0.1, 0.9, (3, n, n, n))
    spec = O.LossSpec(kind=O.LOSS_MI, bins=B, f_range=(F.min(), F.max()),
                      m_range=(M.min() - 0.01, M.max() + 0.01))
    v, g = O.similarity_and_grad(F, M, u, spec)
    h = 1e-4
    rms = float(np.sqrt(np.mean(g ** 2)))
    errs = []
    for _ in range(24):
        k = (rng.integers(0, 3),) + tuple(rng.integers(2, n - 2, 3))
        up = u.copy()
        up[k] += h
        um = u.copy()
        um[k] -= h
        vp, _ = O.similarity_and_grad(F, M, up, spec, need_grad=False)
        vm, _ = O.similarity_and_grad(F, M, um, spec, need_grad=False)
        fd = -(vp - vm) / (2 * h)
        # relative to the entry, with a floor at a tenth of the field's RMS so
        # that entries near zero are compared on the FD rounding noise scale
        errs.append(abs(g[k] - fd) / (abs(fd) + 0.1 * rms))
    assert max(errs) < 1e-6, errs


# ---- the hard-binned (approximate) estimator of App. fused MI -----------------
def _snap(v, rng_, B):
    """intensity of the bin centre nearest to v (the estimator's own rule,
    taken in FP32 as the library takes it)"""
    lo, hi = np.float32(rng_[0]), np.float32(rng_[1])
    scale = np.float32(1.0 / (float(hi) - float(lo)))
    t = np.clip((v.astype(np.float32) - lo) * scale, np.float32(0), np.float32(1))
    s = (t.astype(np.float64) * (B - 3) + 1.0).astype(np.float32)
    m = np.clip(np.floor(s + np.float32(0.5)), 1, B - 2).astype(np.float64)
    return float(lo) + (m - 1.0) / (B - 3) * (float(hi) - float(lo))


@pytest.mark.parametrize("B", [8, 32])
def test_hard_binned_equals_parzen_on_bin_centres(rng, B):
    """The estimator is exact for samples on bin centres (App. fused MI): the
    hard-binned MI of (F, J) is the Parzen MI of the snapped intensities, and
    its PMF sums to 1."""
    F = rng.random((9, 10, 11)) * 3.0 - 1.0
    J = 0.5 * F + rng.random((9, 10, 11))
    # ranges representable in FP32, so the snapped centres sit exactly on s = m
    fr, jr = (-1.0, 2.0), (float(np.float32(J.min() - 0.01)), float(np.float32(J.max() + 0.01)))
    v, p = O.mi_hard(F, J, B, fr, jr, with_hist=True)
    assert abs(p.sum() - 1.0) < 1e-12
    Fs, Js = _snap(F, fr, B), _snap(J, jr, B)
    ref = O.mi(O.normalize(Fs, *fr)[0], O.normalize(Js, *jr)[0], B)
    assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref))
    # the paired gradient is the Parzen adjoint with the approximate table:
    # on snapped samples it equals the Parzen gradient
    _, gh = O.mi_hard_grad(Fs, Js, B, fr, jr)
    _, gp = O.mi_grad(O.normalize(Fs, *fr)[0], O.normalize(Js, *jr)[0], B)
    np.testing.assert_allclose(gh.ravel(), gp.ravel(), rtol=1e-9, atol=1e-12 * np.abs(gp).max())


def test_hard_binned_symmetry_and_constant(rng):
    F = rng.random((8, 8, 8))
    J = np.sqrt(F) + 0.1 * rng.random((8, 8, 8))
    a = O.mi_hard(F, J, 16, (0.0, 1.0), (0.0, 1.2))
    b = O.mi_hard(J, F, 16, (0.0, 1.2), (0.0, 1.0))
    assert abs(a - b) < 1e-12
    assert abs(O.mi_hard(F, np.full_like(F, 0.3), 16, (0.0, 1.0), (0.0, 1.0))) < 1e-12
    # an approximation of the Parzen value on continuous intensities
    ref = O.mi(F, np.clip(J / 1.2, 0, 1), 16)
    assert abs(a - ref) < 0.1 * ref


def test_hard_binned_gradient_uses_the_hard_pmf(rng):
    """Off the bin centres the two PMFs differ, and the hard-binned gradient
    is the Parzen adjoint (Eq. gradientmi-threadn) taken with the hard
    estimator's own PMF, not with the Parzen one."""
    B = 16
    F = rng.random((7, 8, 9))
    J = np.sqrt(F) + 0.1 * rng.random((7, 8, 9))
    fr, jr = (0.0, 1.0), (0.0, 1.2)
    _, p_hard = O.mi_hard(F, J, B, fr, jr, with_hist=True)
    _, g = O.mi_hard_grad(F, J, B, fr, jr)
    Fh, Jh = O.normalize(F, *fr)[0].ravel(), O.normalize(J, *jr)[0].ravel()
    ref = O.mi_adjoint_points(Fh, Jh, Fh.size, B, p_hard)
    np.testing.assert_allclose(g.ravel(), ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())
    _, g_parzen = O.mi_grad(Fh, Jh, B)
    assert np.abs(g.ravel() - g_parzen).max() > 1e-3 * np.abs(g_parzen).max()


def test_per_point_adjoint_and_pmf_mi_match_the_whole_volume_forms(rng):
    """The per-voxel adjoint for a given PMF and the MI of a given PMF (used
    for sampled checks of volumes too large for the oracle's own histogram)
    agree with mi_grad / mi on a whole volume."""
    N, B = 3000, 16
    Fh = rng.uniform(0, 1, N)
    Jh = np.clip(Fh + 0.2 * rng.standard_normal(N), 0, 1)
    v, p = O.mi(Fh, Jh, B, with_hist=True)
    v2, g = O.mi_grad(Fh, Jh, B)
    assert abs(O.mi_of_pmf(p, B) - v) <= 1e-14 * abs(v)
    idx = rng.choice(N, 50, replace=False)
    gp = O.mi_adjoint_points(Fh[idx], Jh[idx], N, B, p)
    np.testing.assert_allclose(gp, g[idx], rtol=1e-12, atol=0)


def test_kernel_derivative_sums_to_zero():
    """The derivative of the partition of unity: sum_m beta3'(s - m) = 0 for
    every s, which is why the -1 term of dMI/dp drops out of the adjoint."""
    for s in np.linspace(1.0, 9.0, 37):
        assert abs(sum(O.bspline3_deriv(s - m) for m in range(-2, 14))) <= 1e-15


# ---- the chain through the warp and the intensity map (Sec. 2.2) ------------
def _smooth_pair(rng, shape=(8, 9, 10)):
    from scipy.ndimage import gaussian_filter
    F = gaussian_filter(rng.standard_normal(shape), 1.2)
    M = np.tanh(F) + 0.3 * gaussian_filter(rng.standard_normal(shape), 1.2)
    u = 0.7 * rng.standard_normal((3,) + shape)
    return F, M, u


def test_mi_is_invariant_to_an_intensity_map_carried_by_the_range(rng):
    """Each image is mapped to [0, 1] by its own range, so M' = 3 M + 2 with
    the range mapped the same way gives the same MI and the same dC/du; the
    fixed image's range differs from the moving one's."""
    F, M, u = _smooth_pair(rng)
    fr = (float(F.min()) - 0.1, float(F.max()) + 0.2)
    mr = (float(M.min()) - 0.05, float(M.max()) + 0.1)
    s1, g1 = O.similarity_and_grad(F, M, u, O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=fr, m_range=mr))
    mr2 = (3 * mr[0] + 2, 3 * mr[1] + 2)
    s2, g2 = O.similarity_and_grad(F, 3 * M + 2, u, O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=fr, m_range=mr2))
    assert abs(s1 - s2) <= 1e-12 * abs(s1) and s1 > 0.01
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-10 * np.abs(g1).max())


def test_mi_clamps_intensities_outside_the_range(rng):
    """Intensities outside the stated range count at its ends: with u = 0 (so
    J = M) the MI of M equals that of M clipped to the range, and voxels
    outside it get no gradient."""
    F, M, _ = _smooth_pair(rng)
    u = np.zeros((3,) + F.shape)
    fr = (float(F.min()), float(F.max()))
    lo, hi = np.quantile(M, [0.2, 0.8])
    spec = O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=fr, m_range=(float(lo), float(hi)))
    s1, g = O.similarity_and_grad(F, M, u, spec)
    s2, _ = O.similarity_and_grad(F, np.clip(M, lo, hi), u, spec)
    assert abs(s1 - s2) <= 1e-12 * abs(s2)
    outside = (M < lo) | (M > hi)
    assert outside.sum() > 0.3 * M.size and not g[:, outside].any()


def test_objective_of_mi_is_minus_mi():
    """The MI objective is C = -MI: F = M taking two separated values (MI =
    ln 2 exactly, see the closed form above) gives loss -ln 2 at u = 0."""
    a, b = _bin_value(5.0), _bin_value(20.0)
    F = np.array([a, b] * 256).reshape(8, 8, 8)
    spec = O.LossSpec(kind=O.LOSS_MI, bins=B, f_range=(0.0, 1.0), m_range=(0.0, 1.0))
    obj = O.objective(F, F, np.zeros((3, 8, 8, 8)), spec, 0.5)
    assert abs(obj["loss"] + math.log(2.0)) < 1e-12 and obj["R"] == 0.0
    assert abs(obj["total"] + math.log(2.0)) < 1e-12


def test_hard_binned_chain_uses_the_hard_pmf(rng):
    """Through the warp and the intensity map, the hard-binned estimator's
    dC/du is the Parzen adjoint taken with the hard estimator's own PMF (the
    pairing its C-level gradient is pinned to), chained by dJh/dJ and the
    warp's slope; off the bin centres it differs from the Parzen chain."""
    F, M, u = _smooth_pair(rng)
    fr = (float(F.min()), float(F.max()))
    mr = (float(M.min()) - 0.1, float(M.max()) + 0.1)
    spec = O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=fr, m_range=mr, mi_estimator=1)
    s, g = O.similarity_and_grad(F, M, u, spec)
    J, dJ = O.warp(M, u, O.PAD_BORDER, with_grad=True)
    v, p = O.mi_hard(F, J, 16, fr, mr, with_hist=True)
    Fh, Jh, dJh = O.normalize(F, *fr)[0], *O.normalize(J, *mr)
    gJh = O.mi_adjoint_points(Fh.ravel(), Jh.ravel(), F.size, 16, p).reshape(F.shape)
    assert s == v
    np.testing.assert_allclose(g, (gJh * dJh)[None] * dJ, rtol=1e-12, atol=1e-15 * np.abs(g).max())
    _, g_parzen = O.similarity_and_grad(F, M, u, O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=fr, m_range=mr))
    assert np.abs(g - g_parzen).max() > 1e-3 * np.abs(g_parzen).max()
