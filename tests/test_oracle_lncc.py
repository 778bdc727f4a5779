"""Pins for the oracle's LNCC value and gradient (App. fused LNCC: Eq.
lncc-loss, Eqs. lncc-a..lncc-c, Eq. gradientcc-first).  CPU only."""
import numpy as np
import pytest

import oracle as O


def _smooth(rng, shape):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(rng.standard_normal(shape), 1.5) + 0.05 * rng.standard_normal(shape)


def test_self_similarity_is_one(rng):
    F = _smooth(rng, (9, 10, 11))
    S, n = O.lncc(F, F, 5, 0.0, per_voxel=True)
    np.testing.assert_allclose(n, 1.0, atol=1e-12)
    assert abs(S - 1.0) < 1e-12


@pytest.mark.parametrize("a,b,c,d", [(2.5, -1.0, 1.0, 0.0), (-0.3, 4.0, 7.0, -2.0)])
def test_affine_intensity_invariance(rng, a, b, c, d):
    F = _smooth(rng, (8, 9, 10))
    J = _smooth(rng, (8, 9, 10))
    S0, n0 = O.lncc(F, J, 5, 0.0, per_voxel=True)
    S1, n1 = O.lncc(c * F + d, a * J + b, 5, 0.0, per_voxel=True)
    np.testing.assert_allclose(n1, n0, rtol=1e-9, atol=1e-12)


def test_symmetry_and_bounds(rng):
    F = _smooth(rng, (8, 9, 10))
    J = _smooth(rng, (8, 9, 10))
    S0, n0 = O.lncc(F, J, 7, 1e-3, per_voxel=True)
    S1, n1 = O.lncc(J, F, 7, 1e-3, per_voxel=True)
    np.testing.assert_allclose(n0, n1, rtol=1e-12)
    assert (n0 >= 0).all() and (n0 <= 1.0).all()


def test_closed_form_ramp_against_square():
    """F = x, J = x^2 (constant along y, z).  Inside a window the x-offsets d
    run over an integer range; with X = x + d:  A = cov(X, X^2), B = var(X),
    C = var(X^2), so for the interior window d in {-r..r}:
    n = 4 x^2 V / (4 x^2 V + W) with V = r(r+1)/3 and
    W = var(d^2) = r(r+1)(3r^2+3r-1)/15 - V^2."""
    nx, ny, nz = 20, 7, 7
    r = 2
    x = np.arange(nx, dtype=np.float64)
    F = np.broadcast_to(x, (nz, ny, nx)).copy()
    J = F ** 2
    _, n = O.lncc(F, J, 2 * r + 1, 0.0, per_voxel=True)
    V = r * (r + 1) / 3.0
    W = r * (r + 1) * (3 * r * r + 3 * r - 1) / 15.0 - V * V
    for xi in range(r, nx - r):
        expect = 4 * xi * xi * V / (4 * xi * xi * V + W)
        np.testing.assert_allclose(n[:, :, xi], expect, rtol=1e-11)
    # truncated windows at the x border: moments of the clipped offset range,
    # by direct enumeration of the few values X can take.
    for xi in list(range(0, r)) + list(range(nx - r, nx)):
        X = np.arange(max(0, xi - r), min(nx - 1, xi + r) + 1, dtype=np.float64)
        cov = np.mean(X * X ** 2) - np.mean(X) * np.mean(X ** 2)
        expect = cov ** 2 / (np.var(X) * np.var(X ** 2))
        np.testing.assert_allclose(n[:, :, xi], expect, rtol=1e-10)


def test_constant_window_gives_zero_with_eps_zero():
    F = np.ones((5, 5, 5))
    J = np.ones((5, 5, 5))
    S, n = O.lncc(F, J, 3, 0.0, per_voxel=True)
    assert S == 0.0 and (n == 0).all()


@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_gradient_wrt_J_matches_central_differences(rng, eps):
    F = _smooth(rng, (7, 8, 9))
    J = _smooth(rng, (7, 8, 9))
    win = 5
    S, g = O.lncc_grad(F, J, win, eps)
    assert abs(S - O.lncc(F, J, win, eps)) < 1e-15
    h = 1e-5
    idx = [tuple(rng.integers(0, s) for s in F.shape) for _ in range(30)]
    idx += [(0, 0, 0), (6, 7, 8), (3, 0, 4)]
    for k in idx:
        Jp = J.copy()
        Jp[k] += h
        Jm = J.copy()
        Jm[k] -= h
        fd = -(O.lncc(F, Jp, win, eps) - O.lncc(F, Jm, win, eps)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-11, (k, g[k], fd)


def test_full_chain_gradient_wrt_u_matches_central_differences(rng):
    """dC/du through warp + LNCC on a 16^3 volume, FP64, rel 1e-6."""
    n = 16
    F = _smooth(rng, (n, n, n))
    M = _smooth(rng, (n, n, n))
    u = rng.integers(-1, 2, (3, n, n, n)) + rng.uniform(0.1, 0.9, (3, n, n, n))
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=7, eps=1e-5)
    S, g = O.similarity_and_grad(F, M, u, spec)
    # h = 1e-4 keeps the FP64 cancellation error of the difference quotient
    # (about 1e-16 |S| / h) well below 1e-6 of the smallest sampled entries;
    # the O(h^2) truncation term is ~1e-9 relative here.
    h = 1e-4
    rms = float(np.sqrt(np.mean(g ** 2)))
    errs = []
    for _ in range(24):
        c = rng.integers(0, 3)
        k = (c,) + tuple(rng.integers(2, n - 2, 3))
        up = u.copy()
        up[k] += h
        um = u.copy()
        um[k] -= h
        Sp, _ = O.similarity_and_grad(F, M, up, spec, need_grad=False)
        Sm, _ = O.similarity_and_grad(F, M, um, spec, need_grad=False)
        fd = -(Sp - Sm) / (2 * h)
        # relative to the entry, with a floor at a tenth of the field's RMS so
        # that entries near zero are judged on the FD rounding noise scale
        errs.append(abs(g[k] - fd) / (abs(fd) + 0.1 * rms))
    assert max(errs) < 1e-6, errs


def test_pointwise_gradient_equals_full_field(rng):
    F = _smooth(rng, (9, 11, 10))
    J = _smooth(rng, (9, 11, 10))
    S, g = O.lncc_grad(F, J, 5, 1e-4)
    _, n = O.lncc(F, J, 5, 1e-4, per_voxel=True)
    pts = np.concatenate([[0, F.size - 1], rng.integers(0, F.size, 40)])
    gp, npnt = O.lncc_grad_points(F, J, 5, 1e-4, pts)
    np.testing.assert_allclose(gp, g.ravel()[pts], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(npnt, n.ravel()[pts], rtol=1e-12)


# ---- the ANTs gradient approximation (App. fused LNCC) ----------------------
def _count(k, shape, r):
    """in-volume size of the window of side 2r+1 at linear index k"""
    nz, ny, nx = shape
    z, rem = divmod(k, ny * nx)
    y, x = divmod(rem, nx)
    c = 1
    for v, n in ((x, nx), (y, ny), (z, nz)):
        c *= min(v + r, n - 1) - max(v - r, 0) + 1
    return c


@pytest.mark.parametrize("win,eps", [(3, 1e-5), (5, 1e-9)])
def test_ants_gradient_is_the_own_window_derivative(rng, win, eps):
    """gJ_k = -(c_k / N) d n_k / d J_k: central differences of the voxel's own
    window NCC (corner, face, interior voxels)."""
    shape = (7, 8, 9)
    F = rng.random(shape)
    J = 0.6 * F + 0.4 * rng.random(shape)
    _, g = O.lncc_grad_ants(F, J, win, eps)
    N = F.size
    h = 1e-5
    for k in (0, N - 1, 4 * 72 + 3 * 9 + 4, 2 * 72 + 0 * 9 + 5, 5 * 72 + 7 * 9 + 8):
        Jp, Jm = J.copy(), J.copy()
        Jp.flat[k] += h
        Jm.flat[k] -= h
        dn = (O.lncc(F, Jp, win, eps, per_voxel=True)[1].flat[k] -
              O.lncc(F, Jm, win, eps, per_voxel=True)[1].flat[k]) / (2 * h)
        expect = -_count(k, shape, win // 2) / N * dn
        assert abs(g.flat[k] - expect) <= 1e-6 * max(abs(expect), 1e-12), (k, g.flat[k], expect)


def test_ants_gradient_approximates_the_exact_adjoint():
    """On smooth images the local approximation points along the exact
    gradient (cosine > 0.8 for 5^3 and 7^3 windows) and transforms like it
    under J -> a J + b (the gradient of a scale-free similarity scales 1/a)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(1)
    F = gaussian_filter(rng.standard_normal((16, 16, 16)), 2.0)
    J = gaussian_filter(rng.standard_normal((16, 16, 16)), 2.0) * 0.3 + 0.8 * np.roll(F, 1, axis=2)
    for win in (5, 7):
        _, ge = O.lncc_grad(F, J, win, 0.0)
        _, ga = O.lncc_grad_ants(F, J, win, 0.0)
        cos = float((ge * ga).sum() / np.linalg.norm(ge) / np.linalg.norm(ga))
        assert cos > 0.8, (win, cos)
        _, ga2 = O.lncc_grad_ants(F, 3.0 * J - 2.0, win, 0.0)
        np.testing.assert_allclose(3.0 * ga2, ga, rtol=1e-7, atol=1e-12 * np.abs(ga).max())


@pytest.mark.parametrize("win", [3, 5])
def test_brute_force_windows_on_a_tiny_volume(rng, win):
    """Every voxel's n_i from explicitly extracted windows (truncated at the
    border, two-pass centred moments, pure numpy) equals the oracle's."""
    shape = (5, 4, 6)
    F = rng.standard_normal(shape)
    J = 0.6 * F + 0.5 * rng.standard_normal(shape)
    eps = 1e-3
    r = win // 2
    nz, ny, nx = shape
    ref = np.empty(shape)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                sl = (slice(max(z - r, 0), min(z + r + 1, nz)), slice(max(y - r, 0), min(y + r + 1, ny)),
                      slice(max(x - r, 0), min(x + r + 1, nx)))
                f, j = F[sl].ravel(), J[sl].ravel()
                A = np.mean((f - f.mean()) * (j - j.mean()))
                B = np.mean((f - f.mean()) ** 2)
                C = np.mean((j - j.mean()) ** 2)
                ref[z, y, x] = A * A / (B * C + eps)
    S, n = O.lncc(F, J, win, eps, per_voxel=True)
    np.testing.assert_allclose(n, ref, rtol=1e-12, atol=1e-14)
    assert abs(S - ref.mean()) <= 1e-13


def test_objective_of_lncc_is_one_minus_s(rng):
    """The LNCC objective is C = 1 - S: an image against itself (S = 1) at
    u = 0 gives loss 0, and the regulariser term adds lam R."""
    F = rng.random((6, 7, 8))
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=3, eps=0.0)  # no window of random values is flat
    obj = O.objective(F, F, np.zeros((3, 6, 7, 8)), spec, 0.5)
    assert abs(obj["loss"]) < 1e-13 and obj["R"] == 0.0 and abs(obj["total"]) < 1e-13
    u = np.zeros((3, 6, 7, 8))
    u[0, :, :, 3:] = 0.25  # a step in x: R > 0, and the warp moves J off F
    obj = O.objective(F, F, u, spec, 0.5)
    S = O.lncc(F, O.warp(F, u), 3, 0.0)
    assert abs(obj["loss"] - (1.0 - S)) < 1e-14 and obj["R"] > 0
    assert abs(obj["total"] - (1.0 - S + 0.5 * obj["R"])) < 1e-14
