"""Pins for the oracle's composite affine + deformable transform
phi(p) = A p + t + S u(p) (Sec. 2.1, the composite implicit grid sampler;
Algorithm gridsampler, forward and backward).  CPU only.

The forward is pinned to exact resamplings a reader can check by eye (integer
shifts, a 90-degree rotation, a 2x decimation, a half-voxel shift); the
backward and the loss gradients with respect to A, t and u are pinned to
central differences of the forward."""
import numpy as np
import pytest

import oracle as O

I3 = np.eye(3)


def _smooth(rng, shape):
    v = rng.standard_normal(shape)
    return O.gaussian_smooth(v, 1.0)


def test_identity_transform_is_plain_warp(rng):
    M = rng.standard_normal((5, 6, 7))
    u = 0.7 * rng.standard_normal((3,) + M.shape)
    assert np.array_equal(O.warp_composite(M, I3, (0, 0, 0), (1, 1, 1), u), O.warp(M, u))
    assert np.array_equal(O.warp_composite(M, I3, (0, 0, 0)), M)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
def test_integer_translation(rng, pad):
    M = rng.standard_normal((6, 7, 9))
    nz, ny, nx = M.shape
    t = (3, -2, 1)
    J = O.warp_composite(M, I3, t, pad=pad)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx, sy, sz = x + t[0], y + t[1], z + t[2]
    val = M[np.clip(sz, 0, nz - 1), np.clip(sy, 0, ny - 1), np.clip(sx, 0, nx - 1)]
    if pad == O.PAD_ZEROS:
        ok = (sx >= 0) & (sx < nx) & (sy >= 0) & (sy < ny) & (sz >= 0) & (sz < nz)
        val = np.where(ok, val, 0.0)
    assert np.array_equal(J, val)


def test_quarter_turn_is_a_transpose_and_flip(rng):
    """A maps (x, y, z) to (n-1-y, x, z): J[z, y, x] = M[z, x, n-1-y].  A is
    not symmetric, so using A^T (or reading A column-major) fails."""
    n = 6
    M = rng.standard_normal((4, n, n))
    A = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    J = O.warp_composite(M, A, (n - 1, 0, 0))
    ref = np.swapaxes(M[:, :, ::-1], 1, 2)
    np.testing.assert_allclose(J, ref, rtol=0, atol=1e-14)


def test_scale_two_is_decimation(rng):
    M = rng.standard_normal((8, 10, 12))
    J = O.warp_composite(M, 2.0 * I3, (0, 0, 0))
    np.testing.assert_allclose(J[:4, :5, :6], M[::2, ::2, ::2], rtol=0, atol=1e-14)


def test_half_voxel_shift_is_neighbour_mean(rng):
    M = rng.standard_normal((3, 4, 8))
    J = O.warp_composite(M, I3, (0.5, 0, 0))
    np.testing.assert_allclose(J[:, :, :-1], 0.5 * (M[:, :, :-1] + M[:, :, 1:]), rtol=0, atol=1e-14)


def test_displacement_scale_acts_per_channel(rng):
    M = rng.standard_normal((5, 6, 7))
    u = 0.8 * rng.standard_normal((3,) + M.shape)
    s = (2.0, 0.5, 1.5)
    ref = O.warp(M, np.asarray(s)[:, None, None, None] * u)
    np.testing.assert_allclose(O.warp_composite(M, I3, (0, 0, 0), s, u), ref, rtol=0, atol=1e-14)


def _rand_affine(rng):
    A = I3 + 0.05 * rng.standard_normal((3, 3))
    t = 0.6 * rng.standard_normal(3)
    return A, t


def test_sampler_backward_matches_differences(rng):
    """g_A[i][j] = d/dA_ij of sum_p g(p) J(p), likewise g_t and g_u, by
    central differences (Algorithm gridsampler, backward)."""
    shape = (5, 6, 7)
    M = _smooth(rng, shape)
    u = 0.4 * rng.standard_normal((3,) + shape)
    g = rng.standard_normal(shape)
    A, t = _rand_affine(rng)
    s = (1.3, 0.8, 1.1)
    g_u, g_A, g_t = O.sampler_backward_composite(M, A, t, s, u, g)
    L = lambda A_, t_, u_: float(np.sum(g * O.warp_composite(M, A_, t_, s, u_)))
    h = 1e-6
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            fd = (L(A + E, t, u) - L(A - E, t, u)) / (2 * h)
            assert abs(fd - g_A[i, j]) < 1e-6 * max(1.0, abs(fd)), (i, j, fd, g_A[i, j])
        e = np.zeros(3)
        e[i] = h
        fd = (L(A, t + e, u) - L(A, t - e, u)) / (2 * h)
        assert abs(fd - g_t[i]) < 1e-6 * max(1.0, abs(fd))
    for c, z, y, x in [(0, 2, 3, 4), (1, 0, 5, 1), (2, 4, 0, 6)]:
        du = np.zeros_like(u)
        du[c, z, y, x] = h
        fd = (L(A, t, u + du) - L(A, t, u - du)) / (2 * h)
        assert abs(fd - g_u[c, z, y, x]) < 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("kind", ["lncc", "lncc_ants", "mi"])
def test_loss_gradients_match_differences(rng, kind):
    shape = (7, 6, 8)
    F = _smooth(rng, shape)
    F = (F - F.min()) / (F.max() - F.min())
    A0 = I3 + np.array([[0.02, -0.03, 0.0], [0.03, 0.01, 0.0], [0.0, 0.0, -0.02]])
    M = O.warp_composite(F, A0, (0.3, -0.2, 0.1))
    u = 0.2 * rng.standard_normal((3,) + shape)
    A, t = _rand_affine(rng)
    s = (1.0, 1.0, 1.0)
    if kind == "mi":
        spec = O.LossSpec(kind=O.LOSS_MI, bins=16, f_range=(0.0, 1.0), m_range=(0.0, 1.0))
    else:
        spec = O.LossSpec(kind=O.LOSS_LNCC, window=3, eps=1e-9, lncc_grad=1 if kind == "lncc_ants" else 0)
    sim, g_u, g_A, g_t = O.similarity_and_grad_composite(F, M, A, t, s, u, spec)
    sim_plain, g_plain = O.similarity_and_grad(F, M, O.composite_offset(shape, A, t, s, u), spec)
    assert sim == sim_plain and np.array_equal(g_u, g_plain)
    if kind == "lncc_ants":
        return  # the approximation is not the derivative of the loss
    sign = -1.0

    def C(A_, t_):
        return sign * O.similarity_and_grad_composite(F, M, A_, t_, s, u, spec)[0]

    h = 1e-6
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            fd = (C(A + E, t) - C(A - E, t)) / (2 * h)
            assert abs(fd - g_A[i, j]) < 2e-5 * max(1e-3, np.abs(g_A).max()), (i, j, fd, g_A[i, j])
        e = np.zeros(3)
        e[i] = h
        fd = (C(A, t + e) - C(A, t - e)) / (2 * h)
        assert abs(fd - g_t[i]) < 2e-5 * max(1e-3, np.abs(g_t).max())


# --------------------------------------------------------------------------
# field composition and scaling-and-squaring
# --------------------------------------------------------------------------
def test_compose_translations_add(rng):
    shape = (5, 6, 7)
    a = np.zeros((3,) + shape)
    b = np.zeros((3,) + shape)
    for c, (ta, tb) in enumerate([(0.3, 0.4), (-0.2, 0.7), (0.5, -0.1)]):
        a[c], b[c] = ta, tb
    np.testing.assert_allclose(O.compose_fields(a, b), a + b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
def test_compose_follows_the_padding_mode(pad):
    """a = an integer shift of +2 voxels along x, b = a constant field c:
    w(p) = a + b(p + a) is a + c where p + a lies inside the volume; outside
    it is a + c with BORDER padding and a with ZEROS padding."""
    shape = (4, 5, 6)
    a = np.zeros((3,) + shape)
    a[0] = 2.0
    c = np.array([0.3, -0.4, 0.5])
    b = np.ones((3,) + shape) * c[:, None, None, None]
    w = O.compose_fields(a, b, pad)
    inside = np.arange(shape[2]) + 2 <= shape[2] - 1
    ref = a + b
    if pad == O.PAD_ZEROS:
        ref[:, :, :, ~inside] = a[:, :, :, ~inside]
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-15)


def test_compose_with_linear_field_is_exact(rng):
    """b(p) = B p is linear, so trilinear sampling is exact in the interior:
    w(p) = a(p) + B (p + a(p))."""
    shape = (8, 9, 10)
    B = 0.05 * rng.standard_normal((3, 3))
    X = O.identity_grid(shape)
    b = np.einsum("ij,jzyx->izyx", B, X)
    a = np.clip(0.3 * rng.standard_normal((3,) + shape), -0.9, 0.9)
    w = O.compose_fields(a, b)
    ref = a + np.einsum("ij,jzyx->izyx", B, X + a)
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))  # p + a stays inside
    np.testing.assert_allclose(w[inner], ref[inner], rtol=0, atol=1e-13)


def test_exp_of_linear_field_is_matrix_power(rng):
    """For v(p) = B p about the volume centre, K squarings give exactly
    (I + B / 2^K)^(2^K) (away from the clamped border), which tends to the
    matrix exponential expm(B)."""
    from scipy.linalg import expm
    shape = (24, 24, 24)
    c = np.array([11.5, 11.5, 11.5])
    B = np.array([[0.02, -0.08, 0.01], [0.08, 0.03, 0.0], [-0.01, 0.02, -0.04]])
    X = O.identity_grid(shape)
    Xc = X - c[:, None, None, None]
    v = np.einsum("ij,jzyx->izyx", B, Xc)
    K = 6
    u = O.exp_field(v, K)
    P = np.linalg.matrix_power(np.eye(3) + B / 2 ** K, 2 ** K)
    ref = np.einsum("ij,jzyx->izyx", P - np.eye(3), Xc)
    inner = (slice(None), slice(6, -6), slice(6, -6), slice(6, -6))
    np.testing.assert_allclose(u[inner], ref[inner], rtol=0, atol=1e-11)
    refE = np.einsum("ij,jzyx->izyx", expm(B) - np.eye(3), Xc)
    assert np.abs(u[inner] - refE[inner]).max() < 2e-3


def test_exp_of_translation_is_translation(rng):
    v = np.zeros((3, 4, 5, 6))
    v[0], v[1], v[2] = 1.7, -0.6, 0.25
    np.testing.assert_allclose(O.exp_field(v, 5), v, rtol=0, atol=1e-14)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
def test_warp_adjoint_is_the_transpose(rng, pad):
    """<warp(M, u), g> = <M, warp_adjoint(g, u)> for every M and g (the warp is
    linear in M), displacements reaching outside the volume included."""
    shape = (5, 7, 6)
    u = 1.5 * rng.standard_normal((3,) + shape)
    for _ in range(3):
        M = rng.standard_normal(shape)
        g = rng.standard_normal(shape)
        lhs = float(np.sum(O.warp(M, u, pad) * g))
        rhs = float(np.sum(M * O.warp_adjoint(g, u, pad)))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_warp_adjoint_of_integer_shift_is_reverse_shift(rng):
    shape = (4, 5, 9)
    u = np.zeros((3,) + shape)
    u[0] = 2.0  # x + 2: interior voxels receive the value sampled from them
    g = rng.standard_normal(shape)
    gM = O.warp_adjoint(g, u, O.PAD_ZEROS)
    np.testing.assert_array_equal(gM[:, :, 2:], g[:, :, :-2])
    np.testing.assert_array_equal(gM[:, :, :2], 0.0)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
@pytest.mark.parametrize("scale", [1.0, 0.25])
def test_compose_backward_matches_differences(rng, scale, pad):
    shape = (6, 5, 7)
    a = 0.6 * O.gaussian_smooth(rng.standard_normal((3,) + shape), 1.0) + 0.2 * rng.standard_normal((3,) + shape)
    b = 0.8 * rng.standard_normal((3,) + shape)
    gw = rng.standard_normal((3,) + shape)
    ga, gb = O.compose_fields_backward(a, b, gw, pad=pad, scale=scale)

    def L(a_, b_):
        w = scale * a_ + np.stack([scale * O.warp(b_[c], scale * a_, pad) for c in range(3)])
        return float(np.sum(gw * w))

    h = 1e-6
    for c, z, y, x in [(0, 2, 3, 4), (1, 0, 1, 6), (2, 5, 4, 0), (0, 3, 0, 2)]:
        d = np.zeros_like(a)
        d[c, z, y, x] = h
        fa = (L(a + d, b) - L(a - d, b)) / (2 * h)
        fb = (L(a, b + d) - L(a, b - d)) / (2 * h)
        assert abs(fa - ga[c, z, y, x]) <= 1e-6 * max(1.0, abs(fa)), (fa, ga[c, z, y, x])
        assert abs(fb - gb[c, z, y, x]) <= 1e-7 * max(1.0, abs(fb)), (fb, gb[c, z, y, x])


@pytest.mark.parametrize("steps", [1, 3])
def test_exp_backward_matches_differences(rng, steps):
    shape = (6, 6, 6)
    v = 1.5 * O.gaussian_smooth(rng.standard_normal((3,) + shape), 1.0) + 0.05 * rng.standard_normal((3,) + shape)
    gout = rng.standard_normal((3,) + shape)
    gv = O.exp_field_backward(v, steps, gout)
    L = lambda v_: float(np.sum(gout * O.exp_field(v_, steps)))
    h = 1e-6
    for c, z, y, x in [(0, 2, 3, 4), (1, 5, 0, 1), (2, 3, 3, 3)]:
        d = np.zeros_like(v)
        d[c, z, y, x] = h
        fd = (L(v + d) - L(v - d)) / (2 * h)
        assert abs(fd - gv[c, z, y, x]) <= 1e-6 * max(1.0, abs(fd)), (fd, gv[c, z, y, x])
