"""Pins of the oracle's learned-initialiser operators other than the
convolutions: LeakyReLU and its derivative, 2x average pooling, trilinear
upsampling with voxel-centre alignment (x2 for the network, x s for the
displacement it outputs), channel concat, the field resampling between the
network's grid and the registration grid, the network input and the training
loss.  Each is checked against something other than itself: a library
routine that is a special case (torch's trilinear interpolation with
align_corners=False, NumPy block means and concatenation), closed forms
(constants, linear functions), adjoint identities and central differences."""
import numpy as np
import pytest
import torch

import oracle as O


def _rng(seed):
    return np.random.default_rng(seed)


def test_leaky_relu_values_and_derivative():
    x = np.array([-2.0, -0.5, 0.0, 0.25, 3.0])
    np.testing.assert_allclose(O.leaky(x, 0.2), [-0.4, -0.1, 0.0, 0.25, 3.0], rtol=0, atol=1e-15)
    dy = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    np.testing.assert_allclose(O.leaky_bwd(x, dy, 0.2), [0.2, 0.4, 0.6, 4.0, 5.0], rtol=0, atol=1e-15)
    # central differences away from the kink
    x = _rng(1).standard_normal(200)
    x = x[np.abs(x) > 1e-3]
    h = 1e-6
    fd = (O.leaky(x + h, 0.2) - O.leaky(x - h, 0.2)) / (2 * h)
    np.testing.assert_allclose(O.leaky_bwd(x, np.ones_like(x), 0.2), fd, rtol=1e-8, atol=0)


def test_avgpool2_is_the_block_mean_and_its_adjoint_the_transpose():
    x = _rng(2).standard_normal((6, 4, 8, 3))
    ref = x.reshape(3, 2, 2, 2, 4, 2, 3).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(O.avgpool2(x), ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(O.avgpool2(np.full((4, 6, 2, 2), 1.75)), 1.75, rtol=0, atol=1e-15)
    # <pool x, y> = <x, pool^T y>
    y = _rng(3).standard_normal((3, 2, 4, 3))
    lhs = float((O.avgpool2(x) * y).sum())
    rhs = float((x * O.avgpool2_adjoint(y, (6, 4, 8))).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("s", [2, 4])
def test_upsample_equals_torch_trilinear_without_corner_alignment(s):
    x = _rng(4 + s).standard_normal((3, 5, 4, 2))  # [nz, ny, nx, C]
    got = O.upsample(x, s)
    t = torch.from_numpy(x).permute(3, 0, 1, 2)[None]  # [1, C, nz, ny, nx]
    ref = torch.nn.functional.interpolate(t, scale_factor=s, mode="trilinear", align_corners=False)
    np.testing.assert_allclose(got, ref[0].permute(1, 2, 3, 0).numpy(), rtol=0, atol=1e-13)


def test_upsample_reproduces_linear_functions_inside_and_clamps_at_the_border():
    nz, ny, nx = 4, 5, 6
    zc, yc, xc = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = (0.5 * xc - 2.0 * yc + 3.0 * zc + 1.0)[..., None]
    up = O.upsample(f, 2)[..., 0]
    # fine voxel centre k lies at coarse coordinate (k + 1/2) / 2 - 1/2
    c = lambda k: (k + 0.5) / 2 - 0.5
    Z, Y, X = np.meshgrid(np.arange(2 * nz), np.arange(2 * ny), np.arange(2 * nx), indexing="ij")
    exact = 0.5 * np.clip(c(X), 0, nx - 1) - 2.0 * np.clip(c(Y), 0, ny - 1) + 3.0 * np.clip(c(Z), 0, nz - 1) + 1.0
    np.testing.assert_allclose(up, exact, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.upsample(np.full((2, 3, 2, 1), -0.5), 2), -0.5, rtol=0, atol=1e-15)


@pytest.mark.parametrize("s", [2, 3])
def test_upsample_adjoint_is_the_transpose(s):
    x = _rng(7).standard_normal((3, 2, 4, 2))
    g = _rng(8).standard_normal((3 * s, 2 * s, 4 * s, 2))
    lhs = float((O.upsample(x, s) * g).sum())
    rhs = float((x * O.upsample_adjoint(g, s)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_concat_equals_numpy():
    a = _rng(9).standard_normal((2, 3, 4, 5))
    b = _rng(10).standard_normal((2, 3, 4, 3))
    np.testing.assert_array_equal(O.concat(a, b), np.concatenate([a, b], axis=-1))


def test_field_down2_is_the_halved_block_mean():
    u = _rng(11).standard_normal((3, 4, 6, 8))
    ref = 0.5 * u.reshape(3, 2, 2, 3, 2, 4, 2).mean(axis=(2, 4, 6))
    np.testing.assert_allclose(O.field_down2(u), ref, rtol=0, atol=1e-14)
    # a constant displacement d voxels fine is d / 2 voxels coarse
    d = np.array([1.0, -3.0, 0.25])[:, None, None, None] * np.ones((3, 4, 4, 4))
    np.testing.assert_allclose(O.field_down2(d)[:, 0, 0, 0], [0.5, -1.5, 0.125], rtol=0, atol=1e-15)


@pytest.mark.parametrize("s", [2, 8])
def test_field_upsample_scales_displacements_and_interpolates(s):
    # a constant displacement d voxels coarse is s d voxels fine
    d = np.array([1.0, -3.0, 0.25])[:, None, None, None] * np.ones((3, 2, 3, 2))
    np.testing.assert_allclose(O.field_upsample(d, s), s * d[:, :1, :1, :1] * np.ones((3, 2 * s, 3 * s, 2 * s)),
                               rtol=0, atol=1e-13)
    u = _rng(12 + s).standard_normal((3, 3, 2, 4))
    t = torch.from_numpy(u)[None]  # channels as the batch's channels
    ref = s * torch.nn.functional.interpolate(t, scale_factor=s, mode="trilinear", align_corners=False)[0]
    np.testing.assert_allclose(O.field_upsample(u, s), ref.numpy(), rtol=0, atol=1e-12)


def test_pack_pair_is_the_normalised_block_mean():
    F = _rng(14).uniform(2.0, 5.0, (4, 6, 8))
    M = _rng(15).uniform(-1.0, 1.0, (4, 6, 8))
    got = O.pack_pair(F, M, 2, (2.0, 5.0), (-1.0, 3.0))
    refF = (F.reshape(2, 2, 3, 2, 4, 2).mean(axis=(1, 3, 5)) - 2.0) / 3.0
    refM = (M.reshape(2, 2, 3, 2, 4, 2).mean(axis=(1, 3, 5)) + 1.0) / 4.0
    np.testing.assert_allclose(got[..., 0], refF, rtol=0, atol=1e-14)
    np.testing.assert_allclose(got[..., 1], refM, rtol=0, atol=1e-14)


def test_mse_value_and_gradient():
    p = _rng(16).standard_normal((3, 40))
    t = _rng(17).standard_normal((3, 40))
    loss, g = O.mse(p, t)
    assert abs(loss - float(((p - t) ** 2).mean())) <= 1e-14
    h = 1e-6
    i = (1, 7)
    pp, pm = p.copy(), p.copy()
    pp[i] += h
    pm[i] -= h
    fd = (O.mse(pp, t)[0] - O.mse(pm, t)[0]) / (2 * h)
    assert abs(g[i] - fd) <= 1e-8 * max(1.0, abs(fd))
