"""Pins for the oracle's trilinear warp (Eq. interp of the ring-sampler
appendix; Algorithm gridsampler).  CPU only."""
import numpy as np
import pytest
import torch

import oracle as O


def _vol(rng, shape=(6, 7, 9)):
    return rng.standard_normal(shape)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
def test_zero_displacement_is_identity(rng, pad):
    M = _vol(rng)
    J = O.warp(M, np.zeros((3,) + M.shape), pad)
    assert np.array_equal(J, M)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
def test_integer_translation_is_exact_shift(rng, pad):
    M = _vol(rng)
    nz, ny, nx = M.shape
    t = (2, -1, 1)  # (x, y, z) in voxels
    u = np.zeros((3,) + M.shape)
    for c in range(3):
        u[c] = t[c]
    J = O.warp(M, u, pad)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx, sy, sz = x + t[0], y + t[1], z + t[2]
    if pad == O.PAD_BORDER:
        ref = M[np.clip(sz, 0, nz - 1), np.clip(sy, 0, ny - 1), np.clip(sx, 0, nx - 1)]
    else:
        ok = (sx >= 0) & (sx < nx) & (sy >= 0) & (sy < ny) & (sz >= 0) & (sz < nz)
        ref = np.where(ok, M[np.clip(sz, 0, nz - 1), np.clip(sy, 0, ny - 1), np.clip(sx, 0, nx - 1)], 0.0)
    assert np.array_equal(J, ref)


def test_affine_intensity_is_reproduced_in_interior(rng):
    nz, ny, nx = 8, 9, 10
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b, c, d = 0.7, -1.3, 0.4, 2.0
    M = a * x + b * y + c * z + d
    u = rng.uniform(-0.9, 0.9, (3, nz, ny, nx))
    J, dJ = O.warp(M, u, O.PAD_BORDER, with_grad=True)
    px, py, pz = x + u[0], y + u[1], z + u[2]
    inside = (px >= 0) & (px <= nx - 1) & (py >= 0) & (py <= ny - 1) & (pz >= 0) & (pz <= nz - 1)
    np.testing.assert_allclose(J[inside], (a * px + b * py + c * pz + d)[inside], atol=1e-12)
    np.testing.assert_allclose(dJ[0][inside], a, atol=1e-12)
    np.testing.assert_allclose(dJ[1][inside], b, atol=1e-12)
    np.testing.assert_allclose(dJ[2][inside], c, atol=1e-12)


def test_border_mode_equals_scipy_map_coordinates(rng):
    from scipy.ndimage import map_coordinates
    M = _vol(rng, (7, 8, 9))
    u = rng.uniform(-3, 3, (3,) + M.shape)
    J = O.warp(M, u, O.PAD_BORDER)
    z, y, x = np.meshgrid(*[np.arange(s) for s in M.shape], indexing="ij")
    coords = np.stack([z + u[2], y + u[1], x + u[0]])
    ref = map_coordinates(M, coords, order=1, mode="nearest")
    np.testing.assert_allclose(J, ref, atol=1e-12)


def test_zero_mode_equals_scipy_grid_constant(rng):
    from scipy.ndimage import map_coordinates
    M = _vol(rng, (7, 8, 9))
    u = rng.uniform(-3, 3, (3,) + M.shape)
    J = O.warp(M, u, O.PAD_ZEROS)
    z, y, x = np.meshgrid(*[np.arange(s) for s in M.shape], indexing="ij")
    coords = np.stack([z + u[2], y + u[1], x + u[0]])
    ref = map_coordinates(M, coords, order=1, mode="grid-constant", cval=0.0)
    np.testing.assert_allclose(J, ref, atol=1e-12)


@pytest.mark.parametrize("pad,mode", [(O.PAD_BORDER, "border"), (O.PAD_ZEROS, "zeros")])
def test_value_and_slope_equal_torch_grid_sample(rng, pad, mode):
    """torch grid_sample (align_corners=True) is the library special case of the
    voxel-unit sampler; its autograd slope pins the clamp-aware derivative."""
    M = _vol(rng, (5, 6, 7))
    nz, ny, nx = M.shape
    u = rng.uniform(-2.5, 2.5, (3,) + M.shape)
    J, dJ = O.warp(M, u, pad, with_grad=True)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = torch.tensor(np.stack([x + u[0], y + u[1], z + u[2]], -1), dtype=torch.float64)
    scale = torch.tensor([2.0 / (nx - 1), 2.0 / (ny - 1), 2.0 / (nz - 1)], dtype=torch.float64)
    grid = (phi * scale - 1.0).unsqueeze(0).requires_grad_(True)
    out = torch.nn.functional.grid_sample(torch.tensor(M)[None, None], grid, mode="bilinear",
                                          padding_mode=mode, align_corners=True)
    out.sum().backward()
    np.testing.assert_allclose(J, out[0, 0].detach().numpy(), atol=1e-12)
    slope = (grid.grad[0] * scale).numpy()  # d out / d phi
    # avoid sample points sitting exactly on a clamp boundary (subgradient)
    for c in range(3):
        np.testing.assert_allclose(dJ[c], slope[..., c], atol=1e-10)


def test_zero_mode_partition_identity(rng):
    """Ring-sampler decomposition (Eqs. interp-h, interp-honly): the warp of M
    equals the sum of warps of its zero-padded z-slab shards."""
    M = _vol(rng, (12, 6, 7))
    u = rng.uniform(-3, 3, (3,) + M.shape)
    full = O.warp(M, u, O.PAD_ZEROS)
    acc = np.zeros_like(full)
    for z0, z1 in [(0, 3), (3, 8), (8, 12)]:
        shard = np.zeros_like(M)
        shard[z0:z1] = M[z0:z1]
        acc += O.warp(shard, u, O.PAD_ZEROS)
    np.testing.assert_allclose(acc, full, atol=1e-12)


@pytest.mark.parametrize("pad", [O.PAD_BORDER, O.PAD_ZEROS])
def test_slope_matches_central_differences(rng, pad):
    M = _vol(rng, (6, 7, 8))
    nz, ny, nx = M.shape
    # fractional parts kept in [0.1, 0.9] so no sample sits on a cell face
    u = rng.integers(-2, 3, (3,) + M.shape) + rng.uniform(0.1, 0.9, (3,) + M.shape)
    J, dJ = O.warp(M, u, pad, with_grad=True)
    h = 1e-6
    for c in range(3):
        up = u.copy()
        up[c] += h
        um = u.copy()
        um[c] -= h
        fd = (O.warp(M, up, pad) - O.warp(M, um, pad)) / (2 * h)
        # exclude points whose +-h move crosses the clamp boundary
        n = (nx, ny, nz)[c]
        coord = np.indices(M.shape)[::-1][c] + u[c]
        ok = np.abs(coord - 0.0) > 1e-3
        ok &= np.abs(coord - (n - 1)) > 1e-3
        np.testing.assert_allclose(dJ[c][ok], fd[ok], atol=1e-7)


def test_slope_on_knots_uses_the_upper_cell():
    """On an integer sample point the slope is the forward difference
    M[x+1] - M[x]; on the last knot (phi = n-1, not clamped) it is the
    backward difference M[n-1] - M[n-2] (the cell index is min(floor, n-2))."""
    rng = np.random.default_rng(7)
    M = rng.standard_normal((4, 5, 6))
    J, dJ = O.warp(M, np.zeros((3,) + M.shape), O.PAD_BORDER, with_grad=True)
    fwd = np.diff(M, axis=2)
    np.testing.assert_allclose(dJ[0][:, :, :-1], fwd, atol=1e-15)
    np.testing.assert_allclose(dJ[0][:, :, -1], fwd[:, :, -1], atol=1e-15)
    np.testing.assert_allclose(dJ[2][:-1], np.diff(M, axis=0), atol=1e-15)
    np.testing.assert_allclose(dJ[2][-1], M[-1] - M[-2], atol=1e-15)


def test_downsample2_is_the_block_mean(rng):
    """The coarse level of the multi-scale schedule: the 2x2x2 block mean,
    the same as numpy's reshape-and-mean, and a constant stays constant."""
    img = rng.random((6, 8, 10))
    ref = img.reshape(3, 2, 4, 2, 5, 2).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(O.downsample2(img), ref, rtol=1e-15, atol=0)
    np.testing.assert_allclose(O.downsample2(np.full((4, 4, 4), 0.7)), 0.7, rtol=1e-15)
