"""Pins for the oracle's diffusion regulariser, Adam step, bfloat16
rounding and Jacobian determinant.  CPU only."""
import numpy as np
import pytest
import torch

import oracle as O


def test_diffusion_constant_field_is_zero(rng):
    u = np.ones((3, 5, 6, 7)) * np.array([0.3, -1.0, 2.0])[:, None, None, None]
    R, g = O.diffusion(u)
    assert R == 0.0 and not g.any()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("comp", [0, 1, 2])
def test_diffusion_linear_field_closed_form(axis, comp):
    """u_comp = a * (coordinate along one axis), the other components 0: only
    the n_axis - 1 differences along that axis are non-zero, each a, on every
    line along it; R = a^2 (n_axis - 1) (N / n_axis) / N."""
    shape = (5, 6, 7)  # nz, ny, nx; axis 0 = x
    a = 0.7
    coords = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    u = np.zeros((3,) + shape)
    u[comp] = a * coords[2 - axis]
    R, _ = O.diffusion(u)
    N = int(np.prod(shape))
    n_ax = shape[2 - axis]
    assert abs(R - a * a * (n_ax - 1) * (N // n_ax) / N) < 1e-14


def test_diffusion_gradient_is_scaled_neumann_laplacian():
    """u_c = x^2 along x: the interior second difference is 2, so
    dR/du = -(2/N) * 2 in the interior; at x=0 the one-sided Neumann
    stencil gives -(2/N)(u1 - u0) = -2/N, at x=n-1 +(2/N)(u_{n-1}-u_{n-2})."""
    nz, ny, nx = 3, 4, 9
    N = nx * ny * nz
    x = np.arange(nx, dtype=np.float64)
    u = np.zeros((3, nz, ny, nx))
    u[0] = x ** 2
    _, g = O.diffusion(u)
    np.testing.assert_allclose(g[0][:, :, 1:-1], -4.0 / N, atol=1e-14)
    np.testing.assert_allclose(g[0][:, :, 0], -(2.0 / N) * 1.0, atol=1e-14)
    np.testing.assert_allclose(g[0][:, :, -1], (2.0 / N) * (64 - 49), atol=1e-14)
    assert not g[1].any() and not g[2].any()


def test_diffusion_gradient_matches_central_differences(rng):
    u = rng.standard_normal((3, 4, 5, 6))
    R, g = O.diffusion(u)
    h = 1e-6
    for _ in range(20):
        k = tuple(rng.integers(0, s) for s in u.shape)
        up = u.copy()
        up[k] += h
        um = u.copy()
        um[k] -= h
        fd = (O.diffusion(up, False) - O.diffusion(um, False)) / (2 * h)
        assert abs(fd - g[k]) < 1e-8


def test_adam_equals_torch_adam_step_for_step(rng):
    n = 64
    u0 = rng.standard_normal(n)
    p = torch.tensor(u0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
    u, m, v = u0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.standard_normal(n) * (1e-3 if t % 2 else 10.0)
        p.grad = torch.tensor(g)
        opt.step()
        u, m, v = O.adam(u, m, v, g, t, lr=0.1)
        np.testing.assert_allclose(u, p.detach().numpy(), rtol=1e-13, atol=1e-14)
        st = opt.state[p]
        np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-13)
        np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-13)


def test_adam_grad_scale_is_input_scaling(rng):
    n = 32
    u0, g = rng.standard_normal(n), rng.standard_normal(n)
    a = O.adam(u0, np.zeros(n), np.zeros(n), g, 1, 0.1, grad_scale=1000.0)
    b = O.adam(u0, np.zeros(n), np.zeros(n), 1000.0 * g, 1, 0.1)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-14)


def test_bf16_round_equals_torch_conversion(rng):
    # includes exact ties with even (1 + 2^-8) and odd (1 + 2^-7 + 2^-8) last kept bit
    x = np.concatenate([rng.standard_normal(500) * 10.0 ** rng.integers(-20, 20, 500),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -1.01171875, 1.005859375, 3e38, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float64).to(torch.float32).to(torch.bfloat16).to(torch.float64)
    np.testing.assert_array_equal(O.bf16_round(x), ref.numpy())


def test_adam_bf16_moments_are_rounded_after_use(rng):
    n = 50
    u0, g = rng.standard_normal(n), rng.standard_normal(n)
    uf, mf, vf = O.adam(u0, np.zeros(n), np.zeros(n), g, 1, 0.05)
    ub, mb, vb = O.adam(u0, np.zeros(n), np.zeros(n), g, 1, 0.05, bf16_moments=True)
    np.testing.assert_array_equal(ub, uf)
    np.testing.assert_array_equal(mb, O.bf16_round(mf))
    np.testing.assert_array_equal(vb, O.bf16_round(vf))


def test_jacdet_identity_and_linear_maps(rng):
    shape = (5, 6, 7)
    assert (O.jacdet(np.zeros((3,) + shape)) == 1.0).all()
    A = rng.uniform(-0.3, 0.3, (3, 3))
    z, y, x = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    X = np.stack([x, y, z])
    u = np.einsum("cd,dzyx->czyx", A, X)
    d = O.jacdet(u)
    np.testing.assert_allclose(d, np.linalg.det(np.eye(3) + A), rtol=1e-13)


def test_jacdet_detects_folding():
    u = np.zeros((3, 4, 4, 8))
    x = np.arange(8, dtype=np.float64)
    u[0] = -2.0 * x  # phi_x = -x : orientation reversed
    assert (O.jacdet(u) < 0).all()


# ---- Gaussian smoothing of gradient / warp (the sigma_grad / sigma_warp
# regularisation the paper runs with) ------------------------------------------
@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.3])
def test_gaussian_smooth_equals_scipy(rng, sigma):
    """A library special case: scipy.ndimage.gaussian_filter with mode
    'nearest' and truncate 4 (the same radius floor(4 sigma + 1/2))."""
    from scipy.ndimage import gaussian_filter
    u = rng.standard_normal((3, 7, 11, 13))
    s = O.gaussian_smooth(u, sigma)
    for c in range(3):
        ref = gaussian_filter(u[c], sigma, mode="nearest", truncate=4.0)
        np.testing.assert_allclose(s[c], ref, rtol=1e-12, atol=1e-12)


def test_gaussian_smooth_preserves_constants_and_mass(rng):
    u = np.full((2, 5, 6, 7), 3.25)
    np.testing.assert_allclose(O.gaussian_smooth(u, 1.5), u, rtol=1e-14)
    # a linear ramp is preserved away from the borders (symmetric kernel)
    x = np.broadcast_to(np.arange(40, dtype=np.float64), (3, 3, 40)).copy()
    s = O.gaussian_smooth(x, 1.0)
    np.testing.assert_allclose(s[:, :, 8:32], x[:, :, 8:32], rtol=0, atol=1e-12)


def test_objective_gradient_is_the_derivative_of_its_total(rng):
    """The iteration's objective C + lam R (lam != 1): its gradient in u equals
    central differences of its own total at random components."""
    from scipy.ndimage import gaussian_filter
    shape = (6, 7, 8)
    F = gaussian_filter(rng.standard_normal(shape), 1.0)
    M = gaussian_filter(rng.standard_normal(shape), 1.0)
    u = 0.8 * rng.standard_normal((3,) + shape)
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=3, eps=1e-3)
    lam = 2.5
    obj = O.objective(F, M, u, spec, lam)
    assert obj["total"] == obj["loss"] + lam * obj["R"]
    h = 1e-6
    for _ in range(16):
        k = tuple(rng.integers(0, s) for s in u.shape)
        up = u.copy()
        up[k] += h
        um = u.copy()
        um[k] -= h
        fd = (O.objective(F, M, up, spec, lam)["total"] - O.objective(F, M, um, spec, lam)["total"]) / (2 * h)
        assert abs(fd - obj["grad"][k]) <= 1e-6 * (1.0 + abs(fd))


def test_first_iteration_moves_each_component_by_lr(rng):
    """The iteration feeds Adam N times the gradient (per-voxel gradients of
    a mean over N voxels are O(1/N), far below Adam's eps otherwise): the
    first step is then lr times the sign of the descent direction, to within
    lr * eps / |N g|, on every component with |N g| above 0.1."""
    from scipy.ndimage import gaussian_filter
    shape = (8, 9, 10)
    F = gaussian_filter(rng.standard_normal(shape), 1.0)
    M = gaussian_filter(rng.standard_normal(shape), 1.0)
    u = 0.5 * rng.standard_normal((3,) + shape)
    spec = O.LossSpec(kind=O.LOSS_LNCC, window=3, eps=1e-3)
    lr = 0.1
    z = np.zeros_like(u)
    out = O.iterate(F, M, u, z, z, 1, spec, lam=0.5, lr=lr)
    g = out["grad"] * F.size
    big = np.abs(g) > 0.1
    assert big.mean() > 0.5
    np.testing.assert_allclose((u - out["u"])[big], lr * np.sign(g[big]), rtol=0, atol=1e-7 * lr)
