"""Seeded synthetic volume pairs shaped like the paper's workloads.

The paper registers OASIS / faux-OASIS brains, 250 um and 100 um ex-vivo
volumes and random N^3 pairs (App. fused LNCC, Table cc-ablation); none of
these datasets ships here, so these generators stand in for them.

This module holds none of the registration method's arithmetic: it draws
random numbers, sums Gaussian blobs, paints label maps, smooths with a
Gaussian (torch conv1d; replicate padding for images, periodic for the random
displacement fields) and builds the moving image with
``torch.nn.functional.grid_sample`` (library trilinear sampling,
align_corners=True, border padding).  Both the CUDA path and the CPU oracle
take their inputs from here.

Random draws: for volumes up to 512^3 they come from numpy's PCG64
(``default_rng(seed)``) on the host, so they are identical on every machine;
the 1280^3 case draws on the GPU from torch's Philox generator seeded with
the same seed (recorded in the returned dict).
"""
from __future__ import annotations

import math

import numpy as np
import torch


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
def gaussian_smooth(vol: torch.Tensor, sigma: float, truncate: float = 4.0, periodic: bool = False) -> torch.Tensor:
    """Separable Gaussian of a [..., nz, ny, nx] tensor with 'nearest'
    borders, or periodic ones (periodic=True: the result of smoothing white
    noise is then stationary, with no inflated variance at the faces)."""
    if sigma <= 0:
        return vol
    r = int(truncate * sigma + 0.5)
    x = torch.arange(-r, r + 1, dtype=torch.float64)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    k = (k / k.sum()).to(vol.dtype).to(vol.device).view(1, 1, -1)
    out = vol
    nd = vol.dim()
    for ax in (nd - 1, nd - 2, nd - 3):
        t = out.movedim(ax, -1)
        shp = t.shape
        flat = t.reshape(-1, 1, shp[-1])
        chunks = []
        step = max(1, (1 << 27) // max(1, shp[-1] + 2 * r))
        for i in range(0, flat.shape[0], step):
            if periodic:
                idx = torch.arange(-r, shp[-1] + r, device=flat.device) % shp[-1]
                part = flat[i:i + step].index_select(-1, idx)
            else:
                part = torch.nn.functional.pad(flat[i:i + step], (r, r), mode="replicate")
            chunks.append(torch.nn.functional.conv1d(part, k))
        out = torch.cat(chunks, 0).reshape(shp).movedim(-1, ax).contiguous()
        del flat, chunks
    return out


def _sample_trilinear(M: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """M(p + u(p)) by torch grid_sample, voxel units, border padding."""
    nz, ny, nx = M.shape
    dev, dt = M.device, M.dtype
    out = torch.empty_like(M)
    # process in z-slabs to bound the temporary grid
    slab = max(1, (1 << 26) // (nx * ny))
    xs = torch.arange(nx, device=dev, dtype=dt)
    ys = torch.arange(ny, device=dev, dtype=dt)
    sx, sy, sz = 2.0 / max(nx - 1, 1), 2.0 / max(ny - 1, 1), 2.0 / max(nz - 1, 1)
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        zs = torch.arange(z0, z1, device=dev, dtype=dt)
        gz, gy, gx = torch.meshgrid(zs, ys, xs, indexing="ij")
        grid = torch.stack([(gx + u[0, z0:z1]) * sx - 1.0,
                            (gy + u[1, z0:z1]) * sy - 1.0,
                            (gz + u[2, z0:z1]) * sz - 1.0], -1)[None]
        out[z0:z1] = torch.nn.functional.grid_sample(
            M[None, None], grid, mode="bilinear", padding_mode="border", align_corners=True)[0, 0]
        del grid, gx, gy, gz
    return out


def smooth_field(shape, sigma: float, max_norm: float, rng=None, gen=None, device="cpu") -> torch.Tensor:
    """3 channels of N(0,1) white noise, Gaussian-smoothed (sigma voxels,
    periodic borders so the field is stationary), then scaled so that
    max_p |u(p)|_2 = max_norm.  Returns [3, nz, ny, nx] float32."""
    nz, ny, nx = shape
    if gen is not None:
        noise = torch.randn((3, nz, ny, nx), generator=gen, device=device, dtype=torch.float32)
    else:
        noise = torch.from_numpy(rng.standard_normal((3, nz, ny, nx), dtype=np.float32)).to(device)
    u = gaussian_smooth(noise, sigma, periodic=True)
    del noise
    norm = torch.sqrt((u.double() ** 2).sum(0)).max().item() if u.numel() < (1 << 28) else \
        max(torch.sqrt((u[:, z:z + 64].double() ** 2).sum(0)).max().item() for z in range(0, nz, 64))
    if max_norm <= 0 or norm == 0:
        return torch.zeros_like(u)
    u.mul_(max_norm / norm)
    return u


def _uniform(rng, gen, lo, hi, n, device):
    if gen is not None:
        return (torch.rand(n, generator=gen, device=device, dtype=torch.float64) * (hi - lo) + lo).cpu().numpy()
    return rng.uniform(lo, hi, n)


def blobs(shape, n_blobs: int, sigma_range, amp_range=(0.2, 1.0), noise_std=0.02, rng=None, gen=None,
          device="cpu") -> torch.Tensor:
    """Sum of isotropic 3-D Gaussian blobs (centres uniform in the volume) plus
    white noise N(0, noise_std^2).  float32 [nz, ny, nx]."""
    nz, ny, nx = shape
    cx = _uniform(rng, gen, 0, nx - 1, n_blobs, device)
    cy = _uniform(rng, gen, 0, ny - 1, n_blobs, device)
    cz = _uniform(rng, gen, 0, nz - 1, n_blobs, device)
    sg = _uniform(rng, gen, sigma_range[0], sigma_range[1], n_blobs, device)
    amp = _uniform(rng, gen, amp_range[0], amp_range[1], n_blobs, device)
    xs = torch.arange(nx, device=device, dtype=torch.float32)
    ys = torch.arange(ny, device=device, dtype=torch.float32)
    zs = torch.arange(nz, device=device, dtype=torch.float32)
    F = torch.zeros(shape, device=device, dtype=torch.float32)
    for j in range(n_blobs):
        gx = torch.exp(-0.5 * ((xs - cx[j]) / sg[j]) ** 2)
        gy = torch.exp(-0.5 * ((ys - cy[j]) / sg[j]) ** 2)
        gz = float(amp[j]) * torch.exp(-0.5 * ((zs - cz[j]) / sg[j]) ** 2)
        F.add_(gz[:, None, None] * (gy[:, None] * gx[None, :])[None])
    if noise_std > 0:
        if gen is not None:
            F.add_(torch.randn(shape, generator=gen, device=device, dtype=torch.float32), alpha=noise_std)
        else:
            F.add_(torch.from_numpy(rng.standard_normal(shape, dtype=np.float32)).to(device), alpha=noise_std)
    return F


def ellipsoid_labels(shape, n_labels: int, rng=None, gen=None, device="cpu") -> torch.Tensor:
    """Background 0 plus n_labels random ellipsoids (labels 1..n, later ones
    overwrite earlier ones).  Sizes are fractions of the volume, so the same
    recipe scales with the grid.  uint8 [nz, ny, nx]."""
    nz, ny, nx = shape
    n = np.array([nx, ny, nz], dtype=np.float64)
    lab = torch.zeros(shape, dtype=torch.uint8, device=device)
    xs = torch.arange(nx, device=device, dtype=torch.float32)
    ys = torch.arange(ny, device=device, dtype=torch.float32)
    zs = torch.arange(nz, device=device, dtype=torch.float32)
    for l in range(1, n_labels + 1):
        c = _uniform(rng, gen, 0.25, 0.75, 3, device) * n
        ax = _uniform(rng, gen, 0.10, 0.32, 3, device) * n
        ang = _uniform(rng, gen, 0.0, math.pi, 3, device)
        ca, sa = np.cos(ang), np.sin(ang)
        Rz = np.array([[ca[0], -sa[0], 0], [sa[0], ca[0], 0], [0, 0, 1]])
        Ry = np.array([[ca[1], 0, sa[1]], [0, 1, 0], [-sa[1], 0, ca[1]]])
        Rx = np.array([[1, 0, 0], [0, ca[2], -sa[2]], [0, sa[2], ca[2]]])
        R = torch.tensor(Rz @ Ry @ Rx, dtype=torch.float32, device=device)
        for z0 in range(0, nz, 64):
            z1 = min(nz, z0 + 64)
            dz = (zs[z0:z1] - float(c[2]))[:, None, None]
            dy = (ys - float(c[1]))[None, :, None]
            dx = (xs - float(c[0]))[None, None, :]
            q = 0.0
            for k in range(3):
                comp = R[0, k] * dx + R[1, k] * dy + R[2, k] * dz
                q = q + (comp / float(ax[k])) ** 2
            lab[z0:z1][q <= 1.0] = l
    return lab


def _paint(labels: torch.Tensor, table: np.ndarray, noise_std: float, smooth_sigma: float, rng=None, gen=None):
    t = torch.tensor(table, dtype=torch.float32, device=labels.device)
    img = t[labels.long()]
    if noise_std > 0:
        if gen is not None:
            img.add_(torch.randn(img.shape, generator=gen, device=img.device, dtype=torch.float32), alpha=noise_std)
        else:
            img.add_(torch.from_numpy(rng.standard_normal(tuple(img.shape), dtype=np.float32)).to(img.device),
                     alpha=noise_std)
    return gaussian_smooth(img, smooth_sigma)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def mono_pair(n: int, seed: int, blob_sigma=(2.0, 8.0), field_sigma=4.0, max_disp=3.0, n_blobs=40,
              device="cpu", gpu_rng: bool = False):
    """Mono-modal pair as the workload states it: F = B + N(0, 0.02^2), the
    blob image B (sum of Gaussian blobs) with its noise, and M = F o (id +
    u_true) for a smooth field u_true (white noise smoothed at field_sigma,
    scaled to max |u| = max_disp).  The noise is part of the imaged texture
    and moves with it, so LNCC windows on the flat parts of the blobs still
    carry a matching signal."""
    shape = (n, n, n)
    rng = None if gpu_rng else np.random.default_rng(seed)
    gen = None
    if gpu_rng:
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
    F = blobs(shape, n_blobs, blob_sigma, noise_std=0.0, rng=rng, gen=gen, device=device)
    u_true = smooth_field(shape, field_sigma, max_disp, rng=rng, gen=gen, device=device)
    if gen is not None:
        F.add_(torch.randn(shape, generator=gen, device=device, dtype=torch.float32), alpha=0.02)
    else:
        F.add_(torch.from_numpy(rng.standard_normal(shape, dtype=np.float32)).to(device), alpha=0.02)
    M = _sample_trilinear(F, u_true)
    return dict(F=F, M=M, u_true=u_true, seed=seed, rng="philox" if gpu_rng else "pcg64")


def label_images(shape, n_labels: int, noise_std: float, smooth_sigma: float, rng=None, gen=None, device="cpu"):
    """Two modalities of one phantom: an n_labels ellipsoid map painted through
    a random intensity table (U[0,1] per label) and through a second random
    table that is not monotone in the first, each with N(0, noise_std^2) and
    Gaussian smoothing at smooth_sigma.  Returns (first, second), aligned."""
    lab = ellipsoid_labels(shape, n_labels, rng=rng, gen=gen, device=device)
    tF = _uniform(rng, gen, 0.0, 1.0, n_labels + 1, device)
    while True:
        tM = _uniform(rng, gen, 0.0, 1.0, n_labels + 1, device)
        order = np.argsort(tF)
        d = np.diff(tM[order])
        if (d > 0).any() and (d < 0).any():
            break
    F = _paint(lab, tF, noise_std, smooth_sigma, rng=rng, gen=gen)
    M = _paint(lab, tM, noise_std, smooth_sigma, rng=rng, gen=gen)
    return F, M


def multimodal_pair(n: int, seed: int, field_sigma=6.0, max_disp=5.0, n_labels=6, device="cpu",
                    gpu_rng: bool = False):
    """Multi-modal phantom pair: a 6-label ellipsoid map; F paints the labels
    with a random table (U[0,1]) + N(0, 0.03^2), smoothed at sigma 1; M paints
    the same labels through a random non-monotone table, same noise and
    smoothing, then is warped by a smooth field.  Returns intensity ranges."""
    shape = (n, n, n)
    rng = None if gpu_rng else np.random.default_rng(seed)
    gen = None
    if gpu_rng:
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
    F, M0 = label_images(shape, n_labels, 0.03, 1.0, rng=rng, gen=gen, device=device)
    u_true = smooth_field(shape, field_sigma, max_disp, rng=rng, gen=gen, device=device)
    M = _sample_trilinear(M0, u_true)
    del M0
    f_range = (float(F.min()), float(F.max()))
    m_range = (float(M.min()), float(M.max()))
    return dict(F=F, M=M, u_true=u_true, f_range=f_range, m_range=m_range, seed=seed,
                rng="philox" if gpu_rng else "pcg64")


CONFIGS = {
    # name: (kind, n, generator kwargs, loss/optimiser settings)
    "c0": dict(kind="lncc", n=64, seed=0, window=7, lam=0.1, lr=0.1, iters=50, dtype="f32",
               gen=dict(blob_sigma=(2.0, 8.0), field_sigma=4.0, max_disp=3.0)),
    "c1": dict(kind="mi", n=192, seed=1, bins=32, lam=0.05, lr=0.1, iters=200, dtype="f32",
               gen=dict(field_sigma=6.0, max_disp=5.0)),
    "c2": dict(kind="lncc", n=512, seed=2, window=9, lam=0.1, lr=0.1, iters=300, dtype="bf16",
               gen=dict(blob_sigma=(16.0, 64.0), field_sigma=16.0, max_disp=12.0)),
    "c4": dict(kind="mi", n=1280, seed=4, bins=32, lam=0.05, lr=0.1, iters=200, dtype="bf16",
               gen=dict(field_sigma=40.0, max_disp=30.0)),
}


def make(config: str, device="cpu", n: int | None = None, seed: int | None = None):
    """Generate the pair of a named workload (optionally at another size)."""
    c = CONFIGS[config]
    n = c["n"] if n is None else n
    seed = c["seed"] if seed is None else seed
    big = n > 512
    if c["kind"] == "lncc":
        g = dict(c["gen"])
        out = mono_pair(n, seed, device=device, gpu_rng=big, **g)
    else:
        out = multimodal_pair(n, seed, device=device, gpu_rng=big, **c["gen"])
    out["config"] = dict(c, n=n, seed=seed)
    return out
