"""Shared helpers for the GPU parity tests: seeded inputs and the tolerance
checks (the bars come from the method's stated accuracy targets)."""
import numpy as np
import torch

from paper_2509_25044_gb300 import synth

# FP32 path vs FP64 oracle
WARP_TOL = 1e-5          # max-abs, times the image range
LOSS_RTOL = 1e-5         # similarity, relative
GRAD_RTOL = 1e-4         # gradient, relative L2
# BF16 storage vs the FP32-input oracle
LOSS_RTOL_BF16 = 2e-3
GRAD_RTOL_BF16 = 5e-3


def smooth_noise(shape, sigma, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    t = torch.from_numpy(rng.standard_normal(shape).astype(np.float32))
    t = synth.gaussian_smooth(t, sigma)
    t = t / t.abs().max() * scale
    return t


def field(shape, sigma, max_disp, seed):
    rng = np.random.default_rng(seed)
    return synth.smooth_field(shape, sigma, max_disp, rng=rng)


def mono_images(shape, seed):
    """Blob image F and a smooth intensity-perturbed moving image M."""
    rng = np.random.default_rng(seed)
    n = max(shape)
    F = synth.blobs(shape, 12, (max(1.5, n / 16), max(3.0, n / 5)), rng=rng)
    M = F + 0.3 * smooth_noise(shape, 2.0, seed + 1)
    return F, M


def multimodal_images(shape, seed):
    rng = np.random.default_rng(seed)
    lab = synth.ellipsoid_labels(shape, 6, rng=rng)
    tF = rng.uniform(0, 1, 7)
    tM = rng.permutation(rng.uniform(0, 1, 7))
    F = synth._paint(lab, tF, 0.03, 1.0, rng=rng)
    M = synth._paint(lab, tM, 0.03, 1.0, rng=rng)
    return F, M


def to64(t):
    return t.detach().double().cpu().numpy()


def bf16_values(t):
    """The values a bfloat16 copy of t holds (as float32 on the same device)."""
    return t.to(torch.bfloat16).float()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_rel(a, b, rtol, what=""):
    a, b = float(a), float(b)
    assert abs(a - b) <= rtol * abs(b), f"{what}: {a} vs {b} (rel {abs(a - b) / max(abs(b), 1e-300):.3e})"


def assert_bf16_drift(g_gpu, g_bf16_oracle, g_f32_oracle, what=""):
    """Against the FP32 images, the BF16-stored path may differ by no more
    than the oracle itself does when fed the BF16 values (the drift that the
    input rounding causes) plus the FP32 parity bar on top of it (triangle
    inequality: |G - O32| <= |G - Obf| + |Obf - O32|, with |G - Obf| <=
    GRAD_RTOL |Obf| asserted separately).  Both are printed."""
    drift = rel_l2(g_bf16_oracle, g_f32_oracle)
    err = rel_l2(g_gpu, g_f32_oracle)
    print(f"{what}: gradient vs the FP32-image oracle {err:.3e}; the oracle's own BF16-input drift {drift:.3e}")
    assert err <= drift + GRAD_RTOL * (1.0 + drift), (what, err, drift)
