"""The seeded input recipe (paper_2509_25044_gb300.synth), on the CPU: the
generators are deterministic per seed, the fields have the stated size, and
the moving image is the fixed one seen through the ground-truth field in the
same convention the oracle's warp uses (channel 0 along x, BORDER padding)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_25044_gb300 import synth


def test_same_seed_same_bits_other_seed_other_pair():
    a = synth.make("c0", n=16)
    b = synth.make("c0", n=16)
    for k in ("F", "M", "u_true"):
        assert torch.equal(a[k], b[k]), k
    c = synth.make("c0", n=16, seed=7)
    assert not torch.equal(a["F"], c["F"])
    m1, m2 = synth.make("c1", n=16), synth.make("c1", n=16)
    assert torch.equal(m1["M"], m2["M"]) and m1["f_range"] == m2["f_range"]


@pytest.mark.parametrize("max_norm", [0.0, 2.5])
def test_smooth_field_has_the_stated_maximum_norm(max_norm):
    u = synth.smooth_field((12, 10, 14), 2.0, max_norm, rng=np.random.default_rng(3))
    assert u.shape == (3, 12, 10, 14) and u.dtype == torch.float32
    norm = torch.sqrt((u.double() ** 2).sum(0))
    assert abs(float(norm.max()) - max_norm) <= 1e-6 * max(1.0, max_norm)


def test_gaussian_smooth_equals_scipy_nearest():
    from scipy.ndimage import gaussian_filter
    v = np.random.default_rng(4).standard_normal((9, 11, 13))
    out = synth.gaussian_smooth(torch.from_numpy(v), 1.3).numpy()
    np.testing.assert_allclose(out, gaussian_filter(v, 1.3, mode="nearest", truncate=4.0), atol=1e-12)


@pytest.mark.parametrize("config", ["c0", "c1"])
def test_moving_image_is_the_warp_by_the_true_field(config):
    """M(p) = M0(p + u_true(p)) with the oracle's trilinear warp: for the
    mono-modal pair M0 = F; the phantom's unwarped M0 is not returned, so
    there the check is that the generator's sampler equals the oracle's on
    the returned field and image."""
    d = synth.make(config, n=20)
    u = d["u_true"].double().numpy()
    if config == "c0":
        ref = O.warp(d["F"].double().numpy(), u, O.PAD_BORDER)
        np.testing.assert_allclose(d["M"].double().numpy(), ref, atol=2e-6 * float(d["F"].abs().max()))
    else:
        M = d["M"]
        ref = O.warp(M.double().numpy(), u, O.PAD_BORDER)
        got = synth._sample_trilinear(M, d["u_true"]).double().numpy()
        np.testing.assert_allclose(got, ref, atol=2e-6 * float(M.abs().max()))
        assert d["f_range"] == (float(d["F"].min()), float(d["F"].max()))
        assert d["m_range"] == (float(M.min()), float(M.max()))
