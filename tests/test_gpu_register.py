"""The registration driver on the small mono-modal and multimodal workloads:
the objective decreases, the field does not fold, and a replay is bitwise
identical."""
import numpy as np
import pytest
import torch

from paper_2509_25044_gb300 import synth
from paper_2509_25044_gb300.register import RegConfig, Registration, register

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_c0_lncc_converges_without_folding():
    d = synth.make("c0", device=DEV)
    # lam = 2: with the noise texture shared by F and M, lam = 1 folds a voxel or two
    cfg = RegConfig(loss="lncc", window=7, eps=1e-9, lam=2.0, lr=0.1)
    res = register(d["F"], d["M"], cfg, 50)
    assert np.all(np.isfinite(res.objective))
    assert res.objective[-1] < res.objective[0]
    assert res.extra["min_det"] > 0 and res.extra["n_fold"] == 0
    again = register(d["F"], d["M"], cfg, 50)
    assert torch.equal(res.u, again.u)


def test_c1_mi_small_converges():
    d = synth.make("c1", device=DEV, n=64)
    # lam = 2: at lam = 1 the MI run folds a few voxels of the 64^3 grid
    cfg = RegConfig(loss="mi", bins=32, f_range=d["f_range"], m_range=d["m_range"], lam=2.0, lr=0.1)
    reg = Registration(d["F"], d["M"], cfg)
    res = reg.run(60)
    assert res.objective[-1] < res.objective[0]  # MI increases: -MI + lam R decreases
    assert res.sim[-1] > res.sim[0]
    assert reg.fold_check()["n_fold"] == 0


def test_multiscale_schedule():
    """Coarse-to-fine (scales 4, 2, 1): every level decreases its objective,
    the returned field is full size, and its full-resolution objective is
    below the objective at zero displacement."""
    from paper_2509_25044_gb300.register import register_multiscale
    d = synth.make("c0", device=DEV)
    cfg = RegConfig(loss="lncc", window=7, eps=1e-9, lam=2.0, lr=0.1)
    out = register_multiscale(d["F"], d["M"], cfg, scales=(4, 2, 1), iters=(30, 30, 30))
    assert [lv["scale"] for lv in out["levels"]] == [4, 2, 1]
    n = tuple(d["F"].shape)
    assert [lv["shape"] for lv in out["levels"]] == [tuple(s // 4 for s in n), tuple(s // 2 for s in n), n]
    for lv in out["levels"]:
        obj = lv["result"].objective
        assert np.all(np.isfinite(obj)) and obj[-1] < obj[0]
    assert tuple(out["u"].shape) == (3,) + n
    r = Registration(d["F"], d["M"], cfg)
    zero = r.objective()["objective"]
    fin = Registration(d["F"], d["M"], cfg, u0=out["u"]).objective()["objective"]
    assert fin < zero
    assert out["ms"] > 0
    with pytest.raises(ValueError):
        register_multiscale(d["F"], d["M"], cfg, scales=(2, 4, 1), iters=(1, 1, 1))
