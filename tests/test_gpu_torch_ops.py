"""The autograd front end (paper_2509_25044_gb300.torch_ops): values and
gradients in u through torch.autograd equal the FP64 oracle's."""
import numpy as np
import pytest
import torch

import oracle as O
from _util import GRAD_RTOL, LOSS_RTOL, WARP_TOL, assert_rel, field, mono_images, multimodal_images, rel_l2, to64

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ops():
    from paper_2509_25044_gb300 import build, capi, torch_ops
    build.build()
    capi.load()
    return torch_ops


@pytest.mark.parametrize("pad", [0, 1])
def test_warp_autograd_matches_oracle(ops, pad):
    shape = (12, 10, 33)
    _, M = mono_images(shape, 91)
    u = field(shape, 3.0, 2.0, 92)
    g = torch.from_numpy(np.random.default_rng(93).standard_normal(shape).astype(np.float32))
    ud = u.to(DEV).requires_grad_()
    J = ops.Warp.apply(M.to(DEV), ud, pad)
    (J * g.to(DEV)).sum().backward()
    torch.cuda.synchronize()
    Jr, dJ = O.warp(to64(M), to64(u), pad, with_grad=True)
    assert np.abs(to64(J.detach()) - Jr).max() <= WARP_TOL * float(M.max() - M.min())
    assert rel_l2(to64(ud.grad), dJ * to64(g)[None]) <= GRAD_RTOL


@pytest.mark.parametrize("kind", ["lncc", "mi"])
def test_losses_autograd_match_oracle(ops, kind):
    shape = (16, 18, 40)
    F, M = (mono_images if kind == "lncc" else multimodal_images)(shape, 94)
    u = field(shape, 3.0, 2.0, 95)
    ud = u.to(DEV).requires_grad_()
    if kind == "lncc":
        C = ops.LNCCLoss.apply(F.to(DEV), M.to(DEV), ud, 5, 1e-4)
        spec = O.LossSpec(kind=O.LOSS_LNCC, window=5, eps=1e-4)
    else:
        fr, mr = (float(F.min()), float(F.max())), (float(M.min()), float(M.max()))
        C = ops.MILoss.apply(F.to(DEV), M.to(DEV), ud, 32, fr, mr)
        spec = O.LossSpec(kind=O.LOSS_MI, bins=32, f_range=fr, m_range=mr)
    (2.0 * C).backward()  # an upstream gradient other than 1
    torch.cuda.synchronize()
    Sr, gr = O.similarity_and_grad(to64(F), to64(M), to64(u), spec)
    Cr = 1.0 - Sr if kind == "lncc" else -Sr
    assert_rel(float(C.detach()), Cr, LOSS_RTOL, "loss")
    assert rel_l2(to64(ud.grad), 2.0 * gr) <= GRAD_RTOL


def test_optimize_decreases_the_objective(ops):
    from paper_2509_25044_gb300 import synth
    from paper_2509_25044_gb300.register import RegConfig
    d = synth.make("c0", device=DEV)
    u, hist = ops.optimize(d["F"], d["M"], RegConfig(loss="lncc", window=7, eps=1e-9, lam=2.0, lr=0.1), iters=30)
    assert tuple(u.shape) == (3,) + tuple(d["F"].shape)
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
