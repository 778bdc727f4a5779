"""The allocation-free MI entry point (reg_mi_loss_grad_noalloc).

It exists for callers that cannot allocate device memory -- an application
or framework that has reserved the whole GPU for its own memory pool, or a
latency-critical loop that must not enter the allocator -- and so keeps its
scratch in a fixed array inside the library instead of a caller workspace.
This test calls it through the C ABI twice in a row, on different inputs
(so a histogram left over from the first call would show), and checks both
results against the workspace entry point reg_loss_grad with the parity
tolerances used everywhere else.  It lives in its own file, collected last.
"""
import pytest
import torch

from _util import GRAD_RTOL, LOSS_RTOL, assert_rel, field, multimodal_images, rel_l2, to64

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def test_noalloc_matches_workspace_entry_point_twice(capi):
    shape = (37, 41, 44)
    F, M = multimodal_images(shape, 101)
    fr = (float(F.min()), float(F.max()))
    mr = (float(M.min()), float(M.max()))
    loss = capi.mi_desc(fr, mr, 32)
    Fd, Md = F.to(DEV), M.to(DEV)
    ws = capi.workspace(loss, Fd)
    for call, seed in enumerate((102, 103)):
        u = field(shape, 3.0, 2.0 + call, seed).to(DEV)
        sim_ref, g_ref = capi.reg_loss_grad(loss, Fd, Md, u, ws)
        sim = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
        g = torch.full_like(u, float("nan"))
        capi.reg_mi_loss_grad_noalloc(loss, Fd, Md, u, sim=sim, grad=g)
        torch.cuda.synchronize()
        assert_rel(sim.item(), sim_ref.item(), LOSS_RTOL, f"MI, call {call + 1}")
        assert rel_l2(to64(g), to64(g_ref)) <= GRAD_RTOL, f"gradient, call {call + 1}"
    assert capi.reg_get_device_error() == 0


def test_noalloc_rejects_bins_beyond_its_scratch(capi):
    shape = (8, 8, 8)
    F = torch.rand(shape, device=DEV)
    u = torch.zeros((3,) + shape, device=DEV)
    with pytest.raises(capi.RegError) as e:
        capi.reg_mi_loss_grad_noalloc(capi.mi_desc((0, 1), (0, 1), 65), F, F, u)
    assert e.value.status == 2  # REG_ERR_SHAPE
    with pytest.raises(capi.RegError) as e:
        capi.reg_mi_loss_grad_noalloc(capi.lncc_desc(7, 1e-5), F, F, u)
    assert e.value.status == 9  # REG_ERR_UNSUPPORTED
