"""The drivers and the autograd front end against a stand-in for the CUDA
library, on the CPU: every entry point returns success and computes nothing,
so these tests check what the Python layer does around the library -- that
every buffer a driver allocates passes the binding's checks (dtype,
contiguity, size), and that each driver calls the entry points in the order
its iteration needs.  Numbers are checked by the GPU tests, not here."""
import ctypes

import pytest
import torch

from paper_2509_25044_gb300 import capi


class _FakeLib:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("reg_"):
            raise AttributeError(name)

        def entry(*args):
            self.calls.append(name)
            return 0
        return entry


class _FakeEvent:
    def __init__(self, *a, **k):
        pass

    def record(self, *a, **k):
        pass

    def elapsed_time(self, other):
        return 0.0


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(capi, "_lib", lambda: lib)
    # host tensors stand in for device memory here (the fake never reads them)
    monkeypatch.setattr(capi, "_ptr", lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))
    monkeypatch.setattr(capi, "_stream", lambda t=None: None)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(capi, "_nn_ready", False)  # the real library's signatures stay untouched
    from paper_2509_25044_gb300.register import Registration
    monkeypatch.setattr(Registration, "_require_device", staticmethod(lambda F: None))
    return lib


def _pair(n=8):
    g = torch.Generator().manual_seed(0)
    return torch.rand((n, n, n), generator=g), torch.rand((n, n, n), generator=g)


def test_svf_driver_orchestration(fake):
    from paper_2509_25044_gb300.register import RegConfig, register_svf
    F, M = _pair()
    out = register_svf(F, M, RegConfig(loss="lncc", window=3, lam=1.0), iters=3, steps=4)
    per_iter = ["reg_exp_field", "reg_loss_grad", "reg_exp_field_backward", "reg_regularize", "reg_step"]
    body = [c for c in fake.calls if c != "reg_workspace_size"]
    assert body == per_iter * 3 + ["reg_exp_field"]
    assert out["objective"].shape == (3,) and tuple(out["u"].shape) == (3, 8, 8, 8)


@pytest.mark.parametrize("on_device", [True, False])
def test_affine_driver_orchestration(fake, on_device):
    from paper_2509_25044_gb300.register import RegConfig, register_affine
    F, M = _pair(16)
    cfg = RegConfig(loss="mi", bins=16)
    out = register_affine(F, M, cfg, scales=(4, 2, 1), iters=(3, 2, 1), on_device=on_device)
    body = [c for c in fake.calls if c != "reg_workspace_size"]
    # the pyramid (F and M at 2x and 4x), then per iteration one composite
    # gradient (on the device: with the transform in device memory, followed
    # by the device Adam step that writes the next transform)
    per_iter = (["reg_loss_grad_composite_dev", "reg_affine_adam_step"] if on_device
                else ["reg_loss_grad_composite"])
    assert body == ["reg_downsample2"] * 4 + per_iter * 6
    assert [lv["scale"] for lv in out["levels"]] == [4, 2, 1]
    assert out["A"].shape == (3, 3) and out["t"].shape == (3,)


@pytest.mark.parametrize("kind", ["lncc", "mi"])
def test_autograd_front_end_calls(fake, kind):
    from paper_2509_25044_gb300 import torch_ops
    F, M = _pair()
    u = torch.zeros((3, 8, 8, 8), requires_grad=True)
    if kind == "lncc":
        C = torch_ops.LNCCLoss.apply(F, M, u, 3, 1e-5)
    else:
        C = torch_ops.MILoss.apply(F, M, u, 16)
    C.backward()
    assert [c for c in fake.calls if c != "reg_workspace_size"] == ["reg_loss", "reg_loss_grad"]
    assert u.grad is not None and tuple(u.grad.shape) == (3, 8, 8, 8)
    fake.calls.clear()
    J = torch_ops.Warp.apply(M, u)
    J.sum().backward()
    assert [c for c in fake.calls if c != "reg_workspace_size"] == ["reg_warp", "reg_warp_composite_backward"]


def test_fake_library_leaves_the_checks_in_place(fake):
    """The stand-in replaces only the library: a short buffer is still
    refused by the binding."""
    F, M = _pair()
    u = torch.zeros((3, 8, 8, 8))
    with pytest.raises(ValueError, match="grad"):
        capi.reg_loss_grad(capi.lncc_desc(3, 1e-5), F, M, u, torch.empty(0), grad=torch.empty(10))
    assert fake.calls == []


def _body(lib):
    return [c for c in lib.calls if c != "reg_workspace_size"]


def test_registration_fused_and_smoothing_paths(fake):
    from paper_2509_25044_gb300.register import RegConfig, Registration
    F, M = _pair()
    r = Registration(F, M, RegConfig(loss="lncc", window=3, moments="bf16"))
    res = r.run(4)
    assert _body(fake) == ["reg_run"] and res.objective.shape == (4,) and r.t == 4
    fake.calls.clear()
    r.objective()
    r.fold_check()
    assert _body(fake) == ["reg_loss", "reg_regularize", "reg_jacdet_min"]
    fake.calls.clear()
    r = Registration(F, M, RegConfig(loss="mi", bins=16, sigma_grad=1.0, sigma_warp=0.5))
    r.run(2)
    it = ["reg_loss_grad", "reg_regularize", "reg_smooth_field", "reg_step", "reg_smooth_field"]
    assert _body(fake) == it * 2
    fake.calls.clear()
    r = Registration(F, M, RegConfig(loss="lncc", window=3, sigma_grad=1.0), affine=capi.affine_desc())
    r.run(1)
    assert _body(fake) == ["reg_loss_grad_composite", "reg_regularize", "reg_smooth_field", "reg_step"]


def test_multiscale_driver_orchestration(fake):
    from paper_2509_25044_gb300.register import RegConfig, register_multiscale
    F, M = _pair(16)
    out = register_multiscale(F, M, RegConfig(loss="lncc", window=3), scales=(4, 2, 1), iters=(2, 2, 2))
    assert _body(fake) == (["reg_downsample2"] * 4 + ["reg_run", "reg_nn_field_upsample", "reg_run",
                                                       "reg_nn_field_upsample", "reg_run"])
    assert [lv["shape"] for lv in out["levels"]] == [(4, 4, 4), (8, 8, 8), (16, 16, 16)]
    assert tuple(out["u"].shape) == (3, 16, 16, 16)
