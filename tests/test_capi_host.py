"""C-ABI library: builds, loads, exports every symbol of include/reg.h, and
rejects bad arguments on the host before anything reaches a GPU.  CPU only:
no call here passes arguments that would launch a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "reg.h")).read()
    return sorted(set(re.findall(r"REG_API[^;(]*?\b(reg_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(capi):
    syms = header_symbols()
    assert len(syms) >= 12
    lib = ctypes.CDLL(capi.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(capi.EXPORTS) == syms


def test_version_and_status_strings(capi):
    assert capi.reg_version() >= 100
    for code in range(10):
        assert capi.reg_status_string(code)
    assert capi.reg_status_string(999) == "unknown status"


def _lib(capi):
    return capi.load()


D = None


def dims(nx=8, ny=8, nz=8):
    from paper_2509_25044_gb300.capi import RegDims
    return RegDims(nx, ny, nz)


def test_workspace_size_host_only(capi):
    lncc = capi.lncc_desc(7, 1e-5)
    mi = capi.mi_desc((0, 1), (0, 1), 32)
    a = capi.reg_workspace_size(lncc, dims(64, 64, 64))
    b = capi.reg_workspace_size(mi, dims(64, 64, 64))
    c = capi.reg_workspace_size(None, dims(64, 64, 64))
    assert a >= 3 * 4 * 64 ** 3  # LNCC keeps three coefficient fields
    assert b < a and c <= b
    with pytest.raises(capi.RegError) as e:
        capi.reg_workspace_size(capi.lncc_desc(8, 1e-5), dims())
    assert e.value.status == 2
    with pytest.raises(capi.RegError):
        capi.reg_workspace_size(capi.mi_desc((1, 0), (0, 1), 32), dims())
    with pytest.raises(capi.RegError):
        capi.reg_workspace_size(capi.mi_desc((0, 1), (0, 1), 100), dims())
    with pytest.raises(capi.RegError):
        capi.reg_workspace_size(None, dims(0, 4, 4))


FAKE = 0x10000  # 16-byte aligned, never dereferenced: validation fails first


def test_warp_validation(capi):
    L = _lib(capi)
    vp = ctypes.c_void_p
    assert L.reg_warp(vp(FAKE), 0, vp(FAKE), dims(0, 4, 4), 0, vp(FAKE), None, None) == 2
    assert L.reg_warp(vp(FAKE), 7, vp(FAKE), dims(), 0, vp(FAKE), None, None) == 3
    assert L.reg_warp(vp(FAKE), 0, vp(FAKE), dims(), 5, vp(FAKE), None, None) == 1
    assert L.reg_warp(None, 0, vp(FAKE), dims(), 0, vp(FAKE), None, None) == 1
    assert L.reg_warp(vp(FAKE + 4), 0, vp(FAKE), dims(), 0, vp(FAKE), None, None) == 4
    assert L.reg_warp(vp(FAKE), 0, vp(FAKE), dims(), 0, vp(FAKE), vp(FAKE + 8), None) == 4


def test_loss_and_iterate_validation(capi):
    L = _lib(capi)
    vp = ctypes.c_void_p
    lncc = capi.lncc_desc(7, 1e-5)
    need = capi.reg_workspace_size(lncc, dims())
    # workspace too small
    assert L.reg_loss(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, vp(FAKE), dims(), 0, vp(FAKE), need - 1,
                      vp(FAKE), None) == 5
    # unknown LNCC gradient mode (neither the exact adjoint nor the ANTs approximation)
    bad_mode = capi.lncc_desc(7, 1e-5)
    bad_mode.lncc_grad = 2
    assert L.reg_loss(ctypes.byref(bad_mode), vp(FAKE), vp(FAKE), 0, vp(FAKE), dims(), 0, vp(FAKE), need,
                      vp(FAKE), None) == 1
    # unknown MI estimator
    bad_est = capi.mi_desc((0.0, 1.0), (0.0, 1.0), 32)
    bad_est.mi_estimator = 5
    assert L.reg_loss(ctypes.byref(bad_est), vp(FAKE), vp(FAKE), 0, vp(FAKE), dims(), 0, vp(FAKE), 1 << 30,
                      vp(FAKE), None) == 1
    # bad eps
    bad = capi.lncc_desc(7, -1.0)
    assert L.reg_loss(ctypes.byref(bad), vp(FAKE), vp(FAKE), 0, vp(FAKE), dims(), 0, vp(FAKE), need,
                      vp(FAKE), None) == 1
    # null similarity output
    assert L.reg_loss_grad(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, vp(FAKE), dims(), 0, vp(FAKE), need, None,
                           vp(FAKE), None) == 1
    adam = capi.adam_desc(0.1, grad_scale=512.0)
    # u_out overlapping u_in
    assert L.reg_iterate(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, vp(FAKE), vp(FAKE + 256), vp(FAKE), vp(FAKE),
                         dims(), 0, 0.1, ctypes.byref(adam), 1, vp(FAKE), need, vp(FAKE), None, None) == 1
    # step count must be >= 1
    assert L.reg_iterate(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, vp(FAKE), vp(FAKE << 8), vp(FAKE), vp(FAKE),
                         dims(), 0, 0.1, ctypes.byref(adam), 0, vp(FAKE), need, vp(FAKE), None, None) == 1
    # multi-iteration run: negative counts, overlapping ping-pong buffers; 0 iterations is a no-op
    def run(t0, iters, ub=FAKE << 8):
        return L.reg_run(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, vp(FAKE), vp(ub), vp(FAKE), vp(FAKE), dims(), 0,
                         0.1, ctypes.byref(adam), t0, iters, vp(FAKE), need, vp(FAKE), T, None)
    T = None
    assert run(0, -1) == 1
    assert run(-1, 5) == 1
    assert run(2 ** 31 - 3, 5) == 1
    assert run(0, 0) == 0
    assert run(0, 3, ub=FAKE + 256) == 1
    T = ctypes.byref(capi.affine_desc(t=(float("inf"), 0.0, 0.0)))  # a non-finite transform
    assert run(0, 3) == 1
    T = None
    badadam = capi.adam_desc(0.1, beta1=1.0)
    assert L.reg_step(vp(FAKE), vp(FAKE), vp(FAKE), vp(FAKE), vp(FAKE), dims(), ctypes.byref(badadam), 1,
                      None) == 1
    bf = capi.adam_desc(0.1, moment_dtype=9)
    assert L.reg_step(vp(FAKE), vp(FAKE), vp(FAKE), vp(FAKE), vp(FAKE), dims(), ctypes.byref(bf), 1, None) == 3
    assert L.reg_regularize(vp(FAKE), dims(), float("nan"), vp(FAKE), 1 << 20, vp(FAKE), None, None) == 1
    assert L.reg_debug_wait_flag(vp(FAKE), 1, 11 * 10 ** 9, None) == 1


def test_composite_validation(capi):
    """Composite sampler entry points reject bad transforms, dtypes and
    buffers before any launch."""
    L = _lib(capi)
    vp = ctypes.c_void_p
    ok = capi.affine_desc()
    nan = capi.affine_desc(A=[[1, 0, 0], [0, float("nan"), 0], [0, 0, 1]])
    inf = capi.affine_desc(s=(1.0, float("inf"), 1.0))
    for T, want in ((nan, 1), (inf, 1)):
        assert L.reg_warp_composite(vp(FAKE), 0, None, dims(), ctypes.byref(T), 0, vp(FAKE), None, None) == want
    assert L.reg_warp_composite(vp(FAKE), 0, None, dims(), None, 0, vp(FAKE), None, None) == 1
    assert L.reg_warp_composite(vp(FAKE), 7, None, dims(), ctypes.byref(ok), 0, vp(FAKE), None, None) == 3
    assert L.reg_warp_composite(vp(FAKE), 0, None, dims(), ctypes.byref(ok), 0, None, None, None) == 1
    assert L.reg_warp_composite(vp(FAKE), 0, vp(FAKE + 4), dims(), ctypes.byref(ok), 0, vp(FAKE), None, None) == 4
    # backward: workspace too small, missing upstream gradient
    need = capi.reg_workspace_size(None, dims())
    assert L.reg_warp_composite_backward(vp(FAKE), 0, None, dims(), ctypes.byref(ok), 0, vp(FAKE), None, None,
                                         vp(FAKE), need - 1, None) == 5
    assert L.reg_warp_composite_backward(vp(FAKE), 0, None, dims(), ctypes.byref(ok), 0, None, None, None,
                                         vp(FAKE), need, None) == 1
    lncc = capi.lncc_desc(7, 1e-5)
    wsl = capi.reg_workspace_size(lncc, dims())
    assert L.reg_loss_grad_composite(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, None, dims(), ctypes.byref(nan), 0,
                                     vp(FAKE), wsl, vp(FAKE), None, None, None) == 1
    assert L.reg_loss_grad_composite(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, None, dims(), ctypes.byref(ok), 0,
                                     vp(FAKE), wsl - 1, vp(FAKE), None, None, None) == 5
    assert L.reg_loss_grad_composite(ctypes.byref(lncc), vp(FAKE), vp(FAKE), 0, None, dims(), ctypes.byref(ok), 0,
                                     vp(FAKE), wsl, None, None, None, None) == 1


def test_field_composition_validation(capi):
    L = _lib(capi)
    vp = ctypes.c_void_p
    F2 = FAKE << 8
    # ga == NULL requires a and b to be one field
    assert L.reg_compose_fields_backward(vp(FAKE), vp(FAKE << 4), vp(FAKE << 6), dims(), 0, None, vp(F2), None) == 1
    # gb overlapping an input
    assert L.reg_compose_fields_backward(vp(FAKE), vp(FAKE), vp(FAKE << 6), dims(), 0, None, vp(FAKE + 64),
                                         None) == 1
    # steps out of range; backward past one step needs the saved fields
    assert L.reg_exp_field(vp(FAKE), dims(), 31, 0, vp(FAKE << 4), vp(F2), None, None) == 1
    assert L.reg_exp_field_backward(vp(FAKE), dims(), 3, 0, None, vp(FAKE << 4), vp(FAKE << 6), vp(F2),
                                    None) == 1
    # the gradient buffers must be distinct
    assert L.reg_exp_field_backward(vp(FAKE), dims(), 1, 0, None, vp(FAKE << 4), vp(FAKE << 4), vp(F2),
                                    None) == 1


def test_autograd_front_end_is_importable():
    """The torch.autograd wrappers load without a GPU (they run only on one)."""
    from paper_2509_25044_gb300 import torch_ops
    import torch
    assert issubclass(torch_ops.Warp, torch.autograd.Function)
    assert callable(torch_ops.LNCCLoss.apply) and callable(torch_ops.MILoss.apply)
    assert callable(torch_ops.optimize)


def test_product_package_has_no_oracle_dependency():
    """The product path must not import, link or execute the oracle."""
    pkg = os.path.join(ROOT, "paper_2509_25044_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "oracle.c" not in txt, f


def test_oracle_has_no_product_dependency():
    """The other direction: the oracle includes only the C standard library
    and imports nothing of the product package, so the two share no code."""
    d = os.path.join(ROOT, "oracle")
    for f in sorted(os.listdir(d)):
        if not f.endswith((".py", ".c", ".h")):
            continue
        txt = open(os.path.join(d, f)).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2509_25044_gb300", txt, re.M), f
        assert "libreg" not in txt, f
        for inc in re.findall(r"#include\s*([<\"][^>\"]+[>\"])", txt):
            assert inc in ("<math.h>", "<stdint.h>", "<stdlib.h>", "<string.h>", "<stdio.h>"), (f, inc)


def test_nn_validation(capi):
    """The learned initialiser's entry points reject bad shapes, enums, null
    and misaligned pointers with their documented codes before any launch."""
    L = capi.nn()
    vp = ctypes.c_void_p
    F, U = vp(FAKE), vp(FAKE + 8)  # aligned / misaligned, never dereferenced
    d = dims()
    # host-only sizes
    assert L.reg_nn_conv_kpad(8) == 256 and L.reg_nn_conv_kpad(16) == 448
    assert L.reg_nn_conv_scratch_bytes(4, 8) == 0
    assert L.reg_nn_dgrad_scratch_bytes(8, 4) == 0
    assert L.reg_nn_wgrad_scratch_bytes(dims(0, 4, 4), 8, 16) == 0
    # forward convolution: (in, Cin, W, bias, Cout, d, epilogue, slope, scratch, bytes, out, stream)
    fwd = L.reg_nn_conv3d_fwd
    assert fwd(F, 8, F, F, 8, dims(0, 4, 4), 0, 0.2, None, 0, F, None) == 2
    assert fwd(F, 12, F, F, 8, d, 0, 0.2, None, 0, F, None) == 2    # Cin % 8
    assert fwd(F, 136, F, F, 8, d, 0, 0.2, None, 0, F, None) == 2   # Cin > 128
    assert fwd(F, 8, F, F, 65, d, 2, 0.2, None, 0, F, None) == 2    # Cout > 64
    assert fwd(F, 8, F, F, 8, d, 3, 0.2, None, 0, F, None) == 1     # epilogue
    assert fwd(F, 8, F, F, 12, d, 0, 0.2, None, 0, F, None) == 2    # BF16 output needs Cout % 8
    assert fwd(None, 8, F, F, 8, d, 0, 0.2, None, 0, F, None) == 1
    assert fwd(U, 8, F, F, 8, d, 0, 0.2, None, 0, F, None) == 4
    assert fwd(F, 8, F, None, 8, d, 0, 0.2, None, 0, F, None) == 1  # bias required
    assert fwd(F, 8, F, None, 8, d, 1, 0.2, U, 1 << 20, F, None) == 4
    # data gradient: (dpre, Cout, W, Cin, d, Wd_scratch, din, stream)
    dg = L.reg_nn_conv3d_dgrad
    assert dg(F, 8, F, 8, dims(4, 0, 4), F, F, None) == 2
    assert dg(F, 12, F, 8, d, F, F, None) == 2
    assert dg(F, 8, F, 136, d, F, F, None) == 2
    assert dg(F, 8, F, 8, d, F, U, None) == 4
    # weight gradient: (in, Cin, dpre, Cout, d, scratch, bytes, dW, stream)
    wg = L.reg_nn_conv3d_wgrad
    assert wg(F, 8, F, 8, d, F, 1 << 20, F, None) == 2    # Cout < 16
    assert wg(F, 8, F, 80, d, F, 1 << 20, F, None) == 2   # Cout > 64
    assert wg(F, 8, F, 16, d, F, 1 << 20, U, None) == 4
    # network input: (F, M, img_dt, d, factor, f_lo, f_hi, m_lo, m_hi, out, stream)
    pp = L.reg_nn_pack_pair
    assert pp(F, F, capi.REG_F32, d, 3, 0.0, 1.0, 0.0, 1.0, F, None) == 2
    assert pp(F, F, capi.REG_F32, d, 0, 0.0, 1.0, 0.0, 1.0, F, None) == 2
    assert pp(F, F, 7, d, 2, 0.0, 1.0, 0.0, 1.0, F, None) == 3
    assert pp(F, F, capi.REG_F32, d, 2, 1.0, 1.0, 0.0, 1.0, F, None) == 1
    assert pp(F, F, capi.REG_F32, d, 2, 0.0, 1.0, 0.0, float("nan"), F, None) == 1
    assert pp(F, F, capi.REG_BF16, d, 2, 0.0, 1.0, 0.0, 1.0, U, None) == 4
    # element-wise and layout operators
    assert L.reg_nn_leaky_bwd(F, F, -1, 0.2, F, None) == 1
    assert L.reg_nn_leaky_bwd(None, F, 16, 0.2, F, None) == 1
    assert L.reg_nn_bias_grad(F, 0, 8, F, F, None) == 1
    assert L.reg_nn_bias_grad(F, 64, 65, F, F, None) == 1
    assert L.reg_nn_bias_grad(F, 64, 8, None, F, None) == 1
    assert L.reg_nn_avgpool2(F, 8, dims(7, 8, 8), F, 0, None) == 2
    assert L.reg_nn_avgpool2(F, 0, d, F, 0, None) == 2
    assert L.reg_nn_avgpool2(None, 8, d, F, 1, None) == 1
    assert L.reg_nn_upsample2(F, 8, dims(0, 4, 4), F, 0, None) == 2
    assert L.reg_nn_upsample2(F, 8, d, None, 1, None) == 1
    assert L.reg_nn_put_channels(F, 8, 64, F, 16, 9, 0, None) == 1   # c0 + Csrc > Cdst
    assert L.reg_nn_put_channels(F, 8, -1, F, 16, 0, 0, None) == 1
    assert L.reg_nn_put_channels(F, 8, 64, F, 16, -1, 0, None) == 1
    assert L.reg_nn_take_channels(F, 16, 9, 64, F, 8, 0, None) == 1  # c0 + Cdst > Csrc
    assert L.reg_nn_mse(F, F, 64, 2, F, F, F, None) == 1             # Cpad < 3
    assert L.reg_nn_mse(F, F, 0, 4, F, F, F, None) == 1
    assert L.reg_nn_mse(F, F, 64, 4, F, F, None, None) == 1
    assert L.reg_nn_field_down2(F, dims(8, 8, 7), F, None) == 2
    assert L.reg_nn_field_down2(None, d, F, None) == 1
    assert L.reg_nn_field_upsample(F, d, 0, F, None) == 2
    assert L.reg_nn_field_upsample(F, d, 2, None, None) == 1
    adam = capi.adam_desc(1e-3, 0.9, 0.999, 1e-8, capi.REG_F32, 1.0)
    assert L.reg_nn_adam(F, F, F, F, 16, ctypes.byref(adam), 0, None, None) == 1
    assert L.reg_nn_adam(F, F, F, F, 0, ctypes.byref(adam), 1, None, None) == 1
    assert L.reg_nn_adam(F, F, F, F, 16, None, 1, None, None) == 1


def test_auxiliary_entry_points_validation(capi):
    """Smoothing, downsampling, det J, the allocation-free MI call, the GEMM
    test hook and the timing-event switch: documented codes, no launch."""
    L = _lib(capi)
    vp = ctypes.c_void_p
    F, F2, U = vp(FAKE), vp(FAKE + 0x100), vp(FAKE + 8)
    d = dims()
    # reg_downsample2(in, dt, d, out, stream)
    assert L.reg_downsample2(F, capi.REG_F32, dims(7, 8, 8), F2, None) == 2
    assert L.reg_downsample2(F, 7, d, F2, None) == 3
    assert L.reg_downsample2(F, capi.REG_BF16, d, F, None) == 1   # in place
    assert L.reg_downsample2(None, capi.REG_F32, d, F2, None) == 1
    assert L.reg_downsample2(F, capi.REG_F32, d, U, None) == 4
    # reg_smooth_field(u, d, sigma, tmp, out, stream)
    assert L.reg_smooth_field(F, d, 0.0, F2, vp(FAKE + 0x200), None) == 1
    assert L.reg_smooth_field(F, d, 8.0, F2, vp(FAKE + 0x200), None) == 1
    assert L.reg_smooth_field(F, d, float("nan"), F2, vp(FAKE + 0x200), None) == 1
    assert L.reg_smooth_field(F, d, 1.0, F, vp(FAKE + 0x200), None) == 1   # u aliases tmp
    assert L.reg_smooth_field(F, d, 1.0, None, vp(FAKE + 0x200), None) == 1
    # reg_jacdet_min(u, d, ws, ws_bytes, min_out, nfold_out, stream)
    assert L.reg_jacdet_min(F, dims(0, 4, 4), None, 0, F2, F2, None) == 2
    assert L.reg_jacdet_min(U, d, None, 0, F2, F2, None) == 4
    assert L.reg_jacdet_min(F, d, None, 0, F2, None, None) == 1
    # reg_debug_gemm_bf16(A, B, C, M, N, K, a_mn_major, b_mn_major, stream)
    g = L.reg_debug_gemm_bf16
    assert g(F, F, F, 100, 64, 64, 0, 0, None) == 2   # M % 128
    assert g(F, F, F, 128, 8, 64, 0, 0, None) == 2    # N < 16
    assert g(F, F, F, 128, 144, 64, 0, 0, None) == 2  # N > 128
    assert g(F, F, F, 128, 64, 32, 0, 0, None) == 2   # K % 64
    assert g(F, F, F, 128, 64, 64, 2, 0, None) == 1
    # reg_mi_loss_grad_noalloc(loss, F, M, img_dt, u, d, pad, sim_out, grad_u, stream)
    na = L.reg_mi_loss_grad_noalloc
    mi = capi.mi_desc((0, 1), (0, 1), 32)
    assert na(None, F, F, capi.REG_F32, F, d, 0, F, None, None) == 1
    assert na(ctypes.byref(capi.lncc_desc(7)), F, F, capi.REG_F32, F, d, 0, F, None, None) == 9
    assert na(ctypes.byref(capi.mi_desc((0, 1), (0, 1), 4)), F, F, capi.REG_F32, F, d, 0, F, None, None) == 2
    assert na(ctypes.byref(capi.mi_desc((0, 1), (0, 1), 65)), F, F, capi.REG_F32, F, d, 0, F, None, None) == 2
    assert na(ctypes.byref(capi.mi_desc((1, 1), (0, 1), 32)), F, F, capi.REG_F32, F, d, 0, F, None, None) == 1
    assert na(ctypes.byref(mi), F, F, 7, F, d, 0, F, None, None) == 3
    assert na(ctypes.byref(mi), F, F, capi.REG_F32, F, d, 5, F, None, None) == 1
    assert na(ctypes.byref(mi), F, F, capi.REG_F32, F, dims(0, 4, 4), 0, F, None, None) == 2
    assert na(ctypes.byref(mi), None, F, capi.REG_F32, F, d, 0, F, None, None) == 1
    assert na(ctypes.byref(mi), F, F, capi.REG_F32, F, d, 0, F, U, None) == 4
    # reg_set_timing_events(events, n): a positive multiple of three events
    # (three per reg_run iteration) or (NULL, 0) to disarm
    assert L.reg_set_timing_events(None, 0) == 0
    assert L.reg_set_timing_events(None, 3) == 1
    two = (ctypes.c_void_p * 2)(FAKE, FAKE)
    assert L.reg_set_timing_events(two, 2) == 1
    four = (ctypes.c_void_p * 4)(FAKE, FAKE, FAKE, FAKE)
    assert L.reg_set_timing_events(four, 4) == 1
    six = (ctypes.c_void_p * 6)(*([FAKE] * 6))
    assert L.reg_set_timing_events(six, 6) == 0  # armed (no call records them) ...
    assert L.reg_set_timing_events(None, 0) == 0  # ... and cleared


def _c_params(txt):
    """name -> (return type, [parameter types]) of every REG_API prototype."""
    out = {}
    for ret, name, params in re.findall(r"REG_API\s+([^;{]*?)\b(reg_\w+)\s*\(([^)]*)\)\s*;", txt):
        params = " ".join(params.split())
        types = [] if params in ("", "void") else [re.sub(r"\s*\b\w+$", "", p.strip()) for p in params.split(",")]
        out[name] = (" ".join(ret.split()), types)
    return out


def _kind_of_c(t):
    t = t.replace("const", "").strip()
    if "*" in t:
        return "ptr"
    return {"int": "i4", "unsigned": "u4", "unsigned int": "u4", "long long": "i8", "unsigned long long": "u8",
            "size_t": "u8", "float": "f4", "double": "f8", "reg_status": "i4", "reg_dims": "reg_dims"}[" ".join(t.split())]


def _kind_of_ctypes(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    if t.__name__ == "RegDims":
        return "reg_dims"
    if t in (ctypes.c_float, ctypes.c_double):
        return f"f{ctypes.sizeof(t)}"
    signed = t(-1).value == -1
    return f"{'i' if signed else 'u'}{ctypes.sizeof(t)}"


def test_binding_argtypes_match_the_header(capi):
    """Every entry point's ctypes signature in the binding has the header's
    parameter count, and each parameter the same kind (pointer, struct by
    value, integer or float of the same width and signedness); functions that
    return size_t or a string declare it."""
    protos = _c_params(open(os.path.join(ROOT, "include", "reg.h")).read())
    assert set(protos) == set(header_symbols())
    capi.load()
    L = capi.nn()
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        argtypes = fn.argtypes or []
        assert len(argtypes) == len(params), (name, len(argtypes), len(params))
        for i, (a, p) in enumerate(zip(argtypes, params)):
            assert _kind_of_ctypes(a) == _kind_of_c(p), (name, i, a, p)
        if ret == "size_t":
            assert fn.restype is ctypes.c_size_t, name
        elif ret == "const char *":
            assert fn.restype is ctypes.c_char_p, name
        else:
            assert ret in ("reg_status", "int"), (name, ret)
            assert fn.restype in (ctypes.c_int, None) or fn.restype.__name__ == "c_int", name


def test_binding_refuses_host_tensors(capi):
    """A host tensor never reaches a kernel: the binding refuses it before the
    call (no host path, no silent copy)."""
    import torch
    M = torch.zeros(4, 4, 4)
    u = torch.zeros(3, 4, 4, 4)
    with pytest.raises(ValueError, match="device memory"):
        capi.reg_warp(M, u, J=torch.empty(4, 4, 4))
    with pytest.raises(ValueError, match="device memory"):
        capi.ptr(M)
    assert capi.ptr(None) is None


def test_binding_checks_caller_buffers_before_the_call(capi):
    """Caller-supplied outputs and state are checked for dtype, contiguity
    and room for what the library writes, before any pointer is taken (so a
    short buffer is an error, never an out-of-bounds write)."""
    import torch
    F = torch.zeros(4, 4, 4)
    u = torch.zeros(3, 4, 4, 4)
    lncc = capi.lncc_desc(3, 1e-5)
    ws = torch.empty(16)
    with pytest.raises(TypeError, match="sim"):
        capi.reg_loss(lncc, F, F, u, ws, sim=torch.empty(1, dtype=torch.float32))
    with pytest.raises(ValueError, match="grad"):
        capi.reg_loss_grad(lncc, F, F, u, ws, grad=torch.empty(3, 4, 4, 3))
    adam = capi.adam_desc(0.1)
    mb = torch.zeros(3, 4, 4, 4, dtype=torch.bfloat16)
    with pytest.raises(TypeError, match="m dtype"):
        capi.reg_iterate(lncc, F, F, u, u.clone(), mb, mb.clone(), 0.1, adam, 1, ws)
    with pytest.raises(ValueError, match="obj_hist"):
        capi.reg_run(lncc, F, F, u, u.clone(), u.clone(), u.clone(), 0.1, adam, 0, 5, ws,
                     obj_hist=torch.empty(4, 2, dtype=torch.float64))
    with pytest.raises(ValueError, match="saved"):
        capi.reg_exp_field(u, 4, saved=torch.empty(2, 3, 4, 4, 4))
    with pytest.raises(ValueError, match="contiguous"):
        capi.reg_compose_fields(u, u, out=torch.empty(4, 4, 4, 3).permute(3, 0, 1, 2))
    with pytest.raises(ValueError, match="A holds"):
        capi.reg_debug_gemm_bf16(torch.empty(64, 64, dtype=torch.bfloat16), torch.empty(16, 64, dtype=torch.bfloat16),
                                 128, 16, 64)
    with pytest.raises(ValueError, match="shape"):
        capi.reg_jacdet_min(torch.zeros(2, 4, 4, 4))
    # the fixed image sets the dims: an expanded (strided) F is refused before
    # its pointer is taken, in the workspace and the no-workspace entry points
    Fx = torch.zeros(1, 1, 1).expand(4, 4, 4)
    mi = capi.mi_desc((0.0, 1.0), (0.0, 1.0), 16)
    with pytest.raises(ValueError, match="contiguous"):
        capi.reg_loss_grad(lncc, Fx, F, u, ws)
    with pytest.raises(ValueError, match="contiguous"):
        capi.reg_mi_loss_grad_noalloc(mi, Fx, F, u)
    with pytest.raises(ValueError, match="contiguous"):
        capi.reg_iterate(mi, Fx, F, u, u.clone(), u.clone(), u.clone(), 0.1, adam, 1, ws)


def test_binding_refuses_tensors_off_the_current_device(capi, monkeypatch):
    """A tensor on another GPU than the current one (where the library
    launches) is refused before its address is taken."""
    import torch

    class Fake:  # a contiguous CUDA tensor on device 1 (no GPU needed)
        device = torch.device("cuda", 1)

        def is_contiguous(self):
            return True

        def data_ptr(self):
            raise AssertionError("the address of a tensor on another device was taken")

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    with pytest.raises(ValueError, match="current device"):
        capi._ptr(Fake())
