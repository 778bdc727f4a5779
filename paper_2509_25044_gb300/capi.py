"""ctypes binding of the C ABI in include/reg.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks dtypes / shapes of torch tensors, passes
their device pointers, the current CUDA stream and the descriptor structs,
and turns a non-zero reg_status into a RegError.  All compute runs in
libreg_gb300.so; if that library is missing the import fails loudly (there is
no CPU or PyTorch fallback).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libreg_gb300.so")

REG_OK = 0
REG_F32, REG_BF16 = 0, 1
REG_PAD_BORDER, REG_PAD_ZEROS = 0, 1
REG_LOSS_LNCC, REG_LOSS_MI = 0, 1
STATUS = {0: "REG_OK", 1: "REG_ERR_INVALID_ARG", 2: "REG_ERR_SHAPE", 3: "REG_ERR_DTYPE", 4: "REG_ERR_ALIGN",
          5: "REG_ERR_WORKSPACE", 6: "REG_ERR_NONFINITE", 7: "REG_ERR_TIMEOUT", 8: "REG_ERR_CUDA",
          9: "REG_ERR_UNSUPPORTED"}

# every C entry point declared in include/reg.h
EXPORTS = ("reg_version", "reg_status_string", "reg_workspace_size", "reg_warp", "reg_loss", "reg_loss_grad",
           "reg_regularize", "reg_step", "reg_iterate", "reg_jacdet_min", "reg_get_device_error",
           "reg_debug_wait_flag", "reg_set_timing_events", "reg_mi_loss_grad_noalloc",
           "reg_debug_gemm_bf16", "reg_smooth_field", "reg_downsample2", "reg_run", "reg_warp_composite",
           "reg_warp_composite_backward", "reg_loss_grad_composite", "reg_compose_fields", "reg_exp_field",
           "reg_compose_fields_backward", "reg_exp_field_backward", "reg_loss_grad_composite_dev",
           "reg_affine_adam_step")


class RegError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_lib().reg_status_string(status).decode()})")


class RegDims(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class RegLossDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("window", ctypes.c_int), ("eps", ctypes.c_float), ("bins", ctypes.c_int),
                ("f_lo", ctypes.c_float), ("f_hi", ctypes.c_float), ("m_lo", ctypes.c_float),
                ("m_hi", ctypes.c_float), ("lncc_grad", ctypes.c_int), ("mi_estimator", ctypes.c_int)]


class RegAdamDesc(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("moment_dtype", ctypes.c_int), ("grad_scale", ctypes.c_float)]


class RegAffineAdamDesc(ctypes.Structure):
    """The affine stage's Adam step (reg_affine_adam_step)."""
    _fields_ = [("lr_A", ctypes.c_double), ("lr_t", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("final_lr", ctypes.c_double),
                ("iters", ctypes.c_int), ("scale", ctypes.c_double), ("centre", ctypes.c_double * 3),
                ("loss_kind", ctypes.c_int)]


class RegAffine(ctypes.Structure):
    """phi(p) = A p + t + diag(s) u(p); A row-major over (x, y, z)."""
    _fields_ = [("A", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("s", ctypes.c_float * 3)]


def affine_desc(A=None, t=(0.0, 0.0, 0.0), s=(1.0, 1.0, 1.0)) -> RegAffine:
    """Descriptor of the composite transform from a 3x3 A (row-major nested
    sequence, array or tensor; default identity), t and s."""
    import numpy as _np
    A = _np.eye(3) if A is None else _np.asarray(A.tolist() if hasattr(A, "tolist") else A, dtype=_np.float64)
    T = RegAffine()
    for i, v in enumerate(A.reshape(9)):
        T.A[i] = float(v)
    for i in range(3):
        T.t[i] = float(t[i])
        T.s[i] = float(s[i])
    return T


_L = None
_vp = ctypes.c_void_p
_st = ctypes.c_int


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2509_25044_gb300.build.build() "
                              "(nvcc, sm_103a); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        L.reg_version.restype = ctypes.c_int
        L.reg_status_string.argtypes = [_st]
        L.reg_status_string.restype = ctypes.c_char_p
        L.reg_workspace_size.argtypes = [ctypes.POINTER(RegLossDesc), RegDims, ctypes.POINTER(ctypes.c_size_t)]
        L.reg_warp.argtypes = [_vp, ctypes.c_int, _vp, RegDims, ctypes.c_int, _vp, _vp, _vp]
        L.reg_loss.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp, RegDims, ctypes.c_int, _vp,
                               ctypes.c_size_t, _vp, _vp]
        L.reg_loss_grad.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp, RegDims, ctypes.c_int,
                                    _vp, ctypes.c_size_t, _vp, _vp, _vp]
        L.reg_regularize.argtypes = [_vp, RegDims, ctypes.c_float, _vp, ctypes.c_size_t, _vp, _vp, _vp]
        L.reg_step.argtypes = [_vp, _vp, _vp, _vp, _vp, RegDims, ctypes.POINTER(RegAdamDesc), ctypes.c_int, _vp]
        L.reg_iterate.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, RegDims,
                                  ctypes.c_int, ctypes.c_float, ctypes.POINTER(RegAdamDesc), ctypes.c_int, _vp,
                                  ctypes.c_size_t, _vp, _vp, _vp]
        L.reg_jacdet_min.argtypes = [_vp, RegDims, _vp, ctypes.c_size_t, _vp, _vp, _vp]
        L.reg_get_device_error.argtypes = [_vp]
        L.reg_debug_wait_flag.argtypes = [_vp, ctypes.c_uint, ctypes.c_ulonglong, _vp]
        L.reg_set_timing_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
        L.reg_debug_gemm_bf16.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _vp]
        L.reg_mi_loss_grad_noalloc.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp, RegDims,
                                               ctypes.c_int, _vp, _vp, _vp]
        L.reg_smooth_field.argtypes = [_vp, RegDims, ctypes.c_float, _vp, _vp, _vp]
        L.reg_downsample2.argtypes = [_vp, ctypes.c_int, RegDims, _vp, _vp]
        _aff = ctypes.POINTER(RegAffine)
        L.reg_warp_composite.argtypes = [_vp, ctypes.c_int, _vp, RegDims, _aff, ctypes.c_int, _vp, _vp, _vp]
        L.reg_warp_composite_backward.argtypes = [_vp, ctypes.c_int, _vp, RegDims, _aff, ctypes.c_int, _vp, _vp, _vp,
                                                  _vp, ctypes.c_size_t, _vp]
        L.reg_loss_grad_composite.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp, RegDims,
                                              _aff, ctypes.c_int, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp]
        L.reg_loss_grad_composite_dev.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp,
                                                  RegDims, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp, _vp, _vp,
                                                  _vp]
        L.reg_affine_adam_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(RegAffineAdamDesc), ctypes.c_int, _vp,
                                           _vp]
        L.reg_compose_fields.argtypes = [_vp, _vp, RegDims, ctypes.c_int, _vp, _vp]
        L.reg_exp_field.argtypes = [_vp, RegDims, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.reg_compose_fields_backward.argtypes = [_vp, _vp, _vp, RegDims, ctypes.c_int, _vp, _vp, _vp]
        L.reg_exp_field_backward.argtypes = [_vp, RegDims, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
        L.reg_run.argtypes = [ctypes.POINTER(RegLossDesc), _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, RegDims,
                              ctypes.c_int, ctypes.c_float, ctypes.POINTER(RegAdamDesc), ctypes.c_int, ctypes.c_int,
                              _vp, ctypes.c_size_t, _vp, ctypes.POINTER(RegAffine), _vp]
        for name in EXPORTS:
            if name not in ("reg_version", "reg_status_string"):
                getattr(L, name).restype = _st
        _L = L
    return _L


def load():
    """Load the library (raises ImportError if it has not been built)."""
    return _lib()


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _check(status: int, where: str):
    if status != REG_OK:
        raise RegError(status, where)


def _ptr(t):
    """Device address of a tensor, taken only after three checks:
    - it is contiguous: the library indexes every array densely from its
      dims, so an expanded or strided view would be read past its storage;
    - it is device memory: every entry point reads and writes device memory
      only, and there is no host path;
    - it lives on the current CUDA device, where the library launches its
      kernels (select another GPU with torch.cuda.device / set_device)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("a non-contiguous tensor was passed: every array must be dense and contiguous")
    if t.device.type != "cuda":
        raise ValueError(f"a {t.device.type} tensor was passed where device memory is required "
                         "(the library runs on the GPU only)")
    cur = torch.cuda.current_device()
    if t.device.index is not None and t.device.index != cur:
        raise ValueError(f"a tensor on {t.device} was passed while cuda:{cur} is the current device "
                         "(the library launches on the current device)")
    return ctypes.c_void_p(t.data_ptr())


def _stream(t=None):
    if t is not None and t.device.type == "cuda":
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _img_dtype(t) -> int:
    if t.dtype == torch.float32:
        return REG_F32
    if t.dtype == torch.bfloat16:
        return REG_BF16
    raise TypeError(f"image dtype must be float32 or bfloat16, got {t.dtype}")


def dims_of(vol) -> RegDims:
    nz, ny, nx = vol.shape[-3:]
    return RegDims(int(nx), int(ny), int(nz))


def _need(t, shape, dtype, name):
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} shape {tuple(t.shape)} != {tuple(shape)}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} dtype {t.dtype} != {dtype}")


def _buf(t, numel: int, dtype, name):
    """A caller-supplied output buffer: contiguous, of the given dtype, with
    room for the `numel` elements the library writes."""
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} dtype {t.dtype} != {dtype}")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements; {numel} are written")


def _field(t, vol_shape, name):
    """A displacement-shaped FP32 field [3][nz][ny][nx] of the given volume."""
    _need(t, (3,) + tuple(vol_shape), torch.float32, name)


def _moments(m, v, vol_shape, adam):
    mt = torch.bfloat16 if adam.moment_dtype == REG_BF16 else torch.float32
    _need(m, (3,) + tuple(vol_shape), mt, "m")
    _need(v, (3,) + tuple(vol_shape), mt, "v")


REG_LNCC_GRAD_EXACT, REG_LNCC_GRAD_ANTS = 0, 1


def lncc_desc(window: int = 7, eps: float = 1e-5, ants: bool = False) -> RegLossDesc:
    """ants=True: the ANTs gradient approximation (no second box sum)."""
    return RegLossDesc(REG_LOSS_LNCC, int(window), float(eps), 0, 0.0, 1.0, 0.0, 1.0,
                       REG_LNCC_GRAD_ANTS if ants else REG_LNCC_GRAD_EXACT)


REG_MI_PARZEN, REG_MI_HARD = 0, 1


def mi_desc(f_range, m_range, bins: int = 32, hard: bool = False) -> RegLossDesc:
    """hard=True: the hard-binned approximate histogram estimator."""
    return RegLossDesc(REG_LOSS_MI, 0, 0.0, int(bins), float(f_range[0]), float(f_range[1]), float(m_range[0]),
                       float(m_range[1]), 0, REG_MI_HARD if hard else REG_MI_PARZEN)


def adam_desc(lr: float, beta1=0.9, beta2=0.999, eps=1e-8, moment_dtype=REG_F32, grad_scale=1.0) -> RegAdamDesc:
    return RegAdamDesc(float(lr), float(beta1), float(beta2), float(eps), int(moment_dtype), float(grad_scale))


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def reg_version() -> int:
    return _lib().reg_version()


def reg_status_string(status: int) -> str:
    return _lib().reg_status_string(int(status)).decode()


def reg_workspace_size(loss: RegLossDesc | None, dims: RegDims) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib().reg_workspace_size(ctypes.byref(loss) if loss is not None else None, dims, ctypes.byref(out)),
           "reg_workspace_size")
    return int(out.value)


def workspace(loss, vol) -> torch.Tensor:
    """Allocate (with torch) a workspace sized by reg_workspace_size."""
    n = reg_workspace_size(loss, dims_of(vol))
    return torch.empty(n, dtype=torch.uint8, device=vol.device)


def reg_warp(M, u, pad: int = REG_PAD_BORDER, J=None, dJ=None, with_slope: bool = False):
    d = dims_of(M)
    _need(u, (3,) + tuple(M.shape), torch.float32, "u")
    if J is None:
        J = torch.empty(M.shape, dtype=torch.float32, device=M.device)
    _buf(J, M.numel(), torch.float32, "J")
    if with_slope and dJ is None:
        dJ = torch.empty_like(u)
    if dJ is not None:
        _buf(dJ, u.numel(), torch.float32, "dJ")
    _check(_lib().reg_warp(_ptr(M), _img_dtype(M), _ptr(u), d, int(pad), _ptr(J), _ptr(dJ), _stream(M)), "reg_warp")
    return (J, dJ) if dJ is not None else J


def reg_warp_composite(M, T: RegAffine, u=None, pad: int = REG_PAD_BORDER, with_slope: bool = False):
    """J = M o (A p + t + S u) (u may be None) and optionally dJ/dphi."""
    d = dims_of(M)
    if u is not None:
        _need(u, (3,) + tuple(M.shape), torch.float32, "u")
    J = torch.empty(M.shape, dtype=torch.float32, device=M.device)
    dJ = torch.empty((3,) + tuple(M.shape), dtype=torch.float32, device=M.device) if with_slope else None
    _check(_lib().reg_warp_composite(_ptr(M), _img_dtype(M), _ptr(u), d, ctypes.byref(T), int(pad), _ptr(J), _ptr(dJ),
                                     _stream(M)), "reg_warp_composite")
    return (J, dJ) if with_slope else J


def reg_warp_composite_backward(M, T: RegAffine, g, u=None, pad: int = REG_PAD_BORDER, ws=None, need_u: bool = True):
    """(g_u or None, grad_affine double[12]) for the upstream gradient g = dL/dJ."""
    d = dims_of(M)
    _need(g, M.shape, torch.float32, "g")
    if u is not None:
        _need(u, (3,) + tuple(M.shape), torch.float32, "u")
    if ws is None:
        ws = workspace(None, M)
    g_u = torch.empty((3,) + tuple(M.shape), dtype=torch.float32, device=M.device) if need_u else None
    ga = torch.empty(12, dtype=torch.float64, device=M.device)
    _check(_lib().reg_warp_composite_backward(_ptr(M), _img_dtype(M), _ptr(u), d, ctypes.byref(T), int(pad), _ptr(g),
                                              _ptr(g_u), _ptr(ga), _ptr(ws), ws.numel(), _stream(M)),
           "reg_warp_composite_backward")
    return g_u, ga


def reg_loss_grad_composite(loss: RegLossDesc, F, M, T: RegAffine, u=None, ws=None, pad: int = REG_PAD_BORDER,
                            need_u: bool = True, need_affine: bool = True, sim=None, grad_u=None, grad_affine=None):
    """(sim double[1], dC/du or None, dC/dA|dC/dt double[12] or None) for the composite transform."""
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    if u is not None:
        _need(u, (3,) + tuple(F.shape), torch.float32, "u")
    if ws is None:
        ws = workspace(loss, F)
    if sim is None:
        sim = torch.empty(2, dtype=torch.float64, device=F.device)
    _buf(sim, 1, torch.float64, "sim")
    if need_u and grad_u is None:
        grad_u = torch.empty((3,) + tuple(F.shape), dtype=torch.float32, device=F.device)
    if need_u:
        _buf(grad_u, 3 * F.numel(), torch.float32, "grad_u")
    if need_affine and grad_affine is None:
        grad_affine = torch.empty(12, dtype=torch.float64, device=F.device)
    if need_affine:
        _buf(grad_affine, 12, torch.float64, "grad_affine")
    _check(_lib().reg_loss_grad_composite(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u), d,
                                          ctypes.byref(T), int(pad), _ptr(ws), ws.numel(), _ptr(sim),
                                          _ptr(grad_u if need_u else None), _ptr(grad_affine if need_affine else None),
                                          _stream(F)), "reg_loss_grad_composite")
    return sim, (grad_u if need_u else None), (grad_affine if need_affine else None)


def reg_loss_grad_composite_dev(loss: RegLossDesc, F, M, T_dev, u=None, ws=None, pad: int = REG_PAD_BORDER,
                                need_u: bool = True, need_affine: bool = True, sim=None, grad_u=None,
                                grad_affine=None):
    """As reg_loss_grad_composite with the transform in device memory (T_dev:
    float32[15], the reg_affine layout A, t, s)."""
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    _buf(T_dev, 15, torch.float32, "T_dev")
    if u is not None:
        _need(u, (3,) + tuple(F.shape), torch.float32, "u")
    if ws is None:
        ws = workspace(loss, F)
    if sim is None:
        sim = torch.empty(2, dtype=torch.float64, device=F.device)
    _buf(sim, 1, torch.float64, "sim")
    if need_u and grad_u is None:
        grad_u = torch.empty((3,) + tuple(F.shape), dtype=torch.float32, device=F.device)
    if need_u:
        _buf(grad_u, 3 * F.numel(), torch.float32, "grad_u")
    if need_affine and grad_affine is None:
        grad_affine = torch.empty(12, dtype=torch.float64, device=F.device)
    if need_affine:
        _buf(grad_affine, 12, torch.float64, "grad_affine")
    _check(_lib().reg_loss_grad_composite_dev(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u), d,
                                              _ptr(T_dev), int(pad), _ptr(ws), ws.numel(), _ptr(sim),
                                              _ptr(grad_u if need_u else None),
                                              _ptr(grad_affine if need_affine else None), _stream(F)),
           "reg_loss_grad_composite_dev")
    return sim, (grad_u if need_u else None), (grad_affine if need_affine else None)


def affine_adam_desc(lr_A, lr_t, iters, scale, centre, loss_kind, beta1=0.9, beta2=0.999, eps=1e-8,
                     final_lr=0.1) -> RegAffineAdamDesc:
    d = RegAffineAdamDesc(float(lr_A), float(lr_t), float(beta1), float(beta2), float(eps), float(final_lr),
                          int(iters), float(scale))
    for i in range(3):
        d.centre[i] = float(centre[i])
    d.loss_kind = int(loss_kind)
    return d


def reg_affine_adam_step(grad_affine, sim, state, T_dev, desc: RegAffineAdamDesc, k: int, obj=None):
    """One device Adam step of the affine stage (state float64[36], T_dev
    float32[15] updated in place; obj float64[1] or None receives the
    objective at the input transform)."""
    _buf(grad_affine, 12, torch.float64, "grad_affine")
    _buf(sim, 1, torch.float64, "sim")
    _buf(state, 36, torch.float64, "state")
    _buf(T_dev, 15, torch.float32, "T_dev")
    if obj is not None:
        _buf(obj, 1, torch.float64, "obj")
    _check(_lib().reg_affine_adam_step(_ptr(grad_affine), _ptr(sim), _ptr(state), _ptr(T_dev), ctypes.byref(desc),
                                       int(k), _ptr(obj), _stream(state)), "reg_affine_adam_step")


def reg_compose_fields(a, b, pad: int = REG_PAD_BORDER, out=None):
    """w = a + b o (id + a) for [3][nz][ny][nx] FP32 fields."""
    d = dims_of(a[0])
    _field(a, a.shape[1:], "a")
    _need(b, tuple(a.shape), torch.float32, "b")
    if out is None:
        out = torch.empty_like(a)
    _buf(out, a.numel(), torch.float32, "out")
    _check(_lib().reg_compose_fields(_ptr(a), _ptr(b), d, int(pad), _ptr(out), _stream(a)), "reg_compose_fields")
    return out


def reg_exp_field(v, steps: int, pad: int = REG_PAD_BORDER, out=None, tmp=None, saved=None):
    """Scaling and squaring of the velocity field v ([3][nz][ny][nx] FP32);
    saved (optional, [steps - 1][3][nz][ny][nx]) keeps u_1 .. u_{steps-1}."""
    d = dims_of(v[0])
    _field(v, v.shape[1:], "v")
    if out is None:
        out = torch.empty_like(v)
    _buf(out, v.numel(), torch.float32, "out")
    if tmp is None and saved is None:
        tmp = torch.empty_like(v)
    if tmp is not None:
        _buf(tmp, v.numel(), torch.float32, "tmp")
    if saved is not None:
        _buf(saved, max(int(steps) - 1, 0) * v.numel(), torch.float32, "saved")
    _check(_lib().reg_exp_field(_ptr(v), d, int(steps), int(pad), _ptr(tmp), _ptr(out), _ptr(saved), _stream(v)),
           "reg_exp_field")
    return out


def reg_compose_fields_backward(a, b, gw, pad: int = REG_PAD_BORDER, same: bool = False):
    """(ga, gb) for gw = dL/dw of w = a + b o (id + a); same=True (a is b):
    returns (None, the whole gradient)."""
    d = dims_of(a[0])
    _field(a, a.shape[1:], "a")
    _need(b, tuple(a.shape), torch.float32, "b")
    _need(gw, tuple(a.shape), torch.float32, "gw")
    ga = None if same else torch.empty_like(a)
    gb = torch.empty_like(b)
    _check(_lib().reg_compose_fields_backward(_ptr(a), _ptr(b), _ptr(gw), d, int(pad), _ptr(ga), _ptr(gb),
                                              _stream(a)), "reg_compose_fields_backward")
    return ga, gb


def reg_exp_field_backward(v, steps: int, gout, saved=None, pad: int = REG_PAD_BORDER, gv=None, tmp=None):
    """dL/dv of scaling and squaring for gout = dL/d exp(v)."""
    d = dims_of(v[0])
    _field(v, v.shape[1:], "v")
    _need(gout, tuple(v.shape), torch.float32, "gout")
    if saved is not None:
        _buf(saved, max(int(steps) - 1, 0) * v.numel(), torch.float32, "saved")
    if gv is None:
        gv = torch.empty_like(v)
    _buf(gv, v.numel(), torch.float32, "gv")
    if tmp is None:
        tmp = torch.empty_like(v)
    _buf(tmp, v.numel(), torch.float32, "tmp")
    _check(_lib().reg_exp_field_backward(_ptr(v), d, int(steps), int(pad), _ptr(saved), _ptr(gout), _ptr(tmp),
                                         _ptr(gv), _stream(v)), "reg_exp_field_backward")
    return gv


def reg_loss(loss: RegLossDesc, F, M, u, ws, pad: int = REG_PAD_BORDER, sim=None):
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    _need(u, (3,) + tuple(F.shape), torch.float32, "u")
    if sim is None:
        sim = torch.empty(1, dtype=torch.float64, device=F.device)
    _buf(sim, 1, torch.float64, "sim")
    _check(_lib().reg_loss(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u), d, int(pad), _ptr(ws),
                           ws.numel(), _ptr(sim), _stream(F)), "reg_loss")
    return sim


def reg_loss_grad(loss: RegLossDesc, F, M, u, ws, pad: int = REG_PAD_BORDER, sim=None, grad=None):
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    _need(u, (3,) + tuple(F.shape), torch.float32, "u")
    if sim is None:
        sim = torch.empty(1, dtype=torch.float64, device=F.device)
    _buf(sim, 1, torch.float64, "sim")
    if grad is None:
        grad = torch.empty_like(u)
    _buf(grad, u.numel(), torch.float32, "grad")
    _check(_lib().reg_loss_grad(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u), d, int(pad), _ptr(ws),
                                ws.numel(), _ptr(sim), _ptr(grad), _stream(F)), "reg_loss_grad")
    return sim, grad


def reg_regularize(u, lam: float, ws, r=None, grad=None):
    d = dims_of(u)
    _field(u, u.shape[1:], "u")
    if r is None:
        r = torch.empty(1, dtype=torch.float64, device=u.device)
    _buf(r, 1, torch.float64, "r")
    if grad is not None:
        _buf(grad, u.numel(), torch.float32, "grad")
    _check(_lib().reg_regularize(_ptr(u), d, float(lam), _ptr(ws), ws.numel(), _ptr(r), _ptr(grad), _stream(u)),
           "reg_regularize")
    return r


def reg_smooth_field(u, sigma: float, out=None, tmp=None):
    """Gaussian smoothing of a [3][nz][ny][nx] FP32 field (out != u)."""
    d = dims_of(u[0])
    _field(u, u.shape[1:], "u")
    if out is None:
        out = torch.empty_like(u)
    _buf(out, u.numel(), torch.float32, "out")
    if tmp is None:
        tmp = torch.empty_like(u)
    _buf(tmp, u.numel(), torch.float32, "tmp")
    _check(_lib().reg_smooth_field(_ptr(u), d, float(sigma), _ptr(tmp), _ptr(out), _stream(u)), "reg_smooth_field")
    return out


def reg_downsample2(img):
    """2x2x2 block mean of an even-sized FP32 / BF16 volume."""
    nz, ny, nx = img.shape
    out = torch.empty((nz // 2, ny // 2, nx // 2), dtype=img.dtype, device=img.device)
    _check(_lib().reg_downsample2(_ptr(img), _img_dtype(img), dims_of(img), _ptr(out), _stream(img)),
           "reg_downsample2")
    return out


def reg_step(u_in, u_out, m, v, grad, adam: RegAdamDesc, t: int):
    d = dims_of(u_in)
    vol = u_in.shape[1:]
    _field(u_in, vol, "u_in")
    _field(u_out, vol, "u_out")
    _field(grad, vol, "grad")
    _moments(m, v, vol, adam)
    _check(_lib().reg_step(_ptr(u_in), _ptr(u_out), _ptr(m), _ptr(v), _ptr(grad), d, ctypes.byref(adam), int(t),
                           _stream(u_in)), "reg_step")
    return u_out


def reg_iterate(loss: RegLossDesc, F, M, u_in, u_out, m, v, lam: float, adam: RegAdamDesc, t: int, ws,
                pad: int = REG_PAD_BORDER, obj=None, grad=None):
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    _need(u_in, (3,) + tuple(F.shape), torch.float32, "u_in")
    _need(u_out, (3,) + tuple(F.shape), torch.float32, "u_out")
    _moments(m, v, F.shape, adam)
    if obj is None:
        obj = torch.empty(2, dtype=torch.float64, device=F.device)
    _buf(obj, 2, torch.float64, "obj")
    if grad is not None:
        _buf(grad, 3 * F.numel(), torch.float32, "grad")
    _check(_lib().reg_iterate(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u_in), _ptr(u_out), _ptr(m),
                              _ptr(v), d, int(pad), float(lam), ctypes.byref(adam), int(t), _ptr(ws), ws.numel(),
                              _ptr(obj), _ptr(grad), _stream(F)), "reg_iterate")
    return obj


def reg_run(loss: RegLossDesc, F, M, u_a, u_b, m, v, lam: float, adam: RegAdamDesc, t0: int, iters: int, ws,
            pad: int = REG_PAD_BORDER, obj_hist=None, affine: RegAffine | None = None):
    """`iters` fused iterations t0+1..t0+iters in one native call; the last
    iterate ends in u_a (iters even) or u_b (odd).  Returns obj_hist
    [iters][2] = {similarity, R} per iteration."""
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    _need(u_a, (3,) + tuple(F.shape), torch.float32, "u_a")
    _need(u_b, (3,) + tuple(F.shape), torch.float32, "u_b")
    _moments(m, v, F.shape, adam)
    if obj_hist is None:
        obj_hist = torch.empty((max(iters, 1), 2), dtype=torch.float64, device=F.device)
    _buf(obj_hist, 2 * max(int(iters), 0), torch.float64, "obj_hist")
    _check(_lib().reg_run(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u_a), _ptr(u_b), _ptr(m), _ptr(v),
                          d, int(pad), float(lam), ctypes.byref(adam), int(t0), int(iters), _ptr(ws), ws.numel(),
                          _ptr(obj_hist), ctypes.byref(affine) if affine is not None else None, _stream(F)),
           "reg_run")
    return obj_hist


def reg_jacdet_min(u, out_min=None, out_nfold=None):
    d = dims_of(u)
    _field(u, u.shape[1:], "u")
    if out_min is None:
        out_min = torch.empty(4, dtype=torch.float32, device=u.device)
    _buf(out_min, 1, torch.float32, "out_min")
    if out_nfold is None:
        out_nfold = torch.empty(2, dtype=torch.int64, device=u.device)
    _buf(out_nfold, 1, torch.int64, "out_nfold")
    _check(_lib().reg_jacdet_min(_ptr(u), d, None, 0, _ptr(out_min), _ptr(out_nfold), _stream(u)), "reg_jacdet_min")
    return out_min[:1], out_nfold[:1]


def reg_get_device_error(stream_of=None) -> int:
    """Synchronises the stream and returns (and clears) the device error code."""
    return int(_lib().reg_get_device_error(_stream(stream_of)))


def reg_debug_wait_flag(flag, expect: int, timeout_ns: int):
    _check(_lib().reg_debug_wait_flag(_ptr(flag), int(expect), int(timeout_ns), _stream(flag)), "reg_debug_wait_flag")


def reg_set_timing_events(events):
    """Arm the timing hook with torch.cuda.Event objects (or None to clear):
    three for the next reg_iterate, or three per iteration (flat, iteration
    k's at 3k .. 3k + 2) for the next reg_run of that many iterations."""
    if events is None:
        _check(_lib().reg_set_timing_events(None, 0), "reg_set_timing_events")
        return
    events = list(events)
    for e in events:
        if not e.cuda_event:  # torch creates the CUDA event on its first record
            e.record()
    arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _check(_lib().reg_set_timing_events(arr, len(events)), "reg_set_timing_events")


def reg_mi_loss_grad_noalloc(loss: RegLossDesc, F, M, u, pad: int = REG_PAD_BORDER, sim=None, grad=None,
                             with_grad: bool = True):
    """MI similarity (+ gradient) through the entry point that needs no
    workspace.  For callers that cannot allocate device memory the outputs
    must be passed in (``sim``, ``grad``); allocating them here is only a
    convenience for tests."""
    d = dims_of(F)
    _need(M, F.shape, F.dtype, "M")
    _need(u, (3,) + tuple(F.shape), torch.float32, "u")
    if sim is None:
        sim = torch.empty(1, dtype=torch.float64, device=F.device)
    _buf(sim, 1, torch.float64, "sim")
    if with_grad and grad is None:
        grad = torch.empty_like(u)
    if with_grad:
        _buf(grad, u.numel(), torch.float32, "grad")
    _check(_lib().reg_mi_loss_grad_noalloc(ctypes.byref(loss), _ptr(F), _ptr(M), _img_dtype(F), _ptr(u), d,
                                           int(pad), _ptr(sim), _ptr(grad if with_grad else None), _stream(F)),
           "reg_mi_loss_grad_noalloc")
    return (sim, grad) if with_grad else sim


def reg_debug_gemm_bf16(A, B, M: int, N: int, K: int, a_mn_major: bool = False, b_mn_major: bool = False, C=None):
    """C = A B^T on the tensor cores (test hook); A, B bf16 in the stated layouts."""
    _buf(A, int(M) * int(K), torch.bfloat16, "A")
    _buf(B, int(N) * int(K), torch.bfloat16, "B")
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _buf(C, int(M) * int(N), torch.float32, "C")
    _check(_lib().reg_debug_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), int(M), int(N), int(K), int(bool(a_mn_major)),
                                      int(bool(b_mn_major)), _stream(A)), "reg_debug_gemm_bf16")
    return C


# ---------------------------------------------------------------------------
# learned-initialiser operators (reg_nn_*): argument marshalling only
# ---------------------------------------------------------------------------
_SZ = ctypes.c_size_t
_NN = {
    "reg_nn_conv_kpad": ([ctypes.c_int], _SZ),
    "reg_nn_conv_scratch_bytes": ([ctypes.c_int, ctypes.c_int], _SZ),
    "reg_nn_conv3d_fwd": ([_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, RegDims, ctypes.c_int, ctypes.c_float, _vp,
                           ctypes.c_size_t, _vp, _vp],
                          _st),
    "reg_nn_dgrad_scratch_bytes": ([ctypes.c_int, ctypes.c_int], _SZ),
    "reg_nn_conv3d_dgrad": ([_vp, ctypes.c_int, _vp, ctypes.c_int, RegDims, _vp, _vp, _vp], _st),
    "reg_nn_wgrad_scratch_bytes": ([RegDims, ctypes.c_int, ctypes.c_int], _SZ),
    "reg_nn_conv3d_wgrad": ([_vp, ctypes.c_int, _vp, ctypes.c_int, RegDims, _vp, _SZ, _vp, _vp], _st),
    "reg_nn_pack_pair": ([_vp, _vp, ctypes.c_int, RegDims, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, ctypes.c_float, _vp, _vp], _st),
    "reg_nn_leaky_bwd": ([_vp, _vp, ctypes.c_longlong, ctypes.c_float, _vp, _vp], _st),
    "reg_nn_bias_grad_scratch_bytes": ([ctypes.c_int], _SZ),
    "reg_nn_bias_grad": ([_vp, ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp], _st),
    "reg_nn_avgpool2": ([_vp, ctypes.c_int, RegDims, _vp, ctypes.c_int, _vp], _st),
    "reg_nn_upsample2": ([_vp, ctypes.c_int, RegDims, _vp, ctypes.c_int, _vp], _st),
    "reg_nn_put_channels": ([_vp, ctypes.c_int, ctypes.c_longlong, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
                            _st),
    "reg_nn_take_channels": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _vp, ctypes.c_int, ctypes.c_int,
                              _vp], _st),
    "reg_nn_mse_scratch_bytes": ([], _SZ),
    "reg_nn_mse": ([_vp, _vp, ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp, _vp], _st),
    "reg_nn_field_down2": ([_vp, RegDims, _vp, _vp], _st),
    "reg_nn_field_upsample": ([_vp, RegDims, ctypes.c_int, _vp, _vp], _st),
    "reg_nn_adam": ([_vp, _vp, _vp, _vp, ctypes.c_longlong, ctypes.POINTER(RegAdamDesc), ctypes.c_int, _vp, _vp],
                    _st),
}
EXPORTS = EXPORTS + tuple(_NN)
_nn_ready = False


def nn():
    """The library with the reg_nn_* signatures declared."""
    global _nn_ready
    L = _lib()
    if not _nn_ready:
        for name, (args, res) in _NN.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _nn_ready = True
    return L


def nn_check(status, where):
    _check(status, where)


def ptr(t):
    return _ptr(t)


def stream_of(t=None):
    return _stream(t)
