"""FP64 CPU oracle for the registration hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2509_25044_gb300``)
never imports, links or executes anything in here, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
z-planes with a fixed summation order).  This module loads it through ctypes
and composes the per-step functions into one registration iteration by the
chain rule, in the paper's order (Sec. 1 Eq. image-reg; Fig. 1b): warp ->
similarity -> its adjoint -> sampler adjoint -> regulariser -> Adam.

Conventions: volumes ``[nz, ny, nx]`` (x fastest), displacement ``u`` is
``[3, nz, ny, nx]`` with channels (x, y, z) in voxel units, phi(p) = p + u(p).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .build import build as _build_lib

PAD_BORDER = 0
PAD_ZEROS = 1
LOSS_LNCC = 0
LOSS_MI = 1

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build_lib()  # compiles oracle.c when the library is missing or older than it
        lib = ctypes.CDLL(path)
        lib.or_warp.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.or_warp.restype = None
        lib.or_warp_adjoint.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        lib.or_warp_adjoint.restype = None
        lib.or_lncc.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, _dp, _dp]
        lib.or_lncc.restype = ctypes.c_double
        lib.or_lncc_grad.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, _dp]
        lib.or_lncc_grad.restype = ctypes.c_double
        cf = ctypes.c_float
        lib.or_mi_hard.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_int, cf, cf, cf, cf, _dp]
        lib.or_mi_hard.restype = ctypes.c_double
        lib.or_mi_hard_grad.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_long, ctypes.c_int, cf, cf, cf, cf, _dp]
        lib.or_mi_hard_grad.restype = ctypes.c_double
        lib.or_downsample2.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        lib.or_downsample2.restype = None
        lib.or_gaussian_smooth.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, _dp]
        lib.or_gaussian_smooth.restype = None
        lib.or_lncc_grad_ants.argtypes = lib.or_lncc_grad.argtypes
        lib.or_lncc_grad_ants.restype = ctypes.c_double
        lib.or_lncc_grad_points.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.POINTER(ctypes.c_long), ctypes.c_int, _dp, _dp]
        lib.or_lncc_grad_points.restype = None
        lib.or_bspline3.argtypes = [ctypes.c_double]
        lib.or_bspline3.restype = ctypes.c_double
        lib.or_bspline3_deriv.argtypes = [ctypes.c_double]
        lib.or_bspline3_deriv.restype = ctypes.c_double
        lib.or_mi.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_int, _dp]
        lib.or_mi.restype = ctypes.c_double
        lib.or_mi_grad.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_int, _dp]
        lib.or_mi_grad.restype = ctypes.c_double
        lib.or_mi_of_pmf.argtypes = [_dp, ctypes.c_int]
        lib.or_mi_of_pmf.restype = ctypes.c_double
        lib.or_mi_adjoint_points.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_long, ctypes.c_int, _dp, _dp]
        lib.or_mi_adjoint_points.restype = None
        lib.or_diffusion.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        lib.or_diffusion.restype = ctypes.c_double
        lib.or_bf16_round.argtypes = [ctypes.c_double]
        lib.or_bf16_round.restype = ctypes.c_double
        lib.or_adam.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.or_adam.restype = None
        lib.or_jacdet.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        lib.or_jacdet.restype = None
        ci = ctypes.c_int
        lib.or_conv3d.argtypes = [_dp, ci, _dp, _dp, ci, ci, ci, ci, _dp]
        lib.or_conv3d.restype = None
        lib.or_conv3d_dgrad.argtypes = [_dp, ci, _dp, ci, ci, ci, ci, _dp]
        lib.or_conv3d_dgrad.restype = None
        lib.or_conv3d_wgrad.argtypes = [_dp, ci, _dp, ci, ci, ci, ci, _dp]
        lib.or_conv3d_wgrad.restype = None
        cl, cd = ctypes.c_long, ctypes.c_double
        lib.or_leaky.argtypes = [_dp, cl, cd, _dp]
        lib.or_leaky_bwd.argtypes = [_dp, _dp, cl, cd, _dp]
        lib.or_avgpool2.argtypes = [_dp, ci, ci, ci, ci, _dp]
        lib.or_avgpool2_adjoint.argtypes = [_dp, ci, ci, ci, ci, _dp]
        lib.or_upsample.argtypes = [_dp, ci, ci, ci, ci, ci, _dp]
        lib.or_upsample_adjoint.argtypes = [_dp, ci, ci, ci, ci, ci, _dp]
        lib.or_concat.argtypes = [_dp, ci, _dp, ci, cl, _dp]
        lib.or_field_down2.argtypes = [_dp, ci, ci, ci, _dp]
        lib.or_field_upsample.argtypes = [_dp, ci, ci, ci, ci, _dp]
        lib.or_pack_pair.argtypes = [_dp, _dp, ci, ci, ci, ci, cd, cd, cd, cd, _dp]
        lib.or_mse.argtypes = [_dp, _dp, cl, _dp]
        lib.or_mse.restype = cd
        for f in ("or_leaky", "or_leaky_bwd", "or_avgpool2", "or_avgpool2_adjoint", "or_upsample",
                  "or_upsample_adjoint", "or_concat", "or_field_down2", "or_field_upsample", "or_pack_pair"):
            getattr(lib, f).restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _dims(vol: np.ndarray):
    nz, ny, nx = vol.shape
    return nx, ny, nz


# --------------------------------------------------------------------------
# per-step functions
# --------------------------------------------------------------------------
def warp(M, u, pad: int = PAD_BORDER, with_grad: bool = False):
    """J = M o (id+u) (trilinear) and optionally dJ/dphi [3, nz, ny, nx]."""
    M = _f64(M)
    u = _f64(u)
    assert u.shape == (3,) + M.shape
    nx, ny, nz = _dims(M)
    J = np.empty_like(M)
    dJ = np.empty_like(u) if with_grad else None
    _load().or_warp(_ptr(M), _ptr(u), nx, ny, nz, int(pad), _ptr(J), _ptr(dJ))
    return (J, dJ) if with_grad else J


def lncc(F, J, win: int, eps: float, per_voxel: bool = False):
    """S = mean_i n_i (LNCC similarity); the loss is 1 - S."""
    F = _f64(F)
    J = _f64(J)
    nx, ny, nz = _dims(F)
    n = np.empty_like(F) if per_voxel else None
    S = _load().or_lncc(_ptr(F), _ptr(J), nx, ny, nz, int(win), float(eps), _ptr(n), None)
    return (S, n) if per_voxel else S


def lncc_grad(F, J, win: int, eps: float):
    """(S, dL/dJ) for L = 1 - S."""
    F = _f64(F)
    J = _f64(J)
    nx, ny, nz = _dims(F)
    g = np.empty_like(F)
    S = _load().or_lncc_grad(_ptr(F), _ptr(J), nx, ny, nz, int(win), float(eps), _ptr(g))
    return S, g


def lncc_grad_ants(F, J, win: int, eps: float):
    """(S, approximate dL/dJ) with the convolution of the gamma family skipped
    (the ANTs gradient approximation, App. fused LNCC)."""
    F = _f64(F)
    J = _f64(J)
    nx, ny, nz = _dims(F)
    g = np.empty_like(F)
    S = _load().or_lncc_grad_ants(_ptr(F), _ptr(J), nx, ny, nz, int(win), float(eps), _ptr(g))
    return S, g


def lncc_grad_points(F, J, win: int, eps: float, points):
    """(dL/dJ, n) at the listed voxels (linear indices), for L = 1 - S of the
    whole volume; for volumes too large for lncc_grad."""
    F = _f64(F)
    J = _f64(J)
    nx, ny, nz = _dims(F)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int64))
    g = np.empty(pts.size, dtype=np.float64)
    n = np.empty(pts.size, dtype=np.float64)
    _load().or_lncc_grad_points(_ptr(F), _ptr(J), nx, ny, nz, int(win), float(eps),
                                pts.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), int(pts.size), _ptr(g), _ptr(n))
    return g, n


def bspline3(t: float) -> float:
    return _load().or_bspline3(float(t))


def bspline3_deriv(t: float) -> float:
    return _load().or_bspline3_deriv(float(t))


def mi(Fh, Jh, bins: int, with_hist: bool = False):
    """Parzen MI of intensities already mapped to [0,1]."""
    Fh = _f64(Fh).ravel()
    Jh = _f64(Jh).ravel()
    p = np.empty((bins, bins), dtype=np.float64) if with_hist else None
    v = _load().or_mi(_ptr(Fh), _ptr(Jh), Fh.size, int(bins), _ptr(p))
    return (v, p) if with_hist else v


def mi_grad(Fh, Jh, bins: int):
    """(MI, dL/dJh) for L = -MI."""
    shape = np.shape(Jh)
    Fh = _f64(Fh).ravel()
    Jh = _f64(Jh).ravel()
    g = np.empty_like(Jh)
    v = _load().or_mi_grad(_ptr(Fh), _ptr(Jh), Fh.size, int(bins), _ptr(g))
    return v, g.reshape(shape)


def _range32(rng):
    """(lo, scale) as the library forms them: float lo, hi; scale = float(1 / (hi - lo))."""
    lo, hi = float(np.float32(rng[0])), float(np.float32(rng[1]))
    return lo, float(np.float32(1.0 / (hi - lo)))


def mi_of_pmf(p, bins: int) -> float:
    """MI of a given joint PMF [bins, bins] (Eq. mi)."""
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(bins, bins))
    return float(_load().or_mi_of_pmf(_ptr(p), int(bins)))


def mi_adjoint_points(Fh, Jh, n_total: int, bins: int, p):
    """dL/dJh (L = -MI) at the given voxels of a volume of n_total voxels with
    joint PMF p (Eq. gradientmi-threadn): the per-voxel form of mi_grad for
    sampled checks of volumes the oracle cannot histogram itself."""
    Fh = np.ascontiguousarray(np.asarray(Fh, dtype=np.float64).ravel())
    Jh = np.ascontiguousarray(np.asarray(Jh, dtype=np.float64).ravel())
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(bins, bins))
    g = np.empty_like(Jh)
    _load().or_mi_adjoint_points(_ptr(Fh), _ptr(Jh), len(Jh), int(n_total), int(bins), _ptr(p), _ptr(g))
    return g


def mi_hard(F, J, bins: int, f_range, m_range, with_hist: bool = False):
    """Hard-binned (approximate) MI of raw intensities F, J (App. fused MI)."""
    F = _f64(F).ravel()
    J = _f64(J).ravel()
    p = np.empty((bins, bins), dtype=np.float64) if with_hist else None
    (fl, fs), (ml, ms) = _range32(f_range), _range32(m_range)
    v = _load().or_mi_hard(_ptr(F), _ptr(J), F.size, int(bins), fl, fs, ml, ms, _ptr(p))
    return (v, p) if with_hist else v


def mi_hard_grad(F, J, bins: int, f_range, m_range):
    """(approximate MI, dL/dJh) for L = -MI: the Parzen adjoint with the
    hard-binned PMF's table."""
    shape = np.shape(J)
    Fr = _f64(F).ravel()
    Jr = _f64(J).ravel()
    Fh, _ = normalize(Fr, *f_range)
    Jh, _ = normalize(Jr, *m_range)
    g = np.empty_like(Jr)
    (fl, fs), (ml, ms) = _range32(f_range), _range32(m_range)
    v = _load().or_mi_hard_grad(_ptr(Fr), _ptr(Jr), _ptr(Fh), _ptr(Jh), Fr.size, int(bins), fl, fs, ml, ms, _ptr(g))
    return v, g.reshape(shape)


def normalize(v, lo: float, hi: float):
    """Map intensities to [0,1]: vh = clamp((v-lo)/(hi-lo), 0, 1), and dvh/dv."""
    v = _f64(v)
    t = (v - lo) / (hi - lo)
    d = np.where((t >= 0.0) & (t <= 1.0), 1.0 / (hi - lo), 0.0)
    return np.clip(t, 0.0, 1.0), d


def downsample2(img):
    """2x2x2 block mean of an even-sized volume [nz][ny][nx]."""
    img = _f64(img)
    nx, ny, nz = _dims(img)
    out = np.empty((nz // 2, ny // 2, nx // 2))
    _load().or_downsample2(_ptr(img), nx, ny, nz, _ptr(out))
    return out


def gaussian_smooth(u, sigma: float):
    """Separable Gaussian (radius floor(4 sigma + 1/2), nearest borders) of
    every channel of u [C][nz][ny][nx] (or of one volume [nz][ny][nx])."""
    u = _f64(u)
    v = u[None] if u.ndim == 3 else u
    out = np.empty_like(v)
    nx, ny, nz = _dims(v[0])
    _load().or_gaussian_smooth(_ptr(np.ascontiguousarray(v)), nx, ny, nz, v.shape[0], float(sigma), _ptr(out))
    return out[0] if u.ndim == 3 else out


def diffusion(u, with_grad: bool = True):
    u = _f64(u)
    nx, ny, nz = _dims(u[0])
    g = np.empty_like(u) if with_grad else None
    R = _load().or_diffusion(_ptr(u), nx, ny, nz, _ptr(g))
    return (R, g) if with_grad else R


def bf16_round(a):
    a = _f64(a)
    f = _load().or_bf16_round
    return np.vectorize(f, otypes=[np.float64])(a) if a.size else a.copy()


def adam(u, m, v, g, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8, grad_scale: float = 1.0, bf16_moments: bool = False):
    """Returns (u', m', v') after one Adam step (inputs are not modified)."""
    u = _f64(u).copy()
    m = _f64(m).copy()
    v = _f64(v).copy()
    g = _f64(g)
    _load().or_adam(_ptr(u), _ptr(m), _ptr(v), _ptr(g), u.size, float(lr), float(beta1), float(beta2),
                    float(eps), float(grad_scale), int(t), int(bool(bf16_moments)))
    return u, m, v


def jacdet(u):
    u = _f64(u)
    nx, ny, nz = _dims(u[0])
    d = np.empty(u.shape[1:], dtype=np.float64)
    _load().or_jacdet(_ptr(u), nx, ny, nz, _ptr(d))
    return d


def conv3d(x, w, bias=None):
    """x: [nz, ny, nx, Cin] channels-last; w: [Cout, 27, Cin]; returns [nz, ny, nx, Cout]."""
    x = _f64(x)
    w = _f64(w)
    nz, ny, nx, cin = x.shape
    cout = w.shape[0]
    out = np.empty((nz, ny, nx, cout))
    b = _f64(bias) if bias is not None else None
    _load().or_conv3d(_ptr(x), cin, _ptr(w), _ptr(b), cout, nx, ny, nz, _ptr(out))
    return out


def conv3d_dgrad(dout, w):
    dout = _f64(dout)
    w = _f64(w)
    nz, ny, nx, cout = dout.shape
    cin = w.shape[2]
    din = np.empty((nz, ny, nx, cin))
    _load().or_conv3d_dgrad(_ptr(dout), cout, _ptr(w), cin, nx, ny, nz, _ptr(din))
    return din


def conv3d_wgrad(x, dout):
    x = _f64(x)
    dout = _f64(dout)
    nz, ny, nx, cin = x.shape
    cout = dout.shape[3]
    dw = np.empty((cout, 27, cin))
    _load().or_conv3d_wgrad(_ptr(x), cin, _ptr(dout), cout, nx, ny, nz, _ptr(dw))
    return dw


# --------------------------------------------------------------------------
# the learned initialiser's other operators (channels-last activations
# [nz, ny, nx, C]; displacement fields [3, nz, ny, nx])
# --------------------------------------------------------------------------
def leaky(x, slope: float = 0.2):
    x = _f64(x)
    y = np.empty_like(x)
    _load().or_leaky(_ptr(x), x.size, float(slope), _ptr(y))
    return y


def leaky_bwd(x, dy, slope: float = 0.2):
    """dL/dx of y = LeakyReLU(x) for the upstream gradient dy."""
    x, dy = _f64(x), _f64(dy)
    dx = np.empty_like(x)
    _load().or_leaky_bwd(_ptr(x), _ptr(dy), x.size, float(slope), _ptr(dx))
    return dx


def avgpool2(x):
    x = _f64(x)
    nz, ny, nx, c = x.shape
    out = np.empty((nz // 2, ny // 2, nx // 2, c))
    _load().or_avgpool2(_ptr(x), c, nx, ny, nz, _ptr(out))
    return out


def avgpool2_adjoint(g, fine_shape):
    g = _f64(g)
    nz, ny, nx = fine_shape
    c = g.shape[3]
    out = np.empty((nz, ny, nx, c))
    _load().or_avgpool2_adjoint(_ptr(g), c, nx, ny, nz, _ptr(out))
    return out


def upsample(x, s: int = 2):
    x = _f64(x)
    nz, ny, nx, c = x.shape
    out = np.empty((s * nz, s * ny, s * nx, c))
    _load().or_upsample(_ptr(x), c, nx, ny, nz, int(s), _ptr(out))
    return out


def upsample_adjoint(g, s: int = 2):
    g = _f64(g)
    nz, ny, nx, c = g.shape
    out = np.empty((nz // s, ny // s, nx // s, c))
    _load().or_upsample_adjoint(_ptr(g), c, nx // s, ny // s, nz // s, int(s), _ptr(out))
    return out


def concat(a, b):
    a, b = _f64(a), _f64(b)
    V = a.size // a.shape[-1]
    out = np.empty(a.shape[:-1] + (a.shape[-1] + b.shape[-1],))
    _load().or_concat(_ptr(a), a.shape[-1], _ptr(b), b.shape[-1], V, _ptr(out))
    return out


def field_down2(u):
    u = _f64(u)
    _, nz, ny, nx = u.shape
    out = np.empty((3, nz // 2, ny // 2, nx // 2))
    _load().or_field_down2(_ptr(u), nx, ny, nz, _ptr(out))
    return out


def field_upsample(u, s: int):
    u = _f64(u)
    _, nz, ny, nx = u.shape
    out = np.empty((3, s * nz, s * ny, s * nx))
    _load().or_field_upsample(_ptr(u), nx, ny, nz, int(s), _ptr(out))
    return out


def pack_pair(F, M, factor: int, f_range, m_range):
    """[nz/f, ny/f, nx/f, 2]: block means of F and M mapped by their ranges."""
    F, M = _f64(F), _f64(M)
    nz, ny, nx = F.shape
    out = np.empty((nz // factor, ny // factor, nx // factor, 2))
    _load().or_pack_pair(_ptr(F), _ptr(M), nx, ny, nz, int(factor), float(f_range[0]), float(f_range[1]),
                         float(m_range[0]), float(m_range[1]), _ptr(out))
    return out


def mse(pred, target):
    """(loss, dloss/dpred) for [3, V] (or [3, ...]) fields."""
    pred, target = _f64(pred), _f64(target)
    g = np.empty_like(pred)
    loss = _load().or_mse(_ptr(pred), _ptr(target), pred.size // 3, _ptr(g))
    return loss, g


# --------------------------------------------------------------------------
# composite affine + deformable transform (Sec. 2.1, the composite implicit
# grid sampler; Algorithm gridsampler): phi(p) = A p + t + S u(p), A a 3x3
# matrix acting on the voxel coordinates p = (x, y, z), t a translation in
# voxels, S = diag(s) the scale of the displacement.  The oracle writes phi as
# p + u_eff(p) and reuses the pinned deformable functions; the affine
# gradients follow by the chain rule.
# --------------------------------------------------------------------------
def identity_grid(shape):
    """[3, nz, ny, nx] FP64 voxel coordinates, channels (x, y, z)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return np.stack([x, y, z])


def composite_offset(shape, A, t, s=(1.0, 1.0, 1.0), u=None):
    """u_eff(p) = A p + t + S u(p) - p, so that phi(p) = p + u_eff(p)."""
    A = np.asarray(A, dtype=np.float64).reshape(3, 3)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    s = np.asarray(s, dtype=np.float64).reshape(3)
    X = identity_grid(shape)
    phi = np.einsum("ij,jzyx->izyx", A, X) + t[:, None, None, None]
    if u is not None:
        phi = phi + s[:, None, None, None] * _f64(u)
    return phi - X


def warp_composite(M, A, t, s=(1.0, 1.0, 1.0), u=None, pad: int = PAD_BORDER, with_grad: bool = False):
    """J(p) = M(A p + t + S u(p)) (Algorithm gridsampler, forward); with_grad
    adds dJ/dphi [3, nz, ny, nx]."""
    M = _f64(M)
    return warp(M, composite_offset(M.shape, A, t, s, u), pad, with_grad)


def _affine_grads(gX, s):
    """g_u = S gX, g_A = sum_p gX(p) p^T, g_t = sum_p gX(p) for the gradient gX
    with respect to the sampling location."""
    X = identity_grid(gX.shape[1:])
    s = np.asarray(s, dtype=np.float64).reshape(3)
    g_A = np.einsum("izyx,jzyx->ij", gX, X)
    g_t = gX.reshape(3, -1).sum(axis=1)
    return s[:, None, None, None] * gX, g_A, g_t


def sampler_backward_composite(M, A, t, s, u, g, pad: int = PAD_BORDER):
    """Algorithm gridsampler, backward, without the image gradient: for an
    upstream gradient g = dL/dJ returns (g_u, g_A, g_t)."""
    _, dJ = warp_composite(M, A, t, s, u, pad, with_grad=True)
    return _affine_grads(dJ * _f64(g)[None], s)


def similarity_and_grad_composite(F, M, A, t, s=(1.0, 1.0, 1.0), u=None, spec=None, pad: int = PAD_BORDER):
    """(similarity, dC/du, dC/dA, dC/dt) of C(F, M o phi) for the composite
    phi; C = 1 - S (LNCC) or -MI."""
    F = _f64(F)
    sim, gX = similarity_and_grad(F, M, composite_offset(F.shape, A, t, s, u), spec, pad)
    g_u, g_A, g_t = _affine_grads(gX, s)
    return sim, g_u, g_A, g_t


# --------------------------------------------------------------------------
# composition of displacement fields and scaling-and-squaring (the
# exponential of a stationary velocity field that the paper's grid sampler
# serves, Sec. 4 ablations): (id + w) = (id + b) o (id + a), i.e.
# w(p) = a(p) + b(p + a(p)), each channel of b sampled with the pinned
# trilinear warp.
# --------------------------------------------------------------------------
def compose_fields(a, b, pad: int = PAD_BORDER):
    """w = a + b o (id + a) for fields [3, nz, ny, nx]."""
    a = _f64(a)
    b = _f64(b)
    return a + np.stack([warp(b[c], a, pad) for c in range(3)])


def warp_adjoint(g, u, pad: int = PAD_BORDER):
    """gM = the transpose of M -> M o (id+u) applied to g (the scatter of the
    sampler backward): <warp(M, u), g> = <M, warp_adjoint(g, u)>."""
    g = _f64(g)
    u = _f64(u)
    nx, ny, nz = _dims(g)
    gM = np.empty_like(g)
    _load().or_warp_adjoint(_ptr(g), _ptr(u), nx, ny, nz, int(pad), _ptr(gM))
    return gM


def compose_fields_backward(a, b, gw, pad: int = PAD_BORDER, scale: float = 1.0):
    """Adjoint of w = s a + s b o (id + s a) (s = scale): returns (dL/da, dL/db)
    for gw = dL/dw.  dL/da = s gw + s^2 (grad b)^T gw at the sample points;
    dL/db = s times the scatter of gw."""
    a = _f64(a)
    b = _f64(b)
    gw = _f64(gw)
    sa = scale * a
    ga = scale * gw.copy()
    gb = np.empty_like(b)
    for d in range(3):
        _, dJ = warp(b[d], sa, pad, with_grad=True)
        ga += scale * scale * gw[d][None] * dJ
        gb[d] = scale * warp_adjoint(gw[d], sa, pad)
    return ga, gb


def exp_field(v, steps: int, pad: int = PAD_BORDER):
    """Scaling and squaring: u = v / 2^steps, then steps times u <- u + u o (id + u)."""
    u = _f64(v) / float(2 ** steps)
    for _ in range(steps):
        u = compose_fields(u, u, pad)
    return u


def exp_field_backward(v, steps: int, gout, pad: int = PAD_BORDER):
    """dL/dv for gout = dL/d exp(v): the forward steps are replayed, then each
    squaring u <- u + u o (id + u) is differentiated with respect to its one
    input (both adjoint terms), last step first; the 2^-steps of the first
    step scales the result."""
    v = _f64(v)
    if steps == 0:
        return _f64(gout).copy()
    us = [v / float(2 ** steps)]
    for _ in range(steps - 1):
        us.append(compose_fields(us[-1], us[-1], pad))
    g = _f64(gout)
    for u in reversed(us):
        ga, gb = compose_fields_backward(u, u, g, pad)
        g = ga + gb
    return g / float(2 ** steps)


# --------------------------------------------------------------------------
# one iteration, composed by the chain rule
# --------------------------------------------------------------------------
@dataclass
class LossSpec:
    kind: int = LOSS_LNCC
    window: int = 7
    eps: float = 1e-5
    lncc_grad: int = 0  # 0: exact adjoint, 1: ANTs approximation
    bins: int = 32
    f_range: tuple = (0.0, 1.0)
    m_range: tuple = (0.0, 1.0)
    mi_estimator: int = 0  # 0: Parzen, 1: hard-binned approximation


def similarity_and_grad(F, M, u, spec: LossSpec, pad: int = PAD_BORDER, need_grad: bool = True):
    """Returns (similarity, dC/du or None) with C = 1 - S (LNCC) or -MI (MI)."""
    J, dJ = warp(M, u, pad, with_grad=True)
    if spec.kind == LOSS_LNCC:
        if not need_grad:
            return lncc(F, J, spec.window, spec.eps), None
        S, gJ = (lncc_grad_ants if spec.lncc_grad == 1 else lncc_grad)(F, J, spec.window, spec.eps)
        return S, gJ[None] * dJ
    Fh, _ = normalize(F, *spec.f_range)
    Jh, dJh = normalize(J, *spec.m_range)
    if spec.mi_estimator == 1:
        if not need_grad:
            return mi_hard(F, J, spec.bins, spec.f_range, spec.m_range), None
        v, gJh = mi_hard_grad(F, J, spec.bins, spec.f_range, spec.m_range)
        return v, (gJh * dJh)[None] * dJ
    if not need_grad:
        return mi(Fh, Jh, spec.bins), None
    v, gJh = mi_grad(Fh, Jh, spec.bins)
    return v, (gJh * dJh)[None] * dJ


def objective(F, M, u, spec: LossSpec, lam: float, pad: int = PAD_BORDER):
    """Returns dict(sim, R, loss, total, grad) for C(F, M o (id+u)) + lam R(u)."""
    sim, g = similarity_and_grad(F, M, u, spec, pad)
    R, gR = diffusion(u)
    loss = 1.0 - sim if spec.kind == LOSS_LNCC else -sim
    return dict(sim=sim, R=R, loss=loss, total=loss + lam * R, grad=g + lam * gR)


def iterate(F, M, u, m, v, t: int, spec: LossSpec, lam: float, lr: float, beta1=0.9, beta2=0.999,
            eps=1e-8, grad_scale=None, bf16_moments=False, pad: int = PAD_BORDER):
    """One full iteration; grad_scale defaults to N (the Adam input is N * grad)."""
    obj = objective(F, M, u, spec, lam, pad)
    if grad_scale is None:
        grad_scale = float(np.prod(np.shape(F)))
    u2, m2, v2 = adam(u, m, v, obj["grad"], t, lr, beta1, beta2, eps, grad_scale, bf16_moments)
    obj.update(u=u2, m=m2, v=v2)
    return obj
