/*
 * reg.h -- C ABI of the GB300 (sm_103a) registration hot path.
 *
 * One iteration of  argmin_u  C(F, M o (id + u)) + lambda R(u)   (Sec. 1,
 * Eq. image-reg) on a dense 3-D displacement field u: trilinear warp of the
 * moving image (Sec. 2.1), windowed LNCC (Sec. 2.3, App. fused LNCC) or
 * Parzen mutual information (Sec. 2.2, App. fused MI), their hand-written
 * adjoints back to dC/du, a diffusion regulariser and an Adam step.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Volumes are dense [nz][ny][nx] arrays, x fastest, voxel spacing 1.
 *  - u (and every gradient) is FP32, structure of arrays [3][nz][ny][nx]:
 *    channel 0, 1, 2 = x, y, z displacement in voxel units;
 *    phi(p) = p + u(p) for integer voxel centres p.
 *  - Every pointer argument is a DEVICE pointer unless stated otherwise, and
 *    must be 16-byte aligned (REG_ERR_ALIGN otherwise).  Any nx, ny, nz >= 1
 *    is accepted (no padding or pitch requirement).
 *  - Ownership: the caller allocates and owns every buffer, including the
 *    workspace; the library allocates no memory on these paths and keeps no
 *    pointer after a call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls only enqueue work; outputs are valid once the stream
 *    has been synchronised.
 *  - Errors: arguments are validated on the host before anything is
 *    launched; a failing check returns its code and enqueues nothing.  A
 *    launch failure returns REG_ERR_CUDA.  Non-finite loss or regulariser
 *    partials found on the device are latched in a device error word, read
 *    (and cleared) by reg_get_device_error().  No kernel traps or asserts.
 *  - Determinism: identical inputs give bitwise-identical outputs
 *    (fixed-order FP64 reductions, integer MI histograms), except where an
 *    entry point's own comment says otherwise (the scatters of
 *    reg_compose_fields_backward and reg_exp_field_backward).
 *  - Device set-up: the library looks up the device address of its error
 *    word (and reg_mi_loss_grad_noalloc that of its scratch array) once per
 *    device, the first time it is used with that device current.  A process
 *    that calls cudaDeviceReset must not use the library on that device
 *    afterwards.
 */
#ifndef REG_H
#define REG_H

#include <stddef.h>

#if defined(__GNUC__)
#define REG_API __attribute__((visibility("default")))
#else
#define REG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum reg_status {
    REG_OK = 0,
    REG_ERR_INVALID_ARG = 1, /* null pointer, bad enum or out-of-range parameter */
    REG_ERR_SHAPE = 2,       /* dims < 1, too large, or window/bins unsupported */
    REG_ERR_DTYPE = 3,       /* unknown reg_dtype */
    REG_ERR_ALIGN = 4,       /* a pointer is not 16-byte aligned */
    REG_ERR_WORKSPACE = 5,   /* ws_bytes smaller than reg_workspace_size() */
    REG_ERR_NONFINITE = 6,   /* device error word: a non-finite partial sum was seen */
    REG_ERR_TIMEOUT = 7,     /* device error word: a bounded device wait expired */
    REG_ERR_CUDA = 8,        /* a CUDA runtime call or kernel launch failed */
    REG_ERR_UNSUPPORTED = 9  /* a valid request the library does not implement */
} reg_status;

typedef enum reg_dtype { REG_F32 = 0, REG_BF16 = 1 } reg_dtype;

/* Out-of-volume sampling.  BORDER: the sample point is clamped into the
 * volume per axis (the slope along a clamped axis is 0).  ZEROS: voxels
 * outside the volume read as 0 (Algorithm gridsampler). */
typedef enum reg_pad { REG_PAD_BORDER = 0, REG_PAD_ZEROS = 1 } reg_pad;

typedef struct reg_dims {
    int nx, ny, nz;
} reg_dims;

typedef enum reg_loss_kind { REG_LOSS_LNCC = 0, REG_LOSS_MI = 1 } reg_loss_kind;

/* Similarity description.
 *   LNCC (App. fused LNCC, Eq. lncc-loss): `window` odd in [3, 15]; a uniform
 *     box of that side centred at each voxel, truncated at the volume border
 *     and normalised by the in-volume count; eps >= 0 is added to B_i C_i.
 *     Similarity S = mean_i A_i^2 / (B_i C_i + eps); loss C = 1 - S.
 *   MI (Sec. 2.2, Eq. mi): `bins` in [8, 64]; cubic B-spline Parzen kernel.
 *     Intensities are mapped to [0,1] by (v - lo) / (hi - lo) and clamped;
 *     the kernel of bin m sits at s = m with s = v (bins - 3) + 1.
 *     Similarity = MI (natural log); loss C = -MI.
 *     Requires f_hi > f_lo and m_hi > m_lo (the fixed / moving ranges).
 *   lncc_grad (LNCC gradients only): REG_LNCC_GRAD_EXACT (0) is the exact
 *     adjoint (the coefficient fields box-summed a second time);
 *     REG_LNCC_GRAD_ANTS (1) is the ANTs approximation of App. fused LNCC,
 *     which skips that second convolution: dL/dJ_k = c_k (a_J + 2 J_k a_JJ +
 *     F_k a_FJ)_k with the coefficients of voxel k's own window (c_k its
 *     in-volume size).  The similarity value is the same in both modes.
 *   mi_estimator (MI only): REG_MI_PARZEN (0) is the Parzen estimate above;
 *     REG_MI_HARD (1) is the approximate histogram estimator of App. fused MI:
 *     each sample adds 1 to its nearest bin (m = floor(s + 1/2) of its bin
 *     coordinate s, taken in FP32), and the count histogram / N is convolved
 *     with kappa(a) kappa(b), a, b in {-1, 0, 1} (1/6, 2/3, 1/6) -- exact for
 *     samples on bin centres.  Its gradient is the Parzen adjoint evaluated
 *     with the approximate PMF's table. */
typedef enum reg_lncc_grad { REG_LNCC_GRAD_EXACT = 0, REG_LNCC_GRAD_ANTS = 1 } reg_lncc_grad;
typedef enum reg_mi_estimator { REG_MI_PARZEN = 0, REG_MI_HARD = 1 } reg_mi_estimator;
typedef struct reg_loss_desc {
    int kind;   /* reg_loss_kind */
    int window; /* LNCC */
    float eps;  /* LNCC */
    int bins;   /* MI */
    float f_lo, f_hi, m_lo, m_hi; /* MI intensity ranges */
    int lncc_grad;    /* reg_lncc_grad */
    int mi_estimator; /* reg_mi_estimator */
} reg_loss_desc;

/* Adam (the optimiser state m1, m2 of Sec. 3.1), torch.optim.Adam semantics
 * with bias correction.  The gradient fed to Adam is grad_scale * dL/du
 * (use grad_scale = N = nx ny nz: C and R are voxel means, so dL/du is
 * O(1/N) and eps would otherwise dominate).  moment_dtype: REG_F32 or
 * REG_BF16 (m, v stored in bfloat16, round-to-nearest-even, updated in FP32). */
typedef struct reg_adam_desc {
    float lr, beta1, beta2, eps;
    int moment_dtype; /* reg_dtype */
    float grad_scale;
} reg_adam_desc;

/* Gaussian smoothing of a field (the sigma_grad / sigma_warp smoothing
 * regularisation the paper runs its registrations with, FireANTs style:
 * the gradient is smoothed before the optimiser step, the warp after it).
 * u, tmp, out: SoA FP32 [3][nz][ny][nx] device buffers, 16-byte aligned,
 * pairwise distinct (tmp is scratch).  Each channel is convolved separably
 * along x, y, z with w_k = exp(-k^2 / (2 sigma^2)) / sum over |k| <=
 * floor(4 sigma + 1/2), borders repeating the edge voxel.
 * 0 < sigma <= 7.9, else REG_ERR_INVALID_ARG. */
REG_API reg_status reg_smooth_field(const float *u, reg_dims d, float sigma, float *tmp, float *out, void *stream);

/* 2x downsampling of an image for the coarse levels of a multi-scale
 * registration (the coarse-to-fine schedules the paper runs with):
 * out[z][y][x] = mean of the 2x2x2 block of `in` at (2x, 2y, 2z), FP32 sums,
 * stored in the image dtype.  nx, ny, nz even (else REG_ERR_SHAPE); out has
 * (nx/2, ny/2, nz/2) voxels and may not alias in. */
REG_API reg_status reg_downsample2(const void *in, int dt, reg_dims d, void *out, void *stream);

/* Library version (major * 10000 + minor * 100 + patch). */
REG_API int reg_version(void);

/* Static description of a status code; never NULL. */
REG_API const char *reg_status_string(reg_status s);

/* Bytes of device workspace that reg_loss, reg_loss_grad, reg_regularize,
 * reg_iterate, reg_run and reg_jacdet_min need for these dims (loss may be
 * NULL for the regulariser / det J alone; LNCC adds 24 bytes per voxel: the
 * warped image, three adjoint coefficient fields and F's window mean and
 * variance).  *bytes is a HOST pointer. */
REG_API reg_status reg_workspace_size(const reg_loss_desc *loss, reg_dims d, size_t *bytes);

/* J = M o (id + u): trilinear warp of M (img_dt) by u (Sec. 2.1, the
 * deformable part of fused_grid_sampler with A = I, t = 0, S = I;
 * Algorithm gridsampler, forward).  J_out: FP32 N (overwritten).
 * dJ_out: optional (may be NULL) FP32 [3][N] receiving dJ/dphi per axis. */
REG_API reg_status reg_warp(const void *M, int img_dt, const float *u, reg_dims d, int pad, float *J_out,
                    float *dJ_out, void *stream);

/* Similarity of F and M o (id+u) (LNCC or MI per `loss`).  sim_out: device
 * double[1], receives S (LNCC) or MI.  F and M share img_dt.  The warped
 * image is recomputed on chip and never stored. */
REG_API reg_status reg_loss(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u,
                    reg_dims d, int pad, void *ws, size_t ws_bytes, double *sim_out, void *stream);

/* As reg_loss, and grad_u (FP32 [3][N], overwritten) = dC/du of the loss
 * C = 1 - S (LNCC) or -MI (MI): the similarity adjoint (LNCC: App. fused
 * LNCC, Eq. gradientcc-first and its moving-image counterpart; MI: Eq.
 * gradientmi-threadn) chained through the sampler slope (Algorithm
 * gridsampler, backward: g_u = dv/dX g). */
REG_API reg_status reg_loss_grad(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u,
                         reg_dims d, int pad, void *ws, size_t ws_bytes, double *sim_out, float *grad_u,
                         void *stream);

/* Diffusion regulariser R(u) = (1/N) sum_c sum_d sum_{p, p+e_d inside}
 * (u_c(p+e_d) - u_c(p))^2 (first-order Sobolev norm, listed among common
 * choices of R in Sec. 1).  r_out: device double[1] receives R(u) (without
 * lambda).  grad_u: FP32 [3][N], lambda * dR/du is ADDED to it (may be NULL). */
REG_API reg_status reg_regularize(const float *u, reg_dims d, float lambda, void *ws, size_t ws_bytes, double *r_out,
                          float *grad_u, void *stream);

/* One Adam step on u (t >= 1 is the 1-based step count):
 * u_out = u_in - lr * mhat / (sqrt(vhat) + eps).  u_out may equal u_in.
 * m, v: [3][N] in adam->moment_dtype, updated in place. */
REG_API reg_status reg_step(const float *u_in, float *u_out, void *m, void *v, const float *grad_u, reg_dims d,
                    const reg_adam_desc *adam, int t, void *stream);

/* One fused iteration: similarity + its gradient + lambda * diffusion
 * gradient + Adam, in two sweeps over the volume (LNCC: window statistics,
 * then adjoint + step; MI: joint histogram, then adjoint + step).
 * u_out must not alias u_in (the stencils read neighbours of u_in).
 * obj_out: device double[2] = {similarity, R(u_in)} at u_in.
 * grad_out: optional FP32 [3][N] receiving the total gradient dL/du fed to
 * Adam (before grad_scale); NULL skips the store. */
REG_API reg_status reg_iterate(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u_in,
                       float *u_out, void *m, void *v, reg_dims d, int pad, float lambda,
                       const reg_adam_desc *adam, int t, void *ws, size_t ws_bytes, double *obj_out,
                       float *grad_out, void *stream);

/* ------------------------------------------------------------------------
 * Composite transform (Sec. 2.1, the composite implicit grid sampler;
 * Algorithm gridsampler):
 *     phi(p) = A p + t + S u(p),   p = (x, y, z) voxel coordinates,
 * A row-major (A[3*i + j] takes coordinate j into output axis i), t in
 * voxels, S = diag(s).  A = I, t = 0, s = 1 is the deformable sampler of
 * reg_warp; a map about the volume centre c is A with t = c - A c.  No
 * coordinate grid is materialised: the kernels form phi per voxel.  Every
 * entry of A, t and s must be finite (else REG_ERR_INVALID_ARG); u may be
 * NULL (u = 0, the affine part alone).
 * ------------------------------------------------------------------------ */
typedef struct reg_affine {
    float A[9];
    float t[3];
    float s[3];
} reg_affine;

/* J = M o phi (FP32 [N]) and optionally dJ/dphi (FP32 [3][N], NULL skips it;
 * Algorithm gridsampler, forward). */
REG_API reg_status reg_warp_composite(const void *M, int img_dt, const float *u, reg_dims d, const reg_affine *T,
                                      int pad, float *J, float *dJ, void *stream);

/* Backward of the composite sampler (Algorithm gridsampler, backward; the
 * gradient with respect to the moving image is not formed): for the upstream
 * gradient g = dL/dJ (FP32 [N]),
 *   g_u = S (dJ/dphi) g            (FP32 [3][N], overwritten; NULL skips it),
 *   grad_affine[0..8]  = dL/dA = sum_p (dJ/dphi g)(p) p^T   (row-major),
 *   grad_affine[9..11] = dL/dt = sum_p (dJ/dphi g)(p)
 * (device double[12], NULL skips it), summed in a fixed order.
 * ws: at least reg_workspace_size(NULL, d) bytes. */
REG_API reg_status reg_warp_composite_backward(const void *M, int img_dt, const float *u, reg_dims d,
                                               const reg_affine *T, int pad, const float *g, float *g_u,
                                               double *grad_affine, void *ws, size_t ws_bytes, void *stream);

/* Similarity of C(F, M o phi) for the composite phi (sim_out as reg_loss)
 * and its gradients: grad_u = dC/du = S dC/dphi (FP32 [3][N], overwritten;
 * NULL skips it) and grad_affine = dC/dA (row-major) then dC/dt (device
 * double[12]; NULL skips it), with C = 1 - S (LNCC) or -MI.  Both NULL
 * computes the similarity alone.  Workspace as reg_loss. */
REG_API reg_status reg_loss_grad_composite(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                                           const float *u, reg_dims d, const reg_affine *T, int pad, void *ws,
                                           size_t ws_bytes, double *sim_out, float *grad_u, double *grad_affine,
                                           void *stream);

/* As reg_loss_grad_composite, with the transform read from DEVICE memory:
 * T_dev holds 15 floats in the layout of reg_affine (A row-major, t, s),
 * for instance written by reg_affine_adam_step, so that an optimiser running
 * on the device can feed the next evaluation without a round trip through
 * the host.  The kernels read T_dev; its entries are not checked on the host
 * and must be finite. */
REG_API reg_status reg_loss_grad_composite_dev(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                                               const float *u, reg_dims d, const float *T_dev, int pad, void *ws,
                                               size_t ws_bytes, double *sim_out, float *grad_u, double *grad_affine,
                                               void *stream);

/* One Adam step of the affine stage (the optimiser state m1, m2 of Sec. 3.1
 * applied to the 12 parameters of phi(p) = A (p - c) + c + tc / s, the map
 * about the centre c of a pyramid level of scale s, tc in voxels of the
 * finest grid), on one device thread in FP64:
 *   gA = dC/dA - (dC/dt) c^T,  gtc = (dC/dt) / s,
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2  (per parameter),
 *   A  -= decay lr_A   mhat / (sqrt(vhat) + eps),
 *   tc -= decay lr_t s mhat / (sqrt(vhat) + eps),
 * with bias correction 1 - beta^(k+1) and decay = 1 - (1 - final_lr) k /
 * max(iters - 1, 1) (the steps shrink linearly to final_lr of their value over
 * the level).  grad_affine: device double[12] as reg_loss_grad_composite
 * writes it (dC/dA row-major, dC/dt) for the transform T_dev held; sim: device
 * double[1], its similarity.  state: device double[36] = A (9), tc (3), m_A
 * (9), v_A (9), m_t (3), v_t (3), updated in place (the caller sets A = I,
 * tc = 0 and the moments to 0 to start, the moments again at a new level).
 * T_dev: device float[15], overwritten with the next transform (A, t = c - A c
 * + tc / s, s = 1).  obj_out (device double[1], may be NULL) receives the
 * objective at the input transform: 1 - S (LNCC) or -MI.  k >= 0 is the
 * step's index within its level. */
typedef struct reg_affine_adam_desc {
    double lr_A, lr_t, beta1, beta2, eps, final_lr;
    int iters;          /* steps in this level (for the decay) */
    double scale;       /* s: the level's voxel size in voxels of the finest grid */
    double centre[3];   /* c: the level's volume centre (voxels of that level, x, y, z) */
    int loss_kind;      /* reg_loss_kind of the objective recorded in obj_out */
} reg_affine_adam_desc;
REG_API reg_status reg_affine_adam_step(const double *grad_affine, const double *sim, double *state, float *T_dev,
                                        const reg_affine_adam_desc *desc, int k, double *obj_out, void *stream);

/* Composition of displacement fields (the fused sampler applied to a
 * 3-channel field): (id + w) = (id + b) o (id + a), i.e.
 *     w(p) = a(p) + b(p + a(p)),
 * all three channels of b sampled trilinearly at one location (padding
 * `pad` as reg_warp).  a, b, w: FP32 [3][N]; w must not overlap a or b
 * (REG_ERR_INVALID_ARG); a and b may be the same field. */
REG_API reg_status reg_compose_fields(const float *a, const float *b, reg_dims d, int pad, float *w, void *stream);

/* Backward of reg_compose_fields for gw = dL/dw (FP32 [3][N]):
 *   ga = gw + (grad b)^T gw, the slope of b taken at the sample points p + a(p);
 *   gb = the scatter of gw onto the 8 corners of every sample with its
 *        trilinear weights (the transpose of sampling b; Algorithm
 *        gridsampler, backward, the moving-image gradient).
 * ga, gb: FP32 [3][N], overwritten, overlapping neither each other nor the
 * inputs.  When a and b are one field, pass ga == NULL: gb then receives the
 * whole gradient (both terms).  gb is accumulated with float atomics, so its
 * last bits can differ between runs. */
REG_API reg_status reg_compose_fields_backward(const float *a, const float *b, const float *gw, reg_dims d, int pad,
                                               float *ga, float *gb, void *stream);

/* Scaling and squaring: the exponential of a stationary velocity field v,
 * u_0 = v / 2^steps, then `steps` times u <- u + u o (id + u) (the
 * composition above; the first step reads v and applies the 2^-steps itself,
 * so no scaled copy is made).  out receives u_steps; tmp is a second [3][N]
 * buffer (ping-pong).  saved (optional, NULL skips it): (steps - 1) x [3][N]
 * floats receiving u_1 .. u_{steps-1} for reg_exp_field_backward (tmp is then
 * not used).  steps in [0, 30] (0 copies v); out, tmp, saved and v must not
 * overlap.  No identity or sampling grid is materialised. */
REG_API reg_status reg_exp_field(const float *v, reg_dims d, int steps, int pad, float *tmp, float *out,
                                 float *saved, void *stream);

/* Backward of scaling and squaring: gv = dL/dv for gout = dL/d exp(v),
 * through every squaring step (both adjoint terms of the composition), last
 * step first.  saved: the u_1 .. u_{steps-1} written by reg_exp_field with the
 * same v, steps and pad (may be NULL when steps <= 1); tmp: a [3][N] buffer;
 * gv: FP32 [3][N], overwritten.  gout, tmp, gv and the inputs must not
 * overlap.  Float atomics as in reg_compose_fields_backward. */
REG_API reg_status reg_exp_field_backward(const float *v, reg_dims d, int steps, int pad, const float *saved,
                                          const float *gout, float *tmp, float *gv, void *stream);

/* `iters` fused iterations (as reg_iterate) in one call, numbered t0 + 1 ..
 * t0 + iters, without returning to the caller between them: iteration k
 * (0-based) reads u[k % 2] and writes u[(k + 1) % 2] with u = {u_a, u_b}, so
 * the last iterate is in u_a when iters is even and in u_b when it is odd.
 * obj_hist: device double[2 * iters]; entry 2k, 2k + 1 = {similarity,
 * R} at iteration k's input.  The launches are those of `iters`
 * reg_iterate calls on `stream` (MI: the same results bit for bit); only the
 * host work between them is gone, which is what bounds small volumes.  LNCC:
 * F does not change during the call, so the window mean and variance of F
 * are formed once, before the first iteration, and every iteration's window
 * statistics box-sum only J, J^2 and FJ (the results then differ from
 * reg_iterate's in the last bits).
 * iters = 0 does nothing; iters < 0 or t0 < 0 is REG_ERR_INVALID_ARG; u_a
 * and u_b must not overlap.
 * T (optional, NULL = the plain phi = p + u): a composite transform
 * (reg_affine); the iterations then optimise u under phi = A p + t + S u with
 * A, t, S fixed -- the loss gradient S dC/dphi, the diffusion term on u and
 * Adam, fused as in the plain case. */
REG_API reg_status reg_run(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, float *u_a,
                           float *u_b, void *m, void *v, reg_dims d, int pad, float lambda,
                           const reg_adam_desc *adam, int t0, int iters, void *ws, size_t ws_bytes,
                           double *obj_hist, const reg_affine *T, void *stream);

/* Fold check of phi = id + u: min over voxels of det(I + grad u) (central
 * differences, one-sided at the border) and the number of voxels with
 * det <= 0.  min_out: device float[1]; nfold_out: device unsigned long long[1]. */
REG_API reg_status reg_jacdet_min(const float *u, reg_dims d, void *ws, size_t ws_bytes, float *min_out,
                          unsigned long long *nfold_out, void *stream);

/* Synchronises `stream`, returns the device error word accumulated by
 * earlier calls on this device (REG_OK, REG_ERR_NONFINITE or
 * REG_ERR_TIMEOUT; the first latched code wins) and clears it. */
REG_API reg_status reg_get_device_error(void *stream);

/* MI similarity and (optionally) its gradient, like reg_loss_grad with an
 * MI descriptor, but with no workspace argument: for callers that cannot
 * allocate device memory -- a host application or framework that has
 * reserved all GPU memory for its own pool and allows no other allocation,
 * or a latency-critical loop that must never enter the allocator (cudaMalloc
 * and cudaFree can synchronise the device).  The paper has no counterpart;
 * this is a property of the library, not of the method.
 *   - Scratch: a fixed 112 KiB array inside the library (joint histogram
 *     u64[64*64] + adjoint table f32[64*64] and its 4-wide rows
 *     f32x4[64*64]), held by every GPU that loads
 *     the library until the process exits.  bins must be in [8, 64]; larger
 *     counts do not fit and return REG_ERR_SHAPE; a non-MI descriptor returns
 *     REG_ERR_UNSUPPORTED.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address and keeps it for the life of the process (so
 *     not across a cudaDeviceReset); make that first call before any stream
 *     capture.
 *   - Every call shares the one array (it keeps the previous call's
 *     contents; the histogram is cleared at the start of each call), so calls
 *     that may overlap on the GPU -- different streams, or several host
 *     threads -- race and must be serialised by the caller.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * sim_out: device double[1] (MI); grad_u: FP32 [3][N] or NULL (dC/du of
 * C = -MI, overwritten).  Other arguments as reg_loss_grad. */
REG_API reg_status reg_mi_loss_grad_noalloc(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                                            const float *u, reg_dims d, int pad, double *sim_out, float *grad_u,
                                            void *stream);

/* Timing hook: the NEXT reg_iterate call on this host thread records the
 * caller's CUDA events (cudaEvent_t passed as void*) on its stream:
 * events[0] before the first sweep, events[1] between the sweeps (after the
 * MI finalisation), events[2] after the second sweep; then the hook clears
 * itself.  With n = 3 * iters events the next reg_run call of `iters`
 * iterations takes them instead: events[3k .. 3k + 2] for iteration k, at
 * the same points.  A reg_run call of another length leaves the hook armed.  n must be a positive multiple
 * of 3 (at most 3 * 2^20), or 0 with events == NULL to clear.  Lets a caller
 * time each sweep inside a long run without synchronising. */
REG_API reg_status reg_set_timing_events(void *const *events, int n);

/* ------------------------------------------------------------------------
 * Learned initialiser: operators of a small 3-D U-Net that predicts a
 * half-resolution initial displacement from a downsampled (F, M) pair.  The
 * paper has no learned initialiser of its own (it trains other networks
 * with its fused losses, Sec. 4); the network is specified alongside the
 * method as an extension.  The convolutions are the only tensor-core work:
 * BF16 implicit GEMMs on tcgen05 with FP32 accumulation in tensor memory.
 *
 * Layouts: activations are channels-last BF16 [nz][ny][nx][C] with C % 8 == 0
 * (8 channels = one 16-byte load); volumes here have fewer than 2^31
 * voxels.  Weights are packed BF16 [rows][Kpad], k = tap * Cin + cin,
 * tap = (kz * 3 + ky) * 3 + kx for the offset (kx-1, ky-1, kz-1), Kpad =
 * reg_nn_conv_kpad(Cin), rows = Cout rounded up to 16 (extra rows and K
 * padding zero).  3 x 3 x 3 taps, zero padding 1, stride 1.  Displacement
 * fields are SoA FP32 [3][nz][ny][nx] in voxel units of their own grid.
 * All entry points validate on the host, enqueue on `stream`, allocate
 * nothing; scratch buffers are the caller's.
 * ------------------------------------------------------------------------ */

/* Kpad (the packed K length, a multiple of 64) for Cin input channels. */
REG_API size_t reg_nn_conv_kpad(int Cin);

/* Scratch for the TMA-fed forward convolution: the weights re-tiled into the
 * tensor cores' shared-memory layout (0 when Cin % 16 != 0: that shape has
 * only the gather kernel). */
REG_API size_t reg_nn_conv_scratch_bytes(int Cin, int Cout);

/* out = epilogue(conv(in, W)): epilogue 0 = LeakyReLU(acc + bias, slope) ->
 * BF16 channels-last (Cout % 8 == 0); 1 = acc -> BF16 (no bias); 2 = acc +
 * bias -> FP32 SoA [Cout][N voxels] (any Cout <= 64).  Cin in [8, 128].
 * With scratch (>= reg_nn_conv_scratch_bytes bytes, 16-byte aligned,
 * else REG_ERR_WORKSPACE / REG_ERR_ALIGN) and Cin % 16 == 0, nx <= 254 the
 * input brick of each output tile is loaded by TMA and every tap is one
 * shifted tensor-core operand; otherwise (scratch NULL) each CTA gathers
 * its im2col tile from global memory.  Both give the same sums up to FP32
 * accumulation order. */
REG_API reg_status reg_nn_conv3d_fwd(const void *in, int Cin, const void *W, const float *bias, int Cout, reg_dims d,
                                     int epilogue, float slope, void *scratch, size_t scratch_bytes, void *out,
                                     void *stream);

/* Data gradient: din (BF16 channels-last, Cin) = conv^T(dpre (Cout), W): the
 * weights are flipped and transposed into Wd_scratch
 * (reg_nn_dgrad_scratch_bytes, which also holds their re-tiled copy), then
 * the forward kernel runs on them (the TMA-fed one when Cout % 16 == 0). */
REG_API size_t reg_nn_dgrad_scratch_bytes(int Cin, int Cout);
REG_API reg_status reg_nn_conv3d_dgrad(const void *dpre, int Cout, const void *W, int Cin, reg_dims d,
                                       void *Wd_scratch, void *din, void *stream);

/* Weight gradient: dW (FP32, packed [Cout][Kpad]) = sum over voxels of
 * in_col (x) dpre, as per-CTA partial sums in scratch
 * (reg_nn_wgrad_scratch_bytes) reduced in a fixed order (deterministic).
 * Cout in {16, 32, 48, 64} (pad a smaller Cout with zero channels).  With
 * Cin % 16 == 0 and nx <= 254, persistent CTAs stream TMA-loaded input
 * bricks and dpre rows through the tensor cores with the 27 per-tap sums in
 * tensor memory; otherwise each CTA gathers im2col tiles. */
REG_API size_t reg_nn_wgrad_scratch_bytes(reg_dims d, int Cin, int Cout);
REG_API reg_status reg_nn_conv3d_wgrad(const void *in, int Cin, const void *dpre, int Cout, reg_dims d,
                                       void *scratch, size_t scratch_bytes, float *dW, void *stream);

/* Network input: average-pool F and M (img_dt, dims d) by `factor`, map each
 * to (v - lo) / (hi - lo), write channels-last BF16 with 16 channels (F, M,
 * 14 zeros) at d / factor. */
REG_API reg_status reg_nn_pack_pair(const void *F, const void *M, int img_dt, reg_dims d, int factor, float f_lo,
                                    float f_hi, float m_lo, float m_hi, void *out, void *stream);

/* dpre = dout * (out > 0 ? 1 : slope) over n BF16 elements (LeakyReLU backward
 * from its output, which has the sign of its input). */
REG_API reg_status reg_nn_leaky_bwd(const void *out, const void *dout, long long n, float slope, void *dpre,
                                    void *stream);

/* dbias[c] = sum over V voxels of dpre[v][c] (fixed-order FP64 partials). */
REG_API size_t reg_nn_bias_grad_scratch_bytes(int C);
REG_API reg_status reg_nn_bias_grad(const void *dpre, long long V, int C, void *scratch, float *dbias, void *stream);

/* 2x average pooling of a channels-last BF16 volume of dims d_in (even), or
 * its backward (in = gradient at d_in / 2, out = gradient at d_in). */
REG_API reg_status reg_nn_avgpool2(const void *in, int C, reg_dims d_in, void *out, int backward, void *stream);

/* 2x trilinear upsampling (voxel-centre aligned, border clamped) of a
 * channels-last BF16 volume of dims d_coarse, or its backward (a gather). */
REG_API reg_status reg_nn_upsample2(const void *in, int C, reg_dims d_coarse, void *out, int backward, void *stream);

/* Channel concat / slice over V voxels: put writes src (Csrc channels) into
 * channels [c0, c0 + Csrc) of dst (Cdst channels); take copies channels
 * [c0, c0 + Cdst) of src into dst; accumulate != 0 adds instead of copying. */
REG_API reg_status reg_nn_put_channels(const void *src, int Csrc, long long V, void *dst, int Cdst, int c0,
                                       int accumulate, void *stream);
REG_API reg_status reg_nn_take_channels(const void *src, int Csrc, int c0, long long V, void *dst, int Cdst,
                                        int accumulate, void *stream);

/* Training loss: loss (device double) = mean of (pred - target)^2 over the 3
 * SoA channels of V voxels; dpred = its gradient as channels-last BF16 with
 * Cpad channels (channels >= 3 zero). */
REG_API size_t reg_nn_mse_scratch_bytes(void);
REG_API reg_status reg_nn_mse(const float *pred, const float *target, long long V, int Cpad, void *dpred,
                              void *scratch, double *loss, void *stream);

/* Displacement resampling: 2x average pooling rescaled to the coarse voxel
 * size (u / 2), and trilinear upsampling by an integer factor rescaled to the
 * fine voxel size (u * factor). */
REG_API reg_status reg_nn_field_down2(const float *u, reg_dims d_fine, float *out, void *stream);
REG_API reg_status reg_nn_field_upsample(const float *u, reg_dims d_coarse, int factor, float *out, void *stream);

/* Adam on FP32 master weights (n elements, grad_scale applied), optionally
 * writing the BF16 copy used by the convolutions. */
REG_API reg_status reg_nn_adam(float *w, float *m, float *v, const float *g, long long n, const reg_adam_desc *adam,
                               int t, void *w_bf16, void *stream);

/* Test hook for the tensor-core engine: C[M x N] (FP32, row-major) =
 * A B^T with BF16 A and B, computed by the tcgen05 mainloop used by the
 * convolutions.  a_mn_major == 0: A is [M][K] (K contiguous), 1: [K][M];
 * likewise B with N.  M % 128 == 0, N % 16 == 0 and N <= 128, K % 64 == 0. */
REG_API reg_status reg_debug_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int a_mn_major,
                                       int b_mn_major, void *stream);

/* Test hook for failure detection: a one-thread kernel polls *flag (device
 * unsigned) until it equals `expect` or `timeout_ns` nanoseconds of device
 * time pass; on expiry it latches REG_ERR_TIMEOUT in the device error word
 * and returns (no trap, the context stays usable).  Used to show that a
 * device wait which never completes is reported, not hung. */
REG_API reg_status reg_debug_wait_flag(const unsigned *flag, unsigned expect, unsigned long long timeout_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* REG_H */
