// capi.cu -- the C ABI of include/reg.h: host-side validation, workspace
// layout and kernel sequencing.  Every entry point validates all arguments
// before enqueueing anything and allocates no memory.
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "checks.h"
#include "kernels.h"

using namespace regk;

namespace {

// ---------------------------------------------------------------------------
// workspace layout (caller-owned, 256-byte aligned sections)
// ---------------------------------------------------------------------------
constexpr size_t WS_HIST = 0;                                        // u64[64*64]
constexpr size_t WS_COUNTERS = WS_HIST + sizeof(unsigned long long) * MAX_BINS * MAX_BINS;  // u32[64]
constexpr size_t WS_ZERO_BYTES = WS_COUNTERS + 256;                  // zeroed by every call
constexpr size_t WS_GTAB = WS_ZERO_BYTES;                            // f32[64*64] + f32x4[64*64]
constexpr size_t WS_SCRATCH = WS_GTAB + MI_TABLE_BYTES;               // f64[32]
constexpr size_t WS_PARTIALS = WS_SCRATCH + 256;                     // f64[12 * max blocks]
constexpr size_t PARTIALS_PER_BLOCK = 12;  // the composite sweeps reduce dC/dA, dC/dt

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

reg_status check_adam(const reg_adam_desc *A, int t) {
    if (!A) return REG_ERR_INVALID_ARG;
    if (t < 1) return REG_ERR_INVALID_ARG;
    if (!(A->lr > 0.0f) || !isfinite(A->lr)) return REG_ERR_INVALID_ARG;
    if (!(A->beta1 >= 0.0f && A->beta1 < 1.0f) || !(A->beta2 >= 0.0f && A->beta2 < 1.0f)) return REG_ERR_INVALID_ARG;
    if (!(A->eps >= 0.0f) || !isfinite(A->eps)) return REG_ERR_INVALID_ARG;
    if (!(A->grad_scale > 0.0f) || !isfinite(A->grad_scale)) return REG_ERR_INVALID_ARG;
    if (A->moment_dtype != REG_F32 && A->moment_dtype != REG_BF16) return REG_ERR_DTYPE;
    return REG_OK;
}

long long max_partial_blocks(const Dims &g, const reg_loss_desc *L) {
    long long nb = diffusion_grid(g).blocks();
    const long long mi = mi_sweep_grid(g).blocks();
    if (mi > nb) nb = mi;
    if (mi_tma_ok(g)) {
        const long long mt = mi_tma_max_blocks(g);
        if (mt > nb) nb = mt;
    }
    if (L && L->kind == REG_LOSS_LNCC) {
        const long long ln = lncc_max_blocks(g);
        if (ln > nb) nb = ln;
    }
    return nb;
}

size_t workspace_bytes(const Dims &g, const reg_loss_desc *L) {
    size_t bytes = align256(WS_PARTIALS + sizeof(double) * PARTIALS_PER_BLOCK * (size_t)max_partial_blocks(g, L));
    // LNCC: three coefficient fields and the warped image
    // LNCC: three coefficient fields, the warped image, F's window mean and variance
    if (L && L->kind == REG_LOSS_LNCC) bytes = align256(bytes + sizeof(float) * 6 * (size_t)g.n);
    return bytes;
}

struct Ws {
    unsigned long long *hist;
    unsigned *counters;
    float *gtab;
    double *scratch;
    double *partials;
    float *coef;   // LNCC: [3][N] adjoint coefficients
    float *warped; // LNCC: [N] warped moving image
    float *fstat;  // LNCC: [2][N] window mean and variance of F (formed once per reg_run)
};

Ws carve(void *ws, const Dims &g, const reg_loss_desc *L) {
    char *b = (char *)ws;
    Ws w;
    w.hist = (unsigned long long *)(b + WS_HIST);
    w.counters = (unsigned *)(b + WS_COUNTERS);
    w.gtab = (float *)(b + WS_GTAB);
    w.scratch = (double *)(b + WS_SCRATCH);
    w.partials = (double *)(b + WS_PARTIALS);
    w.coef = (float *)(b + align256(WS_PARTIALS + sizeof(double) * PARTIALS_PER_BLOCK *
                                               (size_t)max_partial_blocks(g, L)));
    w.warped = w.coef + 3 * (size_t)g.n;
    w.fstat = w.warped + (size_t)g.n;
    return w;
}

MiParams mi_params(const reg_loss_desc *L) {
    MiParams P;
    P.f_lo = L->f_lo;
    P.f_scale = (float)(1.0 / ((double)L->f_hi - (double)L->f_lo));
    P.m_lo = L->m_lo;
    P.m_scale = (float)(1.0 / ((double)L->m_hi - (double)L->m_lo));
    P.bins = L->bins;
    P.hard = L->mi_estimator == REG_MI_HARD;
    return P;
}

StepParams step_params(const reg_adam_desc *A, int t, float lam, const Dims &g) {
    StepParams S;
    S.lam = lam;
    S.two_over_n = (float)(2.0 / (double)g.n);
    const double bc1 = 1.0 - pow((double)A->beta1, (double)t);
    const double bc2 = 1.0 - pow((double)A->beta2, (double)t);
    S.lr_bc1 = (float)((double)A->lr / bc1);
    S.rsqrt_bc2 = (float)(1.0 / sqrt(bc2));
    S.b1 = A->beta1;
    S.b2 = A->beta2;
    S.eps = A->eps;
    S.gscale = A->grad_scale;
    return S;
}

// the timing hook: 3 events for one reg_iterate call, or 3 per iteration
// of a reg_run call; t_base selects the iteration's three
thread_local std::vector<cudaEvent_t> t_events;
thread_local bool t_events_armed = false;
thread_local size_t t_base = 0;

cudaError_t mark(int i, cudaStream_t s) {
    if (!t_events_armed || t_base + i >= t_events.size() || !t_events[t_base + i]) return cudaSuccess;
    return cudaEventRecord(t_events[t_base + i], s);
}

reg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? REG_OK : REG_ERR_CUDA; }

#define REG_TRY(expr)                            \
    do {                                         \
        const reg_status _s = (expr);            \
        if (_s != REG_OK) return _s;             \
    } while (0)

#define REG_CUDA(expr)                                 \
    do {                                               \
        const cudaError_t _e = (expr);                 \
        if (_e != cudaSuccess) return REG_ERR_CUDA;    \
    } while (0)

reg_status check_ptr(const void *p) {
    if (!p) return REG_ERR_INVALID_ARG;
    if (!aligned16(p)) return REG_ERR_ALIGN;
    return REG_OK;
}
reg_status check_opt_ptr(const void *p) { return p ? check_ptr(p) : REG_OK; }

// whether two [3][n] FP32 fields share any byte
bool overlap3(const float *a, const float *b, long long n) {
    const uintptr_t a0 = (uintptr_t)a, a1 = a0 + sizeof(float) * 3 * (size_t)n;
    const uintptr_t b0 = (uintptr_t)b, b1 = b0 + sizeof(float) * 3 * (size_t)n;
    return a0 < b1 && b0 < a1;
}

reg_status check_common(const reg_loss_desc *L, const void *F, const void *M, int img_dt, const float *u,
                        reg_dims d, int pad, void *ws, size_t ws_bytes) {
    REG_TRY(check_dims(d));
    REG_TRY(check_loss(L));
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(F));
    REG_TRY(check_ptr(M));
    REG_TRY(check_ptr(u));
    REG_TRY(check_ptr(ws));
    if (ws_bytes < workspace_bytes(make_dims(d), L)) return REG_ERR_WORKSPACE;
    return REG_OK;
}

bool affine_ok(const reg_affine *T) {
    if (!T) return false;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(T->A[i])) return false;
    for (int i = 0; i < 3; ++i)
        if (!isfinite(T->t[i]) || !isfinite(T->s[i])) return false;
    return true;
}

// the kernels' form: A - I (taken in double, rounded once), t, s
AffineT to_affine(const reg_affine &T) {
    AffineT a;
    for (int i = 0; i < 9; ++i) a.am[i] = (float)((double)T.A[i] - (i % 4 == 0 ? 1.0 : 0.0));
    for (int i = 0; i < 3; ++i) {
        a.t[i] = T.t[i];
        a.s[i] = T.s[i];
    }
    return a;
}

// sweep 1 of either loss: similarity into sim_out (+ LNCC coefficient fields)
reg_status run_sweep1(const reg_loss_desc *L, const void *F, const void *M, int img_dt, const float *u,
                      const Dims &g, int pad, const Ws &w, double *sim_out, bool need_grad, cudaStream_t s,
                      const AffineT *aff = nullptr, const float *fstat = nullptr) {
    REG_CUDA(cudaMemsetAsync(w.hist, 0, WS_ZERO_BYTES, s));
    if (L->kind == REG_LOSS_LNCC) {
        LnccParams P{L->window / 2, L->eps, L->lncc_grad == REG_LNCC_GRAD_ANTS};
        REG_CUDA(launch_warp(M, img_dt, u, g, pad, w.warped, nullptr, s, aff));
        REG_CUDA(launch_lncc_stats(F, w.warped, img_dt, g, P, need_grad ? w.coef : nullptr, w.partials,
                                   w.counters + 0, sim_out, s, fstat));
    } else {
        const MiParams P = mi_params(L);
        REG_CUDA(launch_mi_hist(F, M, img_dt, u, g, pad, P, w.hist, s, aff));
        REG_CUDA(launch_mi_finalize(w.hist, P, g.n, w.gtab, sim_out, s));
    }
    return REG_OK;
}

}  // namespace

extern "C" {

int reg_version(void) { return 100; }

const char *reg_status_string(reg_status s) {
    switch (s) {
        case REG_OK: return "ok";
        case REG_ERR_INVALID_ARG: return "invalid argument";
        case REG_ERR_SHAPE: return "unsupported shape, window or bin count";
        case REG_ERR_DTYPE: return "unknown dtype";
        case REG_ERR_ALIGN: return "pointer not 16-byte aligned";
        case REG_ERR_WORKSPACE: return "workspace too small";
        case REG_ERR_NONFINITE: return "non-finite value in a loss or regulariser reduction";
        case REG_ERR_TIMEOUT: return "bounded device wait expired";
        case REG_ERR_CUDA: return "CUDA runtime error";
        case REG_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

reg_status reg_workspace_size(const reg_loss_desc *loss, reg_dims d, size_t *bytes) {
    if (!bytes) return REG_ERR_INVALID_ARG;
    REG_TRY(check_dims(d));
    if (loss) REG_TRY(check_loss(loss));
    *bytes = workspace_bytes(make_dims(d), loss);
    return REG_OK;
}

reg_status reg_warp(const void *M, int img_dt, const float *u, reg_dims d, int pad, float *J_out, float *dJ_out,
                    void *stream) {
    REG_TRY(check_dims(d));
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(M));
    REG_TRY(check_ptr(u));
    REG_TRY(check_ptr(J_out));
    REG_TRY(check_opt_ptr(dJ_out));
    return cuda_status(launch_warp(M, img_dt, u, make_dims(d), pad, J_out, dJ_out, (cudaStream_t)stream));
}

reg_status reg_loss(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u, reg_dims d,
                    int pad, void *ws, size_t ws_bytes, double *sim_out, void *stream) {
    REG_TRY(check_common(loss, F, M, img_dt, u, d, pad, ws, ws_bytes));
    REG_TRY(check_ptr(sim_out));
    const Dims g = make_dims(d);
    const Ws w = carve(ws, g, loss);
    return run_sweep1(loss, F, M, img_dt, u, g, pad, w, sim_out, false, (cudaStream_t)stream);
}

reg_status reg_loss_grad(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u,
                         reg_dims d, int pad, void *ws, size_t ws_bytes, double *sim_out, float *grad_u,
                         void *stream) {
    REG_TRY(check_common(loss, F, M, img_dt, u, d, pad, ws, ws_bytes));
    REG_TRY(check_ptr(sim_out));
    REG_TRY(check_ptr(grad_u));
    const Dims g = make_dims(d);
    const Ws w = carve(ws, g, loss);
    const cudaStream_t s = (cudaStream_t)stream;
    REG_TRY(run_sweep1(loss, F, M, img_dt, u, g, pad, w, sim_out, true, s));
    StepParams S{};
    if (loss->kind == REG_LOSS_LNCC) {
        LnccParams P{loss->window / 2, loss->eps, loss->lncc_grad == REG_LNCC_GRAD_ANTS};
        REG_CUDA(launch_lncc_sweep2(F, M, img_dt, u, g, pad, P, w.coef, grad_u, false, nullptr, nullptr, nullptr,
                                    REG_F32, S, w.partials, w.counters + 1, w.scratch, s));
    } else {
        REG_CUDA(launch_mi_sweep2(F, M, img_dt, u, g, pad, mi_params(loss), w.gtab, grad_u, false, nullptr, nullptr,
                                  nullptr, REG_F32, S, w.partials, w.counters + 1, w.scratch, s));
    }
    return REG_OK;
}

reg_status reg_regularize(const float *u, reg_dims d, float lambda, void *ws, size_t ws_bytes, double *r_out,
                          float *grad_u, void *stream) {
    REG_TRY(check_dims(d));
    if (!isfinite(lambda)) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(u));
    REG_TRY(check_ptr(ws));
    REG_TRY(check_ptr(r_out));
    REG_TRY(check_opt_ptr(grad_u));
    const Dims g = make_dims(d);
    if (ws_bytes < workspace_bytes(g, nullptr)) return REG_ERR_WORKSPACE;
    const Ws w = carve(ws, g, nullptr);
    const cudaStream_t s = (cudaStream_t)stream;
    REG_CUDA(cudaMemsetAsync(w.counters, 0, 256, s));
    return cuda_status(launch_diffusion(u, g, lambda, grad_u, w.partials, w.counters + 2, r_out, s));
}

reg_status reg_step(const float *u_in, float *u_out, void *m, void *v, const float *grad_u, reg_dims d,
                    const reg_adam_desc *adam, int t, void *stream) {
    REG_TRY(check_dims(d));
    REG_TRY(check_adam(adam, t));
    REG_TRY(check_ptr(u_in));
    REG_TRY(check_ptr(u_out));
    REG_TRY(check_ptr(m));
    REG_TRY(check_ptr(v));
    REG_TRY(check_ptr(grad_u));
    const Dims g = make_dims(d);
    const StepParams S = step_params(adam, t, 0.0f, g);
    return cuda_status(launch_adam(u_in, u_out, m, v, adam->moment_dtype, grad_u, 3 * g.n, S, (cudaStream_t)stream));
}

// one fused iteration; aff: the composite transform (NULL: phi = p + u);
// fcached: F's LNCC window statistics are already in the workspace
static reg_status iterate_impl(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                               const float *u_in, float *u_out, void *m, void *v, reg_dims d, int pad, float lambda,
                               const reg_adam_desc *adam, int t, void *ws, size_t ws_bytes, double *obj_out,
                               float *grad_out, void *stream, const AffineT *aff, bool fcached = false);

reg_status reg_iterate(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u_in,
                       float *u_out, void *m, void *v, reg_dims d, int pad, float lambda, const reg_adam_desc *adam,
                       int t, void *ws, size_t ws_bytes, double *obj_out, float *grad_out, void *stream) {
    return iterate_impl(loss, F, M, img_dt, u_in, u_out, m, v, d, pad, lambda, adam, t, ws, ws_bytes, obj_out,
                        grad_out, stream, nullptr);
}

static reg_status iterate_impl(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                               const float *u_in, float *u_out, void *m, void *v, reg_dims d, int pad, float lambda,
                               const reg_adam_desc *adam, int t, void *ws, size_t ws_bytes, double *obj_out,
                               float *grad_out, void *stream, const AffineT *aff, bool fcached) {
    REG_TRY(check_common(loss, F, M, img_dt, u_in, d, pad, ws, ws_bytes));
    REG_TRY(check_adam(adam, t));
    if (!isfinite(lambda)) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(u_out));
    REG_TRY(check_ptr(m));
    REG_TRY(check_ptr(v));
    REG_TRY(check_ptr(obj_out));
    REG_TRY(check_opt_ptr(grad_out));
    const Dims g = make_dims(d);
    {
        const uintptr_t a0 = (uintptr_t)u_in, a1 = a0 + sizeof(float) * 3 * (size_t)g.n;
        const uintptr_t b0 = (uintptr_t)u_out, b1 = b0 + sizeof(float) * 3 * (size_t)g.n;
        if (a0 < b1 && b0 < a1) return REG_ERR_INVALID_ARG;  // u_out must not overlap u_in
    }
    const Ws w = carve(ws, g, loss);
    const cudaStream_t s = (cudaStream_t)stream;
    REG_CUDA(mark(0, s));
    REG_TRY(run_sweep1(loss, F, M, img_dt, u_in, g, pad, w, obj_out, true, s, aff, fcached ? w.fstat : nullptr));
    REG_CUDA(mark(1, s));
    const StepParams S = step_params(adam, t, lambda, g);
    if (loss->kind == REG_LOSS_LNCC) {
        LnccParams P{loss->window / 2, loss->eps, loss->lncc_grad == REG_LNCC_GRAD_ANTS};
        REG_CUDA(launch_lncc_sweep2(F, M, img_dt, u_in, g, pad, P, w.coef, grad_out, true, u_out, m, v,
                                    adam->moment_dtype, S, w.partials, w.counters + 1, obj_out + 1, s, aff));
    } else {
        REG_CUDA(launch_mi_sweep2(F, M, img_dt, u_in, g, pad, mi_params(loss), w.gtab, grad_out, true, u_out, m, v,
                                  adam->moment_dtype, S, w.partials, w.counters + 1, obj_out + 1, s, aff));
    }
    REG_CUDA(mark(2, s));
    t_events_armed = false;
    return REG_OK;
}

reg_status reg_run(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, float *u_a, float *u_b,
                   void *m, void *v, reg_dims d, int pad, float lambda, const reg_adam_desc *adam, int t0, int iters,
                   void *ws, size_t ws_bytes, double *obj_hist, const reg_affine *T, void *stream) {
    if (iters < 0 || t0 < 0 || (long long)t0 + iters > INT_MAX) return REG_ERR_INVALID_ARG;
    if (T && !affine_ok(T)) return REG_ERR_INVALID_ARG;
    if (iters == 0) return REG_OK;
    AffineT A;
    if (T) A = to_affine(*T);
    // validate once (the per-iteration calls repeat the same checks, which
    // cost nothing next to a launch)
    REG_TRY(check_common(loss, F, M, img_dt, u_a, d, pad, ws, ws_bytes));
    REG_TRY(check_adam(adam, t0 + 1));
    REG_TRY(check_ptr(u_b));
    REG_TRY(check_ptr(obj_hist));
    // everything the iterations check, before the first launch
    if (!isfinite(lambda)) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(m));
    REG_TRY(check_ptr(v));
    if (overlap3(u_a, u_b, make_dims(d).n)) return REG_ERR_INVALID_ARG;
    // the timing hook: this call takes it when it holds three events per
    // iteration, else leaves it armed for the next reg_iterate call
    const bool armed = t_events_armed;
    const bool per_iter = armed && t_events.size() == 3 * (size_t)iters;
    t_events_armed = false;
    // LNCC: F is fixed for the whole run, so its window mean and variance are
    // formed once here and every iteration box-sums only (J, J^2, FJ)
    const bool fcached = loss->kind == REG_LOSS_LNCC;
    if (fcached) {
        const Dims g = make_dims(d);
        const Ws w = carve(ws, g, loss);
        const LnccParams P{loss->window / 2, loss->eps, loss->lncc_grad == REG_LNCC_GRAD_ANTS};
        REG_CUDA(launch_lncc_fstats(F, img_dt, g, P, w.fstat, (cudaStream_t)stream));
    }
    reg_status st = REG_OK;
    for (int k = 0; k < iters && st == REG_OK; ++k) {
        if (per_iter) {
            t_events_armed = true;
            t_base = 3 * (size_t)k;
        }
        float *a = (k % 2) ? u_b : u_a, *b = (k % 2) ? u_a : u_b;
        st = iterate_impl(loss, F, M, img_dt, a, b, m, v, d, pad, lambda, adam, t0 + k + 1, ws, ws_bytes,
                          obj_hist + 2 * (size_t)k, nullptr, stream, T ? &A : nullptr, fcached);
    }
    t_base = 0;
    t_events_armed = per_iter ? false : armed;
    return st;
}

reg_status reg_warp_composite(const void *M, int img_dt, const float *u, reg_dims d, const reg_affine *T, int pad,
                              float *J, float *dJ, void *stream) {
    REG_TRY(check_dims(d));
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    if (!affine_ok(T)) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(M));
    REG_TRY(check_opt_ptr(u));
    REG_TRY(check_ptr(J));
    REG_TRY(check_opt_ptr(dJ));
    const AffineT A = to_affine(*T);
    return cuda_status(launch_warp(M, img_dt, u, make_dims(d), pad, J, dJ, (cudaStream_t)stream, &A));
}

reg_status reg_warp_composite_backward(const void *M, int img_dt, const float *u, reg_dims d, const reg_affine *T,
                                       int pad, const float *g, float *g_u, double *grad_affine, void *ws,
                                       size_t ws_bytes, void *stream) {
    REG_TRY(check_dims(d));
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    if (!affine_ok(T)) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(M));
    REG_TRY(check_opt_ptr(u));
    REG_TRY(check_ptr(g));
    REG_TRY(check_opt_ptr(g_u));
    REG_TRY(check_opt_ptr(grad_affine));
    REG_TRY(check_ptr(ws));
    const Dims gd = make_dims(d);
    if (ws_bytes < workspace_bytes(gd, nullptr)) return REG_ERR_WORKSPACE;
    const Ws w = carve(ws, gd, nullptr);
    const cudaStream_t s = (cudaStream_t)stream;
    const AffineT A = to_affine(*T);
    REG_CUDA(cudaMemsetAsync(w.counters, 0, 256, s));
    return cuda_status(launch_composite_backward(M, img_dt, u, gd, pad, A, g, g_u, w.partials, w.counters + 2,
                                                 grad_affine ? grad_affine : w.scratch, s));
}

namespace {
// the composite similarity and gradients for a transform given by value or,
// through A.dev, in device memory (arguments other than the transform are
// checked here)
reg_status loss_grad_composite(const reg_loss_desc *loss, const void *F, const void *M, int img_dt, const float *u,
                               reg_dims d, const AffineT &A, int pad, void *ws, size_t ws_bytes, double *sim_out,
                               float *grad_u, double *grad_affine, void *stream) {
    REG_TRY(check_dims(d));
    REG_TRY(check_loss(loss));
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(F));
    REG_TRY(check_ptr(M));
    REG_TRY(check_opt_ptr(u));
    REG_TRY(check_ptr(ws));
    REG_TRY(check_ptr(sim_out));
    REG_TRY(check_opt_ptr(grad_u));
    REG_TRY(check_opt_ptr(grad_affine));
    const Dims g = make_dims(d);
    if (ws_bytes < workspace_bytes(g, loss)) return REG_ERR_WORKSPACE;
    const Ws w = carve(ws, g, loss);
    const cudaStream_t s = (cudaStream_t)stream;
    const bool need_grad = grad_u || grad_affine;
    double *aout = grad_affine ? grad_affine : w.scratch;
    REG_CUDA(cudaMemsetAsync(w.hist, 0, WS_ZERO_BYTES, s));
    StepParams S{};
    if (loss->kind == REG_LOSS_LNCC) {
        const LnccParams P{loss->window / 2, loss->eps, loss->lncc_grad == REG_LNCC_GRAD_ANTS};
        REG_CUDA(launch_warp(M, img_dt, u, g, pad, w.warped, nullptr, s, &A));
        REG_CUDA(launch_lncc_stats(F, w.warped, img_dt, g, P, need_grad ? w.coef : nullptr, w.partials,
                                   w.counters + 0, sim_out, s));
        if (need_grad)
            REG_CUDA(launch_lncc_sweep2(F, M, img_dt, u, g, pad, P, w.coef, grad_u, false, nullptr, nullptr, nullptr,
                                        REG_F32, S, w.partials, w.counters + 2, aout, s, &A));
    } else {
        const MiParams P = mi_params(loss);
        REG_CUDA(launch_mi_hist(F, M, img_dt, u, g, pad, P, w.hist, s, &A));
        REG_CUDA(launch_mi_finalize(w.hist, P, g.n, w.gtab, sim_out, s));
        if (need_grad)
            REG_CUDA(launch_mi_sweep2(F, M, img_dt, u, g, pad, P, w.gtab, grad_u, false, nullptr, nullptr, nullptr,
                                      REG_F32, S, w.partials, w.counters + 2, aout, s, &A));
    }
    return REG_OK;
}
}  // namespace

reg_status reg_loss_grad_composite(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                                   const float *u, reg_dims d, const reg_affine *T, int pad, void *ws,
                                   size_t ws_bytes, double *sim_out, float *grad_u, double *grad_affine,
                                   void *stream) {
    if (!affine_ok(T)) return REG_ERR_INVALID_ARG;
    return loss_grad_composite(loss, F, M, img_dt, u, d, to_affine(*T), pad, ws, ws_bytes, sim_out, grad_u,
                               grad_affine, stream);
}

reg_status reg_loss_grad_composite_dev(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                                       const float *u, reg_dims d, const float *T_dev, int pad, void *ws,
                                       size_t ws_bytes, double *sim_out, float *grad_u, double *grad_affine,
                                       void *stream) {
    REG_TRY(check_ptr(T_dev));
    AffineT A{};
    A.dev = T_dev;
    return loss_grad_composite(loss, F, M, img_dt, u, d, A, pad, ws, ws_bytes, sim_out, grad_u, grad_affine, stream);
}

reg_status reg_affine_adam_step(const double *grad_affine, const double *sim, double *state, float *T_dev,
                                const reg_affine_adam_desc *desc, int k, double *obj_out, void *stream) {
    if (!desc || k < 0 || desc->iters < 1) return REG_ERR_INVALID_ARG;
    const double vals[] = {desc->lr_A, desc->lr_t, desc->eps, desc->final_lr, desc->scale,
                           desc->centre[0], desc->centre[1], desc->centre[2]};
    for (double v : vals)
        if (!isfinite(v)) return REG_ERR_INVALID_ARG;
    if (!(desc->lr_A > 0.0) || !(desc->lr_t > 0.0) || !(desc->eps >= 0.0) || !(desc->scale > 0.0))
        return REG_ERR_INVALID_ARG;
    if (!(desc->beta1 >= 0.0 && desc->beta1 < 1.0) || !(desc->beta2 >= 0.0 && desc->beta2 < 1.0))
        return REG_ERR_INVALID_ARG;
    if (desc->loss_kind != REG_LOSS_LNCC && desc->loss_kind != REG_LOSS_MI) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(grad_affine));
    REG_TRY(check_ptr(sim));
    REG_TRY(check_ptr(state));
    REG_TRY(check_ptr(T_dev));
    REG_TRY(check_opt_ptr(obj_out));
    AffineAdam P;
    P.lr_A = desc->lr_A;
    P.lr_t = desc->lr_t;
    P.b1 = desc->beta1;
    P.b2 = desc->beta2;
    P.eps = desc->eps;
    P.scale = desc->scale;
    for (int i = 0; i < 3; ++i) P.c[i] = desc->centre[i];
    P.bc1 = 1.0 - pow(desc->beta1, (double)(k + 1));
    P.bc2 = 1.0 - pow(desc->beta2, (double)(k + 1));
    P.decay = 1.0 - (1.0 - desc->final_lr) * (double)k / (double)(desc->iters > 1 ? desc->iters - 1 : 1);
    P.lncc = desc->loss_kind == REG_LOSS_LNCC;
    return cuda_status(launch_affine_adam(grad_affine, sim, state, T_dev, P, obj_out, (cudaStream_t)stream));
}

reg_status reg_compose_fields(const float *a, const float *b, reg_dims d, int pad, float *w, void *stream) {
    REG_TRY(check_dims(d));
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(a));
    REG_TRY(check_ptr(b));
    REG_TRY(check_ptr(w));
    const Dims g = make_dims(d);
    if (overlap3(w, a, g.n) || overlap3(w, b, g.n)) return REG_ERR_INVALID_ARG;
    return cuda_status(launch_compose(a, b, g, pad, 1.0f, w, (cudaStream_t)stream));
}

reg_status reg_exp_field(const float *v, reg_dims d, int steps, int pad, float *tmp, float *out, float *saved,
                         void *stream) {
    REG_TRY(check_dims(d));
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    if (steps < 0 || steps > 30) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(v));
    REG_TRY(check_ptr(out));
    REG_TRY(check_opt_ptr(saved));
    if (!saved) REG_TRY(check_ptr(tmp));
    const Dims g = make_dims(d);
    if (overlap3(out, v, g.n)) return REG_ERR_INVALID_ARG;
    if (!saved && (overlap3(tmp, v, g.n) || overlap3(out, tmp, g.n))) return REG_ERR_INVALID_ARG;
    if (saved && steps > 1) {
        const uintptr_t s0 = (uintptr_t)saved, s1 = s0 + sizeof(float) * 3 * (size_t)g.n * (size_t)(steps - 1);
        for (const float *f : {v, (const float *)out}) {
            const uintptr_t f0 = (uintptr_t)f, f1 = f0 + sizeof(float) * 3 * (size_t)g.n;
            if (f0 < s1 && s0 < f1) return REG_ERR_INVALID_ARG;
        }
    }
    const cudaStream_t s = (cudaStream_t)stream;
    if (steps == 0)
        return cuda_status(cudaMemcpyAsync(out, v, sizeof(float) * 3 * (size_t)g.n, cudaMemcpyDeviceToDevice, s));
    // destination of step k (1-based): the last one is out; the others are the
    // saved slots, or a ping-pong with tmp chosen so that step `steps` lands in out
    auto dst_of = [&](int k) -> float * {
        if (k == steps) return out;
        if (saved) return saved + (size_t)(k - 1) * 3 * (size_t)g.n;
        return ((steps - k) % 2) ? tmp : out;
    };
    const float *src = v;
    for (int k = 1; k <= steps; ++k) {
        float *dst = dst_of(k);
        REG_CUDA(launch_compose(src, src, g, pad, k == 1 ? (float)ldexp(1.0, -steps) : 1.0f, dst, s));
        src = dst;
    }
    return REG_OK;
}

reg_status reg_compose_fields_backward(const float *a, const float *b, const float *gw, reg_dims d, int pad,
                                       float *ga, float *gb, void *stream) {
    REG_TRY(check_dims(d));
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(a));
    REG_TRY(check_ptr(b));
    REG_TRY(check_ptr(gw));
    REG_TRY(check_opt_ptr(ga));
    REG_TRY(check_ptr(gb));
    const Dims g = make_dims(d);
    if (!ga && a != b) return REG_ERR_INVALID_ARG;
    for (const float *f : {a, b, gw})
        if (overlap3(gb, f, g.n) || (ga && overlap3(ga, f, g.n))) return REG_ERR_INVALID_ARG;
    if (ga && overlap3(ga, gb, g.n)) return REG_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    REG_CUDA(cudaMemsetAsync(gb, 0, sizeof(float) * 3 * (size_t)g.n, s));
    return cuda_status(launch_compose_backward(a, b, gw, g, pad, 1.0f, ga, gb, s));
}

reg_status reg_exp_field_backward(const float *v, reg_dims d, int steps, int pad, const float *saved,
                                  const float *gout, float *tmp, float *gv, void *stream) {
    REG_TRY(check_dims(d));
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    if (steps < 0 || steps > 30) return REG_ERR_INVALID_ARG;
    REG_TRY(check_ptr(v));
    REG_TRY(check_ptr(gout));
    REG_TRY(check_ptr(tmp));
    REG_TRY(check_ptr(gv));
    if (steps > 1) REG_TRY(check_ptr(saved));
    const Dims g = make_dims(d);
    const float *outs[3] = {gout, tmp, gv};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (overlap3(outs[i], outs[j], g.n)) return REG_ERR_INVALID_ARG;
    if (overlap3(tmp, v, g.n) || overlap3(gv, v, g.n)) return REG_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * 3 * (size_t)g.n;
    if (steps == 0) return cuda_status(cudaMemcpyAsync(gv, gout, bytes, cudaMemcpyDeviceToDevice, s));
    // step k maps u_{k-1} to u_k; its adjoint (both terms, a = b = u_{k-1})
    // lands in gv for k = 1 and alternates with tmp before that
    const float *gsrc = gout;
    for (int k = steps; k >= 1; --k) {
        float *dst = (k % 2) ? gv : tmp;
        const float *uin = k == 1 ? v : saved + (size_t)(k - 2) * 3 * (size_t)g.n;
        REG_CUDA(cudaMemsetAsync(dst, 0, bytes, s));
        REG_CUDA(launch_compose_backward(uin, uin, gsrc, g, pad, k == 1 ? (float)ldexp(1.0, -steps) : 1.0f,
                                         nullptr, dst, s));
        gsrc = dst;
    }
    return REG_OK;
}

reg_status reg_smooth_field(const float *u, reg_dims d, float sigma, float *tmp, float *out, void *stream) {
    REG_TRY(check_dims(d));
    REG_TRY(check_ptr(u));
    REG_TRY(check_ptr(tmp));
    REG_TRY(check_ptr(out));
    if (!(sigma > 0.0f) || !(sigma <= 7.9f)) return REG_ERR_INVALID_ARG;
    if (u == tmp || u == out || tmp == out) return REG_ERR_INVALID_ARG;
    return cuda_status(launch_smooth_field(u, make_dims(d), sigma, tmp, out, (cudaStream_t)stream));
}

reg_status reg_downsample2(const void *in, int dt, reg_dims d, void *out, void *stream) {
    REG_TRY(check_dims(d));
    REG_TRY(check_ptr(in));
    REG_TRY(check_ptr(out));
    if (dt != REG_F32 && dt != REG_BF16) return REG_ERR_DTYPE;
    if (d.nx % 2 || d.ny % 2 || d.nz % 2) return REG_ERR_SHAPE;
    if (in == out) return REG_ERR_INVALID_ARG;
    return cuda_status(launch_downsample2(in, dt, make_dims(d), out, (cudaStream_t)stream));
}

reg_status reg_debug_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int a_mn_major,
                               int b_mn_major, void *stream) {
    REG_TRY(check_ptr(A));
    REG_TRY(check_ptr(B));
    REG_TRY(check_ptr(C));
    if (M <= 0 || M % 128 || N < 16 || N > 128 || N % 16 || K <= 0 || K % 64) return REG_ERR_SHAPE;
    if ((a_mn_major & ~1) || (b_mn_major & ~1)) return REG_ERR_INVALID_ARG;
    return cuda_status(launch_gemm_test(A, B, C, M, N, K, a_mn_major, b_mn_major, (cudaStream_t)stream));
}

reg_status reg_set_timing_events(void *const *events, int n) {
    if (n == 0 && events == nullptr) {
        t_events_armed = false;
        return REG_OK;
    }
    if (n < 3 || n % 3 || n > 3 * (1 << 20) || !events) return REG_ERR_INVALID_ARG;
    t_events.assign((cudaEvent_t *)events, (cudaEvent_t *)events + n);
    t_base = 0;
    t_events_armed = true;
    return REG_OK;
}

reg_status reg_jacdet_min(const float *u, reg_dims d, void *ws, size_t ws_bytes, float *min_out,
                          unsigned long long *nfold_out, void *stream) {
    REG_TRY(check_dims(d));
    REG_TRY(check_ptr(u));
    REG_TRY(check_ptr(min_out));
    REG_TRY(check_ptr(nfold_out));
    (void)ws;
    (void)ws_bytes;
    return cuda_status(launch_jacdet(u, make_dims(d), min_out, nfold_out, (cudaStream_t)stream));
}

reg_status reg_get_device_error(void *stream) {
    REG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned *word = error_word();
    if (!word) return REG_ERR_CUDA;
    unsigned v = 0;
    REG_CUDA(cudaMemcpy(&v, word, sizeof(v), cudaMemcpyDeviceToHost));
    REG_CUDA(cudaMemset(word, 0, sizeof(v)));
    if (v == REG_ERR_NONFINITE || v == REG_ERR_TIMEOUT) return (reg_status)v;
    return v == 0 ? REG_OK : REG_ERR_CUDA;
}

reg_status reg_debug_wait_flag(const unsigned *flag, unsigned expect, unsigned long long timeout_ns, void *stream) {
    REG_TRY(check_ptr(flag));
    if (timeout_ns > 10ull * 1000000000ull) return REG_ERR_INVALID_ARG;
    return cuda_status(launch_wait_flag(flag, expect, timeout_ns, (cudaStream_t)stream));
}

}  // extern "C"
