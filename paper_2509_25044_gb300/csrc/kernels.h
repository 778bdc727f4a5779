// kernels.h -- host-side launchers of the sm_103a kernels (internal; the
// public boundary is include/reg.h, implemented in capi.cu).
#pragma once

#include <cuda_runtime.h>

#include "reg_common.cuh"
#include "step_common.cuh"

namespace regk {

// Tile-march geometry shared by every stencil / sweep kernel: a CTA owns a
// 32 x 8 column tile in (x, y) and marches through a chunk of z-planes.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int TILE_THREADS = TX * TY;
constexpr int MAX_BINS = 64;
constexpr int MAX_RADIUS = 7;  // LNCC window <= 15

struct MarchGrid {
    int tiles_x, tiles_y, chunks, zc;
    long long blocks() const { return (long long)tiles_x * tiles_y * chunks; }
};

// target_blocks: roughly how many CTAs to aim for; min_zc: smallest chunk
MarchGrid march_grid(const Dims &g, long long target_blocks, int min_zc);

struct MiParams {
    float f_lo, f_scale, m_lo, m_scale;  // vhat = clamp((v - lo) * scale, 0, 1)
    int bins;
};

struct LnccParams {
    int r;      // window radius, window = 2r + 1
    float eps;  // added to B C
};

// per-kernel grids (used both to launch and to size the workspace)
MarchGrid mi_hist_grid(const Dims &g);
MarchGrid mi_sweep_grid(const Dims &g);
MarchGrid lncc_grid(const Dims &g, int r);
MarchGrid diffusion_grid(const Dims &g);

cudaError_t launch_warp(const void *M, int dt, const float *u, const Dims &g, int pad, float *J, float *dJ,
                        cudaStream_t s);

cudaError_t launch_mi_hist(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                           const MiParams &P, unsigned long long *hist, cudaStream_t s);
cudaError_t launch_mi_finalize(const unsigned long long *hist, const MiParams &P, long long N, float *Gtab,
                               double *sim_out, cudaStream_t s);
// Second MI sweep: adjoint (+ optional diffusion + Adam).
cudaError_t launch_mi_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                             const MiParams &P, const float *Gtab, float *grad_out, bool step, float *u_out,
                             void *m, void *v, int mdt, const StepParams &S, double *partials,
                             unsigned *counter, double *r_out, cudaStream_t s);

// First LNCC sweep: window statistics -> similarity (+ optional adjoint
// coefficient fields, [3][N] floats).
cudaError_t launch_lncc_stats(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                              const LnccParams &P, float *coef, double *partials, unsigned *counter,
                              double *sim_out, cudaStream_t s);
// Second LNCC sweep: box sums of the coefficient fields -> adjoint (+ optional
// diffusion + Adam).
cudaError_t launch_lncc_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                               const LnccParams &P, const float *coef, float *grad_out, bool step,
                               float *u_out, void *m, void *v, int mdt, const StepParams &S,
                               double *partials, unsigned *counter, double *r_out, cudaStream_t s);

cudaError_t launch_diffusion(const float *u, const Dims &g, float lam, float *grad, double *partials,
                             unsigned *counter, double *r_out, cudaStream_t s);
cudaError_t launch_adam(const float *u_in, float *u_out, void *m, void *v, int mdt, const float *grad,
                        long long n3, const StepParams &S, cudaStream_t s);
cudaError_t launch_jacdet(const float *u, const Dims &g, float *min_out, unsigned long long *nfold,
                          cudaStream_t s);
cudaError_t launch_wait_flag(const unsigned *flag, unsigned expect, unsigned long long timeout_ns,
                             cudaStream_t s);

int num_sms();
// device address of the device error word on the current device
unsigned *error_word();

}  // namespace regk
