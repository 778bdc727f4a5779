// kernels.h -- host-side launchers of the sm_103a kernels (internal; the
// public boundary is include/reg.h, implemented in capi.cu).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "reg_common.cuh"
#include "step_common.cuh"

namespace regk {

// compile-time dispatch helpers for the launchers: the padding mode, the
// image storage type and the moment storage type become template arguments
template <int V>
using IC = std::integral_constant<int, V>;
template <typename Fn>
inline void with_pad(int pad, Fn &&fn) {
    if (pad == REG_PAD_ZEROS)
        fn(IC<REG_PAD_ZEROS>{});
    else
        fn(IC<REG_PAD_BORDER>{});
}
template <typename Fn>
inline void with_type(int dt, Fn &&fn) {  // fn receives a null pointer of the element type
    if (dt == REG_BF16)
        fn((__nv_bfloat16 *)nullptr);
    else
        fn((float *)nullptr);
}
template <typename P>
using elem_t = std::remove_pointer_t<P>;
// voxel index type: 32-bit offsets within a channel when the volume has
// fewer than 2^31 voxels (cheaper address arithmetic), 64-bit otherwise
template <typename Fn>
inline void with_index(const Dims &g, Fn &&fn) {
    if (g.n < (1LL << 31))
        fn((int *)nullptr);
    else
        fn((long long *)nullptr);
}

// Tile-march geometry shared by every stencil / sweep kernel: a CTA owns a
// 32 x 8 column tile in (x, y) and marches through a chunk of z-planes.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int TILE_THREADS = TX * TY;
constexpr int MAX_BINS = 64;
constexpr int MAX_RADIUS = 7;  // LNCC window <= 15
// MI histogram fixed point: one unit of kernel weight = 2^20 counts.  One
// shared copy of a CTA's 32-bit bins takes at most MI_MAX_COPY_VOXELS
// voxels before it is added to the global 64-bit histogram, each voxel at
// most (2/3)^2 of a unit per bin: 8192 * 0.445 * 2^20 < 2^32, so a bin
// cannot wrap.
constexpr float MI_FIXED_SCALE = 1048576.0f;
constexpr int MI_MAX_COPY_VOXELS = 8192;

struct MarchGrid {
    int tiles_x, tiles_y, chunks, zc;
    long long blocks() const { return (long long)tiles_x * tiles_y * chunks; }
};

// target_blocks: roughly how many CTAs to aim for; min_zc / max_zc: bounds
// on the z-chunk (max_zc wins)
MarchGrid march_grid(const Dims &g, long long target_blocks, int min_zc, int max_zc = 1 << 30);

// Gaussian smoothing weights: radius r = floor(4 sigma + 1/2) <= SMOOTH_MAX_R
constexpr int SMOOTH_MAX_R = 32;
struct SmoothWeights {
    int r;
    float w[2 * SMOOTH_MAX_R + 1];
};
cudaError_t launch_smooth_field(const float *u, const Dims &g, float sigma, float *tmp, float *out, cudaStream_t s);
cudaError_t launch_downsample2(const void *in, int dt, const Dims &gi, void *out, cudaStream_t s);

struct MiParams {
    float f_lo, f_scale, m_lo, m_scale;  // vhat = clamp((v - lo) * scale, 0, 1)
    int bins;
    int hard;  // 1: hard-binned counts, convolved with the kernel in the finalisation
};

struct LnccParams {
    int r;      // window radius, window = 2r + 1
    float eps;  // added to B C
    int ants;   // 1: gradient with the ANTs approximation (no second box sum)
};

// per-kernel grids (used both to launch and to size the workspace)
MarchGrid mi_sweep_grid(const Dims &g);
// LNCC window-march grid for a kernel with per_sm CTAs resident per SM, and
// the most blocks it can have for any residency (workspace sizing)
constexpr int LNCC_MAX_PER_SM = 8;  // 2048 threads / 256
MarchGrid lncc_grid(const Dims &g, int r, int per_sm);
long long lncc_max_blocks(const Dims &g);
MarchGrid lncc_ants_grid(const Dims &g);
MarchGrid diffusion_grid(const Dims &g);

// aff: the composite transform phi = A p + t + S u (u may then be NULL);
// NULL is the plain deformable warp
cudaError_t launch_warp(const void *M, int dt, const float *u, const Dims &g, int pad, float *J, float *dJ,
                        cudaStream_t s, const AffineT *aff = nullptr);
// Field composition w = s a + s b o (id + s a) (w must not alias a or b)
cudaError_t launch_compose(const float *a, const float *b, const Dims &g, int pad, float scale, float *w,
                           cudaStream_t s);
// Adjoint of the composition: ga (written; NULL when a == b, gb then gets
// the whole gradient) and gb (accumulated with atomics: zero it first)
cudaError_t launch_compose_backward(const float *a, const float *b, const float *gw, const Dims &g, int pad,
                                    float scale, float *ga, float *gb, cudaStream_t s);
// Composite sampler backward: g_u = S gX (optional), out[12] = dL/dA
// (row-major), dL/dt; partials: 12 doubles per block of mi_sweep_grid(g)
cudaError_t launch_composite_backward(const void *M, int dt, const float *u, const Dims &g, int pad,
                                      const AffineT &A, const float *gin, float *g_u, double *partials,
                                      unsigned *counter, double *out, cudaStream_t s);

cudaError_t launch_mi_hist(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                           const MiParams &P, unsigned long long *hist, cudaStream_t s,
                           const AffineT *aff = nullptr);
// The MI adjoint table region: G' (B x B floats, row = fixed-image bin),
// then the same table as 4-wide rows, G4[m][n] = G'[m][n .. n+3] (B x B
// float4, zero past the last bin), which the second sweep copies into shared
// memory with 16-byte loads.
constexpr size_t MI_TABLE_BYTES = (sizeof(float) + sizeof(float4)) * MAX_BINS * MAX_BINS;
__host__ __device__ inline const float4 *mi_table4(const float *Gtab) {
    return reinterpret_cast<const float4 *>(Gtab + MAX_BINS * MAX_BINS);
}
cudaError_t launch_mi_finalize(const unsigned long long *hist, const MiParams &P, long long N, float *Gtab,
                               double *sim_out, cudaStream_t s);
// Second MI sweep: adjoint (+ optional diffusion + Adam).  With aff (the
// composite transform): without the step (u and grad_out may be NULL)
// grad_out = S gX and r_out[12] = dC/dA, dC/dt from 12 partials per block;
// with it, dC/du = S gX feeds the diffusion + Adam update of u.
cudaError_t launch_mi_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                             const MiParams &P, const float *Gtab, float *grad_out, bool step, float *u_out,
                             void *m, void *v, int mdt, const StepParams &S, double *partials,
                             unsigned *counter, double *r_out, cudaStream_t s, const AffineT *aff = nullptr);
// The TMA-staged form of the plain second sweep (mi_tma.cu), used by
// launch_mi_sweep2 when mi_tma_ok(g) and there is no composite transform;
// cudaErrorNotSupported if a tensor map cannot be built or its rings do not
// fit a CTA's shared memory (the caller then runs the plain kernel).  Its
// tiles are 64 x ty voxels (ty = 31 or 20, by what fits); its grid has
// mi_tma_sweep_grid(g, ty).blocks() CTAs (one partial each), at most
// mi_tma_max_blocks(g).
bool mi_tma_ok(const Dims &g);
MarchGrid mi_tma_sweep_grid(const Dims &g, int ty);
long long mi_tma_max_blocks(const Dims &g);
cudaError_t launch_mi_sweep2_tma(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                                 const MiParams &P, const float *Gtab, float *grad_out, bool step, float *u_out,
                                 void *m, void *v, int mdt, const StepParams &S, double *partials,
                                 unsigned *counter, double *r_out, cudaStream_t s);

// First LNCC sweep: window statistics of F and the warped image J (already
// in HBM, FP32) -> similarity (+ optional adjoint coefficient fields, [3][N]).
// fstat (optional): F's window mean and variance ([2][N]) from
// launch_lncc_fstats, so that only the three sums involving J are formed
cudaError_t launch_lncc_stats(const void *F, const float *J, int dt, const Dims &g, const LnccParams &P, float *coef,
                              double *partials, unsigned *counter, double *sim_out, cudaStream_t s,
                              const float *fstat = nullptr);
// F's window mean and variance (fstat [2][N]): F is fixed during a
// registration, so a run of iterations forms them once
cudaError_t launch_lncc_fstats(const void *F, int dt, const Dims &g, const LnccParams &P, float *fstat,
                               cudaStream_t s);
// Second LNCC sweep: box sums of the coefficient fields -> adjoint (+ optional
// diffusion + Adam).  aff as for launch_mi_sweep2.
cudaError_t launch_lncc_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                               const LnccParams &P, const float *coef, float *grad_out, bool step,
                               float *u_out, void *m, void *v, int mdt, const StepParams &S,
                               double *partials, unsigned *counter, double *r_out, cudaStream_t s,
                               const AffineT *aff = nullptr);

// One Adam step on the 12 parameters of an affine map about a centre,
// phi(p) = A (p - c) + c + tc / s, on one device thread (reg_affine_adam_step)
struct AffineAdam {
    double lr_A, lr_t, b1, b2, eps, scale, c[3];
    double bc1, bc2, decay;  // bias corrections 1 - beta^(k+1) and the step's decay factor
    int lncc;                // the objective recorded: 1 - S (LNCC) or -MI
};
cudaError_t launch_affine_adam(const double *grad_affine, const double *sim, double *state, float *T_dev,
                               const AffineAdam &P, double *obj_out, cudaStream_t s);

cudaError_t launch_diffusion(const float *u, const Dims &g, float lam, float *grad, double *partials,
                             unsigned *counter, double *r_out, cudaStream_t s);
cudaError_t launch_adam(const float *u_in, float *u_out, void *m, void *v, int mdt, const float *grad,
                        long long n3, const StepParams &S, cudaStream_t s);
cudaError_t launch_jacdet(const float *u, const Dims &g, float *min_out, unsigned long long *nfold,
                          cudaStream_t s);
cudaError_t launch_wait_flag(const unsigned *flag, unsigned expect, unsigned long long timeout_ns,
                             cudaStream_t s);

// tensor-core GEMM test hook (C = A B^T, BF16 in, FP32 out)
cudaError_t launch_gemm_test(const void *A, const void *B, float *C, int M, int N, int K, int a_mn, int b_mn,
                             cudaStream_t s);

int num_sms();
// device address of the device error word on the current device
unsigned *error_word();

}  // namespace regk

// ---- learned initialiser (unet.cu, unet_ops.cu) -------------------------------
namespace regk {
size_t gemm_smem_bytes();
// convolution epilogues: LeakyReLU(acc + bias) -> BF16, acc -> BF16, acc + bias -> FP32 SoA
enum ConvEpi { EPI_BIAS_LEAKY_BF16 = 0, EPI_PLAIN_BF16 = 1, EPI_BIAS_F32_SOA = 2 };
// TMA-fed convolution (Cin % 16 == 0, nx <= 254): weights re-tiled into
// Wt_scratch (conv_view_weight_bytes); cudaErrorNotSupported if the shape
// has no such path
size_t conv_view_weight_bytes(int Cin, int N);
// TMA-fed weight gradient (Cin % 16 == 0, Cout % 8 == 0, Cout <= 128, nx <= 254): per-CTA
// partials in `part` (conv_wgrad_view_bytes, 0 if the shape has no such path)
size_t conv_wgrad_view_bytes(const Dims &d, int Cin, int Cout);
cudaError_t launch_conv_wgrad_view(const void *in, int Cin, const void *dpre, int Cout, const Dims &d, float *part,
                                   float *dW, int Kpad, cudaStream_t s);
cudaError_t launch_conv_view(const void *in, int Cin, const void *W, int rows, int Kpad, const float *bias, int Cout,
                             int N, const Dims &d, int epi, float slope, void *Wt_scratch, void *out, cudaStream_t s);
cudaError_t launch_conv_fwd(const void *in, int Cin, const void *W, int Kpad, const float *bias, int Cout, int N,
                            const Dims &d, int epi, float slope, void *out, cudaStream_t s);
cudaError_t launch_conv_wgrad(const void *in, int Cin, const void *dpre, int Cout, const Dims &d, float *part,
                              float *dW, int Kpad, cudaStream_t s);
size_t wgrad_part_bytes(const Dims &d, int Cin, int Cout);
cudaError_t launch_repack_dgrad(const void *W, int Cout, int Cin, int Kpad, void *Wd, int Nd, int Kpad_d,
                                cudaStream_t s);
cudaError_t launch_pack_pair(const void *F, const void *M, int dt, const Dims &gin, int factor, float f_lo,
                             float f_scale, float m_lo, float m_scale, void *out, cudaStream_t s);
cudaError_t launch_leaky_bwd(const void *out, const void *dout, long long n, float slope, void *dpre, cudaStream_t s);
int bias_grad_blocks();
cudaError_t launch_bias_grad(const void *dpre, long long V, int C, double *part, float *dbias, cudaStream_t s);
cudaError_t launch_avgpool2(const void *in, int C, const Dims &gi, void *out, cudaStream_t s);
cudaError_t launch_avgpool2_bwd(const void *dout, int C, const Dims &gi, void *din, cudaStream_t s);
cudaError_t launch_upsample2(const void *in, int C, const Dims &gc, void *out, cudaStream_t s);
cudaError_t launch_upsample2_bwd(const void *dout, int C, const Dims &gc, void *din, cudaStream_t s);
cudaError_t launch_put_channels(const void *src, int Csrc, long long V, void *dst, int Cdst, int c0, int acc,
                                cudaStream_t s);
cudaError_t launch_take_channels(const void *src, int Csrc, int c0, long long V, void *dst, int Cdst, int acc,
                                 cudaStream_t s);
int mse_blocks();
cudaError_t launch_mse(const float *pred, const float *tgt, long long V, int Cpad, void *dpred, double *part,
                       double *loss, cudaStream_t s);
cudaError_t launch_field_down2(const float *u, const Dims &gf, float *out, cudaStream_t s);
cudaError_t launch_field_up(const float *u, const Dims &gc, int factor, float *out, cudaStream_t s);
cudaError_t launch_adam_weights(float *w, float *m, float *v, const float *g, long long n, const StepParams &S,
                                void *w_bf16, cudaStream_t s);
}  // namespace regk
