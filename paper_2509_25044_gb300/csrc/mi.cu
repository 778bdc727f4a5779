// mi.cu -- Parzen-window mutual information (Sec. 2.2, Eq. mi; App. fused
// MI) on sm_103a, in two sweeps plus a one-block finalisation:
//
//   sweep 1 (mi_hist_kernel): warp M on chip, map F and the warped value to
//     bin coordinates, add the 4 x 4 cubic B-spline outer product of each
//     voxel into a per-CTA joint histogram in shared memory.  Entries are
//     unsigned fixed point (2^-20 per unit weight: 32-bit per CTA, 64-bit
//     global), so the sums are exact integers and the histogram does not
//     depend on the order of the atomics (deterministic).  Each CTA then adds
//     its non-zero bins to the global histogram (integer atomics, order-
//     free).  No N x B Parzen block is ever materialised (the memory the
//     paper removes).
//   finalise (mi_finalize_kernel): p = hist / (2^20 N) in FP64, marginals
//     as row / column sums, the log ratios in FP32, MI = sum p log(p / (pI
//     pJ)) accumulated in FP64, and the FP32 table
//     G'[m][n] = -(B-3) m_scale / N * log(p / (pI pJ)) of the adjoint.
//   sweep 2 (mi_sweep2_kernel): warp again with slope, the adjoint
//     dL/dJ = sum_{a,b} G'[mF+a][nJ+b] w_a(sF) w'_b(sJ) (Eq. gradientmi-
//     threadn with the 16 non-zero kernel terms), chained through the
//     sampler slope; optionally fused with the diffusion gradient and Adam.
#include <algorithm>

#include "kernels.h"
#include "mi_common.cuh"

namespace regk {

constexpr int HIST_TX = 32;
// Two CTA shapes.  BF16 images with the workloads' 32 bins compiled in:
// 32 x 24 columns, 768 threads at 40 registers and 24 copies of 4 KB (lanes
// 0-7 share theirs with lanes 24-31, the voxels x and x + 24 of a row), two
// CTAs per SM, so 48 warps cover the corner gathers' latency where one
// 1024-thread CTA holding 32 copies gives 32.  Otherwise: 32 x 32 columns,
// 1024 threads at 64 registers, hist_copies(B) copies, one CTA per SM (FP32
// images gather twice the bytes, and the two CTAs' copies leave too little
// L1 for them).
template <int BT, typename T>
struct HistShape {
    static constexpr bool pair = BT == 32 && sizeof(T) == 2;
    static constexpr int ty = pair ? 24 : 32;  // rows = warps
    static constexpr int threads = HIST_TX * ty;
    static constexpr int per_sm = pair ? 2 : 1;
};
__host__ __device__ constexpr int hist_copies_of(int B, bool pair) { return pair ? 24 : hist_copies(B); }
// A copy serves at most ceil(32 / copies) lanes of each of the `warps`
// warps, one voxel per lane and plane, so after this many planes a CTA adds
// its copies to the global histogram and clears them (MI_MAX_COPY_VOXELS
// keeps the 32-bit bins from wrapping).
__host__ __device__ constexpr int hist_batch_planes(int copies, int warps) {
    return MI_MAX_COPY_VOXELS / (warps * ((32 + copies - 1) / copies));
}

// Persistent CTAs (HistShape::per_sm per SM): the volume is cut into 32 x ty
// columns, the (column, plane) pairs are numbered column-major and each CTA
// takes one contiguous range of them, so the work is balanced to within one
// plane.
// Each thread marches its (x, y) column through the planes of its range,
// with F and u of the next plane requested before the current plane is
// computed, and adds the 16 fixed-point products of its voxel's B-spline
// weights to its copy (hist_add_parzen).
// BT > 0: the bin count compiled in (the bin and copy address arithmetic folds
// to constants); BT = 0: P.bins.
template <typename T, int PAD, typename I, bool HARD, bool AFF, int BT = 0>
__global__ void __launch_bounds__(HistShape<BT, T>::threads, HistShape<BT, T>::per_sm)
    mi_hist_kernel(const T *__restrict__ F, const T *__restrict__ M, const float *__restrict__ u, Dims g, MiParams P,
                   int tiles_x, long long total, AffineT Ain, unsigned long long *__restrict__ hist) {
    extern __shared__ unsigned sh[];
    const AffineT A = AFF ? resolve_affine(Ain) : Ain;
    using Sh = HistShape<BT, T>;
    const int B = BT > 0 ? BT : P.bins, BB = B * B;
    const int copies = hist_copies_of(B, Sh::pair), pitch = BB + 1;
    const int tid = threadIdx.y * HIST_TX + threadIdx.x;
    for (int i = tid; i < copies * pitch; i += Sh::threads) sh[i] = 0u;
    __syncthreads();
    unsigned *shc = sh + (threadIdx.x % copies) * pitch;
    const float *u0 = u, *u1 = u + g.n, *u2 = u + 2 * g.n;
    const bool has_u = !AFF || u != nullptr;  // the composite form may omit u
    const I nxy = (I)g.nxy;
    const long long beg = total * blockIdx.x / gridDim.x, end = total * (blockIdx.x + 1) / gridDim.x;
    const int batch = hist_batch_planes(copies, Sh::ty);
    for (long long b0 = beg; b0 < end; b0 += batch) {
        const long long b1 = min(end, b0 + batch);
        for (long long pos = b0; pos < b1;) {
            const long long tile = pos / g.nz;
            const int z0 = (int)(pos - tile * g.nz);
            const int z1 = (int)min((long long)g.nz, (long long)z0 + (b1 - pos));
            pos += z1 - z0;
            const int x = (int)(tile % tiles_x) * HIST_TX + threadIdx.x;
            const int y = (int)(tile / tiles_x) * Sh::ty + threadIdx.y;
            if (x >= g.nx || y >= g.ny) continue;
            I p = (I)z0 * nxy + (I)y * g.nx + x;
            float fv = ld_vox_cs(F, p), ux = 0.0f, uy = 0.0f, uz = 0.0f;
            if (has_u) {
                ux = __ldcs(u0 + p);
                uy = __ldcs(u1 + p);
                uz = __ldcs(u2 + p);
            }
            for (int z = z0; z < z1; ++z, p += nxy) {
                float fn = 0.0f, nx0 = 0.0f, nx1 = 0.0f, nx2 = 0.0f;
                if (z + 1 < z1) {
                    fn = ld_vox_cs(F, p + nxy);
                    if (has_u) {
                        nx0 = __ldcs(u0 + p + nxy);
                        nx1 = __ldcs(u1 + p + nxy);
                        nx2 = __ldcs(u2 + p + nxy);
                    }
                }
                float qx = ux, qy = uy, qz = uz;
                if (AFF) composite_disp(A, x, y, z, qx, qy, qz);
                const float jv = sample<T, PAD, I>(M, g, x, y, z, qx, qy, qz);
                if (HARD) {
                    // one count at the nearest bins; the kernel is applied to
                    // the B x B counts in the finalisation
                    const int mF = nearest_bin(to_bin(fv, P.f_lo, P.f_scale, B), B);
                    const int mJ = nearest_bin(to_bin(jv, P.m_lo, P.m_scale, B), B);
                    atomicAdd(shc + mF * B + mJ, 1u);
                } else {
                    hist_add_parzen(shc, B, to_bin(fv, P.f_lo, P.f_scale, B), to_bin(jv, P.m_lo, P.m_scale, B));
                }
                fv = fn;
                ux = nx0;
                uy = nx1;
                uz = nx2;
            }
        }
        __syncthreads();
        for (int i = tid; i < BB; i += Sh::threads) {
            unsigned long long v = 0;
            for (int c = 0; c < copies; ++c) {
                v += sh[c * pitch + i];
                sh[c * pitch + i] = 0u;
            }
            if (v) atomicAdd(hist + i, v);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) mi_finalize_kernel(const unsigned long long *__restrict__ hist, int B,
                                                           int hard, double inv_total, double gscale,
                                                           float *__restrict__ Gtab, double *__restrict__ sim_out,
                                                           unsigned *err) {
    __shared__ double p[MAX_BINS * MAX_BINS];
    __shared__ double pI[MAX_BINS], pJ[MAX_BINS];
    __shared__ double red[32];
    const int BB = B * B;
    if (!hard) {
        for (int e = threadIdx.x; e < BB; e += blockDim.x) p[e] = (double)hist[e] * inv_total;
    } else {
        // counts at the nearest bins convolved with kappa(a) kappa(b), a, b in {-1, 0, 1}
        const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
        for (int e = threadIdx.x; e < BB; e += blockDim.x) {
            const int m = e / B, n = e % B;
            double acc = 0.0;
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b) {
                    const int mm = m - a, nn = n - b;
                    if (mm < 0 || mm >= B || nn < 0 || nn >= B) continue;
                    acc += w[a + 1] * w[b + 1] * (double)hist[mm * B + nn];
                }
            p[e] = acc * inv_total;
        }
    }
    __syncthreads();
    if (threadIdx.x < B) {
        double s = 0.0;
        for (int n = 0; n < B; ++n) s += p[threadIdx.x * B + n];
        pI[threadIdx.x] = s;
    } else if (threadIdx.x >= 64 && threadIdx.x < 64 + B) {
        const int n = threadIdx.x - 64;
        double s = 0.0;
        for (int m = 0; m < B; ++m) s += p[m * B + n];
        pJ[n] = s;
    }
    __syncthreads();
    // the per-bin log ratio in FP32 (GB300's FP64 rate is a small fraction of
    // its FP32 rate and this block runs on one SM); the MI sum stays in FP64
    double acc = 0.0;
    for (int e = threadIdx.x; e < BB; e += blockDim.x) {
        const double v = p[e];
        float gv = 0.0f;
        if (v > 0.0) {
            const float lr = logf((float)v / (float)(pI[e / B] * pJ[e % B]));
            acc = fma(v, (double)lr, acc);
            gv = (float)gscale * lr;
        }
        Gtab[e] = gv;
    }
    const double mi = block_sum(acc, red);  // (its barriers publish the G' writes above)
    if (threadIdx.x == 0) {
        if (!isfinite(mi)) latch_error(err, REG_ERR_NONFINITE);
        sim_out[0] = mi;
    }
    // the 4-wide rows the second sweep loads: G4[m][n] = G'[m][n .. n+3]
    float4 *G4 = reinterpret_cast<float4 *>(Gtab + MAX_BINS * MAX_BINS);
    for (int e = threadIdx.x; e < BB; e += blockDim.x) {
        const int n = e % B;
        G4[e] = make_float4(Gtab[e], n + 1 < B ? Gtab[e + 1] : 0.0f, n + 2 < B ? Gtab[e + 2] : 0.0f,
                            n + 3 < B ? Gtab[e + 3] : 0.0f);
    }
}

// AFF: the composite transform phi = A p + t + S u.  Without STEP (u and
// grad_out may be NULL): grad_out = S gX and r_out[12] = dC/dA, dC/dt.  With
// STEP: dC/du = S gX enters the diffusion + Adam update of u as usual.
template <typename T, typename MT, bool STEP, int PAD, typename I, bool AFF = false>
__global__ void __launch_bounds__(TILE_THREADS, 4)
    mi_sweep2_kernel(const T *__restrict__ F, const T *__restrict__ M, const float *__restrict__ u, Dims g,
                     MiParams P, int zc, const float *__restrict__ Gtab, float *__restrict__ grad_out,
                     float *__restrict__ u_out, MT *__restrict__ m, MT *__restrict__ v, StepParams S,
                     double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ r_out,
                     unsigned *err, AffineT Ain) {
    const AffineT A = AFF ? resolve_affine(Ain) : Ain;
    // G4[m][n] = G'[m][n .. n+3]: one 16-byte shared load per kernel row
    extern __shared__ float4 G4[];  // B * B entries (dynamic)
    __shared__ double red[32];
    const int B = P.bins, BB = B * B;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const float4 *T4 = mi_table4(Gtab);  // built by the finalisation
    for (int i = tid; i < BB; i += TILE_THREADS) G4[i] = __ldg(T4 + i);
    __syncthreads();

    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(g.nz, z0 + zc);
    float rpart = 0.0f;
    AffineAcc aacc;
    const bool has_u = !AFF || u != nullptr;
    if (x < g.nx && y < g.ny) {
        // per-channel base pointers; voxel offsets within a channel are of type I
        const float *uc[3] = {u, u + g.n, u + 2 * g.n};
        MT *mc[3] = {m, m + g.n, m + 2 * g.n};
        MT *vc[3] = {v, v + g.n, v + 2 * g.n};
        const I nxy = (I)g.nxy, nx = (I)g.nx;
        I p = (I)z0 * nxy + (I)y * nx + x;
        const bool hxm = x > 0, hxp = x + 1 < g.nx, hym = y > 0, hyp = y + 1 < g.ny;
        // registers roll one plane ahead: u at z-1 / z / z+1, and F, m, v of
        // the next plane are requested before the current plane is computed
        float cur[3], prv[3] = {0.f, 0.f, 0.f}, nxt[3] = {0.f, 0.f, 0.f};
        float fcur, mcur[3] = {0.f, 0.f, 0.f}, vcur[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; ++c) cur[c] = has_u ? __ldg(uc[c] + p) : 0.0f;
        fcur = ld_vox(F, p);
        if (STEP) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                mcur[c] = ld_moment(mc[c], p);
                vcur[c] = ld_moment(vc[c], p);
                if (z0 > 0) prv[c] = __ldg(uc[c] + p - nxy);
            }
        }
        for (int z = z0; z < z1; ++z, p += nxy) {
            float fnxt = 0.0f, mnxt[3] = {0.f, 0.f, 0.f}, vnxt[3] = {0.f, 0.f, 0.f};
            if (z + 1 < g.nz && has_u) {
#pragma unroll
                for (int c = 0; c < 3; ++c) nxt[c] = __ldg(uc[c] + p + nxy);
            }
            if (z + 1 < z1) {
                fnxt = ld_vox(F, p + nxy);
                if (STEP) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        mnxt[c] = ld_moment(mc[c], p + nxy);
                        vnxt[c] = ld_moment(vc[c], p + nxy);
                    }
                }
            }
            float sx, sy, sz, qx = cur[0], qy = cur[1], qz = cur[2];
            if (AFF) composite_disp(A, x, y, z, qx, qy, qz);
            const float jv = sample_grad<T, PAD, I>(M, g, x, y, z, qx, qy, qz, sx, sy, sz);
            float wf[4], dj[4];
            const int iF = bspline_weights(to_bin(fcur, P.f_lo, P.f_scale, B), B, wf) - 1;
            const float tj = (jv - P.m_lo) * P.m_scale;
            const int iJ = bspline_dweights(to_bin(jv, P.m_lo, P.m_scale, B), B, dj) - 1;
            float gj = 0.0f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 r = G4[(iF + a) * B + iJ];
                const float t = fmaf(r.x, dj[0], fmaf(r.y, dj[1], fmaf(r.z, dj[2], r.w * dj[3])));
                gj = fmaf(wf[a], t, gj);
            }
            if (!(tj >= 0.0f && tj <= 1.0f)) gj = 0.0f;  // intensity clamp is flat
            const float gs[3] = {gj * sx, gj * sy, gj * sz};
            if (STEP) {
                float gR[3];
                diffusion_ptr<I>(uc, p, nx, hxm, hxp, hym, hyp, z > 0, z + 1 < g.nz, cur, prv, nxt, gR, rpart);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float gt = fmaf(S.lam * S.two_over_n, gR[c], AFF ? A.s[c] * gs[c] : gs[c]);
                    if (grad_out) (grad_out + c * g.n)[p] = gt;
                    (u_out + c * g.n)[p] = adam_fast(cur[c], gt, mcur[c], vcur[c], mc[c], vc[c], p, S);
                }
            } else if (AFF) {
                aacc.add(gs[0], gs[1], gs[2], z);
                if (grad_out) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) (grad_out + c * g.n)[p] = A.s[c] * gs[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) (grad_out + c * g.n)[p] = gs[c];
            }
            fcur = fnxt;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                prv[c] = cur[c];
                cur[c] = nxt[c];
                mcur[c] = mnxt[c];
                vcur[c] = vnxt[c];
            }
        }
    }
    if (AFF && !STEP) affine_reduce(aacc, x, y, partials, counter, r_out, red, err);
    if (STEP) {
        const double bs = block_sum((double)rpart, red);
        const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (tid == 0) partials[bid] = bs;
        if (arrive_last(counter)) {
            const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
            double acc = 0.0;
            // fixed order: thread t sums blocks t, t+256, ... then a fixed tree
            for (long long i = tid; i < nb; i += TILE_THREADS) acc += __ldcg(partials + i);
            const double tot = block_sum(acc, red);
            if (tid == 0) {
                const double R = tot / (double)g.n;
                if (!isfinite(R)) latch_error(err, REG_ERR_NONFINITE);
                r_out[0] = R;
                *counter = 0u;
            }
        }
    }
}

// about four waves of resident CTAs (4 per SM): at 192^3 that is 2304 CTAs of
// 12 planes, 1-2 % faster than twice as many CTAs of 6 planes (each CTA
// builds the 16 KiB adjoint table once); one wave leaves a tail
MarchGrid mi_sweep_grid(const Dims &g) { return march_grid(g, 16LL * num_sms(), 1); }

cudaError_t launch_mi_hist(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                           const MiParams &P, unsigned long long *hist, cudaStream_t s, const AffineT *aff) {
    // the shape of the instantiation dispatched below (the two-CTA shape for
    // the 32-bin non-composite forms on BF16 images)
    using Pair = HistShape<32, __nv_bfloat16>;
    using Single = HistShape<0, float>;
    const bool pair = !aff && P.bins == 32 && dt == REG_BF16;
    const int ty = pair ? Pair::ty : Single::ty;
    const int tiles_x = (g.nx + HIST_TX - 1) / HIST_TX, tiles_y = (g.ny + ty - 1) / ty;
    const long long total = (long long)tiles_x * tiles_y * g.nz;
    if (total <= 0) return cudaSuccess;
    const int per_sm = pair ? Pair::per_sm : Single::per_sm;
    const unsigned grid = (unsigned)std::min<long long>((long long)per_sm * num_sms(), total);
    const dim3 block(HIST_TX, ty);
    const size_t smem = sizeof(unsigned) * (size_t)hist_copies_of(P.bins, pair) * ((size_t)P.bins * P.bins + 1);
    const AffineT A = aff ? *aff : AffineT{};
    cudaError_t e = cudaSuccess;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            auto run = [&](auto kern) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess)
                    kern<<<grid, block, smem, s>>>((const T *)F, (const T *)M, u, g, P, tiles_x, total, A, hist);
            };
            if (aff) {  // the composite form: 64-bit offsets only
                if (P.hard)
                    run(mi_hist_kernel<T, PD, long long, true, true>);
                else
                    run(mi_hist_kernel<T, PD, long long, false, true>);
                return;
            }
            with_index(g, [&](auto ip) {
                using I = elem_t<decltype(ip)>;
                // the workloads' 32 bins compiled in
                if (P.bins == 32)
                    P.hard ? run(mi_hist_kernel<T, PD, I, true, false, 32>)
                           : run(mi_hist_kernel<T, PD, I, false, false, 32>);
                else if (P.hard)
                    run(mi_hist_kernel<T, PD, I, true, false>);
                else
                    run(mi_hist_kernel<T, PD, I, false, false>);
            });
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_mi_finalize(const unsigned long long *hist, const MiParams &P, long long N, float *Gtab,
                               double *sim_out, cudaStream_t s) {
    // Parzen bins hold fixed-point weight (MI_FIXED_SCALE per unit); hard bins hold counts
    const double inv_total = 1.0 / ((P.hard ? 1.0 : (double)MI_FIXED_SCALE) * (double)N);
    const double gscale = -(double)(P.bins - 3) * (double)P.m_scale / (double)N;
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    mi_finalize_kernel<<<1, 1024, 0, s>>>(hist, P.bins, P.hard, inv_total, gscale, Gtab, sim_out, err);
    return cudaGetLastError();
}

cudaError_t launch_mi_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                             const MiParams &P, const float *Gtab, float *grad_out, bool step, float *u_out,
                             void *m, void *v, int mdt, const StepParams &S, double *partials,
                             unsigned *counter, double *r_out, cudaStream_t s, const AffineT *aff) {
    // the TMA-staged form (mi_tma.cu), same arithmetic, where its tensor maps apply
    if (!aff && mi_tma_ok(g)) {
        const cudaError_t e = launch_mi_sweep2_tma(F, M, dt, u, g, pad, P, Gtab, grad_out, step, u_out, m, v, mdt,
                                                   S, partials, counter, r_out, s);
        if (e != cudaErrorNotSupported) return e;
    }
    const MarchGrid G = mi_sweep_grid(g);
    const AffineT A = aff ? *aff : AffineT{};
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    const size_t smem = sizeof(float4) * (size_t)P.bins * P.bins;
    cudaError_t e = cudaSuccess;
    // the G table exceeds the default 48 KiB of dynamic shared memory only for B > 55
    auto prepare = [&](auto kern) {
        if (smem > 48 * 1024 && e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e == cudaSuccess;
    };
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            if (aff && !step) {  // the composite form: gradients only, 64-bit offsets
                if (prepare(mi_sweep2_kernel<T, float, false, PD, long long, true>))
                    mi_sweep2_kernel<T, float, false, PD, long long, true><<<grid, block, smem, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, Gtab, grad_out, nullptr, nullptr, nullptr, S,
                        partials, counter, r_out, err, A);
                return;
            }
            if (aff) {  // the composite form with the step
                with_type(mdt, [&](auto mp) {
                    using MT = elem_t<decltype(mp)>;
                    if (prepare(mi_sweep2_kernel<T, MT, true, PD, long long, true>))
                        mi_sweep2_kernel<T, MT, true, PD, long long, true><<<grid, block, smem, s>>>(
                            (const T *)F, (const T *)M, u, g, P, G.zc, Gtab, grad_out, u_out, (MT *)m, (MT *)v, S,
                            partials, counter, r_out, err, A);
                });
                return;
            }
            with_index(g, [&](auto ip) {
                using I = elem_t<decltype(ip)>;
                if (!step) {
                    if (prepare(mi_sweep2_kernel<T, float, false, PD, I>))
                        mi_sweep2_kernel<T, float, false, PD, I><<<grid, block, smem, s>>>(
                            (const T *)F, (const T *)M, u, g, P, G.zc, Gtab, grad_out, u_out, (float *)m,
                            (float *)v, S, partials, counter, r_out, err, A);
                    return;
                }
                with_type(mdt, [&](auto mp) {
                    using MT = elem_t<decltype(mp)>;
                    if (prepare(mi_sweep2_kernel<T, MT, true, PD, I>))
                        mi_sweep2_kernel<T, MT, true, PD, I><<<grid, block, smem, s>>>(
                            (const T *)F, (const T *)M, u, g, P, G.zc, Gtab, grad_out, u_out, (MT *)m, (MT *)v, S,
                            partials, counter, r_out, err, A);
                });
            });
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace regk
