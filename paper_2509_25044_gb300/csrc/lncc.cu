// lncc.cu -- windowed LNCC (Sec. 2.3; App. fused LNCC, Eq. lncc-loss,
// Eqs. lncc-a..lncc-c) and its adjoint on sm_103a, in two sweeps.
//
// Both sweeps use the same 2.5-D tile march: a CTA owns a 32 x 8 column
// tile in (x, y) and walks a chunk of z-planes.  For every input plane it
// stages the tile plus an r-voxel halo in shared memory, box-sums along x
// (sliding sums over 8-voxel segments), then along y, and keeps the running
// z-sum of the last 2r+1 plane sums per column (a ring in shared memory).
// Nothing N-sized is stored between the window sums and the similarity.
//
// sweep 1 (lncc_stats_kernel): stages F and the warped image J = M o (id+u)
//   (recomputed on chip from M and u), with a per-CTA intensity shift (F and
//   M at the tile centre) so the FP32 variance sums do not cancel.  From the
//   five window sums it forms A, B, C, n_i = A^2 / (B C + eps) and adds n_i
//   into FP64 block partials (fixed-order final sum -> S = mean n_i).  For the
//   gradient it also writes the three per-window adjoint coefficients
//   (dL/dn_i = -1/N):
//     a_FJ = -(1/N) (2A/D) / c,   a_JJ = -(1/N) (-A^2 B / D^2) / c,
//     a_J  = -(a_FJ muF + 2 a_JJ muJ),
//   so that dL/dJ_k = sum_{i: k in W_i} (a_J + 2 J_k a_JJ + F_k a_FJ)_i,
//   the moving-image form of Eq. gradientcc-first (the printed A/(B^2 C)
//   read as A^2/(B^2 C)) with the window-sum derivatives taken directly.
// sweep 2 (lncc_sweep2_kernel): the second box sum of the three coefficient
//   fields (exact adjoint, not the ANTs shortcut), then dL/dJ, chained
//   through the sampler slope to dL/du, optionally fused with the diffusion
//   gradient and the Adam step.
#include "kernels.h"

namespace regk {

__device__ __forceinline__ int win_count(int c, int r, int n) { return min(c + r, n - 1) - max(c - r, 0) + 1; }

template <int K>
__device__ __forceinline__ void xpass(const float *__restrict__ src, float *__restrict__ dst, int RH, int RW,
                                      int r, int tid) {
    // jobs: (quantity k, region row yy, 8-wide segment seg)
    constexpr int SEGS = TX / 8;
    for (int job = tid; job < K * RH * SEGS; job += TILE_THREADS) {
        const int seg = job % SEGS;
        const int rest = job / SEGS;
        const int yy = rest % RH;
        const int k = rest / RH;
        const float *row = src + (k * RH + yy) * RW + seg * 8;
        float *out = dst + (k * RH + yy) * TX + seg * 8;
        float acc = 0.0f;
        for (int d = 0; d <= 2 * r; ++d) acc += row[d];
        out[0] = acc;
#pragma unroll
        for (int i = 1; i < 8; ++i) {
            acc += row[i + 2 * r] - row[i - 1];
            out[i] = acc;
        }
    }
}

size_t lncc_smem_bytes(int r, int K) {
    const int RH = TY + 2 * r, RW = TX + 2 * r, W = 2 * r + 1;
    return sizeof(float) * ((size_t)K * RH * RW + (size_t)K * RH * TX + (size_t)W * K * TILE_THREADS);
}

template <typename T, bool COEF, int PAD>
__global__ void __launch_bounds__(TILE_THREADS)
    lncc_stats_kernel(const T *__restrict__ F, const T *__restrict__ M, const float *__restrict__ u, Dims g,
                      LnccParams P, int zc, float *__restrict__ coef, double *__restrict__ partials,
                      unsigned *__restrict__ counter, double *__restrict__ sim_out, unsigned *err) {
    extern __shared__ float smem[];
    __shared__ double red[32];
    __shared__ float shift[2];
    const int r = P.r, W = 2 * r + 1, RW = TX + 2 * r, RH = TY + 2 * r;
    float *s5 = smem;
    float *hx = s5 + 5 * RH * RW;
    float *ring = hx + 5 * RH * TX;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int z1 = min(g.nz, z0 + zc);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    if (tid == 0) {
        const int cx = min(x0 + TX / 2, g.nx - 1), cy = min(y0 + TY / 2, g.ny - 1), cz = min(z0 + zc / 2, g.nz - 1);
        const long long pc = (long long)cz * g.nxy + (long long)cy * g.nx + cx;
        shift[0] = ld_vox(F, pc);
        shift[1] = ld_vox(M, pc);
    }
    for (int i = tid; i < W * 5 * TILE_THREADS; i += TILE_THREADS) ring[i] = 0.0f;
    __syncthreads();
    const float shF = shift[0], shJ = shift[1];
    const float cxy = active ? (float)(win_count(x, r, g.nx) * win_count(y, r, g.ny)) : 1.0f;
    const float inv_n = 1.0f / (float)g.n;
    float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float nsum = 0.0f;
    int slot = 0;
    const int plane = RH * RW;
    for (int q = z0 - r; q < z1 + r; ++q) {
        const bool qin = q >= 0 && q < g.nz;
        for (int e = tid; e < plane; e += TILE_THREADS) {
            const int yy = e / RW, xx = e - yy * RW;
            const int gx = x0 - r + xx, gy = y0 - r + yy;
            float f = 0.0f, j = 0.0f;
            if (qin && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
                const long long p = (long long)q * g.nxy + (long long)gy * g.nx + gx;
                f = ld_vox(F, p) - shF;
                j = sample<T, PAD>(M, g, gx, gy, q, __ldg(u + p), __ldg(u + g.n + p), __ldg(u + 2 * g.n + p)) - shJ;
            }
            s5[e] = f;
            s5[plane + e] = j;
            s5[2 * plane + e] = f * f;
            s5[3 * plane + e] = j * j;
            s5[4 * plane + e] = f * j;
        }
        __syncthreads();
        xpass<5>(s5, hx, RH, RW, r, tid);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float acc = 0.0f;
            for (int d = 0; d <= 2 * r; ++d) acc += hx[(k * RH + threadIdx.y + d) * TX + threadIdx.x];
            float *rs = ring + (slot * 5 + k) * TILE_THREADS + tid;
            S[k] += acc - *rs;
            *rs = acc;
        }
        slot = slot + 1 == W ? 0 : slot + 1;
        const int zo = q - r;
        if (active && zo >= z0 && zo < z1) {
            const float c = cxy * (float)win_count(zo, r, g.nz);
            const float ic = 1.0f / c;
            const float mF = S[0] * ic, mJ = S[1] * ic;
            const float A = fmaf(S[4], ic, -mF * mJ);
            const float Bv = fmaxf(fmaf(S[2], ic, -mF * mF), 0.0f);
            const float Cv = fmaxf(fmaf(S[3], ic, -mJ * mJ), 0.0f);
            const float D = fmaf(Bv, Cv, P.eps);
            float n = 0.0f, aFJ = 0.0f, aJJ = 0.0f;
            if (D > 0.0f) {
                const float iD = 1.0f / D;
                n = A * A * iD;
                aFJ = -inv_n * (2.0f * A * iD) * ic;
                aJJ = -inv_n * (-A * A * Bv * iD * iD) * ic;
            }
            nsum += n;
            if (COEF) {
                const long long p = (long long)zo * g.nxy + (long long)y * g.nx + x;
                const float aJ = -(aFJ * (mF + shF) + 2.0f * aJJ * (mJ + shJ));
                coef[p] = aJ;
                coef[g.n + p] = aJJ;
                coef[2 * g.n + p] = aFJ;
            }
        }
    }
    const double bs = block_sum((double)nsum, red);
    const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (tid == 0) partials[bid] = bs;
    if (arrive_last(counter)) {
        const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
        double acc = 0.0;
        for (long long i = tid; i < nb; i += TILE_THREADS) acc += __ldcg(partials + i);
        const double tot = block_sum(acc, red);
        if (tid == 0) {
            const double Sv = tot / (double)g.n;
            if (!isfinite(Sv)) latch_error(err, REG_ERR_NONFINITE);
            sim_out[0] = Sv;
            *counter = 0u;
        }
    }
}

template <typename T, typename MT, bool STEP, int PAD>
__global__ void __launch_bounds__(TILE_THREADS)
    lncc_sweep2_kernel(const T *__restrict__ F, const T *__restrict__ M, const float *__restrict__ u, Dims g,
                       LnccParams P, int zc, const float *__restrict__ coef, float *__restrict__ grad_out,
                       float *__restrict__ u_out, MT *__restrict__ m, MT *__restrict__ v, StepParams S,
                       double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ r_out,
                       unsigned *err) {
    extern __shared__ float smem[];
    __shared__ double red[32];
    const int r = P.r, W = 2 * r + 1, RW = TX + 2 * r, RH = TY + 2 * r;
    float *s3 = smem;
    float *hx = s3 + 3 * RH * RW;
    float *ring = hx + 3 * RH * TX;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int z1 = min(g.nz, z0 + zc);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    for (int i = tid; i < W * 3 * TILE_THREADS; i += TILE_THREADS) ring[i] = 0.0f;
    const long long col = active ? (long long)y * g.nx + x : 0;
    float cur[3] = {0.f, 0.f, 0.f}, prv[3] = {0.f, 0.f, 0.f}, nxt[3] = {0.f, 0.f, 0.f};
    if (active) {
        const long long p = (long long)z0 * g.nxy + col;
#pragma unroll
        for (int c = 0; c < 3; ++c) cur[c] = __ldg(u + c * g.n + p);
        if (STEP && z0 > 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) prv[c] = __ldg(u + c * g.n + p - g.nxy);
        }
    }
    __syncthreads();
    float Sa[3] = {0.f, 0.f, 0.f};
    float rpart = 0.0f;
    int slot = 0;
    const int plane = RH * RW;
    for (int q = z0 - r; q < z1 + r; ++q) {
        const bool qin = q >= 0 && q < g.nz;
        for (int e = tid; e < plane; e += TILE_THREADS) {
            const int yy = e / RW, xx = e - yy * RW;
            const int gx = x0 - r + xx, gy = y0 - r + yy;
            float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
            if (qin && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
                const long long p = (long long)q * g.nxy + (long long)gy * g.nx + gx;
                a0 = __ldg(coef + p);
                a1 = __ldg(coef + g.n + p);
                a2 = __ldg(coef + 2 * g.n + p);
            }
            s3[e] = a0;
            s3[plane + e] = a1;
            s3[2 * plane + e] = a2;
        }
        __syncthreads();
        xpass<3>(s3, hx, RH, RW, r, tid);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = 0.0f;
            for (int d = 0; d <= 2 * r; ++d) acc += hx[(k * RH + threadIdx.y + d) * TX + threadIdx.x];
            float *rs = ring + (slot * 3 + k) * TILE_THREADS + tid;
            Sa[k] += acc - *rs;
            *rs = acc;
        }
        slot = slot + 1 == W ? 0 : slot + 1;
        const int zo = q - r;
        if (active && zo >= z0 && zo < z1) {
            const long long p = (long long)zo * g.nxy + col;
            if (zo + 1 < g.nz) {
#pragma unroll
                for (int c = 0; c < 3; ++c) nxt[c] = __ldg(u + c * g.n + p + g.nxy);
            }
            float sx, sy, sz;
            const float jv = sample_grad<T, PAD>(M, g, x, y, zo, cur[0], cur[1], cur[2], sx, sy, sz);
            const float fv = ld_vox(F, p);
            const float gj = fmaf(fv, Sa[2], fmaf(2.0f * jv, Sa[1], Sa[0]));
            const float gs[3] = {gj * sx, gj * sy, gj * sz};
            if (STEP) {
                float gR[3];
                diffusion_at(u, g, x, y, zo, p, cur, prv, nxt, gR, rpart);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float gt = fmaf(S.lam * S.two_over_n, gR[c], gs[c]);
                    if (grad_out) grad_out[c * g.n + p] = gt;
                    u_out[c * g.n + p] = adam_elem(cur[c], gt, m, v, c * g.n + p, S);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) grad_out[c * g.n + p] = gs[c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                prv[c] = cur[c];
                cur[c] = nxt[c];
            }
        }
    }
    if (STEP) {
        const double bs = block_sum((double)rpart, red);
        const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (tid == 0) partials[bid] = bs;
        if (arrive_last(counter)) {
            const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
            double acc = 0.0;
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

MarchGrid lncc_grid(const Dims &g, int r) { return march_grid(g, 6LL * num_sms() * 3, 4 * r > 16 ? 4 * r : 16); }

template <typename K>
static cudaError_t allow_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_lncc_stats(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                              const LnccParams &P, float *coef, double *partials, unsigned *counter,
                              double *sim_out, cudaStream_t s) {
    const MarchGrid G = lncc_grid(g, P.r);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    const size_t smem = lncc_smem_bytes(P.r, 5);
    unsigned *err = error_word();
    cudaError_t e = cudaSuccess;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            if (coef) {
                e = allow_smem(lncc_stats_kernel<T, true, PD>, smem);
                if (e == cudaSuccess)
                    lncc_stats_kernel<T, true, PD><<<grid, block, smem, s>>>((const T *)F, (const T *)M, u, g, P, G.zc,
                                                                             coef, partials, counter, sim_out, err);
            } else {
                e = allow_smem(lncc_stats_kernel<T, false, PD>, smem);
                if (e == cudaSuccess)
                    lncc_stats_kernel<T, false, PD><<<grid, block, smem, s>>>((const T *)F, (const T *)M, u, g, P,
                                                                              G.zc, coef, partials, counter, sim_out,
                                                                              err);
            }
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_lncc_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                               const LnccParams &P, const float *coef, float *grad_out, bool step,
                               float *u_out, void *m, void *v, int mdt, const StepParams &S,
                               double *partials, unsigned *counter, double *r_out, cudaStream_t s) {
    const MarchGrid G = lncc_grid(g, P.r);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    const size_t smem = lncc_smem_bytes(P.r, 3);
    unsigned *err = error_word();
    cudaError_t e = cudaSuccess;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            if (!step) {
                e = allow_smem(lncc_sweep2_kernel<T, float, false, PD>, smem);
                if (e == cudaSuccess)
                    lncc_sweep2_kernel<T, float, false, PD><<<grid, block, smem, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (float *)m, (float *)v, S,
                        partials, counter, r_out, err);
                return;
            }
            with_type(mdt, [&](auto mp) {
                using MT = elem_t<decltype(mp)>;
                e = allow_smem(lncc_sweep2_kernel<T, MT, true, PD>, smem);
                if (e == cudaSuccess)
                    lncc_sweep2_kernel<T, MT, true, PD><<<grid, block, smem, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (MT *)m, (MT *)v, S,
                        partials, counter, r_out, err);
            });
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace regk
