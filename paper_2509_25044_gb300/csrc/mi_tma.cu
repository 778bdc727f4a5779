// mi_tma.cu -- the second MI sweep (Sec. 2.2, Eq. gradientmi-threadn; App.
// fused MI), fused with the diffusion gradient and Adam, with every streamed
// array staged in shared memory by the Tensor Memory Accelerator.
//
// The plain sweep (mi.cu) loads u, F, m and v itself, one plane ahead in
// registers, and spends most of its issue slots on those loads and their
// 64-bit addresses; at gigavoxel sizes its loads are too few in flight to
// cover DRAM latency.  Here a CTA owns a 64 x TY voxel tile (an x pair per
// lane, one warp per row; TY = 31 or 20, SwShape) and marches it through a
// chunk of z-planes with warp specialisation:
//
//   producer (one elected thread of warp TY): for each plane, one tiled TMA
//     copy of u with the diffusion stencil's halo (x0-4 .. x0+67, y0-1 ..
//     y0+TY, all 3 channels; zero outside the volume) into a ring of
//     SwShape::nu plane slots, and one copy each of F, m and v (the tile, 3
//     channels for m and v) into a ring of SW_NS slots.  Each slot's mbarrier
//     completes on the copies' byte count; the producer refills a slot once
//     the TY consumer warps have released it (a second mbarrier per slot).
//   consumers (warps 0 .. TY-1, one row of the tile each, two voxels per
//     lane): u at z-1, z, z+1 and the 4 in-plane neighbours, F, m and v come
//     from shared memory; only the 8 corner gathers of the trilinear sampler
//     go to global memory.  The per-voxel arithmetic (sampler, B-spline
//     weights, 16-term adjoint, diffusion, Adam) is that of mi.cu term for
//     term, so both paths give the same bits for u', m, v and the gradient.
//
// Every wait is bounded: a wait that expires latches REG_ERR_TIMEOUT in the
// device error word, the CTA stops issuing and consuming, waits (bounded)
// for the copies it has in flight and returns.
#include <algorithm>

#include "kernels.h"
#include "mi_common.cuh"
#include "tma.cuh"

namespace regk {

namespace {

constexpr int SW_VL = 2;          // voxels per lane (an x pair)
constexpr int SW_TX = 32 * SW_VL;  // tile width; one warp per tile row
constexpr int SW_UX = SW_TX + 8;   // u box: x0-4 .. x0+SW_TX+3
constexpr int SW_NS = 3;           // F / m / v plane slots

// Two tile heights, one CTA per SM each: 31 rows (1024 threads at 64
// registers) where its rings fit a CTA's shared memory (BF16 images and
// moments), else 20 rows (672 threads at 80 registers).  More consumer warps
// cover more of the corner gathers' latency.
template <int TY>
struct SwShape {
    static constexpr int uy = TY + 2;                  // u box rows: y0-1 .. y0+TY
    static constexpr int uc = SW_UX * uy;              // one u channel of the box
    static constexpr int threads = 32 * (TY + 1);      // TY consumer warps + the producer
    static constexpr int nu = TY >= 31 ? 4 : 5;        // u plane slots: z-1, z, z+1 in use, the rest in flight
    static constexpr uint32_t ubytes = 3u * uc * sizeof(float);
};

__host__ __device__ constexpr size_t al128(size_t v) { return (v + 127) & ~(size_t)127; }

// dynamic shared memory: the adjoint table, the two rings, the mbarriers
template <int TY>
struct SwLayout {
    size_t u, f, m, v, bar, total, fslot, mslot;
    __host__ __device__ SwLayout(int B, int fbytes, int mbytes) {
        using SH = SwShape<TY>;
        fslot = al128((size_t)SW_TX * TY * fbytes);
        mslot = al128((size_t)3 * SW_TX * TY * mbytes);
        u = al128(sizeof(float4) * (size_t)B * B);
        f = u + SH::nu * al128(SH::ubytes);
        m = f + SW_NS * fslot;
        v = m + SW_NS * mslot;
        bar = v + SW_NS * mslot;
        total = bar + sizeof(uint64_t) * 2 * (SH::nu + SW_NS);
    }
};

// two consecutive elements (8-byte aligned FP32 / 4-byte aligned BF16) as floats, and their stores
__device__ __forceinline__ float2 ld_pair(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
__device__ __forceinline__ void st_pair(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
// round-to-nearest-even of each element, as __float2bfloat16_rn
__device__ __forceinline__ void st_pair(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

}  // namespace

// BT > 0: the bin count compiled in (table and ring offsets fold to
// constants); BT = 0: P.bins.
template <int TY, typename T, typename MT, bool STEP, int PAD, typename I, int BT = 0>
__global__ void __launch_bounds__(SwShape<TY>::threads, 1)
    mi_sweep2_tma_kernel(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap fmap,
                         const __grid_constant__ CUtensorMap mmap, const __grid_constant__ CUtensorMap vmap,
                         const T *__restrict__ M, Dims g, MiParams P, int zc, const float *__restrict__ Gtab,
                         float *__restrict__ grad_out, float *__restrict__ u_out, MT *__restrict__ m,
                         MT *__restrict__ v, StepParams S, double *__restrict__ partials,
                         unsigned *__restrict__ counter, double *__restrict__ r_out, unsigned *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double red[32];
    __shared__ volatile int abort_flag;
    constexpr int FB = (int)sizeof(T), MB = STEP ? (int)sizeof(MT) : 0;
    constexpr int SW_TY = TY, SW_UY = SwShape<TY>::uy, SW_UC = SwShape<TY>::uc, SW_NU = SwShape<TY>::nu;
    constexpr int SW_THREADS = SwShape<TY>::threads;
    constexpr uint32_t SW_UBYTES = SwShape<TY>::ubytes;
    (void)SW_UY;
    const int B = BT > 0 ? BT : P.bins, BB = B * B;
    const SwLayout<TY> L(B, FB, MB);
    float4 *G4 = reinterpret_cast<float4 *>(smem);
    uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + L.bar);
    uint64_t *empty_u = full_u + SW_NU, *full_s = empty_u + SW_NU, *empty_s = full_s + SW_NS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float4 *T4 = mi_table4(Gtab);
    for (int i = tid; i < BB; i += SW_THREADS) G4[i] = __ldg(T4 + i);
    if (tid == 0) {
        for (int s = 0; s < SW_NU; ++s) {
            umma::mbar_init(full_u + s, 1);
            umma::mbar_init(empty_u + s, SW_TY);
        }
        for (int s = 0; s < SW_NS; ++s) {
            umma::mbar_init(full_s + s, 1);
            umma::mbar_init(empty_s + s, SW_TY);
        }
        abort_flag = 0;
    }
    __syncthreads();

    const int x0 = blockIdx.x * SW_TX, y0 = blockIdx.y * SW_TY;
    const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc), nzc = z1 - z0;
    double rsum = 0.0;
    if (warp == SW_TY) {
        // ---------------- producer ----------------
        if (lane == 0) {
            const uint32_t sbytes = (uint32_t)(SW_TX * SW_TY * FB + 2 * 3 * SW_TX * SW_TY * MB);
            int ju = 0, ks = 0;  // u planes / F,m,v planes issued
            for (int j = 0; j < nzc + 2 && !abort_flag; ++j) {
                const int su = j % SW_NU;
                if (j >= SW_NU && !umma::mbar_wait(empty_u + su, ((j / SW_NU) - 1) & 1)) {
                    latch_error(err, REG_ERR_TIMEOUT);
                    abort_flag = 1;
                    break;
                }
                tma::expect_tx(full_u + su, SW_UBYTES);
                tma::load_4d(smem + L.u + su * al128(SW_UBYTES), &umap, x0 - 4, y0 - 1, z0 - 1 + j, 0, full_u + su);
                ju = j + 1;
                const int k = j - 1;
                if (k < 0 || k >= nzc) continue;
                const int ss = k % SW_NS;
                if (k >= SW_NS && !umma::mbar_wait(empty_s + ss, ((k / SW_NS) - 1) & 1)) {
                    latch_error(err, REG_ERR_TIMEOUT);
                    abort_flag = 1;
                    break;
                }
                tma::expect_tx(full_s + ss, sbytes);
                tma::load_3d(smem + L.f + ss * L.fslot, &fmap, x0, y0, z0 + k, full_s + ss);
                if (STEP) {
                    tma::load_4d(smem + L.m + ss * L.mslot, &mmap, x0, y0, z0 + k, 0, full_s + ss);
                    tma::load_4d(smem + L.v + ss * L.mslot, &vmap, x0, y0, z0 + k, 0, full_s + ss);
                }
                ks = k + 1;
            }
            // copies still in flight (only after an abort) land before the CTA exits
            for (int j = std::max(0, ju - SW_NU); j < ju; ++j) umma::mbar_wait(full_u + j % SW_NU, (j / SW_NU) & 1);
            for (int k = std::max(0, ks - SW_NS); k < ks; ++k) umma::mbar_wait(full_s + k % SW_NS, (k / SW_NS) & 1);
        }
    } else {
        // ---------------- consumers ----------------
        // lane: the x pair (x, x + 1); the pair is wholly inside or outside the
        // volume (nx % 8 == 0, x even)
        const int x = x0 + SW_VL * lane, y = y0 + warp;
        const bool in = x < g.nx && y < g.ny;
        const bool hxl = x > 0, hxr = x + SW_VL < g.nx, hym = y > 0, hyp = y + 1 < g.ny;
        const I nxy = (I)g.nxy;
        I p = (I)z0 * nxy + (I)y * g.nx + x;
        const int o = (warp + 1) * SW_UX + SW_VL * lane + 4;  // (x, y) in a u channel slot (even: 8-byte aligned)
        const int t = warp * SW_TX + SW_VL * lane;            // (x, y) in an F / m / v slot
        float racc = 0.0f;
        // ring slots of u at z-1, z, z+1 and of F / m / v at z, rotated once per
        // plane, and the parity each slot's next completion will have
        int su0 = 0, su1 = 1, su2 = 2, ss = 0;
        uint32_t uphase = 0u, sphase = 0u;
        for (int zi = 0; zi < nzc; ++zi, p += nxy) {
            const int z = z0 + zi;
            bool ok = true;
            if (zi == 0) {
                ok = umma::mbar_wait(full_u, 0) && umma::mbar_wait(full_u + 1, 0);
                uphase = 3u;
            }
            ok = ok && umma::mbar_wait(full_u + su2, (uphase >> su2) & 1u) &&
                 umma::mbar_wait(full_s + ss, (sphase >> ss) & 1u);
            uphase ^= 1u << su2;
            sphase ^= 1u << ss;
            // the warp leaves together (its lanes meet at __syncwarp below)
            if (!__all_sync(0xffffffffu, ok && !abort_flag)) {
                if (lane == 0) {
                    latch_error(err, REG_ERR_TIMEOUT);
                    abort_flag = 1;
                }
                break;
            }
            const float *Up = reinterpret_cast<const float *>(smem + L.u + su0 * al128(SW_UBYTES));
            const float *Uc = reinterpret_cast<const float *>(smem + L.u + su1 * al128(SW_UBYTES));
            const float *Un = reinterpret_cast<const float *>(smem + L.u + su2 * al128(SW_UBYTES));
            const T *Fs = reinterpret_cast<const T *>(smem + L.f + ss * L.fslot);
            if (in) {
                float cur[3][SW_VL];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 q = ld_pair(Uc + c * SW_UC + o);
                    cur[c][0] = q.x;
                    cur[c][1] = q.y;
                }
                const float2 fq = ld_pair(Fs + t);
                const float fv[SW_VL] = {fq.x, fq.y};
                float gs[3][SW_VL];
#pragma unroll
                for (int e = 0; e < SW_VL; ++e) {
                    float sx, sy, sz;
                    const float jv = sample_grad<T, PAD, I>(M, g, x + e, y, z, cur[0][e], cur[1][e], cur[2][e], sx,
                                                            sy, sz);
                    float wf[4], dj[4];
                    const int iF = bspline_weights(to_bin(fv[e], P.f_lo, P.f_scale, B), B, wf) - 1;
                    const float tj = (jv - P.m_lo) * P.m_scale;
                    const int iJ = bspline_dweights(to_bin(jv, P.m_lo, P.m_scale, B), B, dj) - 1;
                    float gj = 0.0f;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float4 r = G4[(iF + a) * B + iJ];
                        const float tt = fmaf(r.x, dj[0], fmaf(r.y, dj[1], fmaf(r.z, dj[2], r.w * dj[3])));
                        gj = fmaf(wf[a], tt, gj);
                    }
                    if (!(tj >= 0.0f && tj <= 1.0f)) gj = 0.0f;  // intensity clamp is flat
                    gs[0][e] = gj * sx;
                    gs[1][e] = gj * sy;
                    gs[2][e] = gj * sz;
                }
                if (STEP) {
                    const MT *Ms = reinterpret_cast<const MT *>(smem + L.m + ss * L.mslot);
                    const MT *Vs = reinterpret_cast<const MT *>(smem + L.v + ss * L.mslot);
                    const bool hzm = z > 0, hzp = z + 1 < g.nz;
                    float rpart = 0.0f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float *U = Uc + c * SW_UC;
                        const float2 yp = ld_pair(U + o + SW_UX), ym = ld_pair(U + o - SW_UX);
                        const float2 zp = ld_pair(Un + c * SW_UC + o), zm = ld_pair(Up + c * SW_UC + o);
                        const float xl = U[o - 1], xr = U[o + SW_VL];
                        const float ypv[SW_VL] = {yp.x, yp.y}, ymv[SW_VL] = {ym.x, ym.y};
                        const float zpv[SW_VL] = {zp.x, zp.y}, zmv[SW_VL] = {zm.x, zm.y};
                        const float2 m2 = ld_pair(Ms + c * SW_TX * SW_TY + t), v2 = ld_pair(Vs + c * SW_TX * SW_TY + t);
                        const float m0[SW_VL] = {m2.x, m2.y}, v0[SW_VL] = {v2.x, v2.y};
                        float uo[SW_VL], mo[SW_VL], vo[SW_VL], gt[SW_VL];
#pragma unroll
                        for (int e = 0; e < SW_VL; ++e) {
                            // diffusion gradient, same terms and order as diffusion_ptr
                            const float c0 = cur[c][e];
                            const bool hxm = e > 0 || hxl, hxp = e < SW_VL - 1 || hxr;
                            const float xm = e > 0 ? cur[c][e - 1] : xl;
                            const float xp = e < SW_VL - 1 ? cur[c][e + 1] : xr;
                            float acc = 0.0f;
                            if (hxp) {
                                const float d = xp - c0;
                                acc -= d;
                                rpart = fmaf(d, d, rpart);
                            }
                            if (hxm) acc += c0 - xm;
                            if (hyp) {
                                const float d = ypv[e] - c0;
                                acc -= d;
                                rpart = fmaf(d, d, rpart);
                            }
                            if (hym) acc += c0 - ymv[e];
                            if (hzp) {
                                const float d = zpv[e] - c0;
                                acc -= d;
                                rpart = fmaf(d, d, rpart);
                            }
                            if (hzm) acc += c0 - zmv[e];
                            gt[e] = fmaf(S.lam * S.two_over_n, acc, gs[c][e]);
                            // Adam, term for term as adam_fast
                            const float gg = S.gscale * gt[e];
                            mo[e] = fmaf(S.b1, m0[e], (1.0f - S.b1) * gg);
                            vo[e] = fmaf(S.b2, v0[e], (1.0f - S.b2) * gg * gg);
                            const float denom = fmaf(sqrt_approx(vo[e]), S.rsqrt_bc2, S.eps);
                            uo[e] = fmaf(-S.lr_bc1, __fdividef(mo[e], denom), c0);
                        }
                        if (grad_out) st_pair(grad_out + c * g.n + p, gt[0], gt[1]);
                        st_pair(u_out + c * g.n + p, uo[0], uo[1]);
                        st_pair(m + c * g.n + p, mo[0], mo[1]);
                        st_pair(v + c * g.n + p, vo[0], vo[1]);
                    }
                    racc += rpart;
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) st_pair(grad_out + c * g.n + p, gs[c][0], gs[c][1]);
                }
            }
            __syncwarp();
            if (lane == 0) {
                umma::mbar_arrive(empty_u + su0);  // u at z - 1 is no longer needed
                umma::mbar_arrive(empty_s + ss);
            }
            su0 = su1;
            su1 = su2;
            su2 = su2 + 1 == SW_NU ? 0 : su2 + 1;
            ss = ss + 1 == SW_NS ? 0 : ss + 1;
            if ((zi & 15) == 15) {
                rsum += (double)racc;
                racc = 0.0f;
            }
        }
        rsum += (double)racc;
    }
    if (STEP) {
        const double bs = block_sum(rsum, red);
        const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (tid == 0) partials[bid] = bs;
        if (arrive_last(counter)) {
            const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
            double acc = 0.0;
            for (long long i = tid; i < nb; i += SW_THREADS) acc += __ldcg(partials + i);
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

// The TMA path needs every tensor-map stride to be a multiple of 16 bytes
// (BF16 rows: nx % 8 == 0) and no composite transform.
bool mi_tma_ok(const Dims &g) { return g.nx % 8 == 0; }

// Grid of 64 x ty tiles; the z-chunk count minimises (waves of resident CTAs)
// x (planes per CTA + 3), the 3 being each CTA's start-up (its adjoint table
// and the two planes its stencil reads beyond the chunk).
MarchGrid mi_tma_sweep_grid(const Dims &g, int ty) {
    MarchGrid G;
    G.tiles_x = (g.nx + SW_TX - 1) / SW_TX;
    G.tiles_y = (g.ny + ty - 1) / ty;
    static int per_sm[2] = {0, 0};  // 0 until the occupancy calculator has answered
    const int k = ty >= 31 ? 1 : 0;
    int n = per_sm[k];
    if (n == 0) {
        // residency with 32 bins (the instantiations of one shape share its
        // register budget; only larger tables take more shared memory); the
        // grid must not depend on the call's bin count, since it also sizes
        // the workspace
        auto query = [&](auto kern, size_t total, int threads) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, total) != cudaSuccess || n < 1) {
                (void)cudaGetLastError();
                n = 0;
            }
        };
        if (k == 1)
            query(mi_sweep2_tma_kernel<31, __nv_bfloat16, __nv_bfloat16, true, REG_PAD_BORDER, int>,
                  SwLayout<31>(32, 2, 2).total, SwShape<31>::threads);
        else
            query(mi_sweep2_tma_kernel<20, float, float, true, REG_PAD_BORDER, int>, SwLayout<20>(32, 4, 4).total,
                  SwShape<20>::threads);
        if (n > 0)
            per_sm[k] = n;
        else
            n = 1;
    }
    const long long tiles = (long long)G.tiles_x * G.tiles_y;
    const long long slots = (long long)n * num_sms();
    long long best_c = 1;
    double best = -1.0;
    for (long long c = 1; c <= std::min<long long>(g.nz, 256); ++c) {
        const long long zc = (g.nz + c - 1) / c;
        if ((g.nz + zc - 1) / zc != c) continue;
        const long long waves = (tiles * c + slots - 1) / slots;
        const double cost = (double)waves * (double)(zc + 3);
        if (best < 0.0 || cost < best) {
            best = cost;
            best_c = c;
        }
    }
    G.zc = (int)((g.nz + best_c - 1) / best_c);
    G.chunks = (int)((g.nz + G.zc - 1) / G.zc);
    return G;
}

long long mi_tma_max_blocks(const Dims &g) {
    return std::max(mi_tma_sweep_grid(g, 20).blocks(), mi_tma_sweep_grid(g, 31).blocks());
}

cudaError_t launch_mi_sweep2_tma(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                                 const MiParams &P, const float *Gtab, float *grad_out, bool step, float *u_out,
                                 void *m, void *v, int mdt, const StepParams &S, double *partials,
                                 unsigned *counter, double *r_out, cudaStream_t s) {
    // the taller tile where its rings and the adjoint table fit one CTA's
    // shared memory, else the shorter; neither (large bin counts with FP32
    // images and moments): the plain sweep
    const int fb = dt == REG_BF16 ? 2 : 4, mb = step ? (mdt == REG_BF16 ? 2 : 4) : 0;
    int ty = 0;
    {
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return cudaErrorNotSupported;
        if (SwLayout<31>(P.bins, fb, mb).total + 1024 <= (size_t)optin)
            ty = 31;
        else if (SwLayout<20>(P.bins, fb, mb).total + 1024 <= (size_t)optin)
            ty = 20;
        else
            return cudaErrorNotSupported;
    }
    CUtensorMap umap, fmap, mmap, vmap;
    const uint64_t d4[4] = {(uint64_t)g.nx, (uint64_t)g.ny, (uint64_t)g.nz, 3};
    const uint64_t d3[3] = {(uint64_t)g.nx, (uint64_t)g.ny, (uint64_t)g.nz};
    const uint32_t ubox[4] = {SW_UX, (uint32_t)ty + 2, 1, 3}, sbox4[4] = {SW_TX, (uint32_t)ty, 1, 3},
                   sbox3[3] = {SW_TX, (uint32_t)ty, 1};
    if (!tma::make_map(&umap, u, REG_F32, 4, d4, ubox) || !tma::make_map(&fmap, F, dt, 3, d3, sbox3))
        return cudaErrorNotSupported;
    if (step) {
        if (!tma::make_map(&mmap, m, mdt, 4, d4, sbox4) || !tma::make_map(&vmap, v, mdt, 4, d4, sbox4))
            return cudaErrorNotSupported;
    } else {
        mmap = vmap = umap;  // unused without the step
    }
    const MarchGrid G = mi_tma_sweep_grid(g, ty);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    cudaError_t e = cudaSuccess;
    auto shape = [&](auto tyc) {
        constexpr int TY = decltype(tyc)::value;
        with_type(dt, [&](auto tp) {
            using T = elem_t<decltype(tp)>;
            with_pad(pad, [&](auto pd) {
                constexpr int PD = decltype(pd)::value;
                with_index(g, [&](auto ip) {
                    using I = elem_t<decltype(ip)>;
                    auto go = [&](auto kern, auto *mp, bool st) {
                        using MT = std::remove_pointer_t<decltype(mp)>;
                        const size_t smem = SwLayout<TY>(P.bins, (int)sizeof(T), st ? (int)sizeof(MT) : 0).total;
                        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                        if (e != cudaSuccess) return;
                        kern<<<grid, SwShape<TY>::threads, smem, s>>>(umap, fmap, mmap, vmap, (const T *)M, g, P, G.zc,
                                                                      Gtab, grad_out, u_out, (MT *)m, (MT *)v, S,
                                                                      partials, counter, r_out, err);
                    };
                    // the step with the workloads' 32 bins compiled in
                    if (!step)
                        go(mi_sweep2_tma_kernel<TY, T, float, false, PD, I>, (float *)nullptr, false);
                    else if (mdt == REG_BF16 && P.bins == 32)
                        go(mi_sweep2_tma_kernel<TY, T, __nv_bfloat16, true, PD, I, 32>, (__nv_bfloat16 *)nullptr, true);
                    else if (mdt == REG_BF16)
                        go(mi_sweep2_tma_kernel<TY, T, __nv_bfloat16, true, PD, I>, (__nv_bfloat16 *)nullptr, true);
                    else if (P.bins == 32)
                        go(mi_sweep2_tma_kernel<TY, T, float, true, PD, I, 32>, (float *)nullptr, true);
                    else
                        go(mi_sweep2_tma_kernel<TY, T, float, true, PD, I>, (float *)nullptr, true);
                });
            });
        });
    };
    if (ty == 31)
        shape(IC<31>{});
    else
        shape(IC<20>{});
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace regk
