// lncc.cu -- windowed LNCC (Sec. 2.3; App. fused LNCC, Eq. lncc-loss,
// Eqs. lncc-a..lncc-c) and its adjoint on sm_103a, in two sweeps.
//
// The warped image J = M o (id+u) is produced once per evaluation by the
// warp kernel into the workspace (4 bytes per voxel) and read back through
// L2 with its halo, instead of being re-gathered for every halo voxel.
//
// Both sweeps use the same 2.5-D tile march: a CTA owns a 32 x 8 column
// tile in (x, y) and walks a chunk of z-planes.  For every input plane it
// stages the tile plus an r-voxel halo in shared memory, box-sums along x
// (sliding sums over 8-voxel row segments), then along y (sliding sums over
// whole columns, written straight into a ring of the last 2r+1 plane sums),
// and each thread keeps the running z-sum of its own column.  Shared arrays
// use odd pitches so that the row segments of a warp fall in distinct banks.
//
// sweep 1 (lncc_stats_kernel): stages F and J with a per-CTA intensity shift
//   (F and J at the tile centre) so the FP32 variance sums do not cancel.
//   From the five window sums it forms A, B, C, n_i = A^2 / (B C + eps) and
//   adds n_i into FP64 block partials (fixed-order final sum -> S = mean
//   n_i).  For the gradient it also writes the three per-window adjoint
//   coefficients (dL/dn_i = -1/N):
//     a_FJ = -(1/N) (2A/D) / c,   a_JJ = -(1/N) (-A^2 B / D^2) / c,
//     a_J  = -(a_FJ muF + 2 a_JJ muJ),
//   so that dL/dJ_k = sum_{i: k in W_i} (a_J + 2 J_k a_JJ + F_k a_FJ)_i,
//   the moving-image form of Eq. gradientcc-first (the printed A/(B^2 C)
//   read as A^2/(B^2 C)) with the window-sum derivatives taken directly.
// sweep 2 (lncc_sweep2_kernel): the second box sum of the three coefficient
//   fields (exact adjoint, not the ANTs shortcut), then dL/dJ, chained
//   through the sampler slope to dL/du, optionally fused with the diffusion
//   gradient and the Adam step.
#include <algorithm>
#include <mutex>

#include "kernels.h"

namespace regk {

__device__ __forceinline__ int win_count(int c, int r, int n) { return min(c + r, n - 1) - max(c - r, 0) + 1; }

constexpr int SEGW = 8;  // x-pass segment width

// shared-memory layout of one sweep for K quantities and radius r
struct LnccSmem {
    int RH, RW, RWP, HXP, W, K;
    __host__ __device__ LnccSmem(int r, int k)
        : RH(TY + 2 * r), RW(TX + 2 * r), RWP(TX + 2 * r + 1), HXP(TX + 1), W(2 * r + 1), K(k) {}
    __host__ __device__ int stage_words() const { return K * RH * RWP; }  // staged plane + halo
    __host__ __device__ int hx_words() const { return K * RH * HXP; }     // x sums
    __host__ __device__ int ring_words() const { return W * K * TILE_THREADS; }
    __host__ __device__ size_t bytes() const {
        return sizeof(float) * ((size_t)stage_words() + hx_words() + ring_words());
    }
};

size_t lncc_smem_bytes(int r, int K) { return LnccSmem(r, K).bytes(); }

// x box sums of every staged row (sliding over 8-wide segments).  A job is
// (quantity k, staged row yy, segment seg); thread tid owns jobs tid,
// tid + TILE_THREADS, ...  Their offsets depend only on tid, so they are
// computed once per CTA (XJobs) instead of once per plane.
constexpr int MAX_XJOBS = 3;  // K * RH * (TX / SEGW) <= 5 * (8 + 2 * 7) * 4 = 440 < 3 * 256
struct XJobs {
    int n;
    int in[MAX_XJOBS], out[MAX_XJOBS];
};
template <int K>
__device__ __forceinline__ XJobs make_xjobs(const LnccSmem &L, int tid) {
    constexpr int SEGS = TX / SEGW;
    XJobs J;
    J.n = 0;
#pragma unroll
    for (int i = 0; i < MAX_XJOBS; ++i) {
        const int job = tid + i * TILE_THREADS;
        J.in[i] = J.out[i] = 0;
        if (job < K * L.RH * SEGS) {
            const int seg = job % SEGS;
            const int rest = job / SEGS;
            const int yy = rest % L.RH;
            const int k = rest / L.RH;
            J.in[i] = (k * L.RH + yy) * L.RWP + seg * SEGW;
            J.out[i] = (k * L.RH + yy) * L.HXP + seg * SEGW;
            J.n = i + 1;
        }
    }
    return J;
}
__device__ __forceinline__ void xpass(const float *__restrict__ st, float *__restrict__ hx, const XJobs &J, int r) {
#pragma unroll
    for (int i = 0; i < MAX_XJOBS; ++i) {
        if (i >= J.n) break;
        const float *row = st + J.in[i];
        float *out = hx + J.out[i];
        float acc = 0.0f;
        for (int d = 0; d <= 2 * r; ++d) acc += row[d];
        out[0] = acc;
#pragma unroll
        for (int t = 1; t < SEGW; ++t) {
            acc += row[t + 2 * r] - row[t - 1];
            out[t] = acc;
        }
    }
}

// x box sums of every staged row (sliding over 8-wide segments), job
// indices derived per plane (the register-lean form used by sweep 2)
template <int K>
__device__ __forceinline__ void xpass_lean(const float *__restrict__ st, float *__restrict__ hx, const LnccSmem &L, int r,
                                      int tid) {
    constexpr int SEGS = TX / SEGW;
    for (int job = tid; job < K * L.RH * SEGS; job += TILE_THREADS) {
        const int seg = job % SEGS;
        const int rest = job / SEGS;
        const int yy = rest % L.RH;
        const int k = rest / L.RH;
        const float *row = st + (k * L.RH + yy) * L.RWP + seg * SEGW;
        float *out = hx + (k * L.RH + yy) * L.HXP + seg * SEGW;
        float acc = 0.0f;
        for (int d = 0; d <= 2 * r; ++d) acc += row[d];
        out[0] = acc;
#pragma unroll
        for (int i = 1; i < SEGW; ++i) {
            acc += row[i + 2 * r] - row[i - 1];
            out[i] = acc;
        }
    }
}

// y box sums down each column of x sums, written into ring slot `slot`
// (layout [k][y][x] = [k][thread]) -- one job per (quantity, x)
template <int K>
__device__ __forceinline__ void ypass(const float *__restrict__ hx, float *__restrict__ ring, int slot,
                                      const LnccSmem &L, int r, int tid) {
    if (tid < K * TX) {
        const int x = tid % TX, k = tid / TX;
        const float *col = hx + (k * L.RH) * L.HXP + x;
        float *out = ring + (slot * K + k) * TILE_THREADS + x;
        float acc = 0.0f;
        for (int d = 0; d <= 2 * r; ++d) acc += col[d * L.HXP];
        out[0] = acc;
#pragma unroll
        for (int y = 1; y < TY; ++y) {
            acc += col[(y + 2 * r) * L.HXP] - col[(y - 1) * L.HXP];
            out[y * TX] = acc;
        }
    }
}

// Staging of one input plane (tile + r halo) without per-element index
// arithmetic: thread (tx, ty) covers staged columns tx, tx + 32 (RW <= 46)
// and rows ty, ty + 8 [, ty + 16] (NY = 2 for r <= 4, 3 up to r = 7).  The
// slot (j, i) sits at shared offset sbase + 8 j RWP + 32 i and global
// in-plane offset gbase + 8 j nx + 32 i; bit 2 (j * 2 + i) of `smask` says it
// is inside the staged tile, of `gmask` that it is also inside the volume.
// The loads of plane q + 1 are issued before plane q is box-summed.
constexpr int STAGE_NX = 2;
template <typename I>
struct Stage {
    int sbase;
    I gbase;
    unsigned smask, gmask;
};
template <int NY, typename I>
__device__ __forceinline__ Stage<I> make_stage(const LnccSmem &L, int r, int x0, int y0, const Dims &g) {
    Stage<I> S;
    const int tx = threadIdx.x, ty = threadIdx.y;
    S.sbase = ty * L.RWP + tx;
    S.gbase = (I)(y0 - r + ty) * g.nx + (x0 - r + tx);
    S.smask = S.gmask = 0u;
#pragma unroll
    for (int j = 0; j < NY; ++j)
#pragma unroll
        for (int i = 0; i < STAGE_NX; ++i) {
            const int xx = tx + TX * i, yy = ty + TY * j;
            const int gx = x0 - r + xx, gy = y0 - r + yy;
            const unsigned bit = 1u << (j * STAGE_NX + i);
            if (xx < L.RW && yy < L.RH) {
                S.smask |= bit;
                if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) S.gmask |= bit;
            }
        }
    return S;
}

// MODE: LNCC_FULL forms the five box sums of (F, J, F^2, J^2, FJ).
// LNCC_FCACHED forms the three of (J, J^2, FJ) and reads the window mean and
// variance of F from fstat ([2][N]; F is fixed during a registration, so they
// are formed once per run).  LNCC_FSTATS forms the two of (F, F^2) and writes
// that mean and variance to fstat (no J, no similarity).
constexpr int LNCC_FULL = 0, LNCC_FCACHED = 1, LNCC_FSTATS = 2;
template <int MODE>
__host__ __device__ constexpr int lncc_stats_k() {
    return MODE == LNCC_FULL ? 5 : (MODE == LNCC_FCACHED ? 3 : 2);
}

// (the three- and two-sum modes fit 4 CTAs per SM in 64 registers)
// (R as in lncc_sweep2_kernel: the window radius compiled in when >= 0)
template <typename T, bool COEF, typename I, int NY, int MODE = LNCC_FULL, int R = -1>
__global__ void __launch_bounds__(TILE_THREADS, MODE == LNCC_FULL ? 3 : 4)
    lncc_stats_kernel(const T *__restrict__ F, const float *__restrict__ J, Dims g, LnccParams P, int zc,
                      float *__restrict__ coef, float *__restrict__ fstat, double *__restrict__ partials,
                      unsigned *__restrict__ counter, double *__restrict__ sim_out, unsigned *err) {
    constexpr int K = lncc_stats_k<MODE>();
    constexpr bool HAS_J = MODE != LNCC_FSTATS;
    extern __shared__ float smem[];
    __shared__ double red[32];
    __shared__ float shift[2];
    const int r = R >= 0 ? R : P.r;
    const LnccSmem L(r, K);
    float *st = smem;
    float *hx = st + L.stage_words();
    float *ring = hx + L.hx_words();
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int z1 = min(g.nz, z0 + zc);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    const I nxy = (I)g.nxy;
    if (tid == 0) {
        const int cx = min(x0 + TX / 2, g.nx - 1), cy = min(y0 + TY / 2, g.ny - 1), cz = min(z0 + zc / 2, g.nz - 1);
        const I pc = (I)cz * nxy + (I)cy * g.nx + cx;
        shift[0] = ld_vox(F, pc);
        shift[1] = HAS_J ? __ldg(J + pc) : 0.0f;
    }
    for (int i = tid; i < L.ring_words(); i += TILE_THREADS) ring[i] = 0.0f;
    __syncthreads();
    const float shF = shift[0], shJ = shift[1];
    const float cxy = active ? (float)(win_count(x, r, g.nx) * win_count(y, r, g.ny)) : 1.0f;
    const float inv_n = 1.0f / (float)g.n;
    const int kst = L.RH * L.RWP;
    const XJobs xj = make_xjobs<K>(L, tid);
    const Stage<I> sg = make_stage<NY, I>(L, r, x0, y0, g);
    const I rowstep = (I)TY * g.nx;
    float pf[NY][STAGE_NX], pj[NY][STAGE_NX];
    auto fetch = [&](int q) {
        const bool qin = q >= 0 && q < g.nz;
        const I qoff = (I)q * nxy + sg.gbase;
#pragma unroll
        for (int j = 0; j < NY; ++j)
#pragma unroll
            for (int i = 0; i < STAGE_NX; ++i) {
                float f = 0.0f, jv = 0.0f;
                if (qin && (sg.gmask >> (j * STAGE_NX + i) & 1u)) {
                    const I p = qoff + (I)j * rowstep + TX * i;
                    f = ld_vox(F, p) - shF;
                    if (HAS_J) jv = __ldg(J + p) - shJ;
                }
                pf[j][i] = f;
                pj[j][i] = jv;
            }
    };
    fetch(z0 - r);
    float S[K];
#pragma unroll
    for (int k = 0; k < K; ++k) S[k] = 0.0f;
    float nsum = 0.0f;
    int slot = 0;
    // F's cached window mean and variance at the next output voxel, loaded
    // one output plane ahead
    float fm_q = 0.0f, fv_q = 0.0f;
    if (MODE == LNCC_FCACHED && active) {
        const I p0 = (I)z0 * nxy + (I)y * g.nx + x;
        fm_q = __ldg(fstat + p0);
        fv_q = __ldg(fstat + g.n + p0);
    }
    for (int q = z0 - r; q < z1 + r; ++q) {
#pragma unroll
        for (int j = 0; j < NY; ++j)
#pragma unroll
            for (int i = 0; i < STAGE_NX; ++i)
                if (sg.smask >> (j * STAGE_NX + i) & 1u) {
                    const int o = sg.sbase + j * TY * L.RWP + TX * i;
                    const float f = pf[j][i], jv = pj[j][i];
                    if (MODE == LNCC_FULL) {
                        st[o] = f;
                        st[kst + o] = jv;
                        st[2 * kst + o] = f * f;
                        st[3 * kst + o] = jv * jv;
                        st[4 * kst + o] = f * jv;
                    } else if (MODE == LNCC_FCACHED) {
                        st[o] = jv;
                        st[kst + o] = jv * jv;
                        st[2 * kst + o] = f * jv;
                    } else {
                        st[o] = f;
                        st[kst + o] = f * f;
                    }
                }
        if (q + 1 < z1 + r) fetch(q + 1);  // in flight during the box sums of plane q
        __syncthreads();
        xpass(st, hx, xj, r);
        float old[K];
#pragma unroll
        for (int k = 0; k < K; ++k) old[k] = ring[(slot * K + k) * TILE_THREADS + tid];
        __syncthreads();
        ypass<K>(hx, ring, slot, L, r, tid);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) S[k] += ring[(slot * K + k) * TILE_THREADS + tid] - old[k];
        slot = slot + 1 == L.W ? 0 : slot + 1;
        const int zo = q - r;
        if (active && zo >= z0 && zo < z1) {
            const float c = cxy * (float)win_count(zo, r, g.nz);
            const float ic = 1.0f / c;
            const I p = (I)zo * nxy + (I)y * g.nx + x;
            if (MODE == LNCC_FSTATS) {
                const float m = S[0] * ic;
                fstat[p] = m + shF;
                (fstat + g.n)[p] = fmaxf(fmaf(S[1], ic, -m * m), 0.0f);
                continue;
            }
            // means of the shifted values; A, B, C the window covariance and variances
            float mF, mJ, A, Bv, Cv;
            if (MODE == LNCC_FULL) {
                mF = S[0] * ic;
                mJ = S[1] * ic;
                A = fmaf(S[4], ic, -mF * mJ);
                Bv = fmaxf(fmaf(S[2], ic, -mF * mF), 0.0f);
                Cv = fmaxf(fmaf(S[3], ic, -mJ * mJ), 0.0f);
            } else {
                mF = fm_q - shF;
                Bv = fv_q;
                if (zo + 1 < z1) {
                    fm_q = __ldg(fstat + p + nxy);
                    fv_q = __ldg(fstat + g.n + p + nxy);
                }
                mJ = S[0] * ic;
                A = fmaf(S[2], ic, -mF * mJ);
                Cv = fmaxf(fmaf(S[1], ic, -mJ * mJ), 0.0f);
            }
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
                const float aJ = -(aFJ * (mF + shF) + 2.0f * aJJ * (mJ + shJ));
                coef[p] = aJ;
                (coef + g.n)[p] = aJJ;
                (coef + 2 * g.n)[p] = aFJ;
            }
        }
    }
    if (MODE == LNCC_FSTATS) return;
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

// AFF: the composite transform phi = A p + t + S u.  Without STEP (u and
// grad_out may be NULL): grad_out = S gX and r_out[12] = dC/dA, dC/dt.  With
// STEP: dC/du = S gX enters the diffusion + Adam update of u as usual.
// R >= 0: the window radius fixed at compile time (the index arithmetic of
// the staging and the x pass folds to constants); R < 0: P.r.
template <typename T, typename MT, bool STEP, int PAD, typename I, bool AFF = false, int R = -1>
__global__ void __launch_bounds__(TILE_THREADS)
    lncc_sweep2_kernel(const T *__restrict__ F, const T *__restrict__ M, const float *__restrict__ u, Dims g,
                       LnccParams P, int zc, const float *__restrict__ coef, float *__restrict__ grad_out,
                       float *__restrict__ u_out, MT *__restrict__ m, MT *__restrict__ v, StepParams S,
                       double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ r_out,
                       unsigned *err, AffineT Ain) {
    const AffineT A = AFF ? resolve_affine(Ain) : Ain;
    extern __shared__ float smem[];
    __shared__ double red[32];
    const int r = R >= 0 ? R : P.r;
    const LnccSmem L(r, 3);
    float *st = smem;
    float *hx = st + L.stage_words();
    float *ring = hx + L.hx_words();
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int z1 = min(g.nz, z0 + zc);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    const I nxy = (I)g.nxy, nx = (I)g.nx;
    for (int i = tid; i < L.ring_words(); i += TILE_THREADS) ring[i] = 0.0f;
    const float *uc[3] = {u, u + g.n, u + 2 * g.n};
    const float *cf[3] = {coef, coef + g.n, coef + 2 * g.n};
    MT *mc[3] = {m, m + g.n, m + 2 * g.n};
    MT *vc[3] = {v, v + g.n, v + 2 * g.n};
    const I col = active ? (I)y * nx + x : 0;
    const bool hxm = x > 0, hxp = x + 1 < g.nx, hym = y > 0, hyp = y + 1 < g.ny;
    float cur[3] = {0.f, 0.f, 0.f}, prv[3] = {0.f, 0.f, 0.f}, nxt[3] = {0.f, 0.f, 0.f};
    const bool has_u = !AFF || u != nullptr;  // the composite form may omit u
    AffineAcc aacc;
    // the output stage's own operands, one output plane ahead (they land
    // while the plane's box sums run): F, m, v at the next output voxel and
    // u two planes ahead (u at z + 1 is the diffusion stencil's)
    float fq = 0.0f, mq[3] = {0.f, 0.f, 0.f}, vq[3] = {0.f, 0.f, 0.f}, nx2[3] = {0.f, 0.f, 0.f};
    if (active) {
        const I p = (I)z0 * nxy + col;
        fq = ld_vox(F, p);
        if (has_u) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cur[c] = __ldg(uc[c] + p);
                if (STEP && z0 > 0) prv[c] = __ldg(uc[c] + p - nxy);
                if (z0 + 1 < g.nz) nxt[c] = __ldg(uc[c] + p + nxy);
            }
        }
        if (STEP) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                mq[c] = ld_moment(mc[c], p);
                vq[c] = ld_moment(vc[c], p);
            }
        }
    }
    __syncthreads();
    float Sa[3] = {0.f, 0.f, 0.f};
    float rpart = 0.0f;
    int slot = 0;
    const int plane = L.RH * L.RW;
    const int kst = L.RH * L.RWP;
    for (int q = z0 - r; q < z1 + r; ++q) {
        const bool qin = q >= 0 && q < g.nz;
        const I qoff = (I)q * nxy;
        for (int e = tid; e < plane; e += TILE_THREADS) {
            const int yy = e / L.RW, xx = e - yy * L.RW;
            const int gx = x0 - r + xx, gy = y0 - r + yy;
            float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
            if (qin && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
                const I p = qoff + (I)gy * nx + gx;
                a0 = __ldg(cf[0] + p);
                a1 = __ldg(cf[1] + p);
                a2 = __ldg(cf[2] + p);
            }
            const int o = yy * L.RWP + xx;
            st[o] = a0;
            st[kst + o] = a1;
            st[2 * kst + o] = a2;
        }
        __syncthreads();
        xpass_lean<3>(st, hx, L, r, tid);
        float old[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) old[k] = ring[(slot * 3 + k) * TILE_THREADS + tid];
        __syncthreads();
        ypass<3>(hx, ring, slot, L, r, tid);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k) Sa[k] += ring[(slot * 3 + k) * TILE_THREADS + tid] - old[k];
        slot = slot + 1 == L.W ? 0 : slot + 1;
        const int zo = q - r;
        if (active && zo >= z0 && zo < z1) {
            const I p = (I)zo * nxy + col;
            const float fv = fq;
            float m0[3], v0[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                m0[c] = mq[c];
                v0[c] = vq[c];
            }
            if (zo + 1 < z1) {
                fq = ld_vox(F, p + nxy);
                if (STEP) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        mq[c] = ld_moment(mc[c], p + nxy);
                        vq[c] = ld_moment(vc[c], p + nxy);
                    }
                }
                if (zo + 2 < g.nz && has_u) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) nx2[c] = __ldg(uc[c] + p + 2 * nxy);
                }
            }
            float sx, sy, sz, qx = cur[0], qy = cur[1], qz = cur[2];
            if (AFF) composite_disp(A, x, y, zo, qx, qy, qz);
            const float jv = sample_grad<T, PAD, I>(M, g, x, y, zo, qx, qy, qz, sx, sy, sz);
            const float gj = fmaf(fv, Sa[2], fmaf(2.0f * jv, Sa[1], Sa[0]));
            const float gs[3] = {gj * sx, gj * sy, gj * sz};
            if (STEP) {
                float gR[3];
                diffusion_ptr<I>(uc, p, nx, hxm, hxp, hym, hyp, zo > 0, zo + 1 < g.nz, cur, prv, nxt, gR, rpart);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float gt = fmaf(S.lam * S.two_over_n, gR[c], AFF ? A.s[c] * gs[c] : gs[c]);
                    if (grad_out) (grad_out + c * g.n)[p] = gt;
                    (u_out + c * g.n)[p] = adam_fast(cur[c], gt, m0[c], v0[c], mc[c], vc[c], p, S);
                }
            } else if (AFF) {
                aacc.add(gs[0], gs[1], gs[2], zo);
                if (grad_out) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) (grad_out + c * g.n)[p] = A.s[c] * gs[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) (grad_out + c * g.n)[p] = gs[c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                prv[c] = cur[c];
                cur[c] = nxt[c];
                nxt[c] = nx2[c];
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

// Sweep 2 with the ANTs gradient approximation (App. fused LNCC): no second
// box sum, each voxel uses the coefficients of its own window,
//   dL/dJ_k = c_k (a_J + 2 J_k a_JJ + F_k a_FJ)_k,
// so the sweep streams the coefficient fields like the MI sweep streams its
// inputs (plane-ahead prefetch of u, F, the coefficients and the moments).
template <typename T, typename MT, bool STEP, int PAD, typename I, bool AFF = false>
__global__ void __launch_bounds__(TILE_THREADS, 4)
    lncc_sweep2_ants_kernel(const T *__restrict__ F, const T *__restrict__ M, const float *__restrict__ u, Dims g,
                            LnccParams P, int zc, const float *__restrict__ coef, float *__restrict__ grad_out,
                            float *__restrict__ u_out, MT *__restrict__ m, MT *__restrict__ v, StepParams S,
                            double *__restrict__ partials, unsigned *__restrict__ counter,
                            double *__restrict__ r_out, unsigned *err, AffineT Ain) {
    const AffineT A = AFF ? resolve_affine(Ain) : Ain;
    __shared__ double red[32];
    const int r = P.r;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(g.nz, z0 + zc);
    float rpart = 0.0f;
    AffineAcc aacc;
    const bool has_u = !AFF || u != nullptr;
    if (x < g.nx && y < g.ny) {
        const float *uc[3] = {u, u + g.n, u + 2 * g.n};
        const float *cf[3] = {coef, coef + g.n, coef + 2 * g.n};
        MT *mc[3] = {m, m + g.n, m + 2 * g.n};
        MT *vc[3] = {v, v + g.n, v + 2 * g.n};
        const I nxy = (I)g.nxy, nx = (I)g.nx;
        I p = (I)z0 * nxy + (I)y * nx + x;
        const bool hxm = x > 0, hxp = x + 1 < g.nx, hym = y > 0, hyp = y + 1 < g.ny;
        const float cxy = (float)(win_count(x, r, g.nx) * win_count(y, r, g.ny));
        float cur[3], prv[3] = {0.f, 0.f, 0.f}, nxt[3] = {0.f, 0.f, 0.f};
        float fcur, acur[3], mcur[3] = {0.f, 0.f, 0.f}, vcur[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cur[c] = has_u ? __ldg(uc[c] + p) : 0.0f;
            acur[c] = __ldg(cf[c] + p);
        }
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
            float fnxt = 0.0f, anxt[3] = {0.f, 0.f, 0.f}, mnxt[3] = {0.f, 0.f, 0.f}, vnxt[3] = {0.f, 0.f, 0.f};
            if (z + 1 < g.nz && has_u) {
#pragma unroll
                for (int c = 0; c < 3; ++c) nxt[c] = __ldg(uc[c] + p + nxy);
            }
            if (z + 1 < z1) {
                fnxt = ld_vox(F, p + nxy);
#pragma unroll
                for (int c = 0; c < 3; ++c) anxt[c] = __ldg(cf[c] + p + nxy);
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
            const float ck = cxy * (float)win_count(z, r, g.nz);
            const float gj = ck * fmaf(fcur, acur[2], fmaf(2.0f * jv, acur[1], acur[0]));
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
                acur[c] = anxt[c];
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

// Every CTA marches zc + 2r planes (its chunk plus the window's warm-up), one
// plane after the other, so the launch takes about
//     waves x (zc + 2r)   plane steps,   waves = ceil(tiles x chunks / resident CTAs).
// The chunk count minimises that (the fewest chunks on ties: less warm-up
// traffic).  A small volume gets as many chunks as one wave holds; a large one
// long chunks, cut so that the last wave is not left mostly idle.  At most
// LNCC_MAX_CHUNKS chunks, at least 2 planes each.
constexpr long long LNCC_MAX_CHUNKS = 64;
static long long lncc_chunk_cap(const Dims &g) {
    const long long half = (g.nz + 1) / 2;
    return std::max(1LL, std::min(LNCC_MAX_CHUNKS, half));
}
MarchGrid lncc_grid(const Dims &g, int r, int per_sm) {
    const long long tiles = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    const long long slots = (long long)per_sm * num_sms();
    long long best_c = 1, best = -1;
    for (long long c = 1; c <= lncc_chunk_cap(g); ++c) {
        const long long zc = (g.nz + c - 1) / c, chunks = (g.nz + zc - 1) / zc;
        const long long waves = (tiles * chunks + slots - 1) / slots;
        const long long cost = waves * (zc + 2 * r);
        if (best < 0 || cost < best) {
            best = cost;
            best_c = c;
        }
    }
    return march_grid(g, best_c * tiles, 1);
}
long long lncc_max_blocks(const Dims &g) {
    const long long tiles = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    return tiles * lncc_chunk_cap(g);
}

// CTAs of `kernel` (TILE_THREADS threads, `smem` dynamic bytes) resident per
// SM on the current device, cached per (kernel, smem, device)
template <typename K>
static int resident_per_sm(K kernel, size_t smem) {
    struct Entry {
        const void *fn;
        size_t smem;
        int dev, n;
    };
    static std::mutex mu;
    static Entry cache[64];
    static int used = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
        if (cache[i].fn == (const void *)kernel && cache[i].smem == smem && cache[i].dev == dev) return cache[i].n;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, TILE_THREADS, smem) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = 1;
    }
    if (n > LNCC_MAX_PER_SM) n = LNCC_MAX_PER_SM;
    if (used < 64) cache[used++] = Entry{(const void *)kernel, smem, dev, n};
    return n;
}
// the streaming (ANTs) sweep has no warm-up planes: the MI sweep's grid
MarchGrid lncc_ants_grid(const Dims &g) { return march_grid(g, 8LL * num_sms() * 4, 1); }

// staged rows per thread: TY + 2r <= 16 rows fit in 2 passes of 8
template <typename Fn>
inline void with_stage_rows(int r, Fn &&fn) {
    if (TY + 2 * r <= 2 * TY)
        fn(IC<2>{});
    else
        fn(IC<3>{});
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// opt `kernel` in to `smem` bytes and size its grid by its residency
template <typename K>
static cudaError_t prepare_march(K kernel, size_t smem, const Dims &g, int r, MarchGrid &G, dim3 &grid) {
    const cudaError_t e = allow_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    G = lncc_grid(g, r, resident_per_sm(kernel, smem));
    grid = dim3(G.tiles_x, G.tiles_y, G.chunks);
    return cudaSuccess;
}

cudaError_t launch_lncc_stats(const void *F, const float *J, int dt, const Dims &g, const LnccParams &P, float *coef,
                              double *partials, unsigned *counter, double *sim_out, cudaStream_t s,
                              const float *fstat) {
    MarchGrid G;
    dim3 grid;
    const dim3 block(TX, TY);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    cudaError_t e = cudaSuccess;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_index(g, [&](auto ip) {
            using I = elem_t<decltype(ip)>;
            with_stage_rows(P.r, [&](auto ny) {
                constexpr int NY = decltype(ny)::value;
                auto run = [&](auto kern, int K) {
                    const size_t smem = lncc_smem_bytes(P.r, K);
                    e = prepare_march(kern, smem, g, P.r, G, grid);
                    if (e == cudaSuccess)
                        kern<<<grid, block, smem, s>>>((const T *)F, J, g, P, G.zc, coef, (float *)fstat, partials,
                                                       counter, sim_out, err);
                };
                if (fstat) {  // F's window statistics formed beforehand (launch_lncc_fstats)
                    // the workloads' windows (7^3, 9^3) with their radius compiled in
                    if (coef && P.r == 4 && NY == 2)
                        run(lncc_stats_kernel<T, true, I, 2, LNCC_FCACHED, 4>, lncc_stats_k<LNCC_FCACHED>());
                    else if (coef && P.r == 3 && NY == 2)
                        run(lncc_stats_kernel<T, true, I, 2, LNCC_FCACHED, 3>, lncc_stats_k<LNCC_FCACHED>());
                    else if (coef)
                        run(lncc_stats_kernel<T, true, I, NY, LNCC_FCACHED>, lncc_stats_k<LNCC_FCACHED>());
                    else
                        run(lncc_stats_kernel<T, false, I, NY, LNCC_FCACHED>, lncc_stats_k<LNCC_FCACHED>());
                } else if (coef && P.r == 4 && NY == 2) {
                    run(lncc_stats_kernel<T, true, I, 2, LNCC_FULL, 4>, lncc_stats_k<LNCC_FULL>());
                } else if (coef && P.r == 3 && NY == 2) {
                    run(lncc_stats_kernel<T, true, I, 2, LNCC_FULL, 3>, lncc_stats_k<LNCC_FULL>());
                } else if (coef) {
                    run(lncc_stats_kernel<T, true, I, NY>, lncc_stats_k<LNCC_FULL>());
                } else {
                    run(lncc_stats_kernel<T, false, I, NY>, lncc_stats_k<LNCC_FULL>());
                }
            });
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_lncc_fstats(const void *F, int dt, const Dims &g, const LnccParams &P, float *fstat,
                               cudaStream_t s) {
    MarchGrid G;
    dim3 grid;
    const dim3 block(TX, TY);
    const size_t smem = lncc_smem_bytes(P.r, lncc_stats_k<LNCC_FSTATS>());
    cudaError_t e = cudaSuccess;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_index(g, [&](auto ip) {
            using I = elem_t<decltype(ip)>;
            with_stage_rows(P.r, [&](auto ny) {
                constexpr int NY = decltype(ny)::value;
                auto kern = lncc_stats_kernel<T, false, I, NY, LNCC_FSTATS>;
                e = prepare_march(kern, smem, g, P.r, G, grid);
                if (e == cudaSuccess)
                    kern<<<grid, block, smem, s>>>((const T *)F, nullptr, g, P, G.zc, nullptr, fstat, nullptr,
                                                   nullptr, nullptr, nullptr);
            });
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

static cudaError_t launch_lncc_sweep2_ants(const void *F, const void *M, int dt, const float *u, const Dims &g,
                                           int pad, const LnccParams &P, const float *coef, float *grad_out,
                                           bool step, float *u_out, void *m, void *v, int mdt, const StepParams &S,
                                           double *partials, unsigned *counter, double *r_out, cudaStream_t s,
                                           const AffineT *aff) {
    const MarchGrid G = lncc_ants_grid(g);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    const AffineT A = aff ? *aff : AffineT{};
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            if (aff && !step) {  // the composite form: gradients only, 64-bit offsets
                lncc_sweep2_ants_kernel<T, float, false, PD, long long, true><<<grid, block, 0, s>>>(
                    (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, nullptr, nullptr, nullptr, S,
                    partials, counter, r_out, err, A);
                return;
            }
            if (aff) {  // the composite form with the step
                with_type(mdt, [&](auto mp) {
                    using MT = elem_t<decltype(mp)>;
                    lncc_sweep2_ants_kernel<T, MT, true, PD, long long, true><<<grid, block, 0, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (MT *)m, (MT *)v, S,
                        partials, counter, r_out, err, A);
                });
                return;
            }
            with_index(g, [&](auto ip) {
                using I = elem_t<decltype(ip)>;
                if (!step) {
                    lncc_sweep2_ants_kernel<T, float, false, PD, I><<<grid, block, 0, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (float *)m, (float *)v, S,
                        partials, counter, r_out, err, A);
                    return;
                }
                with_type(mdt, [&](auto mp) {
                    using MT = elem_t<decltype(mp)>;
                    lncc_sweep2_ants_kernel<T, MT, true, PD, I><<<grid, block, 0, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (MT *)m, (MT *)v, S,
                        partials, counter, r_out, err, A);
                });
            });
        });
    });
    return cudaGetLastError();
}

cudaError_t launch_lncc_sweep2(const void *F, const void *M, int dt, const float *u, const Dims &g, int pad,
                               const LnccParams &P, const float *coef, float *grad_out, bool step,
                               float *u_out, void *m, void *v, int mdt, const StepParams &S,
                               double *partials, unsigned *counter, double *r_out, cudaStream_t s,
                               const AffineT *aff) {
    if (P.ants)
        return launch_lncc_sweep2_ants(F, M, dt, u, g, pad, P, coef, grad_out, step, u_out, m, v, mdt, S, partials,
                                       counter, r_out, s, aff);
    const AffineT A = aff ? *aff : AffineT{};
    MarchGrid G;
    dim3 grid;
    const dim3 block(TX, TY);
    const size_t smem = lncc_smem_bytes(P.r, 3);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    cudaError_t e = cudaSuccess;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            if (aff && !step) {  // the composite form: gradients only, 64-bit offsets
                e = prepare_march(lncc_sweep2_kernel<T, float, false, PD, long long, true>, smem, g, P.r, G, grid);
                if (e == cudaSuccess)
                    lncc_sweep2_kernel<T, float, false, PD, long long, true><<<grid, block, smem, s>>>(
                        (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, nullptr, nullptr, nullptr, S,
                        partials, counter, r_out, err, A);
                return;
            }
            if (aff) {  // the composite form with the step
                with_type(mdt, [&](auto mp) {
                    using MT = elem_t<decltype(mp)>;
                    e = prepare_march(lncc_sweep2_kernel<T, MT, true, PD, long long, true>, smem, g, P.r, G, grid);
                    if (e == cudaSuccess)
                        lncc_sweep2_kernel<T, MT, true, PD, long long, true><<<grid, block, smem, s>>>(
                            (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (MT *)m, (MT *)v, S,
                            partials, counter, r_out, err, A);
                });
                return;
            }
            with_index(g, [&](auto ip) {
                using I = elem_t<decltype(ip)>;
                if (!step) {
                    e = prepare_march(lncc_sweep2_kernel<T, float, false, PD, I>, smem, g, P.r, G, grid);
                    if (e == cudaSuccess)
                        lncc_sweep2_kernel<T, float, false, PD, I><<<grid, block, smem, s>>>(
                            (const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out, u_out, (float *)m,
                            (float *)v, S, partials, counter, r_out, err, A);
                    return;
                }
                with_type(mdt, [&](auto mp) {
                    using MT = elem_t<decltype(mp)>;
                    auto go = [&](auto kern) {
                        e = prepare_march(kern, smem, g, P.r, G, grid);
                        if (e == cudaSuccess)
                            kern<<<grid, block, smem, s>>>((const T *)F, (const T *)M, u, g, P, G.zc, coef, grad_out,
                                                           u_out, (MT *)m, (MT *)v, S, partials, counter, r_out, err,
                                                           A);
                    };
                    // the windows of the workloads (7^3, 9^3) with their radius compiled in
                    if (P.r == 4)
                        go(lncc_sweep2_kernel<T, MT, true, PD, I, false, 4>);
                    else if (P.r == 3)
                        go(lncc_sweep2_kernel<T, MT, true, PD, I, false, 3>);
                    else
                        go(lncc_sweep2_kernel<T, MT, true, PD, I>);
                });
            });
        });
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace regk
