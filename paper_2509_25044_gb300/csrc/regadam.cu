// regadam.cu -- diffusion regulariser, Adam step, Jacobian-determinant fold
// check, the device error word and the bounded-wait test hook.
#include <mutex>

#include "kernels.h"

namespace regk {

__device__ unsigned int g_reg_error = 0u;

// The word's device address, looked up once per device (with that device
// current) under a lock; nullptr when the runtime cannot give it, which the
// launchers turn into an error return.  The cache outlives a
// cudaDeviceReset: a process that resets a device must not call the library
// on it again.
unsigned *error_word() {
    static std::mutex lock;
    static unsigned *cached[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> guard(lock);
    if (!cached[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reg_error) != cudaSuccess) return nullptr;
        cached[dev] = (unsigned *)p;
    }
    return cached[dev];
}

int num_sms() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            cached = n;
        else
            cached = 152;
    }
    return cached;
}

MarchGrid march_grid(const Dims &g, long long target_blocks, int min_zc, int max_zc) {
    MarchGrid G;
    G.tiles_x = (g.nx + TX - 1) / TX;
    G.tiles_y = (g.ny + TY - 1) / TY;
    const long long tiles = (long long)G.tiles_x * G.tiles_y;
    long long chunks = (target_blocks + tiles - 1) / tiles;
    const long long max_chunks = (g.nz + min_zc - 1) / min_zc;
    if (chunks > max_chunks) chunks = max_chunks;
    const long long min_chunks = (g.nz + max_zc - 1) / max_zc;
    if (chunks < min_chunks) chunks = min_chunks;
    if (chunks < 1) chunks = 1;
    G.zc = (int)((g.nz + chunks - 1) / chunks);
    G.chunks = (g.nz + G.zc - 1) / G.zc;
    return G;
}

MarchGrid diffusion_grid(const Dims &g) { return march_grid(g, 8LL * num_sms() * 4, 1); }

// ---------------------------------------------------------------------------
// diffusion regulariser: value (FP64 fixed-order sum) and lambda * dR/du
// added into grad (grad may be null)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE_THREADS)
    diffusion_kernel(const float *__restrict__ u, Dims g, int zc, float scale, float *__restrict__ grad,
                     double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ r_out,
                     unsigned *err) {
    __shared__ double red[32];
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    float rpart = 0.0f;
    if (x < g.nx && y < g.ny) {
        const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
        const long long col = (long long)y * g.nx + x;
        float cur[3], prv[3] = {0.f, 0.f, 0.f}, nxt[3] = {0.f, 0.f, 0.f};
        const long long p0 = (long long)z0 * g.nxy + col;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cur[c] = __ldg(u + c * g.n + p0);
            if (z0 > 0) prv[c] = __ldg(u + c * g.n + p0 - g.nxy);
        }
        for (int z = z0; z < z1; ++z) {
            const long long p = (long long)z * g.nxy + col;
            if (z + 1 < g.nz) {
#pragma unroll
                for (int c = 0; c < 3; ++c) nxt[c] = __ldg(u + c * g.n + p + g.nxy);
            }
            float gR[3];
            diffusion_at(u, g, x, y, z, p, cur, prv, nxt, gR, rpart);
            if (grad) {
#pragma unroll
                for (int c = 0; c < 3; ++c) grad[c * g.n + p] = fmaf(scale, gR[c], grad[c * g.n + p]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                prv[c] = cur[c];
                cur[c] = nxt[c];
            }
        }
    }
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

cudaError_t launch_diffusion(const float *u, const Dims &g, float lam, float *grad, double *partials,
                             unsigned *counter, double *r_out, cudaStream_t s) {
    const MarchGrid G = diffusion_grid(g);
    const float scale = (float)((double)lam * 2.0 / (double)g.n);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    diffusion_kernel<<<dim3(G.tiles_x, G.tiles_y, G.chunks), dim3(TX, TY), 0, s>>>(u, g, G.zc, scale, grad,
                                                                                   partials, counter, r_out, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam over the 3N displacement components
// ---------------------------------------------------------------------------
template <typename MT>
__global__ void __launch_bounds__(256) adam_kernel(const float *__restrict__ u_in, float *u_out, MT *m, MT *v,
                                                  const float *__restrict__ grad, long long n3, StepParams S) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long long)gridDim.x * blockDim.x) {
        const float uu = u_in[i];
        u_out[i] = adam_elem(uu, __ldg(grad + i), m, v, i, S);
    }
}

cudaError_t launch_adam(const float *u_in, float *u_out, void *m, void *v, int mdt, const float *grad, long long n3,
                        const StepParams &S, cudaStream_t s) {
    long long blocks = (n3 + 255) / 256;
    const long long cap = 16LL * num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (mdt == REG_BF16)
        adam_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(u_in, u_out, (__nv_bfloat16 *)m,
                                                                     (__nv_bfloat16 *)v, grad, n3, S);
    else
        adam_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(u_in, u_out, (float *)m, (float *)v, grad, n3, S);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// det(I + grad u): central differences, one-sided at the border
// ---------------------------------------------------------------------------
__global__ void jacdet_init_kernel(float *min_out, unsigned long long *nfold) {
    min_out[0] = __int_as_float(0x7f800000);  // +inf
    nfold[0] = 0ull;
}

__device__ __forceinline__ void atomic_min_float(float *addr, float val) {
    if (val >= 0.0f)
        atomicMin((int *)addr, __float_as_int(val));
    else
        atomicMax((unsigned *)addr, __float_as_uint(val));
}

__device__ __forceinline__ float central(const float *uc, long long p, int coord, int n, long long stride) {
    if (n == 1) return 0.0f;
    const int lo = coord > 0 ? coord - 1 : coord;
    const int hi = coord < n - 1 ? coord + 1 : coord;
    const float a = __ldg(uc + p + (long long)(hi - coord) * stride);
    const float b = __ldg(uc + p - (long long)(coord - lo) * stride);
    return (a - b) / (float)(hi - lo);
}

__global__ void __launch_bounds__(TILE_THREADS) jacdet_kernel(const float *__restrict__ u, Dims g, int zc,
                                                              float *min_out, unsigned long long *nfold) {
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    float mn = __int_as_float(0x7f800000);
    unsigned cnt = 0;
    if (x < g.nx && y < g.ny) {
        const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
        for (int z = z0; z < z1; ++z) {
            const long long p = (long long)z * g.nxy + (long long)y * g.nx + x;
            float Jm[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *uc = u + c * g.n;
                Jm[c][0] = central(uc, p, x, g.nx, 1) + (c == 0 ? 1.0f : 0.0f);
                Jm[c][1] = central(uc, p, y, g.ny, g.nx) + (c == 1 ? 1.0f : 0.0f);
                Jm[c][2] = central(uc, p, z, g.nz, g.nxy) + (c == 2 ? 1.0f : 0.0f);
            }
            const float det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                              Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                              Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
            if (!(det > 0.0f)) ++cnt;
            if (det == det) mn = fminf(mn, det);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_min_float(min_out, mn);
        if (cnt) atomicAdd(nfold, (unsigned long long)cnt);
    }
}

cudaError_t launch_jacdet(const float *u, const Dims &g, float *min_out, unsigned long long *nfold,
                          cudaStream_t s) {
    jacdet_init_kernel<<<1, 1, 0, s>>>(min_out, nfold);
    const MarchGrid G = march_grid(g, 8LL * num_sms() * 4, 1);
    jacdet_kernel<<<dim3(G.tiles_x, G.tiles_y, G.chunks), dim3(TX, TY), 0, s>>>(u, g, G.zc, min_out, nfold);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bounded device wait (failure-detection test hook)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void wait_flag_kernel(const unsigned *flag, unsigned expect, unsigned long long timeout_ns, unsigned *err) {
    const unsigned long long t0 = global_ns();
    // iteration cap as a second bound in case the timer does not advance
    for (long long it = 0; it < (1LL << 24); ++it) {
        if (*(volatile const unsigned *)flag == expect) return;
        if (global_ns() - t0 > timeout_ns) break;
        __nanosleep(1000);
    }
    latch_error(err, REG_ERR_TIMEOUT);
}

cudaError_t launch_wait_flag(const unsigned *flag, unsigned expect, unsigned long long timeout_ns, cudaStream_t s) {
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    wait_flag_kernel<<<1, 1, 0, s>>>(flag, expect, timeout_ns, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam on the 12 parameters of the affine stage (the optimiser state m1, m2 of
// Sec. 3.1 for phi(p) = A (p - c) + c + tc / s), in FP64 on one thread, fed by
// the fixed-order sums dC/dA, dC/dt of the composite sweeps:
//   dC/dA at fixed tc = dC/dA - (dC/dt) c^T,   dC/dtc = (dC/dt) / s,
// then Adam with bias correction, the step scaled by `decay`, tc's step by s
// (tc is in voxels of the finest grid).  state: A (9), tc (3), m_A (9),
// v_A (9), m_t (3), v_t (3).  T_dev receives the next transform in the layout
// of reg_affine: A, t = c - A c + tc / s, s = 1.
// ---------------------------------------------------------------------------
__global__ void affine_adam_kernel(const double *__restrict__ ga, const double *__restrict__ sim,
                                   double *__restrict__ st, float *__restrict__ T, AffineAdam P,
                                   double *__restrict__ obj) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (obj) obj[0] = P.lncc ? 1.0 - sim[0] : -sim[0];
    double *A = st, *tc = st + 9, *mA = st + 12, *vA = st + 21, *mt = st + 30, *vt = st + 33;
    const double gt[3] = {ga[9], ga[10], ga[11]};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int e = 3 * i + j;
            const double g = ga[e] - gt[i] * P.c[j];
            mA[e] = P.b1 * mA[e] + (1.0 - P.b1) * g;
            vA[e] = P.b2 * vA[e] + (1.0 - P.b2) * g * g;
            A[e] -= P.decay * P.lr_A * (mA[e] / P.bc1) / (sqrt(vA[e] / P.bc2) + P.eps);
        }
    for (int i = 0; i < 3; ++i) {
        const double g = gt[i] / P.scale;
        mt[i] = P.b1 * mt[i] + (1.0 - P.b1) * g;
        vt[i] = P.b2 * vt[i] + (1.0 - P.b2) * g * g;
        tc[i] -= P.decay * P.lr_t * P.scale * (mt[i] / P.bc1) / (sqrt(vt[i] / P.bc2) + P.eps);
    }
    for (int i = 0; i < 3; ++i) {
        const double Ac = A[3 * i] * P.c[0] + A[3 * i + 1] * P.c[1] + A[3 * i + 2] * P.c[2];
        for (int j = 0; j < 3; ++j) T[3 * i + j] = (float)A[3 * i + j];
        T[9 + i] = (float)(P.c[i] - Ac + tc[i] / P.scale);
        T[12 + i] = 1.0f;
    }
}

cudaError_t launch_affine_adam(const double *grad_affine, const double *sim, double *state, float *T_dev,
                               const AffineAdam &P, double *obj_out, cudaStream_t s) {
    affine_adam_kernel<<<1, 32, 0, s>>>(grad_affine, sim, state, T_dev, P, obj_out);
    return cudaGetLastError();
}

}  // namespace regk
