// unet.cu -- BF16 implicit-GEMM 3-D convolutions on the 5th-generation
// tensor cores (tcgen05, FP32 accumulation in TMEM) and the small
// elementwise / resampling kernels of the learned initialiser (a 3-D U-Net
// that predicts a half-resolution displacement from a downsampled pair).
//
// Activations are channels-last BF16 ([nz][ny][nx][C], C a multiple of 8),
// so 8 consecutive channels of one voxel are one 16-byte load -- exactly one
// row of a tensor-core core matrix.
#include "gemm_tc.cuh"
#include "kernels.h"

namespace regk {

// ---------------------------------------------------------------------------
// test hook: C[M x N] = A B^T through the tensor-core mainloop
//   a_mn == 0: A is [M][K] (K contiguous), else [K][M]; likewise B with N.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GEMM_THREADS) gemm_test_kernel(const __nv_bfloat16 *__restrict__ A,
                                                                 const __nv_bfloat16 *__restrict__ B,
                                                                 float *__restrict__ C, int M, int N, int K, int a_mn,
                                                                 int b_mn, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    GemmShared &sh = *reinterpret_cast<GemmShared *>(gsm);
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * GEMM_M;
    gemm_setup(sh, N);
    auto fillA = [&](int c, unsigned char *as) {
        if (!a_mn) {
            for (int u = tid; u < GEMM_M * GEMM_KG; u += GEMM_THREADS) {
                const int row = u / GEMM_KG, kg = u % GEMM_KG;
                const uint4 v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + row) * K + c * GEMM_KC + kg * 8);
                *reinterpret_cast<uint4 *>(as + kmajor_off(row, kg * 8)) = v;
            }
        } else {
            for (int u = tid; u < (GEMM_M / 8) * GEMM_KC; u += GEMM_THREADS) {
                const int g = u / GEMM_KC, k = u % GEMM_KC;
                const uint4 v = *reinterpret_cast<const uint4 *>(A + (size_t)(c * GEMM_KC + k) * M + m0 + g * 8);
                *reinterpret_cast<uint4 *>(as + mnmajor_row_off(g * 8, k)) = v;
            }
        }
    };
    auto fillB = [&](int c, unsigned char *bs) {
        if (!b_mn) {
            for (int u = tid; u < N * GEMM_KG; u += GEMM_THREADS) {
                const int row = u / GEMM_KG, kg = u % GEMM_KG;
                const uint4 v = *reinterpret_cast<const uint4 *>(B + (size_t)row * K + c * GEMM_KC + kg * 8);
                *reinterpret_cast<uint4 *>(bs + kmajor_off(row, kg * 8)) = v;
            }
        } else {
            for (int u = tid; u < (N / 8) * GEMM_KC; u += GEMM_THREADS) {
                const int g = u / GEMM_KC, k = u % GEMM_KC;
                const uint4 v = *reinterpret_cast<const uint4 *>(B + (size_t)(c * GEMM_KC + k) * N + g * 8);
                *reinterpret_cast<uint4 *>(bs + mnmajor_row_off(g * 8, k)) = v;
            }
        }
    };
    const bool ok = gemm_mainloop(sh, N, K / GEMM_KC, a_mn, b_mn, fillA, fillB);
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            gemm_row16(sh, c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) C[(size_t)(m0 + tid) * N + c0 + i] = v[i];
        }
    } else if (tid == 0) {
        latch_error(err, REG_ERR_TIMEOUT);
    }
    gemm_teardown(sh, N);
}

size_t gemm_smem_bytes() { return sizeof(GemmShared) + 1024; }

cudaError_t launch_gemm_test(const void *A, const void *B, float *C, int M, int N, int K, int a_mn, int b_mn,
                             cudaStream_t s) {
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    const size_t smem = gemm_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(gemm_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_test_kernel<<<M / GEMM_M, GEMM_THREADS, smem, s>>>((const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, C, M,
                                                            N, K, a_mn, b_mn, err);
    return cudaGetLastError();
}

}  // namespace regk

namespace regk {

// ---------------------------------------------------------------------------
// implicit-GEMM convolution, 3 x 3 x 3 taps, zero padding 1, stride 1
//   activations: channels-last BF16, C % 8 == 0
//   weights    : packed BF16 [n_rows][Kpad], k = tap * Cin + cin,
//                tap = (kz * 3 + ky) * 3 + kx (offset (kx-1, ky-1, kz-1)),
//                Kpad = 64 * ceil(27 Cin / 64), unused entries zero
// ---------------------------------------------------------------------------
struct ConvGeom {
    int nx, ny, nz;
    long long nvox;
};

__device__ __forceinline__ void vox_xyz(long long v, const ConvGeom &g, int &x, int &y, int &z) {
    const long long r = v / g.nx;
    x = (int)(v - r * g.nx);
    z = (int)(r / g.ny);
    y = (int)(r - (long long)z * g.ny);
}

// 16 bytes (8 channels) of voxel (x+dx, y+dy, z+dz), or zeros outside the volume
__device__ __forceinline__ uint4 tap_load(const __nv_bfloat16 *__restrict__ act, const ConvGeom &g, int C, int x,
                                          int y, int z, int tap, int c0) {
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    const int xx = x + dx, yy = y + dy, zz = z + dz;
    if ((unsigned)xx >= (unsigned)g.nx || (unsigned)yy >= (unsigned)g.ny || (unsigned)zz >= (unsigned)g.nz)
        return make_uint4(0, 0, 0, 0);
    const long long v = ((long long)zz * g.ny + yy) * g.nx + xx;
    return __ldg(reinterpret_cast<const uint4 *>(act + v * C + c0));
}


// forward conv (also the data gradient, with transposed / flipped weights):
// out[v][n] = epi( sum_k in_col[v][k] W[n][k] ), one CTA per 128 voxels
template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS)
    conv_fwd_kernel(const __nv_bfloat16 *__restrict__ in, int Cin, const __nv_bfloat16 *__restrict__ W, int Kpad,
                    const float *__restrict__ bias, int Cout, int N, ConvGeom g, float slope, void *__restrict__ out,
                    unsigned *err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    GemmShared &sh = *reinterpret_cast<GemmShared *>(gsm);
    const int tid = threadIdx.x;
    const long long m0 = (long long)blockIdx.x * GEMM_M;
    const long long v = m0 + tid;
    const bool vin = v < g.nvox;
    int x = 0, y = 0, z = 0;
    if (vin) vox_xyz(v, g, x, y, z);
    const int K = 27 * Cin;
    gemm_setup(sh, N);
    auto fillA = [&](int c, unsigned char *as) {
        // thread tid owns tile row tid (its voxel); 8 core-matrix columns per chunk
#pragma unroll
        for (int kg = 0; kg < GEMM_KG; ++kg) {
            const int k = c * GEMM_KC + kg * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (vin && k < K) val = tap_load(in, g, Cin, x, y, z, k / Cin, k % Cin);
            *reinterpret_cast<uint4 *>(as + kmajor_off(tid, kg * 8)) = val;
        }
    };
    auto fillB = [&](int c, unsigned char *bs) {
        for (int u = tid; u < N * GEMM_KG; u += GEMM_THREADS) {
            const int row = u / GEMM_KG, kg = u % GEMM_KG;
            const uint4 val = __ldg(reinterpret_cast<const uint4 *>(W + (size_t)row * Kpad + c * GEMM_KC + kg * 8));
            *reinterpret_cast<uint4 *>(bs + kmajor_off(row, kg * 8)) = val;
        }
    };
    const bool ok = gemm_mainloop(sh, N, Kpad / GEMM_KC, 0, 0, fillA, fillB);
    if (!ok && tid == 0) latch_error(err, REG_ERR_TIMEOUT);
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float acc[16];
            gemm_row16(sh, c0, acc);
            if (!vin) continue;
            if (EPI == EPI_BIAS_F32_SOA) {
                float *o = reinterpret_cast<float *>(out);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < Cout) o[(size_t)(c0 + i) * g.nvox + v] = acc[i] + bias[c0 + i];
            } else {
                __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out) + v * Cout;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (c0 + 8 * h >= Cout) continue;
                    __align__(16) __nv_bfloat16 t[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float a = acc[8 * h + i];
                        if (EPI == EPI_BIAS_LEAKY_BF16) {
                            a += bias[c0 + 8 * h + i];
                            a = a > 0.0f ? a : slope * a;
                        }
                        t[i] = __float2bfloat16_rn(a);
                    }
                    *reinterpret_cast<uint4 *>(o + c0 + 8 * h) = *reinterpret_cast<const uint4 *>(t);
                }
            }
        }
    }
    gemm_teardown(sh, N);
}

// weight gradient, split over voxel ranges:
//   part[split][k][n] = sum_{v in split} in_col[v][k] dpre[v][n]
// A (rows k, K = voxels) and B (rows n, K = voxels) are MN-major tiles: each
// 16-byte core-matrix row is 8 channels of one voxel.
__global__ void __launch_bounds__(GEMM_THREADS)
    conv_wgrad_kernel(const __nv_bfloat16 *__restrict__ in, int Cin, const __nv_bfloat16 *__restrict__ dpre, int Cout,
                      ConvGeom g, long long vox_per_split, float *__restrict__ part, int Mrows, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    GemmShared &sh = *reinterpret_cast<GemmShared *>(gsm);
    const int tid = threadIdx.x;
    const int mt = blockIdx.x;                    // tile of 128 rows of k = tap * Cin + cin
    const long long vbase = (long long)blockIdx.y * vox_per_split;
    const long long vend = min(g.nvox, vbase + vox_per_split);
    const int nchunks = (int)((vend - vbase + GEMM_KC - 1) / GEMM_KC);
    const int N = Cout;
    const int K = 27 * Cin;
    gemm_setup(sh, N);
    const int kk = tid & (GEMM_KC - 1);   // voxel (K index) handled by this thread
    const int g0 = tid >> 6;              // first of its core-row groups
    auto fillA = [&](int c, unsigned char *as) {
        const long long v = vbase + (long long)c * GEMM_KC + kk;
        const bool vin = v < vend;
        int x = 0, y = 0, z = 0;
        if (vin) vox_xyz(v, g, x, y, z);
#pragma unroll
        for (int j = 0; j < GEMM_M / 8 / 2; ++j) {
            const int grp = g0 + 2 * j;
            const int k = mt * GEMM_M + grp * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (vin && k < K) val = tap_load(in, g, Cin, x, y, z, k / Cin, k % Cin);
            *reinterpret_cast<uint4 *>(as + mnmajor_row_off(grp * 8, kk)) = val;
        }
    };
    auto fillB = [&](int c, unsigned char *bs) {
        const long long v = vbase + (long long)c * GEMM_KC + kk;
        const bool vin = v < vend;
        for (int grp = g0; grp < N / 8; grp += 2) {
            uint4 val = make_uint4(0, 0, 0, 0);
            if (vin) val = __ldg(reinterpret_cast<const uint4 *>(dpre + v * Cout + grp * 8));
            *reinterpret_cast<uint4 *>(bs + mnmajor_row_off(grp * 8, kk)) = val;
        }
    };
    const bool ok = gemm_mainloop(sh, N, nchunks, 1, 1, fillA, fillB);
    if (!ok && tid == 0) latch_error(err, REG_ERR_TIMEOUT);
    const int row = mt * GEMM_M + tid;
    float *dst = part + ((size_t)blockIdx.y * Mrows + row) * N;
    for (int c0 = 0; c0 < N; c0 += 16) {
        float acc[16];
        if (ok && nchunks > 0) {
            gemm_row16(sh, c0, acc);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
        }
        if (row < Mrows) {
#pragma unroll
            for (int i = 0; i < 16; ++i) dst[c0 + i] = acc[i];
        }
    }
    gemm_teardown(sh, N);
}

// dW[n][k] (FP32, packed [Cout][Kpad]) = sum over splits (fixed order) of part[split][k][n]
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int splits, int Mrows, int Cout, int K, int Kpad,
                                    float *__restrict__ dW) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Cout * Kpad) return;
    const int n = idx / Kpad, k = idx % Kpad;
    float acc = 0.0f;
    if (k < K)
        for (int s = 0; s < splits; ++s) acc += part[((size_t)s * Mrows + k) * Cout + n];
    dW[idx] = acc;
}

// data-gradient weights: Wd[cin][tap' * Cout + cout] = W[cout][(26 - tap') * Cin + cin]
__global__ void repack_dgrad_kernel(const __nv_bfloat16 *__restrict__ W, int Cout, int Cin, int Kpad,
                                    __nv_bfloat16 *__restrict__ Wd, int Nd, int Kpad_d) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Nd * Kpad_d) return;
    const int ci = idx / Kpad_d, k = idx % Kpad_d;
    __nv_bfloat16 val = __float2bfloat16_rn(0.0f);
    if (ci < Cin && k < 27 * Cout) {
        const int tapd = k / Cout, co = k % Cout;
        val = W[(size_t)co * Kpad + (26 - tapd) * Cin + ci];
    }
    Wd[idx] = val;
}

cudaError_t launch_conv_fwd(const void *in, int Cin, const void *W, int Kpad, const float *bias, int Cout, int N,
                            const Dims &d, int epi, float slope, void *out, cudaStream_t s) {
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    const size_t smem = gemm_smem_bytes();
    ConvGeom g{d.nx, d.ny, d.nz, d.n};
    const unsigned grid = (unsigned)((d.n + GEMM_M - 1) / GEMM_M);
    cudaError_t e;
    switch (epi) {
        case EPI_BIAS_LEAKY_BF16:
            e = cudaFuncSetAttribute(conv_fwd_kernel<EPI_BIAS_LEAKY_BF16>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            conv_fwd_kernel<EPI_BIAS_LEAKY_BF16><<<grid, GEMM_THREADS, smem, s>>>(
                (const __nv_bfloat16 *)in, Cin, (const __nv_bfloat16 *)W, Kpad, bias, Cout, N, g, slope, out,
                err);
            break;
        case EPI_PLAIN_BF16:
            e = cudaFuncSetAttribute(conv_fwd_kernel<EPI_PLAIN_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            conv_fwd_kernel<EPI_PLAIN_BF16><<<grid, GEMM_THREADS, smem, s>>>(
                (const __nv_bfloat16 *)in, Cin, (const __nv_bfloat16 *)W, Kpad, bias, Cout, N, g, slope, out,
                err);
            break;
        default:
            e = cudaFuncSetAttribute(conv_fwd_kernel<EPI_BIAS_F32_SOA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            conv_fwd_kernel<EPI_BIAS_F32_SOA><<<grid, GEMM_THREADS, smem, s>>>(
                (const __nv_bfloat16 *)in, Cin, (const __nv_bfloat16 *)W, Kpad, bias, Cout, N, g, slope, out,
                err);
    }
    return cudaGetLastError();
}

int wgrad_splits(const Dims &d) {
    long long s = (2LL * num_sms() + 0) ;
    const long long max_s = (d.n + GEMM_KC - 1) / GEMM_KC;
    if (s > max_s) s = max_s;
    return (int)(s < 1 ? 1 : s);
}

cudaError_t launch_conv_wgrad(const void *in, int Cin, const void *dpre, int Cout, const Dims &d, float *part,
                              float *dW, int Kpad, cudaStream_t s) {
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    const size_t smem = gemm_smem_bytes();
    ConvGeom g{d.nx, d.ny, d.nz, d.n};
    const int K = 27 * Cin;
    const int mtiles = (K + GEMM_M - 1) / GEMM_M;
    const int Mrows = mtiles * GEMM_M;
    const int splits = wgrad_splits(d);
    long long vps = (d.n + splits - 1) / splits;
    vps = (vps + GEMM_KC - 1) / GEMM_KC * GEMM_KC;
    cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv_wgrad_kernel<<<dim3(mtiles, splits), GEMM_THREADS, smem, s>>>((const __nv_bfloat16 *)in, Cin,
                                                                       (const __nv_bfloat16 *)dpre, Cout, g, vps, part,
                                                                       Mrows, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int total = Cout * Kpad;
    wgrad_reduce_kernel<<<(total + 255) / 256, 256, 0, s>>>(part, splits, Mrows, Cout, K, Kpad, dW);
    return cudaGetLastError();
}

size_t wgrad_part_bytes(const Dims &d, int Cin, int Cout) {
    const int mtiles = (27 * Cin + GEMM_M - 1) / GEMM_M;
    return sizeof(float) * (size_t)wgrad_splits(d) * mtiles * GEMM_M * Cout;
}

cudaError_t launch_repack_dgrad(const void *W, int Cout, int Cin, int Kpad, void *Wd, int Nd, int Kpad_d,
                                cudaStream_t s) {
    const int total = Nd * Kpad_d;
    repack_dgrad_kernel<<<(total + 255) / 256, 256, 0, s>>>((const __nv_bfloat16 *)W, Cout, Cin, Kpad,
                                                           (__nv_bfloat16 *)Wd, Nd, Kpad_d);
    return cudaGetLastError();
}

}  // namespace regk
