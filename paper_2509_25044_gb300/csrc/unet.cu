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
    const size_t smem = gemm_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(gemm_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_test_kernel<<<M / GEMM_M, GEMM_THREADS, smem, s>>>((const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, C, M,
                                                            N, K, a_mn, b_mn, error_word());
    return cudaGetLastError();
}

}  // namespace regk
