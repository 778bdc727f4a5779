// gemm_tc.cuh -- CTA-level tensor-core mainloop shared by the implicit-GEMM
// convolutions: D[128 x N] (FP32, TMEM) = sum over K-chunks of A B^T, with
// A a 128 x KC and B an N x KC BF16 tile staged in shared memory by caller
// supplied fill functors, double-buffered so that filling chunk c+1
// overlaps the MMAs of chunk c.  One thread issues the MMAs and commits each
// chunk to that buffer's mbarrier; every wait is bounded.
#pragma once

#include "umma.cuh"

namespace regk {

constexpr int GEMM_THREADS = 128;  // 4 warps: one TMEM lane (tile row) per thread
constexpr int GEMM_M = 128;
constexpr int GEMM_KC = 64;        // K elements per staged chunk (4 MMAs of K = 16)
constexpr int GEMM_KG = GEMM_KC / 8;
constexpr int GEMM_MAXN = 128;
constexpr int GEMM_A_BYTES = GEMM_M * GEMM_KC * 2;        // 16 KiB
constexpr int GEMM_B_BYTES = GEMM_MAXN * GEMM_KC * 2;     // 16 KiB
constexpr int GEMM_STAGE_BYTES = GEMM_A_BYTES + GEMM_B_BYTES;

struct GemmShared {
    alignas(128) unsigned char stage[2][GEMM_STAGE_BYTES];
    uint64_t mbar[2];
    uint32_t tmem;
    int failed;
};

__host__ __device__ constexpr uint32_t tmem_cols_for(int N) { return N <= 32 ? 32u : (N <= 64 ? 64u : 128u); }

// byte offset of element (row, k) of a K-major tile in the canonical layout
__device__ __forceinline__ int kmajor_off(int row, int k) {
    return (((row >> 3) * GEMM_KG + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}
// byte offset of the 16-byte core-matrix row holding rows row..row+7 at K index k of an MN-major tile
__device__ __forceinline__ int mnmajor_row_off(int row8, int k) {
    return (((row8 >> 3) * GEMM_KG + (k >> 3)) << 7) + ((k & 7) << 4);
}

// Runs the mainloop.  fillA(chunk, a_smem) / fillB(chunk, b_smem) stage
// chunk `chunk` (called by all 128 threads); a_mn / b_mn give the layouts.
// On return (all threads) the accumulator is complete in TMEM at sh.tmem;
// returns false if a bounded wait expired (the caller must still free TMEM).
template <typename FA, typename FB>
__device__ __forceinline__ bool gemm_mainloop(GemmShared &sh, int N, int nchunks, int a_mn, int b_mn, FA fillA,
                                             FB fillB) {
    const int tid = threadIdx.x;
    const uint32_t idesc = umma::idesc_bf16(GEMM_M, N, a_mn, b_mn);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        if (c >= 2) {
            if (!umma::mbar_wait(&sh.mbar[b], ((c - 2) >> 1) & 1)) ok = false;
            umma::fence_after_sync();
        }
        unsigned char *as = sh.stage[b];
        unsigned char *bs = sh.stage[b] + GEMM_A_BYTES;
        fillA(c, as);
        fillB(c, bs);
        umma::fence_smem_to_async();
        __syncthreads();
        if (tid == 0 && ok) {
            umma::fence_after_sync();
            const uint32_t a0 = umma::smem_addr(as), b0 = umma::smem_addr(bs);
#pragma unroll
            for (int s = 0; s < GEMM_KC / 16; ++s) {
                // K-step s covers core-matrix columns 2s and 2s+1: start address + 256 s
                const uint64_t ad = umma::sdesc(a0 + 256 * s, 128, GEMM_KG * 128);
                const uint64_t bd = umma::sdesc(b0 + 256 * s, 128, GEMM_KG * 128);
                umma::mma_bf16(sh.tmem, ad, bd, idesc, (c > 0 || s > 0) ? 1u : 0u);
            }
            umma::commit(&sh.mbar[b]);
        }
        __syncwarp();
    }
    if (nchunks > 0) {
        const int c = nchunks - 1;
        if (!umma::mbar_wait(&sh.mbar[c & 1], (c >> 1) & 1)) ok = false;
    }
    umma::fence_after_sync();
    return ok;
}

// set up the shared block: mbarriers and TMEM (warp 0 allocates)
__device__ __forceinline__ void gemm_setup(GemmShared &sh, int N) {
    if (threadIdx.x == 0) {
        umma::mbar_init(&sh.mbar[0], 1);
        umma::mbar_init(&sh.mbar[1], 1);
        sh.failed = 0;
    }
    if (threadIdx.x < 32) umma::tmem_alloc(&sh.tmem, tmem_cols_for(N));
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
}

__device__ __forceinline__ void gemm_teardown(GemmShared &sh, int N) {
    umma::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) umma::tmem_dealloc(sh.tmem, tmem_cols_for(N));
}

// this thread's accumulator row: columns [c0, c0+16)
__device__ __forceinline__ void gemm_row16(const GemmShared &sh, int c0, float v[16]) {
    const int warp = threadIdx.x >> 5;
    umma::tmem_ld16(sh.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
}

}  // namespace regk
