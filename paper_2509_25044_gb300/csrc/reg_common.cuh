// reg_common.cuh -- device helpers shared by the sm_103a kernels of the
// registration hot path (trilinear sampling with slope, loads of FP32/BF16
// voxels, block reductions, the device error word).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/reg.h"

namespace regk {

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Dims {
    int nx, ny, nz;
    long long nxy;  // nx * ny
    long long n;    // nx * ny * nz
};

inline Dims make_dims(reg_dims d) {
    Dims g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.nxy = (long long)d.nx * d.ny;
    g.n = g.nxy * d.nz;
    return g;
}

// ---------------------------------------------------------------------------
// voxel loads (read-only path)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ld_vox(const float *p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_vox(const __nv_bfloat16 *p, long long i) {
    return __bfloat162float(__ldg(p + i));
}

// ---------------------------------------------------------------------------
// Trilinear sampling of M at phi = p + u (voxel units), value and slope.
// The cell index is taken from p + floor(u) and the fraction from
// u - floor(u) (exact in FP32), so large coordinates lose no precision.
//   BORDER: phi is clamped into [0, n-1] per axis; cell = min(floor, n-2)
//           (the last knot uses the upper cell); slope 0 along a clamped axis.
//   ZEROS : corners outside the volume read as 0.
// ---------------------------------------------------------------------------
struct Axis {
    int i0;       // lower corner index (may be out of range in ZEROS mode)
    float a;      // fraction in [0,1]
    float slope;  // 1 or 0 (clamped axis)
    bool v0, v1;  // corner validity (ZEROS)
};

__device__ __forceinline__ Axis axis_setup(int p, float uu, int n, int pad) {
    Axis ax;
    // non-finite or absurd displacements are clamped; any |u| > 2^20 voxels
    // is outside every supported volume, so border / zero semantics hold.
    if (!(uu == uu)) uu = 0.0f;
    uu = fminf(fmaxf(uu, -1048576.0f), 1048576.0f);
    const float fl = floorf(uu);
    float a = uu - fl;
    const int f = p + (int)fl;
    if (pad == REG_PAD_BORDER) {
        ax.v0 = ax.v1 = true;
        if (n == 1) {
            ax.i0 = 0;
            ax.a = 0.0f;
            ax.slope = 0.0f;
        } else if (f < 0) {
            ax.i0 = 0;
            ax.a = 0.0f;
            ax.slope = 0.0f;
        } else if (f > n - 2) {
            ax.slope = (f == n - 1 && a == 0.0f) ? 1.0f : 0.0f;
            ax.i0 = n - 2;
            ax.a = 1.0f;
        } else {
            ax.i0 = f;
            ax.a = a;
            ax.slope = 1.0f;
        }
    } else {
        ax.i0 = f;
        ax.a = a;
        ax.slope = 1.0f;
        ax.v0 = (unsigned)f < (unsigned)n;
        ax.v1 = (unsigned)(f + 1) < (unsigned)n;
    }
    return ax;
}

template <typename T>
__device__ __forceinline__ float corner(const T *M, const Dims &g, const Axis &X, const Axis &Y, const Axis &Z,
                                        int bx, int by, int bz) {
    const bool ok = (bx ? X.v1 : X.v0) && (by ? Y.v1 : Y.v0) && (bz ? Z.v1 : Z.v0);
    if (!ok) return 0.0f;
    // BORDER mode with n == 1 uses i0 = 0, i0+1 = 1 with weight 0: clamp index
    const int ix = min(X.i0 + bx, g.nx - 1);
    const int iy = min(Y.i0 + by, g.ny - 1);
    const int iz = min(Z.i0 + bz, g.nz - 1);
    return ld_vox(M, ((long long)iz * g.ny + iy) * g.nx + ix);
}

// (1-a) lo + a hi, exact at a = 0 and a = 1 (so u = 0 reproduces M bit for bit)
__device__ __forceinline__ float lerp1(float a, float lo, float hi) { return fmaf(a, hi, (1.0f - a) * lo); }

// value only
template <typename T>
__device__ __forceinline__ float sample(const T *M, const Dims &g, int x, int y, int z, float ux, float uy,
                                        float uz, int pad) {
    const Axis X = axis_setup(x, ux, g.nx, pad);
    const Axis Y = axis_setup(y, uy, g.ny, pad);
    const Axis Z = axis_setup(z, uz, g.nz, pad);
    const float c000 = corner(M, g, X, Y, Z, 0, 0, 0), c100 = corner(M, g, X, Y, Z, 1, 0, 0);
    const float c010 = corner(M, g, X, Y, Z, 0, 1, 0), c110 = corner(M, g, X, Y, Z, 1, 1, 0);
    const float c001 = corner(M, g, X, Y, Z, 0, 0, 1), c101 = corner(M, g, X, Y, Z, 1, 0, 1);
    const float c011 = corner(M, g, X, Y, Z, 0, 1, 1), c111 = corner(M, g, X, Y, Z, 1, 1, 1);
    const float e00 = lerp1(X.a, c000, c100), e10 = lerp1(X.a, c010, c110);
    const float e01 = lerp1(X.a, c001, c101), e11 = lerp1(X.a, c011, c111);
    const float f0 = lerp1(Y.a, e00, e10), f1 = lerp1(Y.a, e01, e11);
    return lerp1(Z.a, f0, f1);
}

// value and slope dJ/dphi
template <typename T>
__device__ __forceinline__ float sample_grad(const T *M, const Dims &g, int x, int y, int z, float ux, float uy,
                                             float uz, int pad, float &gx, float &gy, float &gz) {
    const Axis X = axis_setup(x, ux, g.nx, pad);
    const Axis Y = axis_setup(y, uy, g.ny, pad);
    const Axis Z = axis_setup(z, uz, g.nz, pad);
    const float c000 = corner(M, g, X, Y, Z, 0, 0, 0), c100 = corner(M, g, X, Y, Z, 1, 0, 0);
    const float c010 = corner(M, g, X, Y, Z, 0, 1, 0), c110 = corner(M, g, X, Y, Z, 1, 1, 0);
    const float c001 = corner(M, g, X, Y, Z, 0, 0, 1), c101 = corner(M, g, X, Y, Z, 1, 0, 1);
    const float c011 = corner(M, g, X, Y, Z, 0, 1, 1), c111 = corner(M, g, X, Y, Z, 1, 1, 1);
    const float d00 = c100 - c000, d10 = c110 - c010, d01 = c101 - c001, d11 = c111 - c011;
    const float e00 = lerp1(X.a, c000, c100), e10 = lerp1(X.a, c010, c110);
    const float e01 = lerp1(X.a, c001, c101), e11 = lerp1(X.a, c011, c111);
    const float f0 = lerp1(Y.a, e00, e10), f1 = lerp1(Y.a, e01, e11);
    const float dy0 = e10 - e00, dy1 = e11 - e01;
    const float dx0 = fmaf(Y.a, d10 - d00, d00), dx1 = fmaf(Y.a, d11 - d01, d01);
    gz = (f1 - f0) * Z.slope;
    gy = fmaf(Z.a, dy1 - dy0, dy0) * Y.slope;
    gx = fmaf(Z.a, dx1 - dx0, dx0) * X.slope;
    return lerp1(Z.a, f0, f1);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int linear_tid() {
    return (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
}

// Fixed-order block sum of a double (every thread passes a value; the
// result is valid in linear thread 0).  `sh` needs (threads / 32) doubles;
// the block size must be a multiple of 32.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int t = linear_tid();
    const int w = t >> 5, l = t & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
        r = l < nw ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// ---------------------------------------------------------------------------
// device error word (first latched code wins)
// ---------------------------------------------------------------------------
// The word lives in a file-scope __device__ variable of regadam.cu; kernels
// receive its device address (error_word()) as an argument.
__device__ __forceinline__ void latch_error(unsigned *err, unsigned code) {
    if (err) atomicCAS(err, 0u, code);
}

// "last block" fixed-order reduction of per-block double partials:
// every block stores its partials, the block that finishes last sums them in
// block-index order (no waiting, deterministic) and re-arms the counter.
// Returns true in the block that must perform the final reduction.
__device__ __forceinline__ bool arrive_last(unsigned *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (linear_tid() == 0) {
        const unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x * gridDim.y * gridDim.z - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

}  // namespace regk
