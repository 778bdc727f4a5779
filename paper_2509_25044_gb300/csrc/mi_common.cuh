// mi_common.cuh -- per-voxel pieces of the Parzen MI sweeps shared by the
// plain kernels (mi.cu) and the TMA-staged second sweep (mi_tma.cu): the
// cubic B-spline weights of a bin coordinate and their derivatives, the
// intensity-to-bin map and the hard-binned estimator's nearest bin.
#pragma once

#include "kernels.h"

namespace regk {

// Cubic B-spline weights of the 4 bins around bin coordinate s in [1, B-2]:
// bins i0-1 .. i0+2 with i0 = min(floor(s), B-3), fraction f = s - i0.
__device__ __forceinline__ int bspline_weights(float s, int B, float w[4]) {
    int i0 = (int)floorf(s);
    i0 = min(max(i0, 1), B - 3);
    const float f = s - (float)i0;
    const float f2 = f * f, f3 = f2 * f, g = 1.0f - f;
    w[0] = g * g * g * (1.0f / 6.0f);
    w[1] = (3.0f * f3 - 6.0f * f2 + 4.0f) * (1.0f / 6.0f);
    w[2] = (-3.0f * f3 + 3.0f * f2 + 3.0f * f + 1.0f) * (1.0f / 6.0f);
    w[3] = f3 * (1.0f / 6.0f);
    return i0;
}

// The same weights times c6 / (1/6): with c6 = (1/6) 2^20 (exactly RN(1/6)
// times a power of two) they are the weights times 2^20, bit for bit, in
// one multiply each instead of two.
__device__ __forceinline__ int bspline_weights_times(float s, int B, float c6, float w[4]) {
    int i0 = (int)floorf(s);
    i0 = min(max(i0, 1), B - 3);
    const float f = s - (float)i0;
    const float f2 = f * f, f3 = f2 * f, g = 1.0f - f;
    w[0] = g * g * g * c6;
    w[1] = (3.0f * f3 - 6.0f * f2 + 4.0f) * c6;
    w[2] = (-3.0f * f3 + 3.0f * f2 + 3.0f * f + 1.0f) * c6;
    w[3] = f3 * c6;
    return i0;
}

// derivatives of the same 4 weights with respect to s
__device__ __forceinline__ int bspline_dweights(float s, int B, float d[4]) {
    int i0 = (int)floorf(s);
    i0 = min(max(i0, 1), B - 3);
    const float f = s - (float)i0;
    const float g = 1.0f - f;
    d[0] = -0.5f * g * g;
    d[1] = 1.5f * f * f - 2.0f * f;
    d[2] = -1.5f * f * f + f + 0.5f;
    d[3] = 0.5f * f * f;
    return i0;
}

__device__ __forceinline__ float to_bin(float v, float lo, float scale, int B) {
    const float t = fminf(fmaxf((v - lo) * scale, 0.0f), 1.0f);
    return fmaf(t, (float)(B - 3), 1.0f);
}

// nearest bin of bin coordinate s (the hard-binned estimator's rule)
__device__ __forceinline__ int nearest_bin(float s, int B) { return min(max((int)floorf(s + 0.5f), 1), B - 2); }

// Shared histogram of one CTA: `copies` private copies, copy c used by the
// lanes with lane % copies == c, each copy padded by one word so that the
// same bin of different copies falls in different banks.  With 32 copies
// the 32 lanes of one atomic instruction never share an address; with
// fewer, two lanes of a copy do when their voxels fall in the same bins
// (the two adds then serialise; the integer sums are the same).  The count
// for the 1024-thread CTA shape, whose copies fill about 131 KB:
__host__ __device__ constexpr int hist_copies(int B) { return B <= 32 ? 32 : (B <= 45 ? 16 : 8); }

// Adds the 16 fixed-point products of a voxel's 4 + 4 B-spline weights to a
// copy of the histogram.  Each product is rounded by one FFMA against 2^23
// (exact round-to-nearest of wf * wj * MI_FIXED_SCALE, which is below 2^22),
// so the bins are sums of integers and the histogram does not depend on the
// order of the atomics (deterministic).
__device__ __forceinline__ void hist_add_parzen(unsigned *shc, int B, float sF, float sJ) {
    constexpr float MAGIC = 8388608.0f;  // 2^23: ulp 1 in [2^23, 2^24)
    float sf[4], wj[4];
    // the fixed-image weights already times MI_FIXED_SCALE (a power of two)
    const int iF = bspline_weights_times(sF, B, (1.0f / 6.0f) * MI_FIXED_SCALE, sf) - 1;
    const int iJ = bspline_weights(sJ, B, wj) - 1;
    unsigned *row = shc + iF * B + iJ;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float sa = sf[a];
#pragma unroll
        for (int b = 0; b < 4; ++b) atomicAdd(row + b, __float_as_uint(fmaf(sa, wj[b], MAGIC)) - 0x4B000000u);
        row += B;
    }
}

}  // namespace regk
