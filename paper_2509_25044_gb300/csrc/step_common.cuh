// step_common.cuh -- the per-voxel tail shared by the fused sweeps: the
// diffusion regulariser's value / gradient at one voxel and the Adam update
// of its three displacement components.
#pragma once

#include "reg_common.cuh"

namespace regk {

struct StepParams {
    float lam;        // regulariser weight lambda
    float two_over_n; // 2 / N (dR/du scale)
    float lr_bc1;     // lr / (1 - beta1^t)
    float rsqrt_bc2;  // 1 / sqrt(1 - beta2^t)
    float b1, b2, eps, gscale;
};

template <typename I>
__device__ __forceinline__ float ld_moment(const float *p, I i) {
    return p[i];
}
template <typename I>
__device__ __forceinline__ float ld_moment(const __nv_bfloat16 *p, I i) {
    return __bfloat162float(p[i]);
}
template <typename I>
__device__ __forceinline__ void st_moment(float *p, I i, float v) {
    p[i] = v;
}
template <typename I>
__device__ __forceinline__ void st_moment(__nv_bfloat16 *p, I i, float v) {
    p[i] = __float2bfloat16_rn(v);
}

// Adam on one element (torch.optim.Adam with bias correction; the update
// uses the new moments in FP32, the stored moments are rounded to MT).
template <typename MT>
__device__ __forceinline__ float adam_elem(float u, float g, MT *m, MT *v, long long i, const StepParams &S) {
    const float gs = S.gscale * g;
    const float mn = fmaf(S.b1, ld_moment(m, i), (1.0f - S.b1) * gs);
    const float vn = fmaf(S.b2, ld_moment(v, i), (1.0f - S.b2) * gs * gs);
    st_moment(m, i, mn);
    st_moment(v, i, vn);
    const float denom = fmaf(sqrtf(vn), S.rsqrt_bc2, S.eps);
    return u - S.lr_bc1 * (mn / denom);
}

// Same update with the old moments already loaded (m0, v0).
template <typename MT>
__device__ __forceinline__ float adam_update(float u, float g, float m0, float v0, MT *m, MT *v, long long i,
                                             const StepParams &S) {
    const float gs = S.gscale * g;
    const float mn = fmaf(S.b1, m0, (1.0f - S.b1) * gs);
    const float vn = fmaf(S.b2, v0, (1.0f - S.b2) * gs * gs);
    st_moment(m, i, mn);
    st_moment(v, i, vn);
    const float denom = fmaf(sqrtf(vn), S.rsqrt_bc2, S.eps);
    return u - S.lr_bc1 * (mn / denom);
}

// Diffusion regulariser at voxel (x,y,z) for all three channels.
//   grad:  gR_c = (2/N) sum_d [ (u_c(p) - u_c(p+e_d)) [p+e_d inside]
//                             + (u_c(p) - u_c(p-e_d)) [p-e_d inside] ]
//   value: adds sum_c sum_d (u_c(p+e_d) - u_c(p))^2 over forward neighbours
//          inside the volume (each pair is counted by its lower voxel).
// cur/prv/nxt hold u at z, z-1, z+1 (prv/nxt ignored at the z borders);
// the x and y neighbours are read through the read-only cache.
__device__ __forceinline__ void diffusion_at(const float *__restrict__ u, const Dims &g, int x, int y, int z,
                                             long long p, const float cur[3], const float prv[3],
                                             const float nxt[3], float gR[3], float &rpart) {
    const bool hxm = x > 0, hxp = x + 1 < g.nx;
    const bool hym = y > 0, hyp = y + 1 < g.ny;
    const bool hzm = z > 0, hzp = z + 1 < g.nz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float *uc = u + (long long)c * g.n;
        const float c0 = cur[c];
        float acc = 0.0f;
        if (hxp) {
            const float d = __ldg(uc + p + 1) - c0;
            acc -= d;
            rpart = fmaf(d, d, rpart);
        }
        if (hxm) acc += c0 - __ldg(uc + p - 1);
        if (hyp) {
            const float d = __ldg(uc + p + g.nx) - c0;
            acc -= d;
            rpart = fmaf(d, d, rpart);
        }
        if (hym) acc += c0 - __ldg(uc + p - g.nx);
        if (hzp) {
            const float d = nxt[c] - c0;
            acc -= d;
            rpart = fmaf(d, d, rpart);
        }
        if (hzm) acc += c0 - prv[c];
        gR[c] = acc;
    }
}

// The same stencil on per-channel base pointers with a voxel index of type I
// (int for volumes below 2^31 voxels); the h* flags say which neighbours lie
// inside the volume.
template <typename I>
__device__ __forceinline__ void diffusion_ptr(const float *const uc[3], I p, I nx, bool hxm, bool hxp, bool hym,
                                              bool hyp, bool hzm, bool hzp, const float cur[3], const float prv[3],
                                              const float nxt[3], float gR[3], float &rpart) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float c0 = cur[c];
        float acc = 0.0f;
        if (hxp) {
            const float d = __ldg(uc[c] + p + 1) - c0;
            acc -= d;
            rpart = fmaf(d, d, rpart);
        }
        if (hxm) acc += c0 - __ldg(uc[c] + p - 1);
        if (hyp) {
            const float d = __ldg(uc[c] + p + nx) - c0;
            acc -= d;
            rpart = fmaf(d, d, rpart);
        }
        if (hym) acc += c0 - __ldg(uc[c] + p - nx);
        if (hzp) {
            const float d = nxt[c] - c0;
            acc -= d;
            rpart = fmaf(d, d, rpart);
        }
        if (hzm) acc += c0 - prv[c];
        gR[c] = acc;
    }
}

// the hardware square-root approximation (sqrt.approx, relative error below
// 2^-22): one instruction instead of the correctly rounded sequence
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Adam on one element with the old moments already loaded; the new moments
// are stored to m[i], v[i]; returns the updated displacement.  The square
// root and the quotient use the fast hardware forms (a few ulp, far inside
// the parity bar).
template <typename MT, typename I>
__device__ __forceinline__ float adam_fast(float u, float g, float m0, float v0, MT *m, MT *v, I i,
                                           const StepParams &S) {
    const float gs = S.gscale * g;
    const float mn = fmaf(S.b1, m0, (1.0f - S.b1) * gs);
    const float vn = fmaf(S.b2, v0, (1.0f - S.b2) * gs * gs);
    st_moment(m, i, mn);
    st_moment(v, i, vn);
    const float denom = fmaf(sqrt_approx(vn), S.rsqrt_bc2, S.eps);
    return fmaf(-S.lr_bc1, __fdividef(mn, denom), u);
}

}  // namespace regk
