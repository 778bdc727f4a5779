// smooth.cu -- Gaussian smoothing of a displacement or gradient field (the
// sigma_grad / sigma_warp smoothing regularisation the paper runs its
// registrations with): each of the three SoA channels is convolved
// separably along x, y and z with w_k = exp(-k^2 / (2 sigma^2)) / sum,
// |k| <= floor(4 sigma + 1/2), borders repeating the edge voxel.  One launch
// per axis; the y and z passes read along rows of 32 consecutive x (coalesced),
// the x pass reads its neighbours through L1.
#include <math.h>

#include "kernels.h"

namespace regk {

template <int AXIS>
__global__ void smooth_axis_kernel(const float *__restrict__ in, float *__restrict__ out, Dims g, SmoothWeights W) {
    const long long total = 3 * g.n;
    const int r = W.r;
    const int n_axis = AXIS == 0 ? g.nx : (AXIS == 1 ? g.ny : g.nz);
    const long long stride = AXIS == 0 ? 1 : (AXIS == 1 ? (long long)g.nx : g.nxy);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i % g.n;
        long long q;
        if (AXIS == 0)
            q = p % g.nx;
        else if (AXIS == 1)
            q = (p / g.nx) % g.ny;
        else
            q = p / g.nxy;
        const float *base = in + (i - q * stride);  // the voxel at coordinate 0 along the axis
        float acc = 0.0f;
        for (int k = -r; k <= r; ++k) {
            long long qq = q + k;
            qq = qq < 0 ? 0 : (qq > n_axis - 1 ? n_axis - 1 : qq);
            acc = fmaf(W.w[k + r], __ldg(base + qq * stride), acc);
        }
        out[i] = acc;
    }
}

SmoothWeights smooth_weights(float sigma) {
    SmoothWeights W;
    W.r = (int)(4.0 * (double)sigma + 0.5);
    double sum = 0.0, w[2 * SMOOTH_MAX_R + 1];
    for (int k = -W.r; k <= W.r; ++k) {
        w[k + W.r] = exp(-0.5 * (double)k * (double)k / ((double)sigma * (double)sigma));
        sum += w[k + W.r];
    }
    for (int k = 0; k <= 2 * W.r; ++k) W.w[k] = (float)(w[k] / sum);
    return W;
}

cudaError_t launch_smooth_field(const float *u, const Dims &g, float sigma, float *tmp, float *out, cudaStream_t s) {
    const SmoothWeights W = smooth_weights(sigma);
    const long long total = 3 * g.n;
    long long blocks = (total + 255) / 256;
    const long long cap = 32LL * num_sms();
    if (blocks > cap) blocks = cap;
    smooth_axis_kernel<0><<<(unsigned)blocks, 256, 0, s>>>(u, out, g, W);
    smooth_axis_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(out, tmp, g, W);
    smooth_axis_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(tmp, out, g, W);
    return cudaGetLastError();
}

// 2x2x2 block mean of an even-sized image (the coarse levels of the
// multi-scale schedule), FP32 or BF16 in and out (the sum is FP32)
template <typename T>
__global__ void downsample2_kernel(const T *__restrict__ in, Dims gi, Dims go, T *__restrict__ out) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < go.n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long x = v % go.nx, y = (v / go.nx) % go.ny, z = v / go.nxy;
        const T *b = in + (2 * z) * gi.nxy + (2 * y) * gi.nx + 2 * x;
        float acc = 0.0f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const T *r = b + dz * gi.nxy + dy * gi.nx;
                acc += ld_vox(r, 0) + ld_vox(r, 1);
            }
        store_vox(out + v, 0.125f * acc);
    }
}

cudaError_t launch_downsample2(const void *in, int dt, const Dims &gi, void *out, cudaStream_t s) {
    const Dims go = make_dims(reg_dims{gi.nx / 2, gi.ny / 2, gi.nz / 2});
    long long blocks = (go.n + 255) / 256;
    if (blocks > 32LL * num_sms()) blocks = 32LL * num_sms();
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        downsample2_kernel<T><<<(unsigned)blocks, 256, 0, s>>>((const T *)in, gi, go, (T *)out);
    });
    return cudaGetLastError();
}

}  // namespace regk
