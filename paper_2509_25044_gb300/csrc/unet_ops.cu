// unet_ops.cu -- the non-GEMM kernels of the learned initialiser: input
// packing (average-pooled, range-normalised pair -> channels-last BF16),
// LeakyReLU backward, bias gradient, 2x average pooling and 2x trilinear
// upsampling (forward and backward, channels-last BF16), channel concat /
// slicing, the L2 training loss, field resampling (SoA FP32) and the weight
// optimiser step.  Everything is deterministic: reductions use fixed-order
// FP64 block partials, the backward resampling is a gather.
#include "kernels.h"

namespace regk {

namespace {

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void xyz_of(long long v, int nx, int ny, int &x, int &y, int &z) {
    const long long r = v / nx;
    x = (int)(v - r * nx);
    z = (int)(r / ny);
    y = (int)(r - (long long)z * ny);
}

// 1-D trilinear x2 upsampling with voxel-centre alignment: fine f samples the
// coarse grid at c = (f + 0.5) / 2 - 0.5, border clamped
__device__ __forceinline__ void up_axis(int f, int n, int &i0, int &i1, float &a) {
    const float c = 0.5f * (float)f - 0.25f;
    const int fl = (int)floorf(c);
    a = c - (float)fl;
    i0 = min(max(fl, 0), n - 1);
    i1 = min(max(fl + 1, 0), n - 1);
}

// weight with which coarse index i contributes to fine index f along one axis
__device__ __forceinline__ float up_weight(int f, int i, int n) {
    int i0, i1;
    float a;
    up_axis(f, n, i0, i1, a);
    return (i0 == i ? 1.0f - a : 0.0f) + (i1 == i ? a : 0.0f);
}

}  // namespace

// ---- input packing ----------------------------------------------------------
template <typename T>
__global__ void pack_pair_kernel(const T *__restrict__ F, const T *__restrict__ M, Dims gin, int factor, float f_lo,
                                 float f_scale, float m_lo, float m_scale, Dims gout, __nv_bfloat16 *__restrict__ out) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= gout.n) return;
    int x, y, z;
    xyz_of(v, gout.nx, gout.ny, x, y, z);
    float sf = 0.0f, sm = 0.0f;
    for (int dz = 0; dz < factor; ++dz)
        for (int dy = 0; dy < factor; ++dy)
            for (int dx = 0; dx < factor; ++dx) {
                const long long p = ((long long)(z * factor + dz) * gin.ny + (y * factor + dy)) * gin.nx + x * factor + dx;
                sf += ld_vox(F, p);
                sm += ld_vox(M, p);
            }
    const float inv = 1.0f / (float)(factor * factor * factor);
    __align__(16) __nv_bfloat16 t[8];
    t[0] = __float2bfloat16_rn((sf * inv - f_lo) * f_scale);
    t[1] = __float2bfloat16_rn((sm * inv - m_lo) * m_scale);
#pragma unroll
    for (int i = 2; i < 8; ++i) t[i] = __float2bfloat16_rn(0.0f);
    // 16 channels (F, M, 14 zeros): the input convolution then takes the TMA-fed path
    *reinterpret_cast<uint4 *>(out + v * 16) = *reinterpret_cast<const uint4 *>(t);
    *reinterpret_cast<uint4 *>(out + v * 16 + 8) = make_uint4(0u, 0u, 0u, 0u);
}

cudaError_t launch_pack_pair(const void *F, const void *M, int dt, const Dims &gin, int factor, float f_lo,
                             float f_scale, float m_lo, float m_scale, void *out, cudaStream_t s) {
    Dims gout = make_dims(reg_dims{gin.nx / factor, gin.ny / factor, gin.nz / factor});
    const unsigned blocks = (unsigned)((gout.n + 255) / 256);
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        pack_pair_kernel<T><<<blocks, 256, 0, s>>>((const T *)F, (const T *)M, gin, factor, f_lo, f_scale, m_lo,
                                                   m_scale, gout, (__nv_bfloat16 *)out);
    });
    return cudaGetLastError();
}

// ---- elementwise ------------------------------------------------------------
__global__ void leaky_bwd_kernel(const __nv_bfloat16 *__restrict__ out, const __nv_bfloat16 *__restrict__ dout,
                                 long long n, float slope, __nv_bfloat16 *__restrict__ dpre) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = bf(dout[i]);
        dpre[i] = __float2bfloat16_rn(bf(out[i]) > 0.0f ? d : slope * d);
    }
}

cudaError_t launch_leaky_bwd(const void *out, const void *dout, long long n, float slope, void *dpre, cudaStream_t s) {
    leaky_bwd_kernel<<<(unsigned)min((n + 255) / 256, 65535LL * 4), 256, 0, s>>>(
        (const __nv_bfloat16 *)out, (const __nv_bfloat16 *)dout, n, slope, (__nv_bfloat16 *)dpre);
    return cudaGetLastError();
}

// dbias[c] = sum_v dpre[v][c]: fixed-order per-block FP64 partials, then one block
__global__ void bias_grad_partial_kernel(const __nv_bfloat16 *__restrict__ dpre, long long V, int C,
                                         long long per_block, double *__restrict__ part) {
    const int c = threadIdx.x;
    if (c >= C) return;
    const long long v0 = (long long)blockIdx.x * per_block, v1 = min(V, v0 + per_block);
    double acc = 0.0;
    for (long long v = v0; v < v1; ++v) acc += (double)bf(dpre[v * C + c]);
    part[(size_t)blockIdx.x * C + c] = acc;
}
__global__ void bias_grad_final_kernel(const double *__restrict__ part, int nblk, int C, float *__restrict__ dbias) {
    const int c = threadIdx.x;
    if (c >= C) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * C + c];
    dbias[c] = (float)acc;
}
int bias_grad_blocks() { return 4 * num_sms(); }
cudaError_t launch_bias_grad(const void *dpre, long long V, int C, double *part, float *dbias, cudaStream_t s) {
    const int nb = bias_grad_blocks();
    const long long per = (V + nb - 1) / nb;
    bias_grad_partial_kernel<<<nb, 64, 0, s>>>((const __nv_bfloat16 *)dpre, V, C, per, part);
    bias_grad_final_kernel<<<1, 64, 0, s>>>(part, nb, C, dbias);
    return cudaGetLastError();
}

// ---- pooling / upsampling (channels-last BF16) -------------------------------
__global__ void avgpool2_kernel(const __nv_bfloat16 *__restrict__ in, int C, Dims gi, Dims go,
                                __nv_bfloat16 *__restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= go.n * C) return;
    const int c = (int)(idx % C);
    const long long v = idx / C;
    int x, y, z;
    xyz_of(v, go.nx, go.ny, x, y, z);
    float acc = 0.0f;
    for (int d = 0; d < 8; ++d) {
        const long long p = ((long long)(2 * z + (d >> 2)) * gi.ny + 2 * y + ((d >> 1) & 1)) * gi.nx + 2 * x + (d & 1);
        acc += bf(in[p * C + c]);
    }
    out[idx] = __float2bfloat16_rn(0.125f * acc);
}
__global__ void avgpool2_bwd_kernel(const __nv_bfloat16 *__restrict__ dout, int C, Dims gi, Dims go,
                                    __nv_bfloat16 *__restrict__ din) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= gi.n * C) return;
    const int c = (int)(idx % C);
    const long long v = idx / C;
    int x, y, z;
    xyz_of(v, gi.nx, gi.ny, x, y, z);
    const long long q = ((long long)(z >> 1) * go.ny + (y >> 1)) * go.nx + (x >> 1);
    din[idx] = __float2bfloat16_rn(0.125f * bf(dout[q * C + c]));
}
__global__ void upsample2_kernel(const __nv_bfloat16 *__restrict__ in, int C, Dims gc, Dims gf,
                                 __nv_bfloat16 *__restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= gf.n * C) return;
    const int c = (int)(idx % C);
    const long long v = idx / C;
    int x, y, z;
    xyz_of(v, gf.nx, gf.ny, x, y, z);
    int x0, x1, y0, y1, z0, z1;
    float ax, ay, az;
    up_axis(x, gc.nx, x0, x1, ax);
    up_axis(y, gc.ny, y0, y1, ay);
    up_axis(z, gc.nz, z0, z1, az);
    auto at = [&](int xx, int yy, int zz) { return bf(in[(((long long)zz * gc.ny + yy) * gc.nx + xx) * C + c]); };
    const float e00 = (1 - ax) * at(x0, y0, z0) + ax * at(x1, y0, z0);
    const float e10 = (1 - ax) * at(x0, y1, z0) + ax * at(x1, y1, z0);
    const float e01 = (1 - ax) * at(x0, y0, z1) + ax * at(x1, y0, z1);
    const float e11 = (1 - ax) * at(x0, y1, z1) + ax * at(x1, y1, z1);
    const float f0 = (1 - ay) * e00 + ay * e10, f1 = (1 - ay) * e01 + ay * e11;
    out[idx] = __float2bfloat16_rn((1 - az) * f0 + az * f1);
}
// transpose of upsample2 as a gather: coarse i collects fine f in [2i-1, 2i+2]
__global__ void upsample2_bwd_kernel(const __nv_bfloat16 *__restrict__ dout, int C, Dims gc, Dims gf,
                                     __nv_bfloat16 *__restrict__ din) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= gc.n * C) return;
    const int c = (int)(idx % C);
    const long long v = idx / C;
    int x, y, z;
    xyz_of(v, gc.nx, gc.ny, x, y, z);
    float acc = 0.0f;
    for (int fz = max(2 * z - 1, 0); fz <= min(2 * z + 2, gf.nz - 1); ++fz) {
        const float wz = up_weight(fz, z, gc.nz);
        if (wz == 0.0f) continue;
        for (int fy = max(2 * y - 1, 0); fy <= min(2 * y + 2, gf.ny - 1); ++fy) {
            const float wy = up_weight(fy, y, gc.ny);
            if (wy == 0.0f) continue;
            for (int fx = max(2 * x - 1, 0); fx <= min(2 * x + 2, gf.nx - 1); ++fx) {
                const float wx = up_weight(fx, x, gc.nx);
                if (wx == 0.0f) continue;
                acc += wz * wy * wx * bf(dout[(((long long)fz * gf.ny + fy) * gf.nx + fx) * C + c]);
            }
        }
    }
    din[idx] = __float2bfloat16_rn(acc);
}

static unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_avgpool2(const void *in, int C, const Dims &gi, void *out, cudaStream_t s) {
    Dims go = make_dims(reg_dims{gi.nx / 2, gi.ny / 2, gi.nz / 2});
    avgpool2_kernel<<<blocks_for(go.n * C), 256, 0, s>>>((const __nv_bfloat16 *)in, C, gi, go, (__nv_bfloat16 *)out);
    return cudaGetLastError();
}
cudaError_t launch_avgpool2_bwd(const void *dout, int C, const Dims &gi, void *din, cudaStream_t s) {
    Dims go = make_dims(reg_dims{gi.nx / 2, gi.ny / 2, gi.nz / 2});
    avgpool2_bwd_kernel<<<blocks_for(gi.n * C), 256, 0, s>>>((const __nv_bfloat16 *)dout, C, gi, go,
                                                             (__nv_bfloat16 *)din);
    return cudaGetLastError();
}
cudaError_t launch_upsample2(const void *in, int C, const Dims &gc, void *out, cudaStream_t s) {
    Dims gf = make_dims(reg_dims{gc.nx * 2, gc.ny * 2, gc.nz * 2});
    upsample2_kernel<<<blocks_for(gf.n * C), 256, 0, s>>>((const __nv_bfloat16 *)in, C, gc, gf, (__nv_bfloat16 *)out);
    return cudaGetLastError();
}
cudaError_t launch_upsample2_bwd(const void *dout, int C, const Dims &gc, void *din, cudaStream_t s) {
    Dims gf = make_dims(reg_dims{gc.nx * 2, gc.ny * 2, gc.nz * 2});
    upsample2_bwd_kernel<<<blocks_for(gc.n * C), 256, 0, s>>>((const __nv_bfloat16 *)dout, C, gc, gf,
                                                              (__nv_bfloat16 *)din);
    return cudaGetLastError();
}

// ---- channel concat / slice -------------------------------------------------
// dst[v][c0 + c] (=|+=) src[v][c] for c < Csrc; dst has Cdst channels
__global__ void put_channels_kernel(const __nv_bfloat16 *__restrict__ src, int Csrc, long long V,
                                    __nv_bfloat16 *__restrict__ dst, int Cdst, int c0, int accumulate) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= V * Csrc) return;
    const long long v = idx / Csrc;
    const int c = (int)(idx % Csrc);
    __nv_bfloat16 *d = dst + v * Cdst + c0 + c;
    const float val = bf(src[idx]);
    *d = __float2bfloat16_rn(accumulate ? bf(*d) + val : val);
}
// dst[v][c] (=|+=) src[v][c0 + c] for c < Cdst; src has Csrc channels
__global__ void take_channels_kernel(const __nv_bfloat16 *__restrict__ src, int Csrc, int c0, long long V,
                                     __nv_bfloat16 *__restrict__ dst, int Cdst, int accumulate) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= V * Cdst) return;
    const long long v = idx / Cdst;
    const int c = (int)(idx % Cdst);
    const float val = bf(src[v * Csrc + c0 + c]);
    dst[idx] = __float2bfloat16_rn(accumulate ? bf(dst[idx]) + val : val);
}
cudaError_t launch_put_channels(const void *src, int Csrc, long long V, void *dst, int Cdst, int c0, int acc,
                                cudaStream_t s) {
    put_channels_kernel<<<blocks_for(V * Csrc), 256, 0, s>>>((const __nv_bfloat16 *)src, Csrc, V,
                                                             (__nv_bfloat16 *)dst, Cdst, c0, acc);
    return cudaGetLastError();
}
cudaError_t launch_take_channels(const void *src, int Csrc, int c0, long long V, void *dst, int Cdst, int acc,
                                 cudaStream_t s) {
    take_channels_kernel<<<blocks_for(V * Cdst), 256, 0, s>>>((const __nv_bfloat16 *)src, Csrc, c0, V,
                                                              (__nv_bfloat16 *)dst, Cdst, acc);
    return cudaGetLastError();
}

// ---- L2 training loss on SoA FP32 fields ------------------------------------
// loss = mean over 3V entries of (pred - target)^2; dpred (channels-last BF16,
// Cpad channels, channels >= 3 zero) = 2 (pred - target) / (3V)
__global__ void mse_kernel(const float *__restrict__ pred, const float *__restrict__ tgt, long long V, int Cpad,
                           __nv_bfloat16 *__restrict__ dpred, double *__restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    const float sc = 2.0f / (3.0f * (float)V);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < Cpad; ++c) {
            float d = 0.0f;
            if (c < 3) {
                d = pred[(size_t)c * V + v] - tgt[(size_t)c * V + v];
                acc += (double)d * d;
            }
            dpred[v * Cpad + c] = __float2bfloat16_rn(sc * d);
        }
    }
    const double bs = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
}
__global__ void mse_final_kernel(const double *__restrict__ part, int nblk, long long V, double *__restrict__ loss) {
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[b];
    loss[0] = acc / (3.0 * (double)V);
}
int mse_blocks() { return 2 * num_sms(); }
cudaError_t launch_mse(const float *pred, const float *tgt, long long V, int Cpad, void *dpred, double *part,
                       double *loss, cudaStream_t s) {
    const int nb = mse_blocks();
    mse_kernel<<<nb, 256, 0, s>>>(pred, tgt, V, Cpad, (__nv_bfloat16 *)dpred, part);
    mse_final_kernel<<<1, 1, 0, s>>>(part, nb, V, loss);
    return cudaGetLastError();
}

// ---- field resampling (SoA FP32, displacements in voxel units) ---------------
// 2x average pooling of a displacement field and rescaling to the coarse voxel size
__global__ void field_down2_kernel(const float *__restrict__ u, Dims gf, Dims gc, float *__restrict__ out) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= gc.n) return;
    int x, y, z;
    xyz_of(v, gc.nx, gc.ny, x, y, z);
    for (int c = 0; c < 3; ++c) {
        float acc = 0.0f;
        for (int d = 0; d < 8; ++d) {
            const long long p = ((long long)(2 * z + (d >> 2)) * gf.ny + 2 * y + ((d >> 1) & 1)) * gf.nx + 2 * x + (d & 1);
            acc += u[(size_t)c * gf.n + p];
        }
        out[(size_t)c * gc.n + v] = 0.125f * acc * 0.5f;
    }
}
// trilinear upsampling by an integer factor s (voxel-centre aligned, border
// clamped), displacements multiplied by s
__global__ void field_up_kernel(const float *__restrict__ u, Dims gc, int s, Dims gf, float *__restrict__ out) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= gf.n) return;
    int x, y, z;
    xyz_of(v, gf.nx, gf.ny, x, y, z);
    const float inv = 1.0f / (float)s;
    auto ax = [&](int f, int n, int &i0, int &i1, float &a) {
        const float cc = ((float)f + 0.5f) * inv - 0.5f;
        const int fl = (int)floorf(cc);
        a = cc - (float)fl;
        i0 = min(max(fl, 0), n - 1);
        i1 = min(max(fl + 1, 0), n - 1);
    };
    int x0, x1, y0, y1, z0, z1;
    float a, b, cz;
    ax(x, gc.nx, x0, x1, a);
    ax(y, gc.ny, y0, y1, b);
    ax(z, gc.nz, z0, z1, cz);
    for (int c = 0; c < 3; ++c) {
        const float *uc = u + (size_t)c * gc.n;
        auto at = [&](int xx, int yy, int zz) { return uc[((long long)zz * gc.ny + yy) * gc.nx + xx]; };
        const float e00 = (1 - a) * at(x0, y0, z0) + a * at(x1, y0, z0);
        const float e10 = (1 - a) * at(x0, y1, z0) + a * at(x1, y1, z0);
        const float e01 = (1 - a) * at(x0, y0, z1) + a * at(x1, y0, z1);
        const float e11 = (1 - a) * at(x0, y1, z1) + a * at(x1, y1, z1);
        const float f0 = (1 - b) * e00 + b * e10, f1 = (1 - b) * e01 + b * e11;
        out[(size_t)c * gf.n + v] = (float)s * ((1 - cz) * f0 + cz * f1);
    }
}
cudaError_t launch_field_down2(const float *u, const Dims &gf, float *out, cudaStream_t s) {
    Dims gc = make_dims(reg_dims{gf.nx / 2, gf.ny / 2, gf.nz / 2});
    field_down2_kernel<<<blocks_for(gc.n), 256, 0, s>>>(u, gf, gc, out);
    return cudaGetLastError();
}
cudaError_t launch_field_up(const float *u, const Dims &gc, int factor, float *out, cudaStream_t s) {
    Dims gf = make_dims(reg_dims{gc.nx * factor, gc.ny * factor, gc.nz * factor});
    field_up_kernel<<<blocks_for(gf.n), 256, 0, s>>>(u, gc, factor, gf, out);
    return cudaGetLastError();
}

// ---- weight optimiser: Adam on FP32 master weights + BF16 copy -----------------
__global__ void adam_weights_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                                    const float *__restrict__ g, long long n, StepParams S,
                                    __nv_bfloat16 *__restrict__ w_bf16) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float nw = adam_update(w[i], g[i], m[i], v[i], m, v, i, S);
        w[i] = nw;
        if (w_bf16) w_bf16[i] = __float2bfloat16_rn(nw);
    }
}
cudaError_t launch_adam_weights(float *w, float *m, float *v, const float *g, long long n, const StepParams &S,
                                void *w_bf16, cudaStream_t s) {
    adam_weights_kernel<<<(unsigned)min((n + 255) / 256, 4096LL), 256, 0, s>>>(w, m, v, g, n, S,
                                                                              (__nv_bfloat16 *)w_bf16);
    return cudaGetLastError();
}

}  // namespace regk
