// warp.cu -- standalone trilinear warp J = M o (id + u) with optional slope
// (Sec. 2.1: the deformable part of the composite implicit grid sampler;
// Algorithm gridsampler, forward), and its composite form
// phi(p) = A p + t + S u(p) with the backward to u, A and t.  The identity
// grid is implicit in the thread index, so no coordinate grid is ever
// materialised.  The fused loss sweeps (lncc.cu, mi.cu) call the same device
// sampler on chip; these kernels serve reg_warp, the composite entry points
// and the tests.
#include "kernels.h"

namespace regk {

template <typename T, bool SLOPE, int PAD, bool AFF>
__global__ void __launch_bounds__(TILE_THREADS) warp_kernel(const T *__restrict__ M, const float *__restrict__ u,
                                                            Dims g, int zc, AffineT Ain, float *__restrict__ J,
                                                            float *__restrict__ dJ) {
    const AffineT A = AFF ? resolve_affine(Ain) : Ain;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const bool has_u = !AFF || u != nullptr;  // the composite form may omit u
    const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
    for (int z = z0; z < z1; ++z) {
        const long long p = (long long)z * g.nxy + (long long)y * g.nx + x;
        float ux = 0.0f, uy = 0.0f, uz = 0.0f;
        if (has_u) {
            ux = __ldg(u + p);
            uy = __ldg(u + g.n + p);
            uz = __ldg(u + 2 * g.n + p);
        }
        if (AFF) composite_disp(A, x, y, z, ux, uy, uz);
        if (SLOPE) {
            float sx, sy, sz;
            J[p] = sample_grad<T, PAD>(M, g, x, y, z, ux, uy, uz, sx, sy, sz);
            dJ[p] = sx;
            dJ[g.n + p] = sy;
            dJ[2 * g.n + p] = sz;
        } else {
            J[p] = sample<T, PAD>(M, g, x, y, z, ux, uy, uz);
        }
    }
}

cudaError_t launch_warp(const void *M, int dt, const float *u, const Dims &g, int pad, float *J, float *dJ,
                        cudaStream_t s, const AffineT *aff) {
    const MarchGrid G = march_grid(g, 8LL * num_sms() * 4, 1);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    const AffineT A = aff ? *aff : AffineT{};
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            auto run = [&](auto kern) { kern<<<grid, block, 0, s>>>((const T *)M, u, g, G.zc, A, J, dJ); };
            if (aff) {
                if (dJ)
                    run(warp_kernel<T, true, PD, true>);
                else
                    run(warp_kernel<T, false, PD, true>);
            } else if (dJ) {
                run(warp_kernel<T, true, PD, false>);
            } else {
                run(warp_kernel<T, false, PD, false>);
            }
        });
    });
    return cudaGetLastError();
}

// Algorithm gridsampler, backward, without the image gradient: for the
// upstream gradient g = dL/dJ, gX = dJ/dphi * g is the gradient with respect
// to the sampling location; g_u = S gX (optional) and the 12 sums dL/dA,
// dL/dt are reduced in a fixed order.
template <typename T, int PAD>
__global__ void __launch_bounds__(TILE_THREADS)
    composite_backward_kernel(const T *__restrict__ M, const float *__restrict__ u, Dims g, int zc, AffineT Ain,
                              const float *__restrict__ gin, float *__restrict__ g_u, double *__restrict__ partials,
                              unsigned *__restrict__ counter, double *__restrict__ out, unsigned *err) {
    __shared__ double red[32];
    const AffineT A = resolve_affine(Ain);
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    AffineAcc acc;
    if (x < g.nx && y < g.ny) {
        const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
        for (int z = z0; z < z1; ++z) {
            const long long p = (long long)z * g.nxy + (long long)y * g.nx + x;
            float ux = 0.0f, uy = 0.0f, uz = 0.0f;
            if (u) {
                ux = __ldg(u + p);
                uy = __ldg(u + g.n + p);
                uz = __ldg(u + 2 * g.n + p);
            }
            composite_disp(A, x, y, z, ux, uy, uz);
            float sx, sy, sz;
            (void)sample_grad<T, PAD>(M, g, x, y, z, ux, uy, uz, sx, sy, sz);
            const float gv = __ldg(gin + p);
            const float gx = gv * sx, gy = gv * sy, gz = gv * sz;
            acc.add(gx, gy, gz, z);
            if (g_u) {
                g_u[p] = A.s[0] * gx;
                g_u[g.n + p] = A.s[1] * gy;
                g_u[2 * g.n + p] = A.s[2] * gz;
            }
        }
    }
    affine_reduce(acc, x, y, partials, counter, out, red, err);
}

cudaError_t launch_composite_backward(const void *M, int dt, const float *u, const Dims &g, int pad,
                                      const AffineT &A, const float *gin, float *g_u, double *partials,
                                      unsigned *counter, double *out, cudaStream_t s) {
    const MarchGrid G = march_grid(g, 8LL * num_sms() * 4, 1);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            composite_backward_kernel<T, decltype(pd)::value><<<grid, block, 0, s>>>(
                (const T *)M, u, g, G.zc, A, gin, g_u, partials, counter, out, err);
        });
    });
    return cudaGetLastError();
}

// Composition of displacement fields, (id + w) = (id + s b) o (id + s a):
// w(p) = s a(p) + s b(p + s a(p)), the three channels of b sampled at one
// location (the same sampler as the warp).  s folds the 2^-K of
// scaling-and-squaring into its first step; s = 1 is the plain composition.
template <int PAD>
__global__ void __launch_bounds__(TILE_THREADS) compose_kernel(const float *__restrict__ a,
                                                               const float *__restrict__ b, Dims g, int zc, float s,
                                                               float *__restrict__ w) {
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
    for (int z = z0; z < z1; ++z) {
        const long long p = (long long)z * g.nxy + (long long)y * g.nx + x;
        const float ux = s * __ldg(a + p), uy = s * __ldg(a + g.n + p), uz = s * __ldg(a + 2 * g.n + p);
        const float bx = sample<float, PAD>(b, g, x, y, z, ux, uy, uz);
        const float by = sample<float, PAD>(b + g.n, g, x, y, z, ux, uy, uz);
        const float bz = sample<float, PAD>(b + 2 * g.n, g, x, y, z, ux, uy, uz);
        w[p] = fmaf(s, bx, ux);
        w[g.n + p] = fmaf(s, by, uy);
        w[2 * g.n + p] = fmaf(s, bz, uz);
    }
}

// Adjoint of w = s a + s b o (id + s a) for gw = dL/dw:
//   ga = s gw + s^2 (grad b)^T gw at the sample point p + s a(p),
//   gb += s gw scattered onto the 8 corners of that sample with its trilinear
//         weights (the same padding as the sampler; the transpose of sampling b).
// SAME (a and b one field): ga is added into gb as well, which then holds the
// whole gradient.  The scatter uses float atomics, so the order of the
// additions -- and the last bits of gb -- can vary between runs.
template <int PAD, bool SAME>
__global__ void __launch_bounds__(TILE_THREADS)
    compose_backward_kernel(const float *__restrict__ a, const float *__restrict__ b, const float *__restrict__ gw,
                            Dims g, int zc, float s, float *__restrict__ ga, float *__restrict__ gb) {
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
    for (int z = z0; z < z1; ++z) {
        const long long p = (long long)z * g.nxy + (long long)y * g.nx + x;
        const float ux = s * __ldg(a + p), uy = s * __ldg(a + g.n + p), uz = s * __ldg(a + 2 * g.n + p);
        const float w0 = __ldg(gw + p), w1 = __ldg(gw + g.n + p), w2 = __ldg(gw + 2 * g.n + p);
        float jx[3], jy[3], jz[3];  // d b_d / d phi_k
#pragma unroll
        for (int d = 0; d < 3; ++d) (void)sample_grad<float, PAD>(b + d * g.n, g, x, y, z, ux, uy, uz, jx[d], jy[d], jz[d]);
        const float s2 = s * s;
        const float gax = fmaf(s2, fmaf(w0, jx[0], fmaf(w1, jx[1], w2 * jx[2])), s * w0);
        const float gay = fmaf(s2, fmaf(w0, jy[0], fmaf(w1, jy[1], w2 * jy[2])), s * w1);
        const float gaz = fmaf(s2, fmaf(w0, jz[0], fmaf(w1, jz[1], w2 * jz[2])), s * w2);
        if (SAME) {
            atomicAdd(gb + p, gax);
            atomicAdd(gb + g.n + p, gay);
            atomicAdd(gb + 2 * g.n + p, gaz);
        } else {
            ga[p] = gax;
            ga[g.n + p] = gay;
            ga[2 * g.n + p] = gaz;
        }
        // the scatter: corner weights of the sample (padding as in the sampler)
        const Axis X = axis_setup<PAD>(x, ux, g.nx), Y = axis_setup<PAD>(y, uy, g.ny), Z = axis_setup<PAD>(z, uz, g.nz);
        const float sw[3] = {s * w0, s * w1, s * w2};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
            const float wt = (bx ? X.a : 1.0f - X.a) * (by ? Y.a : 1.0f - Y.a) * (bz ? Z.a : 1.0f - Z.a);
            const bool valid = (bx ? X.v1 : X.v0) && (by ? Y.v1 : Y.v0) && (bz ? Z.v1 : Z.v0);
            if (!valid || wt == 0.0f) continue;
            const long long q = ((long long)(bz ? Z.i1 : Z.i0) * g.ny + (by ? Y.i1 : Y.i0)) * g.nx + (bx ? X.i1 : X.i0);
#pragma unroll
            for (int d = 0; d < 3; ++d) atomicAdd(gb + d * g.n + q, wt * sw[d]);
        }
    }
}

cudaError_t launch_compose_backward(const float *a, const float *b, const float *gw, const Dims &g, int pad,
                                    float scale, float *ga, float *gb, cudaStream_t s) {
    const MarchGrid G = march_grid(g, 8LL * num_sms() * 4, 1);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    with_pad(pad, [&](auto pd) {
        constexpr int PD = decltype(pd)::value;
        if (ga)
            compose_backward_kernel<PD, false><<<grid, block, 0, s>>>(a, b, gw, g, G.zc, scale, ga, gb);
        else
            compose_backward_kernel<PD, true><<<grid, block, 0, s>>>(a, b, gw, g, G.zc, scale, ga, gb);
    });
    return cudaGetLastError();
}

cudaError_t launch_compose(const float *a, const float *b, const Dims &g, int pad, float scale, float *w,
                           cudaStream_t s) {
    const MarchGrid G = march_grid(g, 8LL * num_sms() * 4, 1);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    with_pad(pad, [&](auto pd) {
        compose_kernel<decltype(pd)::value><<<grid, block, 0, s>>>(a, b, g, G.zc, scale, w);
    });
    return cudaGetLastError();
}

}  // namespace regk
