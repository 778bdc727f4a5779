// warp.cu -- standalone trilinear warp J = M o (id + u) with optional slope
// (Sec. 2.1: the deformable part of the composite implicit grid sampler;
// Algorithm gridsampler, forward).  The identity grid is implicit in the
// thread index, so no coordinate grid is ever materialised.  The fused loss
// sweeps (lncc.cu, mi.cu) call the same device sampler on chip; this kernel
// serves reg_warp and the tests.
#include "kernels.h"

namespace regk {

template <typename T, bool SLOPE, int PAD>
__global__ void __launch_bounds__(TILE_THREADS) warp_kernel(const T *__restrict__ M, const float *__restrict__ u,
                                                            Dims g, int zc, float *__restrict__ J,
                                                            float *__restrict__ dJ) {
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int z0 = blockIdx.z * zc, z1 = min(g.nz, z0 + zc);
    for (int z = z0; z < z1; ++z) {
        const long long p = (long long)z * g.nxy + (long long)y * g.nx + x;
        const float ux = __ldg(u + p), uy = __ldg(u + g.n + p), uz = __ldg(u + 2 * g.n + p);
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
                        cudaStream_t s) {
    const MarchGrid G = march_grid(g, 8LL * num_sms() * 4, 1);
    const dim3 grid(G.tiles_x, G.tiles_y, G.chunks), block(TX, TY);
    with_type(dt, [&](auto tp) {
        using T = elem_t<decltype(tp)>;
        with_pad(pad, [&](auto pd) {
            constexpr int PD = decltype(pd)::value;
            if (dJ)
                warp_kernel<T, true, PD><<<grid, block, 0, s>>>((const T *)M, u, g, G.zc, J, dJ);
            else
                warp_kernel<T, false, PD><<<grid, block, 0, s>>>((const T *)M, u, g, G.zc, J, dJ);
        });
    });
    return cudaGetLastError();
}

}  // namespace regk
