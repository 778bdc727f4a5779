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
template <typename I>
__device__ __forceinline__ float ld_vox(const float *p, I i) {
    return __ldg(p + i);
}
template <typename I>
__device__ __forceinline__ float ld_vox(const __nv_bfloat16 *p, I i) {
    return __bfloat162float(__ldg(p + i));
}

// streaming loads (read once: evict first, so that they do not push the
// reused gather lines of M out of L1)
template <typename I>
__device__ __forceinline__ float ld_vox_cs(const float *p, I i) {
    return __ldcs(p + i);
}
template <typename I>
__device__ __forceinline__ float ld_vox_cs(const __nv_bfloat16 *p, I i) {
    return __bfloat162float(__ldcs(p + i));
}

__device__ __forceinline__ void store_vox(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_vox(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------
// Trilinear sampling of M at phi = p + u (voxel units), value and slope.
// The cell index is taken from p + floor(u) and the fraction from
// u - floor(u) (exact in FP32), so large coordinates lose no precision.
//   BORDER: phi is clamped into [0, n-1] per axis; cell = min(floor, n-2)
//           (the last knot uses the upper cell); slope 0 along a clamped axis.
//   ZEROS : corners outside the volume read as 0.
// ---------------------------------------------------------------------------
struct Axis {
    int i0, i1;   // corner indices (may be out of range in ZEROS mode)
    float a;      // fraction in [0,1]
    float slope;  // 1 or 0 (clamped axis)
    bool v0, v1;  // corner validity (ZEROS)
};

template <int PAD>
__device__ __forceinline__ Axis axis_setup(int p, float uu, int n) {
    Axis ax;
    // non-finite or absurd displacements are clamped; any |u| > 2^20 voxels
    // is outside every supported volume, so border / zero semantics hold.
    uu = (uu == uu) ? fminf(fmaxf(uu, -1048576.0f), 1048576.0f) : 0.0f;
    const float fl = floorf(uu);
    const float a = uu - fl;
    const int f = p + (int)fl;
    if (PAD == REG_PAD_BORDER) {
        const bool lowc = f < 0, highc = f > n - 2;
        ax.slope = (n > 1 && !lowc && (!highc || (f == n - 1 && a == 0.0f))) ? 1.0f : 0.0f;
        ax.i0 = max(lowc ? 0 : (highc ? n - 2 : f), 0);
        ax.i1 = min(ax.i0 + 1, n - 1);
        ax.a = (n == 1 || lowc) ? 0.0f : (highc ? 1.0f : a);
        ax.v0 = ax.v1 = true;
    } else {
        ax.i0 = f;
        ax.i1 = f + 1;
        ax.a = a;
        ax.slope = 1.0f;
        ax.v0 = (unsigned)f < (unsigned)n;
        ax.v1 = (unsigned)(f + 1) < (unsigned)n;
    }
    return ax;
}

// the 8 corner values c[bz*4 + by*2 + bx] (0 outside the volume in ZEROS mode)
// I is the voxel index type: int when the volume has fewer than 2^31 voxels
// (cheaper address arithmetic), long long otherwise.
template <typename T, int PAD, typename I = long long>
__device__ __forceinline__ void gather8(const T *M, const Dims &g, const Axis &X, const Axis &Y, const Axis &Z,
                                        float c[8]) {
    const I r00 = ((I)Z.i0 * g.ny + Y.i0) * g.nx, r01 = ((I)Z.i0 * g.ny + Y.i1) * g.nx;
    const I r10 = ((I)Z.i1 * g.ny + Y.i0) * g.nx, r11 = ((I)Z.i1 * g.ny + Y.i1) * g.nx;
    if (PAD == REG_PAD_BORDER) {
        c[0] = ld_vox(M, r00 + X.i0);
        c[1] = ld_vox(M, r00 + X.i1);
        c[2] = ld_vox(M, r01 + X.i0);
        c[3] = ld_vox(M, r01 + X.i1);
        c[4] = ld_vox(M, r10 + X.i0);
        c[5] = ld_vox(M, r10 + X.i1);
        c[6] = ld_vox(M, r11 + X.i0);
        c[7] = ld_vox(M, r11 + X.i1);
    } else {
        const bool y0z0 = Y.v0 && Z.v0, y1z0 = Y.v1 && Z.v0, y0z1 = Y.v0 && Z.v1, y1z1 = Y.v1 && Z.v1;
        c[0] = (X.v0 && y0z0) ? ld_vox(M, r00 + X.i0) : 0.0f;
        c[1] = (X.v1 && y0z0) ? ld_vox(M, r00 + X.i1) : 0.0f;
        c[2] = (X.v0 && y1z0) ? ld_vox(M, r01 + X.i0) : 0.0f;
        c[3] = (X.v1 && y1z0) ? ld_vox(M, r01 + X.i1) : 0.0f;
        c[4] = (X.v0 && y0z1) ? ld_vox(M, r10 + X.i0) : 0.0f;
        c[5] = (X.v1 && y0z1) ? ld_vox(M, r10 + X.i1) : 0.0f;
        c[6] = (X.v0 && y1z1) ? ld_vox(M, r11 + X.i0) : 0.0f;
        c[7] = (X.v1 && y1z1) ? ld_vox(M, r11 + X.i1) : 0.0f;
    }
}

// (1-a) lo + a hi, exact at a = 0 and a = 1 (so u = 0 reproduces M bit for bit)
__device__ __forceinline__ float lerp1(float a, float lo, float hi) { return fmaf(a, hi, (1.0f - a) * lo); }

// Fast path of both samplers: when every axis has 0 <= p + floor(u) <= n-2
// (a finite displacement whose whole cell lies inside the volume) the two
// padding modes agree -- fraction = u - floor(u), slope 1, all 8 corners
// valid -- and the corners sit at fixed offsets from one base pointer.  The
// test fails for NaN / infinite / huge u (the fraction is not in [0, 1) or
// the index is out of range), which then take the general path above; the
// arithmetic of the interpolation is the same on both paths, so the result
// does not depend on which one ran.
struct Cell {
    int ix, iy, iz;
    float ax, ay, az;
};
__device__ __forceinline__ bool interior_cell(const Dims &g, int x, int y, int z, float ux, float uy, float uz,
                                              Cell &c) {
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
    c.ax = ux - fx;
    c.ay = uy - fy;
    c.az = uz - fz;
    // saturating conversions and wrap-around unsigned sums: a huge or NaN u
    // gives an index or a fraction that fails the test below
    c.ix = (int)((unsigned)x + (unsigned)__float2int_rz(fx));
    c.iy = (int)((unsigned)y + (unsigned)__float2int_rz(fy));
    c.iz = (int)((unsigned)z + (unsigned)__float2int_rz(fz));
    const bool in = (unsigned)c.ix < (unsigned)(g.nx - 1) && (unsigned)c.iy < (unsigned)(g.ny - 1) &&
                    (unsigned)c.iz < (unsigned)(g.nz - 1);
    return in && c.ax >= 0.0f && c.ay >= 0.0f && c.az >= 0.0f;
}
template <typename T, typename I>
__device__ __forceinline__ void gather8_interior(const T *M, const Dims &g, const Cell &c, float v[8]) {
    const T *q = M + ((I)c.iz * g.ny + c.iy) * g.nx + c.ix;
    const I nx = (I)g.nx, nxy = (I)g.nxy;
    const T *q1 = q + nx, *q2 = q + nxy, *q3 = q2 + nx;
    v[0] = ld_vox(q, 0);
    v[1] = ld_vox(q, 1);
    v[2] = ld_vox(q1, 0);
    v[3] = ld_vox(q1, 1);
    v[4] = ld_vox(q2, 0);
    v[5] = ld_vox(q2, 1);
    v[6] = ld_vox(q3, 0);
    v[7] = ld_vox(q3, 1);
}

// A value-only sample split in two: gather_corners issues the 8 corner
// loads and sets the fractions, interp_corners interpolates them.  A caller
// can gather one sample before it interpolates another (software
// pipelining); sample() is the two back to back.
struct Corners {
    float c[8];
    float ax, ay, az;
};
template <typename T, int PAD, typename I = long long>
__device__ __forceinline__ void gather_corners(const T *M, const Dims &g, int x, int y, int z, float ux, float uy,
                                               float uz, Corners &k) {
    Cell cell;
    if (interior_cell(g, x, y, z, ux, uy, uz, cell)) {
        gather8_interior<T, I>(M, g, cell, k.c);
        k.ax = cell.ax;
        k.ay = cell.ay;
        k.az = cell.az;
    } else {
        const Axis X = axis_setup<PAD>(x, ux, g.nx);
        const Axis Y = axis_setup<PAD>(y, uy, g.ny);
        const Axis Z = axis_setup<PAD>(z, uz, g.nz);
        gather8<T, PAD, I>(M, g, X, Y, Z, k.c);
        k.ax = X.a;
        k.ay = Y.a;
        k.az = Z.a;
    }
}
__device__ __forceinline__ float interp_corners(const Corners &k) {
    const float e00 = lerp1(k.ax, k.c[0], k.c[1]), e10 = lerp1(k.ax, k.c[2], k.c[3]);
    const float e01 = lerp1(k.ax, k.c[4], k.c[5]), e11 = lerp1(k.ax, k.c[6], k.c[7]);
    const float f0 = lerp1(k.ay, e00, e10), f1 = lerp1(k.ay, e01, e11);
    return lerp1(k.az, f0, f1);
}

// value only
template <typename T, int PAD, typename I = long long>
__device__ __forceinline__ float sample(const T *M, const Dims &g, int x, int y, int z, float ux, float uy,
                                        float uz) {
    Corners k;
    gather_corners<T, PAD, I>(M, g, x, y, z, ux, uy, uz, k);
    return interp_corners(k);
}

// value and slope dJ/dphi
template <typename T, int PAD, typename I = long long>
__device__ __forceinline__ float sample_grad(const T *M, const Dims &g, int x, int y, int z, float ux, float uy,
                                             float uz, float &gx, float &gy, float &gz) {
    float c[8];
    float ax, ay, az, sx = 1.0f, sy = 1.0f, sz = 1.0f;
    Cell cell;
    if (interior_cell(g, x, y, z, ux, uy, uz, cell)) {
        gather8_interior<T, I>(M, g, cell, c);
        ax = cell.ax;
        ay = cell.ay;
        az = cell.az;
    } else {
        const Axis X = axis_setup<PAD>(x, ux, g.nx);
        const Axis Y = axis_setup<PAD>(y, uy, g.ny);
        const Axis Z = axis_setup<PAD>(z, uz, g.nz);
        gather8<T, PAD, I>(M, g, X, Y, Z, c);
        ax = X.a;
        ay = Y.a;
        az = Z.a;
        sx = X.slope;
        sy = Y.slope;
        sz = Z.slope;
    }
    const float d00 = c[1] - c[0], d10 = c[3] - c[2], d01 = c[5] - c[4], d11 = c[7] - c[6];
    const float e00 = lerp1(ax, c[0], c[1]), e10 = lerp1(ax, c[2], c[3]);
    const float e01 = lerp1(ax, c[4], c[5]), e11 = lerp1(ax, c[6], c[7]);
    const float f0 = lerp1(ay, e00, e10), f1 = lerp1(ay, e01, e11);
    const float dy0 = e10 - e00, dy1 = e11 - e01;
    const float dx0 = fmaf(ay, d10 - d00, d00), dx1 = fmaf(ay, d11 - d01, d01);
    gz = (f1 - f0) * sz;
    gy = fmaf(az, dy1 - dy0, dy0) * sy;
    gx = fmaf(az, dx1 - dx0, dx0) * sx;
    return lerp1(az, f0, f1);
}

// ---------------------------------------------------------------------------
// composite transform phi(p) = A p + t + S u(p) (Sec. 2.1, the composite
// implicit grid sampler; Algorithm gridsampler).  The kernels call the
// deformable sampler with the displacement u' = (A - I) p + t + S u, so that
// phi = p + u' and the interior test, the padding and the interpolation are
// those of the plain sampler.  No coordinate grid is materialised.
// ---------------------------------------------------------------------------
struct AffineT {
    float am[9];  // A - I, row-major: row i is output axis i (x, y, z)
    float t[3];   // translation, voxels
    float s[3];   // S = diag(s)
    // when set, the transform is read on the device instead: 15 floats in the
    // layout of reg_affine (A row-major, t, s), written by an earlier kernel
    const float *dev = nullptr;
};
// The transform a kernel applies: its by-value parameter, or the device copy
// that parameter points to (A - I formed in FP32, the same rounding as the
// host's (float)((double)A - 1) of a float A).
__device__ __forceinline__ AffineT resolve_affine(const AffineT &A) {
    if (A.dev == nullptr) return A;
    AffineT r;
#pragma unroll
    for (int i = 0; i < 9; ++i) r.am[i] = __ldg(A.dev + i) - (i % 4 == 0 ? 1.0f : 0.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r.t[i] = __ldg(A.dev + 9 + i);
        r.s[i] = __ldg(A.dev + 12 + i);
    }
    r.dev = nullptr;
    return r;
}
__device__ __forceinline__ void composite_disp(const AffineT &T, int x, int y, int z, float &ux, float &uy,
                                               float &uz) {
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float ox = fmaf(T.am[0], fx, fmaf(T.am[1], fy, fmaf(T.am[2], fz, T.t[0])));
    const float oy = fmaf(T.am[3], fx, fmaf(T.am[4], fy, fmaf(T.am[5], fz, T.t[1])));
    const float oz = fmaf(T.am[6], fx, fmaf(T.am[7], fy, fmaf(T.am[8], fz, T.t[2])));
    ux = fmaf(T.s[0], ux, ox);
    uy = fmaf(T.s[1], uy, oy);
    uz = fmaf(T.s[2], uz, oz);
}

// Per-thread sums for dC/dA = sum_p gX(p) p^T and dC/dt = sum_p gX(p), gX
// the gradient with respect to the sampling location.  A thread marches one
// (x, y) column, so along it only sum g and sum g z are needed.
struct AffineAcc {
    float G[3] = {0.f, 0.f, 0.f}, Z[3] = {0.f, 0.f, 0.f};
    __device__ __forceinline__ void add(float gx, float gy, float gz, int z) {
        const float fz = (float)z;
        G[0] += gx;
        G[1] += gy;
        G[2] += gz;
        Z[0] = fmaf(gx, fz, Z[0]);
        Z[1] = fmaf(gy, fz, Z[1]);
        Z[2] = fmaf(gz, fz, Z[2]);
    }
};

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

// Fixed-order reduction of every thread's AffineAcc (column (x, y)) into
// out[12] = dC/dA row-major, then dC/dt.  Every thread of the block calls it
// (threads outside the volume with empty sums); partials holds 12 doubles
// per block.
__device__ __forceinline__ void affine_reduce(const AffineAcc &a, int x, int y, double *partials, unsigned *counter,
                                              double *out, double *red, unsigned *err) {
    double v[12];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        v[3 * i + 0] = (double)x * (double)a.G[i];
        v[3 * i + 1] = (double)y * (double)a.G[i];
        v[3 * i + 2] = (double)a.Z[i];
        v[9 + i] = (double)a.G[i];
    }
    const int tid = linear_tid();
    const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll 1
    for (int k = 0; k < 12; ++k) {
        const double bs = block_sum(v[k], red);
        if (tid == 0) partials[bid * 12 + k] = bs;
    }
    if (arrive_last(counter)) {
        const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
        const int nt = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll 1
        for (int k = 0; k < 12; ++k) {
            double acc = 0.0;
            for (long long i = tid; i < nb; i += nt) acc += __ldcg(partials + i * 12 + k);
            const double tot = block_sum(acc, red);
            if (tid == 0) {
                if (!isfinite(tot)) latch_error(err, REG_ERR_NONFINITE);
                out[k] = tot;
            }
        }
        if (tid == 0) *counter = 0u;
    }
}

}  // namespace regk
