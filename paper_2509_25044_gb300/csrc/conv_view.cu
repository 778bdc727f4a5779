// conv_view.cu -- 3 x 3 x 3 convolution (zero padding 1, stride 1) as an
// implicit GEMM on the tcgen05 tensor cores, fed by TMA "views".
//
// A CTA owns an output tile of Tz planes x Ty rows x the whole x extent.  For
// each chunk of 16 input channels it loads, with two tiled TMA copies (one
// per 8-channel group), the input brick that the tile's 27 taps touch:
// (Tz+2) planes x (Ty+2) rows x (nx+2) columns starting at (-1, y0-1, z0-1),
// zero-filled outside the volume -- the zero padding comes for free.  In
// shared memory the brick is position-major (16 bytes = 8 channels per
// position), so the rows of the GEMM's A operand for tap (dx, dy, dz) are
// simply the brick positions shifted by dz (Ty+2)(nx+2) + dy (nx+2) + dx:
// every tap is one matrix descriptor with a different start address and no
// im2col copy is made.  The M dimension runs over brick positions, 128 per
// MMA; positions in the halo columns produce junk rows that the epilogue
// drops (2 of every nx+2).  The chunk's weights arrive by one bulk copy,
// pre-tiled on the device into the canonical K-major layout.  One thread
// issues the copies and the MMAs (FP32 accumulators in TMEM, one 128-lane
// block of Nb columns per M-tile); all waits are bounded and a timeout is
// latched in the device error word.
#include <algorithm>

#include "kernels.h"
#include "tma.cuh"

namespace regk {

namespace tma {
namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
    static const EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiled) nullptr;
        return (EncodeTiled)p;
    }();
    return fn;
}
}  // namespace

bool make_map_bf16_4d(CUtensorMap *map, const void *base, const uint64_t dims[4], const uint32_t box[4]) {
    const EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t gdim[4] = {dims[0], dims[1], dims[2], dims[3]};
    const cuuint64_t gstride[3] = {dims[0] * 2, dims[0] * dims[1] * 2, dims[0] * dims[1] * dims[2] * 2};
    const cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), gdim, gstride, bx, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_map(CUtensorMap *map, const void *base, int dt, int rank, const uint64_t *dims, const uint32_t *box) {
    const EncodeTiled fn = encode_fn();
    if (!fn || rank < 1 || rank > 5) return false;
    const uint64_t es = dt == REG_BF16 ? 2 : 4;
    cuuint64_t gdim[5], gstride[4];
    cuuint32_t bx[5], estr[5];
    uint64_t stride = es;
    for (int i = 0; i < rank; ++i) {
        gdim[i] = dims[i];
        bx[i] = box[i];
        estr[i] = 1;
        if (i > 0) gstride[i - 1] = stride;
        stride *= dims[i];
    }
    return fn(map, dt == REG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
              (cuuint32_t)rank, const_cast<void *>(base), gdim, gstride, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace tma

namespace {

constexpr int VIEW_THREADS = 128;  // one TMEM lane (GEMM row) per thread in the epilogue
constexpr int VIEW_CK = 16;        // input channels per chunk (one MMA K step)

struct ViewGeom {
    int nx, ny, nz;
    int Cin, nchunks;       // nchunks = Cin / 16
    int Cout, Nb;           // real output channels; MMA N per block of columns (multiple of 16, <= 64)
    int Ty, Tz, P, By, Bz;  // tile rows / planes; brick pitch (nx + 2), rows (Ty + 2), planes (Tz + 2)
    int tiles_y;
    int MT;                 // 128-row M-tiles per CTA
    int q0;                 // brick position of the tile's first output (z, y, x) = (1, 1, 1)
    int VGB;                // bytes per 8-channel region of the brick (incl. read slack), multiple of 1024
    int tmem_cols;
    uint32_t tx_bytes;      // bytes landing per chunk (two brick copies + weights)
    uint32_t wbytes;        // weight bytes per chunk
    float slope;
};

__host__ __device__ constexpr int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

// weight tiles: Wt[nb][chunk][tap][kg][ng][r][e] = W[nb Nb + 8 ng + r][tap Cin + 16 chunk + 8 kg + e]
__global__ void tile_weights_kernel(const __nv_bfloat16 *__restrict__ W, int rows, int Kpad, int Cin, int Nb,
                                    int nblocks, __nv_bfloat16 *__restrict__ Wt) {
    const long long total = (long long)nblocks * Nb * 27 * Cin;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int e = (int)(i & 7);
    const int r = (int)((i >> 3) & 7);
    long long rest = i >> 6;
    const int ngs = Nb / 8;
    const int ng = (int)(rest % ngs);
    rest /= ngs;
    const int kg = (int)(rest & 1);
    rest >>= 1;
    const int tap = (int)(rest % 27);
    rest /= 27;
    const int nch = Cin / VIEW_CK;
    const int chunk = (int)(rest % nch);
    const int nb = (int)(rest / nch);
    const int row = nb * Nb + ng * 8 + r;
    const int k = tap * Cin + chunk * VIEW_CK + kg * 8 + e;
    Wt[i] = row < rows ? W[(size_t)row * Kpad + k] : __float2bfloat16_rn(0.0f);
}

template <int EPI>
__global__ void __launch_bounds__(VIEW_THREADS, 1)
    conv_view_kernel(const __grid_constant__ CUtensorMap map, const __nv_bfloat16 *__restrict__ Wt,
                     const float *__restrict__ bias, void *__restrict__ out, ViewGeom G, unsigned *err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (umma::smem_addr(smem_raw) & 1023u)) & 1023u);
    unsigned char *view = sm;                              // 2 regions of VGB bytes
    unsigned char *wts = sm + 2 * (size_t)G.VGB;           // weights of one chunk
    uint64_t *bars = reinterpret_cast<uint64_t *>(wts + G.wbytes);  // [0] loads, [1] MMAs
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2);
    int *flag = reinterpret_cast<int *>(tmem_holder + 1);

    const int tid = threadIdx.x;
    const int tile = blockIdx.x, nb = blockIdx.y;
    const int y0 = (tile % G.tiles_y) * G.Ty, z0 = (tile / G.tiles_y) * G.Tz;

    if (tid == 0) {
        umma::mbar_init(&bars[0], 1);
        umma::mbar_init(&bars[1], 1);
        *flag = 0;
    }
    if (tid < 32) umma::tmem_alloc(tmem_holder, (uint32_t)G.tmem_cols);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    if (tid == 0) {
        bool ok = true;
        const uint32_t idesc = umma::idesc_bf16(128, G.Nb, 0, 0);
        const uint32_t vaddr = umma::smem_addr(view), waddr = umma::smem_addr(wts);
        const int plane = G.By * G.P;
        for (int c = 0; c < G.nchunks && ok; ++c) {
            if (c > 0 && !umma::mbar_wait(&bars[1], (c - 1) & 1)) {  // brick free again
                umma::mbar_wait(&bars[1], (c - 1) & 1);  // one more bounded wait for the MMAs in flight
                ok = false;
                break;
            }
            tma::expect_tx(&bars[0], G.tx_bytes);
            tma::load_4d(view, &map, c * VIEW_CK, -1, y0 - 1, z0 - 1, &bars[0]);
            tma::load_4d(view + G.VGB, &map, c * VIEW_CK + 8, -1, y0 - 1, z0 - 1, &bars[0]);
            tma::load_bulk(wts, Wt + ((size_t)nb * G.nchunks + c) * (G.wbytes / 2), G.wbytes, &bars[0]);
            if (!umma::mbar_wait(&bars[0], c & 1)) {
                umma::mbar_wait(&bars[0], c & 1);  // one more bounded wait for the copies in flight
                ok = false;
                break;
            }
            umma::fence_after_sync();
            // descriptors move by whole 16-byte units: add to the start field
            const uint64_t a_base = umma::sdesc(vaddr + (uint32_t)(G.q0 * 16), (uint32_t)G.VGB, 128u);
            const uint64_t b_base = umma::sdesc(waddr, (uint32_t)(G.Nb / 8) * 128u, 128u);
#pragma unroll 1
            for (int t = 0; t < 27; ++t) {
                const int off = (t / 9 - 1) * plane + ((t / 3) % 3 - 1) * G.P + (t % 3 - 1);
                const uint64_t bd = b_base + (uint64_t)(2 * t * G.Nb);  // t * 32 Nb bytes
                const uint64_t ad0 = a_base + (uint64_t)(int64_t)off;
                const uint32_t acc = (c > 0 || t > 0) ? 1u : 0u;
                for (int j = 0; j < G.MT; ++j)
                    umma::mma_bf16(tmem + (uint32_t)(j * G.Nb), ad0 + (uint64_t)(128 * j), bd, idesc, acc);
            }
            umma::commit(&bars[1]);
        }
        if (!ok) *flag = 1;
    }
    // Only after thread 0 has issued every chunk may the others wait on the
    // MMA barrier: its parity repeats every two chunks.
    __syncthreads();
    bool done = *flag == 0 && umma::mbar_wait(&bars[1], (G.nchunks - 1) & 1);
    umma::fence_after_sync();
    if (!done) {
        if (tid == 0) {
            latch_error(err, REG_ERR_TIMEOUT);
            if (*flag == 0) umma::mbar_wait(&bars[1], (G.nchunks - 1) & 1);  // MMAs still in flight
        }
    } else {
        const int warp = tid >> 5;
        const int plane = G.By * G.P;
        for (int j = 0; j < G.MT; ++j) {
            const int rel = j * 128 + tid;
            const int zz = rel / plane, rem = rel - zz * plane;
            const int yy = rem / G.P, xx = rem - yy * G.P;
            const int z = z0 + zz, y = y0 + yy;
            const bool valid = zz < G.Tz && yy < G.Ty && xx < G.nx && z < G.nz && y < G.ny;
            const long long v = ((long long)z * G.ny + y) * G.nx + xx;
            for (int c0 = 0; c0 < G.Nb; c0 += 16) {
                float acc[16];
                umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * G.Nb + c0), acc);
                if (!valid) continue;
                const int ch0 = nb * G.Nb + c0;
                if (EPI == EPI_BIAS_F32_SOA) {
                    float *o = reinterpret_cast<float *>(out);
                    const long long nvox = (long long)G.nx * G.ny * G.nz;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (ch0 + i < G.Cout) o[(size_t)(ch0 + i) * nvox + v] = acc[i] + bias[ch0 + i];
                } else {
                    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out) + v * G.Cout;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (ch0 + 8 * h >= G.Cout) continue;
                        __align__(16) __nv_bfloat16 tv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float a = acc[8 * h + i];
                            if (EPI == EPI_BIAS_LEAKY_BF16) {
                                a += bias[ch0 + 8 * h + i];
                                a = a > 0.0f ? a : G.slope * a;
                            }
                            tv[i] = __float2bfloat16_rn(a);
                        }
                        *reinterpret_cast<uint4 *>(o + ch0 + 8 * h) = *reinterpret_cast<const uint4 *>(tv);
                    }
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid < 32) umma::tmem_dealloc(tmem, (uint32_t)G.tmem_cols);
}

// N split into blocks of at most 64 columns (multiples of 16)
void n_blocks(int N, int &Nb, int &nblocks) {
    nblocks = (N + 63) / 64;
    Nb = ((N + nblocks - 1) / nblocks + 15) / 16 * 16;
}

size_t view_smem_bytes(const ViewGeom &G) { return 2 * (size_t)G.VGB + G.wbytes + 64 + 1024; }

// Tile choice: the largest useful fraction of the GEMM rows the whole launch
// occupies -- valid outputs / (waves x resident CTAs x MT x 128), with the
// residency each tile's shared and tensor memory allow, so that a last wave
// that leaves most SMs idle counts against a tile -- then the fewest brick
// rows per output row; tiles need at most 113 KB of shared memory and 256
// tensor-memory columns (at least 2 CTAs per SM), with 1 CTA per SM as the
// fallback.
bool choose_geom(const Dims &d, int Cin, int Cout, int N, float slope, ViewGeom &G) {
    if (Cin % VIEW_CK || Cin < VIEW_CK || d.nx + 2 > 256) return false;
    G.nx = d.nx;
    G.ny = d.ny;
    G.nz = d.nz;
    G.Cin = Cin;
    G.nchunks = Cin / VIEW_CK;
    G.Cout = Cout;
    int nblocks;
    n_blocks(N, G.Nb, nblocks);
    G.P = d.nx + 2;
    G.wbytes = (uint32_t)(27 * 32 * G.Nb);
    G.slope = slope;
    for (int pass = 0; pass < 2; ++pass) {
        const size_t smem_cap = pass == 0 ? 113 * 1024 : 220 * 1024;
        const int tmem_cap = pass == 0 ? 256 : 512;
        double best = -1.0;
        ViewGeom bestG = G;
        const int tz_opts[3] = {1, 2, 4};
        for (int zi = 0; zi < 3; ++zi) {
            const int Tz = tz_opts[zi];
            if (Tz > d.nz || Tz + 2 > 256) continue;
            for (int Ty = 1; Ty <= d.ny && Ty + 2 <= 256; ++Ty) {
                ViewGeom g = G;
                g.Ty = Ty;
                g.Tz = Tz;
                g.By = Ty + 2;
                g.Bz = Tz + 2;
                const int plane = g.By * g.P;
                const int span = (Tz - 1) * plane + (Ty - 1) * g.P + d.nx;
                g.MT = (span + 127) / 128;
                g.tmem_cols = pow2_cols(g.MT * g.Nb);
                if (g.MT * g.Nb > tmem_cap) continue;
                g.q0 = plane + g.P + 1;
                const int need = std::max(g.Bz * plane, g.q0 + g.MT * 128 + plane + g.P + 2);
                g.VGB = (need * 16 + 1023) / 1024 * 1024;
                if (view_smem_bytes(g) > smem_cap) continue;
                const int ty_tiles = (d.ny + Ty - 1) / Ty, tz_tiles = (d.nz + Tz - 1) / Tz;
                // CTAs resident per SM: 228 KB of shared memory (1 KB reserved per
                // CTA) and 512 tensor-memory columns per SM, 16 CTAs of 128 threads
                const long long by_smem = (228LL * 1024) / ((long long)view_smem_bytes(g) + 1024);
                const long long by_tmem = 512 / g.tmem_cols;
                const long long per_sm = std::max(1LL, std::min(std::min(by_smem, by_tmem), 16LL));
                const long long slots = per_sm * num_sms();
                const long long ctas = (long long)ty_tiles * tz_tiles * nblocks;
                const long long waves = (ctas + slots - 1) / slots;
                const double eff = (double)d.nx * d.ny * d.nz * nblocks / ((double)waves * slots * g.MT * 128.0);
                const double reuse = (double)(g.By * g.Bz) / (double)(Ty * Tz);
                const double score = eff / (1.0 + 0.01 * reuse);
                if (score > best) {
                    best = score;
                    bestG = g;
                }
            }
        }
        if (best > 0.0) {
            G = bestG;
            G.tiles_y = (d.ny + G.Ty - 1) / G.Ty;
            G.tx_bytes = (uint32_t)(2 * G.Bz * G.By * G.P * 16) + G.wbytes;
            return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores:
//   dW[co][tap][ci] = sum over voxels p of dpre[p][co] * in[p + off(tap)][ci]
// The voxels are the GEMM's K dimension.  Persistent CTAs (one per SM) each
// take a contiguous range of tiles (one plane, Ty rows, the whole x extent)
// and keep the 27 per-tap accumulators D_tap[co][16 ci] in TMEM (27 x 16 of
// the 512 columns) while they stream their tiles through a 2-stage TMA ring:
//   A = dpre^T, MN-major: the tile's rows of dpre (x from -1 to nx, so the two
//       halo columns are zero), one shared region per 8-channel group; M is
//       128, the regions of channel groups >= Cout / 8 stay zero;
//   B = the input brick of the tile (3 planes x Ty+2 rows x nx+2 columns,
//       zero outside the volume) for one 16-channel chunk, MN-major, shifted
//       by the tap's offset exactly as in the forward kernel.
// After its tiles a CTA writes its 27 x 16 partial sums per output channel
// for the chunk; the partials are summed over CTAs in a fixed order.
// ---------------------------------------------------------------------------
constexpr int WG_BOFF = 8;  // zeroed positions in front of each brick region (the tap -1 reads)

struct WgGeom {
    int nx, ny, nz, Cin, Cout, nchunks;
    int Ty, P, By;        // tile rows, row pitch (nx + 2), brick rows (Ty + 2)
    int tiles_y, ntiles;  // ntiles = nz * tiles_y
    int ksteps;           // ceil(Ty P / 16)
    int cgo;              // real 8-channel groups of dpre (Cout / 8)
    int VGX, VGD;         // bytes per brick region / dpre region (multiples of 128)
    uint32_t tx_bytes;    // bytes landing per tile
};

__host__ __device__ inline size_t wg_stage_bytes(const WgGeom &G) { return 2 * (size_t)G.VGX + 16 * (size_t)G.VGD; }
__host__ __device__ inline size_t wg_smem_bytes(const WgGeom &G) { return 2 * wg_stage_bytes(G) + 128 + 1024; }

bool choose_wg(const Dims &d, int Cin, int Cout, WgGeom &G) {
    if (Cin % VIEW_CK || Cin < VIEW_CK || Cout % 8 || Cout < 8 || Cout > 128 || d.nx + 2 > 256) return false;
    G.nx = d.nx;
    G.ny = d.ny;
    G.nz = d.nz;
    G.Cin = Cin;
    G.Cout = Cout;
    G.nchunks = Cin / VIEW_CK;
    G.cgo = Cout / 8;
    G.P = d.nx + 2;
    double best = -1.0;
    WgGeom bestG = G;
    for (int Ty = 1; Ty <= d.ny && Ty + 2 <= 256; ++Ty) {
        WgGeom g = G;
        g.Ty = Ty;
        g.By = Ty + 2;
        g.ksteps = (Ty * g.P + 15) / 16;
        const int brick = 3 * g.By * g.P;
        g.VGX = ((WG_BOFF + brick + 32) * 16 + 127) / 128 * 128;  // reads end within 16 positions of the brick
        g.VGD = ((16 * g.ksteps + 16) * 16 + 127) / 128 * 128;
        if (wg_smem_bytes(g) > 220 * 1024) break;
        g.tiles_y = (d.ny + Ty - 1) / Ty;
        const double useful = (double)d.nx * d.ny / (double)(g.tiles_y * 16 * g.ksteps);
        const double reload = 3.0 * g.By / Ty;
        const double score = useful - 0.02 * reload;
        if (score > best) {
            best = score;
            bestG = g;
        }
    }
    if (best < 0.0) return false;
    G = bestG;
    G.ntiles = G.tiles_y * d.nz;
    // too few tiles to occupy the SMs (a 16^3 level): the gather kernel's
    // voxel split is faster there
    if (G.ntiles < num_sms() / 2) return false;
    G.tx_bytes = (uint32_t)(2 * 3 * G.By * G.P * 16 + G.cgo * G.Ty * G.P * 16);
    return true;
}

__global__ void __launch_bounds__(VIEW_THREADS, 1)
    conv_wgrad_view_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dmap,
                           WgGeom G, float *__restrict__ part, unsigned *err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (umma::smem_addr(smem_raw) & 1023u)) & 1023u);
    const size_t stage_bytes = wg_stage_bytes(G);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * stage_bytes);  // [0,1] loads, [2,3] MMAs
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 4);
    int *flag = reinterpret_cast<int *>(tmem_holder + 1);
    const int tid = threadIdx.x;

    // zero both stages once: the dpre regions of absent channel groups, the
    // slack behind every region and the front guard of the bricks are never
    // written by the copies and must read as 0
    {
        uint4 *z = reinterpret_cast<uint4 *>(sm);
        const size_t n16 = 2 * stage_bytes / 16;
        for (size_t i = tid; i < n16; i += VIEW_THREADS) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) umma::mbar_init(&bars[i], 1);
        *flag = 0;
    }
    if (tid < 32) umma::tmem_alloc(tmem_holder, 512u);
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    const long long t_beg = (long long)G.ntiles * blockIdx.x / gridDim.x;
    const long long t_end = (long long)G.ntiles * (blockIdx.x + 1) / gridDim.x;
    const int per_chunk = (int)(t_end - t_beg);
    const int total = per_chunk * G.nchunks;
    const uint32_t idesc = umma::idesc_bf16(128, 16, 1, 1);
    const int plane = G.By * G.P;
    const int q0 = WG_BOFF + (G.By + 1) * G.P;
    // brick offset of each tap in positions (= 16-byte descriptor units)
    int toff[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) toff[t] = (t / 9 - 1) * plane + ((t / 3) % 3 - 1) * G.P + (t % 3 - 1);

    auto stage_ptr = [&](int st) { return sm + (size_t)st * stage_bytes; };
    auto issue_load = [&](int it) {
        const int st = it & 1;
        const int chunk = it / per_chunk;
        const long long tile = t_beg + it % per_chunk;
        const int z = (int)(tile / G.tiles_y), y0 = (int)(tile % G.tiles_y) * G.Ty;
        unsigned char *xs = stage_ptr(st);
        unsigned char *ds = xs + 2 * (size_t)G.VGX;
        tma::expect_tx(&bars[st], G.tx_bytes);
        for (int g = 0; g < 2; ++g)
            tma::load_4d(xs + (size_t)g * G.VGX + WG_BOFF * 16, &xmap, chunk * VIEW_CK + 8 * g, -1, y0 - 1, z - 1,
                         &bars[st]);
        for (int g = 0; g < G.cgo; ++g) tma::load_4d(ds + (size_t)g * G.VGD, &dmap, 8 * g, -1, y0, z, &bars[st]);
    };

    bool ok = true;
    int it = 0;
    if (tid == 0 && total > 0) issue_load(0);
    for (int chunk = 0; chunk < G.nchunks; ++chunk) {
        if (tid == 0) {
            for (int i = 0; i < per_chunk && ok; ++i, ++it) {
                if (it + 1 < total) {
                    // the stage of iteration it + 1 was last read by iteration it - 1
                    if (it >= 1 && !umma::mbar_wait(&bars[2 + ((it + 1) & 1)], ((it - 1) >> 1) & 1)) {
                        ok = false;
                        break;
                    }
                    issue_load(it + 1);
                }
                if (!umma::mbar_wait(&bars[it & 1], (it >> 1) & 1)) {
                    ok = false;
                    break;
                }
                umma::fence_after_sync();
                const uint32_t xa = umma::smem_addr(stage_ptr(it & 1));
                const uint32_t da = xa + 2 * (uint32_t)G.VGX;
                // descriptors move by whole 16-byte units: add to the start field
                const uint64_t ad0 = umma::sdesc(da, 128u, (uint32_t)G.VGD);
                const uint64_t bd0 = umma::sdesc(xa + (uint32_t)(q0 * 16), 128u, (uint32_t)G.VGX);
                for (int ks = 0; ks < G.ksteps; ++ks) {
                    const uint64_t ad = ad0 + (uint64_t)(16 * ks);
                    const uint64_t bk = bd0 + (uint64_t)(16 * ks);
                    const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                    for (int t = 0; t < 27; ++t)
                        umma::mma_bf16(tmem + (uint32_t)(t * 16), ad, bk + (uint64_t)(int64_t)toff[t], idesc, acc);
                }
                umma::commit(&bars[2 + (it & 1)]);
            }
            if (!ok) *flag = 1;
        }
        __syncthreads();
        if (*flag) break;
        // the chunk's last MMAs complete, then every warp reads its 32 TMEM lanes
        // (only thread 0 advances `it`; every thread derives the last iteration)
        const int last = (chunk + 1) * per_chunk - 1;
        if (per_chunk > 0 && !umma::mbar_wait(&bars[2 + (last & 1)], (last >> 1) & 1)) {
            if (tid == 0) *flag = 1;
        }
        umma::fence_after_sync();
        __syncthreads();
        if (*flag) break;
        const int warp = tid >> 5, row = tid;
        const int K = 27 * G.Cin;
        float *dst = part + ((size_t)blockIdx.x * G.Cout + row) * K + chunk * VIEW_CK;
        for (int t = 0; t < 27; ++t) {
            float acc[16];
            umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 16), acc);
            if (row < G.Cout) {
#pragma unroll
                for (int j = 0; j < 16; ++j) dst[(size_t)t * G.Cin + j] = per_chunk > 0 ? acc[j] : 0.0f;
            }
        }
        umma::fence_before_sync();
        __syncthreads();
    }
    if (*flag) {
        if (tid == 0) {
            latch_error(err, REG_ERR_TIMEOUT);
            // bounded waits for whatever may still be in flight
            if (it >= 1) umma::mbar_wait(&bars[2 + ((it - 1) & 1)], ((it - 1) >> 1) & 1);
            umma::mbar_wait(&bars[it & 1], (it >> 1) & 1);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid < 32) umma::tmem_dealloc(tmem, 512u);
}

// dW[co][k] (FP32, [Cout][Kpad]) = sum over CTAs (fixed order) of part[cta][co][k]
__global__ void wg_reduce_kernel(const float *__restrict__ part, int nparts, int Cout, int K, int Kpad,
                                 float *__restrict__ dW) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Cout * Kpad) return;
    const int co = idx / Kpad, k = idx % Kpad;
    float acc = 0.0f;
    if (k < K)
        for (int c = 0; c < nparts; ++c) acc += part[((size_t)c * Cout + co) * K + k];
    dW[idx] = acc;
}

}  // namespace

size_t conv_view_weight_bytes(int Cin, int N) {
    if (Cin % VIEW_CK || Cin < VIEW_CK) return 0;
    int Nb, nblocks;
    n_blocks(N, Nb, nblocks);
    return sizeof(__nv_bfloat16) * (size_t)nblocks * Nb * 27 * Cin;
}

// Returns cudaErrorNotSupported when the shape has no view path (the caller
// then runs the gather kernel).
cudaError_t launch_conv_view(const void *in, int Cin, const void *W, int rows, int Kpad, const float *bias, int Cout,
                             int N, const Dims &d, int epi, float slope, void *Wt_scratch, void *out, cudaStream_t s) {
    ViewGeom G;
    if (!choose_geom(d, Cin, Cout, N, slope, G)) return cudaErrorNotSupported;
    CUtensorMap map;
    const uint64_t dims[4] = {(uint64_t)Cin, (uint64_t)d.nx, (uint64_t)d.ny, (uint64_t)d.nz};
    const uint32_t box[4] = {8u, (uint32_t)G.P, (uint32_t)G.By, (uint32_t)G.Bz};
    if (!tma::make_map_bf16_4d(&map, in, dims, box)) return cudaErrorNotSupported;
    int Nb, nblocks;
    n_blocks(N, Nb, nblocks);
    const long long total = (long long)nblocks * Nb * 27 * Cin;
    tile_weights_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const __nv_bfloat16 *)W, rows, Kpad, Cin, Nb,
                                                                        nblocks, (__nv_bfloat16 *)Wt_scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = view_smem_bytes(G);
    const dim3 grid((unsigned)(G.tiles_y * ((d.nz + G.Tz - 1) / G.Tz)), (unsigned)nblocks);
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    auto run = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kern<<<grid, VIEW_THREADS, smem, s>>>(map, (const __nv_bfloat16 *)Wt_scratch, bias, out, G, err);
    };
    switch (epi) {
        case EPI_BIAS_LEAKY_BF16: run(conv_view_kernel<EPI_BIAS_LEAKY_BF16>); break;
        case EPI_PLAIN_BF16: run(conv_view_kernel<EPI_PLAIN_BF16>); break;
        default: run(conv_view_kernel<EPI_BIAS_F32_SOA>); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t conv_wgrad_view_bytes(const Dims &d, int Cin, int Cout) {
    WgGeom G;
    if (!choose_wg(d, Cin, Cout, G)) return 0;
    const int grid = (int)std::min<long long>(num_sms(), G.ntiles);
    return sizeof(float) * (size_t)grid * Cout * 27 * Cin;
}

cudaError_t launch_conv_wgrad_view(const void *in, int Cin, const void *dpre, int Cout, const Dims &d, float *part,
                                   float *dW, int Kpad, cudaStream_t s) {
    WgGeom G;
    if (!choose_wg(d, Cin, Cout, G)) return cudaErrorNotSupported;
    CUtensorMap xmap, dmap;
    const uint64_t xdims[4] = {(uint64_t)Cin, (uint64_t)d.nx, (uint64_t)d.ny, (uint64_t)d.nz};
    const uint32_t xbox[4] = {8u, (uint32_t)G.P, (uint32_t)G.By, 3u};
    const uint64_t ddims[4] = {(uint64_t)Cout, (uint64_t)d.nx, (uint64_t)d.ny, (uint64_t)d.nz};
    const uint32_t dbox[4] = {8u, (uint32_t)G.P, (uint32_t)G.Ty, 1u};
    if (!tma::make_map_bf16_4d(&xmap, in, xdims, xbox) || !tma::make_map_bf16_4d(&dmap, dpre, ddims, dbox))
        return cudaErrorNotSupported;
    const int grid = (int)std::min<long long>(num_sms(), G.ntiles);
    const size_t smem = wg_smem_bytes(G);
    cudaError_t e = cudaFuncSetAttribute(conv_wgrad_view_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    unsigned *err = error_word();
    if (!err) return cudaErrorInvalidDevice;
    conv_wgrad_view_kernel<<<grid, VIEW_THREADS, smem, s>>>(xmap, dmap, G, part, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int K = 27 * Cin, total = Cout * Kpad;
    wg_reduce_kernel<<<(total + 255) / 256, 256, 0, s>>>(part, grid, Cout, K, Kpad, dW);
    return cudaGetLastError();
}

}  // namespace regk
