// noalloc.cu -- the Parzen-MI similarity and gradient for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or let a library do it for them): a
// host application or framework that has reserved the whole GPU memory for
// its own pool and forbids any other allocation, or a latency-critical loop
// that must never hit the allocator (cudaMalloc / cudaFree can synchronise
// the device).  reg_loss / reg_loss_grad need a caller-allocated workspace;
// this entry point instead keeps its scratch (the joint histogram and the
// adjoint table) in a fixed-size array compiled into the library, so the
// caller passes only its inputs and outputs.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its 112 KiB until the process exits.  Its device address is
// looked up once per device (cudaGetSymbolAddress) on the first call made
// with that device current; host code never uses the symbol itself.
#include <mutex>

#include "checks.h"
#include "kernels.h"

using namespace regk;

namespace {

constexpr int kNoallocMaxBins = 64;
// the kernels index a histogram and tables of up to MAX_BINS x MAX_BINS entries
static_assert(kNoallocMaxBins <= MAX_BINS, "the scratch must hold the largest histogram the kernels write");
constexpr size_t kHistBytes = sizeof(unsigned long long) * kNoallocMaxBins * kNoallocMaxBins;  // 32 KiB
constexpr size_t kGtabBytes = MI_TABLE_BYTES;  // 80 KiB: G' and its 4-wide rows
constexpr size_t kScratchBytes = kHistBytes + kGtabBytes;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

static __device__ __align__(256) unsigned char g_mi_scratch[kScratchBytes];

namespace {

// Device address of g_mi_scratch on the current device (set-up on first use).
reg_status scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return REG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        unsigned char *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_mi_scratch);
        if (e != cudaSuccess || ptr == nullptr) return REG_ERR_CUDA;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return REG_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" reg_status reg_mi_loss_grad_noalloc(const reg_loss_desc *loss, const void *F, const void *M, int img_dt,
                                               const float *u, reg_dims d, int pad, double *sim_out,
                                               float *grad_u, void *stream) {
    if (!loss || loss->kind != REG_LOSS_MI) return loss ? REG_ERR_UNSUPPORTED : REG_ERR_INVALID_ARG;
    // the same descriptor and dims checks as the workspace entry points; the
    // scratch holds a bins x bins histogram and table, so no count beyond the
    // array's fits
    reg_status st = check_loss(loss);
    if (st != REG_OK) return st;
    if (loss->bins > kNoallocMaxBins) return REG_ERR_SHAPE;
    st = check_dims(d);
    if (st != REG_OK) return st;
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (pad != REG_PAD_BORDER && pad != REG_PAD_ZEROS) return REG_ERR_INVALID_ARG;
    if (!F || !M || !u || !sim_out) return REG_ERR_INVALID_ARG;
    if (!aligned16(F) || !aligned16(M) || !aligned16(u) || !aligned16(sim_out) || (grad_u && !aligned16(grad_u)))
        return REG_ERR_ALIGN;

    unsigned char *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != REG_OK) return st;
    unsigned long long *hist = (unsigned long long *)scratch;
    float *gtab = (float *)(scratch + kHistBytes);

    MiParams P;
    P.f_lo = loss->f_lo;
    P.f_scale = (float)(1.0 / ((double)loss->f_hi - (double)loss->f_lo));
    P.m_lo = loss->m_lo;
    P.m_scale = (float)(1.0 / ((double)loss->m_hi - (double)loss->m_lo));
    P.bins = loss->bins;
    P.hard = loss->mi_estimator == REG_MI_HARD;
    const Dims g = make_dims(d);
    const cudaStream_t s = (cudaStream_t)stream;
    // the histogram is accumulated with atomics and must start at zero on
    // every call (the array keeps whatever the previous call left in it)
    if (cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * loss->bins * loss->bins, s) != cudaSuccess)
        return REG_ERR_CUDA;
    if (launch_mi_hist(F, M, img_dt, u, g, pad, P, hist, s) != cudaSuccess) return REG_ERR_CUDA;
    if (launch_mi_finalize(hist, P, g.n, gtab, sim_out, s) != cudaSuccess) return REG_ERR_CUDA;
    if (grad_u) {
        StepParams S{};
        if (launch_mi_sweep2(F, M, img_dt, u, g, pad, P, gtab, grad_u, false, nullptr, nullptr, nullptr, REG_F32, S,
                             nullptr, nullptr, nullptr, s) != cudaSuccess)
            return REG_ERR_CUDA;
    }
    return REG_OK;
}
