// capi_nn.cu -- C ABI of the learned initialiser's operators (see the
// reg_nn_* declarations in include/reg.h).  Validation on the host, then one
// or two kernel launches each; nothing is allocated.
#include <stdint.h>

#include "kernels.h"

using namespace regk;

namespace {

bool al16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }
reg_status st(cudaError_t e) { return e == cudaSuccess ? REG_OK : REG_ERR_CUDA; }
bool dims_ok(reg_dims d) { return d.nx >= 1 && d.ny >= 1 && d.nz >= 1 && (long long)d.nx * d.ny * d.nz < (1LL << 31); }
bool even(reg_dims d) { return d.nx % 2 == 0 && d.ny % 2 == 0 && d.nz % 2 == 0; }
int kpad_of(int K) { return (K + 63) / 64 * 64; }
// flipped / transposed data-gradient weights, rounded up to 256 bytes (the
// re-tiled copy for the TMA-fed kernel follows them in the scratch)
size_t dgrad_wd_bytes(int Cin, int Cout) {
    return (sizeof(uint16_t) * (size_t)((Cin + 15) / 16 * 16) * kpad_of(27 * Cout) + 255) / 256 * 256;
}

}  // namespace

extern "C" {

size_t reg_nn_conv_kpad(int Cin) { return (size_t)kpad_of(27 * Cin); }

size_t reg_nn_conv_scratch_bytes(int Cin, int Cout) {
    if (Cin < 8 || Cout < 1) return 0;
    return conv_view_weight_bytes(Cin, (Cout + 15) / 16 * 16);
}

reg_status reg_nn_conv3d_fwd(const void *in, int Cin, const void *W, const float *bias, int Cout, reg_dims d,
                             int epilogue, float slope, void *scratch, size_t scratch_bytes, void *out, void *stream) {
    if (!dims_ok(d)) return REG_ERR_SHAPE;
    if (Cin < 8 || Cin % 8 || Cin > 128 || Cout < 1 || Cout > 64) return REG_ERR_SHAPE;
    if (epilogue < 0 || epilogue > 2) return REG_ERR_INVALID_ARG;
    if (epilogue != 2 && Cout % 8) return REG_ERR_SHAPE;
    if (!al16(in) || !al16(W) || !al16(out)) return in && W && out ? REG_ERR_ALIGN : REG_ERR_INVALID_ARG;
    if (epilogue != 1 && !bias) return REG_ERR_INVALID_ARG;
    if (scratch && !al16(scratch)) return REG_ERR_ALIGN;
    const int N = (Cout + 15) / 16 * 16, Kpad = kpad_of(27 * Cin);
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t need = conv_view_weight_bytes(Cin, N);
    if (scratch && need) {
        if (scratch_bytes < need) return REG_ERR_WORKSPACE;
        const cudaError_t e = launch_conv_view(in, Cin, W, N, Kpad, bias, Cout, N, make_dims(d), epilogue, slope,
                                               scratch, out, s);
        if (e != cudaErrorNotSupported) return st(e);
    }
    return st(launch_conv_fwd(in, Cin, W, Kpad, bias, Cout, N, make_dims(d), epilogue, slope, out, s));
}

reg_status reg_nn_conv3d_dgrad(const void *dpre, int Cout, const void *W, int Cin, reg_dims d, void *Wd_scratch,
                               void *din, void *stream) {
    if (!dims_ok(d)) return REG_ERR_SHAPE;
    if (Cin < 8 || Cin % 8 || Cin > 128 || Cout < 8 || Cout % 8 || Cout > 128) return REG_ERR_SHAPE;
    if (!al16(dpre) || !al16(W) || !al16(Wd_scratch) || !al16(din)) return REG_ERR_ALIGN;
    const int Kpad = kpad_of(27 * Cin), Kpad_d = kpad_of(27 * Cout), Nd = (Cin + 15) / 16 * 16;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_repack_dgrad(W, Cout, Cin, Kpad, Wd_scratch, Nd, Kpad_d, s);
    if (e != cudaSuccess) return REG_ERR_CUDA;
    if (conv_view_weight_bytes(Cout, Nd)) {
        void *tiles = (unsigned char *)Wd_scratch + dgrad_wd_bytes(Cin, Cout);
        e = launch_conv_view(dpre, Cout, Wd_scratch, Nd, Kpad_d, nullptr, Cin, Nd, make_dims(d), 1, 0.0f, tiles,
                             din, s);
        if (e != cudaErrorNotSupported) return st(e);
    }
    return st(launch_conv_fwd(dpre, Cout, Wd_scratch, Kpad_d, nullptr, Cin, Nd, make_dims(d), 1, 0.0f, din, s));
}

size_t reg_nn_dgrad_scratch_bytes(int Cin, int Cout) {
    if (Cin < 8 || Cout < 8) return 0;
    return dgrad_wd_bytes(Cin, Cout) + conv_view_weight_bytes(Cout, (Cin + 15) / 16 * 16);
}

size_t reg_nn_wgrad_scratch_bytes(reg_dims d, int Cin, int Cout) {
    if (!dims_ok(d)) return 0;
    const Dims g = make_dims(d);
    const size_t a = wgrad_part_bytes(g, Cin, Cout), b = conv_wgrad_view_bytes(g, Cin, Cout);
    return a > b ? a : b;
}

reg_status reg_nn_conv3d_wgrad(const void *in, int Cin, const void *dpre, int Cout, reg_dims d, void *scratch,
                               size_t scratch_bytes, float *dW, void *stream) {
    if (!dims_ok(d)) return REG_ERR_SHAPE;
    if (Cin < 8 || Cin % 8 || Cin > 128 || Cout < 16 || Cout % 16 || Cout > 64) return REG_ERR_SHAPE;
    if (!al16(in) || !al16(dpre) || !al16(scratch) || !al16(dW)) return REG_ERR_ALIGN;
    const Dims g = make_dims(d);
    const size_t need_view = conv_wgrad_view_bytes(g, Cin, Cout);
    if (need_view && scratch_bytes >= need_view) {
        const cudaError_t e = launch_conv_wgrad_view(in, Cin, dpre, Cout, g, (float *)scratch, dW, kpad_of(27 * Cin),
                                                     (cudaStream_t)stream);
        if (e != cudaErrorNotSupported) return st(e);
    }
    if (scratch_bytes < wgrad_part_bytes(g, Cin, Cout)) return REG_ERR_WORKSPACE;
    return st(launch_conv_wgrad(in, Cin, dpre, Cout, g, (float *)scratch, dW, kpad_of(27 * Cin),
                                (cudaStream_t)stream));
}

reg_status reg_nn_pack_pair(const void *F, const void *M, int img_dt, reg_dims d, int factor, float f_lo,
                            float f_hi, float m_lo, float m_hi, void *out, void *stream) {
    if (!dims_ok(d) || factor < 1 || d.nx % factor || d.ny % factor || d.nz % factor) return REG_ERR_SHAPE;
    if (img_dt != REG_F32 && img_dt != REG_BF16) return REG_ERR_DTYPE;
    if (!(f_hi > f_lo) || !(m_hi > m_lo)) return REG_ERR_INVALID_ARG;
    if (!al16(F) || !al16(M) || !al16(out)) return REG_ERR_ALIGN;
    return st(launch_pack_pair(F, M, img_dt, make_dims(d), factor, f_lo, 1.0f / (f_hi - f_lo), m_lo,
                               1.0f / (m_hi - m_lo), out, (cudaStream_t)stream));
}

reg_status reg_nn_leaky_bwd(const void *out, const void *dout, long long n, float slope, void *dpre, void *stream) {
    if (n < 0 || !out || !dout || !dpre) return REG_ERR_INVALID_ARG;
    return st(launch_leaky_bwd(out, dout, n, slope, dpre, (cudaStream_t)stream));
}

size_t reg_nn_bias_grad_scratch_bytes(int C) { return sizeof(double) * (size_t)bias_grad_blocks() * C; }

reg_status reg_nn_bias_grad(const void *dpre, long long V, int C, void *scratch, float *dbias, void *stream) {
    if (V < 1 || C < 1 || C > 64 || !dpre || !scratch || !dbias) return REG_ERR_INVALID_ARG;
    return st(launch_bias_grad(dpre, V, C, (double *)scratch, dbias, (cudaStream_t)stream));
}

reg_status reg_nn_avgpool2(const void *in, int C, reg_dims d_in, void *out, int backward, void *stream) {
    if (!dims_ok(d_in) || !even(d_in) || C < 1) return REG_ERR_SHAPE;
    if (!in || !out) return REG_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    return st(backward ? launch_avgpool2_bwd(in, C, make_dims(d_in), out, s)
                       : launch_avgpool2(in, C, make_dims(d_in), out, s));
}

reg_status reg_nn_upsample2(const void *in, int C, reg_dims d_coarse, void *out, int backward, void *stream) {
    if (!dims_ok(d_coarse) || C < 1) return REG_ERR_SHAPE;
    if (!in || !out) return REG_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    return st(backward ? launch_upsample2_bwd(in, C, make_dims(d_coarse), out, s)
                       : launch_upsample2(in, C, make_dims(d_coarse), out, s));
}

reg_status reg_nn_put_channels(const void *src, int Csrc, long long V, void *dst, int Cdst, int c0, int accumulate,
                               void *stream) {
    if (!src || !dst || V < 0 || c0 < 0 || c0 + Csrc > Cdst) return REG_ERR_INVALID_ARG;
    return st(launch_put_channels(src, Csrc, V, dst, Cdst, c0, accumulate, (cudaStream_t)stream));
}

reg_status reg_nn_take_channels(const void *src, int Csrc, int c0, long long V, void *dst, int Cdst, int accumulate,
                                void *stream) {
    if (!src || !dst || V < 0 || c0 < 0 || c0 + Cdst > Csrc) return REG_ERR_INVALID_ARG;
    return st(launch_take_channels(src, Csrc, c0, V, dst, Cdst, accumulate, (cudaStream_t)stream));
}

size_t reg_nn_mse_scratch_bytes(void) { return sizeof(double) * (size_t)mse_blocks(); }

reg_status reg_nn_mse(const float *pred, const float *target, long long V, int Cpad, void *dpred, void *scratch,
                      double *loss, void *stream) {
    if (!pred || !target || !dpred || !scratch || !loss || V < 1 || Cpad < 3) return REG_ERR_INVALID_ARG;
    return st(launch_mse(pred, target, V, Cpad, dpred, (double *)scratch, loss, (cudaStream_t)stream));
}

reg_status reg_nn_field_down2(const float *u, reg_dims d_fine, float *out, void *stream) {
    if (!dims_ok(d_fine) || !even(d_fine)) return REG_ERR_SHAPE;
    if (!u || !out) return REG_ERR_INVALID_ARG;
    return st(launch_field_down2(u, make_dims(d_fine), out, (cudaStream_t)stream));
}

reg_status reg_nn_field_upsample(const float *u, reg_dims d_coarse, int factor, float *out, void *stream) {
    if (!dims_ok(d_coarse) || factor < 1) return REG_ERR_SHAPE;
    if (!u || !out) return REG_ERR_INVALID_ARG;
    return st(launch_field_up(u, make_dims(d_coarse), factor, out, (cudaStream_t)stream));
}

reg_status reg_nn_adam(float *w, float *m, float *v, const float *g, long long n, const reg_adam_desc *adam, int t,
                       void *w_bf16, void *stream) {
    if (!w || !m || !v || !g || !adam || t < 1 || n < 1) return REG_ERR_INVALID_ARG;
    StepParams S{};
    const double bc1 = 1.0 - pow((double)adam->beta1, (double)t), bc2 = 1.0 - pow((double)adam->beta2, (double)t);
    S.lr_bc1 = (float)((double)adam->lr / bc1);
    S.rsqrt_bc2 = (float)(1.0 / sqrt(bc2));
    S.b1 = adam->beta1;
    S.b2 = adam->beta2;
    S.eps = adam->eps;
    S.gscale = adam->grad_scale;
    return st(launch_adam_weights(w, m, v, g, n, S, w_bf16, (cudaStream_t)stream));
}

}  // extern "C"
