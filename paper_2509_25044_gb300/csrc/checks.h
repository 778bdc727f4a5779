// checks.h -- host-side argument checks shared by the C ABI's entry points
// (capi.cu) and the entry point without a workspace (noalloc.cu), so that the
// limits they enforce (volume dims, window, bin count) are stated once.
#pragma once

#include <math.h>

#include "kernels.h"

namespace regk {

inline reg_status check_dims(reg_dims d) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return REG_ERR_SHAPE;
    if (d.nx > (1 << 20) || d.ny > (1 << 19) || d.nz > (1 << 16)) return REG_ERR_SHAPE;
    const long long n = (long long)d.nx * d.ny * d.nz;
    if (n > (1LL << 36)) return REG_ERR_SHAPE;
    return REG_OK;
}

inline reg_status check_loss(const reg_loss_desc *L) {
    if (!L) return REG_ERR_INVALID_ARG;
    if (L->kind == REG_LOSS_LNCC) {
        if (L->window < 3 || L->window > 2 * MAX_RADIUS + 1 || (L->window & 1) == 0) return REG_ERR_SHAPE;
        if (!(L->eps >= 0.0f) || !isfinite(L->eps)) return REG_ERR_INVALID_ARG;
        if (L->lncc_grad != REG_LNCC_GRAD_EXACT && L->lncc_grad != REG_LNCC_GRAD_ANTS) return REG_ERR_INVALID_ARG;
        return REG_OK;
    }
    if (L->kind == REG_LOSS_MI) {
        if (L->bins < 8 || L->bins > MAX_BINS) return REG_ERR_SHAPE;
        if (!isfinite(L->f_lo) || !isfinite(L->f_hi) || !isfinite(L->m_lo) || !isfinite(L->m_hi))
            return REG_ERR_INVALID_ARG;
        if (!(L->f_hi > L->f_lo) || !(L->m_hi > L->m_lo)) return REG_ERR_INVALID_ARG;
        if (L->mi_estimator != REG_MI_PARZEN && L->mi_estimator != REG_MI_HARD) return REG_ERR_INVALID_ARG;
        return REG_OK;
    }
    return REG_ERR_INVALID_ARG;
}

}  // namespace regk
