"""How strong the oracle's pins are: each entry of MUTANTS plants one plausible
mistake in a copy of the oracle (a flipped sign, a dropped factor or term, a
wrong index, a transposed operand, a wrong normalisation or border rule), and
the pin tests (tests/test_oracle_*.py, run against that copy) must fail on
every one.  The unmodified copy must pass them, so a failure means the pin
caught the mistake and not that the harness is broken.  The oracle itself is
never modified: the copies live in a temporary directory, each built with the
oracle's own build script before its pins run."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C = "oracle.c"
PY = "__init__.py"

# (name, file, text, replacement, occurrence of the text to replace, 1-based)
MUTANTS = [
    # trilinear warp and its slope (Eq. interp; Algorithm gridsampler)
    ("warp: corner weights swapped", C,
     "w[k] = bb[k] ? a[k] : 1.0 - a[k];", "w[k] = bb[k] ? 1.0 - a[k] : a[k];", 1),
    ("warp: slope sign flipped", C,
     "dw[k] = bb[k] ? 1.0 : -1.0;", "dw[k] = bb[k] ? -1.0 : 1.0;", 1),
    ("warp: x and y of the voxel swapped", C,
     "const int pc[3] = {x, y, z};", "const int pc[3] = {y, x, z};", 1),
    ("warp: corner offset taken from another axis's bit", C,
     "c[k] = i[k] + bb[k];", "c[k] = i[k] + bb[(k + 1) % 3];", 1),
    ("warp: border slope not flattened outside the volume", C,
     "slope_ok[k] = (phi >= 0.0 && phi <= (double)(n[k] - 1)) ? 1.0 : 0.0;", "slope_ok[k] = 1.0;", 1),
    ("warp: border cell not clamped below the last voxel", C,
     "long f = (long)floor(q);\n                            if (f > n[k] - 2) f = n[k] - 2;",
     "long f = (long)floor(q);", 1),
    ("warp: border point clamped one voxel short of the top", C,
     "if (q > (double)(n[k] - 1)) q = (double)(n[k] - 1);", "if (q > (double)(n[k] - 2)) q = (double)(n[k] - 2);", 1),
    ("warp zeros: slope flattened outside the volume", C,
     "slope_ok[k] = 1.0;\n                        long f = (long)floor(phi);",
     "slope_ok[k] = (phi >= 0.0 && phi <= (double)(n[k] - 1)) ? 1.0 : 0.0;\n"
     "                        long f = (long)floor(phi);", 1),
    ("warp adjoint: corner weights swapped", C,
     "w *= bb[k] ? a[k] : 1.0 - a[k];", "w *= bb[k] ? 1.0 - a[k] : a[k];", 1),
    ("warp adjoint: scatter to the sampling voxel", C,
     "gM[lin((int)c[0], (int)c[1], (int)c[2], nx, ny)] += w * g[p];", "gM[p] += w * g[p];", 1),
    # LNCC (App. fused LNCC, Eqs. lncc-loss, lncc-a..c)
    ("lncc: window one voxel short on the high side", C,
     "*hi = c + r > n - 1 ? n - 1 : c + r;", "*hi = c + r > n - 1 ? n - 1 : c + r - 1;", 1),
    ("lncc: border window not truncated (divides by the full size)", C,
     "const double muF = sF / cnt, muJ = sJ / cnt;",
     "cnt = (double)((2 * r + 1) * (2 * r + 1) * (2 * r + 1));\n"
     "                const double muF = sF / cnt, muJ = sJ / cnt;", 1),
    ("lncc: covariance not normalised", C, "                A /= cnt;\n", "", 1),
    ("lncc: F and J variances taken from the same image", C,
     "C += dj * dj;", "C += df * df;", 1),
    ("lncc: eps dropped", C,
     "const double D = B * C + eps;\n                const double ni", "const double D = B * C;\n                const double ni", 1),
    ("lncc: fixed-image window mean taken from the moving image", C,
     "                            sF += F[k];\n                            sJ += J[k];\n                            cnt += 1.0;",
     "                            sF += J[k];\n                            sJ += J[k];\n                            cnt += 1.0;", 1),
    ("lncc grad: dL/dn sign flipped", C,
     "const double dLdn = -1.0 / (double)N;\n#pragma omp parallel for schedule(static)\n    for (long i = 0;",
     "const double dLdn = 1.0 / (double)N;\n#pragma omp parallel for schedule(static)\n    for (long i = 0;", 1),
    ("lncc grad: dn/dC sign flipped", C,
     "const double dndC = -A[i] * A[i] * B[i] / (D * D);", "const double dndC = A[i] * A[i] * B[i] / (D * D);", 1),
    ("lncc grad: factor 2 of dC/dJ dropped", C,
     "beta[i] = dLdn * dndC * 2.0 / cnt[i];", "beta[i] = dLdn * dndC / cnt[i];", 1),
    ("lncc grad: own window's mean used for every window", C,
     "g += alpha[i] * (F[k] - muF[i]) + beta[i] * (J[k] - muJ[i]);",
     "g += alpha[i] * (F[k] - muF[k]) + beta[i] * (J[k] - muJ[i]);", 1),
    ("lncc grad: dn/dA uses B instead of A", C,
     "const double dndA = 2.0 * A[i] / D;", "const double dndA = 2.0 * B[i] / D;", 1),
    ("lncc ANTs: window size factor dropped", C,
     "g = cnt[k] * (alpha * (F[k] - muF[k]) + beta * (J[k] - muJ[k]));",
     "g = alpha * (F[k] - muF[k]) + beta * (J[k] - muJ[k]);", 1),
    ("lncc ANTs: factor 2 of dC/dJ dropped", C,
     "const double beta = dLdn * (-A[k] * A[k] * B[k] / (D * D)) * 2.0 / cnt[k];",
     "const double beta = dLdn * (-A[k] * A[k] * B[k] / (D * D)) / cnt[k];", 1),
    ("lncc points: factor 2 of dC/dJ dropped", C,
     "dndC * 2.0 * (J[k] - mJ) / c", "dndC * (J[k] - mJ) / c", 1),
    ("lncc points: per-voxel NCC not squared", C,
     "n_out[s] = D > 0.0 ? A * A / D : 0.0;", "n_out[s] = D > 0.0 ? A / D : 0.0;", 1),
    ("lncc points: window statistics at the listed voxel for every window", C,
     "window_stats(F, J, nx, ny, nz, r, xx, yy, zz, eps, &mF, &mJ, &A, &B, &C, &c);",
     "window_stats(F, J, nx, ny, nz, r, x, y, z, eps, &mF, &mJ, &A, &B, &C, &c);", 1),
    ("hard mi: PMF not divided by N", C,
     "p[m * B + n] = acc / (double)N;", "p[m * B + n] = acc;", 1),
    ("gaussian: weights not normalised", C,
     "for (int k = 0; k <= 2 * r; ++k) w[k] /= sum;", ";", 1),
    # Parzen MI (Sec. 2.2, Eq. mi; Eq. gradientmi-threadn)
    ("mi: B-spline cubic term sign flipped", C,
     "return 2.0 / 3.0 - a * a + 0.5 * a * a * a;", "return 2.0 / 3.0 - a * a - 0.5 * a * a * a;", 1),
    ("mi: B-spline derivative sign convention flipped", C,
     "const double s = t < 0.0 ? -1.0 : 1.0;", "const double s = t < 0.0 ? 1.0 : -1.0;", 1),
    ("mi: bin map stretched over all bins", C,
     "return v * (double)(B - 3) + 1.0;", "return v * (double)(B - 1);", 1),
    ("mi: moving bin coordinate from the fixed image", C,
     "const double sF = bin_coord(Fh[k], B), sJ = bin_coord(Jh[k], B);\n            for (int m = 0; m < B; ++m) {\n                wF[m]",
     "const double sF = bin_coord(Fh[k], B), sJ = bin_coord(Fh[k], B);\n            for (int m = 0; m < B; ++m) {\n                wF[m]", 1),
    ("mi: joint histogram not divided by N", C,
     "for (int e = 0; e < BB; ++e) p[e] /= (double)N;", ";", 1),
    ("mi: moving marginal read transposed", C,
     "pJ[n] += p[m * B + n];", "pJ[n] += p[n * B + m];", 1),
    ("mi: log ratio with the wrong marginal bin", C,
     "if (v > 0.0) mi += v * log(v / (pI[m] * pJ[n]));", "if (v > 0.0) mi += v * log(v / (pI[m] * pJ[m]));", 1),
    ("mi adjoint: sign flipped", C,
     "const double scale = -(double)(B - 3) / (double)N;", "const double scale = (double)(B - 3) / (double)N;", 1),
    ("mi adjoint: bin-map slope dropped", C,
     "const double scale = -(double)(B - 3) / (double)N;", "const double scale = -1.0 / (double)N;", 1),
    ("mi adjoint: table read transposed", C,
     "g += G[m * B + n] * wF[m] * dJ[n];", "g += G[n * B + m] * wF[m] * dJ[n];", 1),
    ("mi adjoint: kernel derivative argument reversed", C,
     "dJ[m] = or_bspline3_deriv(sJ - (double)m);", "dJ[m] = or_bspline3_deriv((double)m - sJ);", 1),
    ("mi adjoint: marginal term kept (log ratio without pJ)", C,
     "G[m * B + n] = v > 0.0 ? log(v / (pI[m] * pJ[n])) : 0.0;",
     "G[m * B + n] = v > 0.0 ? log(v / pI[m]) : 0.0;", 1),
    ("mi of a pmf: moving marginal read transposed", C,
     "pJ[n] += p[m * B + n];", "pJ[n] += p[n * B + m];", 3),
    # hard-binned MI (App. fused MI, approximate histogram)
    ("hard mi: bin truncated instead of rounded", C,
     "int m = (int)floorf(sb + 0.5f);", "int m = (int)floorf(sb);", 1),
    ("hard mi: smoothing weights not the B-spline's", C,
     "const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};", "const double w[3] = {0.25, 0.5, 0.25};", 1),
    ("hard mi: fixed and moving bins swapped", C,
     "cnt[hard_bin(F[k], f_lo, f_scale, B) * B + hard_bin(J[k], m_lo, m_scale, B)]",
     "cnt[hard_bin(J[k], m_lo, m_scale, B) * B + hard_bin(F[k], f_lo, f_scale, B)]", 1),
    ("hard mi grad: paired with the Parzen PMF instead of the hard one", C,
     "const double mi = or_mi_hard(F, J, N, B, f_lo, f_scale, m_lo, m_scale, p);\n    mi_adjoint(",
     "const double mi = or_mi_hard(F, J, N, B, f_lo, f_scale, m_lo, m_scale, p);\n"
     "    or_mi(Fh, Jh, N, B, p);\n    mi_adjoint(", 1),
    # Gaussian smoothing, downsampling, regulariser, Adam, det J
    ("gaussian: variance doubled", C,
     "w[k + r] = exp(-0.5 * (double)k * (double)k / (sigma * sigma));",
     "w[k + r] = exp(-(double)k * (double)k / (sigma * sigma));", 1),
    ("gaussian: truncated at 3 sigma instead of 4", C,
     "const int r = (int)(4.0 * sigma + 0.5);", "const int r = (int)(3.0 * sigma + 0.5);", 1),
    ("gaussian: periodic instead of nearest border", C,
     "qq = qq < 0 ? 0 : (qq > n[axis] - 1 ? n[axis] - 1 : qq);",
     "qq = ((qq % n[axis]) + n[axis]) % n[axis];", 1),
    ("gaussian: one axis skipped", C,
     "for (int axis = 0; axis < 3; ++axis) {", "for (int axis = 0; axis < 2; ++axis) {", 1),
    ("downsample: block sum not divided by 8", C,
     "out[lin(x, y, z, mx, my)] = acc / 8.0;", "out[lin(x, y, z, mx, my)] = acc / 4.0;", 1),
    ("downsample: y offset taken from dx", C,
     "in[lin(2 * x + dx, 2 * y + dy, 2 * z + dz, nx, ny)]", "in[lin(2 * x + dx, 2 * y + dx, 2 * z + dz, nx, ny)]", 1),
    ("diffusion: gradient sign at the lower voxel flipped", C,
     "gc[p] -= 2.0 * diff / (double)N;", "gc[p] += 2.0 * diff / (double)N;", 1),
    ("diffusion: z differences dropped", C,
     "const int step_ok[3] = {nx > 1, ny > 1, nz > 1};", "const int step_ok[3] = {nx > 1, ny > 1, 0};", 1),
    ("bf16: ties rounded up instead of to even", C,
     "bits = bits + 0x7fffu + lsb;", "bits = bits + 0x8000u;", 1),
    ("adam: bias correction dropped", C,
     "u[i] -= lr * (mn / bc1) / (sqrt(vn / bc2) + eps);", "u[i] -= lr * mn / (sqrt(vn) + eps);", 1),
    ("adam: eps inside the square root", C,
     "u[i] -= lr * (mn / bc1) / (sqrt(vn / bc2) + eps);", "u[i] -= lr * (mn / bc1) / sqrt(vn / bc2 + eps);", 1),
    ("adam: update from the rounded moments", C,
     "u[i] -= lr * (mn / bc1) / (sqrt(vn / bc2) + eps);\n        m[i] = bf16_moments ? or_bf16_round(mn) : mn;\n"
     "        v[i] = bf16_moments ? or_bf16_round(vn) : vn;",
     "m[i] = bf16_moments ? or_bf16_round(mn) : mn;\n        v[i] = bf16_moments ? or_bf16_round(vn) : vn;\n"
     "        u[i] -= lr * (m[i] / bc1) / (sqrt(v[i] / bc2) + eps);", 1),
    ("adam: gradient scale ignored", C,
     "const double gs = grad_scale * g[i];", "const double gs = g[i];", 1),
    ("adam: second moment from the unscaled gradient", C,
     "(1.0 - b2) * gs * gs;", "(1.0 - b2) * g[i] * g[i];", 1),
    ("jacdet: difference taken backwards", C,
     "deriv = (uc[lin(hi[0], hi[1], hi[2], nx, ny)] -\n                                     uc[lin(lo[0], lo[1], lo[2], nx, ny)]) / h;",
     "deriv = (uc[lin(lo[0], lo[1], lo[2], nx, ny)] -\n                                     uc[lin(hi[0], hi[1], hi[2], nx, ny)]) / h;", 1),
    ("jacdet: cofactor sign flipped", C,
     "Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +",
     "Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) -", 1),
    ("jacdet: identity not added", C,
     "Jm[c][d] = (c == d ? 1.0 : 0.0) + deriv;", "Jm[c][d] = deriv;", 1),
    ("jacdet: border difference divided by 2", C,
     "h = (double)(hi[d] - lo[d]);", "h = 2.0;", 1),
    # the learned initialiser's other operators
    ("leaky: slope applied to the positive side", C,
     "y[i] = x[i] > 0.0 ? x[i] : slope * x[i];", "y[i] = x[i] > 0.0 ? slope * x[i] : x[i];", 1),
    ("leaky backward: derivative 1 on the negative side", C,
     "dx[i] = x[i] > 0.0 ? dy[i] : slope * dy[i];", "dx[i] = dy[i];", 1),
    ("avgpool: divided by 4", C,
     "out[lin(X, Y, Z, mx, my) * C + c] = s / 8.0;", "out[lin(X, Y, Z, mx, my) * C + c] = s / 4.0;", 1),
    ("avgpool: block not offset in z", C,
     "s += in[lin(2 * X + dx, 2 * Y + dy, 2 * Z + dz, nx, ny) * C + c];",
     "s += in[lin(2 * X + dx, 2 * Y + dy, 2 * Z, nx, ny) * C + c];", 1),
    ("avgpool adjoint: weight 1 instead of 1/8", C,
     "gout[lin(x / 2, y / 2, z / 2, mx, my) * C + c] / 8.0;", "gout[lin(x / 2, y / 2, z / 2, mx, my) * C + c];", 1),
    ("upsample: corner-aligned instead of voxel-centre coordinates", C,
     "const double c = ((double)f + 0.5) / (double)s - 0.5;", "const double c = (double)f / (double)s;", 1),
    ("upsample: the two corner weights swapped along x", C,
     "const double w = (bx ? ax : 1.0 - ax)", "const double w = (bx ? 1.0 - ax : ax)", 1),
    ("upsample adjoint: corner weights swapped along y", C,
     "(by ? ay : 1.0 - ay) * (bz ? az : 1.0 - az);\n                        gin",
     "(by ? 1.0 - ay : ay) * (bz ? az : 1.0 - az);\n                        gin", 1),
    ("concat: b written over a's channels", C,
     "out[v * (Ca + Cb) + Ca + c] = b[v * Cb + c];", "out[v * (Ca + Cb) + c] = b[v * Cb + c];", 1),
    ("field down2: displacement not halved", C, "out[ch * m + i] *= 0.5;", "out[ch * m + i] *= 1.0;", 1),
    ("field upsample: displacement not rescaled", C, "out[ch * n + i] *= (double)s;", "out[ch * n + i] *= 1.0;", 1),
    ("pack pair: F normalised by M's range", C,
     "out[2 * v] = (sf / cnt - f_lo) / (f_hi - f_lo);", "out[2 * v] = (sf / cnt - f_lo) / (m_hi - m_lo);", 1),
    ("mse: gradient without the factor 2", C,
     "if (grad) grad[i] = 2.0 * d / (3.0 * (double)V);", "if (grad) grad[i] = d / (3.0 * (double)V);", 1),
    ("mse: mean over V instead of 3V", C, "return s / (3.0 * (double)V);", "return s / (double)V;", 1),
    # convolutions of the learned initialiser
    ("conv: x and z taps swapped", C,
     "const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;",
     "const int xx = x + t / 9 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t % 3 - 1;", 1),
    ("conv: bias dropped", C,
     "double acc = bias ? bias[o] : 0.0;", "double acc = 0.0;", 1),
    ("conv dgrad: gathered instead of scattered", C,
     "din[q * Cin + c] += w[((long)o * 27 + t) * Cin + c] * dout[v * Cout + o];",
     "din[v * Cin + c] += w[((long)o * 27 + t) * Cin + c] * dout[q * Cout + o];", 1),
    ("conv wgrad: input not shifted by the tap", C,
     "acc += dout[lin(x, y, z, nx, ny) * Cout + o] * in[q * Cin + c];",
     "acc += dout[lin(x, y, z, nx, ny) * Cout + o] * in[lin(x, y, z, nx, ny) * Cin + c];", 1),
    # the chain rule and the composite transform, in the Python layer
    ("chain: warp slope dropped from the LNCC gradient", PY,
     "return S, gJ[None] * dJ", "return S, np.repeat(gJ[None], 3, axis=0)", 1),
    ("chain: normalisation slope dropped from the MI gradient", PY,
     "return v, (gJh * dJh)[None] * dJ", "return v, gJh[None] * dJ", 2),
    ("chain: intensity map slope not 1/(hi - lo)", PY,
     "d = np.where((t >= 0.0) & (t <= 1.0), 1.0 / (hi - lo), 0.0)",
     "d = np.where((t >= 0.0) & (t <= 1.0), 1.0, 0.0)", 1),
    ("binding: volume sizes passed to C in z, y, x order", PY,
     "    nz, ny, nx = vol.shape\n    return nx, ny, nz", "    nz, ny, nx = vol.shape\n    return nz, ny, nx", 1),
    ("chain: moving image normalised with the fixed image's range", PY,
     "Jh, dJh = normalize(J, *spec.m_range)", "Jh, dJh = normalize(J, *spec.f_range)", 1),
    ("chain: intensities not clamped to [0, 1]", PY,
     "return np.clip(t, 0.0, 1.0), d", "return t, d", 1),
    ("objective: LNCC loss taken as -S", PY,
     "loss = 1.0 - sim if spec.kind == LOSS_LNCC else -sim", "loss = -sim", 1),
    ("objective: MI loss taken as 1 - MI", PY,
     "loss = 1.0 - sim if spec.kind == LOSS_LNCC else -sim", "loss = 1.0 - sim", 1),
    ("iterate: Adam input not scaled by N", PY,
     "grad_scale = float(np.prod(np.shape(F)))", "grad_scale = 1.0", 1),
    ("chain: the exact and ANTs LNCC gradients dispatched the other way round", PY,
     "(lncc_grad_ants if spec.lncc_grad == 1 else lncc_grad)", "(lncc_grad if spec.lncc_grad == 1 else lncc_grad_ants)", 1),
    ("chain: the hard-binned estimator's gradient taken from the Parzen PMF", PY,
     "v, gJh = mi_hard_grad(F, J, spec.bins, spec.f_range, spec.m_range)",
     "v, gJh = mi_hard(F, J, spec.bins, spec.f_range, spec.m_range), mi_grad(Fh, Jh, spec.bins)[1]", 1),
    ("objective: lambda not applied to the regulariser gradient", PY,
     "grad=g + lam * gR", "grad=g + gR", 1),
    ("composite: A applied transposed", PY,
     'np.einsum("ij,jzyx->izyx", A, X)', 'np.einsum("ji,jzyx->izyx", A, X)', 1),
    ("composite: S not applied to u", PY,
     "phi = phi + s[:, None, None, None] * _f64(u)", "phi = phi + _f64(u)", 1),
    ("composite: translation subtracted", PY,
     "phi = np.einsum(\"ij,jzyx->izyx\", A, X) + t[:, None, None, None]",
     "phi = np.einsum(\"ij,jzyx->izyx\", A, X) - t[:, None, None, None]", 1),
    ("composite: dC/dt averaged instead of summed", PY,
     "g_t = gX.reshape(3, -1).sum(axis=1)", "g_t = gX.reshape(3, -1).mean(axis=1)", 1),
    ("composite: dC/dA transposed", PY,
     'g_A = np.einsum("izyx,jzyx->ij", gX, X)', 'g_A = np.einsum("izyx,jzyx->ji", gX, X)', 1),
    ("composite: S dropped from dC/du", PY,
     "return s[:, None, None, None] * gX, g_A, g_t", "return gX, g_A, g_t", 1),
    ("composite backward: upstream gradient dropped", PY,
     "return _affine_grads(dJ * _f64(g)[None], s)", "return _affine_grads(dJ, s)", 1),
    ("compose: padding mode ignored", PY,
     "return a + np.stack([warp(b[c], a, pad) for c in range(3)])",
     "return a + np.stack([warp(b[c], a) for c in range(3)])", 1),
    ("compose backward: padding mode ignored in the scatter", PY,
     "gb[d] = scale * warp_adjoint(gw[d], sa, pad)", "gb[d] = scale * warp_adjoint(gw[d], sa)", 1),
    ("exp: one squaring fewer", PY,
     "    for _ in range(steps):\n        u = compose_fields(u, u, pad)",
     "    for _ in range(steps - 1):\n        u = compose_fields(u, u, pad)", 1),
    ("warp: padding mode ignored for the composite sampler", PY,
     "return warp(M, composite_offset(M.shape, A, t, s, u), pad, with_grad)",
     "return warp(M, composite_offset(M.shape, A, t, s, u), PAD_BORDER, with_grad)", 1),
    ("compose: fields composed in the other order", PY,
     "return a + np.stack([warp(b[c], a, pad) for c in range(3)])",
     "return b + np.stack([warp(a[c], b, pad) for c in range(3)])", 1),
    ("compose backward: slope term dropped", PY,
     "ga += scale * scale * gw[d][None] * dJ", "pass", 1),
    ("compose backward: scatter replaced by a gather", PY,
     "gb[d] = scale * warp_adjoint(gw[d], sa, pad)", "gb[d] = scale * warp(gw[d], -sa, pad)", 1),
    ("compose backward: scale dropped from the direct term", PY,
     "ga = scale * gw.copy()", "ga = gw.copy()", 1),
    ("exp: velocity scaled by 2^-(steps-1)", PY,
     "u = _f64(v) / float(2 ** steps)\n    for _ in range(steps):",
     "u = _f64(v) / float(2 ** (steps - 1))\n    for _ in range(steps):", 1),
    ("exp backward: 2^-steps dropped", PY,
     "return g / float(2 ** steps)", "return g", 1),
    ("exp backward: scatter term dropped", PY,
     "g = ga + gb", "g = ga", 1),
    ("exp backward: one squaring too many replayed", PY,
     "for _ in range(steps - 1):\n        us.append", "for _ in range(steps):\n        us.append", 1),
]


def _mutate(src: str, text: str, new: str, nth: int) -> str:
    at = -1
    for _ in range(nth):
        at = src.find(text, at + 1)
        assert at >= 0, f"mutation site not found: {text!r} (occurrence {nth})"
    return src[:at] + new + src[at + len(text):]


def _copy_base(dst: str) -> None:
    """The pins and a copy of the oracle (its source and its built library)."""
    import glob
    from oracle import build as ob
    ob.build()
    os.makedirs(os.path.join(dst, "tests"))
    os.makedirs(os.path.join(dst, "oracle", "_build"))
    shutil.copy2(os.path.join(ROOT, "pytest.ini"), dst)
    shutil.copy2(os.path.join(ROOT, "tests", "conftest.py"), os.path.join(dst, "tests"))
    for f in glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py")):
        shutil.copy2(f, os.path.join(dst, "tests"))
    for f in ("oracle.c", "__init__.py", "build.py"):
        shutil.copy2(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle"))
    shutil.copy2(ob.lib_path(), os.path.join(dst, "oracle", "_build"))


def _env():
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTEST_ADDOPTS", None)
    return env


def _run_pins(d: str) -> subprocess.CompletedProcess:
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "tests"],
                          cwd=d, env=_env(), capture_output=True, text=True, timeout=600)


def _check(base: str, work: str, i: int):
    name, fname, text, new, nth = MUTANTS[i]
    d = os.path.join(work, f"m{i:02d}")
    shutil.copytree(base, d)
    path = os.path.join(d, "oracle", fname)
    with open(path) as f:
        src = f.read()
    with open(path, "w") as f:
        f.write(_mutate(src, text, new, nth))
    if fname == C:
        # the mutant must compile, so that a failing pin is the pin's doing
        b = subprocess.run([sys.executable, "-c", "from oracle import build; build.build(force=True)"],
                           cwd=d, env=_env(), capture_output=True, text=True, timeout=300)
        if b.returncode != 0:
            return name, "did not compile: " + b.stderr[-400:]
    r = _run_pins(d)
    if r.returncode == 1:
        return name, None
    return name, f"pins exited {r.returncode}: " + (r.stdout + r.stderr)[-400:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = str(tmp_path / "base")
    _copy_base(base)
    control = _run_pins(base)
    assert control.returncode == 0, "the unmodified copy fails its pins:\n" + control.stdout[-2000:]
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as pool:
        results = list(pool.map(lambda i: _check(base, str(tmp_path), i), range(len(MUTANTS))))
    survivors = [f"{name}: {why}" for name, why in results if why is not None]
    assert not survivors, "mistakes no pin caught:\n" + "\n".join(survivors)
