/*
 * oracle.c -- plain FP64 CPU oracle for one iteration of dense 3-D deformable
 * registration, argmin_u C(F, M o (id+u)) + lambda R(u)  (Sec. 1, Eq. image-reg).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no source, header, table or helper with the
 * CUDA library in paper_2509_25044_gb300/csrc.
 *
 * Every function follows the paper's definition as written, in the obvious
 * order, in double precision.  Global sums are taken per z-plane (serially in
 * x-fastest order) and then over planes in increasing z, so results do not
 * depend on the number of OpenMP threads.
 *
 * Layout conventions (the paper is silent on them):
 *   volumes   [nz][ny][nx], x fastest, voxel spacing 1;
 *   u         structure of arrays [3][nz][ny][nx]; channel 0,1,2 = x,y,z
 *             displacement in voxel units; phi(p) = p + u(p).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PAD_BORDER 0
#define OR_PAD_ZEROS 1

static long lin(int x, int y, int z, int nx, int ny) { return ((long)z * ny + y) * nx + x; }

/* ------------------------------------------------------------------------ */
/* Trilinear warp J = M o (id + u).                                          */
/* Follows the d-linear interpolation formula of the ring-sampler appendix   */
/* (Eq. interp): J = sum_{b in {0,1}^3} prod_k (1-a_k)^(1-b_k) a_k^b_k       */
/* M[i+b], i_k = floor(phi_k), a_k = phi_k - i_k; and Algorithm gridsampler  */
/* (one sample per target voxel, identity grid implicit).                    */
/* Padding: ZEROS = corners outside the volume contribute 0 (Algorithm       */
/* gridsampler).  BORDER = the sample point is first clamped into            */
/* [0, n_k - 1] per axis; the cell index is then min(floor(q), n_k - 2).     */
/* dJ (optional, 3N) receives dJ/dphi_k.  In BORDER mode the derivative      */
/* along k is 0 where phi_k lies outside [0, n_k - 1] (the clamp is flat).   */
/* ------------------------------------------------------------------------ */
void or_warp(const double *M, const double *u, int nx, int ny, int nz, int pad,
             double *J, double *dJ)
{
    const long N = (long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const long p = lin(x, y, z, nx, ny);
                const int pc[3] = {x, y, z};
                long i[3];
                double a[3];
                double slope_ok[3];
                for (int k = 0; k < 3; ++k) {
                    double phi = (double)pc[k] + u[(long)k * N + p];
                    if (pad == OR_PAD_BORDER) {
                        double q = phi;
                        slope_ok[k] = (phi >= 0.0 && phi <= (double)(n[k] - 1)) ? 1.0 : 0.0;
                        if (q < 0.0) q = 0.0;
                        if (q > (double)(n[k] - 1)) q = (double)(n[k] - 1);
                        if (n[k] == 1) {
                            i[k] = 0;
                            a[k] = 0.0;
                        } else {
                            long f = (long)floor(q);
                            if (f > n[k] - 2) f = n[k] - 2;
                            i[k] = f;
                            a[k] = q - (double)f;
                        }
                    } else {
                        slope_ok[k] = 1.0;
                        long f = (long)floor(phi);
                        i[k] = f;
                        a[k] = phi - (double)f;
                    }
                }
                double val = 0.0;
                double der[3] = {0.0, 0.0, 0.0};
                for (int b = 0; b < 8; ++b) {
                    const int bb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
                    long c[3];
                    int inside = 1;
                    for (int k = 0; k < 3; ++k) {
                        c[k] = i[k] + bb[k];
                        if (c[k] < 0 || c[k] > n[k] - 1) inside = 0;
                    }
                    double mv = 0.0;
                    if (inside) {
                        mv = M[lin((int)c[0], (int)c[1], (int)c[2], nx, ny)];
                    } else if (pad == OR_PAD_BORDER) {
                        /* only reachable with zero weight (n_k == 1) */
                        long cc[3];
                        for (int k = 0; k < 3; ++k) cc[k] = c[k] > n[k] - 1 ? n[k] - 1 : c[k];
                        mv = M[lin((int)cc[0], (int)cc[1], (int)cc[2], nx, ny)];
                    }
                    double w[3], dw[3];
                    for (int k = 0; k < 3; ++k) {
                        w[k] = bb[k] ? a[k] : 1.0 - a[k];
                        dw[k] = bb[k] ? 1.0 : -1.0;
                    }
                    val += w[0] * w[1] * w[2] * mv;
                    der[0] += dw[0] * w[1] * w[2] * mv;
                    der[1] += w[0] * dw[1] * w[2] * mv;
                    der[2] += w[0] * w[1] * dw[2] * mv;
                }
                J[p] = val;
                if (dJ) {
                    for (int k = 0; k < 3; ++k) dJ[(long)k * N + p] = der[k] * slope_ok[k];
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the warp with respect to the moving volume (the scatter of     */
/* Algorithm gridsampler, backward, "accumulate g_J into 8 neighbours"):      */
/*   gM[q] = sum_p g[p] w_q(p),                                              */
/* w_q(p) the trilinear weight of voxel q in the sample of M at p + u(p),    */
/* with the padding of or_warp (BORDER: the point clamped first; ZEROS:      */
/* corners outside take no weight).  Serial, so the sums have a fixed order. */
/* ------------------------------------------------------------------------ */
void or_warp_adjoint(const double *g, const double *u, int nx, int ny, int nz, int pad, double *gM)
{
    const long N = (long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
    for (long q = 0; q < N; ++q) gM[q] = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long p = lin(x, y, z, nx, ny);
                const int pc[3] = {x, y, z};
                long i[3];
                double a[3];
                for (int k = 0; k < 3; ++k) {
                    double phi = (double)pc[k] + u[(long)k * N + p];
                    if (pad == OR_PAD_BORDER) {
                        if (phi < 0.0) phi = 0.0;
                        if (phi > (double)(n[k] - 1)) phi = (double)(n[k] - 1);
                        if (n[k] == 1) {
                            i[k] = 0;
                            a[k] = 0.0;
                            continue;
                        }
                        long f = (long)floor(phi);
                        if (f > n[k] - 2) f = n[k] - 2;
                        i[k] = f;
                        a[k] = phi - (double)f;
                    } else {
                        long f = (long)floor(phi);
                        i[k] = f;
                        a[k] = phi - (double)f;
                    }
                }
                for (int b = 0; b < 8; ++b) {
                    const int bb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
                    long c[3];
                    double w = 1.0;
                    int inside = 1;
                    for (int k = 0; k < 3; ++k) {
                        c[k] = i[k] + bb[k];
                        w *= bb[k] ? a[k] : 1.0 - a[k];
                        if (c[k] < 0 || c[k] > n[k] - 1) inside = 0;
                    }
                    if (inside && w != 0.0) gM[lin((int)c[0], (int)c[1], (int)c[2], nx, ny)] += w * g[p];
                }
            }
}

/* ------------------------------------------------------------------------ */
/* LNCC value (App. fused LNCC, Eq. lncc-loss and Eqs. lncc-a .. lncc-c).    */
/* The averaging filter w is a uniform box of side `win` (odd) centred at i; */
/* at the volume border the box is truncated to the voxels inside the volume */
/* and normalised by their count c_i (the paper does not say how borders are */
/* handled).  Two-pass form: means first, then centred sums.                 */
/*   A_i = sum_k w_ik (F_k - muF_i)(J_k - muJ_i), B_i, C_i likewise,          */
/*   n_i = A_i^2 / (B_i C_i + eps), and n_i = 0 where B_i C_i + eps == 0.     */
/* Returns S = (1/N) sum_i n_i; the loss is 1 - S.  n_out (optional, N).     */
/* The per-window quantities (muF, muJ, A, B, C, c) go to win_out (optional, */
/* 6N, [6][N]) for the gradient.                                             */
/* ------------------------------------------------------------------------ */
static void window_bounds(int c, int r, int n, int *lo, int *hi)
{
    *lo = c - r < 0 ? 0 : c - r;
    *hi = c + r > n - 1 ? n - 1 : c + r;
}

double or_lncc(const double *F, const double *J, int nx, int ny, int nz, int win, double eps,
               double *n_out, double *win_out)
{
    const long N = (long)nx * ny * nz;
    const int r = win / 2;
    double *plane_sum = (double *)calloc((size_t)nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        double acc = 0.0;
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int x0, x1, y0, y1, z0, z1;
                window_bounds(x, r, nx, &x0, &x1);
                window_bounds(y, r, ny, &y0, &y1);
                window_bounds(z, r, nz, &z0, &z1);
                double cnt = 0.0, sF = 0.0, sJ = 0.0;
                for (int zz = z0; zz <= z1; ++zz)
                    for (int yy = y0; yy <= y1; ++yy)
                        for (int xx = x0; xx <= x1; ++xx) {
                            long k = lin(xx, yy, zz, nx, ny);
                            sF += F[k];
                            sJ += J[k];
                            cnt += 1.0;
                        }
                const double muF = sF / cnt, muJ = sJ / cnt;
                double A = 0.0, B = 0.0, C = 0.0;
                for (int zz = z0; zz <= z1; ++zz)
                    for (int yy = y0; yy <= y1; ++yy)
                        for (int xx = x0; xx <= x1; ++xx) {
                            long k = lin(xx, yy, zz, nx, ny);
                            const double df = F[k] - muF, dj = J[k] - muJ;
                            A += df * dj;
                            B += df * df;
                            C += dj * dj;
                        }
                A /= cnt;
                B /= cnt;
                C /= cnt;
                const double D = B * C + eps;
                const double ni = D > 0.0 ? A * A / D : 0.0;
                const long p = lin(x, y, z, nx, ny);
                if (n_out) n_out[p] = ni;
                if (win_out) {
                    win_out[0 * N + p] = muF;
                    win_out[1 * N + p] = muJ;
                    win_out[2 * N + p] = A;
                    win_out[3 * N + p] = B;
                    win_out[4 * N + p] = C;
                    win_out[5 * N + p] = cnt;
                }
                acc += ni;
            }
        }
        plane_sum[z] = acc;
    }
    double S = 0.0;
    for (int z = 0; z < nz; ++z) S += plane_sum[z];
    free(plane_sum);
    return S / (double)N;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the LNCC loss L = 1 - (1/N) sum_i n_i with respect to J.      */
/* Differentiates the definition directly (App. fused LNCC, the chain rule  */
/* of Eq. gradientcc-first written for the moving image), with              */
/*   dn/dA = 2A/D,  dn/dC = -A^2 B / D^2,  D = B C + eps,                    */
/*   dA_i/dJ_k = (F_k - muF_i)/c_i,  dC_i/dJ_k = 2 (J_k - muJ_i)/c_i          */
/* for k inside window i, and dL/dn_i = -1/N.  Then                          */
/*   gJ_k = sum_{i : k in W_i} dL/dn_i (dn/dA dA_i/dJ_k + dn/dC dC_i/dJ_k). */
/* (The paper's printed coefficient A/(B^2 C) in Eq. gradientcc-first is     */
/* read as A^2/(B^2 C), as in its next line; eps is kept.)                   */
/* Returns S as or_lncc does.                                                */
/* ------------------------------------------------------------------------ */
double or_lncc_grad(const double *F, const double *J, int nx, int ny, int nz, int win, double eps,
                    double *gJ)
{
    const long N = (long)nx * ny * nz;
    const int r = win / 2;
    double *wq = (double *)malloc(sizeof(double) * 6 * (size_t)N);
    const double S = or_lncc(F, J, nx, ny, nz, win, eps, NULL, wq);
    const double *muF = wq, *muJ = wq + N, *A = wq + 2 * N, *B = wq + 3 * N, *C = wq + 4 * N,
                 *cnt = wq + 5 * N;
    /* per-window coefficients alpha_i (multiplies F_k - muF_i) and beta_i (J_k - muJ_i) */
    double *alpha = (double *)malloc(sizeof(double) * (size_t)N);
    double *beta = (double *)malloc(sizeof(double) * (size_t)N);
    const double dLdn = -1.0 / (double)N;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        const double D = B[i] * C[i] + eps;
        if (D > 0.0) {
            const double dndA = 2.0 * A[i] / D;
            const double dndC = -A[i] * A[i] * B[i] / (D * D);
            alpha[i] = dLdn * dndA / cnt[i];
            beta[i] = dLdn * dndC * 2.0 / cnt[i];
        } else {
            alpha[i] = 0.0;
            beta[i] = 0.0;
        }
    }
    /* k lies in W_i  <=>  i inside the volume and |i - k|_inf <= r */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const long k = lin(x, y, z, nx, ny);
                int x0, x1, y0, y1, z0, z1;
                window_bounds(x, r, nx, &x0, &x1);
                window_bounds(y, r, ny, &y0, &y1);
                window_bounds(z, r, nz, &z0, &z1);
                double g = 0.0;
                for (int zz = z0; zz <= z1; ++zz)
                    for (int yy = y0; yy <= y1; ++yy)
                        for (int xx = x0; xx <= x1; ++xx) {
                            const long i = lin(xx, yy, zz, nx, ny);
                            g += alpha[i] * (F[k] - muF[i]) + beta[i] * (J[k] - muJ[i]);
                        }
                gJ[k] = g;
            }
        }
    }
    free(alpha);
    free(beta);
    free(wq);
    return S;
}

/* ------------------------------------------------------------------------ */
/* The ANTs gradient approximation of the LNCC loss (App. fused LNCC,        */
/* paragraph "ANTs gradient approximation"): the convolution of the gamma   */
/* family with the window weights is skipped, i.e. every voxel k keeps only */
/* the term of its own window.  The exact gradient averages                 */
/*   gamma_i (F_k - muF_i) ... over the c_k windows i that contain k with   */
/* weights 1/c_i; the approximation replaces that average by the term of    */
/* i = k:                                                                    */
/*   gJ_k = c_k [ alpha_k (F_k - muF_k) + beta_k (J_k - muJ_k) ]             */
/* with alpha, beta as in or_lncc_grad (they carry dL/dn = -1/N and 1/c_k).  */
/* Equivalently gJ_k = -(c_k / N) d n_k / d J_k, the derivative of the       */
/* voxel's own window NCC with respect to its centre value.                 */
/* Returns S as or_lncc does.                                                */
/* ------------------------------------------------------------------------ */
double or_lncc_grad_ants(const double *F, const double *J, int nx, int ny, int nz, int win, double eps,
                         double *gJ)
{
    const long N = (long)nx * ny * nz;
    double *wq = (double *)malloc(sizeof(double) * 6 * (size_t)N);
    const double S = or_lncc(F, J, nx, ny, nz, win, eps, NULL, wq);
    const double *muF = wq, *muJ = wq + N, *A = wq + 2 * N, *B = wq + 3 * N, *C = wq + 4 * N,
                 *cnt = wq + 5 * N;
    const double dLdn = -1.0 / (double)N;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < N; ++k) {
        const double D = B[k] * C[k] + eps;
        double g = 0.0;
        if (D > 0.0) {
            const double alpha = dLdn * (2.0 * A[k] / D) / cnt[k];
            const double beta = dLdn * (-A[k] * A[k] * B[k] / (D * D)) * 2.0 / cnt[k];
            g = cnt[k] * (alpha * (F[k] - muF[k]) + beta * (J[k] - muJ[k]));
        }
        gJ[k] = g;
    }
    free(wq);
    return S;
}

/* ------------------------------------------------------------------------ */
/* Cubic B-spline Parzen kernel and its derivative (Sec. 2.2, Eq. mi, with   */
/* the 3rd-order B-spline choice of kappa).                                  */
/* ------------------------------------------------------------------------ */
double or_bspline3(double t)
{
    const double a = fabs(t);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

double or_bspline3_deriv(double t)
{
    const double a = fabs(t);
    const double s = t < 0.0 ? -1.0 : 1.0;
    if (a < 1.0) return s * (-2.0 * a + 1.5 * a * a);
    if (a < 2.0) return s * (-0.5 * (2.0 - a) * (2.0 - a));
    return 0.0;
}

/* Bin coordinate of an intensity v in [0,1] for B bins: the B-spline of     */
/* bin m is centred at s = m, and [0,1] maps onto [1, B-2] so that every     */
/* intensity has its full kernel support inside the B bins.                  */
static double bin_coord(double v, int B) { return v * (double)(B - 3) + 1.0; }

/* ------------------------------------------------------------------------ */
/* Parzen-window mutual information (Sec. 2.2, Eq. mi; App. fused MI).       */
/* Inputs Fh, Jh are intensities already mapped to [0,1].                    */
/*   p_IJ[m][n] = (1/N) sum_k kappa(sF_k - m) kappa(sJ_k - n)                */
/*   p_I[m] = sum_n p_IJ[m][n],  p_J[n] = sum_m p_IJ[m][n]                   */
/*   MI = sum_{m,n : p_IJ > 0} p_IJ log(p_IJ / (p_I p_J))   (natural log)     */
/* p_out (optional, B*B, row m = fixed-image bin).                           */
/* ------------------------------------------------------------------------ */
double or_mi(const double *Fh, const double *Jh, long N, int B, double *p_out)
{
    const int BB = B * B;
    /* one partial histogram per block of voxels, summed in block order */
    const long blk = 4096;
    const long nblk = (N + blk - 1) / blk;
    double *part = (double *)calloc((size_t)nblk * BB, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long b = 0; b < nblk; ++b) {
        double *h = part + b * BB;
        double wF[256], wJ[256];
        const long k1 = (b + 1) * blk < N ? (b + 1) * blk : N;
        for (long k = b * blk; k < k1; ++k) {
            const double sF = bin_coord(Fh[k], B), sJ = bin_coord(Jh[k], B);
            for (int m = 0; m < B; ++m) {
                wF[m] = or_bspline3(sF - (double)m);
                wJ[m] = or_bspline3(sJ - (double)m);
            }
            for (int m = 0; m < B; ++m)
                for (int n = 0; n < B; ++n) h[m * B + n] += wF[m] * wJ[n];
        }
    }
    double *p = (double *)calloc((size_t)BB, sizeof(double));
    for (long b = 0; b < nblk; ++b)
        for (int e = 0; e < BB; ++e) p[e] += part[b * BB + e];
    free(part);
    for (int e = 0; e < BB; ++e) p[e] /= (double)N;
    double pI[256], pJ[256];
    for (int m = 0; m < B; ++m) {
        pI[m] = 0.0;
        pJ[m] = 0.0;
    }
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            pI[m] += p[m * B + n];
            pJ[n] += p[m * B + n];
        }
    double mi = 0.0;
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            const double v = p[m * B + n];
            if (v > 0.0) mi += v * log(v / (pI[m] * pJ[n]));
        }
    if (p_out) memcpy(p_out, p, sizeof(double) * (size_t)BB);
    free(p);
    return mi;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the MI loss L = -MI with respect to Jh (App. fused MI, Eq.    */
/* gradientmi-threadn, with the marginals obtained from the joint).          */
/* With MI = sum p log p - sum p_I log p_I - sum p_J log p_J and the        */
/* marginals taken as row/column sums of the joint,                          */
/*   dMI/dp_IJ[m][n] = log(p_IJ[m][n] / (p_I[m] p_J[n])) - 1,                */
/* and the -1 drops out because sum_{m,n} dp_IJ/dJh_k = 0 (the kernel is a   */
/* partition of unity).  So G[m][n] = log(p_IJ / (p_I p_J)), 0 where         */
/* p_IJ = 0 (no voxel then has a non-zero derivative there).  Then           */
/*   dL/dJh_k = -(1/N) (B-3) sum_{m,n} G[m][n] kappa(sF_k - m) kappa'(sJ_k - n). */
/* Returns MI.                                                               */
/* ------------------------------------------------------------------------ */
/* The Parzen adjoint of MI for a given joint PMF p (B*B): marginals,        */
/* G = log(p / (pI pJ)), then gJh_k = -(B-3)/N sum_mn G[m][n] kappa(sF_k-m)   */
/* kappa'(sJ_k-n)  (Eq. gradientmi-threadn).                                  */
static void mi_adjoint_n(const double *Fh, const double *Jh, long n, long N, int B, const double *p, double *gJh);
static void mi_adjoint(const double *Fh, const double *Jh, long N, int B, const double *p, double *gJh)
{
    mi_adjoint_n(Fh, Jh, N, N, B, p, gJh);
}

/* The same adjoint at n given voxels of a volume of N voxels whose joint     */
/* PMF is p: the per-voxel form used for sampled checks of large volumes.     */
void or_mi_adjoint_points(const double *Fh, const double *Jh, long n, long N, int B, const double *p, double *gJh)
{
    mi_adjoint_n(Fh, Jh, n, N, B, p, gJh);
}

static void mi_adjoint_n(const double *Fh, const double *Jh, long n, long N, int B, const double *p, double *gJh)
{
    const int BB = B * B;
    double pI[256], pJ[256];
    for (int m = 0; m < B; ++m) {
        pI[m] = 0.0;
        pJ[m] = 0.0;
    }
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            pI[m] += p[m * B + n];
            pJ[n] += p[m * B + n];
        }
    double *G = (double *)malloc(sizeof(double) * (size_t)BB);
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            const double v = p[m * B + n];
            G[m * B + n] = v > 0.0 ? log(v / (pI[m] * pJ[n])) : 0.0;
        }
    const double scale = -(double)(B - 3) / (double)N;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        double wF[256], dJ[256];
        const double sF = bin_coord(Fh[k], B), sJ = bin_coord(Jh[k], B);
        for (int m = 0; m < B; ++m) {
            wF[m] = or_bspline3(sF - (double)m);
            dJ[m] = or_bspline3_deriv(sJ - (double)m);
        }
        double g = 0.0;
        for (int m = 0; m < B; ++m)
            for (int n = 0; n < B; ++n) g += G[m * B + n] * wF[m] * dJ[n];
        gJh[k] = scale * g;
    }
    free(G);
}

double or_mi_grad(const double *Fh, const double *Jh, long N, int B, double *gJh)
{
    double *p = (double *)malloc(sizeof(double) * (size_t)B * B);
    const double mi = or_mi(Fh, Jh, N, B, p);
    mi_adjoint(Fh, Jh, N, B, p, gJh);
    free(p);
    return mi;
}

static double mi_of_pmf(const double *p, int B);
/* MI of a given joint PMF (B*B, row = fixed-image bin). */
double or_mi_of_pmf(const double *p, int B) { return mi_of_pmf(p, B); }

static double mi_of_pmf(const double *p, int B)
{
    double pI[256], pJ[256];
    for (int m = 0; m < B; ++m) {
        pI[m] = 0.0;
        pJ[m] = 0.0;
    }
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            pI[m] += p[m * B + n];
            pJ[n] += p[m * B + n];
        }
    double mi = 0.0;
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            const double v = p[m * B + n];
            if (v > 0.0) mi += v * log(v / (pI[m] * pJ[n]));
        }
    return mi;
}

/* ------------------------------------------------------------------------ */
/* The approximate (hard-binned) MI estimator of App. fused MI ("An          */
/* approximate histogram estimator"): each sample adds 1 to the bin nearest  */
/* to it, and the count histogram, divided by N, is convolved with the       */
/* kernel kappa; the PMF is exact for samples on bin centres.  With the bin  */
/* layout of or_mi (kernel of bin m centred at s = m), the nearest bin of s  */
/* is floor(s + 1/2) and the convolution weights are kappa(a) kappa(b) for   */
/* a, b in {-1, 0, 1} (kappa(+-2) = 0): 1/6, 2/3, 1/6.                        */
/* The bin decision is taken in FP32, as the GPU takes it:                   */
/*   t = clamp((v - lo) * scale, 0, 1), s = fma(t, B - 3, 1), m* = floor(s + 1/2). */
/* F, J are raw intensities; p_out (optional, B*B).                          */
/* ------------------------------------------------------------------------ */
static int hard_bin(double v, float lo, float scale, int B)
{
    float t = ((float)v - lo) * scale;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    const float sb = fmaf(t, (float)(B - 3), 1.0f);
    int m = (int)floorf(sb + 0.5f);
    if (m < 1) m = 1;
    if (m > B - 2) m = B - 2;
    return m;
}

double or_mi_hard(const double *F, const double *J, long N, int B, float f_lo, float f_scale, float m_lo,
                  float m_scale, double *p_out)
{
    const int BB = B * B;
    double *cnt = (double *)calloc((size_t)BB, sizeof(double));
    for (long k = 0; k < N; ++k) cnt[hard_bin(F[k], f_lo, f_scale, B) * B + hard_bin(J[k], m_lo, m_scale, B)] += 1.0;
    const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    double *p = (double *)malloc(sizeof(double) * (size_t)BB);
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            double acc = 0.0;
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b) {
                    const int mm = m - a, nn = n - b;
                    if (mm < 0 || mm >= B || nn < 0 || nn >= B) continue;
                    acc += w[a + 1] * w[b + 1] * cnt[mm * B + nn];
                }
            p[m * B + n] = acc / (double)N;
        }
    const double mi = mi_of_pmf(p, B);
    if (p_out) memcpy(p_out, p, sizeof(double) * (size_t)BB);
    free(p);
    free(cnt);
    return mi;
}

/* Gradient paired with the hard-binned forward (the paper gives only the   */
/* forward): the Parzen adjoint (Eq. gradientmi-threadn) evaluated with the */
/* approximate PMF's table G.  Fh, Jh are the intensities mapped to [0,1]    */
/* in FP64 for the kernel derivative at each sample's own position.         */
double or_mi_hard_grad(const double *F, const double *J, const double *Fh, const double *Jh, long N, int B,
                       float f_lo, float f_scale, float m_lo, float m_scale, double *gJh)
{
    double *p = (double *)malloc(sizeof(double) * (size_t)B * B);
    const double mi = or_mi_hard(F, J, N, B, f_lo, f_scale, m_lo, m_scale, p);
    mi_adjoint(Fh, Jh, N, B, p, gJh);
    free(p);
    return mi;
}

/* ------------------------------------------------------------------------ */
/* Gaussian smoothing of a field (the sigma_grad / sigma_warp smoothing      */
/* regularisation the paper runs with, FireANTs style): each of nch SoA      */
/* channels [nch][nz][ny][nx] is convolved separably along x, y, z with       */
/* w_k = exp(-k^2 / (2 sigma^2)) / sum, |k| <= floor(4 sigma + 1/2), borders  */
/* repeating the edge voxel.  out may not alias in.                          */
/* ------------------------------------------------------------------------ */
void or_gaussian_smooth(const double *in, int nx, int ny, int nz, int nch, double sigma, double *out)
{
    const long N = (long)nx * ny * nz;
    const int r = (int)(4.0 * sigma + 0.5);
    double *w = (double *)malloc(sizeof(double) * (size_t)(2 * r + 1));
    double sum = 0.0;
    for (int k = -r; k <= r; ++k) {
        w[k + r] = exp(-0.5 * (double)k * (double)k / (sigma * sigma));
        sum += w[k + r];
    }
    for (int k = 0; k <= 2 * r; ++k) w[k] /= sum;
    double *a = (double *)malloc(sizeof(double) * (size_t)N);
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    const int n[3] = {nx, ny, nz};
    for (int c = 0; c < nch; ++c) {
        memcpy(a, in + (long)c * N, sizeof(double) * (size_t)N);
        for (int axis = 0; axis < 3; ++axis) {
#pragma omp parallel for schedule(static)
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        int q[3] = {x, y, z};
                        const int q0 = q[axis];
                        double acc = 0.0;
                        for (int k = -r; k <= r; ++k) {
                            int qq = q0 + k;
                            qq = qq < 0 ? 0 : (qq > n[axis] - 1 ? n[axis] - 1 : qq);
                            q[axis] = qq;
                            acc += w[k + r] * a[lin(q[0], q[1], q[2], nx, ny)];
                        }
                        b[lin(x, y, z, nx, ny)] = acc;
                    }
            double *t = a;
            a = b;
            b = t;
        }
        memcpy(out + (long)c * N, a, sizeof(double) * (size_t)N);
    }
    free(a);
    free(b);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* 2x downsampling of an image for the multi-scale schedule the paper runs   */
/* (coarse-to-fine levels): out[z][y][x] = mean of in over the 2x2x2 block   */
/* (2x, 2y, 2z); nx, ny, nz even.                                            */
/* ------------------------------------------------------------------------ */
void or_downsample2(const double *in, int nx, int ny, int nz, double *out)
{
    const int mx = nx / 2, my = ny / 2, mz = nz / 2;
    for (int z = 0; z < mz; ++z)
        for (int y = 0; y < my; ++y)
            for (int x = 0; x < mx; ++x) {
                double acc = 0.0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) acc += in[lin(2 * x + dx, 2 * y + dy, 2 * z + dz, nx, ny)];
                out[lin(x, y, z, mx, my)] = acc / 8.0;
            }
}

/* ------------------------------------------------------------------------ */
/* Diffusion regulariser (Sec. 1 lists the Sobolev norm of the gradient as  */
/* a common R; this is its first-order, squared form):                       */
/*   R(u) = (1/N) sum_c sum_d sum_{p : p+e_d inside} (u_c(p+e_d) - u_c(p))^2  */
/* grad (optional, 3N, overwritten) = dR/du, by the chain rule of each       */
/* squared difference.                                                       */
/* ------------------------------------------------------------------------ */
double or_diffusion(const double *u, int nx, int ny, int nz, double *grad)
{
    const long N = (long)nx * ny * nz;
    if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)N);
    const int step_ok[3] = {nx > 1, ny > 1, nz > 1};
    double R = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double *uc = u + (long)c * N;
        double *gc = grad ? grad + (long)c * N : NULL;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long p = lin(x, y, z, nx, ny);
                    const int q[3][3] = {{x + 1, y, z}, {x, y + 1, z}, {x, y, z + 1}};
                    for (int d = 0; d < 3; ++d) {
                        if (!step_ok[d]) continue;
                        if (q[d][0] >= nx || q[d][1] >= ny || q[d][2] >= nz) continue;
                        const long pn = lin(q[d][0], q[d][1], q[d][2], nx, ny);
                        const double diff = uc[pn] - uc[p];
                        R += diff * diff;
                        if (gc) {
                            gc[pn] += 2.0 * diff / (double)N;
                            gc[p] -= 2.0 * diff / (double)N;
                        }
                    }
                }
    }
    return R / (double)N;
}

/* ------------------------------------------------------------------------ */
/* bfloat16 round-to-nearest-even of a value, through its FP32 bit pattern   */
/* (bfloat16 keeps the top 16 bits of an IEEE-754 binary32).                */
/* ------------------------------------------------------------------------ */
double or_bf16_round(double x)
{
    float f = (float)x;
    uint32_t bits;
    memcpy(&bits, &f, 4);
    if ((bits & 0x7f800000u) == 0x7f800000u) { /* inf / nan pass through */
        if (bits & 0x007fffffu) bits |= 0x00400000u;
        bits &= 0xffff0000u;
    } else {
        const uint32_t lsb = (bits >> 16) & 1u;
        bits = bits + 0x7fffu + lsb;
        bits &= 0xffff0000u;
    }
    float out;
    memcpy(&out, &bits, 4);
    return (double)out;
}

/* ------------------------------------------------------------------------ */
/* One Adam step (the optimiser state m1, m2 of Sec. 3.1), with bias         */
/* correction, on n elements:                                                */
/*   gs = grad_scale * g;  m = b1 m + (1-b1) gs;  v = b2 v + (1-b2) gs^2;     */
/*   u -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).                  */
/* bf16_moments: the update uses the new m, v as computed; the stored m, v   */
/* are then rounded to bfloat16 (round to nearest even).                     */
/* ------------------------------------------------------------------------ */
void or_adam(double *u, double *m, double *v, const double *g, long n, double lr, double b1,
             double b2, double eps, double grad_scale, int t, int bf16_moments)
{
    const double bc1 = 1.0 - pow(b1, (double)t);
    const double bc2 = 1.0 - pow(b2, (double)t);
    for (long i = 0; i < n; ++i) {
        const double gs = grad_scale * g[i];
        const double mn = b1 * m[i] + (1.0 - b1) * gs;
        const double vn = b2 * v[i] + (1.0 - b2) * gs * gs;
        u[i] -= lr * (mn / bc1) / (sqrt(vn / bc2) + eps);
        m[i] = bf16_moments ? or_bf16_round(mn) : mn;
        v[i] = bf16_moments ? or_bf16_round(vn) : vn;
    }
}

/* ------------------------------------------------------------------------ */
/* Jacobian determinant of phi = id + u: det(I + grad u), with central       */
/* differences in the interior and one-sided differences at the border      */
/* (0 along an axis of length 1).  Row c = displacement component, column d */
/* = derivative axis.                                                        */
/* ------------------------------------------------------------------------ */
void or_jacdet(const double *u, int nx, int ny, int nz, double *det)
{
    const long N = (long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int pc[3] = {x, y, z};
                double Jm[3][3];
                for (int c = 0; c < 3; ++c) {
                    const double *uc = u + (long)c * N;
                    for (int d = 0; d < 3; ++d) {
                        int lo[3] = {x, y, z}, hi[3] = {x, y, z};
                        double h = 0.0;
                        if (n[d] > 1) {
                            if (pc[d] > 0) lo[d] = pc[d] - 1;
                            if (pc[d] < n[d] - 1) hi[d] = pc[d] + 1;
                            h = (double)(hi[d] - lo[d]);
                        }
                        double deriv = 0.0;
                        if (h > 0.0)
                            deriv = (uc[lin(hi[0], hi[1], hi[2], nx, ny)] -
                                     uc[lin(lo[0], lo[1], lo[2], nx, ny)]) / h;
                        Jm[c][d] = (c == d ? 1.0 : 0.0) + deriv;
                    }
                }
                det[lin(x, y, z, nx, ny)] =
                    Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                    Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                    Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
            }
}

int or_version(void) { return 1; }

/* ------------------------------------------------------------------------ */
/* The same LNCC gradient as or_lncc_grad, evaluated only at listed voxels   */
/* (linear indices pts[0..npts)), for volumes too large for the full field: */
/* for each listed k, every window i with k in W_i is formed from its        */
/* definition and contributes its chain-rule term.  N is the full voxel      */
/* count (dL/dn_i = -1/N).  n_out (optional) receives n_k at the same        */
/* voxels.                                                                   */
/* ------------------------------------------------------------------------ */
static void window_stats(const double *F, const double *J, int nx, int ny, int nz, int r, int x, int y, int z,
                         double eps, double *muF, double *muJ, double *A, double *B, double *C, double *cnt)
{
    int x0, x1, y0, y1, z0, z1;
    window_bounds(x, r, nx, &x0, &x1);
    window_bounds(y, r, ny, &y0, &y1);
    window_bounds(z, r, nz, &z0, &z1);
    double c = 0.0, sF = 0.0, sJ = 0.0;
    for (int zz = z0; zz <= z1; ++zz)
        for (int yy = y0; yy <= y1; ++yy)
            for (int xx = x0; xx <= x1; ++xx) {
                const long k = lin(xx, yy, zz, nx, ny);
                sF += F[k];
                sJ += J[k];
                c += 1.0;
            }
    const double mF = sF / c, mJ = sJ / c;
    double a = 0.0, b = 0.0, cc = 0.0;
    for (int zz = z0; zz <= z1; ++zz)
        for (int yy = y0; yy <= y1; ++yy)
            for (int xx = x0; xx <= x1; ++xx) {
                const long k = lin(xx, yy, zz, nx, ny);
                const double df = F[k] - mF, dj = J[k] - mJ;
                a += df * dj;
                b += df * df;
                cc += dj * dj;
            }
    *muF = mF;
    *muJ = mJ;
    *A = a / c;
    *B = b / c;
    *C = cc / c;
    *cnt = c;
    (void)eps;
}

void or_lncc_grad_points(const double *F, const double *J, int nx, int ny, int nz, int win, double eps,
                         const long *pts, int npts, double *gJ_out, double *n_out)
{
    const long N = (long)nx * ny * nz;
    const int r = win / 2;
    const double dLdn = -1.0 / (double)N;
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < npts; ++s) {
        const long k = pts[s];
        const int x = (int)(k % nx), y = (int)((k / nx) % ny), z = (int)(k / ((long)nx * ny));
        int x0, x1, y0, y1, z0, z1;
        window_bounds(x, r, nx, &x0, &x1);
        window_bounds(y, r, ny, &y0, &y1);
        window_bounds(z, r, nz, &z0, &z1);
        double g = 0.0;
        for (int zz = z0; zz <= z1; ++zz)
            for (int yy = y0; yy <= y1; ++yy)
                for (int xx = x0; xx <= x1; ++xx) {
                    double mF, mJ, A, B, C, c;
                    window_stats(F, J, nx, ny, nz, r, xx, yy, zz, eps, &mF, &mJ, &A, &B, &C, &c);
                    const double D = B * C + eps;
                    if (D > 0.0) {
                        const double dndA = 2.0 * A / D;
                        const double dndC = -A * A * B / (D * D);
                        g += dLdn * (dndA * (F[k] - mF) / c + dndC * 2.0 * (J[k] - mJ) / c);
                    }
                }
        gJ_out[s] = g;
        if (n_out) {
            double mF, mJ, A, B, C, c;
            window_stats(F, J, nx, ny, nz, r, x, y, z, eps, &mF, &mJ, &A, &B, &C, &c);
            const double D = B * C + eps;
            n_out[s] = D > 0.0 ? A * A / D : 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 3-D convolution of the learned initialiser (3x3x3 taps, zero padding 1,  */
/* stride 1), channels-last: in[v][Cin], w[Cout][27][Cin] with tap          */
/* t = (kz*3 + ky)*3 + kx for offset (kx-1, ky-1, kz-1), out[v][Cout].       */
/* The plain definition: out[v][o] = bias[o] + sum_t sum_c w[o][t][c]        */
/* in[v + off(t)][c], and its two adjoints.                                  */
/* ------------------------------------------------------------------------ */
static int tap_neighbour(int x, int y, int z, int t, int nx, int ny, int nz, long *q)
{
    const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
    if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) return 0;
    *q = lin(xx, yy, zz, nx, ny);
    return 1;
}

void or_conv3d(const double *in, int Cin, const double *w, const double *bias, int Cout, int nx, int ny, int nz,
               double *out)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long v = lin(x, y, z, nx, ny);
                for (int o = 0; o < Cout; ++o) {
                    double acc = bias ? bias[o] : 0.0;
                    for (int t = 0; t < 27; ++t) {
                        long q;
                        if (!tap_neighbour(x, y, z, t, nx, ny, nz, &q)) continue;
                        for (int c = 0; c < Cin; ++c) acc += w[((long)o * 27 + t) * Cin + c] * in[q * Cin + c];
                    }
                    out[v * Cout + o] = acc;
                }
            }
}

/* din[q][c] = sum over (v, t) with v + off(t) = q of sum_o w[o][t][c] dout[v][o] */
void or_conv3d_dgrad(const double *dout, int Cout, const double *w, int Cin, int nx, int ny, int nz, double *din)
{
    const long N = (long)nx * ny * nz;
    memset(din, 0, sizeof(double) * (size_t)N * Cin);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long v = lin(x, y, z, nx, ny);
                for (int t = 0; t < 27; ++t) {
                    long q;
                    if (!tap_neighbour(x, y, z, t, nx, ny, nz, &q)) continue;
                    for (int o = 0; o < Cout; ++o)
                        for (int c = 0; c < Cin; ++c)
                            din[q * Cin + c] += w[((long)o * 27 + t) * Cin + c] * dout[v * Cout + o];
                }
            }
}

/* dw[o][t][c] = sum_v dout[v][o] in[v + off(t)][c] */
void or_conv3d_wgrad(const double *in, int Cin, const double *dout, int Cout, int nx, int ny, int nz, double *dw)
{
#pragma omp parallel for schedule(static)
    for (int o = 0; o < Cout; ++o)
        for (int t = 0; t < 27; ++t)
            for (int c = 0; c < Cin; ++c) {
                double acc = 0.0;
                for (int z = 0; z < nz; ++z)
                    for (int y = 0; y < ny; ++y)
                        for (int x = 0; x < nx; ++x) {
                            long q;
                            if (!tap_neighbour(x, y, z, t, nx, ny, nz, &q)) continue;
                            acc += dout[lin(x, y, z, nx, ny) * Cout + o] * in[q * Cin + c];
                        }
                dw[((long)o * 27 + t) * Cin + c] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* The learned initialiser's other operators (the U-Net of the workloads:   */
/* LeakyReLU 0.2, 2x average pooling down, 2x trilinear upsampling plus     */
/* channel concat up, and the resampling of its half-resolution output to   */
/* the registration grid).  Activations are channels-last in[v][C];         */
/* displacement fields are [3][nz][ny][nx] in voxel units of their grid.    */
/* ------------------------------------------------------------------------ */

/* LeakyReLU: x for x > 0, slope * x otherwise; its derivative 1 or slope   */
/* (slope at x = 0).  dx = dy * f'(x).                                       */
void or_leaky(const double *x, long n, double slope, double *y)
{
    for (long i = 0; i < n; ++i) y[i] = x[i] > 0.0 ? x[i] : slope * x[i];
}
void or_leaky_bwd(const double *x, const double *dy, long n, double slope, double *dx)
{
    for (long i = 0; i < n; ++i) dx[i] = x[i] > 0.0 ? dy[i] : slope * dy[i];
}

/* 2x average pooling: out[Z][Y][X][c] = mean of in over the 2x2x2 block at */
/* (2X, 2Y, 2Z); nx, ny, nz (the input's) even.  The adjoint spreads each   */
/* coarse gradient over its block with weight 1/8.                          */
void or_avgpool2(const double *in, int C, int nx, int ny, int nz, double *out)
{
    const int mx = nx / 2, my = ny / 2, mz = nz / 2;
    for (int Z = 0; Z < mz; ++Z)
        for (int Y = 0; Y < my; ++Y)
            for (int X = 0; X < mx; ++X)
                for (int c = 0; c < C; ++c) {
                    double s = 0.0;
                    for (int dz = 0; dz < 2; ++dz)
                        for (int dy = 0; dy < 2; ++dy)
                            for (int dx = 0; dx < 2; ++dx)
                                s += in[lin(2 * X + dx, 2 * Y + dy, 2 * Z + dz, nx, ny) * C + c];
                    out[lin(X, Y, Z, mx, my) * C + c] = s / 8.0;
                }
}
void or_avgpool2_adjoint(const double *gout, int C, int nx, int ny, int nz, double *gin)
{
    const int mx = nx / 2, my = ny / 2;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int c = 0; c < C; ++c)
                    gin[lin(x, y, z, nx, ny) * C + c] = gout[lin(x / 2, y / 2, z / 2, mx, my) * C + c] / 8.0;
}

/* Trilinear upsampling by an integer factor s with voxel-centre alignment: */
/* the centre of fine voxel f lies at coarse coordinate (f + 1/2) / s - 1/2  */
/* (x_fine = s x_coarse + (s - 1) / 2).  Along each axis the value is the    */
/* linear interpolation between the coarse voxels floor(c) and floor(c) + 1, */
/* both clamped into [0, n - 1] (border).  in: coarse [nzc][nyc][nxc][C],    */
/* out: fine (s nxc, s nyc, s nzc) x C.                                      */
static void up_coord(int f, int s, int n, int *i0, int *i1, double *a)
{
    const double c = ((double)f + 0.5) / (double)s - 0.5;
    const double fl = floor(c);
    *a = c - fl;
    int lo = (int)fl, hi = (int)fl + 1;
    *i0 = lo < 0 ? 0 : (lo > n - 1 ? n - 1 : lo);
    *i1 = hi < 0 ? 0 : (hi > n - 1 ? n - 1 : hi);
}

void or_upsample(const double *in, int C, int nxc, int nyc, int nzc, int s, double *out)
{
    const int nx = s * nxc, ny = s * nyc, nz = s * nzc;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int ix[2], iy[2], iz[2];
                double ax, ay, az;
                up_coord(x, s, nxc, &ix[0], &ix[1], &ax);
                up_coord(y, s, nyc, &iy[0], &iy[1], &ay);
                up_coord(z, s, nzc, &iz[0], &iz[1], &az);
                for (int c = 0; c < C; ++c) {
                    double v = 0.0;
                    for (int b = 0; b < 8; ++b) {
                        const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
                        const double w = (bx ? ax : 1.0 - ax) * (by ? ay : 1.0 - ay) * (bz ? az : 1.0 - az);
                        v += w * in[lin(ix[bx], iy[by], iz[bz], nxc, nyc) * C + c];
                    }
                    out[lin(x, y, z, nx, ny) * C + c] = v;
                }
            }
}

/* its adjoint: every fine gradient scattered onto its 8 coarse corners */
void or_upsample_adjoint(const double *gout, int C, int nxc, int nyc, int nzc, int s, double *gin)
{
    const int nx = s * nxc, ny = s * nyc, nz = s * nzc;
    memset(gin, 0, sizeof(double) * (size_t)nxc * nyc * nzc * C);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int ix[2], iy[2], iz[2];
                double ax, ay, az;
                up_coord(x, s, nxc, &ix[0], &ix[1], &ax);
                up_coord(y, s, nyc, &iy[0], &iy[1], &ay);
                up_coord(z, s, nzc, &iz[0], &iz[1], &az);
                for (int c = 0; c < C; ++c)
                    for (int b = 0; b < 8; ++b) {
                        const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
                        const double w = (bx ? ax : 1.0 - ax) * (by ? ay : 1.0 - ay) * (bz ? az : 1.0 - az);
                        gin[lin(ix[bx], iy[by], iz[bz], nxc, nyc) * C + c] += w * gout[lin(x, y, z, nx, ny) * C + c];
                    }
            }
}

/* channel concat of two channels-last volumes of V voxels: out[v] =        */
/* [a[v][0 .. Ca), b[v][0 .. Cb)]                                            */
void or_concat(const double *a, int Ca, const double *b, int Cb, long V, double *out)
{
    for (long v = 0; v < V; ++v) {
        for (int c = 0; c < Ca; ++c) out[v * (Ca + Cb) + c] = a[v * Ca + c];
        for (int c = 0; c < Cb; ++c) out[v * (Ca + Cb) + Ca + c] = b[v * Cb + c];
    }
}

/* Displacement resampling between the network's grid and the registration */
/* grid.  Down: 2x block mean of each channel, halved (the displacement in  */
/* coarse voxels).  Up: trilinear upsampling by s (as or_upsample),          */
/* multiplied by s (the displacement in fine voxels).                        */
void or_field_down2(const double *u, int nx, int ny, int nz, double *out)
{
    const int mx = nx / 2, my = ny / 2, mz = nz / 2;
    const long n = (long)nx * ny * nz, m = (long)mx * my * mz;
    for (int ch = 0; ch < 3; ++ch) {
        or_avgpool2(u + ch * n, 1, nx, ny, nz, out + ch * m);
        for (long i = 0; i < m; ++i) out[ch * m + i] *= 0.5;
    }
}
void or_field_upsample(const double *u, int nxc, int nyc, int nzc, int s, double *out)
{
    const long m = (long)nxc * nyc * nzc, n = m * s * s * s;
    for (int ch = 0; ch < 3; ++ch) {
        or_upsample(u + ch * m, 1, nxc, nyc, nzc, s, out + ch * n);
        for (long i = 0; i < n; ++i) out[ch * n + i] *= (double)s;
    }
}

/* The network input: F and M averaged over factor^3 blocks, each mapped to */
/* (v - lo) / (hi - lo); out[v][0] = F, out[v][1] = M at d / factor.         */
void or_pack_pair(const double *F, const double *M, int nx, int ny, int nz, int factor, double f_lo, double f_hi,
                  double m_lo, double m_hi, double *out)
{
    const int mx = nx / factor, my = ny / factor, mz = nz / factor;
    const double cnt = (double)factor * factor * factor;
    for (int Z = 0; Z < mz; ++Z)
        for (int Y = 0; Y < my; ++Y)
            for (int X = 0; X < mx; ++X) {
                double sf = 0.0, sm = 0.0;
                for (int dz = 0; dz < factor; ++dz)
                    for (int dy = 0; dy < factor; ++dy)
                        for (int dx = 0; dx < factor; ++dx) {
                            const long p = lin(X * factor + dx, Y * factor + dy, Z * factor + dz, nx, ny);
                            sf += F[p];
                            sm += M[p];
                        }
                const long v = lin(X, Y, Z, mx, my);
                out[2 * v] = (sf / cnt - f_lo) / (f_hi - f_lo);
                out[2 * v + 1] = (sm / cnt - m_lo) / (m_hi - m_lo);
            }
}

/* The training loss: mean over the 3 channels and V voxels of              */
/* (pred - target)^2, and its gradient 2 (pred - target) / (3 V).           */
double or_mse(const double *pred, const double *target, long V, double *grad)
{
    double s = 0.0;
    for (long i = 0; i < 3 * V; ++i) {
        const double d = pred[i] - target[i];
        s += d * d;
        if (grad) grad[i] = 2.0 * d / (3.0 * (double)V);
    }
    return s / (3.0 * (double)V);
}
