/*
 * FP64 CPU oracle for the moving-least-squares (MLS) field reconstruction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain statement of what
 * the CUDA path computes.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it; the library never does.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * What it computes, per pixel centre p of a W x H grid over the view
 * rectangle [x0,x1] x [y0,y1] (pixel (u,v) has centre
 * (x0 + (u+1/2)(x1-x0)/W, y0 + (v+1/2)(y1-y0)/H), row-major, v = 0 at y0):
 *
 *   r_i^2 = |x_i - p|^2 over all n points x_i (Section 3.3: every pixel
 *           depends on every data point, Section 4.5 O(whn))
 *   w_i   = weight(r_i)          (Section 3.3, Eq. eq-weights gives the
 *           inverse-distance form 1/r^(2 alpha); the Gaussian exp(-r^2/h^2)
 *           and the Wendland C2 form (1-q)^4 (4q+1), q = r/rho < 1, are the
 *           compact / smooth alternatives)
 *   b(d)  = (1, d_x, d_y [, d_x^2, d_x d_y, d_y^2]),  d = (x_i - p)/s
 *   M     = sum_i w_i b(d_i) b(d_i)^T,   R = sum_i w_i b(d_i) f_i^T
 *   c     = M^{-1} R,   f(p) = b(0)^T c = row 0 of c
 *
 * This is the weighted least-squares polynomial fit evaluated at p; with the
 * linear basis it is the paper's affine MLS (Section 3.3.2, Eq.
 * eq-affinemls with the weighted centroids of Eqs. eq-pstar/eq-qstar), with
 * the constant basis it is the weighted mean of Section 3.3.1 (Eq.
 * eq-meanmls without the displacement term).  Each data dimension f_d is
 * fitted with the same M (the values q_i of the paper are read as the
 * point's data values).
 *
 * Readings where the paper is silent:
 *  - stabilised weights: Gaussian w_i = exp(-(r_i^2 - m)/h^2) and
 *    inverse-distance w_i = (m / r_i^2)^alpha with m = min_i r_i^2; a common
 *    positive factor on every weight leaves c unchanged, so this is the same
 *    fit without underflow;
 *  - inverse distance with a point exactly at p: f(p) is the mean value of
 *    the points at p (the limit of Section 3.3.1 / criterion 2 of Section 3.3);
 *  - degenerate pixels: with k basis terms, if fewer than k points carry a
 *    positive weight (Gaussian and inverse distance: all n points count;
 *    Wendland: points with r < rho), or the Cholesky factorisation of the
 *    diagonally equilibrated Me = S M S (S = diag(M_aa^{-1/2})) fails, or
 *    rcond_1(Me) = 1/(|Me|_1 |Me^{-1}|_1) < rcond_min, the next lower degree
 *    is tried (2 -> 1 -> 0); with no point in support the value is NaN;
 *  - iso-bands (Section 3.4, discrete colours): band_d = #{j : t_dj <= f_d},
 *    255 for NaN.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (contraction off so
 * that the x86 and Arm builds round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_GAUSS 0
#define OR_WENDLAND 1
#define OR_INVDIST 2

/* Basis term a of degree <= 2 evaluated at (dx, dy). */
static double basis_term(int a, double dx, double dy) {
    switch (a) {
    case 0: return 1.0;
    case 1: return dx;
    case 2: return dy;
    case 3: return dx * dx;
    case 4: return dx * dy;
    default: return dy * dy;
    }
}

/* Centre of pixel column (row) u of width s starting at x0 (Section 3.3:
 * the field is evaluated at each pixel's centre). */
static double pixel_centre(double x0, double s, int64_t u) { return x0 + ((double)u + 0.5) * s; }

static int n_terms(int degree) { return (degree + 1) * (degree + 2) / 2; }

/* Cholesky of a k x k symmetric matrix A (row-major) into lower L.
 * Returns 0 on success, -1 if a pivot is not positive. */
static int cholesky(int k, const double *A, double *L) {
    memset(L, 0, sizeof(double) * k * k);
    for (int j = 0; j < k; ++j) {
        double s = A[j * k + j];
        for (int t = 0; t < j; ++t) s -= L[j * k + t] * L[j * k + t];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        L[j * k + j] = ljj;
        for (int i = j + 1; i < k; ++i) {
            double v = A[i * k + j];
            for (int t = 0; t < j; ++t) v -= L[i * k + t] * L[j * k + t];
            L[i * k + j] = v / ljj;
        }
    }
    return 0;
}

/* Solve L L^T x = b in place. */
static void chol_solve(int k, const double *L, double *x) {
    for (int i = 0; i < k; ++i) {
        double v = x[i];
        for (int t = 0; t < i; ++t) v -= L[i * k + t] * x[t];
        x[i] = v / L[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = x[i];
        for (int t = i + 1; t < k; ++t) v -= L[t * k + i] * x[t];
        x[i] = v / L[i * k + i];
    }
}

static double norm1(int k, const double *A) {
    double best = 0.0;
    for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += fabs(A[i * k + j]);
        if (s > best) best = s;
    }
    return best;
}

/* Relative error bound, in units of u = 2^-53, of the computed weight
 * w_i of one pair (first order), for ecoef_fix.  r2 = |x_i - p|^2 carries
 * at most 4 u (two differences, two squares, one sum); a common factor on
 * every weight (the stabiliser m, its rounding included) leaves the fit
 * unchanged, so m counts as exact.
 *  - Gaussian exp(-(r2 - m)/h2): argument error 4 u r2/h2 from r2, u and u
 *    of |r2 - m|/h2 from the subtraction and the quotient, 2 u for exp.
 *  - Wendland t^4 (4q + 1), q = sqrt(r2)/h, t = 1 - q: q carries 4 u, so
 *    t carries (4 q/t + 1) u; t^4 multiplies that by 4 and adds 3 u; the
 *    factor 4q + 1 carries at most 5 u; the final product u.
 *  - inverse distance (m/r2)^alpha: the quotient carries 5 u (m exact, as
 *    above), raised to alpha; 4 u for pow. */
static double weight_rel_error(int32_t weight, double r2, double m, double h2, double h, double alpha) {
    if (weight == OR_GAUSS) return 2.0 + (4.0 * r2 + 2.0 * fabs(r2 - m)) / h2;
    if (weight == OR_WENDLAND) {
        const double qd = sqrt(r2) / h, t = 1.0 - qd;
        return 13.0 + 16.0 * qd / t;
    }
    return 5.0 * alpha + 4.0;
}

/*
 * Evaluate the MLS fit for a list of pixels.
 *
 *   xy       n x 2 positions (row-major), F n x D values (row-major)
 *   degree   0, 1 or 2; weight OR_*; h = Gaussian h / Wendland radius /
 *            inverse-distance basis scale; alpha = inverse-distance exponent
 *   trunc    Gaussian only: 0 for the full sum, or c > 0 for the truncated
 *            Gaussian, whose weight is zero unless |x_i - p_x| < c h and
 *            |y_i - p_y| < c h (a box of half-width c h around the pixel:
 *            every pair left out has weight below exp(-c^2) of the kernel's
 *            peak); its support count is the number of points in the box
 *   pix      npix pixel indices v*W+u (NULL: all W*H pixels in order)
 *   field    out, npix x D
 *   deg_used out, npix (-1: no point in support, value NaN)
 *   rcond    out, npix: rcond_1(Me) at the degree used (1 for degree 0,
 *            0 when no degree was usable)
 *   count    out, npix: points with positive weight under the rule above
 *   mstab    out, npix: m = min_i r_i^2 (0 for Wendland)
 *   amb      out, npix: bit 0 set when an rcond tested lay within a factor
 *            amb_factor of rcond_min; bit 1 set when a Wendland point lay
 *            within a relative amb_boundary of the support radius (or a
 *            truncated-Gaussian point's |dx| or |dy| within a relative
 *            amb_boundary of c h) and could move the count across a k
 *            threshold.  Optional (NULL).
 *   ecoef_sum, ecoef_fix  out, npix x D, optional (NULL): coefficients of a
 *            first-order bound on the rounding error of an FP64 evaluation
 *            of this pixel's value (a test aid: not part of the method).
 *            For any implementation that forms the same weights, basis
 *            terms and moments in this pixel frame, sums each moment in
 *            any order whose longest chain of additions has N terms, and
 *            solves through the explicit inverse of the equilibrated Me,
 *              |f_computed - f_exact| <= (N + 12) u ecoef_sum + ecoef_fix
 *            to first order in the unit roundoff u = 2^-53.  With
 *            y = M^{-1} e_0 and c = M^{-1} R (the value is f = y^T R, and
 *            the normal equations give df = y^T (dR - dM c)):
 *              ecoef_sum = sum_a |y_a| (T_ad + sum_b T_ab |c_bd|),
 *                T_ab = sum_i w_i |b_a b_b|, T_ad = sum_i w_i |b_a f_id|
 *                (the absolute sums that bound each moment's summation
 *                error, 12 u covering the rounding of each basis product);
 *              ecoef_fix = the same form with every w_i multiplied by the
 *                relative error bound of the computed weight (delta_w
 *                below), plus the error of the Cholesky solve Me z = e_0
 *                and the final sum: (3k+3) u s_0 g_0 sum_b |c_bd| / s_b +
 *                (k+3) u sum_c s_0 |z_c| s_c |R_cd|, s_a = M_aa^{-1/2},
 *                g_0 = |z|_1.
 *            0 where the value is NaN.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_mls(int64_t n, int32_t D, const double *xy, const double *F,
               int32_t degree, int32_t weight, double h, double alpha, double trunc,
               int32_t W, int32_t H, double x0, double y0, double x1, double y1,
               int64_t npix, const int64_t *pix, double rcond_min,
               double amb_factor, double amb_boundary,
               double *field, int8_t *deg_used, double *rcond_out,
               int64_t *count_out, double *mstab_out, uint8_t *amb,
               double *ecoef_sum, double *ecoef_fix, int32_t nthreads) {
    if (n < 1 || D < 1 || degree < 0 || degree > 2 || !(h > 0.0) || W < 1 || H < 1)
        return -1;
    if (weight != OR_GAUSS && weight != OR_WENDLAND && weight != OR_INVDIST) return -1;
    if (!(trunc >= 0.0) || (trunc > 0.0 && weight != OR_GAUSS)) return -1;
    if (pix == NULL) npix = (int64_t)W * H;
    const double sx = (x1 - x0) / (double)W;
    const double sy = (y1 - y0) / (double)H;
    const double rho_box = trunc * h;
    const double inv_s = 1.0 / h;
    const double h2 = h * h;
    const double rho2 = h * h;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *wt = (double *)malloc(sizeof(double) * (size_t)n);
        double *r2 = (double *)malloc(sizeof(double) * (size_t)n);
        double M[36], R6[6 * 256], Me[36], L[36], Minv[36], col[6];
        double *Rbuf = (D <= 256) ? R6 : (double *)malloc(sizeof(double) * 6 * (size_t)D);
        /* error-bound sums (ecoef_*): T, Tw (k x k), TR, TRw (k x D) */
        const int want_err = ecoef_sum != NULL && ecoef_fix != NULL;
        double T[36], Tw[36];
        double *TR = want_err ? (double *)malloc(sizeof(double) * 12 * (size_t)D) : NULL;
        double *TRw = want_err ? TR + 6 * (size_t)D : NULL;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t q = 0; q < npix; ++q) {
            const int64_t id = pix ? pix[q] : q;
            const int64_t u = id % W, v = id / W;
            const double px = pixel_centre(x0, sx, u);
            const double py = pixel_centre(y0, sy, v);
            double *out = field + q * D;

            /* squared distances and the stabiliser m = min r^2 */
            double m = INFINITY;
            for (int64_t i = 0; i < n; ++i) {
                const double dx = xy[2 * i] - px, dy = xy[2 * i + 1] - py;
                r2[i] = dx * dx + dy * dy;
                if (r2[i] < m) m = r2[i];
            }
            int64_t count = 0, nboundary = 0;
            int coincident = 0;
            for (int64_t i = 0; i < n; ++i) {
                double w;
                if (weight == OR_GAUSS) {
                    int in_box = 1;
                    if (trunc > 0.0) {
                        const double ax = fabs(xy[2 * i] - px), ay = fabs(xy[2 * i + 1] - py);
                        in_box = ax < rho_box && ay < rho_box;
                        if (fabs(ax / rho_box - 1.0) < amb_boundary || fabs(ay / rho_box - 1.0) < amb_boundary)
                            nboundary++;
                    }
                    if (in_box) {
                        w = exp(-(r2[i] - m) / h2);
                        count++;
                    } else {
                        w = 0.0;
                    }
                } else if (weight == OR_WENDLAND) {
                    const double qd = sqrt(r2[i]) / h;
                    if (r2[i] < rho2) {
                        const double t = 1.0 - qd;
                        w = t * t * t * t * (4.0 * qd + 1.0);
                        count++;
                    } else {
                        w = 0.0;
                    }
                    if (fabs(r2[i] / rho2 - 1.0) < amb_boundary) nboundary++;
                } else {
                    if (m == 0.0) {
                        w = (r2[i] == 0.0) ? 1.0 : 0.0;
                        coincident = 1;
                    } else {
                        w = pow(m / r2[i], alpha);
                    }
                    count++;
                }
                wt[i] = w;
            }
            if (mstab_out) mstab_out[q] = (weight == OR_WENDLAND) ? 0.0 : m;
            if (count_out) count_out[q] = count;
            uint8_t ambq = 0;

            int used = -1;
            double rc_used = 0.0;
            if (want_err)
                for (int d = 0; d < D; ++d) ecoef_sum[q * D + d] = ecoef_fix[q * D + d] = 0.0;
            if (coincident) {
                /* inverse distance, pixel centre on a data point: mean value */
                double sw = 0.0;
                for (int d = 0; d < D; ++d) out[d] = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    if (wt[i] == 0.0) continue;
                    sw += 1.0;
                    for (int d = 0; d < D; ++d) out[d] += F[i * D + d];
                }
                for (int d = 0; d < D; ++d) out[d] /= sw;
                used = 0;
                rc_used = 1.0;
                /* a plain mean: the sum of |f| over the points, per point */
                if (want_err)
                    for (int64_t i = 0; i < n; ++i)
                        if (wt[i] != 0.0)
                            for (int d = 0; d < D; ++d) ecoef_sum[q * D + d] += fabs(F[i * D + d]) / sw;
            } else {
                for (int deg = degree; deg >= 0 && used < 0; --deg) {
                    const int k = n_terms(deg);
                    if (nboundary > 0 &&
                        count - nboundary < k && k <= count + nboundary)
                        ambq |= 2;
                    if (count < k) continue;
                    memset(M, 0, sizeof(M));
                    memset(Rbuf, 0, sizeof(double) * (size_t)k * D);
                    if (want_err) {
                        memset(T, 0, sizeof(T));
                        memset(Tw, 0, sizeof(Tw));
                        memset(TR, 0, sizeof(double) * 12 * (size_t)D);
                    }
                    for (int64_t i = 0; i < n; ++i) {
                        const double w = wt[i];
                        if (w == 0.0) continue;
                        const double dx = (xy[2 * i] - px) * inv_s;
                        const double dy = (xy[2 * i + 1] - py) * inv_s;
                        double b[6];
                        for (int a = 0; a < k; ++a) b[a] = basis_term(a, dx, dy);
                        for (int a = 0; a < k; ++a) {
                            for (int c = 0; c < k; ++c) M[a * k + c] += w * b[a] * b[c];
                            for (int d = 0; d < D; ++d) Rbuf[a * D + d] += w * b[a] * F[i * D + d];
                        }
                        if (want_err) {
                            const double dw = weight_rel_error(weight, r2[i], m, h2, h, alpha) * 0x1p-53;
                            for (int a = 0; a < k; ++a) {
                                for (int c = 0; c < k; ++c) {
                                    const double t = w * fabs(b[a] * b[c]);
                                    T[a * k + c] += t;
                                    Tw[a * k + c] += dw * t;
                                }
                                for (int d = 0; d < D; ++d) {
                                    const double t = w * fabs(b[a] * F[i * D + d]);
                                    TR[a * D + d] += t;
                                    TRw[a * D + d] += dw * t;
                                }
                            }
                        }
                    }
                    /* equilibrate, factor, condition */
                    int ok = 1;
                    double sdiag[6];
                    for (int a = 0; a < k; ++a) {
                        if (!(M[a * k + a] > 0.0)) { ok = 0; break; }
                        sdiag[a] = 1.0 / sqrt(M[a * k + a]);
                    }
                    double rc = 0.0;
                    if (ok) {
                        for (int a = 0; a < k; ++a)
                            for (int c = 0; c < k; ++c) Me[a * k + c] = M[a * k + c] * sdiag[a] * sdiag[c];
                        if (cholesky(k, Me, L) != 0) ok = 0;
                    }
                    if (ok) {
                        for (int c = 0; c < k; ++c) {
                            for (int a = 0; a < k; ++a) col[a] = (a == c) ? 1.0 : 0.0;
                            chol_solve(k, L, col);
                            for (int a = 0; a < k; ++a) Minv[a * k + c] = col[a];
                        }
                        rc = 1.0 / (norm1(k, Me) * norm1(k, Minv));
                        if (rc >= rcond_min / amb_factor && rc <= rcond_min * amb_factor) ambq |= 1;
                        if (!(rc >= rcond_min)) ok = 0;
                    } else if (deg > 0) {
                        /* a failed factorisation is the singular end of the scale */
                        rc = 0.0;
                    }
                    if (!ok) continue;
                    /* f_d = row 0 of M^{-1} R = z^T R with z = M^{-1} e_0,
                     * M^{-1} = S Me^{-1} S: z is column 0 of the inverse,
                     * the one solve Me z' = e_0 (row 0 of the computed
                     * inverse is the same number in exact arithmetic, but
                     * gathers the rounding of every column's solve) */
                    for (int d = 0; d < D; ++d) {
                        double acc = 0.0;
                        for (int c = 0; c < k; ++c)
                            acc += sdiag[0] * Minv[c * k + 0] * sdiag[c] * Rbuf[c * D + d];
                        out[d] = acc;
                    }
                    used = deg;
                    rc_used = rc;
                    if (want_err) {
                        const double u53 = 0x1p-53;
                        double y[6], g[6];
                        for (int a = 0; a < k; ++a) {
                            y[a] = sdiag[a] * Minv[a * k + 0] * sdiag[0];
                            g[a] = 0.0;
                            for (int c = 0; c < k; ++c) g[a] += fabs(Minv[c * k + a]);
                        }
                        for (int d = 0; d < D; ++d) {
                            double cb[6], es = 0.0, ef = 0.0;
                            for (int b2 = 0; b2 < k; ++b2) {
                                cb[b2] = 0.0;
                                for (int c = 0; c < k; ++c)
                                    cb[b2] += sdiag[b2] * Minv[b2 * k + c] * sdiag[c] * Rbuf[c * D + d];
                            }
                            for (int a = 0; a < k; ++a) {
                                double ts = TR[a * D + d], tf = TRw[a * D + d];
                                for (int b2 = 0; b2 < k; ++b2) {
                                    ts += T[a * k + b2] * fabs(cb[b2]);
                                    tf += Tw[a * k + b2] * fabs(cb[b2]);
                                }
                                es += fabs(y[a]) * ts;
                                ef += fabs(y[a]) * tf;
                            }
                            /* the solve (Me + E) z = e_0, |E| <= (3k+3) u (Cholesky with
                             * unit-diagonal Me, and Me's own rounding), moves the value by
                             * s_0 z^T E Me^{-1} S R = s_0 z^T E (c_b / s_b)_b; the final
                             * sum of k products adds (k+3) u of its absolute terms */
                            double cs = 0.0;
                            for (int b2 = 0; b2 < k; ++b2) cs += fabs(cb[b2]) / sdiag[b2];
                            ef += (3.0 * k + 3.0) * u53 * sdiag[0] * g[0] * cs;
                            for (int c = 0; c < k; ++c)
                                ef += (k + 3.0) * u53 * sdiag[0] * fabs(Minv[c * k + 0]) * sdiag[c] * fabs(Rbuf[c * D + d]);
                            ecoef_sum[q * D + d] = es;
                            ecoef_fix[q * D + d] = ef;
                        }
                    }
                }
                if (used < 0)
                    for (int d = 0; d < D; ++d) out[d] = NAN;
            }
            if (deg_used) deg_used[q] = (int8_t)used;
            if (rcond_out) rcond_out[q] = rc_used;
            if (amb) amb[q] = ambq;
        }
        if (Rbuf != R6) free(Rbuf);
        free(TR);
        free(wt);
        free(r2);
    }
    return 0;
}

/*
 * Iso-band labels (Section 3.4, discrete colours): for each pixel and
 * dimension, the number of levels t_dj (ascending, D x L) with t_dj <= f_d;
 * 255 when f_d is NaN.  field and bands are npix x D.
 */
int oracle_bands(int64_t npix, int32_t D, const double *field, const double *levels,
                 int32_t L, uint8_t *bands) {
    if (npix < 0 || D < 1 || L < 0 || L > 254) return -1;
    for (int64_t q = 0; q < npix; ++q)
        for (int d = 0; d < D; ++d) {
            const double f = field[q * D + d];
            if (isnan(f)) { bands[q * D + d] = 255; continue; }
            int c = 0;
            for (int j = 0; j < L; ++j)
                if (levels[d * L + j] <= f) c++;
            bands[q * D + d] = (uint8_t)c;
        }
    return 0;
}

/* w_i of oracle_mls for one pair at offset (dx, dy) from the pixel centre
 * (Eq. eq-weights, the Wendland kernel, the truncated Gaussian's box;
 * m = min r^2 stabiliser). */
static double pair_weight(int32_t weight, double dx, double dy, double m, double h, double alpha,
                          double trunc) {
    const double r2 = dx * dx + dy * dy;
    if (weight == OR_GAUSS && trunc > 0.0 && !(fabs(dx) < trunc * h && fabs(dy) < trunc * h)) return 0.0;
    if (weight == OR_GAUSS) return exp(-(r2 - m) / (h * h));
    if (weight == OR_WENDLAND) {
        if (!(r2 < h * h)) return 0.0;
        const double qd = sqrt(r2) / h, t = 1.0 - qd;
        return t * t * t * t * (4.0 * qd + 1.0);
    }
    return pow(m / r2, alpha);
}

/*
 * The paper's other two MLS mappings of 2-D values (Section 3.3.1 Mean MLS,
 * Eq. eq-meanmls; Section 3.3.3 Rigid MLS, Eqs. eq-rigidmls and
 * eq-rigidmlspartial), for D = 2: the point values q_i are the original
 * positions, p_i = xy_i the distorted ones, v the pixel centre, with the
 * weights w_i of oracle_mls (same stabiliser, support and degenerate rules):
 *
 *   variant 1 (rigid):  p* = sum w p / sum w,  q* = sum w q / sum w,
 *     dp_i = p_i - p*, dq_i = q_i - q*, dv = v - p*,
 *     f'(v) = sum_i w_i dq_i [dp_i ; -dp_i^perp] [dv ; -dv^perp]^T
 *             (dq_i a row vector, the brackets 2 x 2 matrices with the
 *             given rows, (x, y)^perp = (-y, x)),
 *     f(v)  = |dv| f'(v) / |f'(v)| + q*;
 *   variant 2 (mean displacement):  f(v) = v + sum w (q - p) / sum w.
 *
 * The rigid form is dv turned by the rotation that best maps the dp_i onto
 * the dq_i under the weights.  Where that rotation is undetermined -- every
 * point of positive weight at one position (a single point in a Wendland
 * support, duplicates), or f'(v) = 0 -- no rotation is taken: f(v) = dv + q*,
 * the mean mapping.  (The paper's quotient is undefined there.)
 *
 * Inverse distance with points exactly at v: the mean of their q (point
 * identity, criterion 2 of Section 3.3).  No point in support: NaN.
 *
 * aux (NULL or npix x 4): q*_x, q*_y, |dv| and, for the rigid form, the
 * conditioning kappa = sum w |dp| |dq| / |mu| of the rotation, where
 * |mu| = |f'(v)| / |dv| is the size of the weighted cross moment that sets
 * the angle (kappa >= 1; INFINITY where the rotation is undetermined, 0 for
 * the mean form or dv = 0).  A relative error e in the moments turns the
 * result by about e kappa radians.
 */
int oracle_mls_variant(int64_t n, const double *xy, const double *Q, int32_t variant, int32_t weight,
                       double h, double alpha, double trunc, int32_t W, int32_t H, double x0, double y0, double x1,
                       double y1, int64_t npix, const int64_t *pix, double *field, double *aux,
                       int32_t nthreads) {
    if (n < 1 || (variant != 1 && variant != 2) || !(h > 0.0) || W < 1 || H < 1) return -1;
    if (weight != OR_GAUSS && weight != OR_WENDLAND && weight != OR_INVDIST) return -1;
    if (!(trunc >= 0.0) || (trunc > 0.0 && weight != OR_GAUSS)) return -1;
    if (pix == NULL) npix = (int64_t)W * H;
    const double sx = (x1 - x0) / (double)W;
    const double sy = (y1 - y0) / (double)H;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t q = 0; q < npix; ++q) {
        const int64_t id = pix ? pix[q] : q;
        const int64_t u = id % W, v = id / W;
        const double vx = pixel_centre(x0, sx, u);
        const double vy = pixel_centre(y0, sy, v);
        double *out = field + 2 * q;
        double *ax = aux ? aux + 4 * q : NULL;
        if (ax) ax[0] = ax[1] = ax[2] = ax[3] = NAN;
        double m = INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            const double dx = xy[2 * i] - vx, dy = xy[2 * i + 1] - vy;
            const double r2 = dx * dx + dy * dy;
            if (r2 < m) m = r2;
        }
        if (weight == OR_INVDIST && m == 0.0) {
            double sq[2] = {0.0, 0.0}, c = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                const double dx = xy[2 * i] - vx, dy = xy[2 * i + 1] - vy;
                if (dx * dx + dy * dy == 0.0) {
                    sq[0] += Q[2 * i];
                    sq[1] += Q[2 * i + 1];
                    c += 1.0;
                }
            }
            out[0] = sq[0] / c;
            out[1] = sq[1] / c;
            if (ax) {
                ax[0] = out[0];
                ax[1] = out[1];
                ax[2] = ax[3] = 0.0;
            }
            continue;
        }
        /* weights, weighted centroids; whether the support has two positions */
        double sw = 0.0, sp[2] = {0.0, 0.0}, sq[2] = {0.0, 0.0};
        int64_t first = -1;
        int spread = 0;
        for (int64_t i = 0; i < n; ++i) {
            const double dx = xy[2 * i] - vx, dy = xy[2 * i + 1] - vy;
            const double w = pair_weight(weight, dx, dy, m, h, alpha, trunc);
            if (!(w > 0.0)) continue;
            if (first < 0) first = i;
            else if (xy[2 * i] != xy[2 * first] || xy[2 * i + 1] != xy[2 * first + 1]) spread = 1;
            sw += w;
            sp[0] += w * xy[2 * i];
            sp[1] += w * xy[2 * i + 1];
            sq[0] += w * Q[2 * i];
            sq[1] += w * Q[2 * i + 1];
        }
        if (!(sw > 0.0)) {
            out[0] = out[1] = NAN;
            continue;
        }
        const double ps[2] = {sp[0] / sw, sp[1] / sw}, qs[2] = {sq[0] / sw, sq[1] / sw};
        const double dv[2] = {vx - ps[0], vy - ps[1]};
        const double ndv = sqrt(dv[0] * dv[0] + dv[1] * dv[1]);
        if (ax) {
            ax[0] = qs[0];
            ax[1] = qs[1];
            ax[2] = ndv;
            ax[3] = 0.0;
        }
        if (variant == 2) {
            /* v + sum w (q - p) / sum w */
            out[0] = vx + (sq[0] - sp[0]) / sw;
            out[1] = vy + (sq[1] - sp[1]) / sw;
            continue;
        }
        /* the 2 x 2 matrix [dv ; -dv^perp]^T, rows dv and -dv^perp = (dv_y, -dv_x) */
        const double Vm[2][2] = {{dv[0], dv[1]}, {dv[1], -dv[0]}};
        const double VT[2][2] = {{Vm[0][0], Vm[1][0]}, {Vm[0][1], Vm[1][1]}};
        double fp[2] = {0.0, 0.0}, spq = 0.0;
        for (int64_t i = 0; i < n && spread; ++i) {
            const double dx = xy[2 * i] - vx, dy = xy[2 * i + 1] - vy;
            const double w = pair_weight(weight, dx, dy, m, h, alpha, trunc);
            if (!(w > 0.0)) continue;
            const double dp[2] = {xy[2 * i] - ps[0], xy[2 * i + 1] - ps[1]};
            const double dq[2] = {Q[2 * i] - qs[0], Q[2 * i + 1] - qs[1]};
            /* [dp ; -dp^perp]: rows dp and (dp_y, -dp_x) */
            const double Pm[2][2] = {{dp[0], dp[1]}, {dp[1], -dp[0]}};
            /* row vector dq times Pm, then times VT */
            const double t0 = dq[0] * Pm[0][0] + dq[1] * Pm[1][0];
            const double t1 = dq[0] * Pm[0][1] + dq[1] * Pm[1][1];
            fp[0] += w * (t0 * VT[0][0] + t1 * VT[1][0]);
            fp[1] += w * (t0 * VT[0][1] + t1 * VT[1][1]);
            spq += w * sqrt(dp[0] * dp[0] + dp[1] * dp[1]) * sqrt(dq[0] * dq[0] + dq[1] * dq[1]);
        }
        const double nfp = sqrt(fp[0] * fp[0] + fp[1] * fp[1]);
        if (ndv == 0.0) {
            out[0] = qs[0];
            out[1] = qs[1];
        } else if (!spread || nfp == 0.0) {
            out[0] = dv[0] + qs[0];
            out[1] = dv[1] + qs[1];
            if (ax) ax[3] = INFINITY;
        } else {
            out[0] = ndv * fp[0] / nfp + qs[0];
            out[1] = ndv * fp[1] / nfp + qs[1];
            if (ax) ax[3] = spq * ndv / nfp;
        }
    }
    return 0;
}
