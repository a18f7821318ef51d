/*
 * Plain FP64 CPU oracle for the community integration algorithm (CIA).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the CUDA
 * library; the product path never links, loads or calls it.  It shares no code,
 * header, table or constant with the device path.
 *
 * Every function below writes out either the plain definition of a right-hand
 * side (the "direct" sums) or the paper's CIA steps in the paper's order:
 *   (E1) per-community observables, then the dense term from them,
 *   (E2) the sparse sum over S (entries +1 / -1), then f_m added.
 * All loops are sequential per output value; OpenMP only distributes whole
 * output values over threads, so results do not depend on the thread count.
 *
 * Indexing conventions: CSR rows are nodes; the CIA functions work on the
 * permuted state phi_m = theta_{kappa(m)} (Sec. 3.1, step P1), where the
 * communities are the contiguous ranges [off[c], off[c+1]).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* h(x) = sum_{k=1..p} d_sin[k-1] sin(kx) + d_cos[k-1] cos(kx)
 * (higher-harmonics Kuramoto coupling, App. A.4; p = 1, d_sin = 1 is the
 * classical sine coupling of Table tab:NetworkExamples). */
static double coupling_h(double x, int p, const double *d_sin, const double *d_cos) {
    double s = 0.0;
    for (int k = 1; k <= p; ++k)
        s += d_sin[k - 1] * sin(k * x) + d_cos[k - 1] * cos(k * x);
    return s;
}

/* Direct RHS of the phase-oscillator network, eq. GeneralNetworkSystem (Sec. 2) with f_m = omega_m and
 * g(x_l, x_m) = K h(x_l - x_m):
 *   out_m = omega_m + (K/N) sum_l a_ml h(theta_l - theta_m).
 * The sum runs over the CSR neighbours of m (a_ml in {0,1}). */
void ora_kuramoto_direct(int64_t n, const int64_t *rowptr, const int32_t *col,
                         const double *theta, const double *omega, double K,
                         int p, const double *d_sin, const double *d_cos,
                         double *out) {
    const double scale = K / (double)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int64_t e = rowptr[m]; e < rowptr[m + 1]; ++e)
            acc += coupling_h(theta[col[e]] - theta[m], p, d_sin, d_cos);
        out[m] = omega[m] + scale * acc;
    }
}

/* CIA RHS of the phase-oscillator network, Sec. 3.2 (steps E1, E2) and App. A.4.
 *
 * phi, omega: permuted order.  Communities c = 0..M-1 occupy
 * [off[c], off[c+1]); nodes in [off[M], n) belong to no community.
 * S is the sparse remainder of B = D + S in CSR form with values +1
 * (extra inter-community link) or -1 (missing link inside a community block,
 * including the diagonal, since b_mm = 0 while d_mm = 1).
 *
 * (E1.1) q_cos[c][k] = (1/N) sum_{l in c} cos(k phi_l),
 *        q_sin[c][k] = (1/N) sum_{l in c} sin(k phi_l)          (eq. PrecomputeQuantities)
 * (E1.2) dense_m = sum_k d_sin_k (q_sin cos k phi_m - q_cos sin k phi_m)
 *                      + d_cos_k (q_sin sin k phi_m + q_cos cos k phi_m)
 *        (eq. FastHdense, in the d_sin/d_cos form of App. A.4; d_0 = 0)
 * (E2)   sparse_m = (1/N) sum_l s_ml h(phi_l - phi_m)
 * out_m = omega_m + K (dense_m + sparse_m).
 *
 * q_cos, q_sin: caller-provided scratch of M * p doubles each. */
void ora_kuramoto_cia(int64_t n, int64_t M, const int64_t *off,
                      const int64_t *s_rowptr, const int32_t *s_col, const int8_t *s_val,
                      const double *phi, const double *omega, double K,
                      int p, const double *d_sin, const double *d_cos,
                      double *q_cos, double *q_sin, double *out) {
    const double invN = 1.0 / (double)n;
    /* (E1.1) observables, one community per iteration, sequential sum */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < M; ++c) {
        for (int k = 1; k <= p; ++k) {
            double sc = 0.0, ss = 0.0;
            for (int64_t l = off[c]; l < off[c + 1]; ++l) {
                sc += cos(k * phi[l]);
                ss += sin(k * phi[l]);
            }
            q_cos[c * p + (k - 1)] = invN * sc;
            q_sin[c * p + (k - 1)] = invN * ss;
        }
    }
    /* (E1.2) dense term from the observables, (E2) sparse sum, then f_m */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        double dense = 0.0;
        int64_t c = -1;
        /* community of m: the unique c with off[c] <= m < off[c+1] */
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid; else hi = mid;
            }
            c = lo;
        }
        if (c >= 0) {
            for (int k = 1; k <= p; ++k) {
                double qc = q_cos[c * p + (k - 1)], qs = q_sin[c * p + (k - 1)];
                double ck = cos(k * phi[m]), sk = sin(k * phi[m]);
                dense += d_sin[k - 1] * (qs * ck - qc * sk)
                       + d_cos[k - 1] * (qs * sk + qc * ck);
            }
        }
        double sparse = 0.0;
        for (int64_t e = s_rowptr[m]; e < s_rowptr[m + 1]; ++e)
            sparse += (double)s_val[e] * coupling_h(phi[s_col[e]] - phi[m], p, d_sin, d_cos);
        out[m] = omega[m] + K * (dense + invN * sparse);
    }
}

/* Triadic term of the higher-order Kuramoto model on complete community
 * hyperedges (App. A.7, eq. HOKuramoto with n = 2, lambda = (1, 1, -2)), written as the plain
 * sum over ordered pairs of distinct community members other than m:
 *   T_m = (K2/N^2) sum_{j != k, j,k in c(m) \ {m}} sin(phi_j + phi_k - 2 phi_m).
 * Evaluated only for the `count` permuted node ids in `nodes` (O(lambda^2)
 * each); nodes outside every community get 0. */
void ora_ho_triadic_direct(int64_t n, int64_t M, const int64_t *off, const double *phi,
                           double K2, int64_t count, const int64_t *nodes, double *out) {
    const double scale = K2 / ((double)n * (double)n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < count; ++i) {
        int64_t m = nodes[i];
        int64_t c = -1;
        for (int64_t cc = 0; cc < M; ++cc)
            if (off[cc] <= m && m < off[cc + 1]) { c = cc; break; }
        double acc = 0.0;
        if (c >= 0) {
            for (int64_t j = off[c]; j < off[c + 1]; ++j) {
                if (j == m) continue;
                for (int64_t k = off[c]; k < off[c + 1]; ++k) {
                    if (k == m || k == j) continue;
                    acc += sin(phi[j] + phi[k] - 2.0 * phi[m]);
                }
            }
        }
        out[i] = scale * acc;
    }
}

/* Triadic term from community moments, eq. HOKuramoto_fastRHS (App. A.7) adapted to the community
 * hyperedges: with Z1 = sum_{l in c} e^{i phi_l}, Z2 = sum_{l in c} e^{2 i phi_l},
 * the ordered pairs j != k of members other than m sum to
 *   (Z1 - e^{i phi_m})^2 - (Z2 - e^{2 i phi_m}),
 * so T_m = (K2/N^2) Im( [ (Z1 - e^{i phi_m})^2 - (Z2 - e^{2 i phi_m}) ] e^{-2 i phi_m} ).
 * z1re.. : caller scratch of M doubles each. */
void ora_ho_triadic_cia(int64_t n, int64_t M, const int64_t *off, const double *phi,
                        double K2, double *z1re, double *z1im, double *z2re, double *z2im,
                        double *out) {
    const double scale = K2 / ((double)n * (double)n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < M; ++c) {
        double a = 0.0, b = 0.0, e = 0.0, f = 0.0;
        for (int64_t l = off[c]; l < off[c + 1]; ++l) {
            a += cos(phi[l]); b += sin(phi[l]);
            e += cos(2.0 * phi[l]); f += sin(2.0 * phi[l]);
        }
        z1re[c] = a; z1im[c] = b; z2re[c] = e; z2im[c] = f;
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        int64_t c = -1;
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid; else hi = mid;
            }
            c = lo;
        }
        if (c < 0) { out[m] = 0.0; continue; }
        /* u = Z1 - e^{i phi_m}, w = Z2 - e^{2 i phi_m} */
        double ure = z1re[c] - cos(phi[m]), uim = z1im[c] - sin(phi[m]);
        double wre = z2re[c] - cos(2.0 * phi[m]), wim = z2im[c] - sin(2.0 * phi[m]);
        /* q = u^2 - w */
        double qre = ure * ure - uim * uim - wre;
        double qim = 2.0 * ure * uim - wim;
        /* Im(q e^{-2 i phi_m}) = qim cos(2phi) - qre sin(2phi) */
        out[m] = scale * (qim * cos(2.0 * phi[m]) - qre * sin(2.0 * phi[m]));
    }
}

/* Cucker-Smale interaction weight eta(||s_l - s_m||^2) = K (sigma^2 + r^2)^(-beta)
 * (eq. Cucker_Smale, App. A.6). */
static double cs_weight(double dx, double dy, double K, double sigma, double beta) {
    return K * pow(sigma * sigma + dx * dx + dy * dy, -beta);
}

/* Direct Cucker-Smale RHS in the plane (eq. Cucker_Smale, App. A.6, n = 2):
 *   s_m' = v_m,
 *   v_m' = (1/N) sum_l a_ml eta(||s_l - s_m||^2) (v_l - v_m).
 * x: n x 4 rows (s_x, s_y, v_x, v_y); out: same layout. */
void ora_cs_direct(int64_t n, const int64_t *rowptr, const int32_t *col, const double *x,
                   double K, double sigma, double beta, double *out) {
    const double invN = 1.0 / (double)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        const double *xm = x + 4 * m;
        double ax = 0.0, ay = 0.0;
        for (int64_t e = rowptr[m]; e < rowptr[m + 1]; ++e) {
            const double *xl = x + 4 * (int64_t)col[e];
            double w = cs_weight(xl[0] - xm[0], xl[1] - xm[1], K, sigma, beta);
            ax += w * (xl[2] - xm[2]);
            ay += w * (xl[3] - xm[3]);
        }
        out[4 * m + 0] = xm[2];
        out[4 * m + 1] = xm[3];
        out[4 * m + 2] = invN * ax;
        out[4 * m + 3] = invN * ay;
    }
}

/* CIA Cucker-Smale RHS with a separable weight eta(||s_l - s_m||^2) ~
 * sum_r phi_r(l) phi_r(m) (the step-P2 basis: the paper's Fourier modes, or a
 * learned feature map), following eqs. Cucker_Smale_orderParams and Cucker_Smale_fast_RHS with the
 * basis in place
 * of e^{i pi <alpha, s>/L}:
 * (E1.1) U[c][r] = (1/N) sum_{l in c} phi_r(l),
 *        H[c][r] = (1/N) sum_{l in c} phi_r(l) v_l           (eq. Cucker_Smale_orderParams)
 * (E1.2) dense_m = sum_r phi_r(m) (H[c][r] - U[c][r] v_m)     (eq. Cucker_Smale_fast_RHS)
 * (E2)   sparse_m = (1/N) sum_l s_ml eta_exact(l, m) (v_l - v_m)
 * Positions: s_m' = v_m.
 * feat: n x R (permuted order, row m = phi(m)); x: n x 4 permuted.
 * U, H: caller scratch of M*R and M*R*2 doubles. */
void ora_cs_cia(int64_t n, int64_t M, const int64_t *off,
                const int64_t *s_rowptr, const int32_t *s_col, const int8_t *s_val,
                const double *x, const double *feat, int64_t R,
                double K, double sigma, double beta,
                double *U, double *H, double *out) {
    const double invN = 1.0 / (double)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < M; ++c) {
        for (int64_t r = 0; r < R; ++r) {
            double u = 0.0, hx = 0.0, hy = 0.0;
            for (int64_t l = off[c]; l < off[c + 1]; ++l) {
                double ph = feat[l * R + r];
                u += ph;
                hx += ph * x[4 * l + 2];
                hy += ph * x[4 * l + 3];
            }
            U[c * R + r] = invN * u;
            H[(c * R + r) * 2 + 0] = invN * hx;
            H[(c * R + r) * 2 + 1] = invN * hy;
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        const double *xm = x + 4 * m;
        int64_t c = -1;
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid; else hi = mid;
            }
            c = lo;
        }
        double dx = 0.0, dy = 0.0;
        if (c >= 0) {
            for (int64_t r = 0; r < R; ++r) {
                double ph = feat[m * R + r];
                dx += ph * (H[(c * R + r) * 2 + 0] - U[c * R + r] * xm[2]);
                dy += ph * (H[(c * R + r) * 2 + 1] - U[c * R + r] * xm[3]);
            }
        }
        double sx = 0.0, sy = 0.0;
        for (int64_t e = s_rowptr[m]; e < s_rowptr[m + 1]; ++e) {
            const double *xl = x + 4 * (int64_t)s_col[e];
            double w = (double)s_val[e] * cs_weight(xl[0] - xm[0], xl[1] - xm[1], K, sigma, beta);
            sx += w * (xl[2] - xm[2]);
            sy += w * (xl[3] - xm[3]);
        }
        out[4 * m + 0] = xm[2];
        out[4 * m + 1] = xm[3];
        out[4 * m + 2] = dx + invN * sx;
        out[4 * m + 3] = dy + invN * sy;
    }
}

/* ---- polynomial difference coupling with a potential --------------------
 * x_m' = -V'(x_m) + (K/N) sum_l a_ml h(x_l - x_m)
 * (eq. GeneralNetworkPolyDifference, App. A.3, with the potential term of the
 * Desai-Zwanzig model, eq. DesaiZwanzig, App. A.5), where
 *   h(x)  = sum_{a=0..p} c[a] x^a,   V'(x) = sum_{j=0..q} dv[j] x^j.
 * Desai-Zwanzig: p = 1, c = (0, 1). */
static double poly_eval(const double *c, int p, double x) {
    double s = 0.0;
    for (int a = p; a >= 0; --a) s = s * x + c[a];
    return s;
}

/* Direct RHS: the CSR neighbours of m one by one. */
void ora_poly_direct(int64_t n, const int64_t *rowptr, const int32_t *col, const double *x, double K,
                     int p, const double *c, int q, const double *dv, double *out) {
    const double scale = K / (double)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int64_t e = rowptr[m]; e < rowptr[m + 1]; ++e) acc += poly_eval(c, p, x[col[e]] - x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + scale * acc;
    }
}

/* CIA RHS in the paper's steps (permuted state, communities [off[c], off[c+1]),
 * S with values +1 / -1 including the diagonal -1 of every community node):
 * (E1.1) w[c][k] = (1/N) sum_{l in c} x_l^k, k = 0..p            (eq. PolyMoments)
 * (E1.2) dense_m = sum_a c_a sum_{k=0..a} binom(a, k) w[c][k] (-x_m)^{a-k}
 *                                                               (eq. PolyDifferenceRHSfast)
 * (E2)   sparse_m = (1/N) sum_l s_ml h(x_l - x_m)
 *        out_m = -V'(x_m) + K (dense_m + sparse_m).
 * w: caller scratch of M * (p + 1) doubles. */
void ora_poly_cia(int64_t n, int64_t M, const int64_t *off, const int64_t *s_rowptr, const int32_t *s_col,
                  const int8_t *s_val, const double *x, double K, int p, const double *c, int q,
                  const double *dv, double *w, double *out) {
    const double invN = 1.0 / (double)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t cc = 0; cc < M; ++cc) {
        for (int k = 0; k <= p; ++k) {
            double s = 0.0;
            for (int64_t l = off[cc]; l < off[cc + 1]; ++l) s += pow(x[l], (double)k);
            w[cc * (p + 1) + k] = invN * s;
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        int64_t cc = -1;
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid;
                else hi = mid;
            }
            cc = lo;
        }
        double dense = 0.0;
        if (cc >= 0) {
            for (int a = 0; a <= p; ++a) {
                double inner = 0.0, binom = 1.0;
                for (int k = 0; k <= a; ++k) {
                    inner += binom * w[cc * (p + 1) + k] * pow(-x[m], (double)(a - k));
                    binom = binom * (double)(a - k) / (double)(k + 1);
                }
                dense += c[a] * inner;
            }
        }
        double sparse = 0.0;
        for (int64_t e = s_rowptr[m]; e < s_rowptr[m + 1]; ++e)
            sparse += (double)s_val[e] * poly_eval(c, p, x[s_col[e]] - x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + K * (dense + invN * sparse);
    }
}

/* ------------------------------------------------------------------------
 * General polynomial coupling (Sec. "General Network Model - Polynomial
 * Expansion", eq. PolyApprox, eq. PolyMoments, eq. PolyRHS):
 *   x_m' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m),
 *   g(u, y) = sum_{a=0..p} sum_{b=0..p} G[a][b] u^a y^b   (u: the neighbour),
 * G row-major with p + 1 columns. */
static double poly2_eval(const double *G, int p, double u, double y) {
    double s = 0.0;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p; ++b) s += G[a * (p + 1) + b] * pow(u, (double)a) * pow(y, (double)b);
    return s;
}

/* Direct RHS: the CSR neighbours of m one by one. */
void ora_polyg_direct(int64_t n, const int64_t *rowptr, const int32_t *col, const double *x, double K,
                      int p, const double *G, int q, const double *dv, double *out) {
    const double scale = K / (double)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int64_t e = rowptr[m]; e < rowptr[m + 1]; ++e) acc += poly2_eval(G, p, x[col[e]], x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + scale * acc;
    }
}

/* CIA RHS (permuted state, S with its diagonal -1 entries):
 * (E1.1) w[c][a] = (1/N) sum_{l in c} x_l^a, a = 0..p          (eq. PolyMoments)
 * (E1.2) dense_m = sum_a sum_b G[a][b] w[c][a] x_m^b            (eq. PolyRHS)
 * (E2)   sparse_m = (1/N) sum_l s_ml g(x_l, x_m)
 *        out_m = -V'(x_m) + K (dense_m + sparse_m).
 * w: caller scratch of M * (p + 1) doubles. */
void ora_polyg_cia(int64_t n, int64_t M, const int64_t *off, const int64_t *s_rowptr, const int32_t *s_col,
                   const int8_t *s_val, const double *x, double K, int p, const double *G, int q,
                   const double *dv, double *w, double *out) {
    const double invN = 1.0 / (double)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t cc = 0; cc < M; ++cc) {
        for (int a = 0; a <= p; ++a) {
            double s = 0.0;
            for (int64_t l = off[cc]; l < off[cc + 1]; ++l) s += pow(x[l], (double)a);
            w[cc * (p + 1) + a] = invN * s;
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        int64_t cc = -1;
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid;
                else hi = mid;
            }
            cc = lo;
        }
        double dense = 0.0;
        if (cc >= 0)
            for (int a = 0; a <= p; ++a)
                for (int b = 0; b <= p; ++b)
                    dense += G[a * (p + 1) + b] * w[cc * (p + 1) + a] * pow(x[m], (double)b);
        double sparse = 0.0;
        for (int64_t e = s_rowptr[m]; e < s_rowptr[m + 1]; ++e)
            sparse += (double)s_val[e] * poly2_eval(G, p, x[s_col[e]], x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + K * (dense + invN * sparse);
    }
}

/* ------------------------------------------------------------------------
 * Rank-one weighted couplings (Sec. "Rank One Coupling", eq. rank1system,
 * eq. rank1precompute, eq. rank1fast) on a graph: the weights of the links
 * factor as a_ml alpha_m beta_l,
 *   x_m' = -V'(x_m) + (K/N) sum_l a_ml alpha_m beta_l g(x_l, x_m),
 * with the general polynomial g of eq. PolyApprox (G as above). */
void ora_polyw_direct(int64_t n, const int64_t *rowptr, const int32_t *col, const double *x, double K,
                      int p, const double *G, int q, const double *dv, const double *alpha,
                      const double *beta, double *out) {
    const double scale = K / (double)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int64_t e = rowptr[m]; e < rowptr[m + 1]; ++e)
            acc += alpha[m] * beta[col[e]] * poly2_eval(G, p, x[col[e]], x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + scale * acc;
    }
}

/* CIA RHS (permuted state and weights, S with its diagonal -1 entries):
 * (E1.1) r[c][a] = (1/N) sum_{l in c} beta_l x_l^a, a = 0..p   (eq. rank1precompute,
 *        one weighted moment per power as in eq. PolyMoments)
 * (E1.2) dense_m = alpha_m sum_a sum_b G[a][b] r[c][a] x_m^b     (eq. rank1fast with eq. PolyRHS)
 * (E2)   sparse_m = (1/N) sum_l s_ml alpha_m beta_l g(x_l, x_m)
 *        out_m = -V'(x_m) + K (dense_m + sparse_m).
 * w: caller scratch of M * (p + 1) doubles. */
void ora_polyw_cia(int64_t n, int64_t M, const int64_t *off, const int64_t *s_rowptr, const int32_t *s_col,
                   const int8_t *s_val, const double *x, double K, int p, const double *G, int q,
                   const double *dv, const double *alpha, const double *beta, double *w, double *out) {
    const double invN = 1.0 / (double)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t cc = 0; cc < M; ++cc) {
        for (int a = 0; a <= p; ++a) {
            double s = 0.0;
            for (int64_t l = off[cc]; l < off[cc + 1]; ++l) s += beta[l] * pow(x[l], (double)a);
            w[cc * (p + 1) + a] = invN * s;
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        int64_t cc = -1;
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid;
                else hi = mid;
            }
            cc = lo;
        }
        double dense = 0.0;
        if (cc >= 0)
            for (int a = 0; a <= p; ++a)
                for (int b = 0; b <= p; ++b)
                    dense += G[a * (p + 1) + b] * w[cc * (p + 1) + a] * pow(x[m], (double)b);
        dense *= alpha[m];
        double sparse = 0.0;
        for (int64_t e = s_rowptr[m]; e < s_rowptr[m + 1]; ++e)
            sparse += (double)s_val[e] * alpha[m] * beta[s_col[e]] * poly2_eval(G, p, x[s_col[e]], x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + K * (dense + invN * sparse);
    }
}

/* ------------------------------------------------------------------------
 * General coupling by a real 2-D Fourier series (Sec. "Real Fourier Series",
 * eq. FourierRealExpansion, eq. RealOP):
 *   x_m' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m),
 *   g(u, y) = sum_{a,b=0..p} C11[a][b] cos(a w u) cos(b w y) + C12[a][b] cos(a w u) sin(b w y)
 *                          + C21[a][b] sin(a w u) cos(b w y) + C22[a][b] sin(a w u) sin(b w y),
 * w = pi / L, each C row-major with p + 1 columns. */
static double fourier2_eval(const double *C11, const double *C12, const double *C21, const double *C22,
                            int p, double w, double u, double y) {
    double s = 0.0;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p; ++b) {
            const double cu = cos(a * w * u), su = sin(a * w * u);
            const double cy = cos(b * w * y), sy = sin(b * w * y);
            const int i = a * (p + 1) + b;
            s += C11[i] * cu * cy + C12[i] * cu * sy + C21[i] * su * cy + C22[i] * su * sy;
        }
    return s;
}

/* Direct RHS: g link by link. */
void ora_fourierg_direct(int64_t n, const int64_t *rowptr, const int32_t *col, const double *x, double K,
                         int p, double L, const double *C11, const double *C12, const double *C21,
                         const double *C22, int q, const double *dv, double *out) {
    const double scale = K / (double)n, w = 3.14159265358979323846 / L;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int64_t e = rowptr[m]; e < rowptr[m + 1]; ++e)
            acc += fourier2_eval(C11, C12, C21, C22, p, w, x[col[e]], x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + scale * acc;
    }
}

/* CIA RHS (permuted state, S with its diagonal -1 entries):
 * (E1.1) rc[c][a] = (1/N) sum_{l in c} cos(a w x_l), rs[c][a] = (1/N) sum_{l in c} sin(a w x_l),
 *        a = 0..p                                                  (eq. RealOP)
 * (E1.2) dense_m = sum_{a,b} C11 rc_a cos(b w x_m) + C12 rc_a sin(b w x_m)
 *                          + C21 rs_a cos(b w x_m) + C22 rs_a sin(b w x_m)
 * (E2)   sparse_m = (1/N) sum_l s_ml g(x_l, x_m)
 *        out_m = -V'(x_m) + K (dense_m + sparse_m).
 * w: caller scratch of 2 M (p + 1) doubles. */
void ora_fourierg_cia(int64_t n, int64_t M, const int64_t *off, const int64_t *s_rowptr, const int32_t *s_col,
                      const int8_t *s_val, const double *x, double K, int p, double L, const double *C11,
                      const double *C12, const double *C21, const double *C22, int q, const double *dv,
                      double *wbuf, double *out) {
    const double invN = 1.0 / (double)n, w = 3.14159265358979323846 / L;
    double *rc = wbuf, *rs = wbuf + M * (p + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t cc = 0; cc < M; ++cc) {
        for (int a = 0; a <= p; ++a) {
            double sc = 0.0, ss = 0.0;
            for (int64_t l = off[cc]; l < off[cc + 1]; ++l) {
                sc += cos(a * w * x[l]);
                ss += sin(a * w * x[l]);
            }
            rc[cc * (p + 1) + a] = invN * sc;
            rs[cc * (p + 1) + a] = invN * ss;
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t m = 0; m < n; ++m) {
        int64_t cc = -1;
        if (m < off[M]) {
            int64_t lo = 0, hi = M;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) / 2;
                if (off[mid] <= m) lo = mid;
                else hi = mid;
            }
            cc = lo;
        }
        double dense = 0.0;
        if (cc >= 0)
            for (int a = 0; a <= p; ++a)
                for (int b = 0; b <= p; ++b) {
                    const int i = a * (p + 1) + b;
                    const double ca = rc[cc * (p + 1) + a], sa = rs[cc * (p + 1) + a];
                    const double cy = cos(b * w * x[m]), sy = sin(b * w * x[m]);
                    dense += C11[i] * ca * cy + C12[i] * ca * sy + C21[i] * sa * cy + C22[i] * sa * sy;
                }
        double sparse = 0.0;
        for (int64_t e = s_rowptr[m]; e < s_rowptr[m + 1]; ++e)
            sparse += (double)s_val[e] * fourier2_eval(C11, C12, C21, C22, p, w, x[s_col[e]], x[m]);
        out[m] = -poly_eval(dv, q, x[m]) + K * (dense + invN * sparse);
    }
}
