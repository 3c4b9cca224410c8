/*
 * Oracle: Rotne-Prager-Yamakawa mobility apply, plain FP64 C.
 *
 * TEST INFRASTRUCTURE. This file is the reference that the CUDA path is
 * checked against. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the library never does. It shares no code,
 * header or constant with the CUDA sources.
 *
 * What it computes (paper Sec. 2.7.1, "RPY mobility matrix"): for segments
 * with centres Y_n, forces F_m and torques T_m,
 *
 *     V_n     = sum_m  Mtt_nm F_m + Mtr_nm T_m
 *     Omega_n = sum_m  Mrt_nm F_m + Mrr_nm T_m
 *
 * over ALL ordered pairs (n, m), including n == m, with r = Y_n - Y_m,
 * rhat = r / |r|, (eps.rhat)_ij = eps_ijk rhat_k, and
 *
 *   n == m :  Mtt = I/(6 pi eta a),  Mrr = I/(8 pi eta a^3),  Mtr = Mrt = 0
 *   r >= 2a:  Mtt = [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) rhat rhat] / (8 pi eta r)
 *             Mrr = (3 rhat rhat - I) / (16 pi eta r^3)
 *             Mtr = Mrt = eps.rhat / (8 pi eta r^2)
 *
 * The paper prints only the r > 2a form and says that a variant for
 * overlapping spheres exists (it cites Wajnryb et al. 2013 for it). For
 * r < 2a, n != m, this oracle takes the equal-radius overlapping form of
 * that reference:
 *   Mtt = [(1 - 9r/(32a)) I + (3r/(32a)) rhat rhat] / (6 pi eta a)
 *   Mrr = [(1 - 27r/(32a) + 5r^3/(64a^3)) I
 *          + (9r/(32a) - 3r^3/(64a^3)) rhat rhat] / (8 pi eta a^3)
 *   Mtr = Mrt = (r/a)(1 - 3r/(8a)) eps.rhat / (16 pi eta a^2)
 * It meets the far form at r = 2a and the self term at r = 0. At r = 0 with
 * n != m the rhat-dependent parts carry a factor r and vanish, so rhat is
 * taken as 0 there.
 *
 * Also provided, for the mixed-precision error bound: the same sum with every
 * part of every block replaced by its absolute value (|alpha| I + |beta|
 * |rhat||rhat|^T, |gamma| |eps.rhat|) applied to (|F|, |T|).
 *
 * Layout: Y is S x 3 row-major, FT is S x 6 row-major (F then T), VW is S x 6
 * (V then Omega). Everything is FP64.
 */
#include <math.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Coefficients of one pair: Mtt = at I + bt rr, Mrr = ar I + br rr,
 * Mtr = Mrt = g eps.rhat. rhat is returned (0 at r = 0). */
static void pair_coefficients(const double d[3], int same, double a, double eta,
                              double *at, double *bt, double *ar, double *br,
                              double *g, double rhat[3])
{
    const double pi = ORACLE_PI;
    if (same) {
        *at = 1.0 / (6.0 * pi * eta * a);
        *bt = 0.0;
        *ar = 1.0 / (8.0 * pi * eta * a * a * a);
        *br = 0.0;
        *g = 0.0;
        rhat[0] = rhat[1] = rhat[2] = 0.0;
        return;
    }
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r > 0.0) {
        rhat[0] = d[0] / r;
        rhat[1] = d[1] / r;
        rhat[2] = d[2] / r;
    } else {
        rhat[0] = rhat[1] = rhat[2] = 0.0;
    }
    if (r >= 2.0 * a) {
        double c = 1.0 / (8.0 * pi * eta * r);
        *at = c * (1.0 + 2.0 * a * a / (3.0 * r * r));
        *bt = c * (1.0 - 2.0 * a * a / (r * r));
        double c3 = 1.0 / (16.0 * pi * eta * r * r * r);
        *ar = -c3;
        *br = 3.0 * c3;
        *g = 1.0 / (8.0 * pi * eta * r * r);
    } else {
        double ct = 1.0 / (6.0 * pi * eta * a);
        *at = ct * (1.0 - 9.0 * r / (32.0 * a));
        *bt = ct * (3.0 * r / (32.0 * a));
        double cr = 1.0 / (8.0 * pi * eta * a * a * a);
        double r3 = r * r * r, a3 = a * a * a;
        *ar = cr * (1.0 - 27.0 * r / (32.0 * a) + 5.0 * r3 / (64.0 * a3));
        *br = cr * (9.0 * r / (32.0 * a) - 3.0 * r3 / (64.0 * a3));
        *g = (r / a) * (1.0 - 3.0 * r / (8.0 * a)) / (16.0 * pi * eta * a * a);
    }
}

/* The four 3x3 blocks of one pair, row-major. same != 0 means n == m. */
void oracle_rpy_pair_blocks(const double d[3], int same, double a, double eta,
                            double Mtt[9], double Mtr[9], double Mrt[9], double Mrr[9])
{
    double at, bt, ar, br, g, e[3];
    pair_coefficients(d, same, a, eta, &at, &bt, &ar, &br, &g, e);
    /* eps.rhat with (eps.rhat)_ij = eps_ijk rhat_k */
    double E[9] = {0.0, e[2], -e[1],
                   -e[2], 0.0, e[0],
                   e[1], -e[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double dd = e[i] * e[j];
            double id = (i == j) ? 1.0 : 0.0;
            Mtt[3 * i + j] = at * id + bt * dd;
            Mrr[3 * i + j] = ar * id + br * dd;
            Mtr[3 * i + j] = g * E[3 * i + j];
            Mrt[3 * i + j] = g * E[3 * i + j];
        }
}

/* One target row n: VW_n = sum_m M_nm FT_m (and the magnitude sum if absout). */
static void target_row(int S, const double *Y, const double *FT, double a, double eta,
                       int n, double *out, double *absout)
{
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double aba[6] = {0, 0, 0, 0, 0, 0};
    for (int m = 0; m < S; ++m) {
        double d[3] = {Y[3 * n] - Y[3 * m], Y[3 * n + 1] - Y[3 * m + 1],
                       Y[3 * n + 2] - Y[3 * m + 2]};
        double Mtt[9], Mtr[9], Mrt[9], Mrr[9];
        oracle_rpy_pair_blocks(d, n == m, a, eta, Mtt, Mtr, Mrt, Mrr);
        const double *F = FT + 6 * m, *T = FT + 6 * m + 3;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                acc[i] += Mtt[3 * i + j] * F[j] + Mtr[3 * i + j] * T[j];
                acc[3 + i] += Mrt[3 * i + j] * F[j] + Mrr[3 * i + j] * T[j];
            }
        if (absout) {
            double at, bt, ar, br, g, e[3];
            pair_coefficients(d, n == m, a, eta, &at, &bt, &ar, &br, &g, e);
            double aE[9] = {0.0, fabs(e[2]), fabs(e[1]),
                            fabs(e[2]), 0.0, fabs(e[0]),
                            fabs(e[1]), fabs(e[0]), 0.0};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double id = (i == j) ? 1.0 : 0.0;
                    double dd = fabs(e[i] * e[j]);
                    aba[i] += (fabs(at) * id + fabs(bt) * dd) * fabs(F[j])
                              + fabs(g) * aE[3 * i + j] * fabs(T[j]);
                    aba[3 + i] += fabs(g) * aE[3 * i + j] * fabs(F[j])
                                  + (fabs(ar) * id + fabs(br) * dd) * fabs(T[j]);
                }
        }
    }
    for (int i = 0; i < 6; ++i) out[i] = acc[i];
    if (absout)
        for (int i = 0; i < 6; ++i) absout[i] = aba[i];
}

/* Full apply: VW (S x 6) = M(Y) FT. absVW may be NULL. nthreads <= 1: serial. */
void oracle_rpy_apply(int S, const double *Y, const double *FT, double a, double eta,
                      double *VW, double *absVW, int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int n = 0; n < S; ++n)
        target_row(S, Y, FT, a, eta, n, VW + 6 * (size_t)n,
                   absVW ? absVW + 6 * (size_t)n : NULL);
    (void)nthreads;
}

/* Selected rows only: out[k] = row rows[k] of the apply (k < nrows). */
void oracle_rpy_apply_rows(int S, const double *Y, const double *FT, double a, double eta,
                           int nrows, const int *rows, double *VW_rows, double *absVW_rows,
                           int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int k = 0; k < nrows; ++k)
        target_row(S, Y, FT, a, eta, rows[k], VW_rows + 6 * (size_t)k,
                   absVW_rows ? absVW_rows + 6 * (size_t)k : NULL);
    (void)nthreads;
}
