/*
 * FP64 CPU oracle for the long-range part of an Ewald sum.  TEST
 * INFRASTRUCTURE ONLY (like oracle.c): called by the tests, never by the CUDA
 * library, and sharing no code with it.
 *
 * The paper's short-range kernel computes the real-space Ewald term of
 * non-excluded pairs inside rc (Sec. V.A) and runs the reciprocal part (PME,
 * Sec. IV) as a separate task.  Together with the self and exclusion terms the
 * pieces make up the Ewald sum of a neutral periodic system (tin-foil boundary):
 *
 *   E = E_real + E_recip + E_self + E_excl
 *   E_recip = f/(2V) sum_{k != 0} (4 pi / k^2) exp(-k^2 / (4 beta^2)) |S(k)|^2,
 *             S(k) = sum_j q_j exp(i k.r_j),  k = 2 pi (n_x/L_x, n_y/L_y, n_z/L_z)
 *   E_self  = -f beta / sqrt(pi) sum_i q_i^2
 *   E_excl  = -f sum_{excluded pairs} q_i q_j erf(beta r_ij) / r_ij
 *             (removes the reciprocal-space interaction of pairs whose direct
 *              interaction is excluded; minimum-image distance)
 *   f = 138.935458 / eps_r
 *
 * Forces are -dE/dx.  Virial, in the convention W = -1/2 sum_pairs r (x) F of the
 * short-range part (W = 1/2 dE/d(strain)):
 *   W_recip,ab = -1/2 sum_{k != 0} e_k (delta_ab - 2 (1/k^2 + 1/(4 beta^2)) k_a k_b),
 *   e_k the term of E_recip for k;  W_excl = -1/2 sum r (x) F like any pair term.
 *
 * or_ewald_recip evaluates the k-space sum directly over |n_a| <= kmax_a (the
 * plain definition PME approximates); or_ewald_excl the exclusion correction;
 * or_ewald_self the self energy.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_F_COUL 138.935458

/* Direct reciprocal-space sum.  k vectors with |n_a| <= kmax_a, k != 0, taken
 * in the half space (n_x > 0, or n_x = 0 and n_y > 0, or n_x = n_y = 0 and
 * n_z > 0) and doubled, as the terms for k and -k are equal.
 * Outputs: F [n*3] forces (overwritten), E [1], W [9]. */
int or_ewald_recip(int n, const double *x, const double *q, const double *box, double beta, double eps_r,
                   int kmax_x, int kmax_y, int kmax_z, double *F, double *E, double *W) {
    if (n < 0 || beta <= 0.0 || kmax_x < 0 || kmax_y < 0 || kmax_z < 0) return 1;
    const double f = OR_F_COUL / eps_r;
    const double V = box[0] * box[1] * box[2];
    const double two_pi = 2.0 * M_PI;
    /* list of half-space k vectors */
    const int nx = kmax_x + 1, ny = 2 * kmax_y + 1, nz = 2 * kmax_z + 1;
    int64_t nk_max = (int64_t)nx * ny * nz;
    double *kv = (double *)malloc(sizeof(double) * 4 * (size_t)nk_max);  /* kx, ky, kz, A(k) */
    if (!kv) return 2;
    int64_t nk = 0;
    for (int a = 0; a <= kmax_x; a++)
        for (int b = -kmax_y; b <= kmax_y; b++)
            for (int c = -kmax_z; c <= kmax_z; c++) {
                if (a == 0 && (b < 0 || (b == 0 && c <= 0))) continue;
                const double kx = two_pi * a / box[0], ky = two_pi * b / box[1], kz = two_pi * c / box[2];
                const double k2 = kx * kx + ky * ky + kz * kz;
                kv[4 * nk] = kx;
                kv[4 * nk + 1] = ky;
                kv[4 * nk + 2] = kz;
                kv[4 * nk + 3] = 4.0 * M_PI / k2 * exp(-k2 / (4.0 * beta * beta));
                nk++;
            }
    double *S = (double *)calloc((size_t)(2 * nk > 0 ? 2 * nk : 1), sizeof(double)); /* Re, Im of S(k) */
    if (!S) {
        free(kv);
        return 2;
    }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nk; k++) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < n; j++) {
            const double ph = kv[4 * k] * x[3 * j] + kv[4 * k + 1] * x[3 * j + 1] + kv[4 * k + 2] * x[3 * j + 2];
            re += q[j] * cos(ph);
            im += q[j] * sin(ph);
        }
        S[2 * k] = re;
        S[2 * k + 1] = im;
    }
    double e = 0.0, w[9] = {0};
    for (int64_t k = 0; k < nk; k++) {
        const double kx = kv[4 * k], ky = kv[4 * k + 1], kz = kv[4 * k + 2], A = kv[4 * k + 3];
        const double s2 = S[2 * k] * S[2 * k] + S[2 * k + 1] * S[2 * k + 1];
        const double ek = 2.0 * f / (2.0 * V) * A * s2; /* doubled: k and -k */
        e += ek;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double g = 2.0 * (1.0 / k2 + 1.0 / (4.0 * beta * beta));
        const double kk[3] = {kx, ky, kz};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) w[3 * a + b] += -0.5 * ek * ((a == b ? 1.0 : 0.0) - g * kk[a] * kk[b]);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t k = 0; k < nk; k++) {
            const double kx = kv[4 * k], ky = kv[4 * k + 1], kz = kv[4 * k + 2];
            const double ph = kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2];
            /* Im(exp(i k.r_i) conj(S)) = sin(ph) Re S - cos(ph) Im S */
            const double t = kv[4 * k + 3] * (sin(ph) * S[2 * k] - cos(ph) * S[2 * k + 1]);
            fx += t * kx;
            fy += t * ky;
            fz += t * kz;
        }
        const double c = 2.0 * f * q[i] / V; /* doubled: k and -k */
        F[3 * i] = c * fx;
        F[3 * i + 1] = c * fy;
        F[3 * i + 2] = c * fz;
    }
    *E = e;
    memcpy(W, w, sizeof(w));
    free(S);
    free(kv);
    return 0;
}

/* Exclusion correction: every unordered excluded pair (CSR off [n+1], idx)
 * contributes V = -f qi qj erf(beta r)/r at its minimum-image distance.
 * F [n*3] forces (overwritten), E [1], W [9]. */
int or_ewald_excl(int n, const double *x, const double *q, const double *box, const int *off, const int *idx,
                  double beta, double eps_r, double *F, double *E, double *W) {
    if (n < 0 || beta <= 0.0) return 1;
    const double f = OR_F_COUL / eps_r;
    const double two_over_sqrt_pi = 2.0 / sqrt(M_PI);
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    double e = 0.0, w[9] = {0};
    for (int i = 0; i < n; i++) {
        for (int p = off[i]; p < off[i + 1]; p++) {
            const int j = idx[p];
            if (j <= i) continue;
            double d[3];
            for (int a = 0; a < 3; a++) {
                d[a] = x[3 * i + a] - x[3 * j + a];
                d[a] -= box[a] * round(d[a] / box[a]);
            }
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const double r = sqrt(r2);
            const double qq = f * q[i] * q[j];
            const double er = erf(beta * r);
            e += -qq * er / r;
            /* V = -qq erf(br)/r; dV/dr = -qq (2b/sqrt(pi) exp(-b^2 r^2)/r - erf(br)/r^2);
             * force on i = -(dV/dr) d/r */
            const double dvdr = -qq * (two_over_sqrt_pi * beta * exp(-beta * beta * r2) / r - er / r2);
            const double phi = -dvdr / r;
            for (int a = 0; a < 3; a++) {
                F[3 * i + a] += phi * d[a];
                F[3 * j + a] -= phi * d[a];
            }
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) w[3 * a + b] += -0.5 * d[a] * phi * d[b];
        }
    }
    *E = e;
    memcpy(W, w, sizeof(w));
    return 0;
}

/* Self energy -f beta/sqrt(pi) sum q_i^2. */
double or_ewald_self(int n, const double *q, double beta, double eps_r) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += q[i] * q[i];
    return -OR_F_COUL / eps_r * beta / sqrt(M_PI) * s;
}
