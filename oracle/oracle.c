/*
 * FP64 CPU oracle for the short-range non-bonded interactions of the cluster
 * pair method.  TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and
 * the benchmark's CPU-baseline leg call it; the CUDA library never does, and
 * this file shares no code, header, table or constant with the CUDA path.
 *
 * What it computes is the plain definition the cluster algorithm reproduces
 * exactly (Sec. V.A: every non-excluded atom pair inside the cut-off is
 * computed once, excluded and out-of-range pairs contribute nothing; Sec. V.B:
 * the pair list only changes which zero interactions are evaluated):
 *
 *   E = sum over unordered non-excluded pairs (i,j), i != j, r_ij < rc of
 *       V_LJ(r_ij) + V_C(r_ij),  r_ij the minimum-image distance in a
 *       rectangular periodic box (rc < L/2, so the image is unique).
 *
 * The paper gives the interaction types (Sec. II: Lennard-Jones plus
 * electrostatics; Sec. V.A: Ewald real-space correction in the pair kernel;
 * Sec. VI: reaction field) but no formulas; the forms used are:
 *   V_LJ = C12/r^12 - C6/r^6 - (C12/rc^12 - C6/rc^6)          (potential shift)
 *   V_RF = f qi qj (1/r + k_rf r^2 - c_rf),
 *          k_rf = (eps_rf - eps_r) / ((2 eps_rf + eps_r) rc^3)  (eps_rf = inf: 1/(2 rc^3)),
 *          c_rf = 1/rc + k_rf rc^2
 *   V_Ew = f qi qj (erfc(beta r)/r - erfc(beta rc)/rc)
 *   f = 138.935458 / eps_r  kJ mol^-1 nm e^-2
 * The pair parameters of atoms with types a, b are C = (C[a][b] + C[b][a]) / 2
 * (the table entry itself for the symmetric tables callers pass).
 * Forces F_i = -dE/dx_i = sum_j phi(r) r_vec, phi = -(1/r) dV/dr, r_vec = x_i - x_j (image);
 * optionally also Fabs_i = sum_j |phi(r) r_vec|, the size of the terms F_i is the sum of
 * (tests scale the FP32 accumulation error of a force by it).
 * Virial W = -1/2 sum_pairs r_vec (x) F_ij (3x3).
 *
 * Pieces: brute force O(N^2) (or_brute), its own cubic cell list (or_celllist,
 * optionally restricted to a subset of atoms), an evaluator over an explicit
 * set of image pairs (or_listset), the brute-force pair set within a radius
 * (or_pairs_within), the analytic vector-Jacobian product (or_vjp), and sums
 * over the pairs that tests use to size FP32 rounding bounds (or_energy_moments,
 * or_energy_hist).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_COULOMB_RF 0
#define OR_COULOMB_EWALD 1
#define OR_COULOMB_NONE 2 /* Lennard-Jones only */

typedef struct {
    int coulomb;
    double rc, rc2;
    double f;         /* 138.935458 / eps_r */
    double k_rf, c_rf;
    double beta;
    double ew_shift;  /* erfc(beta rc) / rc */
    int T;
    const double *c6, *c12;
} setup_t;

static void make_setup(setup_t *s, int coulomb, double eps_r, double eps_rf, double beta, double rc,
                       int T, const double *c6, const double *c12) {
    s->coulomb = coulomb;
    s->rc = rc;
    s->rc2 = rc * rc;
    s->f = 138.935458 / eps_r;
    if (isinf(eps_rf) || eps_rf <= 0.0)
        s->k_rf = 1.0 / (2.0 * rc * rc * rc);
    else
        s->k_rf = (eps_rf - eps_r) / ((2.0 * eps_rf + eps_r) * rc * rc * rc);
    s->c_rf = 1.0 / rc + s->k_rf * rc * rc;
    s->beta = beta;
    s->ew_shift = erfc(beta * rc) / rc;
    s->T = T;
    s->c6 = c6;
    s->c12 = c12;
}

/* Pair quantities at distance r (r2 = r^2) for parameters qq, c6, c12.
 *   vlj, vc   : potential energies (shifted)
 *   plj, pc   : phi = -(1/r) dV/dr
 *   dplj, dpc : d phi / dr                       (only when want_deriv)
 *   psi_c, v_c: phi_C / (qi qj) and V_C / (qi qj) (only when want_deriv)        */
typedef struct {
    double vlj, vc, plj, pc, dplj, dpc, psi_c, v_c;
} pair_t;

static void pair_terms(const setup_t *s, double r2, double qq, double c6, double c12, int want_deriv,
                       pair_t *o) {
    double r = sqrt(r2);
    double ir = 1.0 / r, ir2 = ir * ir, ir6 = ir2 * ir2 * ir2, ir12 = ir6 * ir6;
    double rc6 = 1.0 / (s->rc2 * s->rc2 * s->rc2), rc12 = rc6 * rc6;
    o->vlj = c12 * ir12 - c6 * ir6 - (c12 * rc12 - c6 * rc6);
    o->plj = (12.0 * c12 * ir12 - 6.0 * c6 * ir6) * ir2;
    double vcu, pcu, dpcu;
    if (s->coulomb == OR_COULOMB_NONE) {
        vcu = pcu = dpcu = 0.0;
    } else if (s->coulomb == OR_COULOMB_RF) {
        vcu = s->f * (ir + s->k_rf * r2 - s->c_rf);
        pcu = s->f * (ir * ir2 - 2.0 * s->k_rf);
        dpcu = s->f * (-3.0 * ir2 * ir2);
    } else {
        double br = s->beta * r;
        double ec = erfc(br);
        double g = 2.0 * s->beta / sqrt(M_PI) * exp(-br * br);
        vcu = s->f * (ec * ir - s->ew_shift);
        pcu = s->f * (ec * ir + g) * ir2;
        dpcu = s->f * (-3.0 * ec * ir2 * ir2 - g * (3.0 * ir * ir2 + 2.0 * s->beta * s->beta * ir));
    }
    o->vc = qq * vcu;
    o->pc = qq * pcu;
    if (want_deriv) {
        o->dplj = -168.0 * c12 * ir12 * ir2 * ir + 48.0 * c6 * ir6 * ir2 * ir;
        o->dpc = qq * dpcu;
        o->psi_c = pcu;
        o->v_c = vcu;
    }
}

static int excluded(const int *off, const int *idx, int i, int j) {
    for (int k = off[i]; k < off[i + 1]; k++)
        if (idx[k] == j) return 1;
    return 0;
}

static inline double pair_c(const double *tab, int T, int a, int b) {
    return 0.5 * (tab[a * T + b] + tab[b * T + a]);
}

static inline void min_image(const double *xi, const double *xj, const double *box, double d[3]) {
    for (int k = 0; k < 3; k++) {
        double v = xi[k] - xj[k];
        d[k] = v - box[k] * nearbyint(v / box[k]);
    }
}

/* ---------------------------------------------------------------- brute force */
int or_brute(int n, const double *x, const double *q, const int *type, int T, const double *c6,
             const double *c12, const int *excl_off, const int *excl_idx, const double *box,
             int coulomb, double eps_r, double eps_rf, double beta, double rc,
             double *F, double *E, double *W, int64_t *npairs, double *Fabs) {
    setup_t s;
    make_setup(&s, coulomb, eps_r, eps_rf, beta, rc, T, c6, c12);
    for (int k = 0; k < 3; k++)
        if (!(rc < 0.5 * box[k])) return 1;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (Fabs) memset(Fabs, 0, sizeof(double) * (size_t)n);
    double elj = 0.0, ec = 0.0, w[9] = {0};
    int64_t np = 0;
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < s.rc2)) continue;
            if (excluded(excl_off, excl_idx, i, j)) continue;
            pair_t p;
            pair_terms(&s, r2, q[i] * q[j], pair_c(c6, T, type[i], type[j]),
                       pair_c(c12, T, type[i], type[j]), 0, &p);
            double phi = p.plj + p.pc;
            for (int k = 0; k < 3; k++) {
                F[3 * i + k] += phi * d[k];
                F[3 * j + k] -= phi * d[k];
            }
            if (Fabs) {
                Fabs[i] += fabs(phi) * sqrt(r2);
                Fabs[j] += fabs(phi) * sqrt(r2);
            }
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) w[3 * a + b] += -0.5 * d[a] * phi * d[b];
            elj += p.vlj;
            ec += p.vc;
            np++;
        }
    }
    E[0] = elj;
    E[1] = ec;
    memcpy(W, w, sizeof(w));
    if (npairs) *npairs = np;
    return 0;
}

/* ---------------------------------------------------------------- cell list */
typedef struct {
    int nc[3];
    double cell[3];
    int *head;   /* [ncells+1] offsets */
    int *atoms;  /* atoms sorted by cell */
} cells_t;

static int cell_of(const cells_t *c, const double *xi, const double *box, int out[3]) {
    for (int k = 0; k < 3; k++) {
        double w = xi[k] - box[k] * floor(xi[k] / box[k]);
        int ic = (int)floor(w / c->cell[k]);
        if (ic < 0) ic = 0;
        if (ic >= c->nc[k]) ic = c->nc[k] - 1;
        out[k] = ic;
    }
    return (out[0] * c->nc[1] + out[1]) * c->nc[2] + out[2];
}

/* Cells of edge >= rcut; returns 0 when fewer than 3 cells fit along some axis. */
static int build_cells(cells_t *c, int n, const double *x, const double *box, double rcut) {
    for (int k = 0; k < 3; k++) {
        c->nc[k] = (int)floor(box[k] / rcut);
        if (c->nc[k] < 3) return 0;
        c->cell[k] = box[k] / c->nc[k];
    }
    int ncell = c->nc[0] * c->nc[1] * c->nc[2];
    c->head = (int *)calloc((size_t)ncell + 1, sizeof(int));
    c->atoms = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int tmp[3];
    for (int i = 0; i < n; i++) {
        cid[i] = cell_of(c, x + 3 * i, box, tmp);
        c->head[cid[i] + 1]++;
    }
    for (int k = 0; k < ncell; k++) c->head[k + 1] += c->head[k];
    int *fill = (int *)calloc((size_t)ncell, sizeof(int));
    for (int i = 0; i < n; i++) c->atoms[c->head[cid[i]] + fill[cid[i]]++] = i;
    free(fill);
    free(cid);
    return 1;
}

static void free_cells(cells_t *c) {
    free(c->head);
    free(c->atoms);
}

/* Per-atom full-neighbour evaluation.  For each atom i in `sub` (or every atom
 * when sub == NULL) sum over all j != i inside rc.  Each atom's sum is formed
 * by one thread in a fixed order, so results do not depend on the thread count.
 * Energies and the virial are returned only when sub == NULL. */
int or_celllist(int n, const double *x, const double *q, const int *type, int T, const double *c6,
                const double *c12, const int *excl_off, const int *excl_idx, const double *box,
                int coulomb, double eps_r, double eps_rf, double beta, double rc, int nsub,
                const int *sub, double *F, double *E, double *W, int64_t *npairs, double *Fabs) {
    setup_t s;
    make_setup(&s, coulomb, eps_r, eps_rf, beta, rc, T, c6, c12);
    for (int k = 0; k < 3; k++)
        if (!(rc < 0.5 * box[k])) return 1;
    cells_t c;
    if (!build_cells(&c, n, x, box, rc)) {
        if (sub != NULL) return 2;
        return or_brute(n, x, q, type, T, c6, c12, excl_off, excl_idx, box, coulomb, eps_r, eps_rf,
                        beta, rc, F, E, W, npairs, Fabs);
    }
    int m = sub ? nsub : n;
    double *e_at = (double *)calloc((size_t)m * 2, sizeof(double));
    double *w_at = (double *)calloc((size_t)m * 9, sizeof(double));
    int64_t *np_at = (int64_t *)calloc((size_t)m, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int t = 0; t < m; t++) {
        int i = sub ? sub[t] : t;
        int ci[3];
        cell_of(&c, x + 3 * i, box, ci);
        double fi[3] = {0, 0, 0}, fa = 0.0;
        for (int dx = -1; dx <= 1; dx++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dz = -1; dz <= 1; dz++) {
                    int a = (ci[0] + dx + c.nc[0]) % c.nc[0];
                    int b = (ci[1] + dy + c.nc[1]) % c.nc[1];
                    int e = (ci[2] + dz + c.nc[2]) % c.nc[2];
                    int cc = (a * c.nc[1] + b) * c.nc[2] + e;
                    for (int p = c.head[cc]; p < c.head[cc + 1]; p++) {
                        int j = c.atoms[p];
                        if (j == i) continue;
                        double d[3];
                        min_image(x + 3 * i, x + 3 * j, box, d);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < s.rc2)) continue;
                        if (excluded(excl_off, excl_idx, i, j)) continue;
                        pair_t pt;
                        pair_terms(&s, r2, q[i] * q[j], pair_c(c6, T, type[i], type[j]),
                                   pair_c(c12, T, type[i], type[j]), 0, &pt);
                        double phi = pt.plj + pt.pc;
                        for (int k = 0; k < 3; k++) fi[k] += phi * d[k];
                        fa += fabs(phi) * sqrt(r2);
                        e_at[2 * t] += 0.5 * pt.vlj;
                        e_at[2 * t + 1] += 0.5 * pt.vc;
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) w_at[9 * t + 3 * u + v] += -0.25 * d[u] * phi * d[v];
                        np_at[t]++;
                    }
                }
        for (int k = 0; k < 3; k++) F[3 * t + k] = fi[k];
        if (Fabs) Fabs[t] = fa;
    }
    if (sub == NULL) {
        double elj = 0, ec = 0, w[9] = {0};
        int64_t np = 0;
        for (int t = 0; t < m; t++) {
            elj += e_at[2 * t];
            ec += e_at[2 * t + 1];
            for (int k = 0; k < 9; k++) w[k] += w_at[9 * t + k];
            np += np_at[t];
        }
        E[0] = elj;
        E[1] = ec;
        memcpy(W, w, sizeof(w));
        if (npairs) *npairs = np / 2;
    }
    free(e_at);
    free(w_at);
    free(np_at);
    free_cells(&c);
    return 0;
}

/* ------------------------------------------------------ explicit image-pair set */
/* pairs: [npairs][5] = (i, j, sx, sy, sz); the pair vector is x_i - x_j + s*L
 * (s integer per axis, no minimum image).  Pairs with r >= rc contribute nothing,
 * unless `frozen` is set: then every listed pair is summed at its distance.
 * Every listed pair is summed as given (exclusions are not re-applied). */
int or_listset(int n, const double *x, const double *q, const int *type, int T, const double *c6,
               const double *c12, const double *box, int coulomb, double eps_r, double eps_rf,
               double beta, double rc, int64_t npairs, const int64_t *pairs, int frozen, double *F,
               double *E, double *W, int64_t *n_in, double *Fabs) {
    setup_t s;
    make_setup(&s, coulomb, eps_r, eps_rf, beta, rc, T, c6, c12);
    /* frozen: every listed pair is summed whatever its distance (the pair set is held
     * fixed, as for finite differences of a frozen list); the potentials keep their
     * shift at rc and continue smoothly beyond it */
    const double rtest2 = frozen ? INFINITY : s.rc2;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (Fabs) memset(Fabs, 0, sizeof(double) * (size_t)n);
    double elj = 0, ec = 0, w[9] = {0};
    int64_t cnt = 0;
    for (int64_t p = 0; p < npairs; p++) {
        const int64_t *e = pairs + 5 * p;
        int i = (int)e[0], j = (int)e[1];
        if (i < 0 || j < 0 || i >= n || j >= n) return 1;
        double d[3];
        for (int k = 0; k < 3; k++) d[k] = x[3 * i + k] - x[3 * j + k] + (double)e[2 + k] * box[k];
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(r2 < rtest2)) continue;
        pair_t pt;
        pair_terms(&s, r2, q[i] * q[j], pair_c(c6, T, type[i], type[j]), pair_c(c12, T, type[i], type[j]), 0,
                   &pt);
        double phi = pt.plj + pt.pc;
        for (int k = 0; k < 3; k++) {
            F[3 * i + k] += phi * d[k];
            F[3 * j + k] -= phi * d[k];
        }
        if (Fabs) {
            Fabs[i] += fabs(phi) * sqrt(r2);
            Fabs[j] += fabs(phi) * sqrt(r2);
        }
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) w[3 * a + b] += -0.5 * d[a] * phi * d[b];
        elj += pt.vlj;
        ec += pt.vc;
        cnt++;
    }
    E[0] = elj;
    E[1] = ec;
    memcpy(W, w, sizeof(w));
    if (n_in) *n_in = cnt;
    return 0;
}

/* ------------------------------------------------- brute-force pair set P(rcut) */
/* All unordered non-excluded pairs i < j with minimum-image distance < rcut,
 * written as (i, j, sx, sy, sz) with pair vector x_i - x_j + s*L.  Requires
 * rcut < L/2 on every axis.  Returns the count (may exceed cap; only cap written). */
int64_t or_pairs_within(int n, const double *x, const double *box, const int *excl_off,
                        const int *excl_idx, double rcut, int64_t cap, int64_t *out) {
    double r2c = rcut * rcut;
    int64_t cnt = 0;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            double d[3], s[3];
            for (int k = 0; k < 3; k++) {
                double v = x[3 * i + k] - x[3 * j + k];
                s[k] = -nearbyint(v / box[k]);
                d[k] = v + s[k] * box[k];
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < r2c)) continue;
            if (excluded(excl_off, excl_idx, i, j)) continue;
            if (cnt < cap) {
                int64_t *e = out + 5 * cnt;
                e[0] = i;
                e[1] = j;
                e[2] = (int64_t)s[0];
                e[3] = (int64_t)s[1];
                e[4] = (int64_t)s[2];
            }
            cnt++;
        }
    return cnt;
}

/* ------------------------------------------------------------ analytic adjoint */
/* Gradients of L = <gF, F> + gE * E (E = E_LJ + E_C) with respect to positions,
 * charges and the C6 / C12 tables.  Per pair, with r_vec = x_i - x_j (image),
 * w = gF_i - gF_j and u = r_vec . w:
 *   dL/dx_i += phi w + (phi'/r) u r_vec - gE phi r_vec      (and minus that on x_j)
 *   dL/dq_i += q_j (psi_C u + gE v_C)                       (phi_C = qi qj psi_C, V_C = qi qj v_C)
 *   dL/dC12 += 12 r^-14 u + gE (r^-12 - rc^-12)
 *   dL/dC6  += -6 r^-8 u - gE (r^-6 - rc^-6)
 * Pair parameters are (C[a][b] + C[b][a]) / 2, so a pair of types a != b puts
 * half of its parameter gradient in [a][b] and half in [b][a]; a == b puts all
 * of it in [a][a].  Uses the brute-force pair loop (intended for N up to a few 10^4). */
int or_vjp(int n, const double *x, const double *q, const int *type, int T, const double *c6,
           const double *c12, const int *excl_off, const int *excl_idx, const double *box, int coulomb,
           double eps_r, double eps_rf, double beta, double rc, const double *gF, double gE, double *gx,
           double *gq, double *gc6, double *gc12) {
    setup_t s;
    make_setup(&s, coulomb, eps_r, eps_rf, beta, rc, T, c6, c12);
    for (int k = 0; k < 3; k++)
        if (!(rc < 0.5 * box[k])) return 1;
    memset(gx, 0, sizeof(double) * 3 * (size_t)n);
    memset(gq, 0, sizeof(double) * (size_t)n);
    memset(gc6, 0, sizeof(double) * (size_t)T * T);
    memset(gc12, 0, sizeof(double) * (size_t)T * T);
    double rc6 = 1.0 / (s.rc2 * s.rc2 * s.rc2), rc12 = rc6 * rc6;
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < s.rc2)) continue;
            if (excluded(excl_off, excl_idx, i, j)) continue;
            int a = type[i], b = type[j];
            pair_t p;
            pair_terms(&s, r2, q[i] * q[j], pair_c(c6, T, a, b), pair_c(c12, T, a, b), 1, &p);
            double r = sqrt(r2);
            double phi = p.plj + p.pc, dphi = p.dplj + p.dpc;
            double w[3], u = 0.0;
            for (int k = 0; k < 3; k++) {
                w[k] = gF[3 * i + k] - gF[3 * j + k];
                u += d[k] * w[k];
            }
            for (int k = 0; k < 3; k++) {
                double g = phi * w[k] + (dphi / r) * u * d[k] - gE * phi * d[k];
                gx[3 * i + k] += g;
                gx[3 * j + k] -= g;
            }
            gq[i] += q[j] * (p.psi_c * u + gE * p.v_c);
            gq[j] += q[i] * (p.psi_c * u + gE * p.v_c);
            double ir2 = 1.0 / r2, ir6 = ir2 * ir2 * ir2, ir12 = ir6 * ir6;
            double g12 = 12.0 * ir12 * ir2 * u + gE * (ir12 - rc12);
            double g6 = -6.0 * ir6 * ir2 * u - gE * (ir6 - rc6);
            if (a == b) {
                gc12[a * T + a] += g12;
                gc6[a * T + a] += g6;
            } else {
                gc12[a * T + b] += 0.5 * g12;
                gc12[b * T + a] += 0.5 * g12;
                gc6[a * T + b] += 0.5 * g6;
                gc6[b * T + a] += 0.5 * g6;
            }
        }
    }
    return 0;
}

/* ----------------------------------------------- rounding-floor moments of E */
/* Sums over unordered pairs inside rc of the squared first-order sensitivities
 * of the pair energies to a relative perturbation of r:
 *   m[0] = sum (r dV_LJ/dr)^2 = sum (12 C12 r^-12 - 6 C6 r^-6)^2
 *   m[1] = sum (r dV_C/dr)^2  (f qi qj / r times the screening factor for Ewald)
 *   m[2] = sum |V_LJ|,  m[3] = sum |V_C|
 * A relative rounding error eps in each r moves E_LJ by about eps sqrt(m[0]) (random
 * signs), so sqrt(m)/|E| is the relative error floor of an energy summed from
 * pair terms computed in a precision with unit roundoff eps. */
int or_energy_moments(int n, const double *x, const double *q, const int *type, int T, const double *c6,
                      const double *c12, const int *excl_off, const int *excl_idx, const double *box, int coulomb,
                      double eps_r, double eps_rf, double beta, double rc, double *m) {
    setup_t s;
    make_setup(&s, coulomb, eps_r, eps_rf, beta, rc, T, c6, c12);
    for (int k = 0; k < 3; k++)
        if (!(rc < 0.5 * box[k])) return 1;
    cells_t c;
    int use_cells = build_cells(&c, n, x, box, rc);
    double *acc = (double *)calloc((size_t)n * 4, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; i++) {
        int ci[3] = {0, 0, 0};
        if (use_cells) cell_of(&c, x + 3 * i, box, ci);
        int span = use_cells ? 1 : 0;
        for (int dx = -span; dx <= span; dx++)
            for (int dy = -span; dy <= span; dy++)
                for (int dz = -span; dz <= span; dz++) {
                    int lo = 0, hi = n;
                    if (use_cells) {
                        int a = (ci[0] + dx + c.nc[0]) % c.nc[0];
                        int b = (ci[1] + dy + c.nc[1]) % c.nc[1];
                        int e = (ci[2] + dz + c.nc[2]) % c.nc[2];
                        int cc = (a * c.nc[1] + b) * c.nc[2] + e;
                        lo = c.head[cc];
                        hi = c.head[cc + 1];
                    }
                    for (int p = lo; p < hi; p++) {
                        int j = use_cells ? c.atoms[p] : p;
                        if (j == i) continue;
                        double d[3];
                        min_image(x + 3 * i, x + 3 * j, box, d);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < s.rc2)) continue;
                        if (excluded(excl_off, excl_idx, i, j)) continue;
                        pair_t pt;
                        pair_terms(&s, r2, q[i] * q[j], pair_c(c6, T, type[i], type[j]),
                                   pair_c(c12, T, type[i], type[j]), 0, &pt);
                        /* r dV/dr = -phi r^2 */
                        double slj = pt.plj * r2, sc = pt.pc * r2;
                        acc[4 * i] += 0.5 * slj * slj;
                        acc[4 * i + 1] += 0.5 * sc * sc;
                        acc[4 * i + 2] += 0.5 * fabs(pt.vlj);
                        acc[4 * i + 3] += 0.5 * fabs(pt.vc);
                    }
                }
    }
    m[0] = m[1] = m[2] = m[3] = 0.0;
    for (int i = 0; i < n; i++)
        for (int k = 0; k < 4; k++) m[k] += acc[4 * i + k];
    free(acc);
    if (use_cells) free_cells(&c);
    return 0;
}

/* Radial histogram of the pair terms inside rc: for nbins equal bins of r on
 * [0, rc), h[6*k + 0..5] = number of pairs, sum of qi qj, sum of V_LJ, sum of
 * V_LJ^2, sum of V_C, sum of V_C^2 over the pairs whose distance falls in bin k.
 * The bins add up to the energies of or_celllist.  Tests combine them with a
 * model of FP32 rounding per distance to bound the error of an FP32 energy sum. */
int or_energy_hist(int n, const double *x, const double *q, const int *type, int T, const double *c6,
                   const double *c12, const int *excl_off, const int *excl_idx, const double *box, int coulomb,
                   double eps_r, double eps_rf, double beta, double rc, int nbins, double *h) {
    setup_t s;
    make_setup(&s, coulomb, eps_r, eps_rf, beta, rc, T, c6, c12);
    for (int k = 0; k < 3; k++)
        if (!(rc < 0.5 * box[k])) return 1;
    if (nbins < 1) return 2;
    cells_t c;
    int use_cells = build_cells(&c, n, x, box, rc);
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nt * nbins * 6, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *ht = acc + (size_t)tid * nbins * 6;
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; i++) {
            int ci[3] = {0, 0, 0};
            if (use_cells) cell_of(&c, x + 3 * i, box, ci);
            int span = use_cells ? 1 : 0;
            for (int dx = -span; dx <= span; dx++)
                for (int dy = -span; dy <= span; dy++)
                    for (int dz = -span; dz <= span; dz++) {
                        int lo = 0, hi = n;
                        if (use_cells) {
                            int a = (ci[0] + dx + c.nc[0]) % c.nc[0];
                            int b = (ci[1] + dy + c.nc[1]) % c.nc[1];
                            int e = (ci[2] + dz + c.nc[2]) % c.nc[2];
                            int cc = (a * c.nc[1] + b) * c.nc[2] + e;
                            lo = c.head[cc];
                            hi = c.head[cc + 1];
                        }
                        for (int p = lo; p < hi; p++) {
                            int j = use_cells ? c.atoms[p] : p;
                            if (j <= i) continue; /* each unordered pair once */
                            double d[3];
                            min_image(x + 3 * i, x + 3 * j, box, d);
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (!(r2 < s.rc2)) continue;
                            if (excluded(excl_off, excl_idx, i, j)) continue;
                            pair_t pt;
                            double qq = q[i] * q[j];
                            pair_terms(&s, r2, qq, pair_c(c6, T, type[i], type[j]), pair_c(c12, T, type[i], type[j]),
                                       0, &pt);
                            int k = (int)(sqrt(r2) / rc * nbins);
                            if (k >= nbins) k = nbins - 1;
                            double *b = ht + 6 * k;
                            b[0] += 1.0;
                            b[1] += qq;
                            b[2] += pt.vlj;
                            b[3] += pt.vlj * pt.vlj;
                            b[4] += pt.vc;
                            b[5] += pt.vc * pt.vc;
                        }
                    }
        }
    }
    memset(h, 0, sizeof(double) * 6 * (size_t)nbins);
    for (int t = 0; t < nt; t++)
        for (int k = 0; k < 6 * nbins; k++) h[k] += acc[(size_t)t * nbins * 6 + k];
    free(acc);
    if (use_cells) free_cells(&c);
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
