/*
 * mfs_oracle.c -- plain FP64 CPU oracle of the paper's Algorithm 1
 * ("A First-Order Numerical Algorithm without Matrix Operations", arXiv 2203.05027).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library. The product (the CUDA path behind include/mfs.h) never
 * links, imports or calls it, and it shares no code with it: no header, no helper, no table.
 *
 * What it computes, in the paper's order and notation, with no blocking or fusion:
 *   Sec. IV, eq. (UU)/(VV): U = sum_k a_k e_{i_k} edot_k^T (values), V[j_k, k] = 1 (locations),
 *     with the nonzeros taken in column-major order (Example 1 lists them that way).
 *   Algorithm 1, steps 2-3: F_U = (I + U U^T)^{-1}, F_V = (I + V V^T)^{-1}, both diagonal.
 *   Algorithm 1, steps 5-10 (one iteration, each step reads the newest values):
 *     x      <- F_V ( V (y + gamma/mu) + z + delta/mu - c/mu )                 (eq. vvt)
 *     y      <- (I - U^T F_U U) ( U^T (b - lambda/mu) + V^T x - gamma/mu )     (y-step + Woodbury)
 *     z      <- proj_K( x - delta/mu )                                          (z-step, eq. proj)
 *     lambda <- lambda + mu (U y - b)
 *     gamma  <- gamma  + mu (y - V^T x)
 *     delta  <- delta  + mu (z - x)
 *   The y and gamma vectors have length o (one entry per nonzero), exactly as in the paper.
 *
 * Residuals (the paper's stopping rules mix forms; Sec. V): this file evaluates, at the current
 * (x, lambda), the raw norms from explicit COO loops for A x and A^T lambda, and the relative
 * KKT measure used for termination:
 *   r_p = ||Ax-b||_2 / (1+||b||_2),   r_k = ||x - P_K x||_2 / (1+||x||_2),
 *   r_d = ||s - P_K s||_2 / (1+||c||_2) with s = c + A^T lambda (K is self-dual),
 *   r_g = |c^T x + b^T lambda| / (1 + |c^T x| + |b^T lambda|),    kkt = max of the four.
 *
 * Precision: IEEE FP64 throughout; build with -ffp-contract=off so no FMA contraction happens.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CONE_NONNEG 0 /* nonnegative orthant of the given size = product of size-1 Lorentz cones */
#define ORC_CONE_SOC 1    /* one Lorentz (second-order) cone of the given size */

#define ORC_OK 0
#define ORC_ERR_INVALID 2
#define ORC_ERR_OOM 4

typedef struct orc {
    int64_t m, n, o;
    /* UV decomposition: nonzero k sits at row ik[k], column jk[k], value ak[k]. */
    int64_t *ik, *jk;
    double *ak;
    double *FU; /* length m: diagonal of (I + U U^T)^{-1} */
    double *FV; /* length n: diagonal of (I + V V^T)^{-1} */
    double *b, *c;
    int64_t ncones;
    int32_t *cone_kind;
    int64_t *cone_size;
    double mu;
    /* iterate of Algorithm 1 */
    double *x, *y, *z, *lam, *gam, *del;
    /* work vectors */
    double *wn, *wm, *wo, *wo2;
} orc;

static void *xcalloc(size_t count, size_t elem) {
    if (count == 0) count = 1;
    return calloc(count, elem);
}

void orc_destroy(orc *P) {
    if (!P) return;
    free(P->ik); free(P->jk); free(P->ak);
    free(P->FU); free(P->FV); free(P->b); free(P->c);
    free(P->cone_kind); free(P->cone_size);
    free(P->x); free(P->y); free(P->z); free(P->lam); free(P->gam); free(P->del);
    free(P->wn); free(P->wm); free(P->wo); free(P->wo2);
    free(P);
}

/*
 * Build the problem: COO triplets (row, col, val) in any order. Entries with equal (row, col)
 * are summed; entries whose (summed) value is exactly zero are dropped, since a stored zero
 * would count in V V^T. The remaining nonzeros are numbered k = 0..o-1 column by column,
 * rows ascending within a column (the order of Example 1). cones: ncones (kind, size) pairs
 * covering x's coordinates in order, sizes summing to n.
 */
int orc_create(int64_t m, int64_t n, int64_t nnz, const int64_t *row, const int64_t *col,
               const double *val, const double *b, const double *c, int64_t ncones,
               const int32_t *cone_kind, const int64_t *cone_size, double mu, orc **out) {
    *out = NULL;
    if (m < 0 || n < 0 || nnz < 0 || ncones < 0 || !(mu > 0)) return ORC_ERR_INVALID;
    int64_t total = 0;
    for (int64_t q = 0; q < ncones; q++) {
        if (cone_size[q] < 1) return ORC_ERR_INVALID;
        if (cone_kind[q] != ORC_CONE_NONNEG && cone_kind[q] != ORC_CONE_SOC) return ORC_ERR_INVALID;
        total += cone_size[q];
    }
    if (total != n) return ORC_ERR_INVALID;
    for (int64_t t = 0; t < nnz; t++)
        if (row[t] < 0 || row[t] >= m || col[t] < 0 || col[t] >= n) return ORC_ERR_INVALID;

    orc *P = (orc *)calloc(1, sizeof(orc));
    if (!P) return ORC_ERR_OOM;
    P->m = m; P->n = n; P->mu = mu; P->ncones = ncones;

    /* Column-major ordering by two stable counting sorts: first by row, then by column. */
    int64_t *perm1 = (int64_t *)xcalloc(nnz, sizeof(int64_t));
    int64_t *perm2 = (int64_t *)xcalloc(nnz, sizeof(int64_t));
    int64_t *cnt = (int64_t *)xcalloc((m > n ? m : n) + 1, sizeof(int64_t));
    if (!perm1 || !perm2 || !cnt) { free(perm1); free(perm2); free(cnt); orc_destroy(P); return ORC_ERR_OOM; }
    memset(cnt, 0, sizeof(int64_t) * (size_t)(m + 1));
    for (int64_t t = 0; t < nnz; t++) cnt[row[t] + 1]++;
    for (int64_t i = 0; i < m; i++) cnt[i + 1] += cnt[i];
    for (int64_t t = 0; t < nnz; t++) perm1[cnt[row[t]]++] = t;
    memset(cnt, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t t = 0; t < nnz; t++) cnt[col[t] + 1]++;
    for (int64_t j = 0; j < n; j++) cnt[j + 1] += cnt[j];
    for (int64_t s = 0; s < nnz; s++) { int64_t t = perm1[s]; perm2[cnt[col[t]]++] = t; }
    free(cnt);
    free(perm1);

    P->ik = (int64_t *)xcalloc(nnz, sizeof(int64_t));
    P->jk = (int64_t *)xcalloc(nnz, sizeof(int64_t));
    P->ak = (double *)xcalloc(nnz, sizeof(double));
    if (!P->ik || !P->jk || !P->ak) { free(perm2); orc_destroy(P); return ORC_ERR_OOM; }
    int64_t o = 0;
    int64_t s = 0;
    while (s < nnz) {
        int64_t t = perm2[s];
        int64_t i = row[t], j = col[t];
        double a = val[t];
        s++;
        while (s < nnz && row[perm2[s]] == i && col[perm2[s]] == j) { a += val[perm2[s]]; s++; }
        if (a != 0.0) { P->ik[o] = i; P->jk[o] = j; P->ak[o] = a; o++; }
    }
    free(perm2);
    P->o = o;

    /* Algorithm 1, steps 2-3: diagonal factors. (U U^T)_ii = sum of a_k^2 over row i;
       (V V^T)_jj = number of nonzeros in column j. */
    P->FU = (double *)xcalloc(m, sizeof(double));
    P->FV = (double *)xcalloc(n, sizeof(double));
    if (!P->FU || !P->FV) { orc_destroy(P); return ORC_ERR_OOM; }
    for (int64_t k = 0; k < o; k++) {
        P->FU[P->ik[k]] += P->ak[k] * P->ak[k];
        P->FV[P->jk[k]] += 1.0;
    }
    for (int64_t i = 0; i < m; i++) P->FU[i] = 1.0 / (1.0 + P->FU[i]);
    for (int64_t j = 0; j < n; j++) P->FV[j] = 1.0 / (1.0 + P->FV[j]);

    P->b = (double *)xcalloc(m, sizeof(double));
    P->c = (double *)xcalloc(n, sizeof(double));
    P->cone_kind = (int32_t *)xcalloc(ncones, sizeof(int32_t));
    P->cone_size = (int64_t *)xcalloc(ncones, sizeof(int64_t));
    P->x = (double *)xcalloc(n, sizeof(double));
    P->z = (double *)xcalloc(n, sizeof(double));
    P->del = (double *)xcalloc(n, sizeof(double));
    P->lam = (double *)xcalloc(m, sizeof(double));
    P->y = (double *)xcalloc(o, sizeof(double));
    P->gam = (double *)xcalloc(o, sizeof(double));
    P->wn = (double *)xcalloc(n, sizeof(double));
    P->wm = (double *)xcalloc(m, sizeof(double));
    P->wo = (double *)xcalloc(o, sizeof(double));
    P->wo2 = (double *)xcalloc(o, sizeof(double));
    if (!P->b || !P->c || !P->cone_kind || !P->cone_size || !P->x || !P->z || !P->del || !P->lam ||
        !P->y || !P->gam || !P->wn || !P->wm || !P->wo || !P->wo2) {
        orc_destroy(P);
        return ORC_ERR_OOM;
    }
    if (m) memcpy(P->b, b, sizeof(double) * (size_t)m);
    if (n) memcpy(P->c, c, sizeof(double) * (size_t)n);
    if (ncones) {
        memcpy(P->cone_kind, cone_kind, sizeof(int32_t) * (size_t)ncones);
        memcpy(P->cone_size, cone_size, sizeof(int64_t) * (size_t)ncones);
    }
    *out = P;
    return ORC_OK;
}

int64_t orc_nnz(const orc *P) { return P->o; }

/* Export the UV decomposition: U[ik[k], k] = ak[k], V[jk[k], k] = 1, and the diagonal factors. */
void orc_get_uv(const orc *P, int64_t *ik, int64_t *jk, double *ak, double *FU, double *FV) {
    if (ik) memcpy(ik, P->ik, sizeof(int64_t) * (size_t)P->o);
    if (jk) memcpy(jk, P->jk, sizeof(int64_t) * (size_t)P->o);
    if (ak) memcpy(ak, P->ak, sizeof(double) * (size_t)P->o);
    if (FU) memcpy(FU, P->FU, sizeof(double) * (size_t)P->m);
    if (FV) memcpy(FV, P->FV, sizeof(double) * (size_t)P->n);
}

/* Set / read the full iterate (x, y, z, lambda, gamma, delta). NULL leaves a vector unchanged
   (set) or skips it (get). y and gamma have length o, in the nonzero order above. */
void orc_set_state(orc *P, const double *x, const double *y, const double *z, const double *lam,
                   const double *gam, const double *del) {
    if (x) memcpy(P->x, x, sizeof(double) * (size_t)P->n);
    if (y) memcpy(P->y, y, sizeof(double) * (size_t)P->o);
    if (z) memcpy(P->z, z, sizeof(double) * (size_t)P->n);
    if (lam) memcpy(P->lam, lam, sizeof(double) * (size_t)P->m);
    if (gam) memcpy(P->gam, gam, sizeof(double) * (size_t)P->o);
    if (del) memcpy(P->del, del, sizeof(double) * (size_t)P->n);
}

void orc_get_state(const orc *P, double *x, double *y, double *z, double *lam, double *gam, double *del) {
    if (x) memcpy(x, P->x, sizeof(double) * (size_t)P->n);
    if (y) memcpy(y, P->y, sizeof(double) * (size_t)P->o);
    if (z) memcpy(z, P->z, sizeof(double) * (size_t)P->n);
    if (lam) memcpy(lam, P->lam, sizeof(double) * (size_t)P->m);
    if (gam) memcpy(gam, P->gam, sizeof(double) * (size_t)P->o);
    if (del) memcpy(del, P->del, sizeof(double) * (size_t)P->n);
}

void orc_set_mu(orc *P, double mu) { P->mu = mu; }

/*
 * Projection onto one Lorentz cone of size s (eq. proj): with alpha = ||w_{2..s}||_2,
 *   alpha <= -w_1  ->  0
 *   alpha <=  w_1  ->  w
 *   otherwise      ->  w/2 + [alpha/2, w_1 w_2/(2 alpha), ..., w_1 w_s/(2 alpha)].
 * The first test is taken first, so the tie alpha = -w_1 = 0 (w = 0) maps to 0 = w as well.
 * in and out may alias.
 */
void orc_proj_lorentz(int64_t s, const double *in, double *out) {
    double w1 = in[0];
    double ss = 0.0;
    for (int64_t t = 1; t < s; t++) ss += in[t] * in[t];
    double alpha = sqrt(ss);
    if (alpha <= -w1) {
        for (int64_t t = 0; t < s; t++) out[t] = 0.0;
    } else if (alpha <= w1) {
        for (int64_t t = 0; t < s; t++) out[t] = in[t];
    } else {
        out[0] = in[0] / 2.0 + alpha / 2.0;
        for (int64_t t = 1; t < s; t++) out[t] = in[t] / 2.0 + w1 * in[t] / (2.0 * alpha);
    }
}

/* proj_K over the product cone: a nonnegative orthant of size s is s Lorentz cones of size 1. */
void orc_proj_K(const orc *P, const double *in, double *out) {
    int64_t off = 0;
    for (int64_t q = 0; q < P->ncones; q++) {
        int64_t s = P->cone_size[q];
        if (P->cone_kind[q] == ORC_CONE_SOC) {
            orc_proj_lorentz(s, in + off, out + off);
        } else {
            for (int64_t t = 0; t < s; t++) orc_proj_lorentz(1, in + off + t, out + off + t);
        }
        off += s;
    }
}

/* Algorithm 1, step 5 (eq. vvt): x <- F_V ( V (y + gamma/mu) + z + delta/mu - c/mu ). */
void orc_step_x(orc *P) {
    const double mu = P->mu;
    double *Vq = P->wn;
    for (int64_t j = 0; j < P->n; j++) Vq[j] = 0.0;
    for (int64_t k = 0; k < P->o; k++) Vq[P->jk[k]] += P->y[k] + P->gam[k] / mu;
    for (int64_t j = 0; j < P->n; j++)
        P->x[j] = P->FV[j] * (Vq[j] + P->z[j] + P->del[j] / mu - P->c[j] / mu);
}

/* Algorithm 1, step 6: y <- (I - U^T F_U U) w with w = U^T (b - lambda/mu) + V^T x - gamma/mu
   (the y-step's closed form after the matrix inversion lemma). */
void orc_step_y(orc *P) {
    const double mu = P->mu;
    double *w = P->wo;
    double *Uw = P->wm;
    for (int64_t k = 0; k < P->o; k++)
        w[k] = P->ak[k] * (P->b[P->ik[k]] - P->lam[P->ik[k]] / mu) + P->x[P->jk[k]] - P->gam[k] / mu;
    for (int64_t i = 0; i < P->m; i++) Uw[i] = 0.0;
    for (int64_t k = 0; k < P->o; k++) Uw[P->ik[k]] += P->ak[k] * w[k];
    for (int64_t k = 0; k < P->o; k++) P->y[k] = w[k] - P->ak[k] * (P->FU[P->ik[k]] * Uw[P->ik[k]]);
}

/* Algorithm 1, step 7: z <- proj_K( x - delta/mu ). */
void orc_step_z(orc *P) {
    const double mu = P->mu;
    double *arg = P->wn;
    for (int64_t j = 0; j < P->n; j++) arg[j] = P->x[j] - P->del[j] / mu;
    orc_proj_K(P, arg, P->z);
}

/* Algorithm 1, step 8: lambda <- lambda + mu (U y - b). */
void orc_step_lambda(orc *P) {
    const double mu = P->mu;
    double *Uy = P->wm;
    for (int64_t i = 0; i < P->m; i++) Uy[i] = 0.0;
    for (int64_t k = 0; k < P->o; k++) Uy[P->ik[k]] += P->ak[k] * P->y[k];
    for (int64_t i = 0; i < P->m; i++) P->lam[i] = P->lam[i] + mu * (Uy[i] - P->b[i]);
}

/* Algorithm 1, step 9: gamma <- gamma + mu (y - V^T x). */
void orc_step_gamma(orc *P) {
    const double mu = P->mu;
    for (int64_t k = 0; k < P->o; k++) P->gam[k] = P->gam[k] + mu * (P->y[k] - P->x[P->jk[k]]);
}

/* Algorithm 1, step 10: delta <- delta + mu (z - x). */
void orc_step_delta(orc *P) {
    const double mu = P->mu;
    for (int64_t j = 0; j < P->n; j++) P->del[j] = P->del[j] + mu * (P->z[j] - P->x[j]);
}

/* Algorithm 1, steps 5-10, repeated iters times. */
void orc_iterate(orc *P, int64_t iters) {
    for (int64_t it = 0; it < iters; it++) {
        orc_step_x(P);
        orc_step_y(P);
        orc_step_z(P);
        orc_step_lambda(P);
        orc_step_gamma(P);
        orc_step_delta(P);
    }
}

/*
 * The literal state that a given primal-dual pair (x, lambda) stands for after an iteration:
 * y = V^T x + U^T F_U (b - A x) and gamma = -U^T lambda. The lambda- and gamma-updates together
 * with the y-step give gamma = -U^T lambda after every iteration; given that, the next y-step
 * gives y of the form above. So every iterate from the second on (from the first, if the start
 * already has gamma = -U^T lambda) is of this form, and this is how a warm start from
 * (x, lambda) enters the literal iteration. Writes y and gamma.
 */
void orc_consistent_y_gamma(const orc *P, const double *x, const double *lam, double *y, double *gam) {
    double *rho = (double *)xcalloc(P->m, sizeof(double));
    for (int64_t k = 0; k < P->o; k++) rho[P->ik[k]] += P->ak[k] * x[P->jk[k]];
    for (int64_t i = 0; i < P->m; i++) rho[i] = P->FU[i] * (P->b[i] - rho[i]);
    for (int64_t k = 0; k < P->o; k++) {
        y[k] = x[P->jk[k]] + P->ak[k] * rho[P->ik[k]];
        gam[k] = -P->ak[k] * lam[P->ik[k]];
    }
    free(rho);
}

/* A x and A^T lambda from the nonzeros (explicit loops). */
void orc_matvec(const orc *P, const double *x, double *Ax) {
    for (int64_t i = 0; i < P->m; i++) Ax[i] = 0.0;
    for (int64_t k = 0; k < P->o; k++) Ax[P->ik[k]] += P->ak[k] * x[P->jk[k]];
}

void orc_rmatvec(const orc *P, const double *lam, double *ATl) {
    for (int64_t j = 0; j < P->n; j++) ATl[j] = 0.0;
    for (int64_t k = 0; k < P->o; k++) ATl[P->jk[k]] += P->ak[k] * lam[P->ik[k]];
}

/*
 * Residuals at the current (x, lambda). out[] receives, in order:
 *  0 r_prim  = ||Ax-b||_2 / (1+||b||_2)
 *  1 r_dual  = ||s - P_K s||_2 / (1+||c||_2),  s = c + A^T lambda
 *  2 r_cone  = ||x - P_K x||_2 / (1+||x||_2)
 *  3 r_gap   = |c^T x + b^T lambda| / (1 + |c^T x| + |b^T lambda|)
 *  4 kkt     = max(out[0..3])
 *  5 pobj    = c^T x
 *  6 dobj    = -b^T lambda
 *  7 ||Ax-b||_2        8 ||b||_2         9 ||x-P_K x||_2     10 ||x||_2
 * 11 ||s-P_K s||_2    12 ||c||_2        13 ||A^T lambda + c||_2
 * 14 ||Ax-b||_inf     15 ||Ax||_inf     16 ||b||_inf
 * 17 ||A^T lambda + c||_inf             18 ||A^T lambda||_inf 19 ||c||_inf
 * 20 ||x||_inf       21 ||x-P_K x||_inf 22 ||s-P_K s||_inf
 */
void orc_residuals(const orc *P, double *out) {
    const int64_t m = P->m, n = P->n;
    double *Ax = (double *)xcalloc(m, sizeof(double));
    double *s = (double *)xcalloc(n, sizeof(double));
    double *ps = (double *)xcalloc(n, sizeof(double));
    double *px = (double *)xcalloc(n, sizeof(double));
    orc_matvec(P, P->x, Ax);
    orc_rmatvec(P, P->lam, s); /* s = A^T lambda for now */
    double rp2 = 0, b2 = 0, rpinf = 0, axinf = 0, binf = 0;
    for (int64_t i = 0; i < m; i++) {
        double r = Ax[i] - P->b[i];
        rp2 += r * r;
        b2 += P->b[i] * P->b[i];
        if (fabs(r) > rpinf) rpinf = fabs(r);
        if (fabs(Ax[i]) > axinf) axinf = fabs(Ax[i]);
        if (fabs(P->b[i]) > binf) binf = fabs(P->b[i]);
    }
    double atlinf = 0, cinf = 0, sinf = 0, s2 = 0, c2 = 0, ctx = 0, x2 = 0;
    for (int64_t j = 0; j < n; j++) {
        if (fabs(s[j]) > atlinf) atlinf = fabs(s[j]);
        if (fabs(P->c[j]) > cinf) cinf = fabs(P->c[j]);
        s[j] = s[j] + P->c[j];
        if (fabs(s[j]) > sinf) sinf = fabs(s[j]);
        s2 += s[j] * s[j];
        c2 += P->c[j] * P->c[j];
        ctx += P->c[j] * P->x[j];
        x2 += P->x[j] * P->x[j];
    }
    double btl = 0;
    for (int64_t i = 0; i < m; i++) btl += P->b[i] * P->lam[i];
    orc_proj_K(P, s, ps);
    orc_proj_K(P, P->x, px);
    double ds2 = 0, dx2 = 0, dsinf = 0, dxinf = 0, xinf = 0;
    for (int64_t j = 0; j < n; j++) {
        ds2 += (s[j] - ps[j]) * (s[j] - ps[j]);
        dx2 += (P->x[j] - px[j]) * (P->x[j] - px[j]);
        if (fabs(s[j] - ps[j]) > dsinf) dsinf = fabs(s[j] - ps[j]);
        if (fabs(P->x[j] - px[j]) > dxinf) dxinf = fabs(P->x[j] - px[j]);
        if (fabs(P->x[j]) > xinf) xinf = fabs(P->x[j]);
    }
    double nrp = sqrt(rp2), nb = sqrt(b2), nds = sqrt(ds2), nc = sqrt(c2), ndx = sqrt(dx2), nx = sqrt(x2);
    out[0] = nrp / (1.0 + nb);
    out[1] = nds / (1.0 + nc);
    out[2] = ndx / (1.0 + nx);
    out[3] = fabs(ctx + btl) / (1.0 + fabs(ctx) + fabs(btl));
    double kkt = out[0];
    for (int q = 1; q < 4; q++) if (out[q] > kkt) kkt = out[q];
    out[4] = kkt;
    out[5] = ctx;
    out[6] = -btl;
    out[7] = nrp; out[8] = nb; out[9] = ndx; out[10] = nx;
    out[11] = nds; out[12] = nc; out[13] = sqrt(s2);
    out[14] = rpinf; out[15] = axinf; out[16] = binf;
    out[17] = sinf; out[18] = atlinf; out[19] = cinf;
    out[20] = xinf; out[21] = dxinf; out[22] = dsinf;
    free(Ax); free(s); free(ps); free(px);
}
