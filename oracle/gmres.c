/*
 * gmres.c -- oracle GMRES(m), deflated and augmented recycling, and GMRES-IR
 * (TEST INFRASTRUCTURE; see oracle.h).
 *
 * Paper passages followed:
 *  - Sec. 3, Eq. x_k_expression and the paragraph after it: GMRES is the
 *    minimal-residual projection with S_k = K_k(A, r0), C_k = A S_k; the
 *    iterate is not formed from the reduced system naively but through the
 *    Arnoldi relation A V_j = V_{j+1} Hbar_j and Givens rotations.
 *  - Sec. 1: GMRES(m) restarts every m steps.
 *  - Sec. 4.2, Eq. projection_guess / projection_t_s: x0 = U E^{-1} U^T b with
 *    E = U^T A U (here x0 = x_in + U E^{-1} U^T (b - A x_in), which is the
 *    paper's formula for x_in = 0).
 *  - Sec. 3.2, Eq. left_deflation and Table 1 row "deflated oblique": Krylov
 *    operator P A and start vector P r0 with P = I - A U E^{-1} U^T; M_D A U = 0.
 *  - Sec. 3.3, Eq. equivalence_oblique: with start vector r0 instead of P r0
 *    (Table 1 "augmented oblique") the iterates coincide when P r0 = r0.
 *  - Sec. 3.1, Eq. def_aug_S_space / def_aug_C_space: augmented search space
 *    S = K_j(A, r0) + span U and constraint space A S.
 *  - Left Jacobi preconditioning (not the paper's SSOR, which is sequential):
 *    GMRES on D^{-1} A x = D^{-1} b with the true-residual stopping test.
 *  - Sec. 4.2 alone (ORC_GUESS): the projection initial guess, then GMRES(m)
 *    on A itself (the "proj" column of Table 2).
 *  - Sec. 3.3, Table 1 (and Eq. P_A_variant): the other two projectors of the
 *    deflated family, orthogonal P = I - U (U^T U)^{-1} U^T and least squares
 *    P = I - A U (U^T A^T A U)^{-1} U^T A^T; Sec. 4.4, Eq. augmented_iterate:
 *    with the orthogonal projector every cycle starts from the projection guess.
 * Readings where the paper is silent: Arnoldi uses classical Gram-Schmidt with
 * one full re-orthogonalisation (CGS2); the stopping test is the true relative
 * residual ||b - A x|| / ||b|| <= rtol at the end of each cycle, with the
 * Givens estimate |g_{j+1}| ending a cycle early; happy breakdown when
 * h_{j+1,j} <= 1e-14 ||A v_j||; after each deflated cycle the coarse correction
 * x += U E^{-1} U^T (b - A x) is applied (P A x = P b alone does not give
 * A x = b); with the least-squares projector the correction is
 * x += U (W^T W)^{-1} W^T (b - A x), W = A U, for which I - A Q equals P as
 * U E^{-1} U^T does for the oblique one, so the true residual after the
 * correction is the minimised one; the orthogonal projector has no such Q and
 * keeps the oblique correction (the projection guess of the next cycle); in augmented mode the k columns A U are appended to the Arnoldi
 * basis at the end of each cycle and the least-squares problem is solved over
 * K_J(A, r) + span U; E is declared singular when an LU pivot falls below
 * 1e-13 times max(largest pivot, max_i ||u_i|| ||A u_i||), and the solve then
 * runs plain GMRES.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* round to binary32 on store when f32 is set (GMRES-IR inner solve) */
static double rd(int f32, double v) { return f32 ? (double)(float)v : v; }

static void spmv_vals(const orc_csr *A, const double *val, const double *x, double *y, int f32)
{
    for (int64_t r = 0; r < A->n; ++r) {
        double s = 0.0;
        for (int64_t k = A->rowptr[r]; k < A->rowptr[r + 1]; ++k) s += val[k] * x[A->col[k]];
        y[r] = rd(f32, s);
    }
}

int orc_spmv(const orc_csr *A, const double *x, double *y)
{
    if (!A || !x || !y) return ORC_E_ARG;
    spmv_vals(A, A->val, x, y, 0);
    return ORC_OK;
}

/* LU with partial pivoting of a k x k column-major matrix (in place).  E is
 * declared singular when a pivot falls below 1e-13 times
 * max(largest pivot, scale), scale = max_i ||u_i|| ||A u_i|| (the size E's
 * entries would have without cancellation). */
static int lu_factor(int k, double *E, int *piv, double scale)
{
    double maxp = scale, minp = INFINITY;
    for (int j = 0; j < k; ++j) {
        int p = j;
        for (int i = j + 1; i < k; ++i)
            if (fabs(E[i + j * k]) > fabs(E[p + j * k])) p = i;
        piv[j] = p;
        if (p != j)
            for (int c = 0; c < k; ++c) {
                double t = E[j + c * k]; E[j + c * k] = E[p + c * k]; E[p + c * k] = t;
            }
        double d = E[j + j * k];
        if (fabs(d) > maxp) maxp = fabs(d);
        if (fabs(d) < minp) minp = fabs(d);
        if (d == 0.0) return ORC_W_SINGULAR_COARSE;
        for (int i = j + 1; i < k; ++i) {
            E[i + j * k] /= d;
            for (int c = j + 1; c < k; ++c) E[i + c * k] -= E[i + j * k] * E[j + c * k];
        }
    }
    if (k > 0 && minp < 1e-13 * maxp) return ORC_W_SINGULAR_COARSE;
    return ORC_OK;
}

static void lu_solve(int k, const double *LU, const int *piv, double *x)
{
    for (int j = 0; j < k; ++j)
        if (piv[j] != j) { double t = x[j]; x[j] = x[piv[j]]; x[piv[j]] = t; }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) x[i] -= LU[i + j * k] * x[j];
    for (int i = k - 1; i >= 0; --i) {
        for (int j = i + 1; j < k; ++j) x[i] -= LU[i + j * k] * x[j];
        x[i] /= LU[i + i * k];
    }
}

static double coarse_scale(int64_t n, int k, const double *U, const double *W)
{
    double s = 0.0;
    for (int i = 0; i < k; ++i) {
        double t = sqrt(dot(n, U + i * n, U + i * n) * dot(n, W + i * n, W + i * n));
        if (t > s) s = t;
    }
    return s;
}

int orc_coarse_setup(const orc_csr *A, const double *U, int k, double *W, double *E)
{
    const int64_t n = A->n;
    for (int j = 0; j < k; ++j) orc_spmv(A, U + j * n, W + j * n);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) E[i + j * k] = dot(n, U + i * n, W + j * n);
    return ORC_OK;
}

int orc_apply_oblique(int64_t n, int k, const double *U, const double *W, const double *E,
                      const double *v_in, double *v_out)
{
    double *LU = malloc(sizeof(double) * k * k + 1), *c = malloc(sizeof(double) * k + 1);
    int *piv = malloc(sizeof(int) * k + 1);
    memcpy(LU, E, sizeof(double) * k * k);
    int rc = lu_factor(k, LU, piv, coarse_scale(n, k, U, W));
    for (int i = 0; i < k; ++i) c[i] = dot(n, U + i * n, v_in);
    lu_solve(k, LU, piv, c);
    for (int64_t r = 0; r < n; ++r) {
        double s = v_in[r];
        for (int i = 0; i < k; ++i) s -= W[r + i * n] * c[i];
        v_out[r] = s;
    }
    free(LU); free(c); free(piv);
    return rc;
}

int orc_apply_projector(int64_t n, int k, const double *U, const double *W, int proj,
                        const double *v_in, double *v_out)
{
    if (n < 1 || k < 1 || !U || !W || !v_in || !v_out || proj < 0 || proj > 2) return ORC_E_ARG;
    if (proj == ORC_PROJ_OBLIQUE) {
        double *E = malloc(sizeof(double) * k * k);
        if (!E) return ORC_E_NOMEM;
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < k; ++i) E[i + j * k] = dot(n, U + i * n, W + j * n);
        int rc = orc_apply_oblique(n, k, U, W, E, v_in, v_out);
        free(E);
        return rc;
    }
    const double *Y = (proj == ORC_PROJ_LS) ? W : U;
    double *G = malloc(sizeof(double) * k * k), *cv = malloc(sizeof(double) * k);
    int *piv = malloc(sizeof(int) * k);
    if (!G || !cv || !piv) { free(G); free(cv); free(piv); return ORC_E_NOMEM; }
    double sc = 0.0;
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < k; ++i) G[i + j * k] = dot(n, Y + i * n, Y + j * n);
        if (G[j + j * k] > sc) sc = G[j + j * k];
    }
    int rc = lu_factor(k, G, piv, sc);
    for (int i = 0; i < k; ++i) cv[i] = dot(n, Y + i * n, v_in);
    lu_solve(k, G, piv, cv);
    for (int64_t r = 0; r < n; ++r) {
        double s = v_in[r];
        for (int i = 0; i < k; ++i) s -= Y[r + i * n] * cv[i];
        v_out[r] = s;
    }
    free(G); free(cv); free(piv);
    return rc;
}

/* ||w .* r|| (w NULL: ||r||) */
static double wnrm2(int64_t n, const double *r, const double *w)
{
    if (!w) return nrm2(n, r);
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += (w[i] * r[i]) * (w[i] * r[i]);
    return sqrt(s);
}

/* Left Jacobi: d_i = A_ii (1 where the diagonal is absent or zero), the row-
 * scaled values D^{-1} A into vs and b / d into bs. */
static void jacobi_scale(const orc_csr *A, const double *b, double *vs, double *bs, double *d)
{
    for (int64_t i = 0; i < A->n; ++i) {
        double di = 0.0;
        for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
            if (A->col[e] == i) di += A->val[e];
        if (di == 0.0) di = 1.0;
        d[i] = di;
        for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) vs[e] = A->val[e] / di;
        bs[i] = b[i] / di;
    }
}

/* ---- the solver core, shared by the FP64 solve and the IR inner solve ---- */
typedef struct {
    const orc_csr *A;
    const double *val;      /* operator values (FP64 or binary32-rounded)          */
    int f32;                /* round stored vectors to binary32                     */
    int mode, m, start_r, k;
    const double *U, *W;    /* n x k, already rounded when f32                     */
    const double *LU;       /* LU of E = U^T A U (FP64): projection guess          */
    const int *piv;
    /* deflated family (Table 1): P w = w - Zp Gp^{-1} Yp^T w, and the cycle-end
     * correction x += U Gc^{-1} Yc^T (b - A x) */
    const double *Yp, *Zp, *LUP, *Yc, *LUC;
    const int *pivP, *pivC;
    int maxit, max_cycles;
    double tol_abs;         /* stop when ||b - A x|| <= tol_abs                     */
    double tol_in;          /* in-cycle exit: |g_{j+1}| <= tol_in                    */
    const double *wts;      /* true residual = wts .* (residual of the solved
                               system) (left Jacobi: wts = diag(A)), or NULL      */
    double *hist;
    int hist_len, hist_count;
} core_t;

/* x <- x + U G^{-1} Y^T (b - A x) */
static void correct(core_t *c, const double *Y, const double *LU, const int *piv,
                    const double *b, double *x, double *r, double *cv)
{
    const int64_t n = c->A->n;
    spmv_vals(c->A, c->val, x, r, c->f32);
    for (int64_t i = 0; i < n; ++i) r[i] = rd(c->f32, b[i] - r[i]);
    for (int i = 0; i < c->k; ++i) cv[i] = dot(n, Y + i * n, r);
    lu_solve(c->k, LU, piv, cv);
    for (int64_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int j = 0; j < c->k; ++j) s += c->U[i + j * n] * cv[j];
        x[i] = rd(c->f32, s);
    }
}

/* x <- x + U E^{-1} U^T (b - A x) : the projection guess (Eq. projection_t_s) */
static void coarse_correct(core_t *c, const double *b, double *x, double *r, double *cv)
{
    correct(c, c->U, c->LU, c->piv, b, x, r, cv);
}

/* the correction after a deflated cycle */
static void cycle_correct(core_t *c, const double *b, double *x, double *r, double *cv)
{
    correct(c, c->Yc, c->LUC, c->pivC, b, x, r, cv);
}

/* w <- P w = w - Zp Gp^{-1} Yp^T w */
static void project(core_t *c, double *w, double *cv)
{
    const int64_t n = c->A->n;
    for (int i = 0; i < c->k; ++i) cv[i] = dot(n, c->Yp + i * n, w);
    lu_solve(c->k, c->LUP, c->pivP, cv);
    for (int64_t i = 0; i < n; ++i) {
        double s = w[i];
        for (int j = 0; j < c->k; ++j) s -= c->Zp[i + j * n] * cv[j];
        w[i] = rd(c->f32, s);
    }
}

/* Factor E (in LU on entry) and, for the orthogonal and least-squares
 * projectors, the Gram matrix G = Y^T Y of Y = U or Y = W into LUP; wire the
 * projector and the cycle-end correction of the method into c.  Y, Z given to
 * c are Uv / Wv (the stored, possibly binary32-rounded copies). */
static int recycle_setup(core_t *c, int64_t n, int k, const double *U, const double *W,
                         const double *Uv, const double *Wv, int proj, double *LU, int *piv,
                         double *LUP, int *pivP)
{
    if (lu_factor(k, LU, piv, coarse_scale(n, k, U, W)) != ORC_OK) return ORC_W_SINGULAR_COARSE;
    c->U = Uv; c->W = Wv; c->LU = LU; c->piv = piv; c->k = k;
    if (proj == ORC_PROJ_ORTHOGONAL || proj == ORC_PROJ_LS) {
        const double *Y = (proj == ORC_PROJ_LS) ? W : U;
        double sc = 0.0;
        for (int j = 0; j < k; ++j) {
            for (int i = 0; i < k; ++i) LUP[i + j * k] = dot(n, Y + i * n, Y + j * n);
            if (LUP[j + j * k] > sc) sc = LUP[j + j * k];
        }
        if (lu_factor(k, LUP, pivP, sc) != ORC_OK) return ORC_W_SINGULAR_COARSE;
        const double *Yv = (proj == ORC_PROJ_LS) ? Wv : Uv;
        c->Yp = Yv; c->Zp = Yv; c->LUP = LUP; c->pivP = pivP;
        if (proj == ORC_PROJ_LS) { c->Yc = Wv; c->LUC = LUP; c->pivC = pivP; }
        else { c->Yc = Uv; c->LUC = LU; c->pivC = piv; }
    } else {
        c->Yp = Uv; c->Zp = Wv; c->LUP = LU; c->pivP = piv;
        c->Yc = Uv; c->LUC = LU; c->pivC = piv;
    }
    return ORC_OK;
}

/* classical Gram-Schmidt with one re-orthogonalisation against V[:, 0..nb-1];
 * h receives the summed coefficients. */
static void cgs2(int64_t n, int nb, const double *V, double *w, double *h, double *h2, int f32)
{
    for (int i = 0; i < nb; ++i) h[i] = dot(n, V + i * n, w);
    for (int64_t r = 0; r < n; ++r) {
        double s = w[r];
        for (int i = 0; i < nb; ++i) s -= V[r + i * n] * h[i];
        w[r] = rd(f32, s);
    }
    for (int i = 0; i < nb; ++i) h2[i] = dot(n, V + i * n, w);
    for (int64_t r = 0; r < n; ++r) {
        double s = w[r];
        for (int i = 0; i < nb; ++i) s -= V[r + i * n] * h2[i];
        w[r] = rd(f32, s);
    }
    for (int i = 0; i < nb; ++i) h[i] += h2[i];
}

/* Apply the stored rotations 0..col-1 to column col of H (leading dim ldh),
 * then make rotation col from rows (col, col+1). */
static void givens_column(double *H, int ldh, int col, double *cs, double *sn, double *g)
{
    double *hc = H + (int64_t)col * ldh;
    for (int i = 0; i < col; ++i) {
        double a = hc[i], b = hc[i + 1];
        hc[i] = cs[i] * a + sn[i] * b;
        hc[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double a = hc[col], b = hc[col + 1];
    double r = hypot(a, b);
    if (r == 0.0) { cs[col] = 1.0; sn[col] = 0.0; }
    else { cs[col] = a / r; sn[col] = b / r; }
    hc[col] = r;
    hc[col + 1] = 0.0;
    g[col + 1] = -sn[col] * g[col];
    g[col] = cs[col] * g[col];
}

static int core_solve(core_t *c, const double *b, double *x, int *iters_out, int *cycles_out,
                      double *res_out)
{
    const int64_t n = c->A->n;
    const int m = c->m, kk = (c->mode == ORC_AUGMENTED) ? c->k : 0;
    const int ncol_max = m + kk, nrow_max = ncol_max + 1;
    double *V = calloc((size_t)n * nrow_max, sizeof(double));
    double *H = calloc((size_t)nrow_max * ncol_max, sizeof(double));
    double *r = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * nrow_max), *h2 = malloc(sizeof(double) * nrow_max);
    double *cs = malloc(sizeof(double) * nrow_max), *sn = malloc(sizeof(double) * nrow_max);
    double *g = malloc(sizeof(double) * (nrow_max + 1)), *y = malloc(sizeof(double) * nrow_max);
    double *cv = malloc(sizeof(double) * (c->k + 1));
    int *aug_idx = malloc(sizeof(int) * (c->k + 1));
    if (!V || !H || !r || !w || !h || !h2 || !cs || !sn || !g || !y || !cv || !aug_idx) {
        free(V); free(H); free(r); free(w); free(h); free(h2); free(cs); free(sn);
        free(g); free(y); free(cv); free(aug_idx);
        return ORC_E_NOMEM;
    }
    int iters = 0, cycles = 0;
    spmv_vals(c->A, c->val, x, r, c->f32);
    for (int64_t i = 0; i < n; ++i) r[i] = rd(c->f32, b[i] - r[i]);
    double beta = wnrm2(n, r, c->wts);

    while (beta > c->tol_abs && iters < c->maxit && cycles < c->max_cycles) {
        ++cycles;
        /* start vector: r, or P r for the deflated oblique method */
        memcpy(w, r, sizeof(double) * n);
        if (c->mode == ORC_DEFLATED && !c->start_r) project(c, w, cv);
        double bs = nrm2(n, w);
        memset(H, 0, sizeof(double) * nrow_max * ncol_max);
        memset(g, 0, sizeof(double) * (nrow_max + 1));
        int J = 0;
        if (bs > 0.0) {
            for (int64_t i = 0; i < n; ++i) V[i] = rd(c->f32, w[i] / bs);
            g[0] = bs;
            for (int j = 0; j < m && iters < c->maxit; ++j) {
                spmv_vals(c->A, c->val, V + (int64_t)j * n, w, c->f32);
                double wn0 = nrm2(n, w);                /* ||A v_j||, breakdown reference */
                if (c->mode == ORC_DEFLATED) project(c, w, cv);
                ++iters;
                cgs2(n, j + 1, V, w, h, h2, c->f32);
                double hn = nrm2(n, w);
                double *hc = H + (int64_t)j * nrow_max;
                for (int i = 0; i <= j; ++i) hc[i] = h[i];
                hc[j + 1] = hn;
                givens_column(H, nrow_max, j, cs, sn, g);
                J = j + 1;
                if (c->hist && c->hist_count < c->hist_len) c->hist[c->hist_count++] = fabs(g[j + 1]);
                if (hn <= 1e-14 * wn0) {        /* happy breakdown: v_{j+1} := 0 */
                    for (int64_t i = 0; i < n; ++i) V[i + (int64_t)(j + 1) * n] = 0.0;
                    break;
                }
                for (int64_t i = 0; i < n; ++i) V[i + (int64_t)(j + 1) * n] = rd(c->f32, w[i] / hn);
                if (fabs(g[j + 1]) <= c->tol_in) break;
            }
        }
        /* augmentation: append A u_i as extra columns of the Arnoldi relation */
        int naug = 0;
        if (c->mode == ORC_AUGMENTED && J > 0) {
            for (int i = 0; i < c->k; ++i) {
                int col = J + naug, nb = col + 1;
                for (int64_t t = 0; t < n; ++t) w[t] = c->W[t + (int64_t)i * n];
                double wn0 = nrm2(n, w);
                if (wn0 == 0.0) continue;
                cgs2(n, nb, V, w, h, h2, c->f32);
                double hn = nrm2(n, w);
                /* candidate column after the stored rotations */
                double *hc = H + (int64_t)col * nrow_max;
                for (int t = 0; t < nb; ++t) hc[t] = h[t];
                hc[nb] = hn;
                for (int t = 0; t < col; ++t) {
                    double a = hc[t], bb = hc[t + 1];
                    hc[t] = cs[t] * a + sn[t] * bb;
                    hc[t + 1] = -sn[t] * a + cs[t] * bb;
                }
                if (hypot(hc[col], hc[col + 1]) <= 1e-14 * wn0) {   /* dependent: drop u_i */
                    memset(hc, 0, sizeof(double) * nrow_max);
                    continue;
                }
                /* re-run the full column through givens_column from unrotated data */
                for (int t = 0; t < nb; ++t) hc[t] = h[t];
                hc[nb] = hn;
                for (int t = nb + 1; t < nrow_max; ++t) hc[t] = 0.0;
                givens_column(H, nrow_max, col, cs, sn, g);
                if (hn <= 1e-14 * wn0)
                    for (int64_t t = 0; t < n; ++t) V[t + (int64_t)nb * n] = 0.0;
                else
                    for (int64_t t = 0; t < n; ++t) V[t + (int64_t)nb * n] = rd(c->f32, w[t] / hn);
                aug_idx[naug++] = i;
            }
        }
        /* least squares: R y = g, R the rotated (J+naug) x (J+naug) leading block */
        const int nc = J + naug;
        for (int i = nc - 1; i >= 0; --i) {
            double s = g[i];
            for (int j = i + 1; j < nc; ++j) s -= H[i + (int64_t)j * nrow_max] * y[j];
            double d = H[i + (int64_t)i * nrow_max];
            y[i] = (d != 0.0) ? s / d : 0.0;
        }
        for (int64_t t = 0; t < n; ++t) {
            double s = x[t];
            for (int j = 0; j < J; ++j) s += V[t + (int64_t)j * n] * y[j];
            for (int a = 0; a < naug; ++a) s += c->U[t + (int64_t)aug_idx[a] * n] * y[J + a];
            x[t] = rd(c->f32, s);
        }
        if (c->mode == ORC_DEFLATED) cycle_correct(c, b, x, r, cv);
        spmv_vals(c->A, c->val, x, r, c->f32);
        for (int64_t i = 0; i < n; ++i) r[i] = rd(c->f32, b[i] - r[i]);
        double beta_new = wnrm2(n, r, c->wts);
        if (J == 0 && !(beta_new < beta)) { beta = beta_new; break; }   /* stagnation */
        beta = beta_new;
    }
    *iters_out = iters;
    *cycles_out = cycles;
    *res_out = beta;
    free(V); free(H); free(r); free(w); free(h); free(h2); free(cs); free(sn);
    free(g); free(y); free(cv); free(aug_idx);
    return ORC_OK;
}

int orc_gmres(const orc_csr *A, const double *b, double *x, const double *U, int k,
              const orc_opts *o, orc_stats *st, double *hist, int hist_len)
{
    if (!A || !b || !x || !o || o->m < 1 || k < 0 || o->mode < ORC_PLAIN || o->mode > ORC_GUESS)
        return ORC_E_ARG;
    const int64_t n = A->n;
    orc_stats s0 = {0, 0, 0, ORC_OK, 0.0};
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        if (st) *st = s0;
        return ORC_OK;
    }
    /* left Jacobi: solve D^-1 A x = D^-1 b (the true residual is D times its residual) */
    orc_csr As = *A;
    double *vs = NULL, *bs = NULL, *dw = NULL;
    const double *bb = b;
    if (o->precond == ORC_PRECOND_JACOBI) {
        const int64_t nnz = A->rowptr[n];
        vs = malloc(sizeof(double) * (nnz + 1));
        bs = malloc(sizeof(double) * n);
        dw = malloc(sizeof(double) * n);
        if (!vs || !bs || !dw) { free(vs); free(bs); free(dw); return ORC_E_NOMEM; }
        jacobi_scale(A, b, vs, bs, dw);
        As.val = vs;
        bb = bs;
        A = &As;
    }
    core_t c;
    memset(&c, 0, sizeof c);
    c.A = A; c.val = A->val; c.f32 = 0;
    c.mode = (k > 0 && U) ? o->mode : ORC_PLAIN;
    c.m = o->m; c.start_r = o->start_r; c.k = 0;
    c.maxit = o->maxit; c.max_cycles = 1 << 30;
    c.tol_abs = o->rtol * bnorm;
    c.tol_in = dw ? o->rtol * nrm2(n, bb) : c.tol_abs;
    c.wts = dw;
    c.hist = hist; c.hist_len = hist ? hist_len : 0;
    double *W = NULL, *LU = NULL, *LUP = NULL, *cv = NULL, *r = NULL;
    int *piv = NULL, *pivP = NULL;
    int status = ORC_OK;
    if (c.mode != ORC_PLAIN) {
        W = malloc(sizeof(double) * n * k);
        LU = malloc(sizeof(double) * k * k);
        LUP = malloc(sizeof(double) * k * k);
        piv = malloc(sizeof(int) * k);
        pivP = malloc(sizeof(int) * k);
        cv = malloc(sizeof(double) * k);
        r = malloc(sizeof(double) * n);
        orc_coarse_setup(A, U, k, W, LU);
        if (recycle_setup(&c, n, k, U, W, U, W, o->proj, LU, piv, LUP, pivP) != ORC_OK) {
            status = ORC_W_SINGULAR_COARSE;
            c.mode = ORC_PLAIN;
            c.k = 0;
        } else {
            coarse_correct(&c, bb, x, r, cv);     /* projection initial guess */
        }
    }
    int iters, cycles;
    double res;
    int rc = core_solve(&c, bb, x, &iters, &cycles, &res);
    free(W); free(LU); free(LUP); free(piv); free(pivP); free(cv); free(r);
    free(vs); free(bs); free(dw);
    if (rc) return rc;
    if (hist) for (int i = 0; i < c.hist_count; ++i) hist[i] /= bnorm;
    if (status == ORC_OK && res > o->rtol * bnorm) status = ORC_W_NOT_CONVERGED;
    if (st) {
        st->iters = iters; st->cycles = cycles; st->k_used = c.k;
        st->status = status; st->true_relres = res / bnorm;
    }
    return status;
}

int orc_gmres_ir(const orc_csr *A, const double *b, double *x, const double *U, int k,
                 const orc_opts *o, double inner_rtol, int inner_cycles,
                 int max_refinements, orc_stats *st, int *refinements)
{
    if (!A || !b || !x || !o || o->m < 1 || k < 0) return ORC_E_ARG;
    if (o->precond != ORC_PRECOND_NONE) return ORC_E_ARG;   /* Jacobi: binary64 solves only */
    if (o->mode < ORC_PLAIN || o->mode > ORC_GUESS) return ORC_E_ARG;
    const int64_t n = A->n, nnz = A->rowptr[n];
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        if (st) { st->iters = 0; st->cycles = 0; st->k_used = 0; st->status = 0; st->true_relres = 0; }
        if (refinements) *refinements = 0;
        return ORC_OK;
    }
    int mode = (k > 0 && U) ? o->mode : ORC_PLAIN, status = ORC_OK;
    double *Af = malloc(sizeof(double) * nnz), *r = malloc(sizeof(double) * n);
    double *d = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    double *LU = NULL, *LUP = NULL, *Uf = NULL, *Wf = NULL, *cv = NULL;
    int *piv = NULL, *pivP = NULL;
    for (int64_t i = 0; i < nnz; ++i) Af[i] = (double)(float)A->val[i];
    core_t c;
    memset(&c, 0, sizeof c);
    c.A = A; c.val = Af; c.f32 = 1; c.m = o->m; c.start_r = o->start_r;
    c.maxit = o->maxit; c.max_cycles = inner_cycles;
    if (mode != ORC_PLAIN) {
        LU = malloc(sizeof(double) * k * k);
        LUP = malloc(sizeof(double) * k * k); pivP = malloc(sizeof(int) * k);
        piv = malloc(sizeof(int) * k); cv = malloc(sizeof(double) * k);
        Uf = malloc(sizeof(double) * n * k); Wf = malloc(sizeof(double) * n * k);
        /* U and W = A U are used only inside the binary32 inner solve: W is
         * formed from the binary32 operator and U and stored in binary32, and
         * E = U^T W (and the projector's Gram matrix) is accumulated in FP64
         * from the stored columns, so that the inner projector is exact for
         * the vectors it is applied with; E and its LU stay FP64 */
        for (int64_t i = 0; i < n * k; ++i) Uf[i] = (double)(float)U[i];
        for (int j = 0; j < k; ++j) spmv_vals(A, Af, Uf + (int64_t)j * n, Wf + (int64_t)j * n, 1);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < k; ++i) LU[i + j * k] = dot(n, Uf + (int64_t)i * n, Wf + (int64_t)j * n);
        if (recycle_setup(&c, n, k, Uf, Wf, Uf, Wf, o->proj, LU, piv, LUP, pivP) != ORC_OK) {
            status = ORC_W_SINGULAR_COARSE;
            mode = ORC_PLAIN;
            c.k = 0;
        } else {
            /* FP64 projection initial guess on the outer iterate
             * (x += U E^{-1} U^T (b - A x): U in FP64, E as above) */
            core_t c64 = c;
            c64.val = A->val; c64.f32 = 0; c64.U = U;
            coarse_correct(&c64, b, x, r, cv);
        }
    }
    c.mode = mode;
    int iters = 0, cycles = 0, nref = 0;
    double res = 0.0;
    for (;;) {
        orc_spmv(A, x, r);                                   /* FP64 residual */
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        res = nrm2(n, r);
        if (res <= o->rtol * bnorm || nref >= max_refinements || iters >= o->maxit) break;
        ++nref;
        double rf_norm = 0.0;
        for (int64_t i = 0; i < n; ++i) { r[i] = (double)(float)r[i]; rf_norm += r[i] * r[i]; }
        rf_norm = sqrt(rf_norm);
        memset(d, 0, sizeof(double) * n);
        /* inner_rtol of the current residual, but no further than half the
         * outer target: the refinement loop checks the binary64 residual */
        c.tol_abs = fmax(inner_rtol * rf_norm, 0.5 * o->rtol * bnorm);
        c.tol_in = c.tol_abs;       /* the Givens estimate ends a cycle early, as in every solve */
        c.maxit = o->maxit - iters;
        int it, cy;
        double rr;
        if (mode != ORC_PLAIN) coarse_correct(&c, r, d, tmp, cv);   /* inner guess */
        core_solve(&c, r, d, &it, &cy, &rr);
        iters += it; cycles += cy;
        for (int64_t i = 0; i < n; ++i) x[i] += d[i];                /* FP64 update */
    }
    if (status == ORC_OK && res > o->rtol * bnorm) status = ORC_W_NOT_CONVERGED;
    if (st) {
        st->iters = iters; st->cycles = cycles; st->k_used = (mode != ORC_PLAIN) ? k : 0;
        st->status = status; st->true_relres = res / bnorm;
    }
    if (refinements) *refinements = nref;
    free(Af); free(r); free(d); free(tmp); free(LU); free(LUP); free(piv); free(pivP);
    free(Uf); free(Wf); free(cv);
    return status;
}
