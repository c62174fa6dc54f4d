/*
 * sequence.c -- oracle time-step sequence with Algorithm 1 (TEST
 * INFRASTRUCTURE; see oracle.h).
 *
 * Sec. 2: the systems A_i = A(t_i, x_{i-1}), b_i = b(t_i, x_{i-1}) arrive one
 * at a time.  Algorithm 1: solve A_i x_i = b_i with a recycling scheme, store
 * x_i in the window X of the m most recent solutions (the oldest column leaves
 * when it is full), and every ell steps replace the recycle space by the s
 * leading left singular vectors of X.
 * Readings: the window holds exactly `window` solver outputs (u0 is not one);
 * before it is full all c stored columns are used with k_eff = min(k, c);
 * singular values below rel_drop * sigma_1 are dropped; step 1 runs plain;
 * with a recycle space the solve starts from x_in = 0 (so the initial guess is
 * the paper's x0 = U E^{-1} U^T b), without one from the previous solution.
 * With cfg->precision = 1 every solve is the mixed-precision iterative
 * refinement of orc_gmres_ir (binary32 inner recycled GMRES, FP64 residual and
 * update) with the same recycle space.
 * With cfg->guess = g > 0, x_in is instead the extrapolation of order g
 * (Sec. 4.1) once g+1 solutions are stored (the window must hold them).
 * cfg->velocity / nmodes select Sec. 6.1's own benchmark (cellular velocity,
 * random forcing with the coefficients of step i at forcing[(i-1) nmodes]).
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>
#include <time.h>

static double now_s(void)
{
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

int orc_sequence(const orc_seq_cfg *cfg, const double *u0, double *x_all, double *x_final,
                 int *iters, int *k_used, double *relres, int *status)
{
    return orc_sequence_timed(cfg, u0, x_all, x_final, iters, k_used, relres, status, NULL, NULL);
}

int orc_sequence_timed(const orc_seq_cfg *cfg, const double *u0, double *x_all, double *x_final,
                       int *iters, int *k_used, double *relres, int *status,
                       double *step_seconds, int *refinements)
{
    if (!cfg || !u0 || cfg->steps < 1 || cfg->window < 1 || cfg->nmodes < 0 ||
        (cfg->nmodes > 0 && !cfg->forcing))
        return ORC_E_ARG;
    const int p = cfg->p, N = cfg->N;
    const int64_t n = orc_fe_ndofs(p, N);
    const int64_t nnz = orc_fe_pattern(p, N, 1, NULL, NULL);
    int64_t *rowptr = malloc(sizeof(int64_t) * (n + 1));
    int32_t *col = malloc(sizeof(int32_t) * nnz);
    double *val = malloc(sizeof(double) * nnz), *b = malloc(sizeof(double) * n);
    double *u = malloc(sizeof(double) * n), *x = malloc(sizeof(double) * n);
    double *X = malloc(sizeof(double) * n * cfg->window);
    double *U = malloc(sizeof(double) * n * (cfg->k > 0 ? cfg->k : 1));
    double *vf = malloc(sizeof(double) * 3 * n);     /* nodal bx | by | f */
    if (!rowptr || !col || !val || !b || !u || !x || !X || !U || !vf) {
        free(rowptr); free(col); free(val); free(b); free(u); free(x); free(X); free(U); free(vf);
        return ORC_E_NOMEM;
    }
    double *bxn = vf, *byn = vf + n, *fn = vf + 2 * n;
    if (cfg->velocity == 1) {
        orc_fe_paper_velocity(p, N, bxn, byn);
    } else {
        for (int64_t r = 0; r < n; ++r) { bxn[r] = cfg->bx; byn[r] = cfg->by; }
    }
    orc_fe_pattern(p, N, 1, rowptr, col);
    orc_csr A = {n, rowptr, col, val};
    memcpy(u, u0, sizeof(double) * n);
    int count = 0, k_eff = 0, rc = ORC_OK;
    for (int i = 1; i <= cfg->steps; ++i) {
        double t0 = now_s();
        if (cfg->velocity == 0 && cfg->nmodes == 0) {
            rc = orc_fe_step_system(p, N, cfg->eps, cfg->dt, cfg->bx, cfg->by, u, rowptr, col, val, b);
        } else {
            if (cfg->nmodes > 0)
                orc_fe_paper_forcing(p, N, cfg->nmodes, cfg->forcing + (int64_t)(i - 1) * cfg->nmodes,
                                     cfg->fC, fn);
            rc = orc_fe_step_system_field(p, N, cfg->eps, cfg->dt, bxn, byn,
                                          cfg->nmodes > 0 ? fn : NULL, u, rowptr, col, val, b);
        }
        if (rc) break;
        int use_u = (cfg->mode != ORC_PLAIN && k_eff > 0);
        if (use_u) memset(x, 0, sizeof(double) * n);
        else memcpy(x, u, sizeof(double) * n);
        if (cfg->guess > 0 && count >= cfg->guess + 1) {
            /* x_{i-1}, x_{i-2}, ... are window columns count-1, count-2, ... */
            double *P = malloc(sizeof(double) * n * (cfg->guess + 1));
            if (!P) { rc = ORC_E_NOMEM; break; }
            for (int j = 0; j <= cfg->guess; ++j)
                memcpy(P + (int64_t)j * n, X + (int64_t)(count - 1 - j) * n, sizeof(double) * n);
            orc_extrapolate(n, cfg->guess + 1, P, n, x);
            free(P);
        }
        orc_opts o = {cfg->mode, cfg->m, cfg->rtol, cfg->maxit, 0, cfg->proj, cfg->precond};
        orc_stats st;
        int s, nref = 0;
        if (cfg->precision == 1)
            s = orc_gmres_ir(&A, b, x, use_u ? U : NULL, use_u ? k_eff : 0, &o, cfg->inner_rtol,
                             cfg->inner_cycles, cfg->max_refinements, &st, &nref);
        else
            s = orc_gmres(&A, b, x, use_u ? U : NULL, use_u ? k_eff : 0, &o, &st, NULL, 0);
        if (refinements) refinements[i - 1] = nref;
        if (s < 0) { rc = s; break; }
        if (iters) iters[i - 1] = st.iters;
        if (k_used) k_used[i - 1] = st.k_used;
        if (relres) relres[i - 1] = st.true_relres;
        if (status) status[i - 1] = st.status;
        if (x_all) memcpy(x_all + (int64_t)(i - 1) * n, x, sizeof(double) * n);
        /* FIFO window, oldest column first */
        if (count == cfg->window) {
            memmove(X, X + n, sizeof(double) * n * (cfg->window - 1));
            --count;
        }
        memcpy(X + (int64_t)count * n, x, sizeof(double) * n);
        ++count;
        if (cfg->mode != ORC_PLAIN && cfg->k > 0 && i % cfg->ell == 0) {
            rc = orc_recycle_from_window(n, count, X, cfg->k, cfg->select_smallest,
                                         cfg->rel_drop, U, &k_eff);
            if (rc) break;
        }
        memcpy(u, x, sizeof(double) * n);
        if (step_seconds) step_seconds[i - 1] = now_s() - t0;
    }
    if (x_final && rc == ORC_OK) memcpy(x_final, u, sizeof(double) * n);
    free(rowptr); free(col); free(val); free(b); free(u); free(x); free(X); free(U); free(vf);
    return rc;
}

int orc_extrapolate(int64_t n, int s, const double *P, int64_t ldp, double *x0)
{
    if (n < 0 || s < 1 || s > 4 || !P || !x0) return ORC_E_ARG;
    /* binomial coefficients C(s, j) with alternating signs */
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double binom = 1.0;
    for (int j = 1; j <= s; ++j) {
        binom = binom * (double)(s - j + 1) / (double)j;
        c[j] = (j % 2 == 1) ? binom : -binom;
    }
    for (int64_t r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int j = 1; j <= s; ++j) acc += c[j] * P[r + (int64_t)(j - 1) * ldp];
        x0[r] = acc;
    }
    return ORC_OK;
}
