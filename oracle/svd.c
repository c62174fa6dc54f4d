/*
 * svd.c -- oracle thin SVD of the snapshot window (TEST INFRASTRUCTURE; see
 * oracle.h).
 *
 * Sec. 5.2 and Algorithm 1: the m previous solutions are stored column-wise in
 * X; its SVD X = Psi Sigma Phi^T is computed and the s left singular vectors
 * with the largest (or smallest) singular values span the recycle space.  By
 * the Schmidt-Eckart-Young theorem (Eq. best_rank_s / opt_svd) the leading s
 * modes give the best rank-s approximation of X in the Frobenius norm.
 *
 * Route (textbook, no LAPACK): Householder QR X = Q R, one-sided (Hestenes)
 * Jacobi on the c x c factor R until every column pair is orthogonal to
 * 1e-15 relative, accumulating the right singular vectors Phi; singular values
 * as the column norms, left singular vectors of X = Q times those of R.
 * Sorted by descending sigma, ties by index.
 *
 * The recycle space is formed from the identity psi_i = X phi_i / sigma_i and
 * then orthonormalised (modified Gram-Schmidt, twice) inside its own span:
 * Algorithm 1 takes singular modes of X_m, which lie in range(X_m), and this
 * form keeps V_s there to rounding, whereas Q Psi_R carries the QR's backward
 * error (relative eps sigma_1 / sigma_i) out of range(X_m) in the trailing
 * directions.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

int orc_svd_left(int64_t n, int c, const double *X, double *sigma, double *Psi)
{
    return orc_svd_full(n, c, X, sigma, Psi, NULL);
}

int orc_svd_full(int64_t n, int c, const double *X, double *sigma, double *Psi, double *Phi)
{
    if (n < 1 || c < 1 || n < c) return ORC_E_ARG;
    double *A = malloc(sizeof(double) * n * c);       /* working copy, then reflectors */
    double *R = calloc((size_t)c * c, sizeof(double));
    double *B = malloc(sizeof(double) * c * c);
    double *F = calloc((size_t)c * c, sizeof(double));     /* accumulated rotations */
    double *Y = calloc((size_t)n * c, sizeof(double));
    double *tau = malloc(sizeof(double) * c);
    int *ord = malloc(sizeof(int) * c);
    double *sg = malloc(sizeof(double) * c);
    if (!A || !R || !B || !F || !Y || !tau || !ord || !sg) {
        free(A); free(R); free(B); free(F); free(Y); free(tau); free(ord); free(sg);
        return ORC_E_NOMEM;
    }
    for (int i = 0; i < c; ++i) F[i + i * c] = 1.0;
    memcpy(A, X, sizeof(double) * n * c);
    /* Householder QR: H_j = I - tau_j v_j v_j^T with v_j stored in A[j:, j], v_j[0] = 1 */
    for (int j = 0; j < c; ++j) {
        double *a = A + (int64_t)j * n;
        double s = 0.0;
        for (int64_t i = j; i < n; ++i) s += a[i] * a[i];
        double nrm = sqrt(s);
        if (nrm == 0.0) { tau[j] = 0.0; R[j + j * c] = 0.0; continue; }
        double alpha = (a[j] > 0.0) ? -nrm : nrm;
        double v0 = a[j] - alpha;
        for (int64_t i = j + 1; i < n; ++i) a[i] /= v0;
        a[j] = 1.0;
        double vtv = 1.0;
        for (int64_t i = j + 1; i < n; ++i) vtv += a[i] * a[i];
        tau[j] = 2.0 / vtv;
        for (int q = j + 1; q < c; ++q) {
            double *b = A + (int64_t)q * n;
            double d = 0.0;
            for (int64_t i = j; i < n; ++i) d += a[i] * b[i];
            d *= tau[j];
            for (int64_t i = j; i < n; ++i) b[i] -= d * a[i];
        }
        R[j + j * c] = alpha;
        for (int q = j + 1; q < c; ++q) R[j + q * c] = A[j + (int64_t)q * n];
    }
    /* one-sided Jacobi on the columns of R */
    memcpy(B, R, sizeof(double) * c * c);
    for (int sweep = 0; sweep < 80; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < c - 1; ++p)
            for (int q = p + 1; q < c; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < c; ++i) {
                    al += B[i + p * c] * B[i + p * c];
                    be += B[i + q * c] * B[i + q * c];
                    ga += B[i + p * c] * B[i + q * c];
                }
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                rotated = 1;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < c; ++i) {
                    double bp = B[i + p * c], bq = B[i + q * c];
                    B[i + p * c] = cs * bp - sn * bq;
                    B[i + q * c] = sn * bp + cs * bq;
                    double fp = F[i + p * c], fq = F[i + q * c];
                    F[i + p * c] = cs * fp - sn * fq;
                    F[i + q * c] = sn * fp + cs * fq;
                }
            }
        if (!rotated) break;
    }
    for (int j = 0; j < c; ++j) {
        double s = 0.0;
        for (int i = 0; i < c; ++i) s += B[i + j * c] * B[i + j * c];
        sg[j] = sqrt(s);
        ord[j] = j;
    }
    /* stable insertion sort, descending */
    for (int i = 1; i < c; ++i) {
        int o = ord[i], j = i - 1;
        while (j >= 0 && sg[ord[j]] < sg[o]) { ord[j + 1] = ord[j]; --j; }
        ord[j + 1] = o;
    }
    /* Y = [Psi_R; 0], then Psi = H_0 ... H_{c-1} Y */
    for (int jj = 0; jj < c; ++jj) {
        int j = ord[jj];
        sigma[jj] = sg[j];
        if (sg[j] > 0.0)
            for (int i = 0; i < c; ++i) Y[i + (int64_t)jj * n] = B[i + j * c] / sg[j];
        if (Phi)
            for (int i = 0; i < c; ++i) Phi[i + jj * c] = F[i + j * c];
    }
    for (int j = c - 1; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
        const double *v = A + (int64_t)j * n;
        for (int q = 0; q < c; ++q) {
            double *y = Y + (int64_t)q * n;
            double d = 0.0;
            for (int64_t i = j; i < n; ++i) d += v[i] * y[i];
            d *= tau[j];
            for (int64_t i = j; i < n; ++i) y[i] -= d * v[i];
        }
    }
    for (int jj = 0; jj < c; ++jj)
        if (sigma[jj] == 0.0) memset(Y + (int64_t)jj * n, 0, sizeof(double) * n);
    memcpy(Psi, Y, sizeof(double) * n * c);
    free(A); free(R); free(B); free(F); free(Y); free(tau); free(ord); free(sg);
    return ORC_OK;
}

int orc_recycle_from_window(int64_t n, int c, const double *X, int k, int select_smallest,
                            double rel_drop, double *U, int *k_eff)
{
    if (c < 1 || k < 0) { if (k_eff) *k_eff = 0; return c < 1 ? ORC_OK : ORC_E_ARG; }
    double *sigma = malloc(sizeof(double) * c), *Psi = malloc(sizeof(double) * n * c);
    double *Phi = malloc(sizeof(double) * c * c);
    if (!sigma || !Psi || !Phi) { free(sigma); free(Psi); free(Phi); return ORC_E_NOMEM; }
    int rc = orc_svd_full(n, c, X, sigma, Psi, Phi);
    if (rc) { free(sigma); free(Psi); free(Phi); return rc; }
    int nz = 0;                                   /* numerically nonzero modes */
    while (nz < c && sigma[nz] > 0.0 && sigma[nz] >= rel_drop * sigma[0]) ++nz;
    int ke = k < nz ? k : nz;
    int first = select_smallest ? nz - ke : 0;
    /* psi_l = X phi_l / sigma_l */
    for (int l = 0; l < ke; ++l) {
        const double *ph = Phi + (int64_t)(first + l) * c;
        const double s = sigma[first + l];
        double *u = U + (int64_t)l * n;
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int m = 0; m < c; ++m) acc += X[i + (int64_t)m * n] * ph[m];
            u[i] = acc / s;
        }
    }
    /* modified Gram-Schmidt, twice, inside span U */
    for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < ke; ++j) {
            double *uj = U + (int64_t)j * n;
            for (int i = 0; i < j; ++i) {
                const double *ui = U + (int64_t)i * n;
                double d = 0.0;
                for (int64_t t = 0; t < n; ++t) d += ui[t] * uj[t];
                for (int64_t t = 0; t < n; ++t) uj[t] -= d * ui[t];
            }
            double nr = 0.0;
            for (int64_t t = 0; t < n; ++t) nr += uj[t] * uj[t];
            nr = sqrt(nr);
            for (int64_t t = 0; t < n; ++t) uj[t] /= nr;
        }
    *k_eff = ke;
    free(sigma); free(Psi); free(Phi);
    return ORC_OK;
}
