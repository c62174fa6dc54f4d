/*
 * fe.c -- oracle finite-element system of the paper's benchmark (TEST
 * INFRASTRUCTURE; see oracle.h).
 *
 * Sec. 2, Eq. linear_pde / def_Axb: one implicit time step of a linearised PDE
 * gives A = beta_0 M + L(u~) and b = F + sum beta_a M u^{k-a}.  Sec. 6.1 gives
 * the discrete problem for implicit Euler with the convection coefficient
 * lagged at u^{n-1} (the D_u L term is dropped, Sec. 2):
 *   (1/dt)(v, u^n - u^{n-1}) + eps (grad v, grad u^n)
 *       + (v, u^{n-1} beta . grad u^n) = (v, f).
 * The paper's own benchmark (Sec. 6.1) takes beta as the cellular field
 * b = (-sin(pi x) cos(pi y), cos(pi x) sin(pi y)) through its nodal interpolant
 * and a forcing f of 16 random Laplace modes through its nodal interpolant
 * (orc_fe_paper_velocity / orc_fe_paper_forcing / orc_fe_step_system_field).
 * Q_p Lagrange elements on a uniform N x N grid of [0,1]^2 with Gauss-Lobatto
 * nodes in each cell, lexicographic dof numbering (x fastest) on the
 * (pN+1)^2 node lattice, (p+1)^2 Gauss points per cell.  Homogeneous
 * Dirichlet data: boundary rows become identity rows with b_i = 0 and boundary
 * columns are dropped from interior rows.
 *
 * Everything is computed the plain way: element loop, quadrature loop, scatter
 * into CSR by binary search of the column.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Legendre P_n(t) and P_n'(t) on [-1,1] by the three-term recurrence. */
static void legendre(int n, double t, double *P, double *dP)
{
    double p0 = 1.0, p1 = t;
    if (n == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
    }
    *P = p1;
    /* (1 - t^2) P_n' = n (P_{n-1} - t P_n) */
    *dP = n * (p0 - t * p1) / (1.0 - t * t);
}

int orc_gauss_rule(int q, double *x, double *w)
{
    if (q < 1 || q > 64) return ORC_E_ARG;
    for (int i = 0; i < q; ++i) {
        double t = cos(M_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(q, t, &P, &dP);
            double dt = P / dP;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double P, dP;
        legendre(q, t, &P, &dP);
        /* ascending order on [0,1] */
        x[q - 1 - i] = 0.5 * (t + 1.0);
        w[q - 1 - i] = 1.0 / ((1.0 - t * t) * dP * dP);   /* 2/(...) halved */
    }
    return ORC_OK;
}

int orc_gll_nodes(int p, double *xi)
{
    if (p < 1 || p > 32) return ORC_E_ARG;
    xi[0] = 0.0;
    xi[p] = 1.0;
    /* interior nodes: roots of P_p'(t), found by Newton with P_p'' from
     * Legendre's equation (1-t^2)P'' = 2 t P' - p(p+1) P. */
    for (int i = 1; i < p; ++i) {
        double t = -cos(M_PI * i / p);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(p, t, &P, &dP);
            double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
            double dt = dP / d2P;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        xi[i] = 0.5 * (t + 1.0);
    }
    return ORC_OK;
}

int orc_lagrange(int p, const double *nodes, double x, double *phi, double *dphi)
{
    for (int a = 0; a <= p; ++a) {
        double v = 1.0;
        for (int b = 0; b <= p; ++b)
            if (b != a) v *= (x - nodes[b]) / (nodes[a] - nodes[b]);
        phi[a] = v;
        double d = 0.0;
        for (int c = 0; c <= p; ++c) {
            if (c == a) continue;
            double t = 1.0 / (nodes[a] - nodes[c]);
            for (int b = 0; b <= p; ++b)
                if (b != a && b != c) t *= (x - nodes[b]) / (nodes[a] - nodes[b]);
            d += t;
        }
        dphi[a] = d;
    }
    return ORC_OK;
}

int64_t orc_fe_ndofs(int p, int N)
{
    int64_t L = (int64_t)p * N + 1;
    return L * L;
}

int orc_fe_node_coords(int p, int N, double *x, double *y)
{
    if (p < 1 || N < 1) return ORC_E_ARG;
    double xi[33];
    orc_gll_nodes(p, xi);
    int64_t L = (int64_t)p * N + 1;
    double h = 1.0 / N;
    double *c1 = malloc(sizeof(double) * L);
    if (!c1) return ORC_E_NOMEM;
    for (int64_t I = 0; I < L; ++I) {
        int64_t cell = I / p, a = I % p;
        c1[I] = (cell == N) ? 1.0 : (cell + xi[a]) * h;
    }
    for (int64_t Iy = 0; Iy < L; ++Iy)
        for (int64_t Ix = 0; Ix < L; ++Ix) {
            x[Iy * L + Ix] = c1[Ix];
            y[Iy * L + Ix] = c1[Iy];
        }
    free(c1);
    return ORC_OK;
}

/* 1D coupling range of lattice node I: all nodes that share a cell with it. */
static void range1d(int p, int N, int64_t I, int64_t *lo, int64_t *hi)
{
    int64_t L = (int64_t)p * N + 1;
    if (I % p == 0) {           /* cell vertex: in cells I/p - 1 and I/p */
        *lo = I - p < 0 ? 0 : I - p;
        *hi = I + p > L - 1 ? L - 1 : I + p;
    } else {                    /* inside cell I/p only */
        *lo = (I / p) * p;
        *hi = *lo + p;
    }
}

static int on_boundary(int p, int N, int64_t dof)
{
    int64_t L = (int64_t)p * N + 1;
    int64_t Ix = dof % L, Iy = dof / L;
    return Ix == 0 || Iy == 0 || Ix == L - 1 || Iy == L - 1;
}

int64_t orc_fe_pattern(int p, int N, int dirichlet, int64_t *rowptr, int32_t *col)
{
    if (p < 1 || N < 1) return ORC_E_ARG;
    int64_t L = (int64_t)p * N + 1, n = L * L, nnz = 0;
    if (rowptr) rowptr[0] = 0;
    for (int64_t r = 0; r < n; ++r) {
        int64_t Ix = r % L, Iy = r / L;
        if (dirichlet && on_boundary(p, N, r)) {
            if (col) col[nnz] = (int32_t)r;
            ++nnz;
        } else {
            int64_t xl, xh, yl, yh;
            range1d(p, N, Ix, &xl, &xh);
            range1d(p, N, Iy, &yl, &yh);
            for (int64_t jy = yl; jy <= yh; ++jy)
                for (int64_t jx = xl; jx <= xh; ++jx) {
                    int64_t c = jy * L + jx;
                    if (dirichlet && on_boundary(p, N, c)) continue;
                    if (col) col[nnz] = (int32_t)c;
                    ++nnz;
                }
        }
        if (rowptr) rowptr[r + 1] = nnz;
    }
    return nnz;
}

static int64_t find_col(const int64_t *rowptr, const int32_t *col, int64_t r, int64_t c)
{
    int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (col[mid] == c) return mid;
        if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Tabulated 1D basis at the Gauss points of one cell (reference coordinates). */
typedef struct {
    int p, q;
    double gx[33], gw[33];
    double phi[33][33], dphi[33][33];   /* [gauss point][basis] */
} tab1d;

static void make_tab(int p, tab1d *t)
{
    double xi[33];
    t->p = p;
    t->q = p + 1;
    orc_gll_nodes(p, xi);
    orc_gauss_rule(t->q, t->gx, t->gw);
    for (int g = 0; g < t->q; ++g) orc_lagrange(p, xi, t->gx[g], t->phi[g], t->dphi[g]);
}

/* Shared by the constant-velocity and the nodal-velocity assembly: with
 * bxn/byn set, the velocity at a quadrature point is its nodal interpolant
 * sum_l b_l phi_l; otherwise (bx, by). */
static int assemble_impl(int p, int N, double cm, double ck, double cn, double bx, double by,
                         const double *bxn, const double *byn, const double *u, int dirichlet,
                         const int64_t *rowptr, const int32_t *col, double *val)
{
    if (p < 1 || p > 32 || N < 1) return ORC_E_ARG;
    tab1d t;
    make_tab(p, &t);
    const int nl = (p + 1) * (p + 1), q = t.q;
    const int64_t L = (int64_t)p * N + 1, n = L * L;
    const double h = 1.0 / N;
    memset(val, 0, sizeof(double) * rowptr[n]);
    double *Ae = malloc(sizeof(double) * nl * nl);
    int64_t *gdof = malloc(sizeof(int64_t) * nl);
    if (!Ae || !gdof) { free(Ae); free(gdof); return ORC_E_NOMEM; }
    int rc = ORC_OK;
    for (int cy = 0; cy < N && rc == ORC_OK; ++cy)
        for (int cx = 0; cx < N && rc == ORC_OK; ++cx) {
            for (int b = 0; b <= p; ++b)
                for (int a = 0; a <= p; ++a)
                    gdof[b * (p + 1) + a] = ((int64_t)cy * p + b) * L + ((int64_t)cx * p + a);
            memset(Ae, 0, sizeof(double) * nl * nl);
            for (int gy = 0; gy < q; ++gy)
                for (int gx = 0; gx < q; ++gx) {
                    double W = t.gw[gx] * t.gw[gy] * h * h;
                    /* u (and a nodal velocity) at this quadrature point */
                    double uq = 0.0, bxq = bx, byq = by;
                    if (u && cn != 0.0)
                        for (int l = 0; l < nl; ++l) {
                            int la = l % (p + 1), lb = l / (p + 1);
                            uq += u[gdof[l]] * t.phi[gx][la] * t.phi[gy][lb];
                        }
                    if (bxn && cn != 0.0) {
                        bxq = 0.0;
                        byq = 0.0;
                        for (int l = 0; l < nl; ++l) {
                            int la = l % (p + 1), lb = l / (p + 1);
                            bxq += bxn[gdof[l]] * t.phi[gx][la] * t.phi[gy][lb];
                            byq += byn[gdof[l]] * t.phi[gx][la] * t.phi[gy][lb];
                        }
                    }
                    for (int i = 0; i < nl; ++i) {
                        int ia = i % (p + 1), ib = i / (p + 1);
                        double phii = t.phi[gx][ia] * t.phi[gy][ib];
                        double dxi = t.dphi[gx][ia] * t.phi[gy][ib] / h;
                        double dyi = t.phi[gx][ia] * t.dphi[gy][ib] / h;
                        for (int j = 0; j < nl; ++j) {
                            int ja = j % (p + 1), jb = j / (p + 1);
                            double phij = t.phi[gx][ja] * t.phi[gy][jb];
                            double dxj = t.dphi[gx][ja] * t.phi[gy][jb] / h;
                            double dyj = t.phi[gx][ja] * t.dphi[gy][jb] / h;
                            double v = cm * phii * phij + ck * (dxi * dxj + dyi * dyj)
                                     + cn * phii * uq * (bxq * dxj + byq * dyj);
                            Ae[i * nl + j] += W * v;       /* row i (test), column j (trial) */
                        }
                    }
                }
            for (int i = 0; i < nl; ++i) {
                int64_t r = gdof[i];
                if (dirichlet && on_boundary(p, N, r)) continue;
                for (int j = 0; j < nl; ++j) {
                    int64_t c = gdof[j];
                    if (dirichlet && on_boundary(p, N, c)) continue;
                    int64_t pos = find_col(rowptr, col, r, c);
                    if (pos < 0) { rc = ORC_E_PATTERN; break; }
                    val[pos] += Ae[i * nl + j];
                }
            }
        }
    if (rc == ORC_OK && dirichlet)
        for (int64_t r = 0; r < n; ++r)
            if (on_boundary(p, N, r)) {
                int64_t pos = find_col(rowptr, col, r, r);
                if (pos < 0) { rc = ORC_E_PATTERN; break; }
                val[pos] = 1.0;
            }
    free(Ae);
    free(gdof);
    return rc;
}

int orc_fe_assemble(int p, int N, double cm, double ck, double cn, double bx, double by,
                    const double *u, int dirichlet, const int64_t *rowptr,
                    const int32_t *col, double *val)
{
    return assemble_impl(p, N, cm, ck, cn, bx, by, NULL, NULL, u, dirichlet, rowptr, col, val);
}

int orc_fe_assemble_field(int p, int N, double cm, double ck, double cn, const double *bxn,
                          const double *byn, const double *u, int dirichlet,
                          const int64_t *rowptr, const int32_t *col, double *val)
{
    if (!bxn || !byn) return ORC_E_ARG;
    return assemble_impl(p, N, cm, ck, cn, 0.0, 0.0, bxn, byn, u, dirichlet, rowptr, col, val);
}

int orc_fe_load(int p, int N, orc_scalar_fn f, void *ctx, double *F)
{
    if (p < 1 || p > 32 || N < 1) return ORC_E_ARG;
    tab1d t;
    make_tab(p, &t);
    const int nl = (p + 1) * (p + 1), q = t.q;
    const int64_t L = (int64_t)p * N + 1, n = L * L;
    const double h = 1.0 / N;
    memset(F, 0, sizeof(double) * n);
    for (int cy = 0; cy < N; ++cy)
        for (int cx = 0; cx < N; ++cx)
            for (int gy = 0; gy < q; ++gy)
                for (int gx = 0; gx < q; ++gx) {
                    double W = t.gw[gx] * t.gw[gy] * h * h;
                    double fx = f ? f((cx + t.gx[gx]) * h, (cy + t.gx[gy]) * h, ctx) : 1.0;
                    for (int i = 0; i < nl; ++i) {
                        int ia = i % (p + 1), ib = i / (p + 1);
                        int64_t g = ((int64_t)cy * p + ib) * L + ((int64_t)cx * p + ia);
                        F[g] += W * fx * t.phi[gx][ia] * t.phi[gy][ib];
                    }
                }
    return ORC_OK;
}

/* b = M u_prev / dt + (v, f) with the full (not Dirichlet-reduced) mass
 * matrix; (v, f) = F(f = 1) by quadrature when fn is NULL, else M fn (the
 * load of the nodal interpolant); b_i = 0 on Dirichlet rows. */
static int step_rhs(int p, int N, double dt, const double *u_prev, const double *fn, double *b)
{
    const int64_t n = orc_fe_ndofs(p, N);
    int64_t nnzf = orc_fe_pattern(p, N, 0, NULL, NULL);
    int64_t *rp = malloc(sizeof(int64_t) * (n + 1));
    int32_t *cl = malloc(sizeof(int32_t) * nnzf);
    double *mv = malloc(sizeof(double) * nnzf);
    if (!rp || !cl || !mv) { free(rp); free(cl); free(mv); return ORC_E_NOMEM; }
    orc_fe_pattern(p, N, 0, rp, cl);
    int rc = orc_fe_assemble(p, N, 1.0, 0.0, 0.0, 0.0, 0.0, NULL, 0, rp, cl, mv);
    if (rc == ORC_OK) {
        if (!fn) orc_fe_load(p, N, NULL, NULL, b);
        for (int64_t r = 0; r < n; ++r) {
            double s = 0.0;
            for (int64_t k = rp[r]; k < rp[r + 1]; ++k) s += mv[k] * u_prev[cl[k]];
            if (fn) {
                double sf = 0.0;
                for (int64_t k = rp[r]; k < rp[r + 1]; ++k) sf += mv[k] * fn[cl[k]];
                b[r] = s / dt + sf;
            } else {
                b[r] += s / dt;
            }
            if (on_boundary(p, N, r)) b[r] = 0.0;
        }
    }
    free(rp); free(cl); free(mv);
    return rc;
}

int orc_fe_step_system(int p, int N, double eps, double dt, double bx, double by,
                       const double *u_prev, const int64_t *rowptr, const int32_t *col,
                       double *val, double *b)
{
    int rc = orc_fe_assemble(p, N, 1.0 / dt, eps, 1.0, bx, by, u_prev, 1, rowptr, col, val);
    if (rc) return rc;
    return step_rhs(p, N, dt, u_prev, NULL, b);
}

int orc_fe_step_system_field(int p, int N, double eps, double dt, const double *bxn,
                             const double *byn, const double *fn, const double *u_prev,
                             const int64_t *rowptr, const int32_t *col, double *val, double *b)
{
    int rc = orc_fe_assemble_field(p, N, 1.0 / dt, eps, 1.0, bxn, byn, u_prev, 1, rowptr, col, val);
    if (rc) return rc;
    return step_rhs(p, N, dt, u_prev, fn, b);
}

int orc_fe_paper_velocity(int p, int N, double *bxn, double *byn)
{
    const int64_t n = orc_fe_ndofs(p, N);
    double *x = malloc(sizeof(double) * n), *y = malloc(sizeof(double) * n);
    if (!x || !y) { free(x); free(y); return ORC_E_NOMEM; }
    int rc = orc_fe_node_coords(p, N, x, y);
    if (rc == ORC_OK)
        for (int64_t i = 0; i < n; ++i) {
            bxn[i] = -sin(M_PI * x[i]) * cos(M_PI * y[i]);
            byn[i] = cos(M_PI * x[i]) * sin(M_PI * y[i]);
        }
    free(x); free(y);
    return rc;
}

int orc_fe_paper_forcing(int p, int N, int nmodes, const double *c, double C, double *fn)
{
    if (nmodes < 0 || (nmodes > 0 && !c)) return ORC_E_ARG;
    const int64_t n = orc_fe_ndofs(p, N);
    double *x = malloc(sizeof(double) * n), *y = malloc(sizeof(double) * n);
    if (!x || !y) { free(x); free(y); return ORC_E_NOMEM; }
    int rc = orc_fe_node_coords(p, N, x, y);
    if (rc == ORC_OK)
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 1; j <= nmodes; ++j)
                s += c[j - 1] * exp(-(double)(j * j) / 20.0) * sin(2.0 * j * M_PI * x[i])
                     * sin(2.0 * j * M_PI * y[i]);
            fn[i] = 0.5 * C * s;
        }
    free(x); free(y);
    return rc;
}

int orc_fe_u0(int p, int N, const double *a8, double *u0)
{
    const int64_t n = orc_fe_ndofs(p, N);
    double *x = malloc(sizeof(double) * n), *y = malloc(sizeof(double) * n);
    if (!x || !y) { free(x); free(y); return ORC_E_NOMEM; }
    orc_fe_node_coords(p, N, x, y);
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        if (!on_boundary(p, N, i))
            for (int j = 1; j <= 8; ++j) s += a8[j - 1] * sin(j * M_PI * x[i]) * sin(j * M_PI * y[i]);
        u0[i] = s;
    }
    free(x); free(y);
    return ORC_OK;
}
