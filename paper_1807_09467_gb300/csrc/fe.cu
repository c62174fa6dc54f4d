// fe.cu -- the Sec. 6.1 time-step systems assembled on the device (the
// workload the solver is measured on; see include/rgmres.h).
//
// Discrete problem (Sec. 6.1, implicit Euler, convection coefficient lagged):
//   (1/dt)(v, u^n - u^{n-1}) + eps (grad v, grad u^n) + (v, u^{n-1} beta.grad u^n) = (v, 1)
// on Q_p elements, p = 1..32, with Gauss-Lobatto nodes and (p+1)^2 Gauss points
// per cell.  Uniform grid => one set of reference tables: the 1D mass M1 and
// stiffness K1, the load F1, and the reference convection tensor
//   T[(i),(j),(l)] = sum_q w_q phi_i(q) phi_l(q) (beta . grad_ref phi_j)(q)
// so that N_ij = h sum_l u_l T[i][j][l] on each cell.  With the tensor-product
// basis and Gauss rule T factors into 1D tables,
//   T = beta_x A1[ia][ja][la] B1[ib][jb][lb] + beta_y B1[ia][ja][la] A1[ib][jb][lb],
//   A1[i][j][l] = sum_g w_g phi_i phi_l phi_j',  B1[i][j][l] = sum_g w_g phi_i phi_j phi_l,
// so a first kernel forms each cell's convection matrix sum_l u_l T[i][j][l] by
// sum factorisation (contract lb, then la: 2 (p+1)^5 FMAs a cell instead of
// (p+1)^6), adds the cell's mass/dt and diffusion matrix (the same on every
// cell) and stores the result in a per-cell buffer (p <= 4; higher orders take
// the quadrature path below).  Assembly then gathers row by row (one warp per
// row, one lane per stored entry, cells visited in a fixed order), so it is
// deterministic and needs no atomics.
//
// Sec. 6.1's own benchmark replaces beta by the cellular field
// b = (-sin(pi x) cos(pi y), cos(pi x) sin(pi y)) through its nodal interpolant
// and the load (v, 1) by (v, f_h), f_h the interpolant of 16 random Laplace
// modes: then a first kernel forms, per cell and Gauss point q,
//   C_x = w_q h u(q) b_x(q),  C_y = w_q h u(q) b_y(q)
// (u, b interpolated), and N_ij sums phi_i (C_x d_x phi_j + C_y d_y phi_j) over
// the shared cells' Gauss points; the load is M f_h.
#include "../../include/rgmres.h"
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

void rgm_note_cuda_error(int err, const char *what, int line);   // solver.cu

extern "C" int rgm_internal_nnz(rgm_solver s, int64_t *nnz);
extern "C" int rgm_internal_config(rgm_solver s, rgm_config *cfg);

#define CKF(call)                                                            \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            rgm_note_cuda_error((int)e_, #call, __LINE__);                   \
            return (e_ == cudaErrorMemoryAllocation) ? RGM_E_OOM : RGM_E_CUDA; \
        }                                                                    \
    } while (0)

struct rgm_fe_s {
    int p = 1, N = 1;
    double eps = 0, dt = 1, bx = 0, by = 0, h = 1;
    cudaStream_t st = nullptr;
    int64_t L = 0, n = 0, nnz = 0;
    std::vector<int64_t> h_rowptr;
    std::vector<int32_t> h_col;
    int64_t *rowptr = nullptr;
    int32_t *col = nullptr;
    double *tabs = nullptr;   // M1 | K1 | F1 | T  (device)
    double *val = nullptr;    // assembly target when not writing into a solver
    double *b = nullptr;
    double *x = nullptr;      // solve scratch for rgm_fe_time_step
    // Sec. 6.1 benchmark fields (null: constant beta, f = 1)
    double *bxn = nullptr, *byn = nullptr;   // nodal velocity
    double *coef = nullptr;                  // C_x, C_y per cell and Gauss point
    double *fn = nullptr;                    // nodal forcing
    double *cmodes = nullptr;                // forcing coefficients (RGM_FE_MAX_MODES)
    double *elm = nullptr;                   // per-cell matrices (p <= 4, constant velocity), N^2 nl^2
    int64_t ntab = 0;                        // doubles in tabs
};

namespace {

// Gauss-Lobatto nodes on [0,1] for p <= 4 and Gauss-Legendre rules on [0,1]
// for q <= 5, from their closed forms on [-1,1].
void gll_closed(int p, double *xi)
{
    double t[5];
    if (p == 1) { t[0] = -1; t[1] = 1; }
    else if (p == 2) { t[0] = -1; t[1] = 0; t[2] = 1; }
    else if (p == 3) { t[0] = -1; t[1] = -1 / std::sqrt(5.0); t[2] = -t[1]; t[3] = 1; }
    else { t[0] = -1; t[1] = -std::sqrt(3.0 / 7.0); t[2] = 0; t[3] = -t[1]; t[4] = 1; }
    for (int i = 0; i <= p; ++i) xi[i] = 0.5 * (t[i] + 1.0);
}

void gauss_closed(int q, double *x, double *w)
{
    double t[5], c[5];
    if (q == 2) { t[0] = -1 / std::sqrt(3.0); t[1] = -t[0]; c[0] = c[1] = 1; }
    else if (q == 3) { t[0] = -std::sqrt(0.6); t[1] = 0; t[2] = -t[0]; c[0] = c[2] = 5.0 / 9; c[1] = 8.0 / 9; }
    else if (q == 4) {
        double a = std::sqrt(3.0 / 7 - 2.0 / 7 * std::sqrt(1.2)), b = std::sqrt(3.0 / 7 + 2.0 / 7 * std::sqrt(1.2));
        double wa = (18 + std::sqrt(30.0)) / 36, wb = (18 - std::sqrt(30.0)) / 36;
        t[0] = -b; t[1] = -a; t[2] = a; t[3] = b; c[0] = wb; c[1] = wa; c[2] = wa; c[3] = wb;
    } else {
        double a = std::sqrt(5 - 2 * std::sqrt(10.0 / 7)) / 3, b = std::sqrt(5 + 2 * std::sqrt(10.0 / 7)) / 3;
        double wa = (322 + 13 * std::sqrt(70.0)) / 900, wb = (322 - 13 * std::sqrt(70.0)) / 900;
        t[0] = -b; t[1] = -a; t[2] = 0; t[3] = a; t[4] = b; c[0] = wb; c[1] = wa; c[2] = 128.0 / 225; c[3] = wa; c[4] = wb;
    }
    for (int i = 0; i < q; ++i) { x[i] = 0.5 * (t[i] + 1.0); w[i] = 0.5 * c[i]; }
}

// Legendre P_k(t) and P_k'(t), k = 0..kmax, by Bonnet's recurrence and
// P_k' = P_{k-2}' + (2k - 1) P_{k-1}.
void legendre_table(int kmax, double t, double *P, double *dP)
{
    P[0] = 1.0; dP[0] = 0.0;
    if (kmax >= 1) { P[1] = t; dP[1] = 1.0; }
    for (int k = 2; k <= kmax; ++k) {
        P[k] = ((2.0 * k - 1.0) * t * P[k - 1] - (k - 1.0) * P[k - 2]) / k;
        dP[k] = dP[k - 2] + (2.0 * k - 1.0) * P[k - 1];
    }
}

// Gauss-Lobatto nodes on [0,1] for any p: the zeros of P_{p+1} - P_{p-1}
// (which vanish exactly at the Lobatto points, ends included), by Newton from
// the Chebyshev-Lobatto points.  p <= 4: closed forms.
void gll_nodes(int p, double *xi)
{
    if (p <= 4) { gll_closed(p, xi); return; }
    double P[40], dP[40];
    xi[0] = 0.0;
    xi[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double t = -std::cos(M_PI * i / p);
        for (int it = 0; it < 60; ++it) {
            legendre_table(p + 1, t, P, dP);
            const double q = P[p + 1] - P[p - 1], dq = dP[p + 1] - dP[p - 1];
            const double step = q / dq;
            t -= step;
            if (std::fabs(step) <= 1e-16) break;
        }
        xi[i] = 0.5 * (t + 1.0);
    }
}

// Gauss-Legendre rule on [0,1] for any q: zeros of P_q by Newton, weights
// 2 / ((1 - t^2) P_q'(t)^2) (halved for [0,1]).  q <= 5: closed forms.
void gauss_rule(int q, double *x, double *w)
{
    if (q <= 5) { gauss_closed(q, x, w); return; }
    double P[40], dP[40];
    for (int i = 0; i < q; ++i) {
        double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 60; ++it) {
            legendre_table(q, t, P, dP);
            const double step = P[q] / dP[q];
            t -= step;
            if (std::fabs(step) <= 1e-16) break;
        }
        legendre_table(q, t, P, dP);
        x[i] = 0.5 * (t + 1.0);
        w[i] = 1.0 / ((1.0 - t * t) * dP[q] * dP[q]);
    }
}

// Lagrange basis on `nodes` and its derivative at x (product rule).
void basis(int p, const double *nodes, double x, double *phi, double *dphi)
{
    for (int a = 0; a <= p; ++a) {
        double den = 1.0;
        for (int b = 0; b <= p; ++b) if (b != a) den *= nodes[a] - nodes[b];
        double num = 1.0;
        for (int b = 0; b <= p; ++b) if (b != a) num *= x - nodes[b];
        phi[a] = num / den;
        double d = 0.0;
        for (int skip = 0; skip <= p; ++skip) {
            if (skip == a) continue;
            double pr = 1.0;
            for (int b = 0; b <= p; ++b) if (b != a && b != skip) pr *= x - nodes[b];
            d += pr;
        }
        dphi[a] = d / den;
    }
}

__device__ __forceinline__ void cell_range(int64_t I, int p, int N, int *c0, int *c1)
{
    // cells containing lattice node I along one axis
    const int64_t c = I / p;
    if (I % p == 0) { *c0 = (int)(c > 0 ? c - 1 : 0); *c1 = (int)(c < N ? c : N - 1); }
    else { *c0 = (int)c; *c1 = (int)c; }
}

__device__ __forceinline__ bool on_bnd(int64_t dof, int64_t L)
{
    int64_t ix = dof % L, iy = dof / L;
    return ix == 0 || iy == 0 || ix == L - 1 || iy == L - 1;
}

struct FeDev {
    int p, N, nl;
    int64_t L, n;
    double h, inv_dt, eps;
    const double *M1, *K1, *F1;
    const double *A1, *B1;            // 1D factors of the convection tensor (p <= 4)
    double bx, by;                    // constant velocity
    const double *PH, *DPH, *GW;   // phi_a, phi_a' at Gauss point g ([g][a]), Gauss weights
    const double *XI;              // Gauss-Lobatto nodes of a cell on [0,1]
    const double *ME;              // p <= 4: the cell's mass/dt + diffusion matrix, nl x nl
    const double *AX, *BY;         // p <= 4: h beta_x A1 and h beta_y B1
};

// Coordinate of lattice node I along one axis (GLL nodes inside each cell).
__device__ __forceinline__ double node_coord(const FeDev &f, int64_t I)
{
    const int64_t cell = I / f.p;
    return cell == f.N ? 1.0 : ((double)cell + f.XI[I % f.p]) * f.h;
}

// Sec. 6.1's cellular velocity at the nodes.
__global__ void fe_velocity_kernel(FeDev f, double *bxn, double *byn)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    const double x = node_coord(f, i % f.L), y = node_coord(f, i / f.L);
    bxn[i] = -sin(M_PI * x) * cos(M_PI * y);
    byn[i] = cos(M_PI * x) * sin(M_PI * y);
}

// A constant velocity as a nodal field (the quadrature path of p > 4).
__global__ void fe_fill2_kernel(double *a, double va, double *b, double vb, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) { a[i] = va; b[i] = vb; }
}

// Sec. 6.1's forcing at the nodes: (C/2) sum_j c_j exp(-j^2/20) sin(2 j pi x) sin(2 j pi y).
__global__ void fe_forcing_kernel(FeDev f, int nmodes, const double *c, double C, double *fn)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    const double x = node_coord(f, i % f.L), y = node_coord(f, i / f.L);
    double s = 0.0;
    for (int j = 1; j <= nmodes; ++j)
        s += c[j - 1] * exp(-(double)(j * j) / 20.0) * sin(2.0 * j * M_PI * x) * sin(2.0 * j * M_PI * y);
    fn[i] = 0.5 * C * s;
}

// C_x, C_y per (cell, Gauss point): one thread each.
__global__ void fe_conv_coef_kernel(FeDev f, const double *u, const double *bxn, const double *byn,
                                    double *coef)
{
    const int q1 = f.p + 1, nq = q1 * q1;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)f.N * f.N * nq) return;
    const int g = (int)(t % nq), gx = g % q1, gy = g / q1;
    const int64_t cell = t / nq, cx = cell % f.N, cy = cell / f.N;
    double uq = 0.0, bx = 0.0, by = 0.0;
    for (int lb = 0; lb <= f.p; ++lb)
        for (int la = 0; la <= f.p; ++la) {
            const double ph = f.PH[gx * q1 + la] * f.PH[gy * q1 + lb];
            const int64_t d = (cy * f.p + lb) * f.L + cx * f.p + la;
            uq += u[d] * ph;
            bx += bxn[d] * ph;
            by += byn[d] * ph;
        }
    const double w = f.GW[gx] * f.GW[gy] * f.h;
    coef[2 * t] = w * uq * bx;
    coef[2 * t + 1] = w * uq * by;
}

// Matrices of the cells (constant velocity, p <= 4), one warp per cell:
// elm[cell][i][j] = ME[i][j] + h sum_l u_l T[i][j][l], i = (ia, ib), j = (ja, jb)
// local node indices (ME: mass/dt and diffusion, the same on every cell), the
// convection part by sum factorisation over the two directions:
//   Y1[la][ib][jb] = sum_lb B1[ib][jb][lb] u[la][lb],  Y2 likewise with A1,
//   elm = ME + sum_la (AX[ia][ja][la] Y1[la][ib][jb] + BY[ia][ja][la] Y2[la][ib][jb])
// with AX = h beta_x A1 and BY = h beta_y B1 scaled once on the host, so an
// entry of the second stage costs 2 (p+1) binary64 FMAs and nothing more.
#define FE_ELM_WARPS 8
__global__ void __launch_bounds__(32 * FE_ELM_WARPS) fe_elem_conv_kernel(FeDev f, const double *u, double *elm)
{
    constexpr int QM = 5;                               // p + 1 <= 5
    __shared__ double A1[QM * QM * QM], B1[QM * QM * QM], AX[QM * QM * QM], BY[QM * QM * QM];
    __shared__ double us[FE_ELM_WARPS][QM * QM], Y1[FE_ELM_WARPS][QM * QM * QM], Y2[FE_ELM_WARPS][QM * QM * QM];
    const int q1 = f.p + 1, q3 = q1 * q1 * q1, nl = f.nl;
    for (int t = threadIdx.x; t < q3; t += blockDim.x) {
        A1[t] = f.A1[t]; B1[t] = f.B1[t]; AX[t] = f.AX[t]; BY[t] = f.BY[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t cell = (int64_t)blockIdx.x * FE_ELM_WARPS + w;
    if (cell >= (int64_t)f.N * f.N) return;             // warp-uniform; no block barrier follows
    const int64_t cx = cell % f.N, cy = cell / f.N;
    if (lane < nl) {
        const int la = lane % q1, lb = lane / q1;
        us[w][la * QM + lb] = u[(cy * f.p + lb) * f.L + cx * f.p + la];
    }
    __syncwarp();
    for (int t = lane; t < q3; t += 32) {               // t = (la, ib, jb)
        const int la = t / (q1 * q1), ib = (t / q1) % q1, jb = t % q1;
        const double *ul = &us[w][la * QM];
        double y1 = 0.0, y2 = 0.0;
        for (int lb = 0; lb < q1; ++lb) {
            const int k = (ib * q1 + jb) * q1 + lb;
            y1 = fma(B1[k], ul[lb], y1);
            y2 = fma(A1[k], ul[lb], y2);
        }
        Y1[w][t] = y1;
        Y2[w][t] = y2;
    }
    __syncwarp();
    double *out = elm + cell * nl * nl;
    for (int t = lane; t < nl * nl; t += 32) {          // t = i nl + j, i = ib q1 + ia, j = jb q1 + ja
        const int i = t / nl, j = t % nl;
        const int ia = i % q1, ib = i / q1, ja = j % q1, jb = j / q1;
        double s = f.ME[t];
        for (int la = 0; la < q1; ++la) {
            const int k = (ia * q1 + ja) * q1 + la, y = (la * q1 + ib) * q1 + jb;
            s = fma(AX[k], Y1[w][y], s);
            s = fma(BY[k], Y2[w][y], s);
        }
        out[t] = s;
    }
}

// Quadrature path (nodal velocity, or p > 4): one warp per row, a lane per
// stored entry, the entry's (p+1)^2 Gauss points summed for each shared cell.
__global__ void fe_assemble_kernel(FeDev f, const int64_t *rowptr, const int32_t *col,
                                   const double *coef, double *val)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= f.n) return;
    const int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
    if (on_bnd(row, f.L)) {
        for (int64_t e = e0 + lane; e < e1; e += 32) val[e] = 1.0;
        return;
    }
    const int p = f.p, q1 = p + 1;
    const int64_t Ix = row % f.L, Iy = row / f.L;
    int ax0, ax1, ay0, ay1;
    cell_range(Ix, p, f.N, &ax0, &ax1);
    cell_range(Iy, p, f.N, &ay0, &ay1);
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int64_t cj = col[e];
        const int64_t Jx = cj % f.L, Jy = cj / f.L;
        int bx0, bx1, by0, by1;
        cell_range(Jx, p, f.N, &bx0, &bx1);
        cell_range(Jy, p, f.N, &by0, &by1);
        double v = 0.0;
        for (int cy = max(ay0, by0); cy <= min(ay1, by1); ++cy)
            for (int cx = max(ax0, bx0); cx <= min(ax1, bx1); ++cx) {
                const int ia = (int)(Ix - (int64_t)cx * p), ib = (int)(Iy - (int64_t)cy * p);
                const int ja = (int)(Jx - (int64_t)cx * p), jb = (int)(Jy - (int64_t)cy * p);
                const double mx = f.M1[ia * q1 + ja], my = f.M1[ib * q1 + jb];
                const double kx = f.K1[ia * q1 + ja], ky = f.K1[ib * q1 + jb];
                // nodal velocity: quadrature with the per-point coefficients
                const double *cc = coef + 2 * (((int64_t)cy * f.N + cx) * f.nl);
                double conv = 0.0;
                for (int gy = 0; gy <= p; ++gy)
                    for (int gx = 0; gx <= p; ++gx) {
                        const double pi = f.PH[gx * q1 + ia] * f.PH[gy * q1 + ib];
                        const int g = gy * q1 + gx;
                        conv += pi * (cc[2 * g] * f.DPH[gx * q1 + ja] * f.PH[gy * q1 + jb] +
                                      cc[2 * g + 1] * f.PH[gx * q1 + ja] * f.DPH[gy * q1 + jb]);
                    }
                v += f.h * f.h * mx * my * f.inv_dt + f.eps * (kx * my + mx * ky) + conv;
            }
        val[e] = v;
    }
}

// Per-cell matrix path (constant velocity, p <= 4): the value of entry (I, J)
// is the sum of elm[cell][i][j] over the (at most four) cells holding both
// nodes.  One warp per row, a lane per stored entry.  A row's columns are the
// product of its two 1D coupling ranges with the boundary nodes left out, in
// y-major order (the pattern rgm_fe_create builds), so a lane finds its
// column from its offset in the row instead of reading col; with P a
// compile-time constant and 32-bit node indices (L^2 <= 2^31) no 64-bit
// division remains.
template <int P>
__global__ void fe_assemble_elm_kernel(FeDev f, const int64_t *rowptr, const double *elm, double *val)
{
    constexpr int Q1 = P + 1, NL = Q1 * Q1;
    const int lane = threadIdx.x & 31;
    const int64_t wrow = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wrow >= f.n) return;
    const int row = (int)wrow, L = (int)f.L, N = f.N;
    const int64_t e0 = rowptr[row];
    const int len = (int)(rowptr[row + 1] - e0);
    const int Iy = row / L, Ix = row - Iy * L;
    if (Ix == 0 || Iy == 0 || Ix == L - 1 || Iy == L - 1) {
        for (int k = lane; k < len; k += 32) val[e0 + k] = 1.0;
        return;
    }
    // 1D coupling range of a node, clipped to the interior nodes 1 .. L-2
    auto crange = [&](int I, int *lo, int *hi) {
        if (I % P == 0) { *lo = max(I - P, 1); *hi = min(I + P, L - 2); }
        else { *lo = max((I / P) * P, 1); *hi = min((I / P) * P + P, L - 2); }
    };
    // cells holding a node along one axis
    auto cells = [&](int I, int *c0, int *c1) {
        const int c = I / P;
        if (I % P == 0) { *c0 = c > 0 ? c - 1 : 0; *c1 = c < N ? c : N - 1; }
        else { *c0 = c; *c1 = c; }
    };
    int xl, xh, yl, yh, ax0, ax1, ay0, ay1;
    crange(Ix, &xl, &xh);
    crange(Iy, &yl, &yh);
    cells(Ix, &ax0, &ax1);
    cells(Iy, &ay0, &ay1);
    const int wx = xh - xl + 1;
    // k / wx for k < 2^10 and wx <= 2P + 1 <= 9: (k + 1/2) / wx lies at least
    // 1/(2 wx) from an integer, far above binary32's rounding of the product
    const float rwx = 1.0f / (float)wx;
    // at most (2P + 1)^2 entries a row: all of a lane's entries and their (at
    // most four) cells' loads are issued before the first sum
    constexpr int KMAX = ((2 * P + 1) * (2 * P + 1) + 31) / 32;
#pragma unroll
    for (int it = 0; it < KMAX; ++it) {
        const int k = lane + 32 * it;
        if (k >= len) break;
        const int dy = (int)(((float)k + 0.5f) * rwx);
        const int Jy = yl + dy, Jx = xl + (k - dy * wx);
        int bx0, bx1, by0, by1;
        cells(Jx, &bx0, &bx1);
        cells(Jy, &by0, &by1);
        const int cy0 = max(ay0, by0), cy1 = min(ay1, by1), cx0 = max(ax0, bx0), cx1 = min(ax1, bx1);
        double t[4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int cy = cy0 + a, cx = cx0 + c;
                const int il = (Iy - cy * P) * Q1 + (Ix - cx * P);
                const int jl = (Jy - cy * P) * Q1 + (Jx - cx * P);
                t[2 * a + c] = (cy <= cy1 && cx <= cx1)
                                   ? __ldg(&elm[((int64_t)cy * N + cx) * (NL * NL) + il * NL + jl]) : 0.0;
            }
        // the cells in a fixed order (absent ones add +0)
        val[e0 + k] = ((t[0] + t[1]) + t[2]) + t[3];
    }
}

// b = M u / dt + F over the full neighbourhood (boundary columns included),
// then b_i = 0 on Dirichlet rows; with a nodal forcing fn, F = M fn.  One
// thread per row.  The cell mass matrix is h^2 (M1 x M1), so a cell's
// contribution is h^2 sum_jb M1[ib][jb] (sum_ja M1[ia][ja] u[jb][ja]): 2 (p+1)
// products per column line instead of (p+1)^2 per cell node.
__global__ void fe_rhs_kernel(FeDev f, const double *u, const double *fn, double *b)
{
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= f.n) return;
    if (on_bnd(row, f.L)) { b[row] = 0.0; return; }
    const int p = f.p, q1 = p + 1;
    const int64_t Ix = row % f.L, Iy = row / f.L;
    int ax0, ax1, ay0, ay1;
    cell_range(Ix, p, f.N, &ax0, &ax1);
    cell_range(Iy, p, f.N, &ay0, &ay1);
    double mu = 0.0, F = 0.0;
    for (int cy = ay0; cy <= ay1; ++cy)
        for (int cx = ax0; cx <= ax1; ++cx) {
            const int ia = (int)(Ix - (int64_t)cx * p), ib = (int)(Iy - (int64_t)cy * p);
            const double *mxr = f.M1 + ia * q1, *myr = f.M1 + ib * q1;
            if (!fn) F += f.F1[ia] * f.F1[ib];
            for (int jb = 0; jb <= p; ++jb) {
                const int64_t c0 = ((int64_t)cy * p + jb) * f.L + (int64_t)cx * p;
                double su = 0.0, sf = 0.0;
                for (int ja = 0; ja <= p; ++ja) {
                    su = fma(mxr[ja], u[c0 + ja], su);
                    if (fn) sf = fma(mxr[ja], fn[c0 + ja], sf);
                }
                mu = fma(myr[jb], su, mu);
                if (fn) F = fma(myr[jb], sf, F);
            }
        }
    b[row] = f.h * f.h * (mu * f.inv_dt + F);
}

// The same right-hand side for p <= 4 in two 1D passes.  The global mass
// matrix of the tensor-product grid is h^2 (M_y x M_x), M_x and M_y the
// assembled 1D mass matrices (the 2D cells are the products of the 1D cells),
// and the load of f = 1 is h^2 F_x F_y likewise.  A first pass applies M_x
// along every lattice row, a second M_y along the columns: (p + 1) FMAs per
// cell of a node per pass, and lanes of a warp (consecutive nodes of one
// lattice row) differ in their cell count only in the first pass.  With a
// nodal forcing the first pass applies M_x to u / dt + fn.
template <bool FN>
__global__ void fe_rhs_x_kernel(FeDev f, const double *u, const double *fn, double *t)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    const int p = f.p, q1 = p + 1;
    const int64_t Iy = i / f.L, Ix = i - Iy * f.L;
    int c0, c1;
    cell_range(Ix, p, f.N, &c0, &c1);
    const double *ur = u + Iy * f.L, *fr = FN ? fn + Iy * f.L : nullptr;
    double s = 0.0;
    for (int c = c0; c <= c1; ++c) {
        const double *m = f.M1 + (Ix - (int64_t)c * p) * q1;
        const int64_t j0 = (int64_t)c * p;
        for (int a = 0; a <= p; ++a)
            s = fma(m[a], FN ? fma(ur[j0 + a], f.inv_dt, fr[j0 + a]) : ur[j0 + a], s);
    }
    t[i] = s;
}

template <bool FN>
__global__ void fe_rhs_y_kernel(FeDev f, const double *t, double *b)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    if (on_bnd(i, f.L)) { b[i] = 0.0; return; }
    const int p = f.p, q1 = p + 1;
    const int64_t Iy = i / f.L, Ix = i - Iy * f.L;
    int c0, c1;
    cell_range(Iy, p, f.N, &c0, &c1);
    double s = 0.0, fy = 0.0;
    for (int c = c0; c <= c1; ++c) {
        const int ib = (int)(Iy - (int64_t)c * p);
        const double *m = f.M1 + ib * q1;
        const double *tc = t + (int64_t)c * p * f.L + Ix;
        for (int a = 0; a <= p; ++a) s = fma(m[a], tc[a * f.L], s);
        if (!FN) fy += f.F1[ib];
    }
    if (FN) { b[i] = f.h * f.h * s; return; }
    int x0, x1;
    cell_range(Ix, p, f.N, &x0, &x1);
    double fx = 0.0;
    for (int c = x0; c <= x1; ++c) fx += f.F1[Ix - (int64_t)c * p];
    b[i] = f.h * f.h * (s * f.inv_dt + fx * fy);
}

__global__ void fe_u0_kernel(FeDev f, const double *a8, double *u0)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    if (on_bnd(i, f.L)) { u0[i] = 0.0; return; }
    const double x = node_coord(f, i % f.L), y = node_coord(f, i / f.L);
    double s = 0.0;
    for (int j = 1; j <= 8; ++j) s += a8[j - 1] * sin(j * M_PI * x) * sin(j * M_PI * y);
    u0[i] = s;
}

__global__ void fe_select_kernel(double *x, const double *u, int64_t n, int zero)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = zero ? 0.0 : u[i];
}

FeDev dev_view(const rgm_fe_s *fe)
{
    const int q1 = fe->p + 1;
    FeDev f;
    f.p = fe->p; f.N = fe->N; f.nl = q1 * q1; f.L = fe->L; f.n = fe->n; f.h = fe->h;
    f.inv_dt = 1.0 / fe->dt; f.eps = fe->eps;
    f.M1 = fe->tabs; f.K1 = f.M1 + q1 * q1; f.F1 = f.K1 + q1 * q1; f.A1 = f.F1 + q1;
    f.B1 = f.A1 + q1 * q1 * q1;
    f.PH = f.A1 + (fe->p <= 4 ? 2 * q1 * q1 * q1 : 0);
    f.DPH = f.PH + q1 * q1; f.GW = f.DPH + q1 * q1; f.XI = f.GW + q1;
    f.bx = fe->bx; f.by = fe->by;
    f.ME = f.XI + q1;
    f.AX = f.ME + q1 * q1 * q1 * q1; f.BY = f.AX + q1 * q1 * q1;
    if (fe->p > 4) f.A1 = f.B1 = f.ME = f.AX = f.BY = nullptr;
    return f;
}

}  // namespace

extern "C" {

int rgm_fe_create(rgm_fe *out, int p, int N, double eps, double dt, double beta_x, double beta_y,
                  void *cuda_stream)
{
    if (!out || p < 1 || p > RGM_FE_MAX_P || N < 1 || !(dt > 0)) return RGM_E_ARG;
    *out = nullptr;
    const int64_t L = (int64_t)p * N + 1;
    if (L * L > (int64_t)1 << 31) return RGM_E_ARG;
    rgm_fe_s *fe = new (std::nothrow) rgm_fe_s();
    if (!fe) return RGM_E_OOM;
    fe->p = p; fe->N = N; fe->eps = eps; fe->dt = dt; fe->bx = beta_x; fe->by = beta_y;
    fe->h = 1.0 / N; fe->st = (cudaStream_t)cuda_stream; fe->L = L; fe->n = L * L;
    // Dirichlet pattern: rows = product of 1D coupling ranges, boundary filtered
    auto range1 = [&](int64_t I, int64_t *lo, int64_t *hi) {
        if (I % p == 0) { *lo = I - p < 0 ? 0 : I - p; *hi = I + p > L - 1 ? L - 1 : I + p; }
        else { *lo = (I / p) * p; *hi = *lo + p; }
    };
    auto bnd = [&](int64_t d) { int64_t ix = d % L, iy = d / L; return ix == 0 || iy == 0 || ix == L - 1 || iy == L - 1; };
    fe->h_rowptr.resize(fe->n + 1);
    fe->h_rowptr[0] = 0;
    for (int64_t r = 0; r < fe->n; ++r) {
        if (bnd(r)) fe->h_col.push_back((int32_t)r);
        else {
            int64_t xl, xh, yl, yh;
            range1(r % L, &xl, &xh);
            range1(r / L, &yl, &yh);
            for (int64_t jy = yl; jy <= yh; ++jy)
                for (int64_t jx = xl; jx <= xh; ++jx) {
                    int64_t c = jy * L + jx;
                    if (!bnd(c)) fe->h_col.push_back((int32_t)c);
                }
        }
        fe->h_rowptr[r + 1] = (int64_t)fe->h_col.size();
    }
    fe->nnz = (int64_t)fe->h_col.size();
    // reference tables
    const int q1 = p + 1, nl = q1 * q1;
    // p <= 4: the 1D factors A1, B1 of the reference convection tensor; above,
    // the quadrature path
    const size_t nT = p <= 4 ? 2 * (size_t)q1 * q1 * q1 : 0;
    double xi[RGM_FE_MAX_P + 1], gx[RGM_FE_MAX_P + 1], gw[RGM_FE_MAX_P + 1];
    std::vector<double> phv((size_t)q1 * q1), dphv((size_t)q1 * q1);
    gll_nodes(p, xi);
    gauss_rule(q1, gx, gw);
    for (int g = 0; g < q1; ++g) basis(p, xi, gx[g], &phv[(size_t)g * q1], &dphv[(size_t)g * q1]);
    auto ph = [&](int g, int a) { return phv[(size_t)g * q1 + a]; };
    auto dph = [&](int g, int a) { return dphv[(size_t)g * q1 + a]; };
    const size_t nME = p <= 4 ? (size_t)nl * nl : 0;
    std::vector<double> tab(2 * q1 * q1 + q1 + nT + 2 * q1 * q1 + q1 + q1 + nME + nT, 0.0);
    double *M1 = tab.data(), *K1 = M1 + q1 * q1, *F1 = K1 + q1 * q1, *A1 = F1 + q1;
    double *B1 = A1 + (nT ? q1 * q1 * q1 : 0);
    double *PH = A1 + nT, *DPH = PH + q1 * q1, *GW = DPH + q1 * q1, *XI = GW + q1, *ME = XI + q1;
    double *AX = ME + nME, *BY = AX + (nT ? q1 * q1 * q1 : 0);
    for (int g = 0; g < q1; ++g) {
        GW[g] = gw[g];
        XI[g] = xi[g];
        for (int a = 0; a <= p; ++a) { PH[g * q1 + a] = ph(g, a); DPH[g * q1 + a] = dph(g, a); }
    }
    for (int a = 0; a <= p; ++a) {
        for (int c = 0; c <= p; ++c)
            for (int g = 0; g < q1; ++g) {
                M1[a * q1 + c] += gw[g] * ph(g, a) * ph(g, c);
                K1[a * q1 + c] += gw[g] * dph(g, a) * dph(g, c);
            }
        for (int g = 0; g < q1; ++g) F1[a] += gw[g] * ph(g, a);
    }
    for (int i = 0; i <= p && nT > 0; ++i)
        for (int j = 0; j <= p; ++j)
            for (int l = 0; l <= p; ++l) {
                double a = 0.0, bb = 0.0;
                for (int g = 0; g < q1; ++g) {
                    a += gw[g] * ph(g, i) * ph(g, l) * dph(g, j);
                    bb += gw[g] * ph(g, i) * ph(g, j) * ph(g, l);
                }
                A1[(i * q1 + j) * q1 + l] = a;
                B1[(i * q1 + j) * q1 + l] = bb;
                AX[(i * q1 + j) * q1 + l] = fe->h * beta_x * a;
                BY[(i * q1 + j) * q1 + l] = fe->h * beta_y * bb;
            }
    // the same on every cell of the uniform grid: h^2 (M1 x M1) / dt + eps (K1 x M1 + M1 x K1)
    for (int i = 0; i < nl && nME > 0; ++i)
        for (int j = 0; j < nl; ++j) {
            const int ia = i % q1, ib = i / q1, ja = j % q1, jb = j / q1;
            const double mx = M1[ia * q1 + ja], my = M1[ib * q1 + jb];
            const double kx = K1[ia * q1 + ja], ky = K1[ib * q1 + jb];
            ME[(size_t)i * nl + j] = fe->h * fe->h * mx * my / dt + eps * (kx * my + mx * ky);
        }
    cudaError_t e = cudaMalloc((void **)&fe->rowptr, sizeof(int64_t) * (fe->n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&fe->col, sizeof(int32_t) * fe->nnz);
    fe->ntab = (int64_t)tab.size();
    if (e == cudaSuccess) e = cudaMalloc((void **)&fe->tabs, sizeof(double) * tab.size());
    if (e == cudaSuccess) e = cudaMalloc((void **)&fe->val, sizeof(double) * fe->nnz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&fe->b, sizeof(double) * fe->n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&fe->x, sizeof(double) * fe->n);
    if (e == cudaSuccess && p <= 4)
        e = cudaMalloc((void **)&fe->elm, sizeof(double) * (size_t)fe->N * fe->N * nl * nl);
    if (e == cudaSuccess) e = cudaMemcpy(fe->rowptr, fe->h_rowptr.data(), sizeof(int64_t) * (fe->n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fe->col, fe->h_col.data(), sizeof(int32_t) * fe->nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fe->tabs, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rgm_fe_destroy(fe);
        return e == cudaErrorMemoryAllocation ? RGM_E_OOM : RGM_E_CUDA;
    }
    if (p > 4) {   // no T table: the constant velocity goes through the quadrature path
        const int rc = rgm_fe_set_velocity(fe, RGM_FE_VELOCITY_CONSTANT);
        if (rc) { rgm_fe_destroy(fe); return rc; }
    }
    *out = fe;
    return RGM_OK;
}

int rgm_fe_device_bytes(rgm_fe fe, int64_t *bytes)
{
    if (!fe || !bytes) return RGM_E_ARG;
    int64_t b = 8 * (fe->n + 1) + 4 * fe->nnz + 8 * fe->ntab + 8 * fe->nnz + 16 * fe->n;
    if (fe->bxn) b += 16 * fe->n + 8 * 2 * (int64_t)fe->N * fe->N * (fe->p + 1) * (fe->p + 1);
    if (fe->fn) b += 8 * fe->n + 8 * RGM_FE_MAX_MODES;
    if (fe->elm) b += 8 * (int64_t)fe->N * fe->N * (fe->p + 1) * (fe->p + 1) * (fe->p + 1) * (fe->p + 1);
    *bytes = b;
    return RGM_OK;
}

int rgm_fe_destroy(rgm_fe fe)
{
    if (!fe) return RGM_E_ARG;
    void *p[] = {fe->rowptr, fe->col, fe->tabs, fe->val, fe->b, fe->x, fe->bxn, fe->byn, fe->coef,
                 fe->fn, fe->cmodes, fe->elm};
    for (void *q : p)
        if (q) cudaFree(q);
    delete fe;
    return RGM_OK;
}

int rgm_fe_sizes(rgm_fe fe, int64_t *n, int64_t *nnz)
{
    if (!fe || !n || !nnz) return RGM_E_ARG;
    *n = fe->n;
    *nnz = fe->nnz;
    return RGM_OK;
}

int rgm_fe_pattern(rgm_fe fe, int64_t *rowptr, int32_t *col, int flags)
{
    if (!fe || !rowptr || !col) return RGM_E_ARG;
    cudaMemcpyKind k = (flags & RGM_DEVICE_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    CKF(cudaMemcpy(rowptr, fe->h_rowptr.data(), sizeof(int64_t) * (fe->n + 1), k));
    CKF(cudaMemcpy(col, fe->h_col.data(), sizeof(int32_t) * fe->nnz, k));
    return RGM_OK;
}

static int fe_assemble_dev(rgm_fe fe, const double *u_dev, double *val_dev, double *b_dev)
{
    FeDev f = dev_view(fe);
    const int64_t warps = fe->n;
    const int tpb = 256;
    if (fe->bxn) {
        const int64_t nt = (int64_t)fe->N * fe->N * f.nl;
        fe_conv_coef_kernel<<<(unsigned)((nt + tpb - 1) / tpb), tpb, 0, fe->st>>>(f, u_dev, fe->bxn, fe->byn, fe->coef);
    }
    if (!fe->bxn) {
        const int64_t cells = (int64_t)fe->N * fe->N;
        fe_elem_conv_kernel<<<(unsigned)((cells + FE_ELM_WARPS - 1) / FE_ELM_WARPS), 32 * FE_ELM_WARPS, 0,
                              fe->st>>>(f, u_dev, fe->elm);
    }
    const unsigned ablocks = (unsigned)((warps * 32 + tpb - 1) / tpb);
    if (fe->bxn)
        fe_assemble_kernel<<<ablocks, tpb, 0, fe->st>>>(f, fe->rowptr, fe->col, fe->coef, val_dev);
    else if (fe->p == 1)
        fe_assemble_elm_kernel<1><<<ablocks, tpb, 0, fe->st>>>(f, fe->rowptr, fe->elm, val_dev);
    else if (fe->p == 2)
        fe_assemble_elm_kernel<2><<<ablocks, tpb, 0, fe->st>>>(f, fe->rowptr, fe->elm, val_dev);
    else if (fe->p == 3)
        fe_assemble_elm_kernel<3><<<ablocks, tpb, 0, fe->st>>>(f, fe->rowptr, fe->elm, val_dev);
    else
        fe_assemble_elm_kernel<4><<<ablocks, tpb, 0, fe->st>>>(f, fe->rowptr, fe->elm, val_dev);
    const unsigned nblocks = (unsigned)((fe->n + tpb - 1) / tpb);
    if (fe->elm) {
        // p <= 4: two 1D passes through the cell-matrix buffer (n <= N^2 (p+1)^4
        // doubles), free once the row gather before it on this stream has run
        if (fe->fn) {
            fe_rhs_x_kernel<true><<<nblocks, tpb, 0, fe->st>>>(f, u_dev, fe->fn, fe->elm);
            fe_rhs_y_kernel<true><<<nblocks, tpb, 0, fe->st>>>(f, fe->elm, b_dev);
        } else {
            fe_rhs_x_kernel<false><<<nblocks, tpb, 0, fe->st>>>(f, u_dev, nullptr, fe->elm);
            fe_rhs_y_kernel<false><<<nblocks, tpb, 0, fe->st>>>(f, fe->elm, b_dev);
        }
    } else {
        fe_rhs_kernel<<<nblocks, tpb, 0, fe->st>>>(f, u_dev, fe->fn, b_dev);
    }
    CKF(cudaGetLastError());
    return RGM_OK;
}

int rgm_fe_assemble(rgm_fe fe, const double *u_prev, double *val, double *b, int flags)
{
    if (!fe || !u_prev || !val || !b) return RGM_E_ARG;
    if (flags & RGM_DEVICE_PTRS) {
        int rc = fe_assemble_dev(fe, u_prev, val, b);
        if (rc) return rc;
        CKF(cudaStreamSynchronize(fe->st));
        return RGM_OK;
    }
    CKF(cudaMemcpyAsync(fe->x, u_prev, sizeof(double) * fe->n, cudaMemcpyHostToDevice, fe->st));
    int rc = fe_assemble_dev(fe, fe->x, fe->val, fe->b);
    if (rc) return rc;
    CKF(cudaMemcpyAsync(val, fe->val, sizeof(double) * fe->nnz, cudaMemcpyDeviceToHost, fe->st));
    CKF(cudaMemcpyAsync(b, fe->b, sizeof(double) * fe->n, cudaMemcpyDeviceToHost, fe->st));
    CKF(cudaStreamSynchronize(fe->st));
    return RGM_OK;
}

int rgm_fe_set_velocity(rgm_fe fe, int kind)
{
    if (!fe || kind < RGM_FE_VELOCITY_CONSTANT || kind > RGM_FE_VELOCITY_CELLULAR) return RGM_E_ARG;
    if (kind == RGM_FE_VELOCITY_CONSTANT && fe->p <= 4) {
        CKF(cudaStreamSynchronize(fe->st));
        void *p[] = {fe->bxn, fe->byn, fe->coef};
        for (void *q : p)
            if (q) cudaFree(q);
        fe->bxn = fe->byn = fe->coef = nullptr;
        return RGM_OK;
    }
    if (!fe->bxn) {
        const int64_t ncoef = 2 * (int64_t)fe->N * fe->N * (fe->p + 1) * (fe->p + 1);
        CKF(cudaMalloc((void **)&fe->bxn, sizeof(double) * fe->n));
        CKF(cudaMalloc((void **)&fe->byn, sizeof(double) * fe->n));
        CKF(cudaMalloc((void **)&fe->coef, sizeof(double) * ncoef));
    }
    if (kind == RGM_FE_VELOCITY_CONSTANT)
        fe_fill2_kernel<<<(unsigned)((fe->n + 255) / 256), 256, 0, fe->st>>>(fe->bxn, fe->bx, fe->byn, fe->by, fe->n);
    else
        fe_velocity_kernel<<<(unsigned)((fe->n + 255) / 256), 256, 0, fe->st>>>(dev_view(fe), fe->bxn, fe->byn);
    CKF(cudaGetLastError());
    CKF(cudaStreamSynchronize(fe->st));
    return RGM_OK;
}

int rgm_fe_set_forcing(rgm_fe fe, int nmodes, const double *c, double C, int flags)
{
    if (!fe || nmodes < 0 || nmodes > RGM_FE_MAX_MODES || (nmodes > 0 && !c)) return RGM_E_ARG;
    if (nmodes == 0) {
        CKF(cudaStreamSynchronize(fe->st));
        if (fe->fn) cudaFree(fe->fn);
        if (fe->cmodes) cudaFree(fe->cmodes);
        fe->fn = nullptr;
        fe->cmodes = nullptr;
        return RGM_OK;
    }
    if (!fe->fn) {
        CKF(cudaMalloc((void **)&fe->fn, sizeof(double) * fe->n));
        CKF(cudaMalloc((void **)&fe->cmodes, sizeof(double) * RGM_FE_MAX_MODES));
    }
    CKF(cudaMemcpyAsync(fe->cmodes, c, sizeof(double) * nmodes,
                        (flags & RGM_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, fe->st));
    fe_forcing_kernel<<<(unsigned)((fe->n + 255) / 256), 256, 0, fe->st>>>(dev_view(fe), nmodes, fe->cmodes,
                                                                          C, fe->fn);
    CKF(cudaGetLastError());
    if (!(flags & RGM_DEVICE_PTRS)) CKF(cudaStreamSynchronize(fe->st));
    return RGM_OK;
}

int rgm_fe_initial_field(rgm_fe fe, const double *a8, double *u0, int flags)
{
    if (!fe || !a8 || !u0) return RGM_E_ARG;
    double *a8d = nullptr;
    CKF(cudaMalloc((void **)&a8d, sizeof(double) * 8));
    cudaError_t e = cudaMemcpyAsync(a8d, a8, sizeof(double) * 8, cudaMemcpyHostToDevice, fe->st);
    double *dst = (flags & RGM_DEVICE_PTRS) ? u0 : fe->x;
    if (e == cudaSuccess) {
        fe_u0_kernel<<<(unsigned)((fe->n + 255) / 256), 256, 0, fe->st>>>(dev_view(fe), a8d, dst);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !(flags & RGM_DEVICE_PTRS))
        e = cudaMemcpyAsync(u0, fe->x, sizeof(double) * fe->n, cudaMemcpyDeviceToHost, fe->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(fe->st);
    cudaFree(a8d);
    return e == cudaSuccess ? RGM_OK : RGM_E_CUDA;
}

int rgm_fe_time_step(rgm_fe fe, rgm_solver s, double *u_dev, rgm_stats *st)
{
    if (!fe || !s || !u_dev) return RGM_E_ARG;
    int64_t snnz = 0;
    int rc = rgm_internal_nnz(s, &snnz);
    if (rc) return rc;
    if (snnz != fe->nnz) return RGM_E_STATE;
    if ((rc = fe_assemble_dev(fe, u_dev, fe->val, fe->b))) return rc;
    CKF(cudaStreamSynchronize(fe->st));
    if ((rc = rgm_set_operator_values(s, fe->val, RGM_DEVICE_PTRS))) return rc;
    int kcur = 0;
    rgm_get_recycle_space(s, nullptr, 0, &kcur, 0);
    rgm_config cfg;
    if ((rc = rgm_internal_config(s, &cfg))) return rc;
    const int zero = (cfg.mode != RGM_PLAIN && kcur > 0) ? 1 : 0;
    fe_select_kernel<<<(unsigned)((fe->n + 255) / 256), 256, 0, fe->st>>>(fe->x, u_dev, fe->n, zero);
    CKF(cudaGetLastError());
    CKF(cudaStreamSynchronize(fe->st));
    rc = rgm_solve(s, fe->b, fe->x, RGM_DEVICE_PTRS, st);
    if (rc < 0) return rc;
    int rc2 = rgm_update_recycle_svd(s, fe->x, RGM_DEVICE_PTRS, nullptr);
    if (rc2 < 0) return rc2;
    CKF(cudaMemcpyAsync(u_dev, fe->x, sizeof(double) * fe->n, cudaMemcpyDeviceToDevice, fe->st));
    CKF(cudaStreamSynchronize(fe->st));
    return rc;
}

}  // extern "C"
