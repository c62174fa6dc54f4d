// vec_kernels.cuh -- the fused vector kernel of the Arnoldi cycle and its
// finalisation phases (included by solver.cu).
//
// One launch = one pass over the rows: produce a vector w (SpMV, residual
// b - A x, copy, or AXPY against [W | Vraw | U]), store it, take its dot
// products with a set of columns [U | Vraw | W | w itself], reduce them to
// per-block partials, and let the last block to finish reduce the partials and
// run the scalar step that follows (Gram-Schmidt coefficients, Hessenberg
// column, Givens rotation, convergence test, ...).  Every scalar decision
// stays on the device; the host only reads back once per GMRES cycle.
#pragma once
#include "common.cuh"

enum Src { SRC_SPMV = 0, SRC_RES = 1, SRC_COPY = 2, SRC_AXPY = 3, SRC_NONE = 4 };
enum Gate { GATE_NONE = 0, GATE_KRYLOV = 1, GATE_APPEND = 2 };
enum Fin {
    FIN_NONE = 0,
    FIN_BNORM,       // ||b||, tol
    FIN_RESNORM,     // beta = ||r||, converged flag
    FIN_COARSE,      // coefU = E^{-1} (U^T r)
    FIN_START_PLAIN, // v_0 = r / ||r||
    FIN_START_DEF1,  // coefW = -E^{-1} U^T r  (start vector P r)
    FIN_START_DEF2,  // v_0 = P r / ||P r||, VtW row 0
    FIN_ARN1,        // first CGS pass coefficients (with the oblique projection)
    FIN_ARN2,        // second CGS pass coefficients
    FIN_ARN3,        // Hessenberg column, Givens, flags
    FIN_AUG1,        // appended column: first pass
    FIN_AUG3,        // appended column: accept / drop, Givens
    FIN_DOTS         // store the reduced dots in Small::dots
};

template <typename T>
struct VecOp {
    int64_t n;
    int rpb;                 // rows per block
    int nblocks;
    int src;
    const int64_t *rowptr;
    const int32_t *col;
    const T *val;
    const T *x;              // SpMV / residual input
    int xscale;              // index into colscale, -1 for none
    const T *b;              // residual right-hand side
    const T *win;            // COPY / AXPY input (may equal out)
    int nW, nV, nU;          // AXPY columns used: out = win + W cW + Vraw cV + U cU
    T *out;
    const T *U; int64_t ldu;
    const T *V; int64_t ldv;
    const T *W; int64_t ldw;
    int ndU, ndV, ndW, dnorm;  // dot columns: U[0..ndU), Vraw[0..ndV), W[0..ndW), ||w||^2
    double *partials;
    unsigned *counter;
    Small *sm;
    int fin;
    int gate;
    int arg;                 // phase argument (Krylov index j / appended column i)
    int dyn;                 // DYN_* bits: counts and output column read from Small
};

enum Dyn {
    DYN_NDV_NB = 1,   // ndV = s->nb
    DYN_NV_NB = 2,    // nV  = s->nb
    DYN_NV_J = 4,     // nV  = s->J
    DYN_OUT_VNB = 8   // out = Vraw[:, s->nb]
};

// ---------------------------------------------------------------- scalar helpers
__device__ inline void lu_solve_small(int k, const double *LU, const int *piv, double *x)
{
    for (int j = 0; j < k; ++j)
        if (piv[j] != j) { double t = x[j]; x[j] = x[piv[j]]; x[piv[j]] = t; }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) x[i] -= LU[i + j * RGM_KMAX] * x[j];
    for (int i = k - 1; i >= 0; --i) {
        for (int j = i + 1; j < k; ++j) x[i] -= LU[i + j * RGM_KMAX] * x[j];
        x[i] /= LU[i + i * RGM_KMAX];
    }
}

// Apply rotations 0..col-1 to column col of H, then make rotation col.
__device__ inline void givens_column(Small *s, int col)
{
    double *hc = s->H + (int64_t)col * RGM_HLD;
    for (int i = 0; i < col; ++i) {
        double a = hc[i], b = hc[i + 1];
        hc[i] = s->cs[i] * a + s->sn[i] * b;
        hc[i + 1] = -s->sn[i] * a + s->cs[i] * b;
    }
    double a = hc[col], b = hc[col + 1];
    double r = hypot(a, b);
    double c = 1.0, sn = 0.0;
    if (r != 0.0) { c = a / r; sn = b / r; }
    s->cs[col] = c;
    s->sn[col] = sn;
    hc[col] = r;
    hc[col + 1] = 0.0;
    s->g[col + 1] = -sn * s->g[col];
    s->g[col] = c * s->g[col];
}

// The scalar step after a reduction.  d[] holds the reduced dots in the
// column order [U | Vraw | W | norm].  Runs on one thread.
template <typename T>
__device__ void finalize_scalar(const VecOp<T> &op, const double *d)
{
    Small *s = op.sm;
    const double *dU = d, *dV = d + op.ndU, *dW = d + op.ndU + op.ndV;
    const double nrm2 = op.dnorm ? d[op.ndU + op.ndV + op.ndW] : 0.0;
    const int k = s->k;
    switch (op.fin) {
    case FIN_BNORM:
        s->bnorm = sqrt(nrm2);
        break;
    case FIN_RESNORM:
        s->beta = sqrt(nrm2);
        s->converged = (s->beta <= s->tol_abs) ? 1 : 0;
        break;
    case FIN_COARSE: {
        double c[RGM_KMAX];
        for (int i = 0; i < k; ++i) c[i] = dU[i];
        lu_solve_small(k, s->LU, s->piv, c);
        for (int i = 0; i < k; ++i) s->coefU[i] = c[i];
        break;
    }
    case FIN_START_PLAIN: {
        double bs = sqrt(nrm2);
        s->bs = bs;
        s->J = 0;
        s->nb = 1;
        s->naug = 0;
        s->g[0] = bs;
        s->colscale[0] = bs > 0.0 ? 1.0 / bs : 0.0;
        s->done = (bs > 0.0) ? 0 : 1;
        s->breakdown = 0;
        break;
    }
    case FIN_START_DEF1: {
        double c[RGM_KMAX];
        for (int i = 0; i < k; ++i) c[i] = dU[i];
        lu_solve_small(k, s->LU, s->piv, c);
        for (int i = 0; i < k; ++i) s->coefW[i] = -c[i];
        break;
    }
    case FIN_START_DEF2: {
        double bs = sqrt(nrm2);
        s->bs = bs;
        s->J = 0;
        s->nb = 1;
        s->naug = 0;
        s->g[0] = bs;
        double sc = bs > 0.0 ? 1.0 / bs : 0.0;
        s->colscale[0] = sc;
        for (int l = 0; l < op.ndW; ++l) s->VtW[0 + l * RGM_HLD] = dW[l] * sc;
        s->done = (bs > 0.0) ? 0 : 1;
        s->breakdown = 0;
        break;
    }
    case FIN_ARN1: {
        // w = A v_j (unprojected).  Deflated: P w = w - W d, d = E^{-1} U^T w,
        // and V^T P w = V^T w - (V^T W) d.
        const int nb = s->nb;
        s->wn0 = sqrt(nrm2);
        double dd[RGM_KMAX];
        int kk = op.ndU;
        for (int i = 0; i < kk; ++i) dd[i] = dU[i];
        if (kk) lu_solve_small(kk, s->LU, s->piv, dd);
        for (int i = 0; i < kk; ++i) s->coefW[i] = -dd[i];
        for (int i = 0; i < nb; ++i) {
            double h = dV[i] * s->colscale[i];
            for (int l = 0; l < kk; ++l) h -= s->VtW[i + l * RGM_HLD] * dd[l];
            s->hsum[i] = h;
            s->coefV[i] = -h * s->colscale[i];
        }
        break;
    }
    case FIN_ARN2: {
        const int nb = s->nb;
        for (int i = 0; i < nb; ++i) {
            double h = dV[i] * s->colscale[i];
            s->hsum[i] += h;
            s->coefV[i] = -h * s->colscale[i];
        }
        break;
    }
    case FIN_ARN3: {
        const int j = s->J, nb = s->nb;
        const double hn = sqrt(nrm2);
        double *hc = s->H + (int64_t)j * RGM_HLD;
        for (int i = 0; i < nb; ++i) hc[i] = s->hsum[i];
        hc[nb] = hn;
        givens_column(s, j);
        s->J = j + 1;
        s->iters += 1;
        if (hn <= 1e-14 * s->wn0) {                 // happy breakdown: v_{j+1} := 0
            s->colscale[nb] = 0.0;
            for (int l = 0; l < op.ndW; ++l) s->VtW[nb + l * RGM_HLD] = 0.0;
            s->breakdown = 1;
            s->done = 1;
        } else {
            const double sc = 1.0 / hn;
            s->colscale[nb] = sc;
            for (int l = 0; l < op.ndW; ++l) s->VtW[nb + l * RGM_HLD] = dW[l] * sc;
        }
        s->nb = nb + 1;
        if (fabs(s->g[j + 1]) <= s->tol_abs) s->done = 1;
        if (s->iters >= s->maxit || s->J >= s->m) s->done = 1;
        break;
    }
    case FIN_AUG1: {
        const int nb = s->nb;
        s->wn0 = sqrt(nrm2);
        s->skip = (s->wn0 == 0.0) ? 1 : 0;
        for (int i = 0; i < nb; ++i) {
            double h = dV[i] * s->colscale[i];
            s->hsum[i] = h;
            s->coefV[i] = -h * s->colscale[i];
        }
        break;
    }
    case FIN_AUG3: {
        const int nb = s->nb, col = s->J + s->naug;
        const double hn = sqrt(nrm2);
        // the candidate column after the stored rotations
        double c[RGM_HLD + 1];
        for (int i = 0; i < nb; ++i) c[i] = s->hsum[i];
        c[nb] = hn;
        for (int i = nb + 1; i <= col + 1 && i <= RGM_HLD; ++i) c[i] = 0.0;
        for (int i = 0; i < col; ++i) {
            double a = c[i], b = c[i + 1];
            c[i] = s->cs[i] * a + s->sn[i] * b;
            c[i + 1] = -s->sn[i] * a + s->cs[i] * b;
        }
        if (hypot(c[col], c[col + 1]) <= 1e-14 * s->wn0) break;    // dependent: drop
        double *hc = s->H + (int64_t)col * RGM_HLD;
        for (int i = 0; i < RGM_HLD; ++i) hc[i] = 0.0;
        for (int i = 0; i < nb; ++i) hc[i] = s->hsum[i];
        hc[nb] = hn;
        givens_column(s, col);
        s->colscale[nb] = (hn <= 1e-14 * s->wn0) ? 0.0 : 1.0 / hn;
        s->aug_idx[s->naug] = op.arg;
        s->naug += 1;
        s->nb = nb + 1;
        break;
    }
    case FIN_DOTS: {
        const int nd = op.ndU + op.ndV + op.ndW + op.dnorm;
        for (int i = 0; i < nd; ++i) s->dots[i] = d[i];
        break;
    }
    default:
        break;
    }
}

// Pointer to dot column c of [U | Vraw | W | out].
template <typename T>
__device__ __forceinline__ const T *dot_col(const VecOp<T> &op, int c)
{
    if (c < op.ndU) return op.U + (int64_t)c * op.ldu;
    c -= op.ndU;
    if (c < op.ndV) return op.V + (int64_t)c * op.ldv;
    c -= op.ndV;
    if (c < op.ndW) return op.W + (int64_t)c * op.ldw;
    return op.out;
}

template <typename T, int SW>
__global__ void __launch_bounds__(RGM_THREADS) vec_kernel(VecOp<T> op)
{
    Small *s = op.sm;
    if (op.gate == GATE_KRYLOV && s->done) return;
    if (op.gate == GATE_APPEND && (s->skip || s->J == 0)) return;
    if (op.dyn) {
        if (op.dyn & DYN_NDV_NB) op.ndV = s->nb;
        if (op.dyn & DYN_NV_NB) op.nV = s->nb;
        if (op.dyn & DYN_NV_J) op.nV = s->J;
        if (op.dyn & DYN_OUT_VNB) op.out = const_cast<T *>(op.V) + (int64_t)s->nb * op.ldv;
    }

    __shared__ double red[(RGM_THREADS / 32) * RGM_CHUNK];
    __shared__ T cW[RGM_KMAX], cU[RGM_KMAX], cV[RGM_HLD];
    __shared__ double xs;
    if (threadIdx.x == 0) xs = (op.xscale >= 0) ? s->colscale[op.xscale] : 1.0;
    if (op.src == SRC_AXPY) {
        for (int i = threadIdx.x; i < op.nW; i += blockDim.x) cW[i] = (T)s->coefW[i];
        for (int i = threadIdx.x; i < op.nV; i += blockDim.x) cV[i] = (T)s->coefV[i];
        for (int i = threadIdx.x; i < op.nU; i += blockDim.x) cU[i] = (T)s->coefU[i];
    }
    __syncthreads();

    const int64_t r0 = (int64_t)blockIdx.x * op.rpb;
    const int64_t r1 = min(op.n, r0 + op.rpb);

    // ---- phase 1: produce and store w on this block's rows
    if (op.src == SRC_SPMV || op.src == SRC_RES) {
        // SW lanes per row; the loop bound is uniform across the warp so every
        // lane reaches the shuffles.
        const int lane = threadIdx.x % SW;
        const int grp = threadIdx.x / SW, ngrp = blockDim.x / SW;
        const T sc = (T)xs;
        for (int64_t base = r0; base < r1; base += ngrp) {
            const int64_t r = base + grp;
            T acc = 0;
            if (r < r1) {
                const int64_t e0 = op.rowptr[r], e1 = op.rowptr[r + 1];
                for (int64_t e = e0 + lane; e < e1; e += SW) acc += op.val[e] * op.x[op.col[e]];
            }
#pragma unroll
            for (int o = SW / 2; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, SW);
            if (r < r1 && lane == 0) op.out[r] = (op.src == SRC_SPMV) ? acc * sc : op.b[r] - acc;
        }
    } else if (op.src == SRC_COPY || op.src == SRC_AXPY) {
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            T acc = op.win[r];
            if (op.src == SRC_AXPY) {
                for (int c = 0; c < op.nW; ++c) acc += cW[c] * op.W[r + (int64_t)c * op.ldw];
                for (int c = 0; c < op.nV; ++c) acc += cV[c] * op.V[r + (int64_t)c * op.ldv];
                for (int c = 0; c < op.nU; ++c) acc += cU[c] * op.U[r + (int64_t)c * op.ldu];
            }
            op.out[r] = acc;
        }
    }
    const int nd = op.ndU + op.ndV + op.ndW + op.dnorm;
    if (nd == 0 && op.fin == FIN_NONE) return;
    __syncthreads();

    // ---- phase 2: block partial dot products, RGM_CHUNK columns per pass.
    // Products and per-thread sums in the vector precision T, the reduction
    // tree across threads and blocks in binary64.
    for (int c0 = 0; c0 < nd; c0 += RGM_CHUNK) {
        T acc[RGM_CHUNK];
        const T *cp[RGM_CHUNK];
#pragma unroll
        for (int i = 0; i < RGM_CHUNK; ++i) {
            acc[i] = 0;
            cp[i] = (c0 + i < nd) ? dot_col(op, c0 + i) : op.out;
        }
        const int nv = min(RGM_CHUNK, nd - c0);
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const T wi = op.out[r];
#pragma unroll
            for (int i = 0; i < RGM_CHUNK; ++i)
                if (i < nv) acc[i] += cp[i][r] * wi;
        }
        double accd[RGM_CHUNK];
#pragma unroll
        for (int i = 0; i < RGM_CHUNK; ++i) accd[i] = (double)acc[i];
        block_reduce_store<RGM_CHUNK>(accd, op.partials + (int64_t)c0 * op.nblocks + blockIdx.x, nv,
                                      op.nblocks, red);
    }

    // ---- phase 3: the last block reduces the partials and runs the scalar step
    if (!last_block(op.counter)) return;
    __shared__ double dsum[RGM_MAXDOTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < nd; c += nw) {
        double v = 0.0;
        const double *p = op.partials + (int64_t)c * op.nblocks;
        for (int b = lane; b < op.nblocks; b += 32) v += __ldcg(p + b);
        v = warp_sum(v);
        if (lane == 0) dsum[c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        finalize_scalar(op, dsum);
        *op.counter = 0u;
    }
}

// Pairwise dot products of columns: out[p] = col(a_p) . col(b_p) for a list of
// pairs over the combined column list [X | Y]; binary64 accumulation.
template <typename T>
struct GramOp {
    int64_t n;
    int rpb, nblocks;
    const T *X; int64_t ldx; int nx;
    const T *Y; int64_t ldy;
    int npairs;
    const int2 *pairs;
    double *partials;
    unsigned *counter;
    double *out;
};

template <typename T>
__device__ __forceinline__ const T *gram_col(const GramOp<T> &op, int c)
{
    return c < op.nx ? op.X + (int64_t)c * op.ldx : op.Y + (int64_t)(c - op.nx) * op.ldy;
}

template <typename T>
__global__ void __launch_bounds__(RGM_THREADS) gram_kernel(GramOp<T> op)
{
    __shared__ double red[(RGM_THREADS / 32) * RGM_CHUNK];
    const int64_t r0 = (int64_t)blockIdx.x * op.rpb;
    const int64_t r1 = min(op.n, r0 + op.rpb);
    for (int p0 = 0; p0 < op.npairs; p0 += RGM_CHUNK) {
        double acc[RGM_CHUNK];
        const T *ca[RGM_CHUNK], *cb[RGM_CHUNK];
        const int nv = min(RGM_CHUNK, op.npairs - p0);
#pragma unroll
        for (int i = 0; i < RGM_CHUNK; ++i) {
            acc[i] = 0.0;
            int2 pr = op.pairs[p0 + (i < nv ? i : 0)];
            ca[i] = gram_col(op, pr.x);
            cb[i] = gram_col(op, pr.y);
        }
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
#pragma unroll
            for (int i = 0; i < RGM_CHUNK; ++i)
                if (i < nv) acc[i] += (double)ca[i][r] * (double)cb[i][r];
        }
        block_reduce_store<RGM_CHUNK>(acc, op.partials + (int64_t)p0 * op.nblocks + blockIdx.x, nv,
                                      op.nblocks, red);
    }
    if (!last_block(op.counter)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < op.npairs; c += nw) {
        double v = 0.0;
        const double *p = op.partials + (int64_t)c * op.nblocks;
        for (int b = lane; b < op.nblocks; b += 32) v += __ldcg(p + b);
        v = warp_sum(v);
        if (lane == 0) op.out[c] = v;
    }
    if (threadIdx.x == 0) *op.counter = 0u;
}

// ---------------------------------------------------------------- cycle-end kernels
// Back substitution R y = g on the rotated (J+naug)^2 block, then the update
// coefficients of x += Vraw[:, :J] (y * colscale) + U[:, aug] y_aug.
__global__ void ls_solve_kernel(Small *s)
{
    __shared__ double g[RGM_HLD];
    const int nc = s->J + s->naug;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) g[i] = s->g[i];
    __syncthreads();
    for (int i = nc - 1; i >= 0; --i) {
        __shared__ double yi;
        if (threadIdx.x == 0) {
            double d = s->H[i + (int64_t)i * RGM_HLD];
            yi = (d != 0.0) ? g[i] / d : 0.0;
            s->y[i] = yi;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < i; t += blockDim.x) g[t] -= s->H[t + (int64_t)i * RGM_HLD] * yi;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < RGM_HLD; i += blockDim.x) s->coefV[i] = 0.0;
    for (int i = threadIdx.x; i < RGM_KMAX; i += blockDim.x) s->coefU[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < s->J; ++c) s->coefV[c] = s->y[c] * s->colscale[c];
        for (int a = 0; a < s->naug; ++a) s->coefU[s->aug_idx[a]] += s->y[s->J + a];
    }
}

// Reset the per-cycle Hessenberg state (before the start vector kernels).
__global__ void cycle_reset_kernel(Small *s)
{
    for (int i = threadIdx.x; i < RGM_HLD * RGM_NCOL; i += blockDim.x) s->H[i] = 0.0;
    for (int i = threadIdx.x; i <= RGM_HLD; i += blockDim.x) s->g[i] = 0.0;
    if (threadIdx.x == 0) {
        s->J = 0;
        s->nb = 0;
        s->naug = 0;
        s->skip = 0;
        s->done = 0;
        s->breakdown = 0;
    }
}

// LU with partial pivoting of E (k x k) in one block; singular when a pivot
// falls below 1e-13 * max(largest pivot, max_i ||u_i|| ||A u_i||).  colnorm2
// holds ||u_i||^2 then ||w_i||^2 (2k values).
__global__ void lu_kernel(Small *s, int k, const double *gram_uw, const double *colnorm2)
{
    __shared__ double M[RGM_KMAX * RGM_KMAX];
    __shared__ int pivrow;
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
        int r = i % k, c = i / k;
        M[r + c * RGM_KMAX] = gram_uw[i];
        s->E[r + c * RGM_KMAX] = gram_uw[i];
    }
    __syncthreads();
    double scale = 0.0;
    for (int i = 0; i < k; ++i) scale = fmax(scale, sqrt(colnorm2[i] * colnorm2[k + i]));
    double maxp = scale, minp = INFINITY;
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            int p = j;
            for (int i = j + 1; i < k; ++i)
                if (fabs(M[i + j * RGM_KMAX]) > fabs(M[p + j * RGM_KMAX])) p = i;
            pivrow = p;
            s->piv[j] = p;
        }
        __syncthreads();
        const int p = pivrow;
        if (p != j)
            for (int c = threadIdx.x; c < k; c += blockDim.x) {
                double t = M[j + c * RGM_KMAX];
                M[j + c * RGM_KMAX] = M[p + c * RGM_KMAX];
                M[p + c * RGM_KMAX] = t;
            }
        __syncthreads();
        const double d = M[j + j * RGM_KMAX];
        maxp = fmax(maxp, fabs(d));
        minp = fmin(minp, fabs(d));
        if (d != 0.0) {
            for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) M[i + j * RGM_KMAX] /= d;
            __syncthreads();
            for (int t = threadIdx.x; t < (k - j - 1) * (k - j - 1); t += blockDim.x) {
                int i = j + 1 + t % (k - j - 1), c = j + 1 + t / (k - j - 1);
                M[i + c * RGM_KMAX] -= M[i + j * RGM_KMAX] * M[j + c * RGM_KMAX];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < RGM_KMAX * RGM_KMAX; i += blockDim.x) s->LU[i] = M[i];
    if (threadIdx.x == 0) {
        int sing = (k > 0 && (minp == 0.0 || minp < 1e-13 * maxp)) ? 1 : 0;
        s->singular = sing;
        s->k = sing ? 0 : k;
    }
}
