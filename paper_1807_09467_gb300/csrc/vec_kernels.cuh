// vec_kernels.cuh -- the fused vector kernel of the Arnoldi cycle, its
// finalisation phases and the Gram kernel (included by solver.cu).
//
// One launch = one pass over the rows: produce a vector w (SpMV, residual
// b - A x, copy, or AXPY against [W | Vraw | U]), store it, take its dot
// products with a set of columns [U | Vraw | W | w itself], reduce them to
// per-block partials, and let the last block to finish reduce the partials and
// run the scalar step that follows (Gram-Schmidt coefficients, Hessenberg
// column, Givens rotation, convergence test, ...).  Every scalar decision
// stays on the device; the host only reads back once per GMRES cycle.
//
// Rows are processed in tiles of RGM_TILE: the tile of w is kept in shared
// memory, and the dot products run one warp per column over the tile, so each
// warp accumulates its columns across tiles and reduces once at the end.  The
// last block stages the small state it needs (LU factors, rotations, the new
// Hessenberg column) in shared memory before the sequential parts.
#pragma once
#include "common.cuh"

#define RGM_TILE RGM_THREADS
#define RGM_RGROUP 32            // blocks per group of the two-level dot reduction

enum Src { SRC_SPMV = 0, SRC_RES = 1, SRC_COPY = 2, SRC_AXPY = 3, SRC_NONE = 4 };
enum Gate {
    GATE_NONE = 0,
    GATE_KRYLOV = 1,   // skip once the cycle's Krylov phase is done
    GATE_APPEND = 2,   // skip a dropped appended column
    GATE_STEP = 3      // run only if Arnoldi step arg - 1 completed (s->J == arg)
};
enum Fin {
    FIN_NONE = 0,
    FIN_BNORM,       // ||b||
    FIN_BNORMP,      // ||D^{-1} b|| (left Jacobi)
    FIN_RESNORM,     // beta = ||r||, converged flag
    FIN_COARSE,      // coefU = E^{-1} (U^T r), coefW = -coefU
    FIN_START_PLAIN, // v_0 = r / ||r||
    FIN_START_DEF1,  // coefW = -E^{-1} U^T r  (start vector P r)
    FIN_START_DEF2,  // v_0 = P r / ||P r||, VtW row 0
    FIN_ARN1,        // first CGS pass coefficients (with the oblique projection)
    FIN_ARN2,        // second CGS pass coefficients (appended columns)
    FIN_ARN2H,       // second CGS pass with ||w - V h2|| from the same reduction:
                     // Hessenberg column, Givens, flags (the third pass is a plain update)
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
    // operator in sliced ELL: 32-row slices, rows sorted by length inside each
    // RGM_TILE-row tile; entry k of the slice's lane l at slice_ptr + 32 k + l
    const int64_t *slice_ptr;
    const int32_t *scol;
    const T *sval;
    const int32_t *perm;     // slice row -> matrix row (-1: padding)
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
    const T *wvec;           // if set, the norm column is ||wvec .* w||^2 (true residual)
    double *partials;        // per-block dot partials, column c at c * nblocks
    unsigned *counter;       // completion counter of the groups
    unsigned *gcount;        // per-group completion counters (RGM_RGROUP blocks a group)
    double *gpart;           // per-group sums, column c at c * ngroups
    int ngroups;
    Small *sm;
    int fin;
    int gate;
    int arg;                 // phase argument (appended column index)
    unsigned release_gen;    // FIN_ARN2H in the cycle kernel: publish this grid-barrier
                             // generation as soon as the next pass's inputs are written
    int lu_sel;              // small solves with E's LU (0) or the projector's (1)
    int dyn;                 // DYN_* bits: counts and output column read from Small
    volatile unsigned *mirror;  // FIN_ARN2H: host-mapped {steps done, cycle done} of the
                                // cycle, for the host launching the passes (may be null)
};

enum Dyn {
    DYN_NDV_NB = 1,   // ndV = s->nb
    DYN_NV_NB = 2,    // nV  = s->nb
    DYN_NV_J = 4,     // nV  = s->J
    DYN_OUT_VNB = 8,  // out = Vraw[:, s->nb]
    DYN_NV_NBM1 = 16, // nV  = s->nb - 1 (after a scalar step that stored column nb)
    DYN_OUT_VNBM1 = 32 // out = Vraw[:, s->nb - 1]
};

// Shared scratch of the finalising block.
struct FinScratch {
    double LU[RGM_KMAX * RGM_KMAX];
    int piv[RGM_KMAX];
    double dd[RGM_KMAX];
    double col[RGM_HLD + 1];
    double cs[RGM_HLD], sn[RGM_HLD];
    double sc[RGM_HLD];
    double h2[RGM_HLD];                       // second-pass coefficients
    double rd[RGM_KMAX];                      // reciprocals of the U pivots
    int perm[RGM_KMAX];                       // composite row permutation of the LU
    double vtw[(RGM_MMAX + 1) * RGM_KMAX];    // V^T W rows 0..nb-1 (leading dim RGM_MMAX+1)
    double g_j, wn0, tol_in;                  // scalars of the Givens step, staged
    int iters, maxit, m;
    int flag;
};
#define RGM_VTW_LD (RGM_MMAX + 1)

// ---------------------------------------------------------------- scalar helpers
// Solve with the LU factors of a k x k matrix (row swaps piv, unit lower L,
// upper U with its pivots' reciprocals rd): no divisions on the serial path.
__device__ inline void lu_solve_small(int k, const double *LU, int ld, const int *piv, const double *rd,
                                      double *x)
{
    for (int j = 0; j < k; ++j)
        if (piv[j] != j) { double t = x[j]; x[j] = x[piv[j]]; x[piv[j]] = t; }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) x[i] -= LU[i + j * ld] * x[j];
    for (int i = k - 1; i >= 0; --i) {
        for (int j = i + 1; j < k; ++j) x[i] -= LU[i + j * ld] * x[j];
        x[i] *= rd[i];
    }
}

// Stage the k x k LU factors, pivots and pivot reciprocals of E in shared
// memory (whole block).
__device__ inline void stage_lu(const Small *s, int k, FinScratch &f, int sel)
{
    const double *LU = sel ? s->LUP : s->LU, *rd = sel ? s->LUPrd : s->LUrd;
    const int *piv = sel ? s->pivP : s->piv, *pm = sel ? s->LUPperm : s->LUperm;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        int i = t % k, j = t / k;
        f.LU[i + j * RGM_KMAX] = LU[i + j * RGM_KMAX];
    }
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        f.piv[t] = piv[t];
        f.rd[t] = rd[t];
        f.perm[t] = pm[t];
    }
}

// Warp-parallel solve with the staged LU factors (k <= 32): lane i enters with
// b[perm[i]] and leaves with x_i.  3k binary64 warp instructions instead of a
// k^2 chain in one thread.
__device__ __forceinline__ double warp_lu_solve(int k, const FinScratch &f, double x)
{
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < k - 1; ++j) {
        const double xj = __shfl_sync(0xffffffffu, x, j);
        if (lane > j && lane < k) x = fma(-f.LU[lane + j * RGM_KMAX], xj, x);
    }
    for (int j = k - 1; j >= 0; --j) {
        if (lane == j) x *= f.rd[j];
        const double xj = __shfl_sync(0xffffffffu, x, j);
        if (lane < j) x = fma(-f.LU[lane + j * RGM_KMAX], xj, x);
    }
    return x;
}

// The new Hessenberg column after the stored rotations, as an affine scan.
// Rotation i maps (t_i, h_{i+1}) to (cs_i t_i + sn_i h_{i+1}, t_{i+1}) with
// t_{i+1} = -sn_i t_i + cs_i h_{i+1}, t_0 = h_0; the recurrence for t is
// composed over the warp in log2(32) steps (chunks of 32 rotations in turn).
// One warp; on return col[0..j-1] hold the rotated entries and the return
// value is t_j (entry j before the new rotation).  h: col on entry.
__device__ __forceinline__ double warp_rotate_column(double *col, const double *cs, const double *sn, int j)
{
    const int lane = threadIdx.x & 31;
    double tin = col[0];
    for (int base = 0; base < j; base += 32) {
        const int i = base + lane;
        const bool ok = i < j;
        const double c = ok ? cs[i] : 1.0, sg = ok ? sn[i] : 0.0, h1 = ok ? col[i + 1] : 0.0;
        double A = ok ? -sg : 1.0, B = ok ? c * h1 : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double A1 = __shfl_up_sync(0xffffffffu, A, o), B1 = __shfl_up_sync(0xffffffffu, B, o);
            if (lane >= o) {
                B = fma(A, B1, B);
                A = A * A1;
            }
        }
        const double tnext = fma(A, tin, B);                   // t_{i+1}
        double tcur = __shfl_up_sync(0xffffffffu, tnext, 1);   // t_i
        if (lane == 0) tcur = tin;
        __syncwarp();
        if (ok) col[i] = fma(c, tcur, sg * h1);
        tin = __shfl_sync(0xffffffffu, tnext, min(31, j - 1 - base));
        __syncwarp();
    }
    return tin;
}

// Rotate column c (in shared memory, rows 0..col+1) by rotations 0..col-1.
__device__ inline void apply_rotations(double *c, const double *cs, const double *sn, int col)
{
    for (int i = 0; i < col; ++i) {
        double a = c[i], b = c[i + 1];
        c[i] = cs[i] * a + sn[i] * b;
        c[i + 1] = -sn[i] * a + cs[i] * b;
    }
}

// Givens rotation from (a, hn), hn = sqrt(hn2) >= 0: c = a / r, s = hn / r,
// r = hypot(a, hn), formed from the pair scaled by t = max(|a|, hn) so that
// no square overflows or underflows before r does (hn2 > 0 is the squared norm
// the reduction gave; its square root is taken once).  r = 0 gives (1, 0).
__device__ __forceinline__ void givens_scaled(double a, double hn2, double *c, double *s, double *r,
                                              double *hn_out)
{
    const double hn = sqrt(hn2);
    const double t = fmax(fabs(a), hn);
    if (t == 0.0) {
        *c = 1.0; *s = 0.0; *r = 0.0; *hn_out = 0.0;
        return;
    }
    const double rt = 1.0 / t, as = a * rt, hs = hn * rt;
    const double rr = t * sqrt(fma(as, as, hs * hs));
    const double ir = 1.0 / rr;
    *c = a * ir;
    *s = hn * ir;
    *r = rr;
    *hn_out = hn;
}

// Finalise one Hessenberg column held in f.col (rows 0..nb, already rotated):
// make rotation col, update g, write the column and the rotation back.
__device__ inline void close_column(Small *s, FinScratch &f, int col)
{
    if (threadIdx.x == 0) {
        double a = f.col[col], b = f.col[col + 1];
        double r = hypot(a, b);
        double c = 1.0, sn = 0.0;
        if (r != 0.0) { c = a / r; sn = b / r; }
        s->cs[col] = c;
        s->sn[col] = sn;
        f.col[col] = r;
        f.col[col + 1] = 0.0;
        double g0 = s->g[col];
        s->g[col + 1] = -sn * g0;
        s->g[col] = c * g0;
    }
    __syncthreads();
    double *hc = s->H + (int64_t)col * RGM_HLD;
    for (int i = threadIdx.x; i <= col + 1; i += blockDim.x) hc[i] = f.col[i];
}

// Loads of the small state the scalar step needs, issued by the finalising
// block together with the loads of the partial sums (one round trip for both).
// Counts come from the pass itself: nb = op.ndV for the first and second CGS
// passes (DYN_NDV_NB), op.nV for the third (DYN_NV_NB).
// The scalars the serial part of the Givens step reads, one load per thread
// (issued together, so the serial part does no dependent global load).
__device__ __forceinline__ void stage_givens_scalars(const Small *s, int j, FinScratch &f)
{
    switch (threadIdx.x) {
    case 0: f.g_j = s->g[j]; break;
    case 1: f.wn0 = s->wn0; break;
    case 2: f.tol_in = s->tol_in; break;
    case 3: f.iters = s->iters; break;
    case 4: f.maxit = s->maxit; break;
    case 5: f.m = s->m; break;
    default: break;
    }
}

template <typename T>
__device__ void fin_stage(const VecOp<T> &op, FinScratch &f)
{
    const Small *s = op.sm;
    const int tid = threadIdx.x;
    switch (op.fin) {
    case FIN_COARSE:
    case FIN_START_DEF1:
        stage_lu(s, op.ndU, f, op.lu_sel);
        break;
    case FIN_ARN1:
    case FIN_AUG1: {
        // every load in flight before the first shared-memory store (a store
        // waits for its data, and a later load would wait behind it)
        const int nb = op.ndV, k = op.ndU, sel = op.lu_sel;
        const double *LU = sel ? s->LUP : s->LU, *rd = sel ? s->LUPrd : s->LUrd;
        const int *piv = sel ? s->pivP : s->piv, *pm = sel ? s->LUPperm : s->LUperm;
        static_assert(RGM_HLD <= RGM_THREADS, "one thread per basis column");
        double lu[2], vt[2], rdv = 0.0, scv = 0.0;
        int pvv = 0, pmv = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = tid + u * RGM_THREADS;
            lu[u] = (t < k * k) ? LU[t % k + (t / k) * RGM_KMAX] : 0.0;
        }
        if (tid < k) { pvv = piv[tid]; rdv = rd[tid]; pmv = pm[tid]; }
        if (tid < nb) scv = s->colscale[tid];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = tid + u * RGM_THREADS;
            vt[u] = (t < nb * k) ? s->VtW[t % nb + (t / nb) * RGM_HLD] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = tid + u * RGM_THREADS;
            if (t < k * k) f.LU[t % k + (t / k) * RGM_KMAX] = lu[u];
        }
        for (int t = tid + 2 * RGM_THREADS; t < k * k; t += RGM_THREADS)
            f.LU[t % k + (t / k) * RGM_KMAX] = LU[t % k + (t / k) * RGM_KMAX];
        if (tid < k) { f.piv[tid] = pvv; f.rd[tid] = rdv; f.perm[tid] = pmv; }
        if (tid < nb) f.sc[tid] = scv;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = tid + u * RGM_THREADS;
            if (t < nb * k) f.vtw[t % nb + (t / nb) * RGM_VTW_LD] = vt[u];
        }
        for (int t = tid + 2 * RGM_THREADS; t < nb * k; t += RGM_THREADS)
            f.vtw[t % nb + (t / nb) * RGM_VTW_LD] = s->VtW[t % nb + (t / nb) * RGM_HLD];
        break;
    }
    case FIN_ARN2:
        for (int i = tid; i < op.ndV; i += blockDim.x) {
            f.sc[i] = s->colscale[i];
            f.col[i] = s->hsum[i];
        }
        break;
    case FIN_ARN2H: {
        // loads first, then stores (as for FIN_ARN1); nb <= RGM_HLD < threads
        const int nb = op.ndV, k = op.ndW;
        double scv = 0.0, hv = 0.0, csv = 0.0, snv = 0.0, vt[2];
        if (tid < nb) { scv = s->colscale[tid]; hv = s->hsum[tid]; csv = s->cs[tid]; snv = s->sn[tid]; }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = tid + u * RGM_THREADS;
            vt[u] = (t < nb * k) ? s->VtW[t % nb + (t / nb) * RGM_HLD] : 0.0;
        }
        stage_givens_scalars(s, nb - 1, f);
        if (tid < nb) { f.sc[tid] = scv; f.col[tid] = hv; f.cs[tid] = csv; f.sn[tid] = snv; }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = tid + u * RGM_THREADS;
            if (t < nb * k) f.vtw[t % nb + (t / nb) * RGM_VTW_LD] = vt[u];
        }
        for (int t = tid + 2 * RGM_THREADS; t < nb * k; t += RGM_THREADS)
            f.vtw[t % nb + (t / nb) * RGM_VTW_LD] = s->VtW[t % nb + (t / nb) * RGM_HLD];
        break;
    }
    case FIN_ARN3:
        stage_givens_scalars(s, op.nV - 1, f);
        for (int i = tid; i < op.nV; i += blockDim.x) {
            f.col[i] = s->hsum[i];
            f.cs[i] = s->cs[i];
            f.sn[i] = s->sn[i];
        }
        break;
    default:
        break;
    }
}

// The scalar step after a reduction, run by the whole finalising block.
// d[] holds the reduced dots in the column order [U | Vraw | W | norm].
template <typename T>
__device__ void finalize_block(const VecOp<T> &op, const double *d, FinScratch &f)
{
    Small *s = op.sm;
    const double *dU = d, *dV = d + op.ndU, *dW = d + op.ndU + op.ndV;
    const double nrm2 = op.dnorm ? d[op.ndU + op.ndV + op.ndW] : 0.0;
    const int tid = threadIdx.x;
    switch (op.fin) {
    case FIN_BNORM:
        if (tid == 0) s->bnorm = sqrt(nrm2);
        break;
    case FIN_BNORMP:
        if (tid == 0) s->bnorm_p = sqrt(nrm2);
        break;
    case FIN_RESNORM:
        if (tid == 0) {
            s->beta = sqrt(nrm2);
            s->converged = (s->beta <= s->tol_abs) ? 1 : 0;
        }
        break;
    case FIN_COARSE:
    case FIN_START_DEF1: {
        const int k = op.ndU;           // LU staged by fin_stage
        if (tid < 32) {
            const double x = warp_lu_solve(k, f, tid < k ? dU[f.perm[tid]] : 0.0);
            if (tid < k) f.dd[tid] = x;
        }
        __syncthreads();
        // FIN_COARSE: x += U c, and r -= W c (W = A U) where the residual of
        // the corrected x is updated instead of recomputed
        for (int i = tid; i < k; i += blockDim.x) {
            if (op.fin == FIN_COARSE) s->coefU[i] = f.dd[i];
            s->coefW[i] = -f.dd[i];
        }
        break;
    }
    case FIN_START_PLAIN:
    case FIN_START_DEF2: {
        const double bs = sqrt(nrm2), sc = bs > 0.0 ? 1.0 / bs : 0.0;
        if (tid == 0) {
            s->bs = bs;
            s->J = 0;
            s->nb = 1;
            s->naug = 0;
            s->g[0] = bs;
            s->colscale[0] = sc;
            s->done = (bs > 0.0) ? 0 : 1;
            s->breakdown = 0;
        }
        for (int l = tid; l < op.ndW; l += blockDim.x) s->VtW[0 + l * RGM_HLD] = dW[l] * sc;
        break;
    }
    case FIN_ARN1:
    case FIN_AUG1: {
        // w = A v_j (or A u_i).  Deflated: P w = w - W d, d = E^{-1} U^T w, and
        // V^T P w = V^T w - (V^T W) d.
        // LU, colscale and V^T W staged by fin_stage (nb = op.ndV)
        const int nb = op.ndV, k = op.ndU;
        if (tid < 32 && k) {
            const double x = warp_lu_solve(k, f, tid < k ? dU[f.perm[tid]] : 0.0);
            if (tid < k) f.dd[tid] = x;
        }
        if (tid == 32) {
            s->wn0 = sqrt(nrm2);
            if (op.fin == FIN_AUG1) s->skip = (nrm2 == 0.0) ? 1 : 0;
        }
        __syncthreads();
        for (int i = tid; i < k; i += blockDim.x) s->coefW[i] = -f.dd[i];
        for (int i = tid; i < nb; i += blockDim.x) {
            double h = dV[i] * f.sc[i];
            for (int l = 0; l < k; ++l) h -= f.vtw[i + l * RGM_VTW_LD] * f.dd[l];
            s->hsum[i] = h;
            s->coefV[i] = -h * f.sc[i];
        }
        break;
    }
    case FIN_ARN2: {
        // colscale and hsum staged by fin_stage (nb = op.ndV)
        const int nb = op.ndV;
        for (int i = tid; i < nb; i += blockDim.x) {
            const double sc = f.sc[i];
            const double h = dV[i] * sc;
            s->hsum[i] = f.col[i] + h;
            s->coefV[i] = -h * sc;
        }
        break;
    }
    case FIN_ARN2H: {
        // w1 = w after the first CGS pass; d: [V^T w1 | W^T w1 | ||w1||^2].  The
        // second pass removes h2 = V^T w1, and since V is orthonormal
        // ||w1 - V h2||^2 = ||w1||^2 - ||h2||^2 (no cancellation: w1 is already
        // orthogonal to V up to rounding); v_{j+1}^T W follows from W^T w1 and
        // the stored rows of V^T W.  Staged: colscale, hsum, cs, sn, V^T W.
        const int nb = op.ndV, j = nb - 1, kw = op.ndW;
        __shared__ double sc_h;
        for (int i = tid; i < nb; i += blockDim.x) {
            const double sc = f.sc[i], h = dV[i] * sc;
            f.h2[i] = h;
            f.col[i] += h;                     // the Hessenberg column h1 + h2
            s->coefV[i] = -h * sc;
        }
        if (tid == 0) {
            s->J = j + 1;
            s->nb = nb + 1;
        }
        __syncthreads();
        // The next pass (v_{j+1} = w1 - V h2, unnormalised) needs only the
        // coefficients and the column count above: with op.release_gen the
        // waiting blocks are released here, and the rest of the scalar step
        // (rotation, scale, flags, V^T W row) overlaps their next pass; its
        // results are published by the barrier that ends that pass.
        if (op.release_gen && tid == 0) st_release_gpu(&s->gen, op.release_gen);
        if (tid < 32) {
            double q = 0.0;
            for (int i = tid; i < nb; i += 32) q = fma(f.h2[i], f.h2[i], q);
            q = warp_sum(q);
            const double hn2 = fmax(nrm2 - q, 0.0);
            // rotated column (warp 0), then the new rotation from (t_j, hn)
            const double a = warp_rotate_column(f.col, f.cs, f.sn, j);
            if (tid == 0) {
                double c, sn, rr, hn;
                givens_scaled(a, hn2, &c, &sn, &rr, &hn);
                const double inv_hn = (hn > 0.0) ? 1.0 / hn : 0.0;
                f.col[j] = rr;
                f.col[j + 1] = 0.0;
                s->cs[j] = c;
                s->sn[j] = sn;
                const double g0 = f.g_j, g1 = -sn * g0;
                s->g[j + 1] = g1;
                s->g[j] = c * g0;
                const bool brk = hn <= 1e-14 * f.wn0;
                const double sc = brk ? 0.0 : inv_hn;
                sc_h = sc;
                const int it = f.iters + 1;
                s->iters = it;
                s->colscale[nb] = sc;          // happy breakdown: v_{j+1} := 0
                int done = 0;
                if (brk) { s->breakdown = 1; done = 1; }
                if (fabs(g1) <= f.tol_in || it >= f.maxit || j + 1 >= f.m) done = 1;
                if (done) s->done = 1;
                if (op.mirror) {          // progress for the host's launch lookahead
                    op.mirror[1] = (unsigned)done;
                    op.mirror[0] = (unsigned)(j + 1);
                    __threadfence_system();
                }
            }
        }
        __syncthreads();
        double *hc = s->H + (int64_t)j * RGM_HLD;
        for (int i = tid; i <= j + 1; i += blockDim.x) hc[i] = f.col[i];
        const double sc = sc_h;
        // one thread per column l (a chain, but the fewest binary64 operations:
        // a warp tree would multiply the pipe's work by 32)
        for (int l = tid; l < kw; l += blockDim.x) {
            double v = dW[l];
            for (int i = 0; i < nb; ++i) v = fma(-f.h2[i], f.vtw[i + l * RGM_VTW_LD], v);
            s->VtW[nb + l * RGM_HLD] = v * sc;
        }
        break;
    }
    case FIN_ARN3: {
        // hsum, cs and sn staged by fin_stage (nb = op.nV = J + 1)
        const int nb = op.nV, j = nb - 1;
        __shared__ double sc_sh;
        if (tid < 32) {
            // rotated column (warp 0), then the new rotation from (t_j, ||w||)
            const double a = warp_rotate_column(f.col, f.cs, f.sn, j);
            if (tid == 0) {
                double c, sn, rr, hn;
                givens_scaled(a, nrm2, &c, &sn, &rr, &hn);
                const double inv_hn = (hn > 0.0) ? 1.0 / hn : 0.0;
                f.col[j] = rr;
                f.col[j + 1] = 0.0;
                s->cs[j] = c;
                s->sn[j] = sn;
                const double g0 = f.g_j, g1 = -sn * g0;
                s->g[j + 1] = g1;
                s->g[j] = c * g0;
                const bool brk = hn <= 1e-14 * f.wn0;
                const double sc = brk ? 0.0 : inv_hn;
                sc_sh = sc;
                s->J = j + 1;
                const int it = f.iters + 1;
                s->iters = it;
                s->colscale[nb] = sc;          // happy breakdown: v_{j+1} := 0
                int done = 0;
                if (brk) { s->breakdown = 1; done = 1; }
                s->nb = nb + 1;
                if (fabs(g1) <= f.tol_in || it >= f.maxit || j + 1 >= f.m) done = 1;
                if (done) s->done = 1;
            }
        }
        __syncthreads();
        double *hc = s->H + (int64_t)j * RGM_HLD;
        for (int i = tid; i <= j + 1; i += blockDim.x) hc[i] = f.col[i];
        const double sc = sc_sh;
        for (int l = tid; l < op.ndW; l += blockDim.x) s->VtW[nb + l * RGM_HLD] = dW[l] * sc;
        break;
    }
    case FIN_AUG3: {
        const int nb = s->nb, col = s->J + s->naug;
        const double hn = sqrt(nrm2);
        for (int i = tid; i <= col + 1 && i <= RGM_HLD; i += blockDim.x) f.col[i] = 0.0;
        __syncthreads();
        for (int i = tid; i < nb; i += blockDim.x) f.col[i] = s->hsum[i];
        for (int i = tid; i < col; i += blockDim.x) { f.cs[i] = s->cs[i]; f.sn[i] = s->sn[i]; }
        if (tid == 0) f.col[nb] = hn;
        __syncthreads();
        if (tid == 0) {
            apply_rotations(f.col, f.cs, f.sn, col);
            // dependent on the columns already in the relation: drop u_i
            f.flag = (hypot(f.col[col], f.col[col + 1]) <= 1e-14 * s->wn0) ? 0 : 1;
        }
        __syncthreads();
        if (!f.flag) break;
        close_column(s, f, col);
        if (tid == 0) {
            s->colscale[nb] = (hn <= 1e-14 * s->wn0) ? 0.0 : 1.0 / hn;
            s->aug_idx[s->naug] = op.arg;
            s->naug += 1;
            s->nb = nb + 1;
        }
        break;
    }
    case FIN_DOTS: {
        const int nd = op.ndU + op.ndV + op.ndW + op.dnorm;
        for (int i = tid; i < nd; i += blockDim.x) s->dots[i] = d[i];
        break;
    }
    default:
        break;
    }
}

// Warp sums of the QMAX per-lane values v[q] (column warp + q * NW of a pass);
// store(c, sum) is called once per column c < nd by one lane.  For power-of-2
// QMAX the butterfly halves the live values at each step (QMAX-1 + 5 -
// log2 QMAX binary64 adds per warp instead of 5 QMAX: the FP64 pipe is narrow).
template <int QMAX, typename Store>
__device__ __forceinline__ void warp_sums_store(double (&v)[QMAX], int nd, Store store)
{
    constexpr int NW = RGM_THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr ((QMAX & (QMAX - 1)) == 0 && QMAX <= 32) {
        warp_multi_reduce<QMAX>(v);
        const int sh = warp_multi_owner_shift<QMAX>();
        const int c = warp + (lane >> sh) * NW;
        if ((lane & ((1 << sh) - 1)) == 0 && c < nd) store(c, v[0]);
    } else {
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            const int c = warp + q * NW;
            if (c < nd) {
                const double t = warp_sum(v[q]);
                if (lane == 0) store(c, t);
            }
        }
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

// ---------------------------------------------------------------- 16-byte vector access
// The streaming loops move 16 bytes per lane per load (4 binary32 or 2 binary64
// values): a quarter (a half) of the load instructions of one value per lane,
// and four (two) times the bytes in flight per instruction.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; using itype = int4; };
template <> struct Vec16<double> { using type = double2; using itype = int2; };

template <typename V, typename T>
__device__ __forceinline__ T vcomp(const V &v, int t) { return reinterpret_cast<const T *>(&v)[t]; }
template <typename V>
__device__ __forceinline__ int icomp(const V &v, int t) { return reinterpret_cast<const int *>(&v)[t]; }

// Loads of the operator's stored values and columns.  They are read once per
// Arnoldi step, while the Krylov basis, W, U and the vector being multiplied
// are read again by the next passes: the operator is loaded with the streaming
// (evict-first) hint so that it does not push those out of L2.
#ifndef RGM_STREAM_A
#define RGM_STREAM_A 1
#endif
template <typename V>
__device__ __forceinline__ V ld_op(const V *p)
{
#if RGM_STREAM_A
    return __ldcs(p);
#else
    return *p;
#endif
}

// The end of a slice's row sums: acc[t] of lane l holds the partial sum of row
// VW (l % (32/VW)) + t over the whole chunks of the slice; lanes l, l + 32/VW,
// .. saw the same rows and are added by a butterfly, then row `lane` takes the
// columns k0 .. wd - 1 past the last whole chunk one entry at a time.
template <typename T>
__device__ __forceinline__ T slice_combine(T (&acc)[16 / sizeof(T)], const T *sval, const int32_t *scol,
                                           const T *x, int64_t p0, int64_t k0, int64_t wd)
{
    constexpr int VW = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 32 / VW; o < 32; o <<= 1)
#pragma unroll
        for (int t = 0; t < VW; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    // row `lane` is component lane % VW of lane lane / VW
    T a = (T)0;
#pragma unroll
    for (int t = 0; t < VW; ++t) {
        const T v = __shfl_sync(0xffffffffu, acc[t], lane / VW);
        if ((lane % VW) == t) a = v;
    }
    for (int64_t k = k0; k < wd; ++k) {
        const int64_t e = p0 + 32 * k + lane;
        a += ld_op(sval + e) * x[ld_op(scol + e)];
    }
    return a;
}

// Row sums of one 32-row slice of the sliced-ELL operator, sum_k sval[p0 +
// 32 k + l] x[scol[p0 + 32 k + l]] for the slice's lane l (returned in lane l).
// The slice's entries are read as 16-byte vectors: in a chunk of VW slice
// columns lane l holds entries VW l .. VW l + VW - 1, i.e. VW consecutive rows
// of one column, and keeps one partial sum per row it sees; the lanes that saw
// the same rows are added by a butterfly at the end (no row is ever written by
// two lanes).  Columns past the last whole chunk are read one per lane.
template <typename T>
__device__ __forceinline__ T slice_rowsum(const T *sval, const int32_t *scol, const T *x, int64_t p0, int64_t p1)
{
    constexpr int VW = 16 / (int)sizeof(T);
    using VT = typename Vec16<T>::type;
    using VI = typename Vec16<T>::itype;
    // chunks in flight per lane (fewer when the register budget is 64)
    constexpr int U = (RGM_MINB >= 4) ? 2 : (sizeof(T) == 4) ? 4 : 2;
    const int lane = threadIdx.x & 31;
    const int64_t wd = (p1 - p0) >> 5;
    const int64_t nch = wd / VW;
    T acc[VW];
#pragma unroll
    for (int t = 0; t < VW; ++t) acc[t] = (T)0;
    const VT *vv = reinterpret_cast<const VT *>(sval + p0) + lane;
    const VI *vc = reinterpret_cast<const VI *>(scol + p0) + lane;
    int64_t ch = 0;
    for (; ch + U <= nch; ch += U) {
        VT v[U];
        VI c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = ld_op(vv + (ch + u) * 32);
            c[u] = ld_op(vc + (ch + u) * 32);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int t = 0; t < VW; ++t) acc[t] += vcomp<VT, T>(v[u], t) * x[icomp(c[u], t)];
    }
    for (; ch < nch; ++ch) {
        const VT v = ld_op(vv + ch * 32);
        const VI c = ld_op(vc + ch * 32);
#pragma unroll
        for (int t = 0; t < VW; ++t) acc[t] += vcomp<VT, T>(v, t) * x[icomp(c, t)];
    }
    return slice_combine<T>(acc, sval, scol, x, p0, nch * VW, wd);
}

// What one block did in a pass: left without touching the completion counter
// (gated off, or nothing to reduce), arrived, or arrived last and finalised.
enum PassResult { PASS_SKIPPED = 0, PASS_ARRIVED = 1, PASS_LAST = 2, PASS_RELEASED = 3 };

// One fused pass over the rows of block `bid` of the pass's grid (body of
// vec_kernel and of each phase of the cycle kernels; bid is the block's index
// among the op.nblocks blocks that run the pass).  PDL: signal programmatic
// dependents once the partials are written.
template <typename T, int QMAX, bool PDL>
__device__ __forceinline__ int vec_pass(VecOp<T> op, const int bid)
{
    constexpr int NW = RGM_THREADS / 32;      // QMAX * NW >= number of dot columns
    Small *s = op.sm;
    if (op.gate == GATE_KRYLOV && s->done) return PASS_SKIPPED;
    if (op.gate == GATE_APPEND && (s->skip || s->J == 0)) return PASS_SKIPPED;
    if (op.gate == GATE_STEP && s->J != op.arg) return PASS_SKIPPED;
    if (op.dyn) {
        if (op.dyn & DYN_NDV_NB) op.ndV = s->nb;
        if (op.dyn & DYN_NV_NB) op.nV = s->nb;
        if (op.dyn & DYN_NV_J) op.nV = s->J;
        if (op.dyn & DYN_OUT_VNB) op.out = const_cast<T *>(op.V) + (int64_t)s->nb * op.ldv;
        if (op.dyn & DYN_NV_NBM1) op.nV = s->nb - 1;
        if (op.dyn & DYN_OUT_VNBM1) op.out = const_cast<T *>(op.V) + (int64_t)(s->nb - 1) * op.ldv;
    }

    constexpr int VW = 16 / (int)sizeof(T);   // values per 16-byte vector
    using VT = typename Vec16<T>::type;
    constexpr int NG = RGM_TILE / VW;          // AXPY: row groups of VW rows in a tile
    constexpr int NPH = RGM_THREADS / NG;      //       column phases (threads per row group)
    static_assert(NPH >= 1 && NG * NPH == RGM_THREADS, "AXPY thread layout");
    __shared__ T cW[RGM_KMAX], cU[RGM_KMAX], cV[RGM_HLD];
    // AXPY columns [W | Vraw | U] as one list: pointer and coefficient
    __shared__ const T *acol[RGM_KMAX + RGM_HLD + RGM_KMAX];
    __shared__ T acoef[RGM_KMAX + RGM_HLD + RGM_KMAX];
    // One pool for the large shared arrays: w on a chunk (binary32) or a tile
    // (binary64) and the binary64 AXPY partial sums per column phase, and -- in
    // the block that finalises, after those are dead -- the scalar step's scratch.
    constexpr int WS_BYTES = ((sizeof(T) == 4) ? 8 : 1) * RGM_TILE * (int)sizeof(T);
    constexpr int AP_BYTES = ((sizeof(T) == 8) ? NPH * RGM_TILE : VW) * (int)sizeof(T);
    constexpr int MAIN_BYTES = WS_BYTES + AP_BYTES;
    constexpr int POOL_BYTES = MAIN_BYTES > (int)sizeof(FinScratch) ? MAIN_BYTES : (int)sizeof(FinScratch);
    __shared__ __align__(16) unsigned char pool[POOL_BYTES];
    T *ws = reinterpret_cast<T *>(pool);
    T *apart = reinterpret_cast<T *>(pool + WS_BYTES);
    __shared__ double xs;
    if (threadIdx.x == 0) xs = (op.xscale >= 0) ? s->colscale[op.xscale] : 1.0;
    const int nac = (op.src == SRC_AXPY) ? op.nW + op.nV + op.nU : 0;
    if (op.src == SRC_AXPY) {
        for (int i = threadIdx.x; i < op.nW; i += blockDim.x) {
            cW[i] = (T)s->coefW[i];
            acol[i] = op.W + (int64_t)i * op.ldw;
            acoef[i] = cW[i];
        }
        for (int i = threadIdx.x; i < op.nV; i += blockDim.x) {
            cV[i] = (T)s->coefV[i];
            acol[op.nW + i] = op.V + (int64_t)i * op.ldv;
            acoef[op.nW + i] = cV[i];
        }
        for (int i = threadIdx.x; i < op.nU; i += blockDim.x) {
            cU[i] = (T)s->coefU[i];
            acol[op.nW + op.nV + i] = op.U + (int64_t)i * op.ldu;
            acoef[op.nW + op.nV + i] = cU[i];
        }
    }
    __syncthreads();

    const int nd = op.ndU + op.ndV + op.ndW + op.dnorm;
    const int ndc_ = op.dnorm ? nd - 1 : -1;          // index of the ||w||^2 column
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)bid * op.rpb;
    const int64_t r1 = min(op.n, r0 + op.rpb);
    double acc[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) acc[q] = 0.0;

    const bool spmv_src = (op.src == SRC_SPMV || op.src == SRC_RES);
    if constexpr (sizeof(T) == 4) {
        // Rows are taken in chunks of up to CHT tiles: phase 1 produces w on every
        // row of the chunk (stored, and kept in shared memory), phase 2 streams each
        // dot column over the whole chunk, one warp per column -- long runs of
        // independent 16-byte loads instead of one short tile at a time.
    #ifndef RGM_CHT
    #define RGM_CHT 8
    #endif
        constexpr int CHT = RGM_CHT;                            // tiles per chunk (8: 8 KB of w)
        static_assert(CHT >= 1 && CHT <= 8, "ws holds 8 tiles");
    #ifndef RGM_DU
    #define RGM_DU 4
    #endif
        constexpr int DU = RGM_DU;                                  // vectors in flight per lane
        for (int64_t cb = r0; cb < r1; cb += (int64_t)CHT * RGM_TILE) {
            const int64_t ce = min(r1, cb + (int64_t)CHT * RGM_TILE);
            const int nr = (int)(ce - cb);
            const int ntc = (nr + RGM_TILE - 1) / RGM_TILE;
            // ---- phase 1: produce and store w on the chunk
            if (spmv_src) {
                // one warp per 32-row slice, one lane per row.  Inside a tile the
                // slices are sorted by width (slice 0 widest), so warp w takes slice
                // w of even tiles and slice NW-1-w of odd ones: every warp gets the
                // same work.
                const T sc = (T)xs;
                for (int t = 0; t < ntc; ++t) {
                    const int64_t base = cb + (int64_t)t * RGM_TILE;
                    const int slot = (t & 1) ? (NW - 1 - warp) : warp;
                    const int64_t sl = (base >> 5) + slot;
                    const int64_t p0 = op.slice_ptr[sl], p1 = op.slice_ptr[sl + 1];
                    const T a = slice_rowsum<T>(op.sval, op.scol, op.x, p0, p1);
                    const int pr = op.perm[(sl << 5) + lane];
                    if (pr >= 0) {
                        const T v = (op.src == SRC_SPMV) ? a * sc : op.b[pr] - a;
                        op.out[pr] = v;
                        ws[pr - cb] = v;
                    }
                }
            } else if (op.src == SRC_AXPY) {
                // thread t takes the 16-byte row groups t, t + 256, .. of the
                // chunk over all columns [W | Vraw | U]: its loads are independent
                // (no per-tile barrier); rows past the last whole group (the end of
                // the matrix only) one per thread
                const int G = nr / VW;
                for (int g = threadIdx.x; g < G; g += RGM_THREADS) {
                    const int64_t r = cb + (int64_t)VW * g;
                    VT a = *reinterpret_cast<const VT *>(op.win + r);
#pragma unroll 8
                    for (int c = 0; c < nac; ++c) {
                        const VT v = *reinterpret_cast<const VT *>(acol[c] + r);
                        const T cf = acoef[c];
#pragma unroll
                        for (int q = 0; q < VW; ++q)
                            reinterpret_cast<T *>(&a)[q] += cf * vcomp<VT, T>(v, q);
                    }
                    *reinterpret_cast<VT *>(op.out + r) = a;
                    reinterpret_cast<VT *>(ws)[g] = a;
                }
                for (int i = VW * G + (int)threadIdx.x; i < nr; i += RGM_THREADS) {
                    const int64_t r = cb + i;
                    T a = op.win[r];
                    for (int c = 0; c < nac; ++c) a += acoef[c] * acol[c][r];
                    op.out[r] = a;
                    ws[i] = a;
                }
            } else if (op.src == SRC_COPY) {
                for (int i = threadIdx.x; i < nr; i += RGM_THREADS) {
                    const T a = op.win[cb + i];
                    op.out[cb + i] = a;
                    ws[i] = a;
                }
            }
            if (nd == 0) continue;     // nothing reads ws; the next chunk's writes need no barrier
            __syncthreads();
            // ---- phase 2: dot products, one warp per column streaming over the
            // chunk: lane l reads the 16-byte vectors l, l + 32, .. of its column
            // (and of w from shared memory), DU of them in flight; binary32 products
            // are summed 4 vectors at a time and those sums added in binary64
            const int G = nr / VW;                               // whole vectors in the chunk
            const VT *wv = reinterpret_cast<const VT *>(ws);
    #pragma unroll
            for (int q = 0; q < QMAX; ++q) {
                const int c = warp + q * NW;
                if (c >= nd) continue;
                const bool norm = (c == ndc_);
                const T *cp = norm ? op.wvec : dot_col(op, c);
                const bool load = !norm || cp != nullptr;
                const VT *cv = load ? reinterpret_cast<const VT *>(cp + cb) : nullptr;
                double sacc = 0.0;
                for (int g0 = 0; g0 < G; g0 += 32 * DU) {
                    VT x[DU];
    #pragma unroll
                    for (int u = 0; u < DU; ++u) {
                        const int gi = g0 + lane + 32 * u;
                        if (load && gi < G) x[u] = cv[gi];
                    }
    #pragma unroll
                    for (int h = 0; h < DU; h += 4) {
                        T a = 0;
    #pragma unroll
                        for (int u = h; u < h + 4 && u < DU; ++u) {
                            const int gi = g0 + lane + 32 * u;
                            if (gi < G) {
                                const VT w = wv[gi];
    #pragma unroll
                                for (int t = 0; t < VW; ++t) {
                                    const T wt = vcomp<VT, T>(w, t);
                                    if (!norm) {
                                        a += vcomp<VT, T>(x[u], t) * wt;
                                    } else {
                                        const T v = load ? wt * vcomp<VT, T>(x[u], t) : wt;
                                        a += v * v;
                                    }
                                }
                            }
                        }
                        sacc += (double)a;
                    }
                }
                // rows past the last whole vector (the end of the matrix only)
                for (int i = VW * G + lane; i < nr; i += 32) {
                    const T wt = ws[i];
                    if (!norm) {
                        sacc += (double)(cp[cb + i] * wt);
                    } else {
                        const T v = load ? wt * cp[cb + i] : wt;
                        sacc += (double)(v * v);
                    }
                }
                acc[q] += sacc;
            }
            __syncthreads();           // ws is rewritten by the next chunk
        }
    } else {
        // binary64: the work is bound by the binary64 pipe rather than by
        // loads in flight, and the tile loop (w of one tile in shared memory,
        // the dots of each tile right after it) measured faster than chunks
        const int ntiles_blk = (int)((r1 - r0 + RGM_TILE - 1) / RGM_TILE);
        if (spmv_src && ntiles_blk > 1) {
            // SpMV over all of the block's slices first.  Inside a tile the slices
            // are sorted by width (slice 0 widest), so warp w takes slice w of even
            // tiles and slice NW-1-w of odd ones: every warp gets the same work.
            const T sc = (T)xs;
            for (int t = 0; t < ntiles_blk; ++t) {
                const int64_t base = r0 + (int64_t)t * RGM_TILE;
                const int slot = (t & 1) ? (NW - 1 - warp) : warp;
                const int64_t sl = (base >> 5) + slot;
                const int64_t p0 = op.slice_ptr[sl], p1 = op.slice_ptr[sl + 1];
                const T a = slice_rowsum<T>(op.sval, op.scol, op.x, p0, p1);
                const int pr = op.perm[(sl << 5) + lane];
                if (pr >= 0) op.out[pr] = (op.src == SRC_SPMV) ? a * sc : op.b[pr] - a;
            }
            __syncthreads();      // the block's own writes are visible to it now
        }
        for (int64_t base = r0; base < r1; base += RGM_TILE) {
            const int nrow = (int)min((int64_t)RGM_TILE, r1 - base);
            // ---- phase 1: produce and store w on this tile
            if (spmv_src && ntiles_blk > 1) {
                if ((int)threadIdx.x < nrow) ws[threadIdx.x] = op.out[base + threadIdx.x];
            } else if (spmv_src) {
                // one warp per 32-row slice of the tile, one lane per row; the
                // slice's entries are independent loads (unrolled below)
                const int64_t sl = (base >> 5) + warp;
                const int64_t p0 = op.slice_ptr[sl], p1 = op.slice_ptr[sl + 1];
                const T sc = (T)xs;
                const T a = slice_rowsum<T>(op.sval, op.scol, op.x, p0, p1);
                const int pr = op.perm[(sl << 5) + lane];
                if (pr >= 0) {
                    const T v = (op.src == SRC_SPMV) ? a * sc : op.b[pr] - a;
                    op.out[pr] = v;
                    ws[pr - base] = v;
                }
            } else if (op.src == SRC_AXPY && nrow == RGM_TILE) {
                // full tile: thread (g, ph) sums the columns c = ph (mod NPH) over
                // rows base + VW g .. + VW - 1 with 16-byte loads, all of its
                // columns' loads in flight together; the NPH partial sums of a row
                // are added through shared memory
                const int g = threadIdx.x % NG, ph = threadIdx.x / NG;
                const int64_t r = base + (int64_t)VW * g;
                VT a;
    #pragma unroll
                for (int t = 0; t < VW; ++t) reinterpret_cast<T *>(&a)[t] = (T)0;
                if (ph == 0) a = *reinterpret_cast<const VT *>(op.win + r);
    #pragma unroll 8
                for (int c = ph; c < nac; c += NPH) {
                    const VT v = *reinterpret_cast<const VT *>(acol[c] + r);
                    const T cf = acoef[c];
    #pragma unroll
                    for (int t = 0; t < VW; ++t)
                        reinterpret_cast<T *>(&a)[t] += cf * vcomp<VT, T>(v, t);
                }
                reinterpret_cast<VT *>(apart + ph * RGM_TILE)[g] = a;
                __syncthreads();
                const int t = threadIdx.x;
                T sum = apart[t];
    #pragma unroll
                for (int q = 1; q < NPH; ++q) sum += apart[q * RGM_TILE + t];
                op.out[base + t] = sum;
                ws[t] = sum;
                if (nd == 0) __syncthreads();      // apart is rewritten by the next tile
            } else if (op.src == SRC_COPY || op.src == SRC_AXPY) {
                const int t = threadIdx.x;
                if (t < nrow) {
                    const int64_t r = base + t;
                    T a = op.win[r];
                    if (op.src == SRC_AXPY) {
    #pragma unroll 4
                        for (int c = 0; c < op.nW; ++c) a += cW[c] * op.W[r + (int64_t)c * op.ldw];
    #pragma unroll 8
                        for (int c = 0; c < op.nV; ++c) a += cV[c] * op.V[r + (int64_t)c * op.ldv];
    #pragma unroll 4
                        for (int c = 0; c < op.nU; ++c) a += cU[c] * op.U[r + (int64_t)c * op.ldu];
                    }
                    op.out[r] = a;
                    ws[t] = a;
                }
            }
            if (nd == 0) continue;
            __syncthreads();
            // ---- phase 2: dot products, one warp per column over the tile
            if (nrow == RGM_TILE) {
                // full tile: 16-byte loads, lane l holding rows VW l + 32 VW i ..;
                // the loads of QG columns are in flight together
                constexpr int NVL = RGM_TILE / (32 * VW);
                constexpr int QG = (RGM_MINB >= 4) ? 1 : (sizeof(T) == 4) ? 2 : 1;
                VT wl[NVL];
    #pragma unroll
                for (int i = 0; i < NVL; ++i) wl[i] = reinterpret_cast<const VT *>(ws)[lane + 32 * i];
    #pragma unroll
                for (int q0 = 0; q0 < QMAX; q0 += QG) {
                    VT cv[QG][NVL];
    #pragma unroll
                    for (int gq = 0; gq < QG; ++gq) {
                        const int q = q0 + gq, c = warp + q * NW;
                        if (q < QMAX && c < nd && (c != ndc_ || op.wvec)) {
                            const VT *cp = reinterpret_cast<const VT *>(
                                (c == ndc_) ? op.wvec + base : dot_col(op, c) + base);
    #pragma unroll
                            for (int i = 0; i < NVL; ++i) cv[gq][i] = cp[lane + 32 * i];
                        }
                    }
    #pragma unroll
                    for (int gq = 0; gq < QG; ++gq) {
                        const int q = q0 + gq, c = warp + q * NW;
                        if (q < QMAX && c < nd) {
                            T a = 0;
                            if (c == ndc_) {                 // ||w||^2 or ||wvec .* w||^2
    #pragma unroll
                                for (int i = 0; i < NVL; ++i)
    #pragma unroll
                                    for (int t = 0; t < VW; ++t) {
                                        T v = vcomp<VT, T>(wl[i], t);
                                        if (op.wvec) v *= vcomp<VT, T>(cv[gq][i], t);
                                        a += v * v;
                                    }
                            } else {
    #pragma unroll
                                for (int i = 0; i < NVL; ++i)
    #pragma unroll
                                    for (int t = 0; t < VW; ++t)
                                        a += vcomp<VT, T>(cv[gq][i], t) * vcomp<VT, T>(wl[i], t);
                            }
                            acc[q] += (double)a;
                        }
                    }
                }
            } else {
    #pragma unroll
                for (int q = 0; q < QMAX; ++q) {
                    const int c = warp + q * NW;
                    if (c < nd) {
                        T a = 0;
                        if (c == ndc_ && op.wvec) {
                            for (int i = lane; i < nrow; i += 32) {
                                const T v = ws[i] * op.wvec[base + i];
                                a += v * v;
                            }
                        } else {
                            const T *cp = (c == ndc_) ? ws : dot_col(op, c) + base;
                            for (int i = lane; i < nrow; i += 32) a += cp[i] * ws[i];
                        }
                        acc[q] += (double)a;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (nd == 0 && op.fin == FIN_NONE) {
        if (PDL) asm volatile("griddepcontrol.launch_dependents;");
        return PASS_SKIPPED;
    }
    // per-block partials
    {
        double *pp = op.partials + bid;
        const int64_t nbk = op.nblocks;
        warp_sums_store<QMAX>(acc, nd, [&](int c, double t) { pp[(int64_t)c * nbk] = t; });
    }

    // the next pass may start launching; it waits for this grid to complete
    if (PDL) asm volatile("griddepcontrol.launch_dependents;");
    // ---- two-level reduction, deterministic (fixed lane order and trees):
    // the last block of each group of RGM_RGROUP blocks adds the group's
    // partials (one warp per column, one lane per block); the last group adds
    // the group sums and runs the scalar step.  No block waits for another.
    __shared__ double dsum[RGM_MAXDOTS];
    FinScratch &fin = *reinterpret_cast<FinScratch *>(pool);   // the main phase's arrays are dead
    const int g = bid / RGM_RGROUP, gb0 = g * RGM_RGROUP;
    const int gn = min(RGM_RGROUP, op.nblocks - gb0);
    if (!last_of(op.gcount + g, (unsigned)gn)) return PASS_ARRIVED;
    const bool single = (op.ngroups == 1);
    // the partials' loads go out before the staging loads (whose shared-memory
    // stores wait for their data), so the two round trips overlap; the widest
    // variant keeps the other order (its sums would stay live across the
    // staging and spill)
    constexpr bool early = QMAX <= 8;
    if (!early && single) fin_stage(op, fin);
    // one predicated load per column (gn <= 32): all QMAX loads are in
    // flight together (a loop per column would serialise their round trips)
    static_assert(RGM_RGROUP <= 32, "one lane per block of a group");
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
        const int c = warp + q * NW;
        acc[q] = (c < nd && lane < gn) ? __ldcg(op.partials + (int64_t)c * op.nblocks + gb0 + lane) : 0.0;
    }
    if (early && single) fin_stage(op, fin);
    if (single) {
        warp_sums_store<QMAX>(acc, nd, [&](int c, double t) { dsum[c] = t; });
    } else {
        double *gp = op.gpart + g;
        const int64_t ng = op.ngroups;
        warp_sums_store<QMAX>(acc, nd, [&](int c, double t) { gp[(int64_t)c * ng] = t; });
    }
    if (threadIdx.x == 0) op.gcount[g] = 0u;
    if (!single) {
        if (!last_of(op.counter, (unsigned)op.ngroups)) return PASS_ARRIVED;
        if (!early) fin_stage(op, fin);
        // as above: one predicated load per column for the first 32 groups
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            const int c = warp + q * NW;
            acc[q] = (c < nd && lane < op.ngroups) ? __ldcg(op.gpart + (int64_t)c * op.ngroups + lane) : 0.0;
        }
        if (op.ngroups > 32) {
#pragma unroll
            for (int q = 0; q < QMAX; ++q) {
                const int c = warp + q * NW;
                if (c < nd)
                    for (int gg = lane + 32; gg < op.ngroups; gg += 32)
                        acc[q] += __ldcg(op.gpart + (int64_t)c * op.ngroups + gg);
            }
        }
        if (early) fin_stage(op, fin);
        warp_sums_store<QMAX>(acc, nd, [&](int c, double t) { dsum[c] = t; });
    }
    __syncthreads();
    finalize_block(op, dsum, fin);
    if (threadIdx.x == 0 && !single) *op.counter = 0u;
    return (op.release_gen && op.fin == FIN_ARN2H) ? PASS_RELEASED : PASS_LAST;
}

template <typename T, int QMAX>
__global__ void __launch_bounds__(RGM_THREADS, RGM_MINB) vec_kernel(VecOp<T> op)
{
    // programmatic dependent launch: blocks may be scheduled while the previous
    // pass finishes; nothing it wrote is read before this wait returns
    asm volatile("griddepcontrol.wait;" ::: "memory");
    vec_pass<T, QMAX, true>(op, blockIdx.x);
}

// ---------------------------------------------------------------- persistent cycle
// All Arnoldi steps of one GMRES cycle in one cooperative launch.  The three
// fused passes of a step run back to back in every block, separated by a grid
// barrier that the block finishing a pass last -- the one that reduced the
// partials and ran the scalar step -- releases.  Every block reads the cycle
// state after a barrier, so all of them leave the loop at the same step, and
// the arithmetic is that of the per-pass launches (same code, same reduction
// order).  Waits are bounded: a block that waits longer than RGM_GRID_WAIT_NS
// (or sees Small::fault set) sets Small::fault and returns, the others follow
// at their next wait, and the host reports RGM_E_TIMEOUT.
#define RGM_GRID_WAIT_NS 1000000000ull

template <typename T>
struct CycleOp {
    VecOp<T> pass[3];    // A v_j + dots (first CGS pass), second CGS pass with the norm and
                         // the Givens step, the plain update that stores v_{j+1}
    int m;               // Arnoldi steps at most
    unsigned *arrive;    // arrival counter of the plain barrier
    int cap2;            // host side: co-resident blocks of the two-blocks-per-SM build
};

// After a pass: the last block publishes generation `target`, the others wait
// for it, at most limit_ns.  False when the wait gave up.
__device__ __forceinline__ bool grid_barrier(int pass_rc, Small *s, unsigned target,
                                             unsigned long long limit_ns = RGM_GRID_WAIT_NS)
{
    __shared__ int ok;
    if (pass_rc == PASS_LAST) {
        __syncthreads();                  // the scalar step is complete
        if (threadIdx.x == 0) st_release_gpu(&s->gen, target);
        return true;
    }
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned long long t0 = globaltimer_ns();
        // a second bound that holds even if the timer stalled: one poll is an
        // L2 round trip (hundreds of ns), so this cap is far above limit_ns
        const unsigned long long cap = limit_ns / 16ull + 1024ull;
        for (unsigned long long it = 1; ld_acquire_gpu(&s->gen) < target; ++it) {
            if ((it & 63ull) == 0 && (ld_acquire_gpu(&s->fault) != 0u || it > cap ||
                                      globaltimer_ns() - t0 > limit_ns)) {
                atomicExch(&s->fault, 1u);
                good = 0;
                break;
            }
            if (it > 256) __nanosleep(64);     // spin first: the release is usually close
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Barrier after a pass with no reduction: the last of the n blocks to arrive
// clears the counter and publishes generation `target`; the others wait.
__device__ __forceinline__ bool grid_barrier_arrive(Small *s, unsigned *counter, unsigned n, unsigned target)
{
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        last = (atom_add_acq_rel_gpu(counter, 1u) == n - 1u) ? 1 : 0;
        if (last) {
            *counter = 0u;
            st_release_gpu(&s->gen, target);
        }
    }
    __syncthreads();
    if (last) return true;
    return grid_barrier(PASS_ARRIVED, s, target);
}

// The Arnoldi steps of one cycle as run by block `bid` of the cycle's
// c.pass[0].nblocks blocks.
template <typename T, int QMAX>
__device__ __forceinline__ void cycle_body(const CycleOp<T> &c, const int bid)
{
    Small *s = c.pass[0].sm;
    unsigned gen = 0;
    for (int j = 0; j < c.m; ++j) {
        if (*(volatile int *)&s->done) break;       // same value in every block
        VecOp<T> op = c.pass[0];
        op.x = op.V + (int64_t)j * op.ldv;
        op.xscale = j;
        if (!grid_barrier(vec_pass<T, QMAX, false>(op, bid), s, ++gen)) return;
        VecOp<T> op1 = c.pass[1];
        op1.release_gen = gen + 1;
        const int rc1 = vec_pass<T, QMAX, false>(op1, bid);
        ++gen;
        // the finalising block released the others in mid scalar step
        if (rc1 != PASS_RELEASED && !grid_barrier(rc1, s, gen)) return;
        // plain update storing v_{j+1} (also after the last step: the augmented
        // relation orthogonalises against it)
        vec_pass<T, QMAX, false>(c.pass[2], bid);
        if (!grid_barrier_arrive(s, c.arrive, (unsigned)c.pass[2].nblocks, ++gen)) return;
    }
}

// Built twice: for RGM_MINB resident blocks per SM (the grids never hold
// more), and for two, with twice the registers a thread, which a grid of at
// most two blocks per SM takes (small systems, where every pass is short and
// latency-bound: no spills in the scalar steps).
template <typename T, int QMAX, int MINB>
__global__ void __launch_bounds__(RGM_THREADS, MINB) cycle_kernel(CycleOp<T> c)
{
    cycle_body<T, QMAX>(c, blockIdx.x);
}

// Batched cycles: the GMRES cycles of nsys independent systems in one
// cooperative launch.  Blocks first[i] .. first[i+1]-1 run system i's cycle as
// its blocks 0 .. first[i+1]-first[i]-1 (ops[i] carries that block count).  A
// system's blocks meet only at that system's own barriers (its counters and
// generation in its own Small), so each system ends its cycle at its own step
// and the others carry on; co-residency of the whole grid (the cooperative
// launch) keeps every barrier's blocks resident together.
template <typename T, int QMAX>
__global__ void __launch_bounds__(RGM_THREADS, RGM_MINB)
    batch_cycle_kernel(const CycleOp<T> *__restrict__ ops, const int *__restrict__ first, int nsys)
{
    int lo = 0, hi = nsys - 1;                  // the last i with first[i] <= blockIdx.x
    const int b = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    cycle_body<T, QMAX>(ops[lo], b - first[lo]);
}

// Self-test of the bounded wait: no block ever finishes a pass last, so the
// generation these blocks wait for is never published; each block records in
// *gave_up whether its wait ended by the limit (or by another block's fault).
static __global__ void wait_selftest_kernel(Small *s, unsigned long long limit_ns, int *gave_up)
{
    const bool ok = grid_barrier(PASS_ARRIVED, s, 1u, limit_ns);
    if (threadIdx.x == 0 && !ok) atomicAdd(gave_up, 1);
}

// Host-side dispatch (vec_dispatch.cu): the per-warp column tier is
// chosen from the largest dot-column count the launch can see (nd_max;
// dynamic counts resolve on the device and never exceed it).  Each
// (precision, tier) pair is compiled in a translation unit of its own
// (vec_<precision>_q<tier>.cu, RGM_VEC_DEFINE) so that the build runs in
// parallel; RGM_VEC_DECLARE names what they define.
// Return the cudaError_t of the launch (0 = success).
int launch_vec(const VecOp<double> &op, int nd_max, cudaStream_t st);
int launch_vec(const VecOp<float> &op, int nd_max, cudaStream_t st);
// cycle_kernel: blocks that can be resident at once for this column bound
// (0 if the device cannot launch it cooperatively) in the build for minb
// (RGM_MINB or 2) blocks per SM, and the launch itself.
int cycle_capacity(const CycleOp<double> &c, int nd_max, int minb);
int cycle_capacity(const CycleOp<float> &c, int nd_max, int minb);
int launch_cycle(const CycleOp<double> &c, int nd_max, cudaStream_t st);
int launch_cycle(const CycleOp<float> &c, int nd_max, cudaStream_t st);
// batch_cycle_kernel: blocks that can be resident at once (0 if not
// cooperatively launchable), and the launch of nblocks blocks over nsys
// systems (ops and first in device memory, first[nsys] == nblocks).
int batch_cycle_capacity(const CycleOp<double> *, int nd_max);
int batch_cycle_capacity(const CycleOp<float> *, int nd_max);
int launch_batch_cycle(const CycleOp<double> *ops, const int *first, int nsys, int nblocks, int nd_max,
                       cudaStream_t st);
int launch_batch_cycle(const CycleOp<float> *ops, const int *first, int nsys, int nblocks, int nd_max,
                       cudaStream_t st);

template <typename T, int Q>
static cudaError_t launch_vec_pdl(const VecOp<T> &op, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(op.nblocks);
    cfg.blockDim = dim3(RGM_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, vec_kernel<T, Q>, op);
}

template <typename T, int Q, int MINB>
static int cycle_capacity_q(int dev)
{
    int coop = 0, nsm = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cycle_kernel<T, Q, MINB>, RGM_THREADS, 0) !=
        cudaSuccess)
        return 0;
    return per_sm * nsm;
}

template <typename T, int Q>
static cudaError_t launch_cycle_q(const CycleOp<T> &c, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.pass[0].nblocks);
    cfg.blockDim = dim3(RGM_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all blocks resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the wider-register build when its residency holds the whole grid
    // (c.cap2: the caller's cached capacity of that build on its device)
    return (c.pass[0].nblocks <= c.cap2) ? cudaLaunchKernelEx(&cfg, cycle_kernel<T, Q, 2>, c)
                                         : cudaLaunchKernelEx(&cfg, cycle_kernel<T, Q, RGM_MINB>, c);
}

template <typename T, int Q>
static int batch_capacity_q(int dev)
{
    int coop = 0, nsm = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_cycle_kernel<T, Q>, RGM_THREADS, 0) !=
        cudaSuccess)
        return 0;
    return per_sm * nsm;
}

template <typename T, int Q>
static cudaError_t launch_batch_q(const CycleOp<T> *ops, const int *first, int nsys, int nblocks,
                                  cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(RGM_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all blocks resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_cycle_kernel<T, Q>, ops, first, nsys);
}

#define RGM_QBIG ((RGM_MAXDOTS + RGM_THREADS / 32 - 1) / (RGM_THREADS / 32))

// Entry points of one (precision, column tier) translation unit.
#define RGM_VEC_DECLARE(TN, T, QN)                                                                 \
    int vec_launch_##TN##_##QN(const VecOp<T> &op, cudaStream_t st);                               \
    int vec_cycle_capacity_##TN##_##QN(int dev, int minb);                                         \
    int vec_cycle_launch_##TN##_##QN(const CycleOp<T> &c, cudaStream_t st);                        \
    int vec_batch_capacity_##TN##_##QN(int dev);                                                   \
    int vec_batch_launch_##TN##_##QN(const CycleOp<T> *ops, const int *first, int nsys, int nblocks, \
                                     cudaStream_t st);
#define RGM_VEC_DEFINE_VEC(TN, T, QN, Q)                                                           \
    int vec_launch_##TN##_##QN(const VecOp<T> &op, cudaStream_t st)                                \
    {                                                                                              \
        return (int)launch_vec_pdl<T, Q>(op, st);                                                  \
    }
#define RGM_VEC_DEFINE_CYCLE(TN, T, QN, Q)                                                         \
    int vec_cycle_capacity_##TN##_##QN(int dev, int minb)                                          \
    {                                                                                              \
        return minb == 2 ? cycle_capacity_q<T, Q, 2>(dev) : cycle_capacity_q<T, Q, RGM_MINB>(dev); \
    }                                                                                              \
    int vec_cycle_launch_##TN##_##QN(const CycleOp<T> &c, cudaStream_t st)                         \
    {                                                                                              \
        return (int)launch_cycle_q<T, Q>(c, st);                                                   \
    }
#define RGM_VEC_DEFINE_BATCH(TN, T, QN, Q)                                                         \
    int vec_batch_capacity_##TN##_##QN(int dev) { return batch_capacity_q<T, Q>(dev); }            \
    int vec_batch_launch_##TN##_##QN(const CycleOp<T> *ops, const int *first, int nsys, int nblocks, \
                                     cudaStream_t st)                                              \
    {                                                                                              \
        return (int)launch_batch_q<T, Q>(ops, first, nsys, nblocks, st);                           \
    }
#define RGM_VEC_DEFINE(TN, T, QN, Q)                                                               \
    RGM_VEC_DEFINE_VEC(TN, T, QN, Q)                                                               \
    RGM_VEC_DEFINE_CYCLE(TN, T, QN, Q)                                                             \
    RGM_VEC_DEFINE_BATCH(TN, T, QN, Q)
RGM_VEC_DECLARE(f64, double, q4)
RGM_VEC_DECLARE(f64, double, q8)
RGM_VEC_DECLARE(f64, double, qbig)
RGM_VEC_DECLARE(f32, float, q4)
RGM_VEC_DECLARE(f32, float, q8)
RGM_VEC_DECLARE(f32, float, qbig)

// CSR values -> sliced-ELL positions (binary64 and, when given, binary32 copy).
template <typename Tin>
__global__ void sell_scatter_kernel(double *sval, float *sval32, const Tin *val, const int32_t *map,
                                    int64_t nnz)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)val[e];
        const int32_t d = map[e];
        sval[d] = v;
        if (sval32) sval32[d] = (float)v;
    }
}

// CSR values -> sliced-ELL positions, one block per 256-row tile: the tile's
// CSR values (contiguous, rows r0 .. r0 + 255) are read into shared memory
// with coalesced loads, then every sliced-ELL position of the tile (contiguous
// too) is written in order from src[e], its CSR offset inside the tile (-1:
// padding, value 0).  Both global streams are coalesced, unlike the scatter
// above, whose writes land 32 positions apart.  Dynamic shared memory: the
// largest tile's CSR entries in binary64 (up to RGM_GATHER_SMEM_MAX, so few
// blocks fit an SM: each block is RGM_GATHER_THREADS wide to keep loads in
// flight).
#define RGM_GATHER_THREADS 1024
template <typename Tin>
__global__ void __launch_bounds__(RGM_GATHER_THREADS) sell_gather_kernel(double *__restrict__ sval, float *__restrict__ sval32,
                                                          const Tin *__restrict__ val,
                                                          const int64_t *__restrict__ tile_csr,
                                                          const int64_t *__restrict__ slice_ptr,
                                                          const int32_t *__restrict__ src)
{
    extern __shared__ double tv[];
    const int64_t t = blockIdx.x;
    const int64_t c0 = tile_csr[t], c1 = tile_csr[t + 1];
    for (int64_t i = threadIdx.x; i < c1 - c0; i += blockDim.x) tv[i] = (double)val[c0 + i];
    __syncthreads();
    const int64_t s0 = slice_ptr[t * (RGM_TILE / 32)], s1 = slice_ptr[(t + 1) * (RGM_TILE / 32)];
    for (int64_t e = s0 + threadIdx.x; e < s1; e += blockDim.x) {
        const int32_t k = src[e];
        const double v = (k >= 0) ? tv[k] : 0.0;
        sval[e] = v;
        if (sval32) sval32[e] = (float)v;
    }
}

// ---------------------------------------------------------------- Gram matrices
// Pairwise dot products of columns: out[p] = col(a_p) . col(b_p) for a list of
// pairs over the combined column list [X | Y]; binary64 accumulation.  Each
// block stages a tile of rows of all ncol columns in shared memory (padded
// stride, conflict-free), and each thread owns pairs p = tid + k * blockDim.
enum GramMode {
    GRAM_PACKED = 0,   // all pairs i <= j of the nx columns of X (packed, j-major)
    GRAM_UW = 1,       // E pattern: u_i . w_j (i + j nx), then u_i . u_i, then w_i . w_i
    GRAM_COL = 2       // one column against all: x_col . x_j, j < nx
};

template <typename T>
struct GramOp {
    int64_t n;
    int rpb, nblocks;
    const T *X; int64_t ldx; int nx;
    const T *Y; int64_t ldy;
    const int *nx_dev;       // if set, nx is read from the device (dynamic column count)
    int mode;
    int nxmax;               // bound on nx (shared-memory sizing)
    int col;                 // GRAM_COL: the column dotted with all others
    double *partials;        // per-block sums, pair p at p * nblocks
    unsigned *counter;       // completion counter of the groups
    unsigned *gcount;        // per-group completion counters (RGM_RGROUP blocks a group)
    double *gpart;           // per-group sums, pair p at p * ngroups
    int ngroups;
    double *out;
    int tile;                // rows per tile (tile+1 values per column in smem)
};

#define RGM_GRAM_PMAX 16      // pairs per thread: npairs <= RGM_GRAM_PMAX * RGM_THREADS

__device__ __forceinline__ void packed_pair(int p, int *i, int *j)
{
    int jj = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((jj + 1) * (jj + 2) / 2 <= p) ++jj;
    while (jj * (jj + 1) / 2 > p) --jj;
    *j = jj;
    *i = p - jj * (jj + 1) / 2;
}

// sum over r = r0, r0 + step, .. < nrow of a[r] b[r], accumulated in binary64.
// binary32 columns: products and sums of 8 consecutive terms in binary32 (its
// FMA pipe is 64 times wider than the binary64 one on this part), each block
// sum then added in binary64.
__device__ __forceinline__ double pair_dot(const double *a, const double *b, int r0, int nrow, int step,
                                           double acc)
{
    for (int r = r0; r < nrow; r += step) acc = fma(a[r], b[r], acc);
    return acc;
}
__device__ __forceinline__ double pair_dot(const float *a, const float *b, int r0, int nrow, int step,
                                           double acc)
{
    int r = r0;
    for (; r + 7 * step < nrow; r += 8 * step) {
        float f = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) f = fmaf(a[r + t * step], b[r + t * step], f);
        acc += (double)f;
    }
    for (; r < nrow; r += step) acc += (double)(a[r] * b[r]);
    return acc;
}

// PPT: pairs a thread owns at most (1 when npairs <= RGM_THREADS: the per-step
// Gram matrices -- the window's new column, CholQR, E -- which then run with
// few registers and more blocks per SM; RGM_GRAM_PMAX for a full window Gram).
template <typename T, int PPT>
__global__ void __launch_bounds__(RGM_THREADS) gram_kernel(GramOp<T> op)
{
    extern __shared__ __align__(16) unsigned char gsm_raw[];
    T *gsm = reinterpret_cast<T *>(gsm_raw);
    const int nx = op.nx_dev ? *op.nx_dev : op.nx;
    const int ny = (op.mode == GRAM_UW) ? nx : 0;
    const int ncol = nx + ny, ts = op.tile + 1;
    const int npairs = (op.mode == GRAM_UW) ? nx * nx + 2 * nx : (op.mode == GRAM_COL) ? nx : nx * (nx + 1) / 2;
    const int64_t r0 = (int64_t)blockIdx.x * op.rpb;
    const int64_t r1 = min(op.n, r0 + op.rpb);
    auto pair_of = [&](int p, int *a, int *b) {
        *a = 0;
        *b = 0;
        if (p >= npairs) return;
        if (op.mode == GRAM_PACKED) {
            packed_pair(p, a, b);
        } else if (op.mode == GRAM_COL) {
            *a = op.col;
            *b = p;
        } else if (p < nx * nx) {
            *a = p % nx;
            *b = nx + p / nx;
        } else if (p < nx * nx + nx) {
            *a = *b = p - nx * nx;
        } else {
            *a = *b = nx + (p - nx * nx - nx);
        }
    };
    static_assert(PPT >= 1 && PPT <= RGM_GRAM_PMAX, "pairs a thread");
    double acc[PPT];
    int pa[PPT], pb[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        acc[i] = 0.0;
        pair_of(threadIdx.x + i * RGM_THREADS, &pa[i], &pb[i]);
    }
    // few pairs (the window's new column, CholQR, E): the block's threads split
    // each pair's rows into nsl interleaved slices instead of one thread walking
    // all rows of a pair; the slices' sums are added once at the end
    const bool split = npairs > 0 && 2 * npairs <= RGM_THREADS;
    const int nsl = split ? RGM_THREADS / npairs : 1;
    const int sp = split ? (int)threadIdx.x % npairs : 0, srs = split ? (int)threadIdx.x / npairs : 0;
    int spa = 0, spb = 0;
    if (split) pair_of(sp, &spa, &spb);
    double sacc = 0.0;
    for (int64_t base = r0; base < r1; base += op.tile) {
        const int nrow = (int)min((int64_t)op.tile, r1 - base);
        // column by column, one row a thread (tile <= RGM_THREADS): ncol
        // independent coalesced loads in flight per thread
        for (int c = 0; c < ncol; ++c) {
            const T *src = c < nx ? op.X + (int64_t)c * op.ldx : op.Y + (int64_t)(c - nx) * op.ldy;
            for (int r = threadIdx.x; r < nrow; r += RGM_THREADS) gsm[c * ts + r] = src[base + r];
        }
        __syncthreads();
        if (split) {
            if (srs < nsl) sacc = pair_dot(gsm + spa * ts, gsm + spb * ts, srs, nrow, nsl, sacc);
        } else {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                if (threadIdx.x + i * RGM_THREADS < npairs)
                    acc[i] += pair_dot(gsm + pa[i] * ts, gsm + pb[i] * ts, 0, nrow, 1, 0.0);
            }
        }
        __syncthreads();
    }
    if (split) {
        // the launch gives the buffer at least RGM_THREADS doubles
        double *dsm = reinterpret_cast<double *>(gsm_raw);
        dsm[threadIdx.x] = (srs < nsl) ? sacc : 0.0;
        __syncthreads();
        if ((int)threadIdx.x < npairs) {
            double v = 0.0;
            for (int q = 0; q < nsl; ++q) v += dsm[threadIdx.x + q * npairs];
            acc[0] = v;
        }
    }
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int p = threadIdx.x + i * RGM_THREADS;
        if (p < npairs) op.partials[(int64_t)p * op.nblocks + blockIdx.x] = acc[i];
    }
    // two-level reduction, deterministic (fixed order): the last block of each
    // group of RGM_RGROUP blocks adds the group's partials of every pair (one
    // thread per pair, the group's loads in flight together), the last group
    // adds the group sums.  No block waits for another.
    const int g = blockIdx.x / RGM_RGROUP, gb0 = g * RGM_RGROUP;
    const int gn = min(RGM_RGROUP, op.nblocks - gb0);
    if (!last_of(op.gcount + g, (unsigned)gn)) return;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const double *pp = op.partials + (int64_t)p * op.nblocks + gb0;
        double sum = 0.0;
        // eight loads in flight at a time, added in block order
#pragma unroll
        for (int b0 = 0; b0 < RGM_RGROUP; b0 += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (b0 + u < gn) ? __ldcg(pp + b0 + u) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += v[u];
        }
        op.gpart[(int64_t)p * op.ngroups + g] = sum;
    }
    if (threadIdx.x == 0) op.gcount[g] = 0u;
    if (!last_of(op.counter, (unsigned)op.ngroups)) return;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const double *gp = op.gpart + (int64_t)p * op.ngroups;
        double sum = 0.0;
        int gg = 0;
        for (; gg + 8 <= op.ngroups; gg += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(gp + gg + u);
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += v[u];
        }
        for (; gg < op.ngroups; ++gg) sum += __ldcg(gp + gg);
        op.out[p] = sum;
    }
    if (threadIdx.x == 0) *op.counter = 0u;
}

// ---------------------------------------------------------------- cycle-end kernels
// Back substitution R y = g on the rotated (J+naug)^2 block (staged in shared
// memory), then the update coefficients of x += Vraw[:, :J] (y * colscale)
// + U[:, aug] y_aug.
#define RGM_LS_MAX (RGM_NCOL * (RGM_NCOL + 1) / 2)
static __global__ void ls_solve_kernel(Small *s)
{
    __shared__ double R[RGM_LS_MAX];     // packed upper triangle, column j at j(j+1)/2
    __shared__ double g[RGM_HLD], rdg[RGM_HLD], yv[RGM_HLD];
    const int nc = s->J + s->naug;
    for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
        const int i = t % nc, j = t / nc;
        if (i <= j) R[j * (j + 1) / 2 + i] = s->H[i + (int64_t)j * RGM_HLD];
    }
    for (int i = threadIdx.x; i < nc; i += blockDim.x) g[i] = s->g[i];
    __syncthreads();
    // the diagonal's reciprocals at once, then the back substitution in one
    // warp (no block barrier and no division on the serial path)
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const double d = R[i * (i + 1) / 2 + i];
        rdg[i] = (d != 0.0) ? 1.0 / d : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int i = nc - 1; i >= 0; --i) {
            const double y = g[i] * rdg[i];
            __syncwarp();
            if (lane == 0) yv[i] = y;
            for (int t = lane; t < i; t += 32) g[t] = fma(-R[i * (i + 1) / 2 + t], y, g[t]);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) s->y[i] = yv[i];
    for (int i = threadIdx.x; i < RGM_HLD; i += blockDim.x)
        s->coefV[i] = (i < s->J) ? yv[i] * s->colscale[i] : 0.0;
    for (int i = threadIdx.x; i < RGM_KMAX; i += blockDim.x) s->coefU[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int a = 0; a < s->naug; ++a) s->coefU[s->aug_idx[a]] += yv[s->J + a];
}

// Reset the per-cycle Hessenberg state (before the start vector kernels).
static __global__ void cycle_reset_kernel(Small *s)
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
        s->gen = 0u;          // grid-barrier generations restart with each cycle
    }
}

// LU with partial pivoting of a k x k matrix in one block (singular when a
// pivot < 1e-13 * max(largest pivot, scale)).  which = 0: E = U^T W from the
// GRAM_UW output (k x k column-major, then the squared column norms of U and
// W; scale max ||u_i|| ||w_i||) into E, LU, LUrd, piv, LUperm.  which = 1: the
// Gram matrix G = Y^T Y of the orthogonal / least-squares projector from a
// packed pair list (scale max G_ii) into LUP, LUPrd, pivP, LUPperm.  Either
// one singular sets Small::singular and k = 0 (the solve runs without
// recycling).
static __global__ void lu_kernel(Small *s, int k, const double *in, const double *colnorm2, int which)
{
    __shared__ double M[RGM_KMAX * RGM_KMAX];
    __shared__ int pivrow;
    __shared__ double pivrcp;
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
        const int r = i % k, c = i / k;
        double v;
        if (which == 0) {
            v = in[i];
            s->E[r + c * RGM_KMAX] = v;
        } else {
            v = in[r <= c ? c * (c + 1) / 2 + r : r * (r + 1) / 2 + c];
        }
        M[r + c * RGM_KMAX] = v;
    }
    __syncthreads();
    double scale = 0.0;
    if (which == 0)
        for (int i = 0; i < k; ++i) scale = fmax(scale, sqrt(colnorm2[i] * colnorm2[k + i]));
    else
        for (int i = 0; i < k; ++i) scale = fmax(scale, M[i + i * RGM_KMAX]);
    double *LUo = which ? s->LUP : s->LU, *rdo = which ? s->LUPrd : s->LUrd;
    int *pvo = which ? s->pivP : s->piv, *pmo = which ? s->LUPperm : s->LUperm;
    double maxp = scale, minp = INFINITY;
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            int p = j;
            for (int i = j + 1; i < k; ++i)
                if (fabs(M[i + j * RGM_KMAX]) > fabs(M[p + j * RGM_KMAX])) p = i;
            pivrow = p;
            pvo[j] = p;
            const double dp = M[p + j * RGM_KMAX];
            pivrcp = (dp != 0.0) ? 1.0 / dp : 0.0;   // multipliers by one reciprocal
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
            const double rd = pivrcp;
            for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) M[i + j * RGM_KMAX] *= rd;
            __syncthreads();
            for (int t = threadIdx.x; t < (k - j - 1) * (k - j - 1); t += blockDim.x) {
                int i = j + 1 + t % (k - j - 1), c = j + 1 + t / (k - j - 1);
                M[i + c * RGM_KMAX] -= M[i + j * RGM_KMAX] * M[j + c * RGM_KMAX];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < RGM_KMAX * RGM_KMAX; i += blockDim.x) LUo[i] = M[i];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double d = M[i + i * RGM_KMAX];
        rdo[i] = (d != 0.0) ? 1.0 / d : 0.0;
    }
    if (threadIdx.x == 0) {
        // the row swaps as one permutation: (P b)_i = b[perm_i]
        int pm[RGM_KMAX];
        for (int i = 0; i < k; ++i) pm[i] = i;
        for (int j = 0; j < k; ++j) {
            const int p = pvo[j];
            const int t = pm[j]; pm[j] = pm[p]; pm[p] = t;
        }
        for (int i = 0; i < k; ++i) pmo[i] = pm[i];
        const int sing = (k > 0 && (minp == 0.0 || minp < 1e-13 * maxp)) ? 1 : 0;
        if (which == 0) {
            s->singular = sing;
            s->k = sing ? 0 : k;
        } else if (sing) {
            s->singular = 1;
            s->k = 0;
        }
    }
}
