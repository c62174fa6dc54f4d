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

enum Src { SRC_SPMV = 0, SRC_RES = 1, SRC_COPY = 2, SRC_AXPY = 3, SRC_NONE = 4 };
enum Gate { GATE_NONE = 0, GATE_KRYLOV = 1, GATE_APPEND = 2 };
enum Fin {
    FIN_NONE = 0,
    FIN_BNORM,       // ||b||
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
    double *partials;
    unsigned *counter;
    Small *sm;
    int fin;
    int gate;
    int arg;                 // phase argument (appended column index)
    int dyn;                 // DYN_* bits: counts and output column read from Small
};

enum Dyn {
    DYN_NDV_NB = 1,   // ndV = s->nb
    DYN_NV_NB = 2,    // nV  = s->nb
    DYN_NV_J = 4,     // nV  = s->J
    DYN_OUT_VNB = 8   // out = Vraw[:, s->nb]
};

// Shared scratch of the finalising block.
struct FinScratch {
    double LU[RGM_KMAX * RGM_KMAX];
    int piv[RGM_KMAX];
    double dd[RGM_KMAX];
    double col[RGM_HLD + 1];
    double cs[RGM_HLD], sn[RGM_HLD];
    double sc[RGM_HLD];
    int flag;
};

// ---------------------------------------------------------------- scalar helpers
__device__ inline void lu_solve_small(int k, const double *LU, int ld, const int *piv, double *x)
{
    for (int j = 0; j < k; ++j)
        if (piv[j] != j) { double t = x[j]; x[j] = x[piv[j]]; x[piv[j]] = t; }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) x[i] -= LU[i + j * ld] * x[j];
    for (int i = k - 1; i >= 0; --i) {
        for (int j = i + 1; j < k; ++j) x[i] -= LU[i + j * ld] * x[j];
        x[i] /= LU[i + i * ld];
    }
}

// Stage the k x k LU factors and pivots of E in shared memory (whole block).
__device__ inline void stage_lu(const Small *s, int k, FinScratch &f)
{
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        int i = t % k, j = t / k;
        f.LU[i + j * RGM_KMAX] = s->LU[i + j * RGM_KMAX];
    }
    for (int t = threadIdx.x; t < k; t += blockDim.x) f.piv[t] = s->piv[t];
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
    case FIN_RESNORM:
        if (tid == 0) {
            s->beta = sqrt(nrm2);
            s->converged = (s->beta <= s->tol_abs) ? 1 : 0;
        }
        break;
    case FIN_COARSE:
    case FIN_START_DEF1: {
        const int k = op.ndU;
        stage_lu(s, k, f);
        __syncthreads();
        if (tid == 0) {
            for (int i = 0; i < k; ++i) f.dd[i] = dU[i];
            lu_solve_small(k, f.LU, RGM_KMAX, f.piv, f.dd);
        }
        __syncthreads();
        for (int i = tid; i < k; i += blockDim.x) {
            if (op.fin == FIN_COARSE) s->coefU[i] = f.dd[i];
            else s->coefW[i] = -f.dd[i];
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
        const int nb = s->nb, k = op.ndU;
        if (k) stage_lu(s, k, f);
        for (int i = tid; i < nb; i += blockDim.x) f.sc[i] = s->colscale[i];
        __syncthreads();
        if (tid == 0) {
            s->wn0 = sqrt(nrm2);
            if (op.fin == FIN_AUG1) s->skip = (nrm2 == 0.0) ? 1 : 0;
            for (int i = 0; i < k; ++i) f.dd[i] = dU[i];
            if (k) lu_solve_small(k, f.LU, RGM_KMAX, f.piv, f.dd);
        }
        __syncthreads();
        for (int i = tid; i < k; i += blockDim.x) s->coefW[i] = -f.dd[i];
        for (int i = tid; i < nb; i += blockDim.x) {
            double h = dV[i] * f.sc[i];
            for (int l = 0; l < k; ++l) h -= s->VtW[i + l * RGM_HLD] * f.dd[l];
            s->hsum[i] = h;
            s->coefV[i] = -h * f.sc[i];
        }
        break;
    }
    case FIN_ARN2: {
        const int nb = s->nb;
        for (int i = tid; i < nb; i += blockDim.x) {
            const double sc = s->colscale[i];
            const double h = dV[i] * sc;
            s->hsum[i] += h;
            s->coefV[i] = -h * sc;
        }
        break;
    }
    case FIN_ARN3: {
        const int j = s->J, nb = s->nb;
        const double hn = sqrt(nrm2);
        for (int i = tid; i < nb; i += blockDim.x) f.col[i] = s->hsum[i];
        for (int i = tid; i < j; i += blockDim.x) { f.cs[i] = s->cs[i]; f.sn[i] = s->sn[i]; }
        if (tid == 0) f.col[nb] = hn;
        __syncthreads();
        if (tid == 0) apply_rotations(f.col, f.cs, f.sn, j);
        __syncthreads();
        close_column(s, f, j);
        const bool brk = hn <= 1e-14 * s->wn0;
        const double sc = brk ? 0.0 : 1.0 / hn;
        for (int l = tid; l < op.ndW; l += blockDim.x) s->VtW[nb + l * RGM_HLD] = dW[l] * sc;
        if (tid == 0) {
            s->J = j + 1;
            s->iters += 1;
            s->colscale[nb] = sc;          // happy breakdown: v_{j+1} := 0
            if (brk) { s->breakdown = 1; s->done = 1; }
            s->nb = nb + 1;
            if (fabs(s->g[j + 1]) <= s->tol_abs) s->done = 1;
            if (s->iters >= s->maxit || s->J >= s->m) s->done = 1;
        }
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

// What one block did in a pass: left without touching the completion counter
// (gated off, or nothing to reduce), arrived, or arrived last and finalised.
enum PassResult { PASS_SKIPPED = 0, PASS_ARRIVED = 1, PASS_LAST = 2 };

// One fused pass over the block's rows (body of vec_kernel and of each phase
// of cycle_kernel).  PDL: signal programmatic dependents once the partials
// are written.
template <typename T, int QMAX, bool PDL>
__device__ __forceinline__ int vec_pass(VecOp<T> op)
{
    constexpr int NW = RGM_THREADS / 32;      // QMAX * NW >= number of dot columns
    Small *s = op.sm;
    if (op.gate == GATE_KRYLOV && s->done) return PASS_SKIPPED;
    if (op.gate == GATE_APPEND && (s->skip || s->J == 0)) return PASS_SKIPPED;
    if (op.dyn) {
        if (op.dyn & DYN_NDV_NB) op.ndV = s->nb;
        if (op.dyn & DYN_NV_NB) op.nV = s->nb;
        if (op.dyn & DYN_NV_J) op.nV = s->J;
        if (op.dyn & DYN_OUT_VNB) op.out = const_cast<T *>(op.V) + (int64_t)s->nb * op.ldv;
    }

    __shared__ T cW[RGM_KMAX], cU[RGM_KMAX], cV[RGM_HLD];
    __shared__ T ws[RGM_TILE];
    __shared__ double xs;
    if (threadIdx.x == 0) xs = (op.xscale >= 0) ? s->colscale[op.xscale] : 1.0;
    if (op.src == SRC_AXPY) {
        for (int i = threadIdx.x; i < op.nW; i += blockDim.x) cW[i] = (T)s->coefW[i];
        for (int i = threadIdx.x; i < op.nV; i += blockDim.x) cV[i] = (T)s->coefV[i];
        for (int i = threadIdx.x; i < op.nU; i += blockDim.x) cU[i] = (T)s->coefU[i];
    }
    __syncthreads();

    const int nd = op.ndU + op.ndV + op.ndW + op.dnorm;
    const int ndc_ = op.dnorm ? nd - 1 : -1;          // index of the ||w||^2 column
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * op.rpb;
    const int64_t r1 = min(op.n, r0 + op.rpb);
    double acc[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) acc[q] = 0.0;

    const bool spmv_src = (op.src == SRC_SPMV || op.src == SRC_RES);
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
            T a = 0;
#pragma unroll 8
            for (int64_t e = p0 + lane; e < p1; e += 32) a += op.sval[e] * op.x[op.scol[e]];
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
            T a = 0;
#pragma unroll 8
            for (int64_t e = p0 + lane; e < p1; e += 32) a += op.sval[e] * op.x[op.scol[e]];
            const int pr = op.perm[(sl << 5) + lane];
            if (pr >= 0) {
                const T v = (op.src == SRC_SPMV) ? a * sc : op.b[pr] - a;
                op.out[pr] = v;
                ws[pr - base] = v;
            }
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
            // full tile: every load of the warp's columns is issued up front
            T wl[RGM_TILE / 32];
#pragma unroll
            for (int i = 0; i < RGM_TILE / 32; ++i) wl[i] = ws[lane + 32 * i];
#pragma unroll
            for (int q = 0; q < QMAX; ++q) {
                const int c = warp + q * NW;
                if (c < nd) {
                    const T *cp = (c == ndc_) ? ws : dot_col(op, c) + base;
                    T a = 0;
#pragma unroll
                    for (int i = 0; i < RGM_TILE / 32; ++i) a += cp[lane + 32 * i] * wl[i];
                    acc[q] += (double)a;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < QMAX; ++q) {
                const int c = warp + q * NW;
                if (c < nd) {
                    const T *cp = (c == ndc_) ? ws : dot_col(op, c) + base;
                    T a = 0;
                    for (int i = lane; i < nrow; i += 32) a += cp[i] * ws[i];
                    acc[q] += (double)a;
                }
            }
        }
        __syncthreads();
    }
    if (nd == 0 && op.fin == FIN_NONE) {
        if (PDL) asm volatile("griddepcontrol.launch_dependents;");
        return PASS_SKIPPED;
    }
    // per-block partials: one warp reduction per column
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
        const int c = warp + q * NW;
        if (c < nd) {
            const double v = warp_sum(acc[q]);
            if (lane == 0) op.partials[(int64_t)c * op.nblocks + blockIdx.x] = v;
        }
    }

    // the next pass may start launching; it waits for this grid to complete
    if (PDL) asm volatile("griddepcontrol.launch_dependents;");
    // ---- the last block reduces the partials and runs the scalar step
    if (!last_block(op.counter)) return PASS_ARRIVED;
    __shared__ double dsum[RGM_MAXDOTS];
    __shared__ double red2[RGM_THREADS];
    __shared__ FinScratch fin;
    if (nd > 0) {
        // threads split each column's blocks (independent loads); fixed order
        const int tpc = max(1, RGM_THREADS / nd);
        const int ncov = RGM_THREADS / tpc;
        for (int cbase = 0; cbase < nd; cbase += ncov) {
            const int c = cbase + (int)threadIdx.x / tpc, part = (int)threadIdx.x % tpc;
            double v = 0.0;
            if ((int)threadIdx.x < ncov * tpc && c < nd) {
                const double *p = op.partials + (int64_t)c * op.nblocks;
#pragma unroll 8
                for (int b = part; b < op.nblocks; b += tpc) v += __ldcg(p + b);
            }
            red2[threadIdx.x] = v;
            __syncthreads();
            for (int cc = threadIdx.x; cc < ncov && cbase + cc < nd; cc += blockDim.x) {
                double t = 0.0;
                for (int j = 0; j < tpc; ++j) t += red2[cc * tpc + j];
                dsum[cbase + cc] = t;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    finalize_block(op, dsum, fin);
    if (threadIdx.x == 0) *op.counter = 0u;
    return PASS_LAST;
}

template <typename T, int QMAX>
__global__ void __launch_bounds__(RGM_THREADS, 4) vec_kernel(VecOp<T> op)
{
    // programmatic dependent launch: blocks may be scheduled while the previous
    // pass finishes; nothing it wrote is read before this wait returns
    asm volatile("griddepcontrol.wait;" ::: "memory");
    vec_pass<T, QMAX, true>(op);
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
    VecOp<T> pass[3];    // A v_j + dots (first CGS pass), second CGS pass, norm + Givens
    int m;               // Arnoldi steps at most
};

// After a pass: the last block publishes generation `target`, the others wait
// for it, at most limit_ns.  False when the wait gave up.
__device__ __forceinline__ bool grid_barrier(int pass_rc, Small *s, unsigned target,
                                             unsigned long long limit_ns = RGM_GRID_WAIT_NS)
{
    __shared__ int ok;
    if (pass_rc == PASS_LAST) {
        __syncthreads();                  // the scalar step is complete
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(&s->gen, target);
        }
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
            __nanosleep(64);
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

template <typename T, int QMAX>
__global__ void __launch_bounds__(RGM_THREADS, 4) cycle_kernel(CycleOp<T> c)
{
    Small *s = c.pass[0].sm;
    unsigned gen = 0;
    for (int j = 0; j < c.m; ++j) {
        if (*(volatile int *)&s->done) break;       // same value in every block
        VecOp<T> op = c.pass[0];
        op.x = op.V + (int64_t)j * op.ldv;
        op.xscale = j;
        if (!grid_barrier(vec_pass<T, QMAX, false>(op), s, ++gen)) return;
        if (!grid_barrier(vec_pass<T, QMAX, false>(c.pass[1]), s, ++gen)) return;
        if (!grid_barrier(vec_pass<T, QMAX, false>(c.pass[2]), s, ++gen)) return;
    }
}

// Self-test of the bounded wait: no block ever finishes a pass last, so the
// generation these blocks wait for is never published; each block records in
// *gave_up whether its wait ended by the limit (or by another block's fault).
static __global__ void wait_selftest_kernel(Small *s, unsigned long long limit_ns, int *gave_up)
{
    const bool ok = grid_barrier(PASS_ARRIVED, s, 1u, limit_ns);
    if (threadIdx.x == 0 && !ok) atomicAdd(gave_up, 1);
}

// Host-side dispatch (vec_f64.cu / vec_f32.cu): the per-warp column tier is
// chosen from the largest dot-column count the launch can see (nd_max;
// dynamic counts resolve on the device and never exceed it).
// Return the cudaError_t of the launch (0 = success).
int launch_vec(const VecOp<double> &op, int nd_max, cudaStream_t st);
int launch_vec(const VecOp<float> &op, int nd_max, cudaStream_t st);
// cycle_kernel: blocks that can be resident at once for this column bound
// (0 if the device cannot launch it cooperatively), and the launch itself.
int cycle_capacity(const CycleOp<double> &c, int nd_max);
int cycle_capacity(const CycleOp<float> &c, int nd_max);
int launch_cycle(const CycleOp<double> &c, int nd_max, cudaStream_t st);
int launch_cycle(const CycleOp<float> &c, int nd_max, cudaStream_t st);

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

template <typename T>
static int launch_vec_impl(const VecOp<T> &op, int nd_max, cudaStream_t st)
{
    constexpr int NW = RGM_THREADS / 32;
    constexpr int QBIG = (RGM_MAXDOTS + NW - 1) / NW;
    const int q = (nd_max + NW - 1) / NW;
    cudaError_t e;
    if (q <= 4) e = launch_vec_pdl<T, 4>(op, st);
    else if (q <= 8) e = launch_vec_pdl<T, 8>(op, st);
    else e = launch_vec_pdl<T, QBIG>(op, st);
    return (int)e;          // cudaSuccess == 0
}

template <typename T, int Q>
static int cycle_capacity_q(int dev)
{
    int coop = 0, nsm = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cycle_kernel<T, Q>, RGM_THREADS, 0) !=
        cudaSuccess)
        return 0;
    return per_sm * nsm;
}

template <typename T>
static int cycle_capacity_impl(int nd_max)
{
    constexpr int NW = RGM_THREADS / 32;
    constexpr int QBIG = (RGM_MAXDOTS + NW - 1) / NW;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const int q = (nd_max + NW - 1) / NW;
    if (q <= 4) return cycle_capacity_q<T, 4>(dev);
    if (q <= 8) return cycle_capacity_q<T, 8>(dev);
    return cycle_capacity_q<T, QBIG>(dev);
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
    return cudaLaunchKernelEx(&cfg, cycle_kernel<T, Q>, c);
}

template <typename T>
static int launch_cycle_impl(const CycleOp<T> &c, int nd_max, cudaStream_t st)
{
    constexpr int NW = RGM_THREADS / 32;
    constexpr int QBIG = (RGM_MAXDOTS + NW - 1) / NW;
    const int q = (nd_max + NW - 1) / NW;
    cudaError_t e;
    if (q <= 4) e = launch_cycle_q<T, 4>(c, st);
    else if (q <= 8) e = launch_cycle_q<T, 8>(c, st);
    else e = launch_cycle_q<T, QBIG>(c, st);
    return (int)e;          // cudaSuccess == 0
}

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

// ---------------------------------------------------------------- Gram matrices
// Pairwise dot products of columns: out[p] = col(a_p) . col(b_p) for a list of
// pairs over the combined column list [X | Y]; binary64 accumulation.  Each
// block stages a tile of rows of all ncol columns in shared memory (padded
// stride, conflict-free), and each thread owns pairs p = tid + k * blockDim.
enum GramMode {
    GRAM_PACKED = 0,   // all pairs i <= j of the nx columns of X (packed, j-major)
    GRAM_UW = 1        // E pattern: u_i . w_j (i + j nx), then u_i . u_i, then w_i . w_i
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
    double *partials;
    unsigned *counter;
    double *out;
    int tile;                // rows per tile (tile+1 doubles per column in smem)
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

template <typename T>
__global__ void __launch_bounds__(RGM_THREADS) gram_kernel(GramOp<T> op)
{
    extern __shared__ double gsm[];
    const int nx = op.nx_dev ? *op.nx_dev : op.nx;
    const int ny = (op.mode == GRAM_UW) ? nx : 0;
    const int ncol = nx + ny, ts = op.tile + 1;
    const int npairs = (op.mode == GRAM_UW) ? nx * nx + 2 * nx : nx * (nx + 1) / 2;
    const int64_t r0 = (int64_t)blockIdx.x * op.rpb;
    const int64_t r1 = min(op.n, r0 + op.rpb);
    double acc[RGM_GRAM_PMAX];
    int pa[RGM_GRAM_PMAX], pb[RGM_GRAM_PMAX];
#pragma unroll
    for (int i = 0; i < RGM_GRAM_PMAX; ++i) {
        acc[i] = 0.0;
        const int p = threadIdx.x + i * RGM_THREADS;
        int a = 0, b = 0;
        if (p < npairs) {
            if (op.mode == GRAM_PACKED) {
                packed_pair(p, &a, &b);
            } else if (p < nx * nx) {
                a = p % nx;
                b = nx + p / nx;
            } else if (p < nx * nx + nx) {
                a = b = p - nx * nx;
            } else {
                a = b = nx + (p - nx * nx - nx);
            }
        }
        pa[i] = a;
        pb[i] = b;
    }
    for (int64_t base = r0; base < r1; base += op.tile) {
        const int nrow = (int)min((int64_t)op.tile, r1 - base);
        for (int t = threadIdx.x; t < nrow * ncol; t += RGM_THREADS) {
            const int r = t % nrow, c = t / nrow;
            const T *src = c < nx ? op.X + (int64_t)c * op.ldx : op.Y + (int64_t)(c - nx) * op.ldy;
            gsm[c * ts + r] = (double)src[base + r];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RGM_GRAM_PMAX; ++i) {
            if (threadIdx.x + i * RGM_THREADS < npairs) {
                const double *a = gsm + pa[i] * ts, *b = gsm + pb[i] * ts;
                double s = 0.0;
                for (int r = 0; r < nrow; ++r) s += a[r] * b[r];
                acc[i] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RGM_GRAM_PMAX; ++i) {
        const int p = threadIdx.x + i * RGM_THREADS;
        if (p < npairs) op.partials[(int64_t)p * op.nblocks + blockIdx.x] = acc[i];
    }
    if (!last_block(op.counter)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < npairs; c += nw) {
        double v = 0.0;
        const double *p = op.partials + (int64_t)c * op.nblocks;
        for (int b = lane; b < op.nblocks; b += 32) v += __ldcg(p + b);
        v = warp_sum(v);
        if (lane == 0) op.out[c] = v;
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
    __shared__ double g[RGM_HLD];
    __shared__ double yi;
    const int nc = s->J + s->naug;
    for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
        const int i = t % nc, j = t / nc;
        if (i <= j) R[j * (j + 1) / 2 + i] = s->H[i + (int64_t)j * RGM_HLD];
    }
    for (int i = threadIdx.x; i < nc; i += blockDim.x) g[i] = s->g[i];
    __syncthreads();
    for (int i = nc - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            const double d = R[i * (i + 1) / 2 + i];
            yi = (d != 0.0) ? g[i] / d : 0.0;
            s->y[i] = yi;
        }
        __syncthreads();
        const double y = yi;
        for (int t = threadIdx.x; t < i; t += blockDim.x) g[t] -= R[i * (i + 1) / 2 + t] * y;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < RGM_HLD; i += blockDim.x)
        s->coefV[i] = (i < s->J) ? s->y[i] * s->colscale[i] : 0.0;
    for (int i = threadIdx.x; i < RGM_KMAX; i += blockDim.x) s->coefU[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int a = 0; a < s->naug; ++a) s->coefU[s->aug_idx[a]] += s->y[s->J + a];
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

// LU with partial pivoting of E (k x k) in one block; singular when a pivot
// falls below 1e-13 * max(largest pivot, max_i ||u_i|| ||A u_i||).  colnorm2
// holds ||u_i||^2 then ||w_i||^2 (2k values).
static __global__ void lu_kernel(Small *s, int k, const double *gram_uw, const double *colnorm2)
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
