// solver.cu -- librgmres: the C ABI of include/rgmres.h and the host-side
// orchestration of restarted, recycled GMRES on one GPU.
//
// Sec. 3 of the paper defines GMRES as the minimal-residual projection with
// S_k = K_k(A, r0), C_k = A S_k, computed through the Arnoldi relation; Sec. 1
// restarts it every m steps; Sec. 3.1 (augmentation), Sec. 3.2 (deflation with
// P = I - A U E^{-1} U^T) and Table 1 give the recycled variants; Sec. 4.2 the
// projection initial guess x0 = U E^{-1} U^T b; Sec. 5.2 / Algorithm 1 the
// recycle space from a thin SVD of a window of previous solutions.
//
// Host side: one launch per fused pass, stream-ordered, with all scalar state
// (Hessenberg matrix, rotations, flags) on the device; the host synchronises
// once per GMRES cycle to read the residual and decide whether to restart.
#include "../../include/rgmres.h"
#include "common.cuh"
#include "vec_kernels.cuh"
#include "svd_kernels.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

// The CUDA error behind the last RGM_E_CUDA / RGM_E_OOM of this thread
// (rgm_last_error).
static thread_local char g_last_error[320] = "";

void rgm_note_cuda_error(int err, const char *what, int line)
{
    const cudaError_t e = (cudaError_t)err;
    std::snprintf(g_last_error, sizeof g_last_error, "%s (%s) in %s [line %d]", cudaGetErrorName(e),
                  cudaGetErrorString(e), what, line);
}

#define CK(call)                                                             \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            rgm_note_cuda_error((int)e_, #call, __LINE__);                   \
            return (e_ == cudaErrorMemoryAllocation) ? RGM_E_OOM : RGM_E_CUDA; \
        }                                                                    \
    } while (0)

namespace {

struct ProfRec {
    int kind, kry_j;
    double flops, bytes, units, step_bytes;
    cudaEvent_t a, b;
};

// Per-precision device buffers of the Arnoldi process.
template <typename T>
struct Arnoldi {
    const int64_t *slice_ptr = nullptr;
    const int32_t *scol = nullptr;
    const T *sval = nullptr;
    const int32_t *perm = nullptr;
    T *V = nullptr;      // n x (m + k + 1), leading dimension ld
    T *U = nullptr;      // n x kmax
    T *W = nullptr;      // n x kmax (A U)
    T *w = nullptr;      // work vector
    T *r = nullptr;      // residual
    T *b = nullptr;      // right-hand side of this (inner) solve
    T *x = nullptr;      // iterate of this (inner) solve
};

}  // namespace

struct rgm_solver_s {
    rgm_config cfg;
    cudaStream_t st = nullptr;
    int nsm = 0;
    int64_t n = 0, ld = 0, nnz = 0;
    int nblocks = 0, rpb = 0;
    bool have_op = false;
    // operator, sliced ELL (see VecOp); csr2sell maps CSR entry -> ELL slot
    int64_t nslices = 0, nsell = 0;
    int64_t *slice_ptr = nullptr;
    int32_t *scol = nullptr, *perm = nullptr, *csr2sell = nullptr;
    // gather route of new values (sell_gather_kernel): per sliced-ELL entry its
    // CSR offset inside its tile (-1 padding), per tile its first CSR entry, and
    // the shared memory the largest tile needs (0: the scatter route)
    int32_t *sell_src = nullptr;
    int64_t *tile_csr = nullptr;
    size_t gather_smem = 0;
    double *sval = nullptr;
    float *sval32 = nullptr;
    double *val_stage = nullptr;  // host values land here before the scatter
    double *dvec = nullptr;       // left Jacobi: diag(A) of the unscaled operator
    // binary64 vectors
    double *V = nullptr, *U = nullptr, *W = nullptr, *w = nullptr, *r = nullptr, *b = nullptr,
           *x = nullptr;
    // binary32 vectors (GMRES-IR inner solve)
    float *V32 = nullptr, *U32 = nullptr, *W32 = nullptr, *w32 = nullptr, *r32 = nullptr,
          *b32 = nullptr, *x32 = nullptr;
    // recycling
    int k_cur = 0;
    bool k_pending = false;       // a device-side SVD update chose a new k
    bool coarse_stale = true;
    double *X = nullptr;          // snapshot window, n x window (ring)
    int win_count = 0, win_head = 0, updates = 0;
    double *Urow = nullptr;       // row-major copy of U (n x kmax) for the SpMM W = A U
    double *gwin = nullptr;       // window Gram matrix X^T X kept between updates (WMAX^2)
    bool gwin_valid = false;      // gwin matches the stored columns
    int win_last = -1;            // ring slot written by the last update
    // scratch
    double *partials = nullptr;
    unsigned *counter = nullptr;  // [0..3] completion counters, then one per reduction group
    double *gpart = nullptr;      // per-group dot sums (RGM_MAXDOTS x ngroups)
    int ngroups = 0;
    int2 *pairs = nullptr;        // pair list for Gram launches
    double *gram_out = nullptr;
    Small *sm = nullptr;
    Small *hs = nullptr;          // pinned host mirror (header fields)
    // host-mapped {steps done, cycle done} of the running cycle, written by the
    // Givens step: the per-pass launches look at most RGM_LOOKAHEAD steps ahead
    unsigned *prog_host = nullptr, *prog_dev = nullptr;
    int npairs_max = 0;
    // per-launch CUDA-event timing (rgm_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<ProfRec> pending;
    size_t cycle_rec0 = 0;
    rgm_kernel_prof acc[RGM_PROF_KINDS];
    int64_t launches = 0;
    std::vector<double> cyc_flops, cyc_bytes, cyc_step_bytes;   // cost of the first j steps of a cycle launch
    // co-resident capacity of cycle_kernel per precision and dot-column bound
    // (-1: not queried yet)
    int cycle_cap[2][RGM_MAXDOTS + 2];
    int cycle_cap2[2][RGM_MAXDOTS + 2];   // the same for the two-blocks-per-SM build
    bool in_batch = false;        // solving inside rgm_batch_solve: no cooperative launch
    bool zero_guess = false;      // this solve's x_in is zero (RGM_ZERO_GUESS)
    // inside rgm_batch_solve with RGM_BATCH_COOP: the rendezvous this handle's
    // cycle launches join, its index there, and the event marking its inputs ready
    struct BatchCycles *batch = nullptr;
    int batch_idx = 0;
    cudaEvent_t batch_ev = nullptr;
    // device bytes this handle holds, by allocation (rgm_solver_device_bytes)
    std::vector<std::pair<void *, size_t>> allocs;
};

// cudaMalloc that books the allocation on the handle.
static cudaError_t dev_alloc(rgm_solver s, void **p, size_t bytes)
{
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) s->allocs.emplace_back(*p, bytes);
    return e;
}

static void dev_free(rgm_solver s, void *p)
{
    if (!p) return;
    cudaFree(p);
    for (size_t i = 0; i < s->allocs.size(); ++i)
        if (s->allocs[i].first == p) {
            s->allocs[i] = s->allocs.back();
            s->allocs.pop_back();
            break;
        }
}

// Rendezvous of the systems of one rgm_batch_solve(.., RGM_BATCH_COOP, ..): each
// system's host thread runs its own solve and, at every GMRES cycle, hands its
// cycle (the three fused passes of CycleOp) to this object and waits.  When
// every system still solving has arrived, the last one to arrive launches all
// their cycles as one batch_cycle_kernel on the batch's stream (after the
// systems' streams, before their continuations), then wakes the others.
// A system that finishes its solve leaves, which can complete a phase too.
struct BatchCycles {
    struct Req {
        int idx;
        rgm_solver s;
        const void *cyc;          // CycleOp<T> on the waiting thread's stack
        int nd;                   // dot-column bound of the cycle
    };
    std::mutex mu;
    std::condition_variable cv;
    int active = 0;               // systems still inside their solve
    unsigned long long phase = 0; // phases launched so far
    std::vector<Req> arrived;
    std::vector<int> rc;          // per system: result of its last phase
    int precision = RGM_FP64;     // the same for every system of the batch
    cudaStream_t st = nullptr;    // the batch launches' stream
    cudaEvent_t done = nullptr;   // end of the latest phase's launches
    void *d_ops = nullptr;        // CycleOp<T>[nsys] of a phase
    int *d_first = nullptr;       // per wave: first block of each system, then the total
    std::vector<char> h_ops;
    std::vector<int> h_first;
    int cap[RGM_MAXDOTS + 2];     // co-resident blocks by dot-column bound (-1: not queried)
};

static size_t small_header_bytes() { return offsetof(Small, H); }
static int sync_recycle_dim(rgm_solver s);

template <typename T>
static VecOp<T> base_op(rgm_solver s, const Arnoldi<T> &a)
{
    VecOp<T> op;
    std::memset(&op, 0, sizeof op);
    op.n = s->n;
    op.rpb = s->rpb;
    op.nblocks = s->nblocks;
    op.src = SRC_NONE;
    op.slice_ptr = a.slice_ptr;
    op.scol = a.scol;
    op.sval = a.sval;
    op.perm = a.perm;
    op.xscale = -1;
    op.U = a.U;
    op.ldu = s->ld;
    op.V = a.V;
    op.ldv = s->ld;
    op.W = a.W;
    op.ldw = s->ld;
    op.partials = s->partials;
    op.counter = s->counter;
    op.gcount = s->counter + 4;
    op.gpart = s->gpart;
    op.ngroups = s->ngroups;
    op.sm = s->sm;
    op.fin = FIN_NONE;
    op.gate = GATE_NONE;
    op.arg = 0;
    op.lu_sel = 0;
    op.dyn = 0;
    return op;
}

static cudaEvent_t pool_event(rgm_solver s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Algorithmic flops and bytes of one fused pass: what the method must read,
// write and compute (the work vector re-read for the dot pass is not counted).
template <typename T>
static void op_cost(rgm_solver s, const VecOp<T> &op, int nb, int J, double *flops, double *bytes)
{
    const double n = (double)s->n, es = (double)sizeof(T);
    double f = 0.0, b = 0.0;
    int nV = op.nV, ndV = op.ndV;
    if (op.dyn & DYN_NV_NB) nV = nb;
    if (op.dyn & DYN_NV_NBM1) nV = nb;     // nb here is the basis size the step started with
    if (op.dyn & DYN_NV_J) nV = J;
    if (op.dyn & DYN_NDV_NB) ndV = nb;
    if (op.src == SRC_SPMV || op.src == SRC_RES) {
        b += (double)s->nnz * (es + 4.0) + 8.0 * (n + 1) + 2.0 * es * n;
        f += 2.0 * (double)s->nnz;
        if (op.src == SRC_RES) { b += es * n; f += n; }
    } else if (op.src == SRC_COPY) {
        b += 2.0 * es * n;
    } else if (op.src == SRC_AXPY) {
        const int nc = op.nW + nV + op.nU;
        b += es * n * (2.0 + nc);
        f += 2.0 * n * nc;
    }
    const int nd = op.ndU + ndV + op.ndW;
    b += es * n * nd;
    f += 2.0 * n * (nd + op.dnorm);
    *flops = f;
    *bytes = b;
}

// Algorithmic bytes an Arnoldi step with j basis vectors before it must move
// (rgm_kernel_prof::step_bytes): B_j = (e + 4) nnz + e n (j + 2 kdef + 4).
template <typename T>
static double step_bytes(rgm_solver s, int j, int kdef)
{
    const double es = (double)sizeof(T);
    return (es + 4.0) * (double)s->nnz + es * (double)s->n * ((double)j + 2.0 * kdef + 4.0);
}

// NVTX range names, one per profiling kind (a profiler can select or rename
// launches by them; with no tool attached a range push is a no-op call).
static const char *const kNvtxKind[RGM_PROF_KINDS] = {
    "arnoldi_spmv_dots", "arnoldi_cgs1_axpy_dots", "arnoldi_cgs2_axpy_norm", "other_vector", "gram", "small",
    "arnoldi_cycle", "window_svd", "coarse_setup", "operator_values"};

template <typename T>
static int launch(rgm_solver s, const VecOp<T> &op, int kind = RGM_PROF_OTHER, int kry_j = -1,
                  int nb_host = 0, int J_host = 0)
{
    // largest dot-column count this launch can see
    const int nb_bound = (kry_j >= 0) ? kry_j + 1 : (nb_host > 0 ? nb_host : s->cfg.m + s->cfg.k + 1);
    const int nd_max = op.ndU + ((op.dyn & DYN_NDV_NB) ? nb_bound : op.ndV) + op.ndW + op.dnorm;
    ProfRec rec;
    if (s->prof) {
        rec.kind = kind;
        rec.kry_j = kry_j;
        rec.units = (kind == RGM_PROF_ARNOLDI_SPMV) ? 1.0 : 0.0;
        rec.step_bytes = (kind == RGM_PROF_ARNOLDI_SPMV) ? step_bytes<T>(s, kry_j + 1, op.ndU) : 0.0;
        op_cost(s, op, nb_host, J_host, &rec.flops, &rec.bytes);
        rec.a = pool_event(s);
        rec.b = pool_event(s);
        cudaEventRecord(rec.a, s->st);
    }
    nvtxRangePushA(kNvtxKind[kind]);
    const int rc = launch_vec(op, nd_max, s->st);
    nvtxRangePop();
    ++s->launches;
    if (rc) {
        rgm_note_cuda_error(rc, "vec_kernel launch", __LINE__);
        return RGM_E_CUDA;
    }
    if (s->prof) {
        cudaEventRecord(rec.b, s->st);
        s->pending.push_back(rec);
    }
    return RGM_OK;
}

// Launch counting (and optional timing) for the single-block and Gram kernels.
struct ProfScope {
    rgm_solver s;
    ProfRec rec;
    ProfScope(rgm_solver s_, int kind, double flops = 0.0, double bytes = 0.0) : s(s_)
    {
        ++s->launches;
        nvtxRangePushA(kNvtxKind[kind]);
        if (s->prof) {
            rec.kind = kind; rec.kry_j = -1; rec.flops = flops; rec.bytes = bytes; rec.units = 0.0;
            rec.step_bytes = 0.0;
            rec.a = pool_event(s);
            rec.b = pool_event(s);
            cudaEventRecord(rec.a, s->st);
        }
    }
    ~ProfScope()
    {
        nvtxRangePop();
        if (s->prof) {
            cudaEventRecord(rec.b, s->st);
            s->pending.push_back(rec);
        }
    }
};

// After a cycle: Krylov passes launched beyond the J steps actually taken
// returned at once (the device had finished the cycle); book them as overhead.
static void prof_fix_cycle(rgm_solver s, int J)
{
    for (size_t i = s->cycle_rec0; i < s->pending.size(); ++i)
        if (s->pending[i].kind == RGM_PROF_ARNOLDI_CYCLE) {
            const size_t jj = std::min<size_t>((size_t)std::max(J, 0), s->cyc_flops.size() - 1);
            s->pending[i].flops = s->cyc_flops[jj];
            s->pending[i].bytes = s->cyc_bytes[jj];
            s->pending[i].step_bytes = s->cyc_step_bytes[jj];
            s->pending[i].units = (double)jj;
        } else if (s->pending[i].kry_j >= J) {
            s->pending[i].kind = RGM_PROF_OTHER;
            s->pending[i].flops = 0.0;
            s->pending[i].bytes = 0.0;
            s->pending[i].units = 0.0;
            s->pending[i].step_bytes = 0.0;
        }
    s->cycle_rec0 = s->pending.size();
}

static void prof_collect(rgm_solver s)
{
    if (s->pending.empty()) return;
    cudaStreamSynchronize(s->st);
    for (ProfRec &r : s->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        rgm_kernel_prof &a = s->acc[r.kind];
        a.ms += ms;
        a.launches += 1;
        a.flops += r.flops;
        a.bytes += r.bytes;
        a.units += r.units;
        a.step_bytes += r.step_bytes;
        s->ev_pool.push_back(r.a);
        s->ev_pool.push_back(r.b);
    }
    s->pending.clear();
    s->cycle_rec0 = 0;
}

// Gram pairs are generated on the device (no host upload, which for pageable
// memory would synchronise the stream).  nx_dev: optional device count.
template <typename T>
static int launch_gram(rgm_solver s, const T *X, int64_t ldx, int nx, const T *Y, int64_t ldy,
                       int mode, const int *nx_dev, int nxmax, double *out, int col = 0)
{
    if (nxmax <= 0) return RGM_OK;
    const int npmax = (mode == GRAM_UW) ? nxmax * nxmax + 2 * nxmax
                      : (mode == GRAM_COL) ? nxmax : nxmax * (nxmax + 1) / 2;
    if (npmax > s->npairs_max || npmax > RGM_GRAM_PMAX * RGM_THREADS) return RGM_E_ARG;
    GramOp<T> op;
    op.n = s->n;
    op.rpb = s->rpb;
    op.nblocks = s->nblocks;
    op.X = X;
    op.ldx = ldx;
    op.nx = nx;
    op.Y = Y;
    op.ldy = ldy;
    op.nx_dev = nx_dev;
    op.mode = mode;
    op.nxmax = nxmax;
    op.col = col;
    op.partials = s->partials;
    op.counter = s->counter;
    op.gcount = s->counter + 4;
    op.gpart = s->gpart;
    op.ngroups = s->ngroups;
    op.out = out;
    const int ncol = (mode == GRAM_UW) ? 2 * nxmax : nxmax;
    // the row tile of all ncol columns (tile + 1 values each) in dynamic shared
    // memory, within the 48 KB a launch may use without opting in, less the
    // kernel's static shared memory
    // one pair a thread when they fit the block (the per-step Gram matrices)
    const bool one = npmax <= RGM_THREADS;
    static size_t static_smem[2] = {(size_t)-1, (size_t)-1};
    if (static_smem[one] == (size_t)-1) {
        cudaFuncAttributes fa;
        if (one) CK(cudaFuncGetAttributes(&fa, gram_kernel<T, 1>));
        else CK(cudaFuncGetAttributes(&fa, gram_kernel<T, RGM_GRAM_PMAX>));
        static_smem[one] = fa.sharedSizeBytes;
    }
    const int budget = (int)((48 * 1024 - static_smem[one]) / sizeof(T));
    op.tile = std::min(RGM_THREADS, budget / ncol - 1);
    const size_t smem = std::max(sizeof(T) * (size_t)ncol * (op.tile + 1), sizeof(double) * RGM_THREADS);
    {
        const double n = (double)s->n, np_ = (double)npmax;
        ProfScope ps(s, RGM_PROF_GRAM, 2.0 * n * np_, (double)sizeof(T) * n * ncol);
        if (one) gram_kernel<T, 1><<<s->nblocks, RGM_THREADS, smem, s->st>>>(op);
        else gram_kernel<T, RGM_GRAM_PMAX><<<s->nblocks, RGM_THREADS, smem, s->st>>>(op);
    }
    CK(cudaGetLastError());
    return RGM_OK;
}

static int read_header(rgm_solver s)
{
    CK(cudaMemcpyAsync(s->hs, s->sm, small_header_bytes(), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (s->hs->fault) {
        // blocks that gave up left the completion counter mid-count: clear it
        // so that the handle's next solve starts from a clean state
        CK(cudaMemsetAsync(s->counter, 0, sizeof(unsigned) * (4 + s->ngroups), s->st));
        CK(cudaStreamSynchronize(s->st));
        return RGM_E_TIMEOUT;
    }
    return RGM_OK;
}

__global__ void solve_setup_kernel(Small *s, int maxit, int m, int k)
{
    if (threadIdx.x == 0) {
        s->iters = 0;
        s->maxit = maxit;
        s->m = m;
        s->k = k;
        s->converged = 0;
        s->done = 0;
        s->J = 0;
        s->nb = 0;
        s->naug = 0;
        s->skip = 0;
        s->breakdown = 0;
        s->gen = 0u;
        s->fault = 0u;
    }
}

// tol_abs bounds the true residual (never below floor_abs); tol_in the in-cycle
// Givens estimate, which with left Jacobi measures the residual of
// D^{-1} A x = D^{-1} b.
__global__ void set_tol_kernel(Small *s, double rtol, int precond, double floor_abs)
{
    if (threadIdx.x == 0) {
        s->tol_abs = fmax(rtol * s->bnorm, floor_abs);
        s->tol_in = precond ? rtol * s->bnorm_p : s->tol_abs;
    }
}

// W = A U, E = U^T W and the LU of E, once per (operator, recycle space).
// Binary64 solves form them in binary64.  GMRES-IR uses U and W only inside
// its binary32 inner solve, so there W = A U is formed from the binary32
// operator and U (W in binary32, as every vector of the inner solve), and
// E = U^T W is accumulated in binary64 from the stored binary32 columns, so
// that the inner projector is exact for the vectors it is applied with; E
// and its LU stay binary64.
template <typename T>
static int coarse_matrices(rgm_solver s, int k, const T *sval, T *Urow, const T *U, T *W)
{
    const int kp = (k + (16 / (int)sizeof(T)) - 1) / (16 / (int)sizeof(T)) * (16 / (int)sizeof(T));
    if (k > 0) {   // W = A U, one pass over the operator
        {
            ProfScope ps_(s, RGM_PROF_COARSE, 0.0, 2.0 * sizeof(T) * (double)s->n * k);
            urow_kernel<T><<<(unsigned)((s->n + RGM_UROW_ROWS - 1) / RGM_UROW_ROWS), 256, 0, s->st>>>(
                Urow, U, s->n, s->ld, k, kp);
        }
        const int grid = (int)std::min<int64_t>((s->nslices + 7) / 8, 8 * (int64_t)s->nsm);
        const double flops = 2.0 * (double)s->nnz * k;
        const double bytes = (sizeof(T) + 4.0) * (double)s->nnz + sizeof(T) * (double)s->n * (2.0 * k + 1.0);
        ProfScope ps_(s, RGM_PROF_COARSE, flops, bytes);
        spmm_kernel<T><<<grid, 256, 0, s->st>>>(s->slice_ptr, s->scol, sval, s->perm, s->nslices, Urow, k, kp,
                                                W, s->ld);
    }
    CK(cudaGetLastError());
    // E_ij = u_i . w_j, then ||u_i||^2, ||w_i||^2
    int rc = launch_gram<T>(s, U, s->ld, k, W, s->ld, GRAM_UW, nullptr, k, s->gram_out);
    if (rc) return rc;
    { ProfScope ps_(s, RGM_PROF_SMALL); lu_kernel<<<1, 256, 0, s->st>>>(s->sm, k, s->gram_out, s->gram_out + k * k, 0); }
    CK(cudaGetLastError());
    if (s->cfg.proj != RGM_PROJ_OBLIQUE && k > 0) {
        // Gram matrix of the projector's columns: U (orthogonal) or W = A U (least squares)
        const T *Y = (s->cfg.proj == RGM_PROJ_LS) ? W : U;
        if ((rc = launch_gram<T>(s, Y, s->ld, k, Y, s->ld, GRAM_PACKED, nullptr, k, s->gram_out))) return rc;
        { ProfScope ps_(s, RGM_PROF_SMALL); lu_kernel<<<1, 256, 0, s->st>>>(s->sm, k, s->gram_out, nullptr, 1); }
        CK(cudaGetLastError());
    }
    return RGM_OK;
}

static int coarse_setup(rgm_solver s)
{
    const int k = s->k_cur;
    int rc;
    if (s->cfg.precision == RGM_FP32_IR) {
        if (k > 0) {
            ProfScope ps_(s, RGM_PROF_COARSE, 0.0, 12.0 * (double)s->n * k);
            convert_kernel<<<s->nblocks, 256, 0, s->st>>>(s->U32, s->U, s->n, s->ld, k);
        }
        CK(cudaGetLastError());
        rc = coarse_matrices<float>(s, k, s->sval32, reinterpret_cast<float *>(s->Urow), s->U32, s->W32);
    } else {
        rc = coarse_matrices<double>(s, k, s->sval, s->Urow, s->U, s->W);
    }
    if (rc) return rc;
    if ((rc = read_header(s))) return rc;
    s->coarse_stale = false;
    return RGM_OK;
}

// Columns of the deflation projector P w = w - Zp Gp^{-1} Yp^T w (Table 1) and
// of the cycle-end correction x += U Gc^{-1} Yc^T (b - A x), W = A U:
// oblique Yp = U, Zp = W, Gp = E; orthogonal Yp = Zp = U, Gp = U^T U;
// least squares Yp = Zp = W, Gp = W^T W.  The correction uses Yc = U, Gc = E
// except for least squares (Yc = W, Gc = W^T W, so that I - A Q = P).
template <typename T>
struct ProjCols {
    const T *Yp, *Zp, *Yc;
    int psel, csel;      // LU factors: 0 = E's, 1 = the projector's Gram matrix
};

template <typename T>
static ProjCols<T> proj_cols(rgm_solver s, const Arnoldi<T> &a)
{
    ProjCols<T> p;
    const int pj = s->cfg.proj;
    p.Yp = (pj == RGM_PROJ_LS) ? a.W : a.U;
    p.Zp = (pj == RGM_PROJ_ORTHOGONAL) ? a.U : a.W;
    p.Yc = (pj == RGM_PROJ_LS) ? a.W : a.U;
    p.psel = (pj != RGM_PROJ_OBLIQUE) ? 1 : 0;
    p.csel = (pj == RGM_PROJ_LS) ? 1 : 0;
    return p;
}

// The three fused passes of an Arnoldi step with CGS2 (operator P A when kdef
// recycle columns deflate): A v_j and its dots with [U | V], the first
// Gram-Schmidt update and the dots of the second pass, the second update with
// ||w|| and the Givens step.  Step j's input column and scale are set per step.
template <typename T>
static void arnoldi_passes(rgm_solver s, const Arnoldi<T> &a, int kdef, CycleOp<T> &c)
{
    const ProjCols<T> pc = proj_cols(s, a);
    VecOp<T> op = base_op(s, a);
    op.src = SRC_SPMV; op.x = a.V; op.xscale = 0; op.out = a.w;
    op.U = pc.Yp; op.lu_sel = pc.psel;
    op.ndU = kdef; op.dnorm = 1; op.dyn = DYN_NDV_NB; op.fin = FIN_ARN1;
    c.pass[0] = op;
    op = base_op(s, a);
    op.src = SRC_AXPY; op.win = a.w; op.out = a.w; op.nW = kdef; op.W = pc.Zp;
    op.ndW = kdef; op.dnorm = 1;
    op.dyn = DYN_NV_NB | DYN_NDV_NB; op.fin = FIN_ARN2H;
    c.pass[1] = op;
    op = base_op(s, a);
    op.src = SRC_AXPY; op.win = a.w; op.dyn = DYN_NV_NBM1 | DYN_OUT_VNBM1; op.W = pc.Zp;
    op.fin = FIN_NONE;
    c.pass[2] = op;
    c.m = s->cfg.m;
    c.arrive = s->counter + 1;
    c.cap2 = 0;
}

// The cooperative cycle launch applies when the policy allows it and every
// block of the grid can be resident at once (checked by occupancy; the
// cooperative launch itself also refuses a grid that does not fit).
template <typename T>
static bool use_cycle_kernel(rgm_solver s, CycleOp<T> &c, int nd_max)
{
    if (s->cfg.launch_policy != RGM_LAUNCH_AUTO || s->in_batch || nd_max > RGM_MAXDOTS) return false;
    // large systems: the per-pass launches (programmatic dependent launch between
    // passes) beat the grid barriers of the cooperative kernel once a block owns
    // several tiles (measured on GB300: Q4 256x256, 7 tiles a block, 129 against
    // 118 solves/s in GMRES-IR, 101 against 87 in binary64)
    if (s->rpb > RGM_COOP_MAX_TILES * RGM_TILE) return false;
    const int pi = sizeof(T) == 4 ? 1 : 0;
    int &cap = s->cycle_cap[pi][nd_max];
    if (cap < 0) cap = cycle_capacity(c, nd_max, RGM_MINB);
    int &cap2 = s->cycle_cap2[pi][nd_max];
    if (cap2 < 0) cap2 = cycle_capacity(c, nd_max, 2);
    c.cap2 = cap2;
    return s->nblocks <= cap;
}

template <typename T>
static int launch_cycle_prof(rgm_solver s, const CycleOp<T> &c, int nd_max)
{
    ProfRec rec;
    if (s->prof) {
        // algorithmic cost of the first j steps, j = 0..m (booked once J is known):
        // the three passes' flops and bytes, and the steps' B_j
        const int m = c.m;
        s->cyc_flops.assign(m + 1, 0.0);
        s->cyc_bytes.assign(m + 1, 0.0);
        s->cyc_step_bytes.assign(m + 1, 0.0);
        for (int j = 0; j < m; ++j) {
            double f = 0.0, b = 0.0, ft, bt;
            for (int p = 0; p < 3; ++p) {
                op_cost(s, c.pass[p], j + 1, j + 1, &ft, &bt);
                f += ft;
                b += bt;
            }
            s->cyc_flops[j + 1] = s->cyc_flops[j] + f;
            s->cyc_bytes[j + 1] = s->cyc_bytes[j] + b;
            s->cyc_step_bytes[j + 1] = s->cyc_step_bytes[j] + step_bytes<T>(s, j + 1, c.pass[0].ndU);
        }
        rec.kind = RGM_PROF_ARNOLDI_CYCLE;
        rec.kry_j = -1;
        rec.flops = rec.bytes = rec.units = rec.step_bytes = 0.0;
        rec.a = pool_event(s);
        rec.b = pool_event(s);
        cudaEventRecord(rec.a, s->st);
    }
    nvtxRangePushA(kNvtxKind[RGM_PROF_ARNOLDI_CYCLE]);
    const int rc = launch_cycle(c, nd_max, s->st);
    nvtxRangePop();
    ++s->launches;
    if (rc) {
        char what[96];
        std::snprintf(what, sizeof what, "cycle_kernel cooperative launch (%d blocks, capacity %d)",
                      c.pass[0].nblocks, s->cycle_cap[sizeof(T) == 4 ? 1 : 0][nd_max]);
        rgm_note_cuda_error(rc, what, __LINE__);
        return RGM_E_CUDA;
    }
    if (s->prof) {
        cudaEventRecord(rec.b, s->st);
        s->pending.push_back(rec);
    }
    return RGM_OK;
}

// Weights of the true-residual norm: with left Jacobi the stored residual is
// D^{-1} (b - A x), so ||b - A x|| = ||d .* r||.  binary64 solves only.
static const double *res_weights(rgm_solver s, const Arnoldi<double> &) { return s->dvec; }
static const float *res_weights(rgm_solver, const Arnoldi<float> &) { return nullptr; }

// Launch lookahead of the per-pass Arnoldi steps: wait (spinning, at most
// RGM_LOOKAHEAD_WAIT_NS) until the device has finished `steps` steps of the
// cycle or ended it; true when the cycle has ended (launch no more steps).  A
// wait that runs out returns false: the launches go on and the device's own
// done flag still gates them, so nothing depends on the mirror arriving.
static bool progress_done(volatile unsigned *prog, int steps)
{
    if (prog[1]) return true;
    if ((int)prog[0] >= steps) return false;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        if (prog[1]) return true;
        if ((int)prog[0] >= steps) return false;
        if (std::chrono::steady_clock::now() - t0 > std::chrono::nanoseconds(RGM_LOOKAHEAD_WAIT_NS))
            return false;
    }
}

// One recycled GMRES solve of A x = b on the device buffers of `a`, with the
// tolerance tol_abs already in Small.  mode: effective mode (PLAIN if no U).
// Returns the number of cycles through *cycles.
// Block plan of a batched cycle launch (rgm_batch_plan in include/rgmres.h):
// waves of at most cap consecutive systems; a wave whose requests exceed cap
// gives each system one block plus a share of the rest in proportion to its
// work per Arnoldi step (nnz + n x dot columns), never more than it asked for,
// its rows in whole tiles per block.  rpb[i] = 0: the system keeps its own
// partition (blocks[i] = want[i]).  Returns the number of waves.
static int batch_plan(int nsys, const int64_t *n, const int64_t *nnz, const int *nd, const int *want, int cap,
                      int *blocks, int *rpb, int *wave)
{
    int nw = 0;
    for (int w0 = 0; w0 < nsys; ++nw) {
        const int w1 = std::min(nsys, w0 + cap);
        int64_t asked = 0;
        double wsum = 0.0;
        for (int i = w0; i < w1; ++i) {
            asked += want[i];
            wsum += (double)nnz[i] + (double)n[i] * nd[i];
        }
        const int spare = cap - (w1 - w0);
        for (int i = w0; i < w1; ++i) {
            wave[i] = nw;
            blocks[i] = want[i];
            rpb[i] = 0;
            if (asked <= cap) continue;
            const double share = wsum > 0.0 ? ((double)nnz[i] + (double)n[i] * nd[i]) / wsum : 0.0;
            const int nb = std::min(want[i], 1 + (int)std::floor(spare * share));
            if (nb >= want[i]) continue;
            const int64_t ntile = (n[i] + RGM_TILE - 1) / RGM_TILE;
            const int64_t r = (ntile + nb - 1) / nb * RGM_TILE;
            rpb[i] = (int)r;
            blocks[i] = (int)((n[i] + r - 1) / r);
        }
        w0 = w1;
    }
    return nw;
}

// Launch one phase of a batched solve (the caller holds b.mu): the arrived
// systems' cycles in waves of at most `cap` co-resident blocks (batch_plan).
// The plan depends only on the systems of the phase, taken in index order, so
// a batch repeats bit for bit.
template <typename T>
static int batch_phase(BatchCycles &b)
{
    std::vector<BatchCycles::Req> &rq = b.arrived;
    std::sort(rq.begin(), rq.end(),
              [](const BatchCycles::Req &x, const BatchCycles::Req &y) { return x.idx < y.idx; });
    int nd = 0;
    for (const auto &r : rq) nd = std::max(nd, r.nd);
    int &cap = b.cap[nd];
    if (cap < 0) cap = batch_cycle_capacity((const CycleOp<T> *)nullptr, nd);
    if (cap <= 0) {
        rgm_note_cuda_error((int)cudaErrorCooperativeLaunchTooLarge, "batched cycle capacity", __LINE__);
        return RGM_E_CUDA;
    }
    const int ns = (int)rq.size();
    b.h_ops.resize(sizeof(CycleOp<T>) * ns);
    CycleOp<T> *ops = reinterpret_cast<CycleOp<T> *>(b.h_ops.data());
    std::vector<int64_t> vn(ns), vnnz(ns);
    std::vector<int> vnd(ns), want(ns), nblk(ns), rpb(ns), wave(ns);
    for (int i = 0; i < ns; ++i) {
        ops[i] = *static_cast<const CycleOp<T> *>(rq[i].cyc);
        vn[i] = rq[i].s->n;
        vnnz[i] = rq[i].s->nnz;
        vnd[i] = rq[i].nd;
        want[i] = ops[i].pass[0].nblocks;
    }
    batch_plan(ns, vn.data(), vnnz.data(), vnd.data(), want.data(), cap, nblk.data(), rpb.data(), wave.data());
    struct Wave { int s0, s1, f0, nblocks; };
    std::vector<Wave> waves;
    b.h_first.clear();
    for (int i = 0; i < ns; ++i) {
        if (i == 0 || wave[i] != wave[i - 1]) {
            waves.push_back({i, i, (int)b.h_first.size(), 0});
            b.h_first.push_back(0);
        }
        if (rpb[i] > 0)
            for (VecOp<T> &op : ops[i].pass) {
                op.rpb = rpb[i];
                op.nblocks = nblk[i];
                op.ngroups = (nblk[i] + RGM_RGROUP - 1) / RGM_RGROUP;
            }
        Wave &wv = waves.back();
        wv.s1 = i + 1;
        wv.nblocks += nblk[i];
        b.h_first.push_back(wv.nblocks);
    }
    CK(cudaMemcpyAsync(b.d_ops, ops, sizeof(CycleOp<T>) * ns, cudaMemcpyHostToDevice, b.st));
    CK(cudaMemcpyAsync(b.d_first, b.h_first.data(), sizeof(int) * b.h_first.size(), cudaMemcpyHostToDevice,
                       b.st));
    for (const auto &r : rq) CK(cudaStreamWaitEvent(b.st, r.s->batch_ev, 0));
    for (const Wave &wv : waves) {
        nvtxRangePushA(kNvtxKind[RGM_PROF_ARNOLDI_CYCLE]);
        const int rc = launch_batch_cycle(static_cast<const CycleOp<T> *>(b.d_ops) + wv.s0, b.d_first + wv.f0,
                                          wv.s1 - wv.s0, wv.nblocks, nd, b.st);
        nvtxRangePop();
        ++rq[wv.s0].s->launches;
        if (rc) {
            rgm_note_cuda_error(rc, "batch_cycle_kernel launch", __LINE__);
            return RGM_E_CUDA;
        }
    }
    CK(cudaEventRecord(b.done, b.st));
    for (const auto &r : rq) CK(cudaStreamWaitEvent(r.s->st, b.done, 0));
    return RGM_OK;
}

// Complete a phase if every system still solving has arrived (caller holds b.mu).
static void batch_try_launch(BatchCycles &b)
{
    if (b.arrived.empty() || (int)b.arrived.size() < b.active) return;
    const int rc = (b.precision == RGM_FP64) ? batch_phase<double>(b) : batch_phase<float>(b);
    for (const auto &r : b.arrived) b.rc[r.idx] = rc;
    b.arrived.clear();
    ++b.phase;
    b.cv.notify_all();
}

// A system of a batched solve at its cycle launch: join the phase, wait for it.
template <typename T>
static int batch_cycle(rgm_solver s, const CycleOp<T> &c, int nd)
{
    BatchCycles &b = *s->batch;
    CK(cudaEventRecord(s->batch_ev, s->st));
    std::unique_lock<std::mutex> lk(b.mu);
    const unsigned long long ph = b.phase;
    b.arrived.push_back({s->batch_idx, s, &c, nd});
    batch_try_launch(b);
    b.cv.wait(lk, [&] { return b.phase != ph; });
    return b.rc[s->batch_idx];
}

// A system of a batched solve is done (or failed): the others stop waiting for it.
static void batch_leave(BatchCycles &b)
{
    std::lock_guard<std::mutex> lk(b.mu);
    --b.active;
    batch_try_launch(b);
}

template <typename T>
static int gmres_cycles(rgm_solver s, const Arnoldi<T> &a, int mode, int k, int max_cycles,
                        int *cycles_out)
{
    const int m = s->cfg.m;
    int cycles = 0;
    double beta_prev = INFINITY;
    int rc = read_header(s);
    if (rc) return rc;
    while (!s->hs->converged && s->hs->iters < s->hs->maxit && cycles < max_cycles) {
        ++cycles;
        { ProfScope ps_(s, RGM_PROF_SMALL); cycle_reset_kernel<<<1, 256, 0, s->st>>>(s->sm); }
        CK(cudaGetLastError());
        // start vector: r, or P r for the deflated oblique method (Table 1)
        if (mode == RGM_DEFLATED) {
            const ProjCols<T> pc = proj_cols(s, a);
            VecOp<T> op = base_op(s, a);
            if (!s->cfg.start_r) {
                op.src = SRC_COPY; op.win = a.r; op.out = a.w; op.ndU = k; op.fin = FIN_START_DEF1;
                op.U = pc.Yp; op.lu_sel = pc.psel;
                if ((rc = launch(s, op))) return rc;
                op = base_op(s, a);
                op.src = SRC_AXPY; op.win = a.w; op.nW = k;
            } else {
                op.src = SRC_COPY; op.win = a.r;
            }
            op.W = pc.Zp;
            op.out = a.V; op.ndW = k; op.dnorm = 1; op.fin = FIN_START_DEF2;
            if ((rc = launch(s, op))) return rc;
        } else {
            VecOp<T> op = base_op(s, a);
            op.src = SRC_COPY; op.win = a.r; op.out = a.V; op.dnorm = 1; op.fin = FIN_START_PLAIN;
            if ((rc = launch(s, op))) return rc;
        }
        // Arnoldi with CGS2; deflated: operator P A
        const int kdef = (mode == RGM_DEFLATED) ? k : 0;
        CycleOp<T> cyc;
        arnoldi_passes(s, a, kdef, cyc);
        if (s->batch) {
            if ((rc = batch_cycle(s, cyc, kdef + m + 1))) return rc;
        } else if (use_cycle_kernel(s, cyc, kdef + m + 1)) {
            if ((rc = launch_cycle_prof(s, cyc, kdef + m + 1))) return rc;
        } else {
            // the device gates every pass on the cycle's done flag; the host
            // runs at most RGM_LOOKAHEAD steps ahead of the device's progress
            // (host-mapped, written by the Givens step), so that few passes are
            // launched past the step that ends the cycle
            volatile unsigned *prog = s->prog_host;
            prog[0] = 0u;
            prog[1] = 0u;
            for (int j = 0; j < m; ++j) {
                if (j >= RGM_LOOKAHEAD && progress_done(prog, j - RGM_LOOKAHEAD + 1)) break;
                VecOp<T> op = cyc.pass[0];
                op.gate = GATE_KRYLOV;
                op.x = a.V + (int64_t)j * s->ld;
                op.xscale = j;
                if ((rc = launch(s, op, RGM_PROF_ARNOLDI_SPMV, j, j + 1))) return rc;
                op = cyc.pass[1];
                op.gate = GATE_KRYLOV;
                op.mirror = s->prog_dev;
                if ((rc = launch(s, op, RGM_PROF_ARNOLDI_CGS1, j, j + 1))) return rc;
                op = cyc.pass[2];
                op.gate = GATE_STEP;        // also after the step that ended the cycle
                op.arg = j + 1;
                if ((rc = launch(s, op, RGM_PROF_ARNOLDI_CGS2, j, j + 1))) return rc;
            }
        }
        // augmentation: append A u_i to the Arnoldi relation (Sec. 3.1)
        if (mode == RGM_AUGMENTED) {
            for (int i = 0; i < k; ++i) {
                VecOp<T> op = base_op(s, a);
                op.gate = GATE_APPEND;
                op.src = SRC_COPY; op.win = a.W + (int64_t)i * s->ld; op.out = a.w;
                op.dyn = DYN_NDV_NB; op.dnorm = 1; op.fin = FIN_AUG1;
                if ((rc = launch(s, op, RGM_PROF_OTHER, -1, m + 1 + i))) return rc;
                op = base_op(s, a);
                op.gate = GATE_APPEND;
                op.src = SRC_AXPY; op.win = a.w; op.out = a.w; op.dyn = DYN_NV_NB | DYN_NDV_NB;
                op.fin = FIN_ARN2;
                if ((rc = launch(s, op, RGM_PROF_OTHER, -1, m + 1 + i))) return rc;
                op = base_op(s, a);
                op.gate = GATE_APPEND;
                op.src = SRC_AXPY; op.win = a.w; op.dyn = DYN_NV_NB | DYN_OUT_VNB; op.dnorm = 1;
                op.fin = FIN_AUG3; op.arg = i;
                if ((rc = launch(s, op, RGM_PROF_OTHER, -1, m + 1 + i))) return rc;
                { ProfScope ps_(s, RGM_PROF_SMALL); clear_skip_kernel<<<1, 32, 0, s->st>>>(s->sm); }
            }
        }
        { ProfScope ps_(s, RGM_PROF_SMALL); ls_solve_kernel<<<1, 128, 0, s->st>>>(s->sm); }
        CK(cudaGetLastError());
        {   // x += V y (+ U y_aug)
            VecOp<T> op = base_op(s, a);
            op.src = SRC_AXPY; op.win = a.x; op.out = a.x; op.dyn = DYN_NV_J;
            op.nU = (mode == RGM_AUGMENTED) ? k : 0;
            if ((rc = launch(s, op))) return rc;
        }
        if (mode == RGM_DEFLATED) {   // cycle-end correction x += U Gc^{-1} Yc^T (b - A x)
            const ProjCols<T> pc = proj_cols(s, a);
            VecOp<T> op = base_op(s, a);
            op.src = SRC_RES; op.x = a.x; op.b = a.b; op.out = a.r; op.ndU = k; op.fin = FIN_COARSE;
            op.U = pc.Yc; op.lu_sel = pc.csel;
            if ((rc = launch(s, op))) return rc;
            op = base_op(s, a);
            op.src = SRC_AXPY; op.win = a.x; op.out = a.x; op.nU = k;
            if ((rc = launch(s, op))) return rc;
        }
        if (mode == RGM_DEFLATED && sizeof(T) == 4) {
            if ((rc = residual_after_coarse(s, a, k))) return rc;
        } else {
            VecOp<T> op = base_op(s, a);
            op.src = SRC_RES; op.x = a.x; op.b = a.b; op.out = a.r; op.dnorm = 1; op.fin = FIN_RESNORM;
            op.wvec = res_weights(s, a);
            if ((rc = launch(s, op))) return rc;
        }
        if ((rc = read_header(s))) return rc;
        if (s->prof) prof_fix_cycle(s, s->hs->J);
        if (s->hs->J == 0 && !(s->hs->beta < beta_prev)) break;   // stagnation
        beta_prev = s->hs->beta;
    }
    *cycles_out = cycles;
    return RGM_OK;
}

// Projection initial guess / coarse correction on (x, b): x += U E^{-1} U^T (b - A x).
// x_zero: x is known to be zero, so b - A x = b (a copy, no SpMV; same values).
template <typename T>
static int coarse_correct(rgm_solver s, const Arnoldi<T> &a, int k, bool x_zero = false)
{
    VecOp<T> op = base_op(s, a);
    op.src = x_zero ? SRC_COPY : SRC_RES;
    op.x = a.x; op.b = a.b; op.win = a.b; op.out = a.r; op.ndU = k; op.fin = FIN_COARSE;
    int rc = launch(s, op);
    if (rc) return rc;
    op = base_op(s, a);
    op.src = SRC_AXPY; op.win = a.x; op.out = a.x; op.nU = k;
    return launch(s, op);
}

// The residual of x after a coarse correction x += U c: r - W c (W = A U)
// instead of b - A x.  Used by the binary32 inner solve of GMRES-IR, whose
// residuals only steer the inner iteration (the refinement loop recomputes the
// binary64 residual from A); an AXPY over k columns instead of an SpMV.
template <typename T>
static int residual_after_coarse(rgm_solver s, const Arnoldi<T> &a, int k)
{
    VecOp<T> op = base_op(s, a);
    op.src = SRC_AXPY; op.win = a.r; op.out = a.r; op.nW = k; op.W = a.W; op.dnorm = 1;
    op.fin = FIN_RESNORM;
    op.wvec = res_weights(s, a);
    return launch(s, op);
}

template <typename T>
static int residual_norm(rgm_solver s, const Arnoldi<T> &a)
{
    VecOp<T> op = base_op(s, a);
    op.src = SRC_RES; op.x = a.x; op.b = a.b; op.out = a.r; op.dnorm = 1; op.fin = FIN_RESNORM;
    op.wvec = res_weights(s, a);
    return launch(s, op);
}

template <typename T>
static int norm_of(rgm_solver s, const Arnoldi<T> &a, const T *v, int fin)
{
    VecOp<T> op = base_op(s, a);
    op.src = SRC_COPY; op.win = v; op.out = a.w; op.dnorm = 1; op.fin = fin;
    return launch(s, op);
}

static Arnoldi<double> arn64(rgm_solver s)
{
    Arnoldi<double> a;
    a.slice_ptr = s->slice_ptr; a.scol = s->scol; a.sval = s->sval; a.perm = s->perm;
    a.V = s->V; a.U = s->U; a.W = s->W; a.w = s->w; a.r = s->r; a.b = s->b; a.x = s->x;
    return a;
}

static Arnoldi<float> arn32(rgm_solver s)
{
    Arnoldi<float> a;
    a.slice_ptr = s->slice_ptr; a.scol = s->scol; a.sval = s->sval32; a.perm = s->perm;
    a.V = s->V32; a.U = s->U32; a.W = s->W32; a.w = s->w32; a.r = s->r32; a.b = s->b32; a.x = s->x32;
    return a;
}

static int solve_device(rgm_solver s, rgm_stats *out)
{
    const rgm_config &c = s->cfg;
    int status = RGM_OK, rc;
    if ((rc = sync_recycle_dim(s))) return rc;
    int k = (c.mode != RGM_PLAIN) ? s->k_cur : 0;
    if (k > 0 && s->coarse_stale) {
        if ((rc = coarse_setup(s))) return rc;
        if (s->hs->singular) { status = RGM_W_SINGULAR_COARSE; k = 0; }
    } else if (k > 0 && s->hs->singular) {
        status = RGM_W_SINGULAR_COARSE; k = 0;
    }
    // RGM_GUESS: the projection guess below, then plain cycles
    const int mode = (k > 0 && c.mode != RGM_GUESS) ? c.mode : RGM_PLAIN;
    if (c.guess > 0 && s->win_count >= c.guess + 1) {
        // extrapolation from the most recent snapshots replaces the x passed in
        const int newest = (s->win_head - 1 + c.window) % c.window;
        ProfScope ps_(s, RGM_PROF_OTHER, 2.0 * (c.guess + 1) * (double)s->n, 8.0 * (c.guess + 2) * (double)s->n);
        extrap_kernel<<<s->nblocks, 256, 0, s->st>>>(s->x, s->X, s->ld, c.guess + 1, newest, c.window, s->n);
    }
    { ProfScope ps_(s, RGM_PROF_SMALL); solve_setup_kernel<<<1, 32, 0, s->st>>>(s->sm, c.maxit, c.m, k); }
    CK(cudaGetLastError());
    Arnoldi<double> a = arn64(s);
    const int pre = s->dvec != nullptr;
    if ((rc = norm_of(s, a, s->b, FIN_BNORM))) return rc;
    if (pre) {   // left Jacobi: b := D^{-1} b, ||D^{-1} b|| for the in-cycle tolerance
        { ProfScope ps_(s, RGM_PROF_OTHER, (double)s->n, 24.0 * (double)s->n);
          diag_apply_kernel<<<s->nblocks, 256, 0, s->st>>>(s->b, s->dvec, s->n, 1); }
        CK(cudaGetLastError());
        if ((rc = norm_of(s, a, s->b, FIN_BNORMP))) return rc;
    }
    { ProfScope ps_(s, RGM_PROF_SMALL); set_tol_kernel<<<1, 32, 0, s->st>>>(s->sm, c.rtol, pre, 0.0); }
    if (k > 0 && (rc = coarse_correct(s, a, k, s->zero_guess && c.guess == 0))) return rc;   // x0 = x_in + Q (b - A x_in)
    if ((rc = residual_norm(s, a))) return rc;
    if ((rc = read_header(s))) return rc;
    const double bnorm = s->hs->bnorm;
    int cycles = 0, refinements = 0;
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(s->x, 0, sizeof(double) * s->n, s->st));
        CK(cudaStreamSynchronize(s->st));
    } else if (c.precision == RGM_FP64) {
        if ((rc = gmres_cycles(s, a, mode, k, 1 << 30, &cycles))) return rc;
    } else {
        // GMRES-IR: binary64 residual r = b - A x, binary32 recycled GMRES for
        // A d = r to inner_rtol * ||r||, x += d in binary64.
        Arnoldi<float> f = arn32(s);
        int iters_total = 0;
        while (!s->hs->converged && iters_total < c.maxit && refinements < c.max_refinements) {
            ++refinements;
            { ProfScope ps_(s, RGM_PROF_OTHER); convert_kernel<<<s->nblocks, 256, 0, s->st>>>(s->b32, s->r, s->n, s->n, 1); }
            CK(cudaMemsetAsync(s->x32, 0, sizeof(float) * s->n, s->st));
            { ProfScope ps_(s, RGM_PROF_SMALL); solve_setup_kernel<<<1, 32, 0, s->st>>>(s->sm, c.maxit - iters_total, c.m, k); }
            if ((rc = norm_of(s, f, s->b32, FIN_BNORM))) return rc;
            // inner_rtol of the current residual, but no further than half the
            // outer target (the binary64 residual below decides convergence)
            { ProfScope ps_(s, RGM_PROF_SMALL);
              set_tol_kernel<<<1, 32, 0, s->st>>>(s->sm, c.inner_rtol, 0, 0.5 * c.rtol * bnorm); }
            if (k > 0) {     // d = U c from d = 0: residual b32 - W c
                if ((rc = coarse_correct(s, f, k, true))) return rc;
                if ((rc = residual_after_coarse(s, f, k))) return rc;
            } else {         // d = 0: the residual is b32
                VecOp<float> op = base_op(s, f);
                op.src = SRC_COPY; op.win = f.b; op.out = f.r; op.dnorm = 1; op.fin = FIN_RESNORM;
                if ((rc = launch(s, op))) return rc;
            }
            int cy = 0;
            if ((rc = gmres_cycles(s, f, mode, k, c.inner_cycles, &cy))) return rc;
            cycles += cy;
            iters_total += s->hs->iters;
            // x += d (binary64), then the true residual
            { ProfScope ps_(s, RGM_PROF_OTHER); add_f32_kernel<<<s->nblocks, 256, 0, s->st>>>(s->x, s->x32, s->n); }
            { ProfScope ps_(s, RGM_PROF_SMALL); solve_setup_kernel<<<1, 32, 0, s->st>>>(s->sm, c.maxit, c.m, k); }
            if ((rc = norm_of(s, a, s->b, FIN_BNORM))) return rc;
            { ProfScope ps_(s, RGM_PROF_SMALL); set_tol_kernel<<<1, 32, 0, s->st>>>(s->sm, c.rtol, 0, 0.0); }
            if ((rc = residual_norm(s, a))) return rc;
            if ((rc = read_header(s))) return rc;
            s->hs->iters = iters_total;
        }
        s->hs->iters = iters_total;
    }
    const double beta = s->hs->beta;
    const double relres = bnorm > 0.0 ? beta / bnorm : 0.0;
    if (status == RGM_OK && !(relres <= c.rtol)) status = RGM_W_NOT_CONVERGED;
    if (out) {
        out->iters = s->hs->iters;
        out->cycles = cycles;
        out->refinements = refinements;
        out->k_used = k;
        out->status = status;
        out->true_relres = relres;
    }
    return status;
}

// ---------------------------------------------------------------- SVD update (Algorithm 1)
// Everything stays on the device: the chosen dimension k_new is read by the
// kernels that need it, and by the host lazily at the next solve.
static int svd_update(rgm_solver s)
{
    const rgm_config &c = s->cfg;
    const int cnt = s->win_count;
    int rc;
    if (s->gwin_valid) {
        // only the new snapshot's row and column of X^T X change
        if ((rc = launch_gram<double>(s, s->X, s->ld, cnt, s->X, s->ld, GRAM_COL, nullptr, cnt, s->gram_out,
                                      s->win_last)))
            return rc;
        { ProfScope ps_(s, RGM_PROF_SMALL); gram_insert_kernel<<<1, 64, 0, s->st>>>(s->gwin, s->gram_out, s->win_last, cnt); }
    } else {
        if ((rc = launch_gram<double>(s, s->X, s->ld, cnt, s->X, s->ld, GRAM_PACKED, nullptr, cnt, s->gram_out)))
            return rc;
        { ProfScope ps_(s, RGM_PROF_SMALL); gram_unpack_kernel<<<1, 256, 0, s->st>>>(s->gwin, s->gram_out, cnt); }
    }
    CK(cudaGetLastError());
    s->gwin_valid = true;
    { ProfScope ps_(s, RGM_PROF_SMALL); sym_eig_select_kernel<<<1, 512, EIG_SMEM_BYTES, s->st>>>(s->sm, s->gwin, cnt, c.k,
                                                             c.select_smallest, c.rel_drop); }
    CK(cudaGetLastError());
    const int kmax = std::min(c.k, cnt);
    const int *kdev = &s->sm->k_new;
    if (kmax > 0) {
        // U = X Phi_k Sigma_k^{-1} R1^{-1} with the first CholQR pass taken in the
        // window's coordinates, then the second pass on the formed U (k_new read
        // on the device)
        { ProfScope ps_(s, RGM_PROF_SMALL); cholqr_small_kernel<<<1, 256, 0, s->st>>>(s->sm, s->gwin, cnt, kdev); }
        { ProfScope ps_(s, RGM_PROF_SVD); combine_kernel<<<s->nblocks, 256, 0, s->st>>>(s->U, s->X, s->sm->evec, cnt, -1, kdev, s->n, s->ld, RGM_WMAX, 0); }
        CK(cudaGetLastError());
        if ((rc = launch_gram<double>(s, s->U, s->ld, 0, s->U, s->ld, GRAM_PACKED, kdev, kmax, s->gram_out))) return rc;
        { ProfScope ps_(s, RGM_PROF_SMALL); chol_inv_kernel<<<1, 64, 0, s->st>>>(s->sm, s->gram_out, -1, kdev); }
        { ProfScope ps_(s, RGM_PROF_SVD); combine_kernel<<<s->nblocks, 256, 0, s->st>>>(s->U, s->U, s->sm->evec, -1, -1, kdev, s->n, s->ld, RGM_WMAX, 1); }
        CK(cudaGetLastError());
    }
    s->k_pending = true;
    s->coarse_stale = true;
    return RGM_OK;
}

// Pick up the recycle dimension chosen by the last device-side SVD update.
static int sync_recycle_dim(rgm_solver s)
{
    if (!s->k_pending) return RGM_OK;
    int kn = 0;
    CK(cudaMemcpyAsync(&s->hs->k_new, &s->sm->k_new, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    kn = s->hs->k_new;
    s->k_cur = kn;
    s->k_pending = false;
    return RGM_OK;
}

// ================================================================= C ABI
extern "C" {

int rgm_config_default(rgm_config *cfg)
{
    if (!cfg) return RGM_E_ARG;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->m = 30;
    cfg->k = 8;
    cfg->window = 16;
    cfg->svd_interval = 1;
    cfg->mode = RGM_DEFLATED;
    cfg->precision = RGM_FP64;
    cfg->maxit = 20000;
    cfg->inner_cycles = 2;
    cfg->max_refinements = 50;
    cfg->rtol = 1e-10;
    cfg->inner_rtol = 1e-4;
    cfg->rel_drop = 1e-7;
    return RGM_OK;
}

const char *rgm_last_error(void) { return g_last_error; }

const char *rgm_status_string(int code)
{
    switch (code) {
    case RGM_OK: return "ok";
    case RGM_W_NOT_CONVERGED: return "not converged: maxit reached";
    case RGM_W_SINGULAR_COARSE: return "coarse matrix U^T A U singular: solved without recycling";
    case RGM_E_ARG: return "invalid argument";
    case RGM_E_OOM: return "device out of memory";
    case RGM_E_CUDA: return "CUDA error";
    case RGM_E_STATE: return "call out of order";
    case RGM_E_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

static void free_all(rgm_solver s)
{
    void *dp[] = {s->slice_ptr, s->scol, s->perm, s->csr2sell, s->sell_src, s->tile_csr, s->sval, s->sval32, s->val_stage, s->V, s->U, s->W, s->w, s->r, s->b, s->x,
                  s->V32, s->U32, s->W32, s->w32, s->r32, s->b32, s->x32, s->X, s->Urow, s->gwin,
                  s->dvec, s->partials, s->counter, s->gpart, s->pairs, s->gram_out, s->sm};
    for (void *p : dp) dev_free(s, p);
    if (s->hs) cudaFreeHost(s->hs);
    if (s->prog_host) cudaFreeHost(s->prog_host);
    for (ProfRec &r : s->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    if (s->batch_ev) cudaEventDestroy(s->batch_ev);
}

int rgm_solver_create(rgm_solver *out, const rgm_config *cfg)
{
    if (!out || !cfg) return RGM_E_ARG;
    *out = nullptr;
    const rgm_config &c = *cfg;
    if (c.n < 1 || c.m < 1 || c.m > RGM_MMAX || c.k < 0 || c.k > RGM_KMAX || c.window < 1 ||
        c.window > RGM_WMAX || c.svd_interval < 1 || c.mode < RGM_PLAIN || c.mode > RGM_GUESS || c.precision < 0 ||
        c.precision > 1 || c.maxit < 0 || !(c.rtol >= 0) || c.inner_cycles < 1 ||
        c.max_refinements < 1 || !(c.inner_rtol > 0) || !(c.rel_drop >= 0) ||
        c.launch_policy < RGM_LAUNCH_AUTO || c.launch_policy > RGM_LAUNCH_PER_PASS ||
        c.proj < RGM_PROJ_OBLIQUE || c.proj > RGM_PROJ_LS || c.guess < 0 || c.guess > 3 ||
        (c.guess > 0 && c.window < c.guess + 1) || c.precond < RGM_PRECOND_NONE ||
        c.precond > RGM_PRECOND_JACOBI || (c.precond != RGM_PRECOND_NONE && c.precision != RGM_FP64) ||
        c.tiles_per_block < 0)
        return RGM_E_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RGM_E_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RGM_E_CUDA;
    if (cudaFuncSetAttribute(sym_eig_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)EIG_SMEM_BYTES) != cudaSuccess)
        return RGM_E_CUDA;
    if (cudaFuncSetAttribute(sell_gather_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RGM_GATHER_SMEM_MAX) != cudaSuccess)
        return RGM_E_CUDA;
    rgm_solver s = new (std::nothrow) rgm_solver_s();
    if (!s) return RGM_E_OOM;
    for (auto &row : s->cycle_cap)
        for (int &v : row) v = -1;
    for (auto &row : s->cycle_cap2)
        for (int &v : row) v = -1;
    s->cfg = c;
    s->st = (cudaStream_t)c.cuda_stream;
    s->nsm = nsm;
    s->n = c.n;
    s->ld = (c.n + 31) / 32 * 32;
    // blocks own whole RGM_TILE-row tiles (the sliced-ELL sorting windows)
    const int64_t ntile = (s->n + RGM_TILE - 1) / RGM_TILE;
    const int64_t nb_want = std::max<int64_t>(1, std::min<int64_t>(ntile, RGM_MINB * (int64_t)nsm));
    const int64_t tiles_per_block = (c.tiles_per_block > 0) ? std::min<int64_t>(c.tiles_per_block, ntile)
                                                            : (ntile + nb_want - 1) / nb_want;
    s->rpb = (int)(tiles_per_block * RGM_TILE);
    s->nblocks = (int)((s->n + s->rpb - 1) / s->rpb);
    const int kmax = std::max(c.k, 1);
    const int64_t ncolV = c.m + c.k + 1;
    s->npairs_max = RGM_WMAX * (RGM_WMAX + 1) / 2 + RGM_KMAX * RGM_KMAX + 2 * RGM_KMAX;
    cudaError_t e = cudaSuccess;
#define ALLOC(p, bytes) if (e == cudaSuccess) e = dev_alloc(s, (void **)&(p), (bytes))
    ALLOC(s->V, sizeof(double) * s->ld * ncolV);
    ALLOC(s->U, sizeof(double) * s->ld * kmax);
    ALLOC(s->W, sizeof(double) * s->ld * kmax);
    ALLOC(s->w, sizeof(double) * s->ld);
    ALLOC(s->r, sizeof(double) * s->ld);
    ALLOC(s->b, sizeof(double) * s->ld);
    ALLOC(s->x, sizeof(double) * s->ld);
    ALLOC(s->X, sizeof(double) * s->ld * c.window);
    ALLOC(s->Urow, sizeof(double) * s->ld * (kmax + 1));   // rows padded to whole 16-byte vectors
    ALLOC(s->gwin, sizeof(double) * RGM_WMAX * RGM_WMAX);
    ALLOC(s->partials, sizeof(double) * (size_t)std::max(RGM_MAXDOTS, s->npairs_max) * s->nblocks);
    s->ngroups = (s->nblocks + RGM_RGROUP - 1) / RGM_RGROUP;
    ALLOC(s->counter, sizeof(unsigned) * (4 + s->ngroups));
    ALLOC(s->gpart, sizeof(double) * (size_t)std::max(RGM_MAXDOTS, s->npairs_max) * s->ngroups);
    ALLOC(s->pairs, sizeof(int2) * s->npairs_max);
    ALLOC(s->gram_out, sizeof(double) * s->npairs_max);
    ALLOC(s->sm, sizeof(Small));
    if (c.precond == RGM_PRECOND_JACOBI) ALLOC(s->dvec, sizeof(double) * s->ld);
    if (c.precision == RGM_FP32_IR) {
        ALLOC(s->V32, sizeof(float) * s->ld * ncolV);
        ALLOC(s->U32, sizeof(float) * s->ld * kmax);
        ALLOC(s->W32, sizeof(float) * s->ld * kmax);
        ALLOC(s->w32, sizeof(float) * s->ld);
        ALLOC(s->r32, sizeof(float) * s->ld);
        ALLOC(s->b32, sizeof(float) * s->ld);
        ALLOC(s->x32, sizeof(float) * s->ld);
    }
#undef ALLOC
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->hs, sizeof(Small));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->prog_host, 2 * sizeof(unsigned), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s->prog_dev, s->prog_host, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->counter, 0, sizeof(unsigned) * (4 + s->ngroups), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->sm, 0, sizeof(Small), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->V, 0, sizeof(double) * s->ld * ncolV, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
        free_all(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? RGM_E_OOM : RGM_E_CUDA;
    }
    std::memset(s->hs, 0, sizeof(Small));
    *out = s;
    return RGM_OK;
}

int rgm_solver_destroy(rgm_solver s)
{
    if (!s) return RGM_E_ARG;
    cudaStreamSynchronize(s->st);
    free_all(s);
    delete s;
    return RGM_OK;
}

static cudaMemcpyKind kind_in(int flags)
{
    return (flags & RGM_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

static cudaMemcpyKind kind_out(int flags)
{
    return (flags & RGM_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

int rgm_set_operator_csr(rgm_solver s, int64_t n, int64_t nnz, const int64_t *rowptr,
                         const int32_t *col, const double *val, int flags)
{
    if (!s || n != s->n || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val))) return RGM_E_ARG;
    // validate the pattern on a host copy
    const cudaMemcpyKind hk = (flags & RGM_DEVICE_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    std::vector<int64_t> rp(n + 1);
    if (cudaMemcpy(rp.data(), rowptr, sizeof(int64_t) * (n + 1), hk) != cudaSuccess) return RGM_E_CUDA;
    if (rp[0] != 0 || rp[n] != nnz) return RGM_E_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return RGM_E_ARG;
    std::vector<int32_t> cl(nnz);
    if (nnz && cudaMemcpy(cl.data(), col, sizeof(int32_t) * nnz, hk) != cudaSuccess) return RGM_E_CUDA;
    for (int64_t e = 0; e < nnz; ++e)
        if (cl[e] < 0 || cl[e] >= n) return RGM_E_ARG;
    // sliced ELL: inside each tile, rows sorted by length (descending, stable)
    const int64_t ntile = (n + RGM_TILE - 1) / RGM_TILE, nslices = ntile * (RGM_TILE / 32);
    std::vector<int32_t> perm(nslices * 32, -1);
    std::vector<int64_t> sp(nslices + 1, 0);
    std::vector<int> idx(RGM_TILE);
    for (int64_t t = 0; t < ntile; ++t) {
        const int64_t r0 = t * RGM_TILE, cnt = std::min<int64_t>(RGM_TILE, n - r0);
        for (int i = 0; i < cnt; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.begin() + cnt, [&](int a, int b) {
            return rp[r0 + a + 1] - rp[r0 + a] > rp[r0 + b + 1] - rp[r0 + b];
        });
        for (int i = 0; i < cnt; ++i) perm[r0 + i] = (int32_t)(r0 + idx[i]);
    }
    for (int64_t sl = 0; sl < nslices; ++sl) {
        int64_t width = 0;
        for (int l = 0; l < 32; ++l) {
            const int32_t r = perm[sl * 32 + l];
            if (r >= 0) width = std::max<int64_t>(width, rp[r + 1] - rp[r]);
        }
        sp[sl + 1] = sp[sl] + 32 * width;
    }
    const int64_t nsell = sp[nslices];
    if (nsell >= ((int64_t)1 << 31)) return RGM_E_ARG;
    std::vector<int32_t> scol(std::max<int64_t>(nsell, 1));
    std::vector<int32_t> map(std::max<int64_t>(nnz, 1));
    std::vector<int32_t> src(std::max<int64_t>(nsell, 1));
    std::vector<int64_t> tcsr(ntile + 1);
    int64_t tmax = 0;
    for (int64_t t = 0; t <= ntile; ++t) tcsr[t] = rp[std::min<int64_t>(t * RGM_TILE, n)];
    for (int64_t t = 0; t < ntile; ++t) tmax = std::max(tmax, tcsr[t + 1] - tcsr[t]);
    for (int64_t sl = 0; sl < nslices; ++sl) {
        const int64_t width = (sp[sl + 1] - sp[sl]) / 32;
        const int64_t c0 = tcsr[sl / (RGM_TILE / 32)];
        for (int l = 0; l < 32; ++l) {
            const int32_t r = perm[sl * 32 + l];
            const int64_t len = r >= 0 ? rp[r + 1] - rp[r] : 0;
            for (int64_t k = 0; k < width; ++k) {
                const int64_t e = sp[sl] + 32 * k + l;
                if (k < len) {
                    scol[e] = cl[rp[r] + k];
                    map[rp[r] + k] = (int32_t)e;
                    src[e] = (int32_t)(rp[r] + k - c0);
                } else {
                    scol[e] = r >= 0 ? r : 0;       // padding: value 0 on a valid column
                    src[e] = -1;
                }
            }
        }
    }
    // the gather route when the largest tile's values fit in shared memory
    const size_t gsmem = sizeof(double) * (size_t)std::max<int64_t>(tmax, 1);
    const bool gather = gsmem <= RGM_GATHER_SMEM_MAX;
    void *old[] = {s->slice_ptr, s->scol, s->perm, s->csr2sell, s->sell_src, s->tile_csr, s->sval, s->sval32,
                   s->val_stage};
    for (void *p : old) dev_free(s, p);
    s->slice_ptr = nullptr; s->scol = nullptr; s->perm = nullptr; s->csr2sell = nullptr;
    s->sell_src = nullptr; s->tile_csr = nullptr; s->gather_smem = 0;
    s->sval = nullptr; s->sval32 = nullptr; s->val_stage = nullptr;
    CK(dev_alloc(s, (void **)&s->slice_ptr, sizeof(int64_t) * (nslices + 1)));
    CK(dev_alloc(s, (void **)&s->scol, sizeof(int32_t) * std::max<int64_t>(nsell, 1)));
    CK(dev_alloc(s, (void **)&s->perm, sizeof(int32_t) * nslices * 32));
    if (gather) {
        CK(dev_alloc(s, (void **)&s->sell_src, sizeof(int32_t) * std::max<int64_t>(nsell, 1)));
        CK(dev_alloc(s, (void **)&s->tile_csr, sizeof(int64_t) * (ntile + 1)));
    } else {
        CK(dev_alloc(s, (void **)&s->csr2sell, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    }
    CK(dev_alloc(s, (void **)&s->sval, sizeof(double) * std::max<int64_t>(nsell, 1)));
    CK(dev_alloc(s, (void **)&s->val_stage, sizeof(double) * std::max<int64_t>(nnz, 1)));
    if (s->cfg.precision == RGM_FP32_IR)
        CK(dev_alloc(s, (void **)&s->sval32, sizeof(float) * std::max<int64_t>(nsell, 1)));
    CK(cudaMemcpyAsync(s->slice_ptr, sp.data(), sizeof(int64_t) * (nslices + 1), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->scol, scol.data(), sizeof(int32_t) * std::max<int64_t>(nsell, 1), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->perm, perm.data(), sizeof(int32_t) * nslices * 32, cudaMemcpyHostToDevice, s->st));
    if (gather) {
        CK(cudaMemcpyAsync(s->sell_src, src.data(), sizeof(int32_t) * std::max<int64_t>(nsell, 1),
                           cudaMemcpyHostToDevice, s->st));
        CK(cudaMemcpyAsync(s->tile_csr, tcsr.data(), sizeof(int64_t) * (ntile + 1), cudaMemcpyHostToDevice, s->st));
        s->gather_smem = gsmem;
    } else {
        CK(cudaMemcpyAsync(s->csr2sell, map.data(), sizeof(int32_t) * std::max<int64_t>(nnz, 1),
                           cudaMemcpyHostToDevice, s->st));
    }
    CK(cudaMemsetAsync(s->sval, 0, sizeof(double) * std::max<int64_t>(nsell, 1), s->st));
    if (s->sval32) CK(cudaMemsetAsync(s->sval32, 0, sizeof(float) * std::max<int64_t>(nsell, 1), s->st));
    CK(cudaStreamSynchronize(s->st));
    s->nnz = nnz;
    s->nslices = nslices;
    s->nsell = nsell;
    s->have_op = true;
    return rgm_set_operator_values(s, val, flags);
}

int rgm_set_operator_sell(rgm_solver s, int64_t n, int64_t nslices, const int64_t *slice_ptr,
                          const int32_t *perm, const int32_t *col, const double *val, int flags)
{
    if (!s || n != s->n || !slice_ptr || !perm) return RGM_E_ARG;
    const int64_t ntile = (n + RGM_TILE - 1) / RGM_TILE;
    if (nslices != ntile * (RGM_TILE / 32)) return RGM_E_ARG;
    // validate the layout on host copies
    const cudaMemcpyKind hk = (flags & RGM_DEVICE_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    std::vector<int64_t> sp(nslices + 1);
    std::vector<int32_t> pm(nslices * 32);
    if (cudaMemcpy(sp.data(), slice_ptr, sizeof(int64_t) * (nslices + 1), hk) != cudaSuccess) return RGM_E_CUDA;
    if (cudaMemcpy(pm.data(), perm, sizeof(int32_t) * nslices * 32, hk) != cudaSuccess) return RGM_E_CUDA;
    if (sp[0] != 0) return RGM_E_ARG;
    for (int64_t q = 0; q < nslices; ++q)
        if (sp[q + 1] < sp[q] || (sp[q + 1] - sp[q]) % 32 != 0) return RGM_E_ARG;
    const int64_t nsell = sp[nslices];
    if (nsell >= ((int64_t)1 << 31) || (nsell > 0 && (!col || !val))) return RGM_E_ARG;
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < nslices * 32; ++i) {
        const int32_t r = pm[i];
        if (r < 0) continue;
        const int64_t t = i / RGM_TILE;
        if (r >= n || r < t * RGM_TILE || r >= (t + 1) * RGM_TILE || seen[r]) return RGM_E_ARG;
        seen[r] = 1;
    }
    for (int64_t r = 0; r < n; ++r)
        if (!seen[r]) return RGM_E_ARG;
    std::vector<int32_t> cl(std::max<int64_t>(nsell, 1));
    if (nsell && cudaMemcpy(cl.data(), col, sizeof(int32_t) * nsell, hk) != cudaSuccess) return RGM_E_CUDA;
    for (int64_t e = 0; e < nsell; ++e)
        if (cl[e] < 0 || cl[e] >= n) return RGM_E_ARG;
    // values arrive in this layout: the scatter map is the identity
    std::vector<int32_t> map(std::max<int64_t>(nsell, 1));
    for (int64_t e = 0; e < nsell; ++e) map[e] = (int32_t)e;
    void *old[] = {s->slice_ptr, s->scol, s->perm, s->csr2sell, s->sell_src, s->tile_csr, s->sval, s->sval32,
                   s->val_stage};
    for (void *p : old) dev_free(s, p);
    s->slice_ptr = nullptr; s->scol = nullptr; s->perm = nullptr; s->csr2sell = nullptr;
    s->sell_src = nullptr; s->tile_csr = nullptr; s->gather_smem = 0;
    s->sval = nullptr; s->sval32 = nullptr; s->val_stage = nullptr;
    const int64_t ne = std::max<int64_t>(nsell, 1);
    CK(dev_alloc(s, (void **)&s->slice_ptr, sizeof(int64_t) * (nslices + 1)));
    CK(dev_alloc(s, (void **)&s->scol, sizeof(int32_t) * ne));
    CK(dev_alloc(s, (void **)&s->perm, sizeof(int32_t) * nslices * 32));
    CK(dev_alloc(s, (void **)&s->csr2sell, sizeof(int32_t) * ne));
    CK(dev_alloc(s, (void **)&s->sval, sizeof(double) * ne));
    CK(dev_alloc(s, (void **)&s->val_stage, sizeof(double) * ne));
    if (s->cfg.precision == RGM_FP32_IR) CK(dev_alloc(s, (void **)&s->sval32, sizeof(float) * ne));
    CK(cudaMemcpyAsync(s->slice_ptr, sp.data(), sizeof(int64_t) * (nslices + 1), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->scol, cl.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->perm, pm.data(), sizeof(int32_t) * nslices * 32, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->csr2sell, map.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(s->sval, 0, sizeof(double) * ne, s->st));
    if (s->sval32) CK(cudaMemsetAsync(s->sval32, 0, sizeof(float) * ne, s->st));
    CK(cudaStreamSynchronize(s->st));
    s->nnz = nsell;
    s->nslices = nslices;
    s->nsell = nsell;
    s->have_op = true;
    return rgm_set_operator_values(s, val, flags);
}

int rgm_set_operator_values(rgm_solver s, const double *val, int flags)
{
    if (!s || (s->nnz > 0 && !val)) return RGM_E_ARG;
    if (!s->have_op) return RGM_E_STATE;
    if (s->nnz) {
        const double *src = val;
        if (!(flags & RGM_DEVICE_PTRS)) {
            CK(cudaMemcpyAsync(s->val_stage, val, sizeof(double) * s->nnz, cudaMemcpyHostToDevice, s->st));
            src = s->val_stage;
        }
        if (s->gather_smem) {
            ProfScope ps_(s, RGM_PROF_OPERATOR, 0.0, 2.0 * 8.0 * (double)s->nnz + 16.0 * (double)s->nsell);
            sell_gather_kernel<double><<<(unsigned)((s->n + RGM_TILE - 1) / RGM_TILE), RGM_GATHER_THREADS,
                                         s->gather_smem, s->st>>>(
                s->sval, s->sval32, src, s->tile_csr, s->slice_ptr, s->sell_src);
        } else {
            const int g = (int)std::min<int64_t>((s->nnz + 255) / 256, 8 * (int64_t)s->nsm);
            ProfScope ps_(s, RGM_PROF_OPERATOR, 0.0, 2.0 * 8.0 * (double)s->nnz + 16.0 * (double)s->nsell);
            sell_scatter_kernel<double><<<g, 256, 0, s->st>>>(s->sval, s->sval32, src, s->csr2sell, s->nnz);
        }
        CK(cudaGetLastError());
    }
    if (s->dvec) {   // left Jacobi: keep D^{-1} A, remember D
        const int g = (int)std::min<int64_t>((s->nslices + 7) / 8, 8 * (int64_t)s->nsm);
        ProfScope ps_(s, RGM_PROF_OPERATOR);
        jacobi_scale_kernel<<<std::max(g, 1), 256, 0, s->st>>>(s->sval, s->scol, s->slice_ptr, s->perm,
                                                              s->nslices, s->dvec);
        CK(cudaGetLastError());
    }
    s->coarse_stale = true;
    if (!(flags & RGM_DEVICE_PTRS)) CK(cudaStreamSynchronize(s->st));
    return RGM_OK;
}

int rgm_set_recycle_space(rgm_solver s, const double *U, int k, int64_t ld, int flags)
{
    if (!s || k < 0 || k > s->cfg.k || (k > 0 && (!U || ld < s->n))) return RGM_E_ARG;
    for (int i = 0; i < k; ++i)
        CK(cudaMemcpyAsync(s->U + (int64_t)i * s->ld, U + (int64_t)i * ld, sizeof(double) * s->n,
                           kind_in(flags), s->st));
    CK(cudaStreamSynchronize(s->st));
    s->k_cur = k;
    s->k_pending = false;
    s->coarse_stale = true;
    return RGM_OK;
}

int rgm_get_recycle_space(rgm_solver s, double *U, int64_t ld, int *k, int flags)
{
    if (!s || !k) return RGM_E_ARG;
    int rc = sync_recycle_dim(s);
    if (rc) return rc;
    *k = s->k_cur;
    if (!U) return RGM_OK;
    if (ld < s->n) return RGM_E_ARG;
    for (int i = 0; i < s->k_cur; ++i)
        CK(cudaMemcpyAsync(U + (int64_t)i * ld, s->U + (int64_t)i * s->ld, sizeof(double) * s->n,
                           kind_out(flags), s->st));
    CK(cudaStreamSynchronize(s->st));
    return RGM_OK;
}

int rgm_solve(rgm_solver s, const double *b, double *x, int flags, rgm_stats *st)
{
    if (!s || !b || !x) return RGM_E_ARG;
    if (!s->have_op) return RGM_E_STATE;
    CK(cudaMemcpyAsync(s->b, b, sizeof(double) * s->n, kind_in(flags), s->st));
    if (flags & RGM_ZERO_GUESS) CK(cudaMemsetAsync(s->x, 0, sizeof(double) * s->n, s->st));
    else CK(cudaMemcpyAsync(s->x, x, sizeof(double) * s->n, kind_in(flags), s->st));
    s->zero_guess = (flags & RGM_ZERO_GUESS) != 0;
    int rc = solve_device(s, st);
    if (rc < 0) return rc;
    CK(cudaMemcpyAsync(x, s->x, sizeof(double) * s->n, kind_out(flags), s->st));
    CK(cudaStreamSynchronize(s->st));
    return rc;
}

int rgm_batch_plan(int nsys, const int64_t *n, const int64_t *nnz, const int *nd, const int *want, int cap,
                   int *blocks, int *rpb, int *wave)
{
    if (nsys < 0 || cap < 1 || (nsys > 0 && (!n || !nnz || !nd || !want || !blocks || !rpb || !wave)))
        return RGM_E_ARG;
    for (int i = 0; i < nsys; ++i)
        if (n[i] < 1 || nnz[i] < 0 || nd[i] < 0 || want[i] < 1) return RGM_E_ARG;
    return batch_plan(nsys, n, nnz, nd, want, cap, blocks, rpb, wave);
}

int rgm_batch_solve(rgm_solver *handles, int nsys, const double *const *b, double *const *x, int flags,
                    rgm_stats *st)
{
    if (nsys < 0 || (nsys > 0 && (!handles || !b || !x))) return RGM_E_ARG;
    {
        std::vector<rgm_solver> hs(handles, handles + nsys);
        std::sort(hs.begin(), hs.end());
        for (int i = 0; i < nsys; ++i)
            if (!hs[i] || !b[i] || !x[i] || (i > 0 && hs[i] == hs[i - 1])) return RGM_E_ARG;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // batched cycle launches: every handle in the same precision, none forced
    // to per-pass launches, and a device that launches cooperatively
    bool coop = (flags & RGM_BATCH_COOP) && nsys > 0;
    for (int i = 0; coop && i < nsys; ++i)
        coop = handles[i]->cfg.precision == handles[0]->cfg.precision &&
               handles[i]->cfg.launch_policy == RGM_LAUNCH_AUTO;
    if (coop) {
        const CycleOp<double> *p64 = nullptr;
        coop = batch_cycle_capacity(p64, 1) > 0;
    }
    flags &= ~RGM_BATCH_COOP;
    BatchCycles bc;
    if (coop) {
        for (int &v : bc.cap) v = -1;
        bc.active = nsys;
        bc.rc.assign(nsys, RGM_OK);
        bc.precision = handles[0]->cfg.precision;
        const size_t opsz = bc.precision == RGM_FP64 ? sizeof(CycleOp<double>) : sizeof(CycleOp<float>);
        CK(cudaStreamCreateWithFlags(&bc.st, cudaStreamNonBlocking));
        cudaError_t e = cudaEventCreateWithFlags(&bc.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocAsync(&bc.d_ops, opsz * nsys, bc.st);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&bc.d_first, sizeof(int) * (2 * nsys + 2), bc.st);
        for (int i = 0; e == cudaSuccess && i < nsys; ++i) {
            rgm_solver s = handles[i];
            if (!s->batch_ev) e = cudaEventCreateWithFlags(&s->batch_ev, cudaEventDisableTiming);
            s->batch = &bc;
            s->batch_idx = i;
        }
        if (e != cudaSuccess) {
            for (int i = 0; i < nsys; ++i) handles[i]->batch = nullptr;
            if (bc.d_ops) cudaFreeAsync(bc.d_ops, bc.st);
            if (bc.d_first) cudaFreeAsync(bc.d_first, bc.st);
            if (bc.done) cudaEventDestroy(bc.done);
            cudaStreamDestroy(bc.st);
            rgm_note_cuda_error((int)e, "batched cycle setup", __LINE__);
            return e == cudaErrorMemoryAllocation ? RGM_E_OOM : RGM_E_CUDA;
        }
    }
    std::vector<int> rc(nsys, RGM_OK);
    std::atomic<int> next(0);
    std::mutex mu;
    std::string first_error;
    auto solve_one = [&](int i) {
        rgm_solver s = handles[i];
        s->in_batch = true;
        rc[i] = rgm_solve(s, b[i], x[i], flags, st ? &st[i] : nullptr);
        s->in_batch = false;
        if (coop) batch_leave(bc);
        if (rc[i] < 0) {
            std::lock_guard<std::mutex> lk(mu);
            if (first_error.empty()) first_error = g_last_error;
        }
    };
    bool dev_ok = true;
    if (coop) {
        // one thread per system: a system waits at the rendezvous until every
        // other system still solving has reached its own cycle launch
        std::atomic<int> started(0);
        auto one = [&](int i) {
            if (cudaSetDevice(dev) != cudaSuccess) {
                rc[i] = RGM_E_CUDA;
                batch_leave(bc);
                return;
            }
            started.fetch_add(1);
            solve_one(i);
        };
        std::vector<std::thread> pool;
        for (int i = 1; i < nsys; ++i) pool.emplace_back(one, i);
        one(0);
        for (auto &th : pool) th.join();
        dev_ok = started.load() == nsys;
        for (int i = 0; i < nsys; ++i) handles[i]->batch = nullptr;
        cudaFreeAsync(bc.d_ops, bc.st);
        cudaFreeAsync(bc.d_first, bc.st);
        cudaStreamSynchronize(bc.st);
        cudaEventDestroy(bc.done);
        cudaStreamDestroy(bc.st);
    } else {
        auto work = [&]() {
            if (cudaSetDevice(dev) != cudaSuccess) return;
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= nsys) break;
                solve_one(i);
            }
        };
        const int nthr = std::max(1, std::min<int>(nsys, (int)std::max(1u, std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        for (int t = 1; t < nthr; ++t) pool.emplace_back(work);
        work();
        for (auto &th : pool) th.join();
        dev_ok = next.load() >= nsys;
    }
    if (!dev_ok) return RGM_E_CUDA;            // a worker could not select the device
    int worst = RGM_OK;
    for (int r : rc) {
        if (r < 0) { if (worst >= 0) worst = r; }
        else if (worst >= 0 && r > worst) worst = r;
    }
    if (!first_error.empty()) std::snprintf(g_last_error, sizeof g_last_error, "%s", first_error.c_str());
    return worst;
}

int rgm_update_recycle_svd(rgm_solver s, const double *x, int flags, int *k_used)
{
    if (!s || !x) return RGM_E_ARG;
    CK(cudaMemcpyAsync(s->X + (int64_t)s->win_head * s->ld, x, sizeof(double) * s->n, kind_in(flags),
                       s->st));
    // the resident window Gram matrix tracks one new column per update; a
    // column stored without an update (svd_interval > 1) invalidates it
    if (s->win_last >= 0 && !(s->cfg.k > 0 && (s->updates + 1) % s->cfg.svd_interval == 0))
        s->gwin_valid = false;
    s->win_last = s->win_head;
    s->win_head = (s->win_head + 1) % s->cfg.window;
    if (s->win_count < s->cfg.window) ++s->win_count;
    ++s->updates;
    if (s->cfg.k > 0 && s->updates % s->cfg.svd_interval == 0) {
        int rc = svd_update(s);
        if (rc) return rc;
    }
    if (k_used) {
        int rc = sync_recycle_dim(s);
        if (rc) return rc;
        *k_used = s->k_cur;
    }
    // host buffers: the copy must be done before the caller may reuse x
    if (!(flags & RGM_DEVICE_PTRS)) CK(cudaStreamSynchronize(s->st));
    return RGM_OK;
}

int rgm_get_singular_values(rgm_solver s, double *sigma, int *count)
{
    if (!s || !sigma || !count) return RGM_E_ARG;
    CK(cudaStreamSynchronize(s->st));
    CK(cudaMemcpy(s->hs, s->sm, sizeof(Small), cudaMemcpyDeviceToHost));
    const int c = s->win_count;
    for (int i = 0; i < c; ++i) {
        double l = s->hs->eval[s->hs->ord[i]];
        sigma[i] = l > 0 ? std::sqrt(l) : 0.0;
    }
    *count = c;
    return RGM_OK;
}

int rgm_reset_recycling(rgm_solver s)
{
    if (!s) return RGM_E_ARG;
    s->win_count = 0;
    s->win_head = 0;
    s->updates = 0;
    s->gwin_valid = false;
    s->win_last = -1;
    CK(cudaMemsetAsync(&s->sm->phi_c, 0, sizeof(int), s->st));
    CK(cudaStreamSynchronize(s->st));
    s->k_cur = 0;
    s->k_pending = false;
    s->coarse_stale = true;
    return RGM_OK;
}

// Checkpoint layout: StateHeader, then win_used window columns (ring slots
// 0..win_used-1, n doubles each), k_cur columns of U, (gram set) the
// win_used x win_used window Gram matrix the next update builds on, and the
// phi_c x phi_c eigenvectors of the last window Gram matrix that the next
// eigen-decomposition starts from (version 3; version 2 has none).
namespace {
struct StateHeader {
    uint32_t magic, version;
    int64_t n;
    int32_t window, k_cur, win_count, win_head;
    int64_t updates;
    int32_t gram, phi_c;
};
const uint32_t kStateMagic = 0x314d4752u;   // bytes "RGM1" in little-endian order
}  // namespace

int rgm_export_state(rgm_solver s, void *buf, size_t *bytes)
{
    if (!s || !bytes) return RGM_E_ARG;
    int rc = sync_recycle_dim(s);
    if (rc) return rc;
    const int win_used = s->win_count;   // ring slots 0..win_count-1 hold data
    const int with_gram = s->gwin_valid ? 1 : 0;
    int pc = 0;
    CK(cudaStreamSynchronize(s->st));
    CK(cudaMemcpy(&pc, &s->sm->phi_c, sizeof(int), cudaMemcpyDeviceToHost));
    if (pc < 0 || pc > win_used) pc = 0;
    const size_t need = sizeof(StateHeader) + sizeof(double) * ((size_t)s->n * (win_used + s->k_cur) +
                                                                (size_t)with_gram * win_used * win_used +
                                                                (size_t)pc * pc);
    if (!buf) { *bytes = need; return RGM_OK; }
    if (*bytes < need) return RGM_E_ARG;
    StateHeader h;
    h.magic = kStateMagic;
    h.version = 3;
    h.n = s->n;
    h.window = s->cfg.window;
    h.k_cur = s->k_cur;
    h.win_count = s->win_count;
    h.win_head = s->win_head;
    h.updates = s->updates;
    h.gram = with_gram;
    h.phi_c = pc;
    std::memcpy(buf, &h, sizeof h);
    double *d = reinterpret_cast<double *>(static_cast<char *>(buf) + sizeof h);
    for (int i = 0; i < win_used; ++i)
        CK(cudaMemcpyAsync(d + (size_t)i * s->n, s->X + (int64_t)i * s->ld, sizeof(double) * s->n,
                           cudaMemcpyDeviceToHost, s->st));
    d += (size_t)win_used * s->n;
    for (int i = 0; i < s->k_cur; ++i)
        CK(cudaMemcpyAsync(d + (size_t)i * s->n, s->U + (int64_t)i * s->ld, sizeof(double) * s->n,
                           cudaMemcpyDeviceToHost, s->st));
    d += (size_t)s->k_cur * s->n;
    for (int j = 0; j < win_used && with_gram; ++j)
        CK(cudaMemcpyAsync(d + (size_t)j * win_used, s->gwin + (int64_t)j * RGM_WMAX,
                           sizeof(double) * win_used, cudaMemcpyDeviceToHost, s->st));
    d += (size_t)with_gram * win_used * win_used;
    for (int j = 0; j < pc; ++j)
        CK(cudaMemcpyAsync(d + (size_t)j * pc, s->sm->phi + (int64_t)j * RGM_WMAX, sizeof(double) * pc,
                           cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    *bytes = need;
    return RGM_OK;
}

int rgm_import_state(rgm_solver s, const void *buf, size_t bytes)
{
    if (!s || !buf || bytes < sizeof(StateHeader)) return RGM_E_ARG;
    StateHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.version == 2) h.phi_c = 0;          // written before the warm start existed
    if (h.magic != kStateMagic || (h.version != 2 && h.version != 3) || h.n != s->n ||
        h.window != s->cfg.window || h.k_cur < 0 || h.k_cur > s->cfg.k || h.win_count < 0 ||
        h.win_count > h.window || h.win_head < 0 || h.win_head >= h.window || h.updates < h.win_count ||
        h.gram < 0 || h.gram > 1 || h.phi_c < 0 || h.phi_c > h.win_count)
        return RGM_E_ARG;
    const size_t need = sizeof(StateHeader) + sizeof(double) * ((size_t)s->n * (h.win_count + h.k_cur) +
                                                                (size_t)h.gram * h.win_count * h.win_count +
                                                                (size_t)h.phi_c * h.phi_c);
    if (bytes != need) return RGM_E_ARG;
    CK(cudaStreamSynchronize(s->st));
    const double *d = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof h);
    for (int i = 0; i < h.win_count; ++i)
        CK(cudaMemcpyAsync(s->X + (int64_t)i * s->ld, d + (size_t)i * s->n, sizeof(double) * s->n,
                           cudaMemcpyHostToDevice, s->st));
    d += (size_t)h.win_count * s->n;
    for (int i = 0; i < h.k_cur; ++i)
        CK(cudaMemcpyAsync(s->U + (int64_t)i * s->ld, d + (size_t)i * s->n, sizeof(double) * s->n,
                           cudaMemcpyHostToDevice, s->st));
    d += (size_t)h.k_cur * s->n;
    for (int j = 0; j < h.win_count && h.gram; ++j)
        CK(cudaMemcpyAsync(s->gwin + (int64_t)j * RGM_WMAX, d + (size_t)j * h.win_count,
                           sizeof(double) * h.win_count, cudaMemcpyHostToDevice, s->st));
    d += (size_t)h.gram * h.win_count * h.win_count;
    for (int j = 0; j < h.phi_c; ++j)
        CK(cudaMemcpyAsync(s->sm->phi + (int64_t)j * RGM_WMAX, d + (size_t)j * h.phi_c,
                           sizeof(double) * h.phi_c, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(&s->sm->phi_c, &h.phi_c, sizeof(int), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    s->gwin_valid = h.gram != 0;
    s->win_last = -1;
    s->win_count = h.win_count;
    s->win_head = h.win_head;
    s->updates = (int)h.updates;
    s->k_cur = h.k_cur;
    s->k_pending = false;
    s->coarse_stale = true;
    return RGM_OK;
}

int rgm_wait_selftest(int64_t limit_ns, int *blocks_gave_up, int *fault_flag)
{
    if (limit_ns < 1000 || limit_ns > 1000000000 || !blocks_gave_up || !fault_flag) return RGM_E_ARG;
    Small *sm = nullptr;
    int *cnt = nullptr;
    cudaError_t e = cudaMalloc((void **)&sm, sizeof(Small));
    if (e == cudaSuccess) e = cudaMalloc((void **)&cnt, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(sm, 0, sizeof(Small));
    if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(int));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<2, RGM_THREADS>>>(sm, (unsigned long long)limit_ns, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    Small h;
    int c = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&c, cnt, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h, sm, offsetof(Small, H), cudaMemcpyDeviceToHost);
    cudaFree(sm);
    cudaFree(cnt);
    if (e != cudaSuccess) return RGM_E_CUDA;
    *blocks_gave_up = c;
    *fault_flag = h.fault ? 1 : 0;
    return RGM_OK;
}

// Library-internal: the solver's device value buffer (for in-library producers
// such as the FE workload) and a copy of its configuration.
int rgm_solver_device_bytes(rgm_solver s, int64_t *bytes)
{
    if (!s || !bytes) return RGM_E_ARG;
    int64_t b = 0;
    for (const auto &a : s->allocs) b += (int64_t)a.second;
    *bytes = b;
    return RGM_OK;
}

int rgm_internal_nnz(rgm_solver s, int64_t *nnz)
{
    if (!s || !nnz) return RGM_E_ARG;
    if (!s->have_op) return RGM_E_STATE;
    *nnz = s->nnz;
    return RGM_OK;
}

int rgm_internal_config(rgm_solver s, rgm_config *cfg)
{
    if (!s || !cfg) return RGM_E_ARG;
    *cfg = s->cfg;
    return RGM_OK;
}

int rgm_profile(rgm_solver s, int enable)
{
    if (!s) return RGM_E_ARG;
    prof_collect(s);
    for (int i = 0; i < RGM_PROF_KINDS; ++i) s->acc[i] = rgm_kernel_prof{0.0, 0, 0.0, 0.0, 0.0, 0.0};
    s->launches = 0;
    s->prof = enable != 0;
    return RGM_OK;
}

int rgm_profile_read(rgm_solver s, rgm_kernel_prof *out, int nkinds, int64_t *launches)
{
    if (!s || !out || nkinds < 0 || nkinds > RGM_PROF_KINDS) return RGM_E_ARG;
    prof_collect(s);
    for (int i = 0; i < nkinds; ++i) out[i] = s->acc[i];
    if (launches) *launches = s->launches;
    return RGM_OK;
}

int rgm_spmv(rgm_solver s, const double *x, double *y, int flags)
{
    if (!s || !x || !y) return RGM_E_ARG;
    if (!s->have_op) return RGM_E_STATE;
    CK(cudaMemcpyAsync(s->r, x, sizeof(double) * s->n, kind_in(flags), s->st));
    Arnoldi<double> a = arn64(s);
    VecOp<double> op = base_op(s, a);
    op.src = SRC_SPMV;
    op.x = s->r;
    op.out = s->w;
    int rc = launch(s, op);
    if (rc) return rc;
    if (s->dvec) {   // the stored operator is D^{-1} A
        ProfScope ps_(s, RGM_PROF_OTHER, (double)s->n, 24.0 * (double)s->n);
        diag_apply_kernel<<<s->nblocks, 256, 0, s->st>>>(s->w, s->dvec, s->n, 0);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(y, s->w, sizeof(double) * s->n, kind_out(flags), s->st));
    CK(cudaStreamSynchronize(s->st));
    return RGM_OK;
}

}  // extern "C"
