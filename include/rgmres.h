/*
 * rgmres.h -- C ABI of librgmres: recycled GMRES(m) for sequences of linear
 * systems on one NVIDIA GB300 (sm_103a).
 *
 * Method: Pitton & Heltai, "Accelerating the iterative solution of
 * convection-diffusion problems using singular value decomposition"
 * (arXiv 1807.09467).  A sequence A_i x_i = b_i arrives one system at a time
 * (Sec. 2, the systems depend on the previous solution); each is solved by
 * restarted GMRES (Sec. 3) accelerated by a recycle space U, the leading left
 * singular vectors of a window of previous solutions (Sec. 5.2, Algorithm 1),
 * used to deflate (Sec. 3.2) or to augment (Sec. 3.1) the Krylov space.
 *
 * Conventions for every entry point:
 *  - Return value: RGM_OK (0), a positive warning (the call completed) or a
 *    negative error (nothing was changed unless stated).  rgm_status_string
 *    gives the text.
 *  - Pointers are host pointers unless `flags` contains RGM_DEVICE_PTRS, in
 *    which case they are device pointers of the current CUDA device, read or
 *    written in order on the solver's stream.
 *  - The caller owns every array it passes; the library copies what it keeps.
 *    The solver handle owns all device state (operator, Krylov basis, recycle
 *    space, snapshot window, scratch) and frees it in rgm_solver_destroy.
 *  - Dense arrays are column-major with the stated leading dimension.  CSR
 *    uses int64 row pointers and int32 column indices.
 *  - Calls on one handle must not overlap; distinct handles are independent.
 *  - Nothing falls back to the CPU: without a usable CUDA device every call
 *    that needs one returns RGM_E_CUDA.
 */
#ifndef RGMRES_H
#define RGMRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define RGM_OK                  0
#define RGM_W_NOT_CONVERGED     1   /* maxit reached; x holds the last iterate            */
#define RGM_W_SINGULAR_COARSE   2   /* E = U^T A U singular: this solve ran plain GMRES
                                       (the paper takes no measure, Sec. 5.2 end)          */
#define RGM_E_ARG             (-1)  /* invalid argument                                    */
#define RGM_E_OOM             (-2)  /* device allocation failed                            */
#define RGM_E_CUDA            (-3)  /* CUDA runtime error (no device, launch failure, ...) */
#define RGM_E_STATE           (-4)  /* call out of order (e.g. solve before an operator)   */
#define RGM_E_TIMEOUT         (-5)  /* a bounded device wait gave up                       */

#define RGM_DEVICE_PTRS         1   /* flag: pointers are device pointers                  */
#define RGM_BATCH_COOP          2   /* flag of rgm_batch_solve: batched cycle launches     */
#define RGM_ZERO_GUESS          4   /* flag of rgm_solve / rgm_batch_solve: x_in = 0 (x is
                                       output only; b - A x_in = b needs no SpMV)            */

/* ---------------------------------------------------------------- config */
typedef enum {
    RGM_PLAIN = 0,       /* GMRES(m), Sec. 1 / Sec. 3                                       */
    RGM_DEFLATED = 1,    /* Table 1 "deflated oblique": operator P A, start P r,
                            P = I - A U E^{-1} U^T (Eq. left_deflation), plus the coarse
                            correction x += U E^{-1} U^T (b - A x) after each cycle          */
    RGM_AUGMENTED = 2,   /* Sec. 3.1: search space K_j(A, r) + span U, constraint space A S  */
    RGM_GUESS = 3        /* Sec. 4.2 alone: the projection initial guess
                            x0 = x_in + U E^{-1} U^T (b - A x_in), then GMRES(m) on A       */
} rgm_mode;

typedef enum {
    RGM_FP64 = 0,        /* every step in binary64                                          */
    RGM_FP32_IR = 1      /* GMRES-IR: binary32 Arnoldi/SpMV/projections inside a binary64
                            refinement loop (residual, Hessenberg, E and SVD stay binary64)  */
} rgm_precision;

typedef enum {
    RGM_PROJ_OBLIQUE = 0,    /* P = I - W E^{-1} U^T, W = A U, E = U^T W (Table 1 oblique)      */
    RGM_PROJ_ORTHOGONAL = 1, /* P = I - U (U^T U)^{-1} U^T (Table 1 orthogonal, Eq. P_A_variant);
                                each cycle ends with the projection correction
                                x += U E^{-1} U^T (b - A x) (Eq. augmented_iterate)           */
    RGM_PROJ_LS = 2          /* P = I - W (W^T W)^{-1} W^T (Table 1 LS); cycle-end correction
                                x += U (W^T W)^{-1} W^T (b - A x), so I - A Q = P            */
} rgm_projector;

typedef enum {
    RGM_PRECOND_NONE = 0,
    RGM_PRECOND_JACOBI = 1   /* left Jacobi, M = diag(A): GMRES on D^{-1} A x = D^{-1} b (a
                                rows without a nonzero diagonal keep weight 1); the in-cycle
                                exit compares the preconditioned estimate with
                                rtol ||D^{-1} b||, the stopping test stays on the true
                                residual ||b - A x|| <= rtol ||b||.  Binary64 solves only. */
} rgm_precond;

typedef enum {
    RGM_LAUNCH_AUTO = 0,     /* the Arnoldi steps of a cycle run in one cooperative launch
                                (grid barriers between the fused passes) when the grid fits
                                on the device at once and a block owns at most two 256-row
                                tiles; otherwise one launch per pass                        */
    RGM_LAUNCH_PER_PASS = 1  /* one launch per fused pass (same arithmetic)                 */
} rgm_launch_policy;

typedef struct {
    int64_t n;            /* system size (fixed for the handle's life)                      */
    int m;                /* restart length, 1..64                                          */
    int k;                /* recycle dimension s of Algorithm 1, 0..32                      */
    int window;           /* snapshots kept (m of Algorithm 1), k..64                       */
    int svd_interval;     /* ell of Algorithm 1 (>= 1)                                      */
    int select_smallest;  /* 1: keep the trailing singular modes instead of the leading    */
    int mode;             /* rgm_mode                                                       */
    int precision;        /* rgm_precision                                                  */
    int start_r;          /* deflated mode only: 1 = start vector r (Table 1 aug. oblique) */
    int maxit;            /* cap on Arnoldi steps per solve                                 */
    int inner_cycles;     /* FP32_IR: GMRES cycles per refinement                           */
    int max_refinements;  /* FP32_IR: cap on refinement steps                               */
    int launch_policy;    /* rgm_launch_policy                                              */
    int proj;             /* deflated mode: rgm_projector of the Krylov operator P A       */
    int guess;            /* 0: solve from the x passed in; g = 1..3: replace it by the
                             extrapolation of order g (Sec. 4.1, Eq. ext2..ext4) from the
                             g+1 most recent window snapshots once the window holds them
                             (needs window >= g+1); recycling then adds its projection  */
    int precond;          /* rgm_precond (not with RGM_FP32_IR)                              */
    int tiles_per_block;  /* rows each block of the fused passes owns, in 256-row tiles; 0 =
                             automatic (the fewest tiles that keep the grid within the
                             blocks the device holds at once).  Not in the paper: a launch-
                             shape knob for the batched form's autotuner (more tiles a block
                             = fewer blocks a system, so more systems share the device).  A
                             value above the tile count is clamped to it                  */
    double rtol;          /* converged when ||b - A x||_2 <= rtol ||b||_2                   */
    double inner_rtol;    /* FP32_IR: inner solve to max(inner_rtol ||r||, rtol ||b|| / 2)  */
    double rel_drop;      /* drop singular values below rel_drop * sigma_1                 */
    void *cuda_stream;    /* cudaStream_t to run on; NULL = the legacy default stream      */
} rgm_config;

typedef struct {
    int iters;            /* Arnoldi steps (operator applications to basis vectors)         */
    int cycles;           /* GMRES cycles                                                   */
    int refinements;      /* FP32_IR refinement steps                                       */
    int k_used;           /* recycle columns used by this solve                             */
    int status;           /* same code the call returned                                    */
    double true_relres;   /* ||b - A x||_2 / ||b||_2 of the returned x, in binary64         */
} rgm_stats;

typedef struct rgm_solver_s *rgm_solver;

/* Fill *cfg with defaults: m 30, k 8, window 16, ell 1, deflated, FP64,
 * rtol 1e-10, maxit 20000, inner_rtol 1e-4, inner_cycles 2, rel_drop 1e-7. */
int rgm_config_default(rgm_config *cfg);

/* Text of the CUDA error behind the last RGM_E_CUDA or RGM_E_OOM returned on
 * the calling thread (error name, message, failing call); "" if none.  The
 * string belongs to the library and stays valid until the thread's next
 * failing call. */
const char *rgm_last_error(void);

/* Create a solver for systems of size cfg->n on the current device.  Allocates
 * the Krylov basis (n x (m+k+1)), the recycle space and the snapshot window.
 * Errors: RGM_E_ARG (limits above), RGM_E_OOM, RGM_E_CUDA. */
int rgm_solver_create(rgm_solver *out, const rgm_config *cfg);
int rgm_solver_destroy(rgm_solver s);

/* Operator A (n x n) in CSR (Sec. 2, Eq. algebra_pde).  Sets pattern and values;
 * the pattern may change between calls.  Invalidates A U and E.  Column indices
 * must lie in [0, n); rows need not be sorted.  Errors: RGM_E_ARG, RGM_E_OOM. */
int rgm_set_operator_csr(rgm_solver s, int64_t n, int64_t nnz, const int64_t *rowptr,
                         const int32_t *col, const double *val, int flags);
/* Operator A (n x n) in the library's own layout, sliced ELL with 32-row slices
 * (SELL-32-sigma with sorting windows inside 256-row tiles), as the kernels read
 * it.  nslices = 8 * ceil(n / 256); slice q holds slice rows 32q .. 32q + 31.
 *  - perm (nslices * 32 int32): matrix row of each slice row, or -1 for padding;
 *    every matrix row appears exactly once, and the slice rows of tile t
 *    (slices 8t .. 8t + 7) map to matrix rows 256t .. 256t + 255.
 *  - slice_ptr (nslices + 1 int64): slice_ptr[0] = 0, each slice's size a
 *    multiple of 32; entry j of lane l of slice q sits at slice_ptr[q] + 32 j + l.
 *  - col, val (nsell = slice_ptr[nslices] entries): padding entries need a
 *    column in [0, n) and value 0.
 * Slices sorted by width inside a tile run fastest (the kernels balance warps on
 * that order).  After this call rgm_set_operator_values takes nsell values in
 * this layout.  Errors: RGM_E_ARG (any rule above), RGM_E_OOM, RGM_E_CUDA. */
int rgm_set_operator_sell(rgm_solver s, int64_t n, int64_t nslices, const int64_t *slice_ptr,
                          const int32_t *perm, const int32_t *col, const double *val, int flags);
/* New values on the pattern of the last rgm_set_operator_csr (nnz doubles, same
 * order) or rgm_set_operator_sell (nsell doubles, that layout).  This is the
 * per-time-step call of Sec. 2: A_i = A(t_i, x_{i-1}). */
int rgm_set_operator_values(rgm_solver s, const double *val, int flags);

/* Recycle space U (n x k, leading dimension ld >= n) set by the caller instead
 * of by rgm_update_recycle_svd.  Columns should be linearly independent; the
 * library uses them as given (no re-orthonormalisation).  k = 0 clears it. */
int rgm_set_recycle_space(rgm_solver s, const double *U, int k, int64_t ld, int flags);
/* Copy the current recycle space out (n x k_used, leading dimension ld); *k
 * receives k_used.  U may be NULL to query *k only. */
int rgm_get_recycle_space(rgm_solver s, double *U, int64_t ld, int *k, int flags);

/* Solve A x = b.  x: in = x_in, out = solution.  With a recycle space the solve
 * starts from x0 = x_in + U E^{-1} U^T (b - A x_in) (Sec. 4.2, Eq.
 * projection_t_s; the paper's x0 = U E^{-1} U^T b is x_in = 0).  With
 * RGM_ZERO_GUESS in flags x_in = 0 and x is not read (the result is the same
 * as passing zeros; the first residual b - A x_in = b then costs no SpMV).
 * st may be NULL.  Returns RGM_OK, RGM_W_NOT_CONVERGED or
 * RGM_W_SINGULAR_COARSE (x valid in all three), or an error. */
int rgm_solve(rgm_solver s, const double *b, double *x, int flags, rgm_stats *st);

/* Algorithm 1 after a solve: append x (n doubles) to the snapshot window (the
 * oldest column leaves when `window` are stored); if the number of calls so far
 * is a multiple of svd_interval, replace U by the k leading (or trailing) left
 * singular vectors of the window (Sec. 5.2), dropping singular values below
 * rel_drop * sigma_1.  *k_used (may be NULL) receives the new dimension, which
 * makes the call wait for the device; with k_used NULL and RGM_DEVICE_PTRS the
 * work is only queued on the solver's stream (the next call on the handle
 * picks up the new dimension).  With host pointers the call returns after x
 * has been read. */
int rgm_update_recycle_svd(rgm_solver s, const double *x, int flags, int *k_used);

/* Batched solve: nsys independent systems, system i on handle handles[i], solved
 * concurrently (the batched and served forms: the sequences of a batch are
 * independent problems).  Handles must be distinct and should have distinct
 * streams (solves on one stream serialise).  b[i], x[i] and flags as in
 * rgm_solve; st (optional) receives nsys entries.  Returns the first error if
 * any solve failed (rgm_last_error then describes it), else the largest
 * warning, else RGM_OK.
 *
 * Without RGM_BATCH_COOP each handle's work is queued on its own stream from a
 * pool of host threads, one launch per fused pass (no cooperative cycle kernel:
 * cooperative grids on concurrent streams are not guaranteed to be resident
 * together).  With RGM_BATCH_COOP (all handles in one precision, launch policy
 * auto, a device with cooperative launch; otherwise the flag is ignored) every
 * system runs on a host thread of its own and, at each GMRES cycle, waits until
 * all systems still solving have reached theirs; their cycles then run as one
 * cooperative launch of batch_cycle_kernel on a stream of the batch, each
 * system on a block range of its own (its usual block count when all fit, else
 * one block plus a share of the resident capacity in proportion to its work per
 * Arnoldi step).  Results then equal the handle's own solve up to the rounding
 * of its dot-product partition: bit for bit when the system kept its block
 * count, within rounding otherwise; a batch repeats bit for bit. */
int rgm_batch_solve(rgm_solver *handles, int nsys, const double *const *b, double *const *x, int flags,
                    rgm_stats *st);

/* The block plan of one batched cycle launch of rgm_batch_solve(.., RGM_BATCH_COOP,
 * ..), host only (no device work; for inspection and tests).  Inputs, one entry
 * per system in the order of the launch: n rows, nnz stored entries, nd dot
 * columns of an Arnoldi pass, want the blocks of the system's own partition;
 * cap the co-resident blocks of the launch.  Systems run in waves of at most
 * cap consecutive systems.  In a wave whose wants add up to more than cap,
 * system i gets min(want[i], 1 + floor((cap - size) * w_i / sum w)) blocks,
 * w = nnz + n * nd, each block a run of whole 256-row tiles.  Outputs (caller
 * owned, nsys entries): blocks[i] the block count, rpb[i] its rows per block
 * (0: the system keeps its own partition, blocks[i] == want[i]), wave[i] its
 * wave.  Returns the number of waves, or RGM_E_ARG (nsys < 0, cap < 1, a
 * missing array, n < 1, nnz < 0, nd < 0 or want < 1). */
int rgm_batch_plan(int nsys, const int64_t *n, const int64_t *nnz, const int *nd, const int *want, int cap,
                   int *blocks, int *rpb, int *wave);
/* Singular values of the last window SVD, descending (up to `window` values);
 * *count receives how many are valid. */
int rgm_get_singular_values(rgm_solver s, double *sigma, int *count);

/* Clear the snapshot window and the recycle space (and the eigenvectors the
 * next window SVD would start from). */
int rgm_reset_recycling(rgm_solver s);

/* Checkpoint / resume of the recycling state that Algorithm 1 carries from
 * one system of the sequence to the next: the snapshot window (its stored
 * columns, ring position, update count and the window Gram matrix that the
 * next update extends by one column), the recycle space U, and the
 * eigenvectors of the last window Gram matrix, which the next window SVD's
 * Jacobi rotations start from (consecutive windows differ by one column, so
 * they nearly diagonalise the next Gram matrix; the eigenpairs are unchanged,
 * only their rounding depends on the start, hence their place in the state).
 * Buffers written before the eigenvectors were part of the state are still
 * accepted (the next SVD then starts from the identity).  Not
 * described in the paper; it lets a sequence continue in a new handle or a
 * new process with results identical to the uninterrupted run.  The operator
 * is not part of the state (each step sets its own), nor are the singular
 * values of the last update.
 *
 * rgm_export_state: with buf == NULL, *bytes receives the size needed; else
 * *bytes must hold buf's capacity, the state is written to buf (host memory,
 * native byte order) and *bytes receives the size written.  Waits for the
 * handle's stream.  RGM_E_ARG if the capacity is too small.
 * rgm_import_state: buf/bytes as written by rgm_export_state for a handle
 * with the same n, window and k >= the stored recycle dimension; RGM_E_ARG
 * otherwise (the handle is then unchanged).  The next solve rebuilds
 * W = A U and E from the operator it is given. */
int rgm_export_state(rgm_solver s, void *buf, size_t *bytes);
int rgm_import_state(rgm_solver s, const void *buf, size_t bytes);

/* y = A x with the solver's operator (the SpMV of every Arnoldi step). */
int rgm_spmv(rgm_solver s, const double *x, double *y, int flags);

const char *rgm_status_string(int code);

/* ------------------------------------------------------------ measurement
 * Per-launch CUDA-event timing of the solver's kernels on its stream, grouped
 * by kind, with the algorithmic work of each launch (flops and bytes the
 * method must compute and move; not the hardware traffic).  Not part of the
 * method; used to place kernels on the roofline. */
#define RGM_PROF_ARNOLDI_SPMV 0   /* SpMV A v_j + dots with [U|V] (first pass)   */
#define RGM_PROF_ARNOLDI_CGS1 1   /* AXPY of the first Gram-Schmidt pass + dots  */
#define RGM_PROF_ARNOLDI_CGS2 2   /* AXPY of the second pass + norm              */
#define RGM_PROF_OTHER        3   /* residuals, start vectors, coarse, updates   */
#define RGM_PROF_GRAM         4   /* Gram matrices (E, snapshot window, CholQR)  */
#define RGM_PROF_SMALL        5   /* single-block scalar kernels                 */
#define RGM_PROF_ARNOLDI_CYCLE 6  /* all Arnoldi steps of a cycle in one cooperative
                                     launch (RGM_LAUNCH_AUTO)                       */
#define RGM_PROF_SVD          7   /* U = X C combinations of the window SVD          */
#define RGM_PROF_COARSE       8   /* W = A U and the binary32 copy of U              */
#define RGM_PROF_OPERATOR     9   /* new operator values into the sliced ELL         */
#define RGM_PROF_KINDS        10

typedef struct {
    double ms;          /* summed device time of the launches                */
    int64_t launches;
    double flops;       /* summed algorithmic floating-point operations      */
    double bytes;       /* summed algorithmic bytes read and written         */
    double units;       /* Arnoldi steps the launches carried out (Arnoldi kinds; 0 otherwise) */
    double step_bytes;  /* algorithmic bytes of those Arnoldi steps, B_j summed (below) */
} rgm_kernel_prof;
/* bytes: what each launch's passes read and write once (the vectors a pass
 * produces and the columns it reads, the operator for a SpMV).  step_bytes:
 * what an Arnoldi step j (1-based; j basis vectors before it) must move at
 * least -- the operator once, the basis once, 2 k recycle columns when k
 * deflate and about four vector streams (w, the new basis vector, the SpMV
 * input and output):
 *     B_j = (e + 4) nnz + e n (j + 2 k + 4),   e = 8 (binary64) or 4 (binary32),
 * booked on the cycle kind and on the first pass of each step (the SpMV kind).
 * Flops: 2 per stored nonzero and 2 per row per dot or AXPY column of every
 * pass. */

/* Device memory the handle holds now: the sum of its device allocations
 * (operator in sliced ELL, Krylov basis, recycle space, snapshot window,
 * binary32 copies, scratch), in bytes.  RGM_E_ARG for a NULL argument. */
int rgm_solver_device_bytes(rgm_solver s, int64_t *bytes);

/* Reset the counters and switch event timing on (1) or off (0). */
int rgm_profile(rgm_solver s, int enable);
/* Synchronise the stream and copy the per-kind totals out (nkinds entries);
 * *launches receives every kernel launch since the last reset. */
int rgm_profile_read(rgm_solver s, rgm_kernel_prof *out, int nkinds, int64_t *launches);

/* ------------------------------------------------------------ bounded-wait self-test
 * Not part of the method.  The cooperative cycle kernel (RGM_LAUNCH_AUTO)
 * separates its passes by grid barriers whose waits are bounded: a block that
 * waits longer than its limit sets a fault flag and returns, and the solve
 * reports RGM_E_TIMEOUT instead of hanging.  This call exercises exactly that
 * path on the current device: it launches two blocks that wait at such a
 * barrier for a generation nothing ever publishes, with the wait limit
 * limit_ns (1e3 .. 1e9 ns), synchronises, and sets *blocks_gave_up (blocks
 * whose wait ended without the release: 2 when the limit works) and
 * *fault_flag (the device-side fault flag: 1).  Allocates and frees a few
 * hundred KB of device memory; RGM_E_ARG for bad arguments, RGM_E_CUDA on a
 * CUDA error. */
int rgm_wait_selftest(int64_t limit_ns, int *blocks_gave_up, int *fault_flag);

/* ------------------------------------------------------------ allocation-free check
 * The paper has no counterpart to this entry point: it serves callers that
 * cannot allocate device memory (a host framework that owns the allocator, a
 * latency-critical path that must not synchronise on an allocation, a check
 * that must run after memory is exhausted) and so cannot create an rgm_solver.
 *
 * r = b - A x and norms[0] = ||b - A x||_2, norms[1] = ||b||_2 for an n x n CSR
 * matrix.  Every pointer is a device pointer of the current device (r may be
 * NULL): rowptr n+1 int64 entries (rowptr[0] = 0, non-decreasing), col and val
 * rowptr[n] entries (int32, binary64), x, b and r n binary64 entries; r must
 * not alias x or b (it is written while other blocks still read them).  The
 * C entry point cannot check types or extents behind a pointer: an int32
 * rowptr read as int64, for instance, sends the kernel to offsets outside the
 * buffers, so a binding must check them (the Python binding does).  The work
 * is queued on cuda_stream (NULL = legacy default stream) and the call returns
 * without waiting.  Nothing is allocated: the scratch (per-
 * block partial sums and a completion counter) is one static device array of
 * 2 * RGM_NOALLOC_MAX_BLOCKS + 32 doubles that every GPU loading the library
 * holds until exit.  The first call on a device looks its address up once
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array: calls that overlap on
 * the GPU race and give wrong results.  A column index outside [0, n) makes the
 * norms NaN (it is never dereferenced).
 * Errors: RGM_E_ARG for a NULL pointer, n < 1 or n > RGM_NOALLOC_MAX_BLOCKS *
 * RGM_NOALLOC_ROWS_PER_BLOCK (8,388,608 rows); RGM_E_CUDA otherwise. */
#define RGM_NOALLOC_MAX_BLOCKS 4096
#define RGM_NOALLOC_ROWS_PER_BLOCK 2048
int rgm_residual_noalloc(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                         const double *x, const double *b, double *r, double *norms,
                         void *cuda_stream);

/* ------------------------------------------------------------ FE workload
 * The time-step systems of Sec. 6.1 built on the device: Q_p Lagrange elements
 * (p = 1..RGM_FE_MAX_P, Gauss-Lobatto nodes; high p on a coarse grid is the
 * spectral-element discretisation of the paper's Table 4, order 23 on 2 x 2
 * elements) on a uniform N x N grid of the unit square,
 * (p+1)^2 Gauss points per cell, implicit Euler with the convection coefficient
 * lagged one step,
 *   A = M/dt + eps K + N(u_prev; beta),  b = M u_prev / dt + F(f = 1),
 * N_ij = (u_prev beta . grad phi_j, phi_i) (beta constant, or the paper's
 * cellular field, rgm_fe_set_velocity; f = 1 or the paper's random modes,
 * rgm_fe_set_forcing), homogeneous Dirichlet rows
 * (identity, b_i = 0), boundary columns dropped from interior rows.
 * Dofs are numbered lexicographically (x fastest) on the (pN+1)^2 lattice.
 * This is the workload the solver is measured on, not part of the method.  */
typedef struct rgm_fe_s *rgm_fe;
#define RGM_FE_MAX_P 32

int rgm_fe_create(rgm_fe *out, int p, int N, double eps, double dt, double beta_x,
                  double beta_y, void *cuda_stream);
int rgm_fe_destroy(rgm_fe fe);
/* Sizes of the Dirichlet pattern. */
int rgm_fe_sizes(rgm_fe fe, int64_t *n, int64_t *nnz);
/* Device memory the workload holds now (pattern, element tables, values,
 * right-hand side, for p <= 4 the per-cell matrices, velocity and forcing
 * fields when set), in bytes. */
int rgm_fe_device_bytes(rgm_fe fe, int64_t *bytes);
/* Copy the Dirichlet CSR pattern out (rowptr n+1, col nnz). */
int rgm_fe_pattern(rgm_fe fe, int64_t *rowptr, int32_t *col, int flags);
/* Assemble values (nnz, CSR order of rgm_fe_pattern) and b (n) from u_prev (n).
 * Every value is gathered row by row in a fixed order of the cells (no
 * atomics), so repeated assemblies give the same bits.  Host pointers (flags
 * 0) or device pointers (RGM_DEVICE_PTRS); synchronises the handle's stream. */
int rgm_fe_assemble(rgm_fe fe, const double *u_prev, double *val, double *b, int flags);
/* Velocity of the convection term (Sec. 6.1).  RGM_FE_VELOCITY_CONSTANT: the
 * (beta_x, beta_y) given at creation.  RGM_FE_VELOCITY_CELLULAR: the paper's
 * solenoidal field b = (-sin(pi x) cos(pi y), cos(pi x) sin(pi y)) through its
 * nodal interpolant (P_{V_h} b), N_ij = (u_prev b_h . grad phi_j, phi_i).
 * Returns RGM_E_ARG for another kind; device memory for the field (3 vectors
 * of the cell quadrature size) is owned by the handle.  Synchronises. */
typedef enum { RGM_FE_VELOCITY_CONSTANT = 0, RGM_FE_VELOCITY_CELLULAR = 1 } rgm_fe_velocity;
int rgm_fe_set_velocity(rgm_fe fe, int kind);
/* Forcing of the load (v, f) (Sec. 6.1):
 *   f = (C/2) sum_{j=1..nmodes} c_j exp(-j^2/20) sin(2 j pi x) sin(2 j pi y)
 * through its nodal interpolant f_h, so the load is M f_h (the paper: C = 0.1,
 * 16 modes, c_1 = 1 and c_2..c_16 drawn from U[-1, 1] at every step).  c: nmodes
 * coefficients (c[0] = c_1), host or device memory by flags; with
 * RGM_DEVICE_PTRS the call is asynchronous on the handle's stream.  nmodes = 0
 * restores f = 1.  RGM_E_ARG for nmodes outside 0..RGM_FE_MAX_MODES or a null c.
 * The forcing applies to every later assembly until changed. */
#define RGM_FE_MAX_MODES 64
int rgm_fe_set_forcing(rgm_fe fe, int nmodes, const double *c, double C, int flags);
/* Nodal interpolant of u0 = sum_{j=1..8} a_j sin(j pi x) sin(j pi y), zero on the
 * boundary.  a8 is a host array of 8 doubles. */
int rgm_fe_initial_field(rgm_fe fe, const double *a8, double *u0, int flags);
/* One time step on the device: assemble from u_prev, rgm_set_operator_values,
 * rgm_solve with x_in as Algorithm 1 prescribes (0 with a recycle space, u_prev
 * without), then rgm_update_recycle_svd.  u (device, n) holds u_prev on entry
 * and the new solution on return.  The solver must have been given the FE
 * pattern by rgm_set_operator_csr. */
int rgm_fe_time_step(rgm_fe fe, rgm_solver s, double *u_dev, rgm_stats *st);

#ifdef __cplusplus
}
#endif
#endif
