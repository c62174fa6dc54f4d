/*
 * oracle.h -- plain, slow, FP64 CPU oracle for recycled GMRES(m) over a sequence
 * of implicitly time-stepped, linearised convection-diffusion systems
 * (Pitton & Heltai, "Accelerating the iterative solution of convection-diffusion
 * problems using singular value decomposition", arXiv 1807.09467).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path loads, links or calls
 * this code: only the tests, the smoke check of the package entry module and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library; the two meet only through seeded
 * inputs made by the `synth` module.
 *
 * Every routine is written from the paper's definitions, in the paper's order,
 * with no blocking or fusion:
 *   fe.c       Sec. 2 (Eq. linear_pde, def_Axb) and Sec. 6.1 (discrete problem)
 *   gmres.c    Sec. 3 (Eq. x_k_expression; GMRES = C_k = A S_k), Sec. 3.1
 *              (augmentation, Eq. def_aug_S_space), Sec. 3.2 (deflation,
 *              Eq. left_deflation), Sec. 3.3 / Table 1 (projectors), Sec. 4.2
 *              (projection initial guess, Eq. projection_t_s)
 *   svd.c      Sec. 5.2 (Eq. best_rank_s, opt_svd) and Algorithm 1
 *   sequence.c Algorithm 1 driving Sec. 2's time-step sequence
 * All dense arrays are column-major; CSR uses int64 row pointers and int32
 * column indices with ascending columns in each row.
 */
#ifndef RGMRES_ORACLE_H
#define RGMRES_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- status codes ---------------- */
#define ORC_OK                 0
#define ORC_W_NOT_CONVERGED    1   /* maxit reached; x holds the last iterate   */
#define ORC_W_SINGULAR_COARSE  2   /* E = U^T A U singular: solve ran plain     */
#define ORC_E_ARG            (-1)
#define ORC_E_PATTERN        (-2)  /* an assembled entry is outside the pattern */
#define ORC_E_NOMEM          (-3)

/* ---------------- 1D building blocks (fe.c) ---------------- */
int orc_gll_nodes(int p, double *xi);                 /* p+1 Gauss-Lobatto nodes on [0,1] */
int orc_gauss_rule(int q, double *x, double *w);      /* q-point Gauss-Legendre on [0,1]  */
int orc_lagrange(int p, const double *nodes, double x, double *phi, double *dphi);

/* ---------------- FE system of Sec. 6.1 on N x N quads, Q_p (fe.c) ---------------- */
int64_t orc_fe_ndofs(int p, int N);
int orc_fe_node_coords(int p, int N, double *x, double *y);
/* CSR pattern.  dirichlet=0: every pair of dofs sharing an element.
 * dirichlet=1: boundary rows keep only the diagonal, interior rows drop boundary
 * columns.  Returns nnz; rowptr/col may be NULL to query the size only. */
int64_t orc_fe_pattern(int p, int N, int dirichlet, int64_t *rowptr, int32_t *col);
/* val = cm*M + ck*K + cn*N(u; beta) on the given pattern (full or Dirichlet).
 * M_ij = (phi_j, phi_i), K_ij = (grad phi_j, grad phi_i),
 * N_ij = (u beta . grad phi_j, phi_i), u = sum_l u_l phi_l.
 * With dirichlet=1 the boundary rows are set to the identity. */
int orc_fe_assemble(int p, int N, double cm, double ck, double cn, double bx, double by,
                    const double *u, int dirichlet, const int64_t *rowptr,
                    const int32_t *col, double *val);
/* F_i = (f, phi_i) by the (p+1)^2 Gauss rule; f == NULL means f = 1. */
typedef double (*orc_scalar_fn)(double x, double y, void *ctx);
int orc_fe_load(int p, int N, orc_scalar_fn f, void *ctx, double *F);
/* One implicit-Euler step with the lagged (Picard) coefficient:
 *   A = M/dt + eps K + N(u_prev; beta),  b = M u_prev / dt + F(f = 1),
 * then homogeneous Dirichlet rows (identity, b_i = 0). */
int orc_fe_step_system(int p, int N, double eps, double dt, double bx, double by,
                       const double *u_prev, const int64_t *rowptr, const int32_t *col,
                       double *val, double *b);
/* As orc_fe_assemble with the velocity given by nodal values (bxn, byn; n
 * each), interpolated at the quadrature points by the element basis. */
int orc_fe_assemble_field(int p, int N, double cm, double ck, double cn, const double *bxn,
                          const double *byn, const double *u, int dirichlet,
                          const int64_t *rowptr, const int32_t *col, double *val);
/* Sec. 6.1's benchmark step: A = M/dt + eps K + N(u_prev; b_h) with the nodal
 * velocity (bxn, byn), b = M u_prev / dt + M fn (fn: nodal forcing; NULL
 * means (v, 1) as in orc_fe_step_system), Dirichlet rows as there. */
int orc_fe_step_system_field(int p, int N, double eps, double dt, const double *bxn,
                             const double *byn, const double *fn, const double *u_prev,
                             const int64_t *rowptr, const int32_t *col, double *val, double *b);
/* Sec. 6.1: b = (-sin(pi x) cos(pi y), cos(pi x) sin(pi y)) at the nodes. */
int orc_fe_paper_velocity(int p, int N, double *bxn, double *byn);
/* Sec. 6.1: f = (C/2) sum_{j=1..nmodes} c_j exp(-j^2/20) sin(2 j pi x) sin(2 j pi y)
 * at the nodes (the paper: C = 0.1, 16 modes, c_1 = 1, c_j ~ U[-1,1] per step). */
int orc_fe_paper_forcing(int p, int N, int nmodes, const double *c, double C, double *fn);
/* Nodal interpolant of u0 = sum_{j=1..8} a_j sin(j pi x) sin(j pi y), zero on the boundary. */
int orc_fe_u0(int p, int N, const double *a8, double *u0);

/* ---------------- GMRES(m) and recycling (gmres.c) ---------------- */
typedef struct {
    int64_t n;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
} orc_csr;

#define ORC_PLAIN      0   /* GMRES(m)                                            */
#define ORC_DEFLATED   1   /* deflated oblique, Table 1 row 5, + coarse correction */
#define ORC_AUGMENTED  2   /* Sec. 3.1: S = K_m(A, r) + span U, C = A S            */
#define ORC_GUESS      3   /* Sec. 4.2: projection initial guess, then GMRES(m)   */

/* Projector of the ORC_DEFLATED family (Table 1): the Krylov operator is P A. */
#define ORC_PROJ_OBLIQUE    0   /* P = I - W E^{-1} U^T, W = A U, E = U^T W            */
#define ORC_PROJ_ORTHOGONAL 1   /* P = I - U (U^T U)^{-1} U^T (Eq. P_A_variant)       */
#define ORC_PROJ_LS         2   /* P = I - W (W^T W)^{-1} W^T                          */

typedef struct {
    int mode;          /* ORC_PLAIN / ORC_DEFLATED / ORC_AUGMENTED / ORC_GUESS      */
    int m;             /* restart length                                           */
    double rtol;       /* stop when ||b - A x|| <= rtol ||b||                       */
    int maxit;         /* cap on Arnoldi steps (operator applications)             */
    int start_r;       /* DEFLATED only: 1 = start vector r (Table 1 "augmented"
                          rows), 0 = P r (Table 1 "deflated" rows)                 */
    int proj;          /* DEFLATED only: ORC_PROJ_*                                */
    int precond;       /* ORC_PRECOND_NONE / ORC_PRECOND_JACOBI                    */
} orc_opts;

/* Left Jacobi preconditioning (a GPU-friendly preconditioner in place of the
 * paper's SSOR, whose triangular sweeps are sequential): GMRES on D^{-1} A x = D^{-1} b, D = diag(A) (rows
 * without a nonzero diagonal keep weight 1).  The in-cycle exit compares the
 * Givens estimate of the preconditioned residual with rtol ||D^{-1} b||; the
 * stopping test stays on the true residual ||b - A x|| <= rtol ||b||. */
#define ORC_PRECOND_NONE    0
#define ORC_PRECOND_JACOBI  1

typedef struct {
    int iters;           /* Arnoldi steps summed over cycles                       */
    int cycles;
    int k_used;          /* recycle columns actually used                          */
    int status;
    double true_relres;  /* ||b - A x|| / ||b|| on exit                            */
} orc_stats;

int orc_spmv(const orc_csr *A, const double *x, double *y);
/* W = A U, E = U^T W (k x k, column-major). */
int orc_coarse_setup(const orc_csr *A, const double *U, int k, double *W, double *E);
/* v_out = (I - W E^{-1} U^T) v_in ; returns ORC_W_SINGULAR_COARSE if E is singular. */
int orc_apply_oblique(int64_t n, int k, const double *U, const double *W, const double *E,
                      const double *v_in, double *v_out);
/* v_out = P v_in for the projector proj (ORC_PROJ_*), W = A U given. */
int orc_apply_projector(int64_t n, int k, const double *U, const double *W, int proj,
                        const double *v_in, double *v_out);
/* Solve A x = b.  x: in = x_in, out = solution.  U: n x k (k may be 0).
 * hist (optional, length hist_len): relative residual estimate |g_{j+1}|/||b||
 * after every Arnoldi step, in order. */
int orc_gmres(const orc_csr *A, const double *b, double *x, const double *U, int k,
              const orc_opts *o, orc_stats *st, double *hist, int hist_len);
/* Mixed-precision iterative refinement (GMRES-IR): outer FP64 residual, inner
 * recycled GMRES with every stored vector and A's values rounded to binary32
 * (arithmetic in FP64, rounded on store).  The inner solve stops at
 * max(inner_rtol ||r||, rtol ||b|| / 2) (r the current outer residual) or
 * after inner_cycles cycles. */
int orc_gmres_ir(const orc_csr *A, const double *b, double *x, const double *U, int k,
                 const orc_opts *o, double inner_rtol, int inner_cycles,
                 int max_refinements, orc_stats *st, int *refinements);

/* ---------------- thin SVD of the snapshot window (svd.c) ---------------- */
/* X: n x c.  sigma: c values, descending.  Psi: n x c left singular vectors
 * (columns for sigma_i = 0 are left zero).  Householder QR, then one-sided
 * Jacobi on R. */
int orc_svd_left(int64_t n, int c, const double *X, double *sigma, double *Psi);
/* Same, also returning the right singular vectors Phi (c x c, column i for sigma_i). */
int orc_svd_full(int64_t n, int c, const double *X, double *sigma, double *Psi, double *Phi);
/* Recycle space of Algorithm 1: the k leading left singular vectors of X
 * (or trailing if select_smallest), dropping sigma_i < rel_drop * sigma_1,
 * formed as X phi_i / sigma_i and orthonormalised inside their span.
 * Returns k_eff through *k_eff; U is n x k_eff. */
int orc_recycle_from_window(int64_t n, int c, const double *X, int k, int select_smallest,
                            double rel_drop, double *U, int *k_eff);

/* Extrapolated initial guess (Sec. 4.1, Eq. ext2 / ext3 / ext4): the polynomial
 * of degree s-1 through the s most recent solutions, evaluated one time step
 * ahead: x0 = sum_{j=1..s} (-1)^(j+1) C(s, j) x_{i-j}.  Column j-1 of P (leading
 * dimension ldp) is x_{i-j}.  s = 1..4. */
int orc_extrapolate(int64_t n, int s, const double *P, int64_t ldp, double *x0);

/* ---------------- Algorithm 1 over the Sec. 6.1 sequence (sequence.c) ---------------- */
typedef struct {
    int p, N;
    double eps, dt, bx, by;
    int steps;
    int mode, m, k, window, ell, select_smallest;
    double rtol;
    int maxit;
    double rel_drop;
    int guess;         /* 0: previous solution (plain) / zero (recycled) as x_in;
                          g = 1..3: extrapolation of order g from the g+1 most recent
                          solutions (Eq. ext2-ext4) once that many are stored    */
    int velocity;      /* 0: constant (bx, by); 1: Sec. 6.1's cellular field    */
    int nmodes;        /* forcing modes per step (0: f = 1)                      */
    double fC;         /* forcing amplitude C                                    */
    const double *forcing;  /* steps x nmodes coefficients c_j, step-major     */
    int proj;          /* ORC_PROJ_* of the solves                                */
    int precond;       /* ORC_PRECOND_* of the solves                             */
    int precision;     /* 0: FP64 solves; 1: GMRES-IR (orc_gmres_ir) to rtol       */
    double inner_rtol; /* GMRES-IR: inner tolerance relative to the outer residual */
    int inner_cycles;  /* GMRES-IR: cycles per refinement                          */
    int max_refinements; /* GMRES-IR: cap on refinement steps                      */
} orc_seq_cfg;
/* u0: initial nodal field.  x_all (optional): n x steps solutions.
 * iters/k_used/status (length steps) and relres (length steps) are per step. */
int orc_sequence(const orc_seq_cfg *cfg, const double *u0, double *x_all, double *x_final,
                 int *iters, int *k_used, double *relres, int *status);
/* Same, also returning the wall time of each step (assembly + solve + window
 * update, seconds, CLOCK_MONOTONIC) in step_seconds (length steps) and, for
 * GMRES-IR sequences, the refinement steps of each solve in refinements (both
 * optional). */
int orc_sequence_timed(const orc_seq_cfg *cfg, const double *u0, double *x_all, double *x_final,
                       int *iters, int *k_used, double *relres, int *status,
                       double *step_seconds, int *refinements);

#ifdef __cplusplus
}
#endif
#endif
