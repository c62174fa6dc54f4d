// svd_kernels.cuh -- recycle space from the snapshot window (Sec. 5.2,
// Algorithm 1) and small conversion kernels (included by solver.cu).
//
// Route on the device: G = X^T X (binary64 Gram of the c <= 64 window
// columns), G = Phi Lambda Phi^T by cyclic Jacobi with the round-robin
// parallel ordering (c/2 disjoint rotations per step), sigma_i = sqrt(lambda_i)
// sorted descending, U = X Phi_k Sigma_k^{-1} for the kept modes, then two
// CholeskyQR passes so that U^T U = I to rounding.  X's left singular vectors
// are X phi_i / sigma_i, so span U is the paper's Psi_m[1:s].
#pragma once
#include "common.cuh"

__global__ void convert_kernel(float *dst, const double *src, int64_t n, int64_t ld, int ncols)
{
    for (int c = 0; c < ncols; ++c)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            dst[i + c * ld] = (float)src[i + c * ld];
}

__global__ void add_f32_kernel(double *x, const float *d, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

__global__ void clear_skip_kernel(Small *s)
{
    if (threadIdx.x == 0) s->skip = 0;
}

// Left Jacobi (M = diag(A)) on the sliced-ELL operator: one warp per slice,
// one lane per row; d = sum of the row's entries in column i (padding entries
// hold 0 and add nothing), 1 if that sum is 0; the row's values are divided
// by d.  Rows of a slice are interleaved: entry e of the slice belongs to the
// row in lane e mod 32.
__global__ void jacobi_scale_kernel(double *__restrict__ sval, const int32_t *__restrict__ scol,
                                    const int64_t *__restrict__ slice_ptr, const int32_t *__restrict__ perm,
                                    int64_t nslices, double *__restrict__ dvec)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nwarps) {
        const int pr = perm[(sl << 5) + lane];
        if (pr < 0) continue;
        const int64_t p0 = slice_ptr[sl], p1 = slice_ptr[sl + 1];
        double d = 0.0;
        for (int64_t e = p0 + lane; e < p1; e += 32)
            if (scol[e] == pr) d += sval[e];
        if (d == 0.0) d = 1.0;
        dvec[pr] = d;
        for (int64_t e = p0 + lane; e < p1; e += 32) sval[e] = sval[e] / d;
    }
}

// v = v ./ d (div = 1) or v .* d (div = 0)
__global__ void diag_apply_kernel(double *v, const double *d, int64_t n, int div)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = div ? v[i] / d[i] : v[i] * d[i];
}

// Extrapolated initial guess (Sec. 4.1, Eq. ext2 / ext3 / ext4): x = sum over
// j = 1..s of (-1)^(j+1) C(s, j) x_{i-j}, where x_{i-j} sits in ring slot
// (newest - j + 1) mod window of the snapshot window X.
__global__ void extrap_kernel(double *__restrict__ x, const double *__restrict__ X, int64_t ld, int s,
                              int newest, int window, int64_t n)
{
    double c[4];
    int64_t off[4];
    double binom = 1.0;
    for (int j = 1; j <= s; ++j) {
        binom = binom * (double)(s - j + 1) / (double)j;
        c[j - 1] = (j % 2 == 1) ? binom : -binom;
        off[j - 1] = (int64_t)((newest - (j - 1) + window) % window) * ld;
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j) acc += c[j] * X[r + off[j]];
        x[r] = acc;
    }
}

// Row-major copy of the k columns of U (row r at Urow + r k) for the SpMM
// gather, through a shared-memory tile of RGM_UROW_ROWS rows (coalesced on
// both sides).
#define RGM_UROW_ROWS 128
template <typename T>
__global__ void __launch_bounds__(256) urow_kernel(T *__restrict__ Urow, const T *__restrict__ U,
                                                   int64_t n, int64_t ld, int k, int kp)
{
    __shared__ T t[RGM_UROW_ROWS * (RGM_KMAX + 1)];
    const int64_t r0 = (int64_t)blockIdx.x * RGM_UROW_ROWS;
    const int nr = (int)min((int64_t)RGM_UROW_ROWS, n - r0);
    for (int i = threadIdx.x; i < RGM_UROW_ROWS * k; i += blockDim.x) {
        const int r = i % RGM_UROW_ROWS, c = i / RGM_UROW_ROWS;
        if (r < nr) t[r * (RGM_KMAX + 1) + c] = U[r0 + r + (int64_t)c * ld];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * kp; i += blockDim.x) {
        const int r = i / kp, c = i % kp;
        Urow[(r0 + r) * kp + c] = (c < k) ? t[r * (RGM_KMAX + 1) + c] : (T)0;
    }
}

// W = A U for k columns in one pass over the sliced-ELL operator (the operator
// is read once per RGM_SPMM_KB columns instead of once per column): one warp
// per 32-row slice, one lane per row, RGM_SPMM_KB accumulators per lane; the
// gathered rows of U come from the row-major copy (contiguous per entry).
// T = float: the binary32 operator and recycle columns of GMRES-IR (16
// accumulators: k <= 16 reads the operator once).
#define RGM_SPMM_KB ((sizeof(T) == 4) ? 16 : 8)
#ifndef RGM_SPMM_UNROLL
#define RGM_SPMM_UNROLL 2
#endif
constexpr int kSpmmUnroll = RGM_SPMM_UNROLL;   // entries in flight per lane
template <typename T>
__global__ void __launch_bounds__(256) spmm_kernel(const int64_t *__restrict__ slice_ptr,
                                                   const int32_t *__restrict__ scol,
                                                   const T *__restrict__ sval,
                                                   const int32_t *__restrict__ perm, int64_t nslices,
                                                   const T *__restrict__ Urow, int k, int kp,
                                                   T *__restrict__ W, int64_t ldw)
{
    // the gathered row of U is read as 16-byte vectors (row stride kp, a
    // multiple of the vector width; columns k .. kp-1 hold zeros)
    constexpr int VW = 16 / (int)sizeof(T);
    using VT = typename Vec16<T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nwarps) {
        const int64_t p0 = slice_ptr[sl], p1 = slice_ptr[sl + 1];
        const int pr = perm[(sl << 5) + lane];
        for (int c0 = 0; c0 < k; c0 += RGM_SPMM_KB) {
            T acc[RGM_SPMM_KB];
#pragma unroll
            for (int c = 0; c < RGM_SPMM_KB; ++c) acc[c] = (T)0;
            // the iterations are independent but for the accumulators: unrolled,
            // their gathers of U rows overlap
#pragma unroll kSpmmUnroll
            for (int64_t e = p0 + lane; e < p1; e += 32) {
                const T a = sval[e];
                const VT *u = reinterpret_cast<const VT *>(Urow + (int64_t)scol[e] * kp + c0);
#pragma unroll
                for (int cv = 0; cv < RGM_SPMM_KB / VW; ++cv)
                    if (c0 + cv * VW < k) {
                        const VT v = u[cv];
#pragma unroll
                        for (int t = 0; t < VW; ++t)
                            acc[cv * VW + t] = fma(a, vcomp<VT, T>(v, t), acc[cv * VW + t]);
                    }
            }
            if (pr >= 0) {
#pragma unroll
                for (int c = 0; c < RGM_SPMM_KB; ++c)
                    if (c0 + c < k) W[pr + (int64_t)(c0 + c) * ldw] = acc[c];
            }
        }
    }
}

// The window Gram matrix kept between updates (full, leading dimension
// RGM_WMAX): a new snapshot in ring slot `slot` replaces row and column slot
// with its dots against the c stored columns (col[j] = x_slot . x_j).
__global__ void gram_insert_kernel(double *gwin, const double *col, int slot, int c)
{
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        gwin[slot + j * RGM_WMAX] = col[j];
        gwin[j + slot * RGM_WMAX] = col[j];
    }
}

// Full window Gram matrix from the packed pair list (rebuild after a reset).
__global__ void gram_unpack_kernel(double *gwin, const double *packed, int c)
{
    for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
        const int i = t % c, j = t / c;
        gwin[i + j * RGM_WMAX] = packed[i <= j ? j * (j + 1) / 2 + i : i * (i + 1) / 2 + j];
    }
}

// Unpack the Gram matrix of columns 0..c-1 from the pair list (i <= j, j-major).
__device__ inline int packed_index(int i, int j) { return j * (j + 1) / 2 + i; }

// Symmetric eigen-decomposition of the c x c window Gram matrix and the choice
// of the recycle modes.  One block; G, Phi and a product buffer in dynamic
// shared memory (EIG_SMEM_BYTES, above the 48 KB static limit: needs the
// opt-in attribute).
//
// Leading modes (select_smallest == 0): the rotations run on G1 = R R^T, where
// G = R^T R is the pivoted Cholesky factorisation of G (R: r x c, one row per
// pivot step, columns in slot order; pivot steps stop once the largest
// remaining diagonal entry is below 1e-17 lambda_max, so the dropped part is
// far below any mode the selection can keep).  G1 has the eigenvalues of G
// (one step of the Cholesky LR iteration) and is much closer to diagonal on
// graded windows -- the snapshots of a time sequence, whose Gram eigenvalues
// fall geometrically -- so the rotations need 4-6 sweeps instead of about 12;
// an eigenvector q of G1 gives v = R^T q / sqrt(lambda) of G.
//
// Trailing modes (select_smallest): the rotations run on G itself, warm
// started: consecutive windows share all columns but the replaced ones, so the
// eigenvectors Phi0 of the previous window Gram matrix (Small::phi, rows indexed
// by ring slot; slots added since get unit vectors) nearly diagonalise the new
// one.  The rotations run on Phi0^T G Phi0 with Phi accumulated from Phi0 -- a
// similarity transform, so the eigenpairs are those of G.
#define EIG_SMEM_BYTES (4 * RGM_WMAX * RGM_WMAX * sizeof(double))
__global__ void sym_eig_select_kernel(Small *s, const double *gram, int c, int k,
                                      int select_smallest, double rel_drop)
// gram: the full c x c window Gram matrix, leading dimension RGM_WMAX
{
    extern __shared__ double eig_smem[];       // G, Phi, T and R, RGM_WMAX x RGM_WMAX each
    double *G = eig_smem, *P = eig_smem + RGM_WMAX * RGM_WMAX, *T = P + RGM_WMAX * RGM_WMAX;
    double *R = T + RGM_WMAX * RGM_WMAX;        // R[a + m RGM_WMAX]: pivot step a, slot m
    __shared__ double rc[RGM_WMAX / 2], rs[RGM_WMAX / 2];
    __shared__ int rp[RGM_WMAX / 2], rq[RGM_WMAX / 2];
    const bool lr = !select_smallest;           // rotations on R R^T
    const int c0e = c + (c & 1);
    const int pc = s->phi_c;
    const bool warm = !lr && pc > 0 && pc <= c; // the previous window's slots are a prefix
    for (int t = threadIdx.x; t < c0e * c0e; t += blockDim.x) {
        int i = t % c0e, j = t / c0e;
        double v = 0.0;
        if (i < c && j < c) v = gram[i + j * RGM_WMAX];
        G[i + j * RGM_WMAX] = v;
        T[i + j * RGM_WMAX] = v;
        P[i + j * RGM_WMAX] = (warm && i < pc && j < pc) ? s->phi[i + j * RGM_WMAX]
                              : (warm && (i < pc || j < pc)) ? 0.0 : (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();                            // G complete before its diagonal is read
    __shared__ double gmax;
    __shared__ int rsz;                         // size of the matrix the rotations run on
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < c; ++i) m = fmax(m, G[i + i * RGM_WMAX]);
        gmax = m;
        rsz = c;
    }
    __syncthreads();
    if (lr) {
        // pivoted Cholesky G = R^T R on the working copy T (Schur complements);
        // pivot: the largest remaining diagonal entry
        __shared__ int piv_done[RGM_WMAX];
        __shared__ int pj;
        __shared__ double pd;
        for (int i = threadIdx.x; i < c; i += blockDim.x) piv_done[i] = 0;
        const double tau = 1e-17 * gmax;
        int r = 0;
        for (; r < c; ++r) {
            __syncthreads();                    // previous update and flags done
            if (threadIdx.x == 0) {
                int p = -1;
                double d = tau;
                for (int i = 0; i < c; ++i)
                    if (!piv_done[i] && T[i + i * RGM_WMAX] > d) { d = T[i + i * RGM_WMAX]; p = i; }
                pj = p;
                pd = d;
            }
            __syncthreads();
            const int p = pj;
            if (p < 0) break;                   // same value in every thread
            const double rsd = rsqrt(pd), sd = pd * rsd;
            for (int m = threadIdx.x; m < c; m += blockDim.x)
                R[r + m * RGM_WMAX] = (m == p) ? sd : piv_done[m] ? 0.0 : T[p + m * RGM_WMAX] * rsd;
            __syncthreads();
            for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
                const int a = t % c, b = t / c;
                if (a != p && b != p && !piv_done[a] && !piv_done[b])
                    T[a + b * RGM_WMAX] -= R[r + a * RGM_WMAX] * R[r + b * RGM_WMAX];
            }
            if (threadIdx.x == 0) piv_done[p] = 1;
        }
        __syncthreads();
        // G <- R R^T (r x r, zero-padded to even size); P <- identity
        const int re = r + (r & 1);
        for (int t = threadIdx.x; t < c0e * c0e; t += blockDim.x) {
            const int a = t % c0e, b = t / c0e;
            double v = 0.0;
            if (a < r && b < r)
                for (int m = 0; m < c; ++m) v = fma(R[a + m * RGM_WMAX], R[b + m * RGM_WMAX], v);
            G[a + b * RGM_WMAX] = v;
            P[a + b * RGM_WMAX] = (a == b && a < re) ? 1.0 : 0.0;
        }
        if (threadIdx.x == 0) rsz = r;
    }
    if (warm) {
        const int ce = c0e;
        // G <- Phi0^T (G Phi0): T = G Phi0, then the upper triangle of Phi0^T T,
        // mirrored (the rotations below keep G exactly symmetric)
        for (int t = threadIdx.x; t < ce * ce; t += blockDim.x) {
            const int i = t % ce, j = t / ce;
            double v = 0.0;
            for (int m = 0; m < ce; ++m) v = fma(G[i + m * RGM_WMAX], P[m + j * RGM_WMAX], v);
            T[i + j * RGM_WMAX] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ce * ce; t += blockDim.x) {
            const int i = t % ce, j = t / ce;
            if (i > j) continue;
            double v = 0.0;
            for (int m = 0; m < ce; ++m) v = fma(P[m + i * RGM_WMAX], T[m + j * RGM_WMAX], v);
            G[i + j * RGM_WMAX] = v;
            G[j + i * RGM_WMAX] = v;
        }
    }
    __syncthreads();
    const int cs = rsz;                         // c, or the Cholesky rank r
    const int ce = cs + (cs & 1);               // even size for the tournament
    // Stop rotating a pair when its coupling is below 1e-15 of its own
    // diagonal scale or below 2e-16 of the largest eigenvalue.  A rotation of a
    // pair that couples lambda_max with a tiny eigenvalue reintroduces couplings
    // of rounding size (about eps * lambda_max), so without this floor graded
    // windows sweep forever; the floor is the accuracy the Gram matrix carries.
    const double floor_abs = 2e-16 * gmax;
    const double floor2 = floor_abs * floor_abs;
    const int npair = ce / 2, nround = ce - 1;
    __shared__ double rt[RGM_WMAX / 2];
    __shared__ int rot_flag[2];
    if (threadIdx.x == 0) rot_flag[0] = 0;
    __syncthreads();
    for (int sweep = 0; sweep < 30; ++sweep) {
        const int fl = sweep & 1;
        for (int round = 0; round < nround; ++round) {
            // round-robin pairs (circle method): (round, ce-1) and
            // ((round + i) mod (ce-1), (round - i) mod (ce-1)), i = 1 .. npair-1
            for (int t = threadIdx.x; t < npair; t += blockDim.x) {
                int a = round, b = ce - 1;
                if (t > 0) { a = (round + t) % nround; b = (round - t + nround) % nround; }
                const int p = min(a, b), q = max(a, b);
                rp[t] = p; rq[t] = q;
                const double app = G[p + p * RGM_WMAX], aqq = G[q + q * RGM_WMAX], apq = G[p + q * RGM_WMAX];
                double cth = 1.0, sth = 0.0, tt = 0.0;
                const double apq2 = apq * apq;
                if (apq2 > floor2 && apq2 > 1e-30 * fabs(app * aqq)) {
                    // the rotation with tan(2 theta) = 2 apq / d, d = aqq - app,
                    // |theta| <= pi/4: cos(2 theta) = |d| / sqrt(h), sin(2 theta) =
                    // 2 apq sgn(d) / sqrt(h), h = d^2 + 4 apq^2; then cos^2(theta) =
                    // (1 + cos(2 theta)) / 2 and sin(theta) = sin(2 theta) / (2 cos(theta))
                    // (half-angle identities: two reciprocal square roots, no division)
                    const double d = aqq - app;
                    const double h = fma(d, d, 4.0 * apq2);
                    const double num = (d > 0.0) ? 2.0 * apq : (d < 0.0) ? -2.0 * apq : 2.0 * fabs(apq);
                    const double rh = rsqrt(h);
                    const double x = fma(0.5 * fabs(d), rh, 0.5);     // cos^2(theta)
                    const double y = rsqrt(x);                         // 1 / cos(theta)
                    cth = x * y;
                    sth = 0.5 * num * rh * y;
                    tt = sth * y;                                      // tan(theta)
                    rot_flag[fl] = 1;
                }
                rc[t] = cth; rs[t] = sth; rt[t] = tt;
            }
            __syncthreads();
            // clear the next sweep's flag: every thread has read it (end of the
            // previous sweep) before this barrier, and it is next written in the
            // next sweep
            if (round == 0 && threadIdx.x == 0) rot_flag[fl ^ 1] = 0;
            // G <- J^T G J: every 2 x 2 block (pair a rows, pair b columns) with
            // a <= b in one thread (two-sided), mirrored; Phi <- Phi J
            const int nblk = npair * npair;
            for (int x = threadIdx.x; x < nblk + npair * ce; x += blockDim.x) {
                if (x < nblk) {
                    const int ia = x % npair, ib = x / npair;
                    if (ia > ib) continue;
                    const int p1 = rp[ia], q1 = rq[ia];
                    if (ia == ib) {
                        const double tt = rt[ia];
                        if (tt != 0.0) {
                            const double apq = G[p1 + q1 * RGM_WMAX];
                            G[p1 + p1 * RGM_WMAX] -= tt * apq;
                            G[q1 + q1 * RGM_WMAX] += tt * apq;
                            G[p1 + q1 * RGM_WMAX] = 0.0;
                            G[q1 + p1 * RGM_WMAX] = 0.0;
                        }
                        continue;
                    }
                    const int p2 = rp[ib], q2 = rq[ib];
                    const double c1 = rc[ia], s1 = rs[ia], c2 = rc[ib], s2 = rs[ib];
                    const double b00 = G[p1 + p2 * RGM_WMAX], b01 = G[p1 + q2 * RGM_WMAX];
                    const double b10 = G[q1 + p2 * RGM_WMAX], b11 = G[q1 + q2 * RGM_WMAX];
                    const double r00 = c1 * b00 - s1 * b10, r01 = c1 * b01 - s1 * b11;
                    const double r10 = s1 * b00 + c1 * b10, r11 = s1 * b01 + c1 * b11;
                    const double n00 = c2 * r00 - s2 * r01, n01 = s2 * r00 + c2 * r01;
                    const double n10 = c2 * r10 - s2 * r11, n11 = s2 * r10 + c2 * r11;
                    G[p1 + p2 * RGM_WMAX] = n00; G[p2 + p1 * RGM_WMAX] = n00;
                    G[p1 + q2 * RGM_WMAX] = n01; G[q2 + p1 * RGM_WMAX] = n01;
                    G[q1 + p2 * RGM_WMAX] = n10; G[p2 + q1 * RGM_WMAX] = n10;
                    G[q1 + q2 * RGM_WMAX] = n11; G[q2 + q1 * RGM_WMAX] = n11;
                } else {
                    const int y = x - nblk, pr = y / ce, row = y % ce;
                    const int p = rp[pr], q = rq[pr];
                    const double cth = rc[pr], sth = rs[pr];
                    const double vp = P[row + p * RGM_WMAX], vq = P[row + q * RGM_WMAX];
                    P[row + p * RGM_WMAX] = cth * vp - sth * vq;
                    P[row + q * RGM_WMAX] = sth * vp + cth * vq;
                }
            }
            __syncthreads();
        }
        if (!rot_flag[fl]) break;
        // would the next sweep rotate at all?  The same test on every pair of
        // the current matrix (a sweep that rotates nothing leaves it as is), so
        // the sweep that only confirms convergence is not run
        __shared__ int more;
        if (threadIdx.x == 0) more = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < ce * ce; t += blockDim.x) {
            const int p = t % ce, q = t / ce;
            if (p < q) {
                const double app = G[p + p * RGM_WMAX], aqq = G[q + q * RGM_WMAX], apq = G[p + q * RGM_WMAX];
                const double apq2 = apq * apq;
                if (apq2 > floor2 && apq2 > 1e-30 * fabs(app * aqq)) more = 1;
            }
        }
        __syncthreads();
        if (!more) break;
    }
    if (lr) {
        // eigenvectors of G: v_j = R^T q_j / sqrt(lambda_j) for the r eigenpairs
        // of R R^T; the c - r dropped directions get lambda = 0 and v = 0
        for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
            const int m = t % c, j = t / c;
            double v = 0.0;
            if (j < cs) {
                const double lj = G[j + j * RGM_WMAX];
                for (int a = 0; a < cs; ++a) v = fma(R[a + m * RGM_WMAX], P[a + j * RGM_WMAX], v);
                v = (lj > 0.0) ? v * rsqrt(lj) : 0.0;
            }
            T[m + j * RGM_WMAX] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
            const int m = t % c, j = t / c;
            P[m + j * RGM_WMAX] = T[m + j * RGM_WMAX];
            if (m == j && j >= cs) G[j + j * RGM_WMAX] = 0.0;
        }
        if (threadIdx.x == 0) s->phi_c = 0;     // no warm start from this path
        __syncthreads();
    } else {
        // the next update starts from these eigenvectors
        for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
            const int i = t % c, j = t / c;
            s->phi[i + j * RGM_WMAX] = P[i + j * RGM_WMAX];
        }
        if (threadIdx.x == 0) s->phi_c = c;
    }
    // eigenvalues, stable descending order by rank counting (ties by index)
    __shared__ double lam[RGM_WMAX], isg[RGM_WMAX];
    __shared__ int ord[RGM_WMAX];
    __shared__ int sel[2];                       // k_new, first selected rank
    for (int i = threadIdx.x; i < c; i += blockDim.x) lam[i] = G[i + i * RGM_WMAX];
    __syncthreads();
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        const double li = lam[i];
        int r = 0;
        for (int j = 0; j < c; ++j) r += (lam[j] > li || (lam[j] == li && j < i)) ? 1 : 0;
        ord[r] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // keep sigma_i = sqrt(lambda_i) > 0 with sigma_i >= rel_drop sigma_1
        // (compared as squares)
        const double l1 = lam[ord[0]];
        const double thr = (l1 > 0.0) ? rel_drop * rel_drop * l1 : INFINITY;
        int nz = 0;
        while (nz < c && lam[ord[nz]] > 0.0 && lam[ord[nz]] >= thr) ++nz;
        const int kn = k < nz ? k : nz;
        sel[0] = kn;
        sel[1] = select_smallest ? nz - kn : 0;
        s->k_new = kn;
    }
    __syncthreads();
    const int kn = sel[0], first = sel[1];
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        s->eval[i] = lam[i];
        s->ord[i] = ord[i];
    }
    for (int l = threadIdx.x; l < kn; l += blockDim.x) isg[l] = rsqrt(lam[ord[first + l]]);
    __syncthreads();
    // evec[:, l] = phi_e / sigma_e for the selected modes e
    for (int t = threadIdx.x; t < kn * c; t += blockDim.x) {
        const int l = t / c, m = t % c, e = ord[first + l];
        s->evec[m + l * RGM_WMAX] = P[m + e * RGM_WMAX] * isg[l];
    }
}

// out[:, l] = sum_m in[:, m] C[m + l * ldc] for l < kout; in-place safe
// (each row's inputs are read before its outputs are written).  A negative
// cin or kout is read from *kdev (the dimension chosen on the device).
// upper: C is upper triangular (its entries below the diagonal are zeros), so
// the sum stops at m = l -- the same values with half the binary64 FMAs.
__global__ void combine_kernel(double *out, const double *in, const double *C, int cin, int kout,
                               const int *kdev, int64_t n, int64_t ld, int ldc, int upper)
{
    __shared__ double Cs[RGM_WMAX * RGM_KMAX];
    if (cin < 0) cin = *kdev;
    if (kout < 0) kout = *kdev;
    if (kout <= 0) return;
    for (int t = threadIdx.x; t < cin * kout; t += blockDim.x) {
        int m = t % cin, l = t / cin;
        Cs[m + l * RGM_WMAX] = C[m + l * ldc];
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xin[RGM_WMAX];
#pragma unroll 8
        for (int m = 0; m < cin; ++m) xin[m] = in[i + m * ld];
        for (int l = 0; l < kout; ++l) {
            double acc = 0.0;
            const int mend = upper ? min(cin, l + 1) : cin;
            for (int m = 0; m < mend; ++m) acc += xin[m] * Cs[m + l * RGM_WMAX];
            out[i + l * ld] = acc;
        }
    }
}

// First CholQR pass of the recycle space in the window's coordinates: with
// U = X C (C = Phi_k Sigma_k^{-1}, the selected columns of Small::evec) the Gram
// matrix of U is C^T (X^T X) C, formed from the resident window Gram matrix G
// instead of n-length dot products; its Cholesky factor R gives C <- C R^{-1},
// so that the one n-length combination U = X C already carries the first
// pass.  The second pass (Gram of the formed U) then removes the rounding of
// that combination.  One block; c <= RGM_WMAX, k <= RGM_KMAX.
__global__ void cholqr_small_kernel(Small *s, const double *gwin, int c, const int *kdev)
{
    __shared__ double E[RGM_WMAX * RGM_KMAX];    // C, leading dimension RGM_WMAX
    __shared__ double T[RGM_WMAX * RGM_KMAX];    // G C, later R^{-1}
    __shared__ double R[RGM_KMAX * RGM_KMAX];
    __shared__ double rdiag[RGM_KMAX];
    const int k = *kdev;
    if (k <= 0) return;
    for (int t = threadIdx.x; t < c * k; t += blockDim.x) {
        const int m = t % c, l = t / c;
        E[m + l * RGM_WMAX] = s->evec[m + l * RGM_WMAX];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < c * k; t += blockDim.x) {
        const int m = t % c, l = t / c;
        double v = 0.0;
        for (int p = 0; p < c; ++p) v = fma(gwin[m + p * RGM_WMAX], E[p + l * RGM_WMAX], v);
        T[m + l * RGM_WMAX] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int i = t % k, j = t / k;
        double v = 0.0;
        if (i <= j)
            for (int m = 0; m < c; ++m) v = fma(E[m + i * RGM_WMAX], T[m + j * RGM_WMAX], v);
        R[i + j * RGM_KMAX] = v;
    }
    __syncthreads();
    // upper Cholesky, right-looking, pivots by rsqrt (as chol_inv_kernel)
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            const double v = R[j + j * RGM_KMAX];
            const double r = v > 0.0 ? rsqrt(v) : 1.0;
            R[j + j * RGM_KMAX] = v > 0.0 ? v * r : 1.0;
            rdiag[j] = r;
        }
        __syncthreads();
        const double rd = rdiag[j];
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) R[j + i * RGM_KMAX] *= rd;
        __syncthreads();
        for (int t = threadIdx.x; t < (k - j - 1) * (k - j - 1); t += blockDim.x) {
            const int a = j + 1 + t % (k - j - 1), b = j + 1 + t / (k - j - 1);
            if (a <= b) R[a + b * RGM_KMAX] -= R[j + a * RGM_KMAX] * R[j + b * RGM_KMAX];
        }
        __syncthreads();
    }
    // R^{-1} (upper), one thread per column, into T
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        for (int i = 0; i < k; ++i) T[i + j * RGM_KMAX] = 0.0;
        T[j + j * RGM_KMAX] = rdiag[j];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int l = i + 1; l <= j; ++l) v += R[i + l * RGM_KMAX] * T[l + j * RGM_KMAX];
            T[i + j * RGM_KMAX] = -v * rdiag[i];
        }
    }
    __syncthreads();
    // C <- C R^{-1}
    for (int t = threadIdx.x; t < c * k; t += blockDim.x) {
        const int m = t % c, l = t / c;
        double v = 0.0;
        for (int i = 0; i <= l; ++i) v = fma(E[m + i * RGM_WMAX], T[i + l * RGM_KMAX], v);
        s->evec[m + l * RGM_WMAX] = v;
    }
}

// Cholesky factor R of the packed Gram matrix of U (k x k), and its inverse
// into Small::evec so that U R^{-1} has orthonormal columns.  One block:
// the factorisation row by row with the trailing updates in parallel, then one
// thread per column of R^{-1} (back substitution from shared memory).
__global__ void chol_inv_kernel(Small *s, const double *gram, int k, const int *kdev)
{
    __shared__ double R[RGM_KMAX * RGM_KMAX];
    if (k < 0) k = *kdev;
    if (k <= 0) return;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int i = t % k, j = t / k;
        R[i + j * RGM_KMAX] = (i <= j) ? gram[packed_index(i, j)] : 0.0;
    }
    __syncthreads();
    // upper Cholesky G = R^T R, right-looking; the pivots' reciprocals are
    // kept, so no division is on the serial path
    __shared__ double rdiag[RGM_KMAX];
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            const double v = R[j + j * RGM_KMAX];
            const double r = v > 0.0 ? rsqrt(v) : 1.0;
            R[j + j * RGM_KMAX] = v > 0.0 ? v * r : 1.0;
            rdiag[j] = r;
        }
        __syncthreads();
        const double rd = rdiag[j];
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) R[j + i * RGM_KMAX] *= rd;
        __syncthreads();
        for (int t = threadIdx.x; t < (k - j - 1) * (k - j - 1); t += blockDim.x) {
            const int a = j + 1 + t % (k - j - 1), b = j + 1 + t / (k - j - 1);
            if (a <= b) R[a + b * RGM_KMAX] -= R[j + a * RGM_KMAX] * R[j + b * RGM_KMAX];
        }
        __syncthreads();
    }
    // column j of R^{-1}
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double col[RGM_KMAX];
        for (int i = 0; i < k; ++i) col[i] = 0.0;
        col[j] = rdiag[j];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int l = i + 1; l <= j; ++l) v += R[i + l * RGM_KMAX] * col[l];
            col[i] = -v * rdiag[i];
        }
        for (int i = 0; i < k; ++i) s->evec[i + j * RGM_WMAX] = col[i];
    }
}
