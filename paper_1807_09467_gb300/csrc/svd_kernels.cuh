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

// Unpack the Gram matrix of columns 0..c-1 from the pair list (i <= j, j-major).
__device__ inline int packed_index(int i, int j) { return j * (j + 1) / 2 + i; }

// Symmetric eigen-decomposition of the c x c window Gram matrix and the choice
// of the recycle modes.  One block; G and Phi in dynamic shared memory
// (EIG_SMEM_BYTES, above the 48 KB static limit: needs the opt-in attribute).
#define EIG_SMEM_BYTES (2 * RGM_WMAX * RGM_WMAX * sizeof(double))
__global__ void sym_eig_select_kernel(Small *s, const double *gram, int c, int k,
                                      int select_smallest, double rel_drop)
{
    extern __shared__ double eig_smem[];       // G and Phi, RGM_WMAX x RGM_WMAX each
    double *G = eig_smem, *P = eig_smem + RGM_WMAX * RGM_WMAX;
    __shared__ double rc[RGM_WMAX / 2], rs[RGM_WMAX / 2];
    __shared__ int rp[RGM_WMAX / 2], rq[RGM_WMAX / 2];
    __shared__ int perm[RGM_WMAX];
    __shared__ int any_rot;
    const int ce = c + (c & 1);                 // even size for the tournament
    for (int t = threadIdx.x; t < ce * ce; t += blockDim.x) {
        int i = t % ce, j = t / ce;
        double v = 0.0;
        if (i < c && j < c) v = gram[i <= j ? packed_index(i, j) : packed_index(j, i)];
        G[i + j * RGM_WMAX] = v;
        P[i + j * RGM_WMAX] = (i == j) ? 1.0 : 0.0;
    }
    for (int t = threadIdx.x; t < ce; t += blockDim.x) perm[t] = t;
    __shared__ double gmax;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < c; ++i) m = fmax(m, G[i + i * RGM_WMAX]);
        gmax = m;
    }
    __syncthreads();
    // Stop rotating a pair when its coupling is below 1e-15 of its own
    // diagonal scale or below 2e-16 of the largest eigenvalue.  A rotation of a
    // pair that couples lambda_max with a tiny eigenvalue reintroduces couplings
    // of rounding size (about eps * lambda_max), so without this floor graded
    // windows sweep forever; the floor is the accuracy the Gram matrix carries.
    const double floor_abs = 2e-16 * gmax;
    const int npair = ce / 2;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (threadIdx.x == 0) any_rot = 0;
        __syncthreads();
        for (int step = 0; step < ce - 1; ++step) {
            // pairs of this round: (perm[i], perm[ce-1-i])
            for (int t = threadIdx.x; t < npair; t += blockDim.x) {
                int p = perm[t], q = perm[ce - 1 - t];
                if (p > q) { int tmp = p; p = q; q = tmp; }
                rp[t] = p; rq[t] = q;
                double app = G[p + p * RGM_WMAX], aqq = G[q + q * RGM_WMAX], apq = G[p + q * RGM_WMAX];
                double cth = 1.0, sth = 0.0;
                if (fabs(apq) > floor_abs && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
                    double tau = (aqq - app) / (2.0 * apq);
                    double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    cth = 1.0 / sqrt(1.0 + tt * tt);
                    sth = tt * cth;
                    any_rot = 1;
                }
                rc[t] = cth; rs[t] = sth;
            }
            __syncthreads();
            // G <- J^T G (rows p, q), then G <- G J (columns p, q), Phi <- Phi J
            for (int t = threadIdx.x; t < npair * ce; t += blockDim.x) {
                int pr = t / ce, col = t % ce;
                int p = rp[pr], q = rq[pr];
                double cth = rc[pr], sth = rs[pr];
                double gp = G[p + col * RGM_WMAX], gq = G[q + col * RGM_WMAX];
                G[p + col * RGM_WMAX] = cth * gp - sth * gq;
                G[q + col * RGM_WMAX] = sth * gp + cth * gq;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < npair * ce; t += blockDim.x) {
                int pr = t / ce, row = t % ce;
                int p = rp[pr], q = rq[pr];
                double cth = rc[pr], sth = rs[pr];
                double gp = G[row + p * RGM_WMAX], gq = G[row + q * RGM_WMAX];
                G[row + p * RGM_WMAX] = cth * gp - sth * gq;
                G[row + q * RGM_WMAX] = sth * gp + cth * gq;
                double vp = P[row + p * RGM_WMAX], vq = P[row + q * RGM_WMAX];
                P[row + p * RGM_WMAX] = cth * vp - sth * vq;
                P[row + q * RGM_WMAX] = sth * vp + cth * vq;
            }
            __syncthreads();
            // rotate the tournament: keep perm[0], shift the rest
            if (threadIdx.x == 0) {
                int last = perm[ce - 1];
                for (int i = ce - 1; i > 1; --i) perm[i] = perm[i - 1];
                perm[1] = last;
            }
            __syncthreads();
        }
        if (!any_rot) break;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // eigenvalues (clamped at 0), stable descending order
        int ord[RGM_WMAX];
        double lam[RGM_WMAX];
        for (int i = 0; i < c; ++i) { lam[i] = G[i + i * RGM_WMAX]; ord[i] = i; }
        for (int i = 1; i < c; ++i) {
            int o = ord[i], j = i - 1;
            while (j >= 0 && lam[ord[j]] < lam[o]) { ord[j + 1] = ord[j]; --j; }
            ord[j + 1] = o;
        }
        for (int i = 0; i < c; ++i) { s->eval[i] = lam[i]; s->ord[i] = ord[i]; }
        const double s1 = lam[ord[0]] > 0 ? sqrt(lam[ord[0]]) : 0.0;
        int nz = 0;
        while (nz < c) {
            double l = lam[ord[nz]];
            double sg = l > 0 ? sqrt(l) : 0.0;
            if (!(sg > 0.0 && sg >= rel_drop * s1)) break;
            ++nz;
        }
        const int kn = k < nz ? k : nz;
        const int first = select_smallest ? nz - kn : 0;
        for (int l = 0; l < kn; ++l) {
            int e = ord[first + l];
            double sg = sqrt(lam[e]);
            for (int m = 0; m < c; ++m) s->evec[m + l * RGM_WMAX] = P[m + e * RGM_WMAX] / sg;
        }
        s->k_new = kn;
    }
}

// out[:, l] = sum_m in[:, m] C[m + l * ldc] for l < kout; in-place safe
// (each row's inputs are read before its outputs are written).  A negative
// cin or kout is read from *kdev (the dimension chosen on the device).
__global__ void combine_kernel(double *out, const double *in, const double *C, int cin, int kout,
                               const int *kdev, int64_t n, int64_t ld, int ldc)
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
            for (int m = 0; m < cin; ++m) acc += xin[m] * Cs[m + l * RGM_WMAX];
            out[i + l * ld] = acc;
        }
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
    // upper Cholesky G = R^T R, right-looking
    for (int j = 0; j < k; ++j) {
        __shared__ double d;
        if (threadIdx.x == 0) {
            double v = R[j + j * RGM_KMAX];
            d = v > 0.0 ? sqrt(v) : 1.0;
            R[j + j * RGM_KMAX] = d;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) R[j + i * RGM_KMAX] /= d;
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
        col[j] = 1.0 / R[j + j * RGM_KMAX];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int l = i + 1; l <= j; ++l) v += R[i + l * RGM_KMAX] * col[l];
            col[i] = -v / R[i + i * RGM_KMAX];
        }
        for (int i = 0; i < k; ++i) s->evec[i + j * RGM_WMAX] = col[i];
    }
}
