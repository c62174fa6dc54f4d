// common.cuh -- limits, the device-resident solver state and warp/block
// reduction helpers shared by the librgmres translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RGM_MMAX 64                          // restart length limit
#define RGM_KMAX 32                          // recycle dimension limit
#define RGM_WMAX 64                          // snapshot window limit
#define RGM_HLD (RGM_MMAX + RGM_KMAX + 1)    // rows of the Hessenberg matrix
#define RGM_NCOL (RGM_MMAX + RGM_KMAX)       // columns of the Hessenberg matrix
#define RGM_MAXDOTS (RGM_KMAX + RGM_HLD + RGM_KMAX + 1)
#define RGM_THREADS 256
#ifndef RGM_MINB
#define RGM_MINB 4                           // resident blocks per SM every fused kernel is built for
                                             // (65536 / (256 RGM_MINB) registers a thread; grids hold
                                             // at most this many blocks per SM)
#endif
#define RGM_COOP_MAX_TILES 2                 // RGM_LAUNCH_AUTO takes the cooperative cycle kernel when
                                             // a block owns at most this many row tiles
#define RGM_CHUNK 8                          // dot columns per register pass
#define RGM_GATHER_SMEM_MAX (160 * 1024)     // shared memory of sell_gather_kernel at most
#define RGM_LOOKAHEAD 3                      // per-pass launches: Arnoldi steps the host runs ahead
#define RGM_LOOKAHEAD_WAIT_NS 200000000ll    // and the longest it waits for the device's progress

// Small device-resident state of one solve: the Hessenberg least-squares
// problem, Givens rotations, coefficient vectors handed from one fused kernel
// to the next, the coarse matrix E and its LU factors.  Everything is binary64
// whatever the vector precision.  Column i of the stored Krylov basis is
// v_i = colscale[i] * Vraw[:, i] (normalisation is folded into coefficients).
// The fields before H form the header the host reads back once per cycle.
struct Small {
    int done;          // Krylov phase of the current cycle finished
    int J;             // Krylov steps taken in the current cycle
    int nb;            // basis vectors stored in the current cycle
    int iters;         // Arnoldi steps in this solve
    int maxit;
    int m;
    int naug;          // appended recycle columns accepted in this cycle
    int skip;          // the appended column being processed was dropped
    int converged;     // true residual <= tol_abs
    int breakdown;
    int k;             // recycle columns in use
    int singular;      // E was declared singular
    int k_new;         // recycle dimension chosen by the last window SVD
    unsigned gen;      // grid-barrier generation of the persistent cycle kernel
    unsigned fault;    // a bounded device wait gave up (cleared per solve)
    int aug_idx[RGM_KMAX];
    double bnorm, tol_abs, beta, wn0, bs;
    double bnorm_p, tol_in;  // preconditioned ||D^{-1} b|| and the in-cycle tolerance
    double H[RGM_HLD * RGM_NCOL];         // column-major, leading dimension RGM_HLD
    double cs[RGM_HLD], sn[RGM_HLD], g[RGM_HLD + 1], y[RGM_HLD];
    double hsum[RGM_HLD];                 // Gram-Schmidt coefficients of the current column
    double colscale[RGM_HLD];
    double coefW[RGM_KMAX];               // AXPY coefficients on columns of W
    double coefV[RGM_HLD];                // AXPY coefficients on columns of Vraw
    double coefU[RGM_KMAX];               // AXPY coefficients on columns of U
    double VtW[RGM_HLD * RGM_KMAX];       // v_i^T W_l at [i + l * RGM_HLD]
    double E[RGM_KMAX * RGM_KMAX];
    double LU[RGM_KMAX * RGM_KMAX];
    double LUrd[RGM_KMAX];                // reciprocals of the U pivots of LU
    int piv[RGM_KMAX];                    // row swaps of the LU, in order
    int LUperm[RGM_KMAX];                 // the same swaps as one permutation
    double LUP[RGM_KMAX * RGM_KMAX];      // LU of the projector's Gram matrix Y^T Y
    double LUPrd[RGM_KMAX];               //   (orthogonal: Y = U, least squares: Y = A U)
    int pivP[RGM_KMAX];
    int LUPperm[RGM_KMAX];
    double dots[RGM_MAXDOTS];             // last reduced dot products
    double gram[RGM_WMAX * RGM_WMAX];     // last reduced Gram matrix
    double evec[RGM_WMAX * RGM_WMAX];     // eigenvectors of the window Gram matrix
    double eval[RGM_WMAX];
    int ord[RGM_WMAX];
    double wn_dummy;
    // eigenvectors of the last window Gram matrix (rows: ring slots), the
    // starting rotation of the next eigen-decomposition; phi_c = 0: none
    double phi[RGM_WMAX * RGM_WMAX];
    int phi_c;
};

// Reduce NV per-lane values across a warp with a butterfly that halves the
// number of live values at each step (NV-1 + 5-log2(NV) shuffles instead of
// 5*NV).  On return lane l holds the warp sum of value (l >> (5 - log2 NV))
// in v[0].
template <int NV>
__device__ __forceinline__ void warp_multi_reduce(double (&v)[NV])
{
    const int lane = threadIdx.x & 31;
    int live = NV;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (live > 1) {
            const int half = live >> 1;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < NV / 2; ++i) {
                if (i < half) {
                    double send = upper ? v[i] : v[i + half];
                    double keep = upper ? v[i + half] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            live = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

template <int NV>
__device__ __forceinline__ int warp_multi_owner_shift()
{
    return NV == 1 ? 5 : NV == 2 ? 4 : NV == 4 ? 3 : NV == 8 ? 2 : NV == 16 ? 1 : 0;
}

// Block-reduce NV values per thread and store the nvalid block sums to
// dst[c * stride] (c < nvalid).  red: shared scratch of (blockDim/32)*NV doubles.
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double *dst, int nvalid,
                                                   int stride, double *red)
{
    warp_multi_reduce<NV>(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sh = warp_multi_owner_shift<NV>();
    if ((lane & ((1 << sh) - 1)) == 0) red[warp * NV + (lane >> sh)] = v[0];
    __syncthreads();
    if (threadIdx.x < nvalid) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
        dst[(int64_t)threadIdx.x * stride] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Record the CUDA error behind an RGM_E_CUDA / RGM_E_OOM return (solver.cu).
void rgm_note_cuda_error(int err, const char *what, int line);

// Scoped memory operations for the grid barrier of the persistent kernel.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Fetch-and-add with acquire-release semantics at GPU scope: the caller's
// earlier writes (and, through a preceding __syncthreads, those of its whole
// block) are visible to whoever observes the new value, and the caller sees
// everything released by the earlier adds it observes.
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Last-of-n: every one of n blocks calls this once (after writing what the
// last one will read); returns true in exactly the block that arrives last,
// which then sees everything the others wrote before arriving.  Nothing spins.
__device__ __forceinline__ bool last_of(unsigned *counter, unsigned n)
{
    __shared__ bool am_last;
    __syncthreads();                    // the block's writes precede thread 0's release
    if (threadIdx.x == 0) am_last = (atom_add_acq_rel_gpu(counter, 1u) == n - 1u);
    __syncthreads();                    // and its acquire precedes the block's reads
    return am_last;
}

// Last-block-done over the whole grid (see last_of).
__device__ __forceinline__ bool last_block(unsigned *counter) { return last_of(counter, gridDim.x); }
