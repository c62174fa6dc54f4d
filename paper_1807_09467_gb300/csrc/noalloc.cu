// noalloc.cu -- rgm_residual_noalloc: the true-residual check of a solve
// (r = b - A x, ||r||_2, ||b||_2) for callers that cannot allocate device
// memory.
//
// Who cannot allocate: code that runs while another component owns the device
// allocator (a framework that forbids raw cudaMalloc in its process), code on
// a latency-critical path where an allocation's implicit synchronisation is
// not acceptable, and code that must work after device memory is exhausted
// (e.g. a watchdog that verifies a solution before anything is freed).  They
// cannot create an rgm_solver, whose creation allocates.
//
// The scratch this kernel needs (per-block partial sums and the completion
// counter of the last-block reduction) lives in one file-scope device array,
// g_noalloc_scratch, held by every GPU that loads the library until the
// process exits.  Every call shares it: the counter is cleared at the start of
// each call, the partials are rewritten in full, and two calls that overlap on
// the GPU (different streams, or different host threads on one device) race on
// it and give wrong results.  Host code never uses the array's name as an
// address: the first call on a device, with that device current, looks the
// address up once with cudaGetSymbolAddress and caches it (make that first
// call before any stream capture).
#include "../../include/rgmres.h"
#include <cuda_runtime.h>

#include <mutex>

#define NOALLOC_THREADS 256
#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[2 * RGM_NOALLOC_MAX_BLOCKS + 32];

namespace {

std::mutex g_mu;
double *g_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Rows [blk * RGM_NOALLOC_ROWS_PER_BLOCK, ...) of A in CSR, one warp per row;
// per-block sums of r_i^2 and b_i^2, then the last block to finish adds the
// partials in block order (deterministic) and writes the two norms.
__global__ void __launch_bounds__(NOALLOC_THREADS)
residual_noalloc_kernel(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                        const double *__restrict__ val, const double *__restrict__ x,
                        const double *__restrict__ b, double *__restrict__ r, double *__restrict__ norms,
                        double *scratch)
{
    double *part_r = scratch, *part_b = scratch + RGM_NOALLOC_MAX_BLOCKS;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + 2 * RGM_NOALLOC_MAX_BLOCKS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = NOALLOC_THREADS / 32;
    const int64_t r0 = (int64_t)blockIdx.x * RGM_NOALLOC_ROWS_PER_BLOCK;
    const int64_t r1 = min(n, r0 + RGM_NOALLOC_ROWS_PER_BLOCK);
    double sr = 0.0, sb = 0.0;
    for (int64_t row = r0 + warp; row < r1; row += nw) {
        double a = 0.0;
        for (int64_t e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
            const int32_t c = col[e];
            a += (c >= 0 && c < n) ? val[e] * x[c] : __longlong_as_double(0x7ff8000000000000LL);
        }
        for (int o = 16; o >= 1; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) {
            const double ri = b[row] - a;
            if (r) r[row] = ri;
            sr += ri * ri;
            sb += b[row] * b[row];
        }
    }
    __shared__ double red[2][NOALLOC_THREADS / 32];
    if (lane == 0) { red[0][warp] = sr; red[1][warp] = sb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, tb = 0.0;
        for (int w = 0; w < nw; ++w) { tr += red[0][w]; tb += red[1][w]; }
        part_r[blockIdx.x] = tr;
        part_b[blockIdx.x] = tb;
    }
    // last-block-done: no block waits for another
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double tr = 0.0, tb = 0.0;
        for (unsigned i = 0; i < gridDim.x; ++i) { tr += __ldcg(part_r + i); tb += __ldcg(part_b + i); }
        norms[0] = sqrt(tr);
        norms[1] = sqrt(tb);
        *counter = 0u;
    }
}

}  // namespace

extern "C" int rgm_residual_noalloc(int64_t n, const int64_t *rowptr, const int32_t *col,
                                    const double *val, const double *x, const double *b, double *r,
                                    double *norms, void *cuda_stream)
{
    if (n < 1 || !rowptr || !col || !val || !x || !b || !norms) return RGM_E_ARG;
    const int64_t nblocks = (n + RGM_NOALLOC_ROWS_PER_BLOCK - 1) / RGM_NOALLOC_ROWS_PER_BLOCK;
    if (nblocks > RGM_NOALLOC_MAX_BLOCKS) return RGM_E_ARG;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return RGM_E_CUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RGM_E_CUDA;
            g_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the completion counter must start at zero
    if (cudaMemsetAsync(scratch + 2 * RGM_NOALLOC_MAX_BLOCKS, 0, sizeof(unsigned), st) != cudaSuccess)
        return RGM_E_CUDA;
    residual_noalloc_kernel<<<(unsigned)nblocks, NOALLOC_THREADS, 0, st>>>(n, rowptr, col, val, x, b, r,
                                                                          norms, scratch);
    return cudaGetLastError() == cudaSuccess ? RGM_OK : RGM_E_CUDA;
}
