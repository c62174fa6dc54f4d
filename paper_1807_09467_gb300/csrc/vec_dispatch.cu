// vec_dispatch.cu -- host-side choice of the column tier of the fused vector
// kernels: the tier is the smallest number of dot columns per warp that covers
// the largest dot-column count the launch can see (nd_max; dynamic counts
// resolve on the device and never exceed it).  The kernels themselves are
// compiled per precision and tier in vec_<precision>_q<tier>.cu.
#include "vec_kernels.cuh"

namespace {
constexpr int kWarps = RGM_THREADS / 32;
inline int tier(int nd_max) { return (nd_max + kWarps - 1) / kWarps; }
}  // namespace

#define RGM_VEC_DISPATCH(TN, T)                                                                   \
    int launch_vec(const VecOp<T> &op, int nd_max, cudaStream_t st)                               \
    {                                                                                             \
        const int q = tier(nd_max);                                                               \
        return q <= 4 ? vec_launch_##TN##_q4(op, st)                                              \
                      : q <= 8 ? vec_launch_##TN##_q8(op, st) : vec_launch_##TN##_qbig(op, st);   \
    }                                                                                             \
    int cycle_capacity(const CycleOp<T> &, int nd_max, int minb)                                  \
    {                                                                                             \
        int dev = 0;                                                                              \
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;                                         \
        const int q = tier(nd_max);                                                               \
        return q <= 4   ? vec_cycle_capacity_##TN##_q4(dev, minb)                                 \
               : q <= 8 ? vec_cycle_capacity_##TN##_q8(dev, minb)                                 \
                        : vec_cycle_capacity_##TN##_qbig(dev, minb);                              \
    }                                                                                             \
    int launch_cycle(const CycleOp<T> &c, int nd_max, cudaStream_t st)                            \
    {                                                                                             \
        const int q = tier(nd_max);                                                               \
        return q <= 4 ? vec_cycle_launch_##TN##_q4(c, st)                                         \
                      : q <= 8 ? vec_cycle_launch_##TN##_q8(c, st) : vec_cycle_launch_##TN##_qbig(c, st); \
    }                                                                                             \
    int batch_cycle_capacity(const CycleOp<T> *, int nd_max)                                      \
    {                                                                                             \
        int dev = 0;                                                                              \
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;                                         \
        const int q = tier(nd_max);                                                               \
        return q <= 4 ? vec_batch_capacity_##TN##_q4(dev)                                         \
                      : q <= 8 ? vec_batch_capacity_##TN##_q8(dev) : vec_batch_capacity_##TN##_qbig(dev); \
    }                                                                                             \
    int launch_batch_cycle(const CycleOp<T> *ops, const int *first, int nsys, int nblocks, int nd_max, \
                           cudaStream_t st)                                                       \
    {                                                                                             \
        const int q = tier(nd_max);                                                               \
        return q <= 4   ? vec_batch_launch_##TN##_q4(ops, first, nsys, nblocks, st)               \
               : q <= 8 ? vec_batch_launch_##TN##_q8(ops, first, nsys, nblocks, st)               \
                        : vec_batch_launch_##TN##_qbig(ops, first, nsys, nblocks, st);            \
    }

RGM_VEC_DISPATCH(f64, double)
RGM_VEC_DISPATCH(f32, float)
