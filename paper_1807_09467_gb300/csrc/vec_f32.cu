// vec_f32.cu -- instantiations of the fused vector kernel for float vectors
// (compiled as their own translation unit so the build runs in parallel).
#include "vec_kernels.cuh"

int launch_vec(const VecOp<float> &op, int nd_max, cudaStream_t st)
{
    return launch_vec_impl(op, nd_max, st);
}

int cycle_capacity(const CycleOp<float> &, int nd_max)
{
    return cycle_capacity_impl<float>(nd_max);
}

int launch_cycle(const CycleOp<float> &c, int nd_max, cudaStream_t st)
{
    return launch_cycle_impl(c, nd_max, st);
}

int batch_cycle_capacity(const CycleOp<float> *, int nd_max)
{
    return batch_capacity_impl<float>(nd_max);
}

int launch_batch_cycle(const CycleOp<float> *ops, const int *first, int nsys, int nblocks, int nd_max,
                       cudaStream_t st)
{
    return launch_batch_impl(ops, first, nsys, nblocks, nd_max, st);
}
