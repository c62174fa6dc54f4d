// vec_f32.cu -- instantiations of the fused vector kernel for float vectors
// (compiled as their own translation unit so the build runs in parallel).
#include "vec_kernels.cuh"

int launch_vec(const VecOp<float> &op, int nd_max, cudaStream_t st)
{
    return launch_vec_impl(op, nd_max, st);
}
