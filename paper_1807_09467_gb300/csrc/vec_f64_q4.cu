// vec_f64_q4.cu -- the fused vector, cycle and batched-cycle kernels for
// double vectors with up to 4 dot columns per warp (one translation unit per
// precision and column tier, so that the build runs in parallel).
#include "vec_kernels.cuh"

RGM_VEC_DEFINE(f64, double, q4, 4)
