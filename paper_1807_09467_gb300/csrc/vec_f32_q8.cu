// vec_f32_q8.cu -- the fused vector, cycle and batched-cycle kernels for
// float vectors with up to 8 dot columns per warp (one translation unit per
// precision and column tier, so that the build runs in parallel).
#include "vec_kernels.cuh"

RGM_VEC_DEFINE(f32, float, q8, 8)
