// vec_f32_qbig_cycle.cu -- the cycle kernel(s) for float vectors with the widest
// column tier (RGM_QBIG dot columns per warp), in a translation unit of their
// own: the widest tier is the slowest to compile.
#include "vec_kernels.cuh"

RGM_VEC_DEFINE_CYCLE(f32, float, qbig, RGM_QBIG)
