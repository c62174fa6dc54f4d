// vec_f64_qbig_batch.cu -- the batch kernel(s) for double vectors with the widest
// column tier (RGM_QBIG dot columns per warp), in a translation unit of their
// own: the widest tier is the slowest to compile.
#include "vec_kernels.cuh"

RGM_VEC_DEFINE_BATCH(f64, double, qbig, RGM_QBIG)
