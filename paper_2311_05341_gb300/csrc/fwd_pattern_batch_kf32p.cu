// fwd_pattern_batch_kf32p.cu -- the persistent batch pattern kernels and launcher of kind
// kF32P: float32 pairs (64-bit words of two floats, add.f32x2) from the packed copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kF32P)
