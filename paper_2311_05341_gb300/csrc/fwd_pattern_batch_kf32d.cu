// fwd_pattern_batch_kf32d.cu -- the persistent batch pattern kernels and launcher of kind
// kF32D: float32 at bin 1, staged directly.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kF32D)
