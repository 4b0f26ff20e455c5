// fwd_pattern_batch_kf32.cu -- the persistent batch pattern kernels and launcher of kind
// kF32: float32 (one sample per word, unpacked; binned).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kF32)
