// fwd_pattern_kf32.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kF32: float32 (one sample per word, unpacked; binned).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kF32)
