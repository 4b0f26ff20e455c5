// fwd_pattern_kf32d.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kF32D: float32 at bin 1, staged directly.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kF32D)
