// fwd_pattern_kf32d.cu -- the pattern-tile kernels and launchers of kind
// kF32D: float32 at bin 1, staged directly.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kF32D)
