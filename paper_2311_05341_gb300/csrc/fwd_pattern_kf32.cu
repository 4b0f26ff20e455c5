// fwd_pattern_kf32.cu -- the pattern-tile kernels and launchers of kind
// kF32: float32 (one sample per word, unpacked; binned).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kF32)
