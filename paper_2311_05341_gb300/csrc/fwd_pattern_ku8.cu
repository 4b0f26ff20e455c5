// fwd_pattern_ku8.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kU8: uint8 at bin 1 (pairs of samples in 16-bit lanes, unpacked from staged bytes).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kU8)
