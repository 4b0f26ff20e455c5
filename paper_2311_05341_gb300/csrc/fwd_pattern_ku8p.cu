// fwd_pattern_ku8p.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kU8P: uint8 or 4-bit from the packed copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kU8P)
