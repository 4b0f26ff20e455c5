// fwd_pattern_ku16.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kU16: uint16 (one sample per word, unpacked).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kU16)
