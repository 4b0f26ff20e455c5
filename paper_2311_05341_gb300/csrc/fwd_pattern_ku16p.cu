// fwd_pattern_ku16p.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kU16P: uint16 from the widened copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kU16P)
