// fwd_pattern_ku8w.cu -- the one-unit-per-CTA pattern kernels and launcher of kind
// kU8W: uint8 at larger bins (one decimated sample per word).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_FORWARD(kU8W)
