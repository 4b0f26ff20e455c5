// fwd_pattern_ku8w.cu -- the pattern-tile kernels and launchers of kind
// kU8W: uint8 at larger bins (one decimated sample per word).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kU8W)
