// fwd_pattern_ku8p.cu -- the pattern-tile kernels and launchers of kind
// kU8P: uint8 or 4-bit from the packed copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kU8P)
