// fwd_pattern_ku8.cu -- the pattern-tile kernels and launchers of kind
// kU8: uint8 at bin 1 (pairs of samples in 16-bit lanes, unpacked from staged bytes).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kU8)
