// fwd_pattern_ku16.cu -- the pattern-tile kernels and launchers of kind
// kU16: uint16 (one sample per word, unpacked).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kU16)
