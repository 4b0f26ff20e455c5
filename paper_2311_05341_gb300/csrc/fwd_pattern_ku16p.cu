// fwd_pattern_ku16p.cu -- the pattern-tile kernels and launchers of kind
// kU16P: uint16 from the widened copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND(kU16P)
