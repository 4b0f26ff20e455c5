// fwd_pattern_batch_ku16p.cu -- the persistent batch pattern kernels and launcher of kind
// kU16P: uint16 from the widened copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kU16P)
