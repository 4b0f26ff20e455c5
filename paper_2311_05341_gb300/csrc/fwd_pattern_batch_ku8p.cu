// fwd_pattern_batch_ku8p.cu -- the persistent batch pattern kernels and launcher of kind
// kU8P: uint8 or 4-bit from the packed copy.
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kU8P)
