// fwd_pattern_batch_ku4.cu -- the persistent batch pattern kernels and launcher of kind
// kU4: 4-bit samples (pairs in 16-bit lanes, unpacked from staged nibbles).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kU4)
