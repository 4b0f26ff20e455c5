// fwd_pattern_batch_ku8w.cu -- the persistent batch pattern kernels and launcher of kind
// kU8W: uint8 at larger bins (one decimated sample per word).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kU8W)
