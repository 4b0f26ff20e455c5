// fwd_pattern_batch_ku16.cu -- the persistent batch pattern kernels and launcher of kind
// kU16: uint16 (one sample per word, unpacked).
#include "pattern_kernels.cuh"

DD_PATTERN_KIND_BATCH(kU16)
