// fd_batch_d3.cu -- the batched layout kernel for dim = 3 (one translation
// unit per dimension so that they build in parallel).
#define FD_BATCH_DIM 3
#include "fd_batch_inst.cuh"
