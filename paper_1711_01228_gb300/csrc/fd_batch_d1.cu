// fd_batch_d1.cu -- the batched layout kernel for dim = 1 (one translation
// unit per dimension so that they build in parallel).
#define FD_BATCH_DIM 1
#include "fd_batch_inst.cuh"
