// fd_batch_d2.cu -- the batched layout kernel for dim = 2 (one translation
// unit per dimension so that they build in parallel).
#define FD_BATCH_DIM 2
#include "fd_batch_inst.cuh"
