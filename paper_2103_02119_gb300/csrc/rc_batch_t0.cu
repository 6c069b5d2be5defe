// rc_batch_t0.cu -- one of the batch's constant-memory lattice tables and its
// kernels (see batch_table.cuh); a translation unit of its own so that the
// table has a constant bank of its own.
#define LBM_BATCH_SLOT 0
#include "batch_table.cuh"
