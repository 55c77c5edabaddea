// Tensor-core stage kernel instantiation for order N=7 (operator in tensor
// memory, Op_lo's last k-steps in shared memory).
#include "tc_stage_t.cuh"
DG_INSTANTIATE_TT_STAGE(7)
