// Tensor-core stage kernel instantiation for order N=6 (operator in tensor memory).
#include "tc_stage_t.cuh"
DG_INSTANTIATE_TT_STAGE(6)
