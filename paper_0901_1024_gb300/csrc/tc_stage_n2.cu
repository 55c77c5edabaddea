// Tensor-core stage kernel instantiation for order N=2.
#include "tc_stage.cuh"
DG_INSTANTIATE_TC_STAGE(2)
