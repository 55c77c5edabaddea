// Stage kernel instantiation for order N=2.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(2)
