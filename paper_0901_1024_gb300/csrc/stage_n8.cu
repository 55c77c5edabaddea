// Stage kernel instantiation for order N=8.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(8)
