// Stage kernel instantiation for order N=6.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(6)
