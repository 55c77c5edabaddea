// Stage kernel instantiation for order N=7.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(7)
