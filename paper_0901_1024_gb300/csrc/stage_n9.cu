// Stage kernel instantiation for order N=9.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(9)
