// Stage kernel instantiation for order N=4.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(4)
