// Stage kernel instantiation for order N=1.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(1)
