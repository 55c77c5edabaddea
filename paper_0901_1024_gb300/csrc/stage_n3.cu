// Stage kernel instantiation for order N=3.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(3)
