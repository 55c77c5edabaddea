// Stage kernel instantiation for order N=5.
#include "stage_kernel.cuh"
DG_INSTANTIATE_STAGE(5)
