// One persistent launch per RK stage over packs of orders 5 and 6 (the
// tensor-core stage with the operator in tensor memory): as mixed_tc.cu, each
// CTA runs its group's stage (tt_stage_body) as CTA `blockIdx.x - first` of
// the group's `count` CTAs.  (Orders 5, 6 use 512-thread CTAs with up to 127
// registers per thread, orders 1..4 640-thread CTAs with at most 96, so the two
// families launch separately.)
#include "launch.cuh"
#include "tc_stage_t.cuh"

namespace dgdev {

namespace {

template <int N> constexpr int tt_smem() {
  return TtDims<N>::SMEM > 120 * 1024 ? TtDims<N>::SMEM : 120 * 1024;
}
constexpr int kMixedTtSmem = tt_smem<5>() > tt_smem<6>() ? tt_smem<5>() : tt_smem<6>();
static_assert(TtDims<5>::THREADS == TtDims<6>::THREADS, "one CTA shape");

__global__ void __launch_bounds__(TtDims<6>::THREADS, 1)
tt_mixed_kernel(const __grid_constant__ MixedArgs M) {
  pdl_launch_dependents();
  int gi = 0;
  while (gi + 1 < M.ngroups && int(blockIdx.x) >= M.g[gi + 1].first) ++gi;
  const MixedGroup& g = M.g[gi];
  const int cta = int(blockIdx.x) - g.first;
  switch (g.N * 2 + g.ext) {
    case 10: tt_stage_body<5, true, false>(g.a, cta, g.count); break;
    case 11: tt_stage_body<5, true, true>(g.a, cta, g.count); break;
    case 12: tt_stage_body<6, true, false>(g.a, cta, g.count); break;
    case 13: tt_stage_body<6, true, true>(g.a, cta, g.count); break;
    default: break;
  }
}

}  // namespace

cudaError_t launch_tt_mixed(const MixedArgs& m, int grid, cudaStream_t s) {
  static bool attr[16] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (!attr[dev & 15]) {
    err = cudaFuncSetAttribute(tt_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kMixedTtSmem);
    if (err != cudaSuccess) return err;
    attr[dev & 15] = true;
  }
  if (grid <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TtDims<6>::THREADS);
  cfg.dynamicSmemBytes = kMixedTtSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tt_mixed_kernel, m);
}

}  // namespace dgdev
