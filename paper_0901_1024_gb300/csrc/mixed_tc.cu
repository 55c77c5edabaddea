// One persistent launch per RK stage over packs of several orders (1..4).
//
// Each CTA belongs to one group (a packed mesh of one order, with its own
// fields and time steps) and runs that order's fused stage (tc_stage_body) as
// CTA `blockIdx.x - first` of the group's `count` CTAs, so the packs of every
// order advance in the same grid, side by side on the SMs, instead of one
// launch per order in sequence.  A packed element performs exactly the
// arithmetic of the per-order kernel, so results are bit-identical to it.
#include "launch.cuh"
#include "tc_stage.cuh"

namespace dgdev {

namespace {

template <int N> constexpr int tc_smem() {
  return TcDims<N>::SMEM > 120 * 1024 ? TcDims<N>::SMEM : 120 * 1024;
}
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kMixedTcSmem = cmax(cmax(tc_smem<1>(), tc_smem<2>()), cmax(tc_smem<3>(), tc_smem<4>()));
static_assert(TcDims<1>::THREADS == 640 && TcDims<4>::THREADS == 640, "one CTA shape");

__device__ __forceinline__ int mixed_group(const MixedArgs& M) {
  int gi = 0;
  while (gi + 1 < M.ngroups && int(blockIdx.x) >= M.g[gi + 1].first) ++gi;
  return gi;
}

__global__ void __launch_bounds__(640, 1) tc_mixed_kernel(const __grid_constant__ MixedArgs M) {
  pdl_launch_dependents();
  const MixedGroup& g = M.g[mixed_group(M)];
  const int cta = int(blockIdx.x) - g.first;
  switch (g.N * 2 + g.ext) {
    case 2: tc_stage_body<1, true, false>(g.a, cta, g.count); break;
    case 3: tc_stage_body<1, true, true>(g.a, cta, g.count); break;
    case 4: tc_stage_body<2, true, false>(g.a, cta, g.count); break;
    case 5: tc_stage_body<2, true, true>(g.a, cta, g.count); break;
    case 6: tc_stage_body<3, true, false>(g.a, cta, g.count); break;
    case 7: tc_stage_body<3, true, true>(g.a, cta, g.count); break;
    case 8: tc_stage_body<4, true, false>(g.a, cta, g.count); break;
    case 9: tc_stage_body<4, true, true>(g.a, cta, g.count); break;
    default: break;
  }
}

}  // namespace

cudaError_t launch_tc_mixed(const MixedArgs& m, int grid, cudaStream_t s) {
  static bool attr[16] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (!attr[dev & 15]) {
    err = cudaFuncSetAttribute(tc_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kMixedTcSmem);
    if (err != cudaSuccess) return err;
    attr[dev & 15] = true;
  }
  if (grid <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(640);
  cfg.dynamicSmemBytes = kMixedTcSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_mixed_kernel, m);
}

}  // namespace dgdev
