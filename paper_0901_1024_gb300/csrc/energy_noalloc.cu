// dg_energy_noalloc: the discrete energy computed without any allocation.
//
// Some callers must not allocate device memory while they run: a serving
// process whose HBM is carved up ahead of time by its own pool and budget, or
// a time loop that has to keep cudaMalloc/cudaFree (which may synchronise the
// whole device) out of its steady state.  For them this entry point computes
// the same energy as dg_energy(), but its scratch -- one FP64 partial sum per
// block of 64 tetrahedra -- lives in the file-scope device array below instead
// of a buffer the library allocates.  The array is part of the library image:
// every GPU that loads the library holds it (512 KiB) until the process exits.
//
// Limits and sharing: at most kMaxBlocks partial sums, i.e. K <= 4 194 304
// tetrahedra; larger meshes are rejected with DG_ERR_ARG.  Every call, on any
// mesh and any stream of a device, uses the same array, and it keeps the last
// call's contents; each call writes every slot it later reads, so nothing has
// to be cleared, but calls that overlap on the GPU race on it.
//
// Unlike dg_energy() the call does not synchronise: it neither reads the
// pipeline status word of the stage kernels nor checks the energy for
// finiteness (callers test the result themselves, or call dg_energy).
#include <mutex>
#include <string>

#include <cuda.h>            // CUcontext / CUresult types only (no driver library link)
#include <cuda_runtime.h>

#include "device.h"
#include "dg_internal.h"

namespace {

constexpr int kElemsPerBlock = 64;        // 8 warps x 8 tetrahedra
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 65536;         // scratch slots (FP64) = 512 KiB
constexpr int kSumThreads = 1024;

static __device__ __align__(256) double g_energy_partials[kMaxBlocks];

// Block b adds J_k u_kc^T M u_kc (FP32 per element, FP64 across elements) over
// its 64 tetrahedra in a fixed order and writes partials[b].
__global__ void __launch_bounds__(kThreads)
energy_block_sums(const float* __restrict__ u, const float* __restrict__ M,
                  const float* __restrict__ geo, const float4* __restrict__ mat, int K, int Np,
                  double* partials) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int q = 0; q < kElemsPerBlock / (kThreads / 32); ++q) {
    const int k = blockIdx.x * kElemsPerBlock + warp * (kElemsPerBlock / (kThreads / 32)) + q;
    if (k >= K) break;
    float ek = 0.f;
    const float4 mw = mat ? __ldg(mat + size_t(k) * dgdev::kMatVecs) : make_float4(1.f, 1.f, 1.f, 1.f);
    for (int c = 0; c < 6; ++c) {
      const float* uk = u + (size_t(c) * K + k) * Np;
      const float w = c < 3 ? mw.z : mw.w;        // eps for E, mu for H (1 in vacuum)
      for (int i = lane; i < Np; i += 32) {
        float s = 0.f;
        for (int j = 0; j < Np; ++j) s = fmaf(__ldg(M + j * Np + i), __ldg(uk + j), s);
        ek = fmaf(w * __ldg(uk + i), s, ek);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ek += __shfl_xor_sync(0xffffffffu, ek, o);
    acc += double(geo[size_t(k) * dgdev::kGeoWords + 9]) * double(ek);
  }
  __shared__ double sw[kThreads / 32];
  if (lane == 0) sw[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += sw[w];
    partials[blockIdx.x] = t;
  }
}

// One block: thread t adds a contiguous run of partials in order, then a
// fixed-shape tree in shared memory; writes 1/2 of the total to *out.
__global__ void __launch_bounds__(kSumThreads)
energy_final_sum(const double* __restrict__ partials, int n, double* out) {
  __shared__ double s[kSumThreads];
  const int t = threadIdx.x;
  const int chunk = (n + kSumThreads - 1) / kSumThreads;
  double a = 0.0;
  for (int i = t * chunk; i < min(n, (t + 1) * chunk); ++i) a += partials[i];
  s[t] = a;
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if (t < w) s[t] += s[t + w];
    __syncthreads();
  }
  if (t == 0) out[0] = 0.5 * s[0];
}

// Device address of g_energy_partials per device, looked up with that device
// current on the first call made on it, and again whenever the device's
// current context has changed since (after cudaDeviceReset the module is
// loaded anew and the array gets a new address).  cuCtxGetCurrent is reached
// through the runtime's driver entry points, so the library needs no link
// against the driver library.
using CtxGetCurrent = CUresult (*)(CUcontext*);
std::mutex g_mu;
struct SymbolAddr {
  CUcontext ctx = nullptr;
  void* addr = nullptr;
};
SymbolAddr g_addr[64];

CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrent>(p);
  }();
  return fn;
}

struct LaunchCtx {
  const float* u;
  const float* M;
  const float* geo;
  const float4* mat;
  int K, Np, blocks;
  double* partials;
  double* energy;
  cudaStream_t s;
};

int launch_block_sums(void* p) {
  const LaunchCtx& c = *static_cast<const LaunchCtx*>(p);
  energy_block_sums<<<c.blocks, kThreads, 0, c.s>>>(c.u, c.M, c.geo, c.mat, c.K, c.Np, c.partials);
  return static_cast<int>(cudaGetLastError());
}

int launch_final_sum(void* p) {
  const LaunchCtx& c = *static_cast<const LaunchCtx*>(p);
  energy_final_sum<<<1, kSumThreads, 0, c.s>>>(c.partials, c.blocks, c.energy);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace

extern "C" int dg_energy_noalloc(dg_mesh* m, const float* u, double* energy, void* stream) {
  if (!m) { dg::set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (!u || !energy) { dg::set_error("u or energy is NULL"); return DG_ERR_ARG; }
  if (m->N == 0) { dg::set_error("dg_set_order() has not been called"); return DG_ERR_STATE; }
  if (m->K > int64_t(kMaxBlocks) * kElemsPerBlock) {
    dg::set_error("dg_energy_noalloc supports at most 4194304 tetrahedra (K = " +
                  std::to_string(m->K) + "); use dg_energy");
    return DG_ERR_ARG;
  }
  std::string err;
  const float* M = nullptr;
  const void* geo = nullptr;
  const void* mat = nullptr;
  int64_t K = 0;
  int Np = 0;
  if (int rc = dg::device_resident(m, &M, &geo, &mat, &K, &Np, err)) { dg::set_error(err); return rc; }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    dg::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return DG_ERR_CUDA;
  }
  void* partials = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    CUcontext ctx = nullptr;
    if (CtxGetCurrent get = ctx_get_current()) get(&ctx);
    if (!g_addr[dev].addr || g_addr[dev].ctx != ctx) {
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_energy_partials);
      if (e != cudaSuccess) {
        g_addr[dev] = SymbolAddr{};
        dg::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return DG_ERR_CUDA;
      }
      // the first lookup of a context happens before it is cached, after any
      // lazy module load, so the context is read again
      if (CtxGetCurrent get = ctx_get_current()) get(&ctx);
      g_addr[dev] = SymbolAddr{ctx, addr};
    }
    partials = g_addr[dev].addr;
  }
  LaunchCtx c{u, M, static_cast<const float*>(geo), static_cast<const float4*>(mat),
              static_cast<int>(K), Np, static_cast<int>((K + kElemsPerBlock - 1) / kElemsPerBlock),
              static_cast<double*>(partials), energy, static_cast<cudaStream_t>(stream)};
  // launches are traced (dg_trace_enable) like those of dg_energy: kinds 2 and 3
  e = static_cast<cudaError_t>(dg::trace_launch(m, stream, 2, launch_block_sums, &c));
  if (e == cudaSuccess)
    e = static_cast<cudaError_t>(dg::trace_launch(m, stream, 3, launch_final_sum, &c));
  if (e != cudaSuccess) {
    dg::set_error(std::string("energy kernel launch: ") + cudaGetErrorString(e));
    return DG_ERR_CUDA;
  }
  m->last_launches = 2;
  return DG_OK;
}
