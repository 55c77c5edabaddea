// Device buffers of a mesh, kernel dispatch, the energy reduction and the
// host-facing device operations behind the C ABI.
#include <algorithm>
#include <cstdint>
#include <initializer_list>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device.h"
#include "dg_internal.h"
#include "tcgen05.cuh"

namespace dgdev {

template <int N>
cudaError_t launch_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s, int shape);

template <int N>
cudaError_t launch_tc_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s);
template <int N>
cudaError_t launch_tt_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s);

cudaError_t launch_tc_stage(int N, bool rk, const StageArgs& a, int num_sms, cudaStream_t s) {
  switch (N) {
    case 1: return launch_tc_stage_n<1>(rk, a, num_sms, s);
    case 2: return launch_tc_stage_n<2>(rk, a, num_sms, s);
    case 3: return launch_tc_stage_n<3>(rk, a, num_sms, s);
    case 4: return launch_tc_stage_n<4>(rk, a, num_sms, s);
    case 5: return launch_tt_stage_n<5>(rk, a, num_sms, s);
    case 6: return launch_tt_stage_n<6>(rk, a, num_sms, s);
    case 7: return launch_tt_stage_n<7>(rk, a, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stage(int N, bool rk, const StageArgs& a, int num_sms, cudaStream_t s,
                         int shape) {
  switch (N) {
    case 1: return launch_stage_n<1>(rk, a, num_sms, s, shape);
    case 2: return launch_stage_n<2>(rk, a, num_sms, s, shape);
    case 3: return launch_stage_n<3>(rk, a, num_sms, s, shape);
    case 4: return launch_stage_n<4>(rk, a, num_sms, s, shape);
    case 5: return launch_stage_n<5>(rk, a, num_sms, s, shape);
    case 6: return launch_stage_n<6>(rk, a, num_sms, s, shape);
    case 7: return launch_stage_n<7>(rk, a, num_sms, s, shape);
    case 8: return launch_stage_n<8>(rk, a, num_sms, s, shape);
    case 9: return launch_stage_n<9>(rk, a, num_sms, s, shape);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------- energy -----
// E = 1/2 sum_k J_k sum_c u_kc^T M u_kc.  Each block writes one FP64 partial
// (its threads' sums, added in a fixed order) and a one-warp kernel adds the
// partials in a fixed order, so the result is deterministic.
constexpr int kEnergyThreads = 256;
constexpr int kEnergyRows = 128;      // field rows (c, k) per block pass, row kernel

// Row kernel (orders 1, 2, 3, 5): a block stages 128 consecutive field rows (c, k) in shared
// memory per pass (row stride NP | 1: conflict-free), thread r then keeps row r
// in registers and forms u^T M u from M's rows, read as broadcast 16-byte loads.
// The rows arrive by 4-byte cp.async copies (a pass's copies are all in flight
// at once, coalesced); where shared memory allows four blocks per SM the next
// pass's copies are issued before the current pass is computed.
template <int NP>
struct EnergyRowsShape {
  static constexpr int NP4 = (NP + 3) & ~3, RS = NP | 1;
  // Up to 56 nodes M is used as its upper triangle (M symmetric:
  // u^T M u = sum_i u_i (M_ii u_i + 2 sum_{j>i} M_ij u_j)), row i holding
  // M_ii, 2 M_i,i+1, ..., 2 M_i,NP-1 from a 16-byte boundary; above that the
  // full matrix, row-padded to NP4.
  static constexpr bool TRI = NP <= 56;
  __host__ __device__ static constexpr int tri_off(int i) {
    int o = 0;
    for (int r = 0; r < i; ++r) o += (NP - r + 3) & ~3;
    return o;
  }
  static constexpr int M_FLOATS = TRI ? tri_off(NP) : NP * NP4, U_FLOATS = kEnergyRows * RS;
  static constexpr int NBUF = (M_FLOATS + 2 * U_FLOATS) * 4 <= 56 * 1024 ? 2 : 1;
  static constexpr int BYTES = (M_FLOATS + NBUF * U_FLOATS) * 4;
};

template <int NP>
__global__ void __launch_bounds__(kEnergyRows) energy_rows_kernel(const EnergyArgs A) {
  using S = EnergyRowsShape<NP>;
  constexpr int NP4 = S::NP4, RS = S::RS, NBUF = S::NBUF;
  extern __shared__ __align__(16) float esm[];
  float* sM = esm;                       // [NP][NP4], zero padded
  float* sU = esm + S::M_FLOATS;         // [NBUF][kEnergyRows][RS]
  __shared__ int64_t sRow[NBUF][kEnergyRows];
  if constexpr (S::TRI) {
    for (int r = 0; r < NP; ++r)         // row r: columns r .. NP-1, zero padded
      for (int c = threadIdx.x; c < ((NP - r + 3) & ~3); c += kEnergyRows)
        sM[S::tri_off(r) + c] = r + c < NP ? (c ? 2.f : 1.f) * __ldg(A.M + r * NP + r + c) : 0.f;
  } else {
    for (int i = threadIdx.x; i < NP * NP4; i += kEnergyRows) {
      const int r = i / NP4, c = i - r * NP4;
      sM[i] = c < NP ? __ldg(A.M + r * NP + c) : 0.f;
    }
  }
  // rows (c, k) for k0 <= k < k1, numbered c * Kr + (k - k0); pass p of this
  // block covers rows [r0(p), r0(p) + 128)
  const int64_t Kr = A.k1 - A.k0, rows = 6 * Kr;
  const int64_t first = int64_t(blockIdx.x) * kEnergyRows, stride = int64_t(gridDim.x) * kEnergyRows;
  // thread t's row of a pass: its global offset (published for the copies);
  // returns its weight J_k (times eps_k for E rows, mu_k for H rows with
  // materials), loaded a pass ahead with two buffers (> 0), or -1 for no row
  auto row_of = [&](int64_t r0, int b) -> float {
    const int64_t g = r0 + threadIdx.x;
    if (g >= rows) return -1.f;
    const int64_t c = g / Kr, k = A.k0 + (g - c * Kr);
    sRow[b][threadIdx.x] = (c * A.K + k) * NP;
    const float J = __ldg(reinterpret_cast<const float*>(A.geo) + k * kGeoWords + 9);
    if (!A.mat) return J;
    const float4 w = __ldg(A.mat + k * kMatVecs);
    return J * (c < 3 ? w.z : w.w);
  };
  auto issue = [&](int64_t r0, int b) {
    if (r0 < rows) {
      const int nr = int(rows - r0 < kEnergyRows ? rows - r0 : kEnergyRows);
      float* dst = sU + b * S::U_FLOATS;
      for (int i = threadIdx.x; i < nr * NP; i += kEnergyRows) {
        const int r = i / NP, j = i - r * NP;
        tc::cp_async4(dst + r * RS + j, A.u + sRow[b][r] + j);
      }
    }
    tc::cp_async_commit();               // possibly empty: keeps the group count uniform
  };
  double acc = 0.0;
  float J_cur = -1.f;
  if constexpr (NBUF == 2) {
    J_cur = row_of(first, 0);
    __syncthreads();
    issue(first, 0);
  }
  for (int p = 0;; ++p) {
    const int64_t r0 = first + p * stride;
    const int b = NBUF == 2 ? (p & 1) : 0;
    float J_next = -1.f;
    // row offsets of the pass to issue (the next one with two buffers, else
    // this one); its buffer was last read before the previous barrier
    if constexpr (NBUF == 2) {
      if (r0 + stride < rows) J_next = row_of(r0 + stride, b ^ 1);
    } else {
      if (r0 < rows) J_cur = row_of(r0, 0);
    }
    __syncthreads();                     // offsets visible; the previous pass is consumed
    if constexpr (NBUF == 2) issue(r0 + stride, b ^ 1);
    else issue(r0, 0);
    tc::cp_async_wait_group<NBUF - 1>(); // this thread's copies of pass p have landed
    __syncthreads();                     // everyone's have
    if (r0 >= rows) break;
    const float* su = sU + b * S::U_FLOATS + threadIdx.x * RS;
    if (J_cur >= 0.f) {
      float u[NP4];
#pragma unroll
      for (int j = 0; j < NP4; ++j) u[j] = j < NP ? su[j] : 0.f;
      float e = 0.f;
      if constexpr (S::TRI) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const float4* Mi = reinterpret_cast<const float4*>(sM + S::tri_off(i));
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int q = 0; q < (NP - i + 3) / 4; ++q) {
            const float4 m4 = Mi[q];
            const int j = i + 4 * q;
            s0 = fmaf(m4.x, u[j], s0);
            if (j + 1 < NP) s1 = fmaf(m4.y, u[j + 1], s1);
            if (j + 2 < NP) s0 = fmaf(m4.z, u[j + 2], s0);
            if (j + 3 < NP) s1 = fmaf(m4.w, u[j + 3], s1);
          }
          e = fmaf(u[i], s0 + s1, e);
        }
      } else {
#pragma unroll 1
        for (int i = 0; i < NP; ++i) {
          const float4* Mi = reinterpret_cast<const float4*>(sM + i * NP4);
          float s0 = 0.f, s1 = 0.f;        // two chains for instruction-level parallelism
#pragma unroll
          for (int j4 = 0; j4 < NP4 / 4; ++j4) {
            const float4 m4 = Mi[j4];
            s0 = fmaf(m4.x, u[4 * j4], s0);
            s1 = fmaf(m4.y, u[4 * j4 + 1], s1);
            s0 = fmaf(m4.z, u[4 * j4 + 2], s0);
            s1 = fmaf(m4.w, u[4 * j4 + 3], s1);
          }
          e = fmaf(su[i], s0 + s1, e);
        }
      }
      acc += double(J_cur) * double(e);
    }
    if constexpr (NBUF == 2) J_cur = J_next;
  }
  tc::cp_async_wait_all();
  __shared__ double sw[kEnergyRows / 32];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kEnergyRows / 32; ++w) t += sw[w];
    A.partials[blockIdx.x] = t;
  }
}

// Orders 4 and 6..9: M (symmetric) in shared memory as its weighted upper triangle,
// T_ji = M_ij for j = i, 2 M_ij for j > i, 0 below (row j padded to NP8 floats),
// so u^T M u = sum_i u_i s_i with s_i = sum_{j >= i} T_ji u_j.  Each thread takes
// RPT field rows (c, k) of a pass, staged by 4-byte cp.async copies with an odd
// row stride (conflict-free 4-byte reads), and forms s_i for 8 outputs i0..i0+7
// at a time over j >= i0 (row j of T read as two broadcast 16-byte loads, used
// for all RPT rows of the thread), then e += sum_i u_i s_i.  FP32 products,
// FP64 sums of the weighted rows.
template <int NP, int THREADS, int RPT>
struct EnergyWideShape {
  static constexpr int NP8 = (NP + 7) & ~7, RS = NP | 1, ROWS = THREADS * RPT;
  static constexpr int BYTES = (NP * NP8 + ROWS * RS) * 4;
  static_assert(BYTES <= 226 * 1024, "shared memory");
};

template <int NP, int THREADS, int RPT>
__global__ void __launch_bounds__(THREADS) energy_wide_kernel(const EnergyArgs A) {
  using S = EnergyWideShape<NP, THREADS, RPT>;
  constexpr int NP8 = S::NP8, RS = S::RS, ROWS = S::ROWS;
  extern __shared__ __align__(16) float esm[];
  float* sM = esm;                       // T: [NP][NP8], zero padded
  float* sU = esm + NP * NP8;            // [ROWS][RS]
  __shared__ int64_t sRow[ROWS];
  for (int i = threadIdx.x; i < NP * NP8; i += THREADS) {
    const int r = i / NP8, c = i - r * NP8;              // T_rc
    sM[i] = c < NP && r >= c ? (r > c ? 2.f : 1.f) * __ldg(A.M + r * NP + c) : 0.f;
  }
  const int64_t Kr = A.k1 - A.k0, rows = 6 * Kr;
  double acc = 0.0;
  for (int64_t r0 = int64_t(blockIdx.x) * ROWS; r0 < rows; r0 += int64_t(gridDim.x) * ROWS) {
    float w[RPT];                        // J_k (times eps_k or mu_k), or 0: no row
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int lr = threadIdx.x + q * THREADS;
      const int64_t g = r0 + lr;
      w[q] = 0.f;
      if (g < rows) {
        const int64_t c = g / Kr, k = A.k0 + (g - c * Kr);
        sRow[lr] = (c * A.K + k) * NP;
        const float J = __ldg(reinterpret_cast<const float*>(A.geo) + k * kGeoWords + 9);
        w[q] = J;
        if (A.mat) {
          const float4 m = __ldg(A.mat + k * kMatVecs);
          w[q] = J * (c < 3 ? m.z : m.w);
        }
      }
    }
    __syncthreads();                     // row offsets visible; the previous pass is consumed
    const int nr = int(rows - r0 < ROWS ? rows - r0 : ROWS);
    for (int i = threadIdx.x; i < nr * NP; i += THREADS) {
      const int r = i / NP, j = i - r * NP;
      tc::cp_async4(sU + r * RS + j, A.u + sRow[r] + j);
    }
    tc::cp_async_commit();
    tc::cp_async_wait_all();
    __syncthreads();
    if (threadIdx.x < nr) {
      const float* u0 = sU + threadIdx.x * RS;
      float e[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) e[q] = 0.f;
#pragma unroll 1
      for (int i0 = 0; i0 < NP; i0 += 8) {
        float sacc[RPT][8];
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) sacc[q][ii] = 0.f;
#pragma unroll 4
        for (int j = i0; j < NP; ++j) {
          const float4 m0 = *reinterpret_cast<const float4*>(sM + j * NP8 + i0);
          const float4 m1 = *reinterpret_cast<const float4*>(sM + j * NP8 + i0 + 4);
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            const float uj = u0[q * THREADS * RS + j];
            sacc[q][0] = fmaf(m0.x, uj, sacc[q][0]);
            sacc[q][1] = fmaf(m0.y, uj, sacc[q][1]);
            sacc[q][2] = fmaf(m0.z, uj, sacc[q][2]);
            sacc[q][3] = fmaf(m0.w, uj, sacc[q][3]);
            sacc[q][4] = fmaf(m1.x, uj, sacc[q][4]);
            sacc[q][5] = fmaf(m1.y, uj, sacc[q][5]);
            sacc[q][6] = fmaf(m1.z, uj, sacc[q][6]);
            sacc[q][7] = fmaf(m1.w, uj, sacc[q][7]);
          }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int ii = 0; ii < 8; ++ii)
            if (i0 + ii < NP) e[q] = fmaf(u0[q * THREADS * RS + i0 + ii], sacc[q][ii], e[q]);
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (threadIdx.x + q * THREADS < nr) acc += double(w[q]) * double(e[q]);
    }
  }
  tc::cp_async_wait_all();
  __shared__ double sw[(THREADS + 31) / 32];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (THREADS + 31) / 32; ++w) t += sw[w];
    A.partials[blockIdx.x] = t;
  }
}

// Any order: one warp per element, lane i forms (M u_c)_i (M symmetric, read
// column-wise = coalesced) and u_i (M u_c)_i in FP32, scaled by J_k in FP64.
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(const EnergyArgs A) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kEnergyThreads / 32;
  double acc = 0.0;
  for (int k = A.k0 + blockIdx.x * nw + warp; k < A.k1; k += gridDim.x * nw) {
    float ek = 0.f;
    const float4 mw = A.mat ? __ldg(A.mat + size_t(k) * kMatVecs) : make_float4(1.f, 1.f, 1.f, 1.f);
    for (int c = 0; c < 6; ++c) {
      const float* uk = A.u + (size_t(c) * A.K + k) * A.Np;
      const float w = c < 3 ? mw.z : mw.w;          // eps for E, mu for H (1 in vacuum)
      for (int i = lane; i < A.Np; i += 32) {
        float s = 0.f;
        for (int j = 0; j < A.Np; ++j) s = fmaf(__ldg(A.M + j * A.Np + i), __ldg(uk + j), s);
        ek = fmaf(w * __ldg(uk + i), s, ek);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ek += __shfl_xor_sync(0xffffffffu, ek, o);
    const float J = reinterpret_cast<const float*>(A.geo)[size_t(k) * kGeoWords + 9];
    acc += double(J) * double(ek);
  }
  __shared__ double sw[nw];
  if (lane == 0) sw[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sw[w];
    A.partials[blockIdx.x] = t;
  }
}

// One warp: lane l adds partials l, l + 32, ... in order, then a fixed
// butterfly adds the lanes.
__global__ void energy_finalize(const double* partials, int n, double* result) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) t += partials[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) result[0] = 0.5 * t;
}

int energy_grid(int num_sms) { return 4 * num_sms; }

template <int NP>
static cudaError_t launch_energy_rows(const EnergyArgs& a, int grid, cudaStream_t s) {
  constexpr int bytes = EnergyRowsShape<NP>::BYTES;
  static bool attr[16] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (!attr[dev & 15]) {
    err = cudaFuncSetAttribute(energy_rows_kernel<NP>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (err != cudaSuccess) return err;
    attr[dev & 15] = true;
  }
  energy_rows_kernel<NP><<<grid, kEnergyRows, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int NP, int THREADS, int RPT>
static cudaError_t launch_energy_wide(const EnergyArgs& a, int grid, cudaStream_t s) {
  constexpr int bytes = EnergyWideShape<NP, THREADS, RPT>::BYTES;
  auto kern = energy_wide_kernel<NP, THREADS, RPT>;
  static bool attr[16] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (!attr[dev & 15]) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (err != cudaSuccess) return err;
    attr[dev & 15] = true;
  }
  kern<<<grid, THREADS, bytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_energy_partials(const EnergyArgs& a, int grid, cudaStream_t s) {
  switch (a.Np) {
    case 4: return launch_energy_rows<4>(a, grid, s);
    case 10: return launch_energy_rows<10>(a, grid, s);
    case 20: return launch_energy_rows<20>(a, grid, s);
    case 35: return launch_energy_wide<35, 256, 2>(a, grid, s);
    case 56: return launch_energy_rows<56>(a, grid, s);
    case 84: return launch_energy_wide<84, 256, 2>(a, grid, s);
    case 120: return launch_energy_wide<120, 128, 2>(a, grid, s);
    case 165: return launch_energy_wide<165, 64, 2>(a, grid, s);
    case 220: return launch_energy_wide<220, 32, 1>(a, grid, s);
    default:
      energy_kernel<<<grid, kEnergyThreads, 0, s>>>(a);
      return cudaGetLastError();
  }
}

cudaError_t launch_energy_final(const EnergyArgs& a, int grid, cudaStream_t s) {
  energy_finalize<<<1, 32, 0, s>>>(a.partials, grid, a.result);
  return cudaGetLastError();
}

// ------------------------------------------------------- device state -----
struct DeviceState {
  int device = -1;
  int N = 0;
  int64_t K = 0;
  int Np = 0, Nfp = 0;
  int num_sms = 0;
  float4* geo = nullptr;
  float4* D4 = nullptr;
  float4* LIFT4 = nullptr;
  float* M = nullptr;
  unsigned char* fmask = nullptr;
  unsigned char* perm = nullptr;
  float* u_work = nullptr;      // second state buffer for the stage ping-pong
  float* h_u = nullptr;         // device copies for dg_step_host
  float* h_res = nullptr;
  double* partials = nullptr;   // energy partials, one per block
  double* result = nullptr;
  int egrid = 0;
  void* tcB = nullptr;          // tensor-core B pieces (orders <= kTcMaxOrder)
  float4* mat = nullptr;        // material records (meshes with materials), in the arena
  bool absorbing = false;       // some boundary face is absorbing
  float* tcgeo = nullptr;       // word-major geometry for the tensor-core stage
  int tc_geo_stride = 0;
  float tc_inv_bscale = 1.f;
  int* status = nullptr;        // pipeline status word (0 = ok)
  void* arena = nullptr;        // one allocation: geo, tcgeo, status, partials, result
  // D4, LIFT4, M, fmask, perm and tcB belong to the per-(device, order) cache
  // per-launch tracing: event pair 2i, 2i+1 around launch i
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  size_t nrec = 0;
};

void destroy_device_state(DeviceState* d) {
  if (!d) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (d->device >= 0) cudaSetDevice(d->device);
  cudaFree(d->arena); cudaFree(d->u_work); cudaFree(d->h_u); cudaFree(d->h_res);
  for (cudaEvent_t e : d->ev) cudaEventDestroy(e);
  if (cur >= 0) cudaSetDevice(cur);
  delete d;
}

}  // namespace dgdev

namespace dg {
using dgdev::DeviceState;

static int cuda_fail(cudaError_t e, const char* what, std::string& err) {
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

#define DG_CUDA(call, what)                                        \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what, err);        \
  } while (0)

template <class T>
static int upload(T** dst, const std::vector<T>& src, std::string& err) {
  DG_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), src.size() * sizeof(T)), "cudaMalloc");
  DG_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice),
          "cudaMemcpy H2D");
  return DG_OK;
}

// Launches `fn` (returning cudaError_t) and, when tracing, brackets it with a
// pair of events on stream s.
template <class F>
static cudaError_t traced(dg_mesh* m, cudaStream_t s, int kind, F&& fn) {
  DeviceState* d = m->dev;
  if (!m->trace) return fn();
  const size_t i = d->nrec;
  while (d->ev.size() < 2 * i + 2) {
    cudaEvent_t e;
    cudaError_t c = cudaEventCreate(&e);
    if (c != cudaSuccess) return c;
    d->ev.push_back(e);
  }
  if (d->kind.size() < i + 1) d->kind.resize(i + 1);
  cudaError_t c = cudaEventRecord(d->ev[2 * i], s);
  if (c != cudaSuccess) return c;
  if ((c = fn()) != cudaSuccess) return c;
  if ((c = cudaEventRecord(d->ev[2 * i + 1], s)) != cudaSuccess) return c;
  d->kind[i] = kind;
  d->nrec = i + 1;
  return cudaSuccess;
}

int ensure_device(dg_mesh* m, std::string& err);

int trace_launch(dg_mesh* m, void* stream, int kind, int (*launch)(void*), void* ctx) {
  return static_cast<int>(traced(m, static_cast<cudaStream_t>(stream), kind,
                                 [&] { return static_cast<cudaError_t>(launch(ctx)); }));
}

int device_trace_reset(dg_mesh* m, int reserve, std::string& err) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  DeviceState* d = m->dev;
  d->nrec = 0;
  while (d->ev.size() < 2 * static_cast<size_t>(reserve)) {
    cudaEvent_t e;
    DG_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    d->ev.push_back(e);
  }
  d->kind.resize(std::max(d->kind.size(), static_cast<size_t>(reserve)));
  return DG_OK;
}

int device_trace_read(dg_mesh* m, double* ms, int32_t* kind, int64_t cap, int64_t* count,
                      std::string& err) {
  DeviceState* d = m->dev;
  if (!d || d->nrec == 0) { err = "no traced launches recorded"; return DG_ERR_STATE; }
  DG_CUDA(cudaEventSynchronize(d->ev[2 * d->nrec - 1]), "cudaEventSynchronize");
  *count = static_cast<int64_t>(d->nrec);
  for (size_t i = 0; i < d->nrec && static_cast<int64_t>(i) < cap; ++i) {
    float t = 0.f;
    DG_CUDA(cudaEventElapsedTime(&t, d->ev[2 * i], d->ev[2 * i + 1]), "cudaEventElapsedTime");
    ms[i] = t;
    if (kind) kind[i] = d->kind[i];
  }
  return DG_OK;
}

// Order-dependent device operators, shared by every mesh of that order on a
// device (built once, kept for the life of the process): Dr/Ds/Dt as float4
// rows, LIFT, M, the face-node tables and the tensor-core B pieces.
struct OrderOps {
  float4* D4 = nullptr;
  float4* LIFT4 = nullptr;
  float* M = nullptr;
  unsigned char* fmask = nullptr;
  unsigned char* perm = nullptr;
  void* tcB = nullptr;
  float tc_inv_bscale = 1.f;
};

static std::mutex g_ops_mutex;
static std::map<std::pair<int, int>, OrderOps> g_ops;

static int order_ops(const dg_mesh* m, int dev, OrderOps& out, std::string& err) {
  std::lock_guard<std::mutex> lock(g_ops_mutex);
  auto it = g_ops.find({dev, m->N});
  if (it != g_ops.end()) {
    out = it->second;
    return DG_OK;
  }
  OrderOps o;
  const int Np = m->ops.Np, NF = 4 * m->ops.Nfp;
  std::vector<float4> D4(static_cast<size_t>(Np) * Np);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j)
      D4[i * Np + j] = make_float4(static_cast<float>(m->ops.Dr[i * Np + j]),
                                   static_cast<float>(m->ops.Ds[i * Np + j]),
                                   static_cast<float>(m->ops.Dt[i * Np + j]), 0.f);
  int rc;
  if ((rc = upload(&o.D4, D4, err))) return rc;
  std::vector<float4> L4(static_cast<size_t>(Np) * NF / 4);
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < NF / 4; ++q)
      L4[i * (NF / 4) + q] = make_float4(static_cast<float>(m->ops.LIFT[i * NF + 4 * q + 0]),
                                         static_cast<float>(m->ops.LIFT[i * NF + 4 * q + 1]),
                                         static_cast<float>(m->ops.LIFT[i * NF + 4 * q + 2]),
                                         static_cast<float>(m->ops.LIFT[i * NF + 4 * q + 3]));
  if ((rc = upload(&o.LIFT4, L4, err))) return rc;
  std::vector<float> Mf(m->ops.M.begin(), m->ops.M.end());
  if ((rc = upload(&o.M, Mf, err))) return rc;
  std::vector<unsigned char> fm(m->ops.Fmask.begin(), m->ops.Fmask.end());
  if ((rc = upload(&o.fmask, fm, err))) return rc;
  std::vector<unsigned char> pm(m->ops.perm.begin(), m->ops.perm.end());
  if ((rc = upload(&o.perm, pm, err))) return rc;
  if (m->N > 4 && m->N <= dgdev::kTcMaxOrder) {
    // Orders 5..7: Op = [Dr Ds Dt LIFT] (Np x KT, each derivative block padded
    // to KB columns, zero padded), scaled by 2^p, split into FP16 hi + lo, as
    // tensor-memory rows: [piece][lane = node, 128][KT / 2] words, word p of a
    // row holding columns 2p (low half) and 2p + 1.
    const int KB = dgdev::tt_kb(m->N), KT = dgdev::tt_kt(m->N), AC = dgdev::tt_acols(m->N);
    std::vector<double> Op(static_cast<size_t>(Np) * KT, 0.0);
    double mx = 0.0;
    for (int n = 0; n < Np; ++n)
      for (int k = 0; k < KT; ++k) {
        double v = 0.0;
        if (k < 3 * KB) {
          const int mu = k / KB, j = k % KB;
          const std::vector<double>& Dm = mu == 0 ? m->ops.Dr : mu == 1 ? m->ops.Ds : m->ops.Dt;
          if (j < Np) v = Dm[n * Np + j];
        } else if (k < 3 * KB + NF) {
          v = m->ops.LIFT[n * NF + (k - 3 * KB)];
        }
        Op[n * KT + k] = v;
        mx = std::max(mx, std::fabs(v));
      }
    const double sB = std::ldexp(1.0, static_cast<int>(std::floor(std::log2(16384.0 / mx))));
    o.tc_inv_bscale = static_cast<float>(1.0 / sB);
    const size_t piece = static_cast<size_t>(128) * AC * 2;      // halves
    std::vector<__half> P(2 * piece, __float2half_rn(0.f));
    for (int n = 0; n < Np; ++n)
      for (int k = 0; k < KT; ++k) {
        const float x = static_cast<float>(Op[n * KT + k] * sB);
        const __half hi = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(hi));
        const size_t off = static_cast<size_t>(n) * AC * 2 + k;   // word k / 2, half k % 2
        P[off] = hi;
        P[piece + off] = lo;
      }
    if ((rc = upload(reinterpret_cast<__half**>(&o.tcB), P, err))) return rc;
  } else if (m->N <= 4) {
    // B = [Dr Ds Dt LIFT] (Np x KT, zero padded), scaled by 2^p, split into FP16
    // hi + lo, stored in the canonical K-major core-matrix layout.
    const int KB = (Np + 1) & ~1, KT = (3 * KB + NF + 15) & ~15, NN = (Np + 15) & ~15;
    std::vector<double> B(static_cast<size_t>(NN) * KT, 0.0);
    double mx = 0.0;
    for (int n = 0; n < Np; ++n)
      for (int k = 0; k < KT; ++k) {
        double v = 0.0;
        if (k < 3 * KB) {
          const int mu = k / KB, j = k % KB;
          const std::vector<double>& Dm = mu == 0 ? m->ops.Dr : mu == 1 ? m->ops.Ds : m->ops.Dt;
          if (j < Np) v = Dm[n * Np + j];
        } else if (k < 3 * KB + NF) {
          v = m->ops.LIFT[n * NF + (k - 3 * KB)];
        }
        B[n * KT + k] = v;
        mx = std::max(mx, std::fabs(v));
      }
    const double sB = std::ldexp(1.0, static_cast<int>(std::floor(std::log2(16384.0 / mx))));
    o.tc_inv_bscale = static_cast<float>(1.0 / sB);
    const size_t piece = static_cast<size_t>(NN) * KT;
    std::vector<__half> P(2 * piece);
    for (int n = 0; n < NN; ++n)
      for (int k = 0; k < KT; ++k) {
        const float x = static_cast<float>(B[n * KT + k] * sB);
        const __half hi = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(hi));
        const size_t off = ((k / 8) * (NN / 8) + n / 8) * 64 + (n % 8) * 8 + (k % 8);
        P[off] = hi;
        P[piece + off] = lo;
      }
    if ((rc = upload(reinterpret_cast<__half**>(&o.tcB), P, err))) return rc;
  }
  g_ops[{dev, m->N}] = o;
  out = o;
  return DG_OK;
}

// Creates (or re-creates after an order change) the device copy of the mesh:
// the shared order operators plus one arena holding this mesh's geometry
// records, its tiled tensor-core geometry, the status word and the energy
// partial sums (one allocation, one copy).
int ensure_device(dg_mesh* m, std::string& err) {
  if (m->N == 0) { err = "dg_set_order() has not been called"; return DG_ERR_STATE; }
  int cur = 0;
  DG_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (m->dev && m->dev->N == m->N && m->dev->device == cur) return DG_OK;
  if (m->dev) { dgdev::destroy_device_state(m->dev); m->dev = nullptr; }
  auto* d = new DeviceState();
  m->dev = d;
  d->device = cur;
  d->N = m->N;
  d->K = m->K;
  d->Np = m->ops.Np;
  d->Nfp = m->ops.Nfp;
  DG_CUDA(cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, cur),
          "cudaDeviceGetAttribute");
  OrderOps ops;
  int rc = order_ops(m, cur, ops, err);
  if (rc) return rc;
  d->D4 = ops.D4;
  d->LIFT4 = ops.LIFT4;
  d->M = ops.M;
  d->fmask = ops.fmask;
  d->perm = ops.perm;
  d->tcB = ops.tcB;
  d->tc_inv_bscale = ops.tc_inv_bscale;
  const int64_t K = m->K;
  const int Nfp = d->Nfp, NF = 4 * Nfp;
  const bool tc = d->N <= dgdev::kTcMaxOrder;
  const int E = dgdev::tc_tile_elems(d->N);
  const int64_t ntiles = (K + E - 1) / E;
  d->tc_geo_stride = tc ? dgdev::tc_geo_floats(d->N) : 0;
  d->egrid = dgdev::energy_grid(d->num_sms);
  // arena layout (bytes, each part 256-byte aligned)
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t geo_b = static_cast<size_t>(K) * dgdev::kGeoWords * 4;
  const size_t mat_b = m->eps.empty() ? 0 : static_cast<size_t>(K) * dgdev::kMatVecs * 16;
  const size_t tcg_b = tc ? static_cast<size_t>(ntiles) * d->tc_geo_stride * 4 : 0;
  const size_t o_mat = up(geo_b), o_tcg = o_mat + up(mat_b), o_part = o_tcg + up(tcg_b);
  const size_t o_res = o_part + up(sizeof(double) * d->egrid), o_stat = o_res + 256;
  const size_t total = o_stat + 256;
  std::vector<unsigned char> host(o_part, 0);

  // geometry records
  float* geo = reinterpret_cast<float*>(host.data());
  for (int64_t k = 0; k < K; ++k) {
    float* g = &geo[k * dgdev::kGeoWords];
    for (int a = 0; a < 9; ++a) g[a] = static_cast<float>(m->metric[a * K + k]);
    g[9] = static_cast<float>(m->J[k]);
    uint32_t codes = 0;
    for (int f = 0; f < 4; ++f) {
      const int c = m->nbr_code[4 * k + f];
      const bool absorbing = c < 0 && !m->bc.empty() && m->bc[4 * k + f] == DG_BC_ABSORBING;
      d->absorbing = d->absorbing || absorbing;
      codes |= (absorbing ? dgdev::kAbsorbingCode : static_cast<uint32_t>(c + 1)) << (8 * f);
      for (int dd = 0; dd < 3; ++dd)
        g[12 + 4 * f + dd] = static_cast<float>(m->normals[(dd * K + k) * 4 + f]);
      g[15 + 4 * f] = static_cast<float>(m->Fscale[4 * k + f]);
      const int32_t nb = m->nbr_elem[4 * k + f];
      std::memcpy(&g[28 + f], &nb, 4);
    }
    std::memcpy(&g[10], &codes, 4);
  }
  if (mat_b) {
    // material records: 1/eps, 1/mu, eps, mu, then the flux coefficients of each
    // face from the impedances of both sides (the element's own on boundaries)
    float4* mr = reinterpret_cast<float4*>(host.data() + o_mat);
    for (int64_t k = 0; k < K; ++k) {
      const double e = m->eps[k], u = m->mu[k], zm = std::sqrt(u / e);
      mr[k * dgdev::kMatVecs] = make_float4(static_cast<float>(1.0 / e), static_cast<float>(1.0 / u),
                                            static_cast<float>(e), static_cast<float>(u));
      for (int f = 0; f < 4; ++f) {
        const int64_t k2 = m->nbr_code[4 * k + f] < 0 ? k : m->nbr_elem[4 * k + f];
        const double zp = std::sqrt(m->mu[k2] / m->eps[k2]), ym = 1.0 / zm, yp = 1.0 / zp;
        mr[k * dgdev::kMatVecs + 1 + f] =
            make_float4(static_cast<float>(zp), static_cast<float>(1.0 / (zm + zp)),
                        static_cast<float>(yp), static_cast<float>(1.0 / (ym + yp)));
      }
    }
  }
  if (tc) {
    // tiled geometry, one contiguous block per tile: word-major [kTcGeoWords][E]
    // (record words {0..8 metric, 10 codes, 12..27 faces, 28..31 neighbours} ->
    // words {0..8, 9, 10..25, 26..29}), then one byte per face node (e, m):
    // the node of the neighbour across face m / Nfp that matches it (0 on walls)
    float* tg = reinterpret_cast<float*>(host.data() + o_tcg);
    for (int64_t k = 0; k < K; ++k) {
      float* blk = &tg[(k / E) * d->tc_geo_stride];
      for (int w = 0; w < dgdev::kTcGeoWords; ++w) {
        const int src = w < 9 ? w : (w == 9 ? 10 : w + 2);
        blk[w * E + k % E] = geo[k * dgdev::kGeoWords + src];
      }
      unsigned char* nodes = reinterpret_cast<unsigned char*>(blk + dgdev::kTcGeoWords * E);
      for (int f = 0; f < 4; ++f) {
        const int c = m->nbr_code[4 * k + f];
        for (int j = 0; j < Nfp; ++j)
          nodes[(k % E) * NF + f * Nfp + j] =
              c < 0 ? 0 : static_cast<unsigned char>(m->ops.perm[(f * 24 + c) * Nfp + j]);
      }
    }
  }
  DG_CUDA(cudaMalloc(&d->arena, total), "cudaMalloc");
  unsigned char* base = static_cast<unsigned char*>(d->arena);
  DG_CUDA(cudaMemcpy(base, host.data(), host.size(), cudaMemcpyHostToDevice), "cudaMemcpy H2D");
  DG_CUDA(cudaMemset(base + o_stat, 0, 256), "cudaMemset");
  d->geo = reinterpret_cast<float4*>(base);
  d->mat = mat_b ? reinterpret_cast<float4*>(base + o_mat) : nullptr;
  d->tcgeo = tc ? reinterpret_cast<float*>(base + o_tcg) : nullptr;
  d->partials = reinterpret_cast<double*>(base + o_part);
  d->result = reinterpret_cast<double*>(base + o_res);
  d->status = reinterpret_cast<int*>(base + o_stat);
  return DG_OK;
}

// Tensor cores for orders 2..kTcMaxOrder (and 1 on request) unless the CUDA-core
// path is forced.
// The tensor-core kernel moves whole tiles with bulk copies, which need every
// field chunk 16-byte aligned: (K * Np) % 4 == 0 and 16-byte aligned buffers.
static bool use_tc(const dg_mesh* m, std::initializer_list<const void*> bufs) {
  if (m->stage_impl == DG_STAGE_FP32 || m->N > dgdev::kTcMaxOrder) return false;
  // at N = 1 (Np = 4) the FP32 kernel is faster unless tensor cores are asked for
  if (m->stage_impl == DG_STAGE_AUTO && m->N == 1) return false;
  if ((m->K * m->ops.Np) % 4 != 0) return false;
  for (const void* p : bufs)
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
  return true;
}

static dgdev::StageArgs stage_args(dg_mesh* m, bool tc) {
  DeviceState* d = m->dev;
  dgdev::StageArgs a{};
  a.tcB = d->tcB;
  a.tcgeo = d->tcgeo;
  a.tc_geo_stride = d->tc_geo_stride;
  a.tc_inv_bscale = d->tc_inv_bscale;
  a.status = d->status;
  a.geo = d->geo;
  a.mat = d->mat;
  a.absorbing = d->absorbing ? 1 : 0;
  a.D4 = d->D4;
  a.LIFT4 = d->LIFT4;
  a.fmask = d->fmask;
  a.perm = d->perm;
  a.K = static_cast<int>(d->K);
  a.alpha = static_cast<float>(m->alpha);
  const int E = tc ? dgdev::tc_tile_elems(d->N) : dgdev::stage_tile_elems(d->N, m->stage_shape);
  a.num_tiles = static_cast<int>((d->K + E - 1) / E);
  return a;
}

int device_rhs(dg_mesh* m, const float* u, float* rhs, void* stream, std::string& err) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_device(m, err);
  if (rc) return rc;
  const bool tc = use_tc(m, {u, rhs});
  dgdev::StageArgs a = stage_args(m, tc);
  a.u_in = u;
  a.rhs = rhs;
  DG_CUDA(traced(m, s, tc ? 5 : 1, [&] {
            return tc ? dgdev::launch_tc_stage(m->N, false, a, m->dev->num_sms, s)
                             : dgdev::launch_stage(m->N, false, a, m->dev->num_sms, s,
                                                   m->stage_shape);
          }), "stage kernel launch");
  m->last_launches = 1;
  return DG_OK;
}

// LSERK4 coefficients (Carpenter & Kennedy 1994, five stages, two registers).
static const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0,
                               -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0,
                               -1275806237668.0 / 842570457699.0};
static const double kRkB[5] = {1432997174477.0 / 9575080441755.0,
                               5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0,
                               3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};

static int step_impl(dg_mesh* m, float* u, float* res, double dt, int nsteps, cudaStream_t s,
                     std::string& err) {
  DeviceState* d = m->dev;
  const size_t n = static_cast<size_t>(6) * d->K * d->Np;
  if (!d->u_work) DG_CUDA(cudaMalloc(&d->u_work, n * sizeof(float)), "cudaMalloc work state");
  const bool tc = use_tc(m, {u, res, d->u_work});
  dgdev::StageArgs a = stage_args(m, tc);
  a.res = res;
  a.dt = static_cast<float>(dt);
  const float* src = u;
  float* dst = d->u_work;
  int64_t launches = 0;
  for (int st = 0; st < nsteps; ++st)
    for (int i = 0; i < 5; ++i) {
      a.u_in = src;
      a.u_out = dst;
      a.a = static_cast<float>(kRkA[i]);
      a.b = static_cast<float>(kRkB[i]);
      DG_CUDA(traced(m, s, tc ? 4 : 0, [&] {
                return tc ? dgdev::launch_tc_stage(m->N, true, a, d->num_sms, s)
                          : dgdev::launch_stage(m->N, true, a, d->num_sms, s, m->stage_shape);
              }), "stage kernel launch");
      ++launches;
      float* nsrc = dst;
      dst = const_cast<float*>(src);
      src = nsrc;
    }
  if (src != u)  // odd number of stages: the state sits in the work buffer
    DG_CUDA(cudaMemcpyAsync(u, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s),
            "cudaMemcpyAsync D2D");
  m->last_launches = launches;
  return DG_OK;
}

int device_stage_tile(dg_mesh* m, const float* u_in, const float* u_out, const float* res,
                      int* tile, std::string& err) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  *tile = use_tc(m, {u_in, u_out, res}) ? dgdev::tc_tile_elems(m->N)
                                        : dgdev::stage_tile_elems(m->N, m->stage_shape);
  return DG_OK;
}

int device_stage(dg_mesh* m, const float* u_in, float* u_out, float* res, int stage, double dt,
                 const float* dt_elem, void* stream, std::string& err, int64_t k0, int64_t k1) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceState* d = m->dev;
  const bool tc = use_tc(m, {u_in, u_out, res});
  dgdev::StageArgs a = stage_args(m, tc);
  if (k1 >= 0) {                        // elements [k0, k1): whole tiles of the kernel that runs
    const int E = tc ? dgdev::tc_tile_elems(m->N) : dgdev::stage_tile_elems(m->N, m->stage_shape);
    if (k0 < 0 || k1 <= k0 || k1 > m->K || k0 % E != 0 || (k1 % E != 0 && k1 != m->K)) {
      err = "the element range must be [k0, k1) with k0 and k1 multiples of the stage's tile of " +
            std::to_string(E) + " tetrahedra (or k1 = K), 0 <= k0 < k1 <= K";
      return DG_ERR_ARG;
    }
    a.tile0 = static_cast<int>(k0 / E);
    a.num_tiles = static_cast<int>((k1 + E - 1) / E - k0 / E);
  }
  a.u_in = u_in;
  a.u_out = u_out;
  a.res = res;
  a.dt = static_cast<float>(dt);
  a.dt_elem = dt_elem;
  a.a = static_cast<float>(kRkA[stage]);
  a.b = static_cast<float>(kRkB[stage]);
  DG_CUDA(traced(m, s, tc ? 4 : 0, [&] {
            return tc ? dgdev::launch_tc_stage(m->N, true, a, d->num_sms, s)
                      : dgdev::launch_stage(m->N, true, a, d->num_sms, s, m->stage_shape);
          }), "stage kernel launch");
  m->last_launches = 1;
  return DG_OK;
}

// Default cost of one tile on one SM in microseconds, orders 1..6 on the
// tensor cores (GB300: stage time x CTAs / tiles of the order sweep), used to
// split a mixed launch's CTAs when the caller gives no costs.
static double default_tile_cost(int N) {
  static const double c[7] = {1.0, 1.6, 1.9, 2.7, 3.6, 3.1, 3.9};
  return N >= 1 && N <= 6 ? c[N] : 1.0;
}

// CTAs of a mixed launch: one per group at least, `total` in all, each further
// CTA to the group whose span ceil(tiles / ctas) x cost is then the longest
// (so the groups of one launch finish together).
static std::vector<int> split_ctas(const std::vector<int64_t>& tiles,
                                   const std::vector<double>& cost, int total) {
  const size_t n = tiles.size();
  std::vector<int> c(n, 1);
  int used = static_cast<int>(n);
  auto span = [&](size_t g) {
    return static_cast<double>((tiles[g] + c[g] - 1) / c[g]) * cost[g];
  };
  while (used < total) {
    size_t best = n;
    for (size_t g = 0; g < n; ++g)
      if (c[g] < tiles[g] && (best == n || span(g) > span(best))) best = g;
    if (best == n) break;
    ++c[best];
    ++used;
  }
  return c;
}

int device_stage_multi(dg_mesh* const* ms, int n, const float* const* u_in, float* const* u_out,
                       float* const* res, const float* const* dt_elem, int stage, double dt,
                       const double* tile_cost, void* stream, std::string& err) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t launches = 0;
  std::vector<int> fam(n, 0);        // 0: its own launch (order 7, FP32), 1: orders 1..4, 2: orders 5, 6
  for (int i = 0; i < n; ++i) {
    if (int rc = ensure_device(ms[i], err)) return rc;
    if (ms[i]->dev->device != ms[0]->dev->device) {
      err = "every mesh of one call must be on the same device";
      return DG_ERR_ARG;
    }
    if (use_tc(ms[i], {u_in[i], u_out[i], res[i]})) fam[i] = ms[i]->N <= 4 ? 1 : ms[i]->N <= 6 ? 2 : 0;
  }
  for (int i = 0; i < n; ++i)
    if (fam[i] == 0) {
      if (int rc = device_stage(ms[i], u_in[i], u_out[i], res[i], stage, dt,
                                dt_elem ? dt_elem[i] : nullptr, stream, err))
        return rc;
      ++launches;
    }
  const int sms = ms[0]->dev->num_sms;
  for (int f = 1; f <= 2; ++f) {
    std::vector<int> idx;
    for (int i = 0; i < n; ++i)
      if (fam[i] == f) idx.push_back(i);
    for (size_t c0 = 0; c0 < idx.size(); c0 += dgdev::kMaxMixedGroups) {
      const size_t ng = std::min(idx.size() - c0, static_cast<size_t>(dgdev::kMaxMixedGroups));
      std::vector<int64_t> tiles(ng);
      std::vector<double> cost(ng);
      dgdev::MixedArgs M{};
      M.ngroups = static_cast<int>(ng);
      int64_t all = 0;
      for (size_t g = 0; g < ng; ++g) {
        const int i = idx[c0 + g];
        dgdev::StageArgs a = stage_args(ms[i], true);
        a.u_in = u_in[i];
        a.u_out = u_out[i];
        a.res = res[i];
        a.dt = static_cast<float>(dt);
        a.dt_elem = dt_elem ? dt_elem[i] : nullptr;
        a.a = static_cast<float>(kRkA[stage]);
        a.b = static_cast<float>(kRkB[stage]);
        M.g[g].a = a;
        M.g[g].N = ms[i]->N;
        M.g[g].ext = (a.mat || a.absorbing) ? 1 : 0;
        tiles[g] = a.num_tiles;
        cost[g] = tile_cost && tile_cost[i] > 0.0 ? tile_cost[i] : default_tile_cost(ms[i]->N);
        all += a.num_tiles;
      }
      const int total = static_cast<int>(std::min<int64_t>(sms, all));
      const std::vector<int> c = split_ctas(tiles, cost, total);
      int grid = 0;
      for (size_t g = 0; g < ng; ++g) {
        M.g[g].first = grid;
        M.g[g].count = c[g];
        grid += c[g];
      }
      DG_CUDA(traced(ms[0], s, 6, [&] {
                return f == 1 ? dgdev::launch_tc_mixed(M, grid, s)
                              : dgdev::launch_tt_mixed(M, grid, s);
              }), "mixed stage kernel launch");
      ++launches;
    }
  }
  for (int i = 0; i < n; ++i) ms[i]->last_launches = 0;
  ms[0]->last_launches = launches;
  return DG_OK;
}

int device_step(dg_mesh* m, float* u, float* res, double dt, int nsteps, void* stream,
                std::string& err) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  return step_impl(m, u, res, dt, nsteps, static_cast<cudaStream_t>(stream), err);
}

// Reads (and clears) the pipeline status word; only after a synchronisation.
static int check_status(dg_mesh* m, std::string& err) {
  int st = 0;
  DG_CUDA(cudaMemcpy(&st, m->dev->status, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy D2H");
  if (st != 0) {
    DG_CUDA(cudaMemset(m->dev->status, 0, sizeof(int)), "cudaMemset");
    err = "tensor-core stage: an MMA completion wait timed out (results invalid)";
    return DG_ERR_CUDA;
  }
  return DG_OK;
}

int device_wait_selftest(dg_mesh* m, uint32_t polls, double* seconds, std::string& err) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  DeviceState* d = m->dev;
  auto* ns = reinterpret_cast<unsigned long long*>(d->result);   // 8-byte scratch word
  DG_CUDA(dgdev::launch_wait_selftest(d->status, polls, ns, nullptr), "self-test launch");
  unsigned long long h = 0;
  DG_CUDA(cudaMemcpy(&h, ns, sizeof(h), cudaMemcpyDeviceToHost), "cudaMemcpy D2H");
  if (seconds) *seconds = static_cast<double>(h) * 1e-9;
  return check_status(m, err);
}

static int energy_impl(dg_mesh* m, const float* u, double* out, cudaStream_t s,
                       std::string& err, int64_t k0 = 0, int64_t k1 = -1) {
  DeviceState* d = m->dev;
  dgdev::EnergyArgs a{u, d->M, d->geo, static_cast<int>(d->K), d->Np, d->partials, d->result,
                      static_cast<int>(k0), static_cast<int>(k1 < 0 ? d->K : k1), d->mat};
  DG_CUDA(traced(m, s, 2, [&] { return dgdev::launch_energy_partials(a, d->egrid, s); }),
          "energy kernel launch");
  DG_CUDA(traced(m, s, 3, [&] { return dgdev::launch_energy_final(a, d->egrid, s); }),
          "energy kernel launch");
  double h = 0.0;
  DG_CUDA(cudaMemcpyAsync(&h, d->result, sizeof(double), cudaMemcpyDeviceToHost, s),
          "cudaMemcpyAsync D2H");
  DG_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (int rc = check_status(m, err)) return rc;
  *out = h;
  m->last_launches = 2;
  if (!std::isfinite(h)) { err = "energy is not finite (unstable run)"; return DG_ERR_UNSTABLE; }
  return DG_OK;
}

int device_resident(const dg_mesh* m, const float** M, const void** geo, const void** mat,
                    int64_t* K, int* Np, std::string& err) {
  int cur = -1;
  DG_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  const DeviceState* d = m->dev;
  if (!d || d->N != m->N || d->device != cur) {
    err = "mesh data is not on the current device yet (make one dg_rhs, dg_step or "
          "dg_energy call on this device first)";
    return DG_ERR_STATE;
  }
  *M = d->M;
  *geo = d->geo;
  *mat = d->mat;
  *K = d->K;
  *Np = d->Np;
  return DG_OK;
}

int device_energy_range(dg_mesh* m, const float* u, int64_t k0, int64_t k1, double* out,
                        void* stream, std::string& err) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  return energy_impl(m, u, out, static_cast<cudaStream_t>(stream), err, k0, k1);
}

int device_energy(dg_mesh* m, const float* u, double* out, void* stream, std::string& err) {
  int rc = ensure_device(m, err);
  if (rc) return rc;
  return energy_impl(m, u, out, static_cast<cudaStream_t>(stream), err);
}

int device_step_host(dg_mesh* m, float* u, float* res, double dt, int nsteps, double* energy,
                     void* stream, std::string& err) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_device(m, err);
  if (rc) return rc;
  DeviceState* d = m->dev;
  const size_t bytes = static_cast<size_t>(6) * d->K * d->Np * sizeof(float);
  if (!d->h_u) DG_CUDA(cudaMalloc(&d->h_u, bytes), "cudaMalloc");
  if (!d->h_res) DG_CUDA(cudaMalloc(&d->h_res, bytes), "cudaMalloc");
  DG_CUDA(cudaMemcpyAsync(d->h_u, u, bytes, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync H2D");
  // without a host RK register the device one starts from zero (the first
  // LSERK4 stage has a = 0, so a step's result does not depend on it)
  if (res) DG_CUDA(cudaMemcpyAsync(d->h_res, res, bytes, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync H2D");
  else DG_CUDA(cudaMemsetAsync(d->h_res, 0, bytes, s), "cudaMemsetAsync");
  // energy-growth check (opt-in): the energy of the incoming state first
  const bool check = m->energy_check >= 0.0;
  double e_in = 0.0;
  int64_t launches = 0;
  if (check) {
    if ((rc = energy_impl(m, d->h_u, &e_in, s, err))) return rc;
    launches += 2;
  }
  if ((rc = step_impl(m, d->h_u, d->h_res, dt, nsteps, s, err))) return rc;
  launches += m->last_launches;
  DG_CUDA(cudaMemcpyAsync(u, d->h_u, bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync D2H");
  if (res) DG_CUDA(cudaMemcpyAsync(res, d->h_res, bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync D2H");
  if (energy || check) {
    double e_out = 0.0;
    rc = energy_impl(m, d->h_u, &e_out, s, err);
    launches += 2;
    m->last_launches = launches;
    if (energy) *energy = e_out;
    if (rc) return rc;                       // includes a non-finite energy (DG_ERR_UNSTABLE)
    if (check && e_out > e_in * (1.0 + m->energy_check)) {
      char buf[160];
      std::snprintf(buf, sizeof buf, "energy grew from %.9g to %.9g over %d steps "
                    "(allowed factor 1 + %g): unstable run", e_in, e_out, nsteps, m->energy_check);
      err = buf;
      return DG_ERR_UNSTABLE;
    }
  } else {
    DG_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if ((rc = check_status(m, err))) return rc;
  }
  m->last_launches = launches;
  return DG_OK;
}

}  // namespace dg
