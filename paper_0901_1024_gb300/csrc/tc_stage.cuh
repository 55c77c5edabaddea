// Tensor-core RK stage of the nodal DG Maxwell operator (tcgen05, sm_103a).
//
// The volume term and the lifted surface term of Eq. semidiscrete-dg are one
// dense contraction per (field c, element e).  The metric terms of an affine
// tetrahedron are constants (Eq. dg-reference-matrices), so the chain rule can
// be applied before differentiating: with d/dx_nu = sum_mu (dr_mu/dx_nu) d/dr_mu
// every curl component of Eq. maxwells-claws is
//     rhs_c(e, i) = sum_mu sum_j D^mu_ij g^mu_c(e, j) + sum_m LIFT_im flux_c(e, m),
//     g^mu_c = sign_c (r_mu,a U_a - r_mu,b U_b)   (two fields of the other kind),
// i.e.  rhs[(c,e), :] = [g^r g^s g^t flux][(c,e), :] x [Dr Ds Dt LIFT]^T.
// That is an M x N x K GEMM with M = 6 * 20 rows per tile (128 with padding),
// N = Np (padded to 16), K = 3 Np + 4 Nfp (padded), computed on the tensor
// cores in FP32-class precision as three FP16 products
//     A_hi B_hi + A_hi B_lo + A_lo B_hi,      A = A_hi + A_lo,  B = B_hi + B_lo,
// with every A row scaled by a power of two (so FP16's range does not matter)
// and B = [Dr Ds Dt LIFT] scaled by a power of two; both scales are removed in
// the epilogue.
//
// Per persistent CTA (one per SM, 16 warps, all 512 tensor-memory columns):
//   * B and the face-node tables are staged once in shared memory;
//   * each tile's fields, RK register and geometry arrive by bulk copies
//     (TMA engine, mbarrier completion) one tile ahead, into a 3-slot ring;
//   * flux extraction (Alg. 2 of the paper): the neighbour values of faces that
//     leave the tile are requested first (cp.async into a shared ghost
//     buffer), the g^mu part of the A rows is computed while they are in
//     flight, then the upwind flux of every face node goes to a shared
//     [row][m] buffer (PEC ghost state on walls);
//   * A rows are built by the warps owning their tensor-memory lane quarter
//     (warp w: lanes 32 (w % 4).., K-range w / 4), split into FP16 hi/lo and
//     written straight into tensor memory (tcgen05.st);
//   * one thread issues the 3 x K/16 MMAs into a double-buffered FP32
//     accumulator in tensor memory and commits them to an mbarrier;
//   * while they run, the epilogue of tile t-1 reads its accumulator rows
//     (tcgen05.ld), unscales them and applies the LSERK4 update
//     res <- a res + dt rhs, u <- u + b res in place in shared memory; bulk
//     copies write u_out and res back.
#pragma once

#include <cuda_runtime.h>

#include "device.h"
#include "tcgen05.cuh"

namespace dgdev {

template <int N> struct TcDims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int E = kTcTileElems;             // elements per tile
  static constexpr int ROWS = 6 * E;                  // 120 <= 128
  static constexpr int KB = (Np + 1) & ~1;            // one mu block, even
  static constexpr int KG = 3 * KB;                   // g part
  static constexpr int KT = (KG + NF + 15) & ~15;     // total K, multiple of 16
  static constexpr int KSTEPS = KT / 16;
  static constexpr int ACOLS = KT / 2;                // tensor-memory columns per A piece
  static constexpr int NN = (Np + 15) & ~15;          // MMA N
  static constexpr int BUF_COLS = 256;                // columns per pipeline buffer
  static_assert(2 * ACOLS + NN <= BUF_COLS, "tensor-memory buffer overflow");
  static constexpr int COLS_G = KB / 2;               // columns of one mu block
  static constexpr int COLS_F = (KT - KG) / 2;        // columns of the flux block
  static constexpr int ECOLS = NN / 4;                // epilogue columns per warp
  static constexpr int FSTR = NF | 1;                 // flux buffer row stride (odd)
  static constexpr int THREADS = 512;
  static constexpr int ITEMS = (E * NF + THREADS - 1) / THREADS;   // flux items per thread
  // shared memory (bytes)
  static constexpr int U_FLOATS = 6 * E * Np;         // one tile of one state array
  static constexpr int G_FLOATS = E * kTcGeoWords;   // word-major: [w][E]
  static constexpr int F_FLOATS = ROWS * FSTR;
  static constexpr int B_BYTES = NN * KT * 2;         // one FP16 piece
  static constexpr int TAB_BYTES = (4 * Nfp + 96 * Nfp + 15) & ~15;
  static constexpr int OFF_B = 0;                     // 2 pieces
  static constexpr int OFF_U = OFF_B + 2 * B_BYTES;   // 3 slots
  static constexpr int OFF_R = OFF_U + 3 * U_FLOATS * 4;
  static constexpr int OFF_G = OFF_R + 3 * U_FLOATS * 4;
  static constexpr int OFF_F = OFF_G + 3 * G_FLOATS * 4;
  static constexpr int OFF_MAX = OFF_F + F_FLOATS * 4;   // [4][128] float
  static constexpr int OFF_SC = OFF_MAX + 4 * 128 * 4;   // [2][128] float
  static constexpr int OFF_TAB = OFF_SC + 2 * 128 * 4;
  static constexpr int GH_STR = 7;                       // ghost record stride (odd)
  static constexpr int OFF_GH = OFF_TAB + TAB_BYTES;     // [E*NF][GH_STR] neighbour values
  static constexpr int OFF_IT = OFF_GH + E * NF * GH_STR * 4;   // [E*NF] packed item words
  static constexpr int OFF_DESC = OFF_IT + E * NF * 4;   // [3][KSTEPS] B descriptors
  static constexpr int SMEM = OFF_DESC + ((3 * KSTEPS * 8 + 15) & ~15);
  static_assert((U_FLOATS * 4) % 16 == 0 && (E * Np * 4) % 16 == 0, "bulk-copy alignment");
  static_assert(OFF_U % 16 == 0 && OFF_R % 16 == 0 && OFF_G % 16 == 0 && OFF_F % 16 == 0 &&
                OFF_TAB % 16 == 0 && OFF_IT % 16 == 0 && OFF_DESC % 16 == 0, "alignment");
  static_assert((E * 4) % 16 == 0, "geometry word chunks must be 16-byte multiples");
  static_assert(SMEM <= 220 * 1024, "shared memory budget");
};

static_assert(tc_b_bytes(4) == 2 * TcDims<4>::B_BYTES, "B buffer size formula");

template <int NC>
__device__ __forceinline__ void tmem_store_cols(uint32_t taddr, const uint32_t* v) {
  if constexpr (NC >= 16) {
    tc::tmem_st<16>(taddr, v);
    tmem_store_cols<NC - 16>(taddr + 16, v + 16);
  } else if constexpr (NC >= 8) {
    tc::tmem_st<8>(taddr, v);
    tmem_store_cols<NC - 8>(taddr + 8, v + 8);
  } else if constexpr (NC >= 4) {
    tc::tmem_st<4>(taddr, v);
    tmem_store_cols<NC - 4>(taddr + 4, v + 4);
  } else if constexpr (NC >= 2) {
    tc::tmem_st<2>(taddr, v);
    tmem_store_cols<NC - 2>(taddr + 2, v + 2);
  } else if constexpr (NC == 1) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" :: "r"(taddr), "r"(v[0])
                 : "memory");
  }
}

// Scales 2*NC values, splits them into FP16 hi/lo pairs and stores the NC
// packed columns of each piece, at most 16 columns at a time.
template <int NC>
__device__ __forceinline__ void split_store(const float* v, float s, uint32_t t_hi, uint32_t t_lo) {
  constexpr int CH = NC < 16 ? NC : 16;
  uint32_t hi[CH], lo[CH];
#pragma unroll
  for (int p = 0; p < CH; ++p) tc::split2(v[2 * p] * s, v[2 * p + 1] * s, hi[p], lo[p]);
  tmem_store_cols<CH>(t_hi, hi);
  tmem_store_cols<CH>(t_lo, lo);
  if constexpr (NC > CH) split_store<NC - CH>(v + 2 * CH, s, t_hi + CH, t_lo + CH);
}

template <int NC>
__device__ __forceinline__ void tmem_load_cols(uint32_t taddr, uint32_t* v) {
  if constexpr (NC >= 16) {
    tc::tmem_ld<16>(taddr, v);
    tmem_load_cols<NC - 16>(taddr + 16, v + 16);
  } else if constexpr (NC >= 8) {
    tc::tmem_ld<8>(taddr, v);
    tmem_load_cols<NC - 8>(taddr + 8, v + 8);
  } else if constexpr (NC >= 4) {
    tc::tmem_ld<4>(taddr, v);
    tmem_load_cols<NC - 4>(taddr + 4, v + 4);
  } else {
    static_assert(NC == 0, "epilogue columns must be a multiple of 4");
  }
}

// Power-of-two scale bringing the largest |value| of a row to [2^14, 2^15).
__device__ __forceinline__ float row_scale(float rmax) {
  const int ex = int((__float_as_uint(rmax) >> 23) & 0xff);
  return ex == 0 ? 1.f : __uint_as_float(uint32_t(max(1, min(254, 268 - ex))) << 23);
}

// One thread: bulk copies of tile `tile` (fields, RK register, geometry block)
// into ring slot buffers, completing on `bar`.
template <int N, bool RK>
__device__ __forceinline__ void tc_issue_loads(const StageArgs& A, int tile, float* su, float* sr,
                                               float* sg, uint64_t* bar) {
  using D = TcDims<N>;
  const int K = A.K, k0 = tile * D::E, Ev = min(D::E, K - k0);
  const uint32_t fb = uint32_t(Ev) * D::Np * 4;
  constexpr uint32_t gb = kTcGeoWords * D::E * 4;      // one tiled geometry block
  tc::mbar_expect_tx(bar, (RK ? 12u : 6u) * fb + gb);
  for (int c = 0; c < 6; ++c) {
    tc::bulk_g2s(su + c * D::E * D::Np, A.u_in + (size_t(c) * K + k0) * D::Np, fb, bar);
    if (RK) tc::bulk_g2s(sr + c * D::E * D::Np, A.res + (size_t(c) * K + k0) * D::Np, fb, bar);
  }
  tc::bulk_g2s(sg, A.tcgeo + size_t(tile) * A.tc_geo_stride, gb, bar);
}

template <int N, bool RK>
__global__ void __launch_bounds__(TcDims<N>::THREADS, 1) tc_stage_kernel(const StageArgs A) {
  using D = TcDims<N>;
  constexpr int E = D::E, Np = D::Np, Nfp = D::Nfp, NF = D::NF, FSTR = D::FSTR;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mma_bar[2];
  __shared__ __align__(8) uint64_t s_load_bar[3];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, part = warp >> 2;     // lane quarter, K-range / column part
  const int K = A.K;
  const int ntiles_cta = (A.num_tiles - int(blockIdx.x) + int(gridDim.x) - 1) / int(gridDim.x);
  if (ntiles_cta <= 0) return;

  float* sU = reinterpret_cast<float*>(smem + D::OFF_U);
  float* sR = reinterpret_cast<float*>(smem + D::OFF_R);
  float* sG = reinterpret_cast<float*>(smem + D::OFF_G);
  float* sF = reinterpret_cast<float*>(smem + D::OFF_F);
  float* sMax = reinterpret_cast<float*>(smem + D::OFF_MAX);
  float* sScale = reinterpret_cast<float*>(smem + D::OFF_SC);
  float* sGhost = reinterpret_cast<float*>(smem + D::OFF_GH);
  uint32_t* sItem = reinterpret_cast<uint32_t*>(smem + D::OFF_IT);
  unsigned char* sFmask = smem + D::OFF_TAB;
  unsigned char* sPerm = sFmask + 4 * Nfp;

  // ---- set-up: B pieces, tables, tensor memory, barriers, first loads ------
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.tcB);
    uint4* dst = reinterpret_cast<uint4*>(smem + D::OFF_B);
    for (int i = tid; i < 2 * D::B_BYTES / 16; i += D::THREADS) dst[i] = __ldg(src + i);
    for (int i = tid; i < 4 * Nfp; i += D::THREADS) sFmask[i] = __ldg(A.fmask + i);
    for (int i = tid; i < 96 * Nfp; i += D::THREADS) sPerm[i] = __ldg(A.perm + i);
    // flux item idx -> e | m << 5 | f << 13 | j << 15 | idM << 21, face nodes of
    // one element consecutive: a warp's gathers hit the same neighbour blocks
    for (int idx = tid; idx < E * NF; idx += D::THREADS) {
      const int m = idx % NF, e = idx / NF, f = m / Nfp, j = m - f * Nfp;
      sItem[idx] = uint32_t(e) | uint32_t(m) << 5 | uint32_t(f) << 13 | uint32_t(j) << 15 |
                   uint32_t(__ldg(A.fmask + f * Nfp + j)) << 21;
    }
  }
  tc::fence_proxy_async_smem();
  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  if (tid == 0) {
    tc::mbar_init(&s_mma_bar[0], 1);
    tc::mbar_init(&s_mma_bar[1], 1);
    for (int i = 0; i < 3; ++i) tc::mbar_init(&s_load_bar[i], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0 && tc::elect_one()) tc_issue_loads<N, RK>(A, blockIdx.x, sU, sR, sG, &s_load_bar[0]);
  const uint32_t tbase = s_tmem;
  const uint32_t lane_off = uint32_t(quarter * 32) << 16;
  const int row = quarter * 32 + lane;               // A / D row owned by this thread
  const int rc = row / E, re = row - (row / E) * E;  // field, element of that row
  constexpr uint32_t IDESC = tc::idesc_f16(128, D::NN);
  constexpr uint32_t WAIT_LIMIT = 1u << 26;

  for (int t = 0; t <= ntiles_cta; ++t) {
    const int buf = t & 1;
    if (t < ntiles_cta) {
      const int slot = t % 3;
      const int tile = blockIdx.x + t * gridDim.x;
      const int k0 = tile * E, Ev = min(E, K - k0);
      float* su = sU + slot * D::U_FLOATS;
      float* sg = sG + slot * D::G_FLOATS;
      if (!tc::mbar_wait_bounded(&s_load_bar[slot], (t / 3) & 1, WAIT_LIMIT) && A.status)
        atomicExch(A.status, 1);
      __syncthreads();                                  // previous epilogue done everywhere

      // ---- flux, step 1: request neighbour values that leave the tile -----
      uint32_t item[D::ITEMS];
      int kind[D::ITEMS];        // 0 skip, 1 wall, 2 in tile (offset in ofs), 3 gathered
      int ofs[D::ITEMS];
#pragma unroll
      for (int q = 0; q < D::ITEMS; ++q) {
        const int idx = tid + q * D::THREADS;
        kind[q] = 0;
        ofs[q] = 0;
        item[q] = 0;
        if (idx < E * NF) {
          const uint32_t it = sItem[idx];
          item[q] = it;
          const int e = it & 31, f = (it >> 13) & 3, j = (it >> 15) & 63;
          if (e < Ev) {
            const unsigned code = (__float_as_uint(sg[9 * E + e]) >> (8 * f)) & 0xffu;
            if (code == 0u) {
              kind[q] = 1;
            } else {
              const int k2 = __float_as_int(sg[(26 + f) * E + e]);
              const int i2 = sPerm[(f * 24 + int(code) - 1) * Nfp + j];
              const int e2 = k2 - k0;
              if (e2 >= 0 && e2 < Ev) {
                kind[q] = 2;
                ofs[q] = e2 * Np + i2;
              } else {
                kind[q] = 3;
                const float* src = A.u_in + size_t(k2) * Np + i2;
#pragma unroll
                for (int c = 0; c < 6; ++c)
                  tc::cp_async4(sGhost + idx * D::GH_STR + c, src + size_t(c) * K * Np);
              }
            }
          }
        }
      }

      // ---- g^mu part of the A rows (parts 0..2), while the loads fly ------
      const bool live = row < D::ROWS && re < Ev;
      float v[D::KB];
      float mx = 0.f;
      if (part < 3) {
        if (live) {
          // curl component o of the other field kind: rhs_E = curl H, rhs_H = -curl E
          const int o = rc % 3;
          const int fa = rc < 3 ? 3 + (o + 2) % 3 : (o + 2) % 3;
          const int fb = rc < 3 ? 3 + (o + 1) % 3 : (o + 1) % 3;
          const float sgn = rc < 3 ? 1.f : -1.f;
          const float ca = sgn * sg[(3 * part + (o + 1) % 3) * E + re];
          const float cb = -sgn * sg[(3 * part + (o + 2) % 3) * E + re];
          const float* ua = su + (fa * E + re) * Np;
          const float* ub = su + (fb * E + re) * Np;
#pragma unroll
          for (int j = 0; j < D::KB; ++j) {
            v[j] = j < Np ? fmaf(ca, ua[j], cb * ub[j]) : 0.f;
            mx = fmaxf(mx, fabsf(v[j]));
          }
        } else {
#pragma unroll
          for (int j = 0; j < D::KB; ++j) v[j] = 0.f;
        }
      }

      // ---- flux, step 2: upwind flux of every face node -> sF -------------
      tc::cp_async_wait_all();                          // this thread's gathers
#pragma unroll 1
      for (int q = 0; q < D::ITEMS; ++q) {
        if (kind[q] == 0) continue;
        const int idx = tid + q * D::THREADS;
        const uint32_t it = item[q];
        const int e = it & 31, m = (it >> 5) & 255, f = (it >> 13) & 3, idM = it >> 21;
        float uM[6], up[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) uM[c] = su[(c * E + e) * Np + idM];
        if (kind[q] == 1) {
#pragma unroll
          for (int c = 0; c < 3; ++c) { up[c] = -uM[c]; up[c + 3] = uM[c + 3]; }
        } else if (kind[q] == 2) {
#pragma unroll
          for (int c = 0; c < 6; ++c) up[c] = su[c * E * Np + ofs[q]];
        } else {
#pragma unroll
          for (int c = 0; c < 6; ++c) up[c] = sGhost[idx * D::GH_STR + c];
        }
        const float nx = sg[(10 + 4 * f) * E + e], ny = sg[(11 + 4 * f) * E + e];
        const float nz = sg[(12 + 4 * f) * E + e];
        const float sc = 0.5f * sg[(13 + 4 * f) * E + e];
        const float dEx = uM[0] - up[0], dEy = uM[1] - up[1], dEz = uM[2] - up[2];
        const float dHx = uM[3] - up[3], dHy = uM[4] - up[4], dHz = uM[5] - up[5];
        const float ndE = nx * dEx + ny * dEy + nz * dEz;
        const float ndH = nx * dHx + ny * dHy + nz * dHz;
        const float al = A.alpha;
        float* fr = sF + e * FSTR + m;
        fr[0 * E * FSTR] = sc * (-(ny * dHz - nz * dHy) + al * (nx * ndE - dEx));
        fr[1 * E * FSTR] = sc * (-(nz * dHx - nx * dHz) + al * (ny * ndE - dEy));
        fr[2 * E * FSTR] = sc * (-(nx * dHy - ny * dHx) + al * (nz * ndE - dEz));
        fr[3 * E * FSTR] = sc * ((ny * dEz - nz * dEy) + al * (nx * ndH - dHx));
        fr[4 * E * FSTR] = sc * ((nz * dEx - nx * dEz) + al * (ny * ndH - dHy));
        fr[5 * E * FSTR] = sc * ((nx * dEy - ny * dEx) + al * (nz * ndH - dHz));
      }
      __syncthreads();

      // ---- flux part of the A rows (part 3), row scales, split, store -----
      constexpr int KF = D::KT - D::KG;
      const float* frow = sF + (rc * E + re) * FSTR;
      if (part == 3 && live) {
#pragma unroll 4
        for (int m = 0; m < NF; ++m) mx = fmaxf(mx, fabsf(frow[m]));
      }
      sMax[part * 128 + row] = mx;
      __syncthreads();
      const float s = row_scale(fmaxf(fmaxf(sMax[row], sMax[128 + row]),
                                      fmaxf(sMax[256 + row], sMax[384 + row])));
      const uint32_t a_hi = tbase + lane_off + buf * D::BUF_COLS;
      const uint32_t a_lo = a_hi + D::ACOLS;
      if (part < 3) {
        if (part == 0) sScale[buf * 128 + row] = s;
        split_store<D::COLS_G>(v, s, a_hi + part * D::COLS_G, a_lo + part * D::COLS_G);
      } else {
        // second pass over the flux row, 32 values (16 columns) at a time
#pragma unroll
        for (int c0 = 0; c0 < D::COLS_F; c0 += 16) {
          constexpr int CH = 16;
          float w[2 * CH];
#pragma unroll
          for (int q = 0; q < 2 * CH; ++q) {
            const int m = 2 * c0 + q;
            w[q] = (live && m < NF) ? frow[m] : 0.f;
          }
          if (c0 + CH <= D::COLS_F) {
            split_store<CH>(w, s, a_hi + 3 * D::COLS_G + c0, a_lo + 3 * D::COLS_G + c0);
          } else {
            split_store<D::COLS_F % CH>(w, s, a_hi + 3 * D::COLS_G + c0, a_lo + 3 * D::COLS_G + c0);
          }
        }
      }
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncthreads();

      // ---- warp 0: issue the MMAs of tile t, then the loads of tile t+1 ---
      if (warp == 0) {
        tc::fence_after_sync();
        const uint32_t d_acc = tbase + buf * D::BUF_COLS + 2 * D::ACOLS;
        const uint32_t a_base = tbase + buf * D::BUF_COLS;
        constexpr uint32_t LBO = (D::NN / 8) * 128;
        const uint64_t b_hi = tc::smem_desc(tc::smem_u32(smem + D::OFF_B), LBO, 128);
        const uint64_t b_lo = b_hi + uint64_t(D::B_BYTES >> 4);
#pragma unroll
        for (int i = 0; i < 3 * D::KSTEPS; ++i) {
          const int p = i / D::KSTEPS, ks = i - p * D::KSTEPS;   // passes: hi.hi, hi.lo, lo.hi
          const uint64_t bd = (p == 1 ? b_lo : b_hi) + uint64_t((ks * 2 * LBO) >> 4);
          const uint32_t ad = a_base + (p == 2 ? D::ACOLS : 0) + ks * 8;
          tc::mma_f16_ts_warp(d_acc, ad, bd, IDESC, i > 0 ? 1u : 0u);
        }
        tc::mma_commit_warp(&s_mma_bar[buf]);
        __syncwarp();
        if (t + 1 < ntiles_cta && tc::elect_one()) {
          const int ns = (t + 1) % 3;
          tc::bulk_wait_read_all();                     // stores of tile t-2 left that slot
          tc::fence_proxy_async_smem();
          tc_issue_loads<N, RK>(A, tile + gridDim.x, sU + ns * D::U_FLOATS, sR + ns * D::U_FLOATS,
                                sG + ns * D::G_FLOATS, &s_load_bar[ns]);
        }
        __syncwarp();
      }
    }

    // ---- epilogue of tile t-1 ---------------------------------------------
    if (t >= 1) {
      const int tp = t - 1, pbuf = tp & 1, pslot = tp % 3;
      const int tile = blockIdx.x + tp * gridDim.x;
      const int k0 = tile * E, Ev = min(E, K - k0);
      float* su = sU + pslot * D::U_FLOATS;
      float* sr = sR + pslot * D::U_FLOATS;
      if (!tc::mbar_wait_bounded(&s_mma_bar[pbuf], (tp >> 1) & 1, WAIT_LIMIT) && A.status)
        atomicExch(A.status, 1);
      tc::fence_after_sync();
      uint32_t acc[D::ECOLS];
      tmem_load_cols<D::ECOLS>(tbase + lane_off + pbuf * D::BUF_COLS + 2 * D::ACOLS +
                               part * D::ECOLS, acc);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
      if (row < D::ROWS && re < Ev) {
        const float inv = A.tc_inv_bscale / sScale[pbuf * 128 + row];
        const int base = (rc * E + re) * Np;
#pragma unroll
        for (int q = 0; q < D::ECOLS; ++q) {
          const int i = part * D::ECOLS + q;
          if (i < Np) {
            const float r = __uint_as_float(acc[q]) * inv;
            if (RK) {
              const float rn = fmaf(A.a, sr[base + i], A.dt * r);
              sr[base + i] = rn;
              su[base + i] = fmaf(A.b, rn, su[base + i]);
            } else {
              sr[base + i] = r;
            }
          }
        }
      }
      tc::fence_proxy_async_smem();
      __syncthreads();
      if (warp == 0 && tc::elect_one()) {
        const uint32_t fb = uint32_t(Ev) * Np * 4;
        for (int c = 0; c < 6; ++c) {
          const size_t g = (size_t(c) * K + k0) * Np;
          if (RK) {
            tc::bulk_s2g(A.u_out + g, su + c * E * Np, fb);
            tc::bulk_s2g(A.res + g, sr + c * E * Np, fb);
          } else {
            tc::bulk_s2g(A.rhs + g, sr + c * E * Np, fb);
          }
        }
        tc::bulk_commit();
      }
    }
  }
  if (warp == 0 && tc::elect_one()) tc::bulk_wait_all();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

template <int N>
cudaError_t launch_tc_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s) {
  using D = TcDims<N>;
  static bool attr[2][16] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  dev &= 15;
  auto kern = rk ? tc_stage_kernel<N, true> : tc_stage_kernel<N, false>;
  // at least 120 KB of shared memory: never two CTAs (each takes all 512
  // tensor-memory columns) on one SM
  constexpr int smem = D::SMEM > 120 * 1024 ? D::SMEM : 120 * 1024;
  if (!attr[rk ? 1 : 0][dev]) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    attr[rk ? 1 : 0][dev] = true;
  }
  const int grid = a.num_tiles < num_sms ? a.num_tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, D::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dgdev

#define DG_INSTANTIATE_TC_STAGE(NN)                                                        \
  namespace dgdev {                                                                         \
  template cudaError_t launch_tc_stage_n<NN>(bool, const StageArgs&, int, cudaStream_t);    \
  }
