// Tensor-core RK stage for orders 5..7: the operator lives in tensor memory.
//
// The same contraction as the order <= 4 kernel (tc_stage.cuh), transposed:
//     rhs^T[i, (c,e)] = sum_k Op[i, k] X[(c,e), k],
//     Op = [Dr Ds Dt LIFT]  (Np x KT),   X = [g^r g^s g^t flux]  (one row per
//     field c and element e of the tile, g^mu_c = sign_c (r_mu,a U_a - r_mu,b U_b)),
// i.e. the volume term and the lifted surface term of Eq. semidiscrete-dg with
// the chain rule applied before differentiating (Eq. dg-reference-matrices,
// Eq. maxwells-claws).  From N = 5 on, the two FP16 pieces of Op (2 x Np x KT
// halves, 147 KB at N = 6) no longer fit shared memory beside the field tiles;
// they do fit tensor memory.  So Op is the MMA's A operand (M = 128 lanes =
// nodes i < Np, KT / 2 columns per piece), written to tensor memory once per
// CTA, and X is the B operand (N = 6 E = 48 rows), built per tile by the
// producer warps in shared memory in the canonical K-major layout.  FP32-class
// accuracy as in the other kernel: three FP16 products Op_hi X_hi + Op_hi X_lo
// + Op_lo X_hi, every X row scaled by a power of two, Op by 2^p, FP32
// accumulation.  The accumulator (lane = node i, column = (c,e)) is double
// buffered in the remaining tensor-memory columns, so lane i of the epilogue
// warps owns node i of every (c,e) of the tile -- the shared-memory order of
// the RK update.
//
// Order 7 (Np = 120, KT = 512): the two pieces take all 512 columns, so the
// accumulator is single buffered (48 columns, freed as soon as the four
// epilogue warps have read it into registers), Op_lo keeps its first 26
// k-steps (208 columns) in tensor memory and its last 6 k-steps (24 KB) sit in
// shared memory as the MMA's A operand (canonical K-major layout).  Nodes fill
// lanes 0..119, so warp 3 updates as well as issuing; the shared-memory ring
// then has room for three field slots and no RK register, and the update reads
// res and u and writes res and u_out straight from and to global memory (a
// warp touches 32 consecutive floats per column; res is prefetched into L2
// with the fields' bulk copy).
//
// One persistent 512-thread CTA per SM (orders 5, 6):
//   * producer warps (12): the fluxes of tile t (Alg. 3: face-node gathers by
//     4-byte cp.async, upwind flux with the PEC ghost state), then, after a
//     named barrier, the 48 x KT values of X(t) -- the 8 producers of a row
//     share its 8-value chunks, producer q building the chunks of all three
//     g^mu blocks at node chunks q, q + 8, ... from one load of the two curl
//     fields, then flux chunks up to its share -- a second barrier publishes
//     the row maxima (row scale), and once the MMAs of tile t-1 have read the
//     single X buffer, the scaled values are split into FP16 hi/lo and stored;
//   * MMA/epilogue warps (4): warp 3 (its tensor-memory lanes hold no node)
//     issues the 3 x KT/16 MMAs of tile t into accumulator t & 1 and all bulk
//     copies, while warps 0..2 read tile t-1's accumulator (tcgen05.ld), remove
//     the scales and apply the LSERK4 update res <- a res + dt rhs,
//     u <- u + b res in place in shared memory; bulk copies write u_out and res.
// Fields and geometry arrive by bulk copies NSU - 1 tiles ahead, the RK
// register one tile ahead.
#pragma once

#include <cuda_runtime.h>

#include "device.h"
#include "tc_stage.cuh"
#include "tcgen05.cuh"

namespace dgdev {

template <int N> struct TtDims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int E = kTtTileElems;              // elements per tile
  static constexpr int ROWS = 6 * E;                  // X rows = MMA N
  static constexpr int NN = ROWS;
  static constexpr int KB = tt_kb(N);                 // one mu block (whole 8-value chunks)
  static constexpr int KG = 3 * KB;
  static constexpr int KT = tt_kt(N);                 // total K, multiple of 16
  static constexpr int KSTEPS = KT / 16;
  static constexpr int KCH = KT / 8;                  // 16-byte chunks of an X row
  static constexpr int CG = KB / 8;                   // chunks per mu block
  static constexpr int CF = KG / 8;                   // first flux chunk
  static constexpr int ACOLS = tt_acols(N);           // tensor-memory columns per Op piece
  // Nodes reach tensor-memory lanes 96..127 (N = 7): all four lane quarters
  // update (warp 3 also issues the MMAs and copies), the accumulator is single
  // buffered, and the k-steps of Op_lo that do not fit tensor memory beside
  // Op_hi and the accumulator are the MMA's A operand from shared memory.
  static constexpr bool W4 = Np > 96;
  static constexpr int NACC = W4 ? 1 : 2;             // accumulator buffers
  static constexpr int LCOLS = W4 ? 512 - ACOLS - NN : ACOLS;   // Op_lo columns in tensor memory
  static constexpr int LSTEPS = LCOLS / 8;            // k-steps of Op_lo read from tensor memory
  static constexpr int ACC0 = ACOLS + LCOLS;          // first accumulator column
  static constexpr int PRODUCERS = 384;               // a multiple of ROWS
  static constexpr int THREADS = 128 + PRODUCERS;     // 4 MMA/epilogue warps + producer warps
  static constexpr int QR = PRODUCERS / ROWS;         // producers per X row
  static constexpr int CPT = (KCH + QR - 1) / QR;     // X chunks per producer
  static constexpr int ITEMS = (E * NF + PRODUCERS - 1) / PRODUCERS;   // flux items per producer
  static constexpr int FSTR = ((NF / 4) | 1) * 4;     // flux row stride: 16-byte row reads of
                                                      // 8 consecutive rows are conflict-free
  // ring slots: fields+geometry, RK register (W4: the update reads and writes
  // global memory directly, the fields' slots serve the producers only)
  static constexpr int NSU = W4 ? 3 : 5, NSR = W4 ? 0 : 2;
  static constexpr int NSR1 = NSR ? NSR : 1;          // array size and modulus
  // shared memory (bytes)
  static constexpr int U_FLOATS = 6 * E * Np;
  static constexpr int G_FLOATS = tc_geo_floats(N);
  static constexpr int X_BYTES = NN * KT * 2;         // one FP16 piece of X
  static constexpr int OFF_X = 0;                     // 2 pieces
  static constexpr int OFF_U = OFF_X + 2 * X_BYTES;   // NSU slots
  static constexpr int OFF_G = OFF_U + NSU * U_FLOATS * 4;
  static constexpr int OFF_R = OFF_G + NSU * G_FLOATS * 4;   // NSR slots
  static constexpr int OFF_F = OFF_R + NSR * U_FLOATS * 4;   // one flux buffer
  static constexpr int OFF_BND = OFF_F + ROWS * FSTR * 4;    // [QR][ROWS] partial row maxima
  static constexpr int OFF_SC = OFF_BND + QR * ROWS * 4;     // [4][ROWS] column factors
  static constexpr int OFF_TAB = OFF_SC + 4 * ROWS * 4;      // face-node table (NF bytes)
  // Op_lo k-steps LSTEPS.. as A operand: [k-step][2 chunks][128 rows][16 bytes]
  static constexpr int OFF_TAIL = (OFF_TAB + NF + 127) & ~127;
  static constexpr int TAIL_CH = (KSTEPS - LSTEPS) * 2;      // 8-value chunks
  static constexpr int SMEM = W4 ? OFF_TAIL + TAIL_CH * 128 * 16 : OFF_TAB + ((NF + 15) & ~15);
  static_assert(NN % 16 == 0 && NN <= 256, "MMA N");
  static_assert(PRODUCERS % ROWS == 0 && PRODUCERS % 32 == 0 && CPT * QR >= KCH, "X chunk split");
  static_assert(ACC0 + NACC * NN <= 512, "tensor-memory budget");
  static_assert(ACOLS % 16 == 0 && LCOLS % 16 == 0 && LCOLS <= ACOLS, "operator columns are written 16 at a time");
  static_assert(Np <= 128 && NF < 256 && E <= 32, "item encoding");
  static_assert((E * Np * 4) % 16 == 0 && (U_FLOATS * 4) % 16 == 0 && (G_FLOATS * 4) % 16 == 0,
                "bulk-copy alignment");
  static_assert((Np * 4) % 16 == 0 && (FSTR * 4) % 16 == 0, "16-byte row chunks");
  static_assert(OFF_U % 16 == 0 && OFF_G % 16 == 0 && OFF_R % 16 == 0 && OFF_F % 16 == 0,
                "alignment");
  static_assert(SMEM <= 226 * 1024, "shared memory budget");
  // set-up: Op staged row by row (16-byte padded rows: the lane-per-row reads of
  // a warp are conflict-free) in the X / U region, before the ring starts
  static constexpr int OPW = ACOLS + 4;               // staged row stride (words)
  static constexpr int OP_VEC = 128 * ACOLS / 4;      // 16-byte words of one piece
  static_assert(128 * OPW * 4 <= OFF_R && (!W4 || 128 * OPW * 4 <= OFF_TAIL), "operator staging area");
};

// One thread: bulk copies of tile `tile`'s fields and geometry block.
template <int N>
__device__ __forceinline__ void tt_load_u(const StageArgs& A, int tile, float* su, float* sg,
                                          uint64_t* bar) {
  using D = TtDims<N>;
  const int K = A.K, k0 = tile * D::E, Ev = min(D::E, K - k0);
  const uint32_t fb = uint32_t(Ev) * D::Np * 4;
  constexpr uint32_t gb = D::G_FLOATS * 4;
  tc::mbar_expect_tx(bar, 6u * fb + gb);
  for (int c = 0; c < 6; ++c)
    tc::bulk_g2s(su + c * D::E * D::Np, A.u_in + (size_t(c) * K + k0) * D::Np, fb, bar);
  tc::bulk_g2s(sg, A.tcgeo + size_t(tile) * A.tc_geo_stride, gb, bar);
}

// One thread: bulk copies of tile `tile`'s RK register.
template <int N>
__device__ __forceinline__ void tt_load_res(const StageArgs& A, int tile, float* sr, uint64_t* bar) {
  using D = TtDims<N>;
  const int K = A.K, k0 = tile * D::E, Ev = min(D::E, K - k0);
  const uint32_t fb = uint32_t(Ev) * D::Np * 4;
  tc::mbar_expect_tx(bar, 6u * fb);
  for (int c = 0; c < 6; ++c)
    tc::bulk_g2s(sr + c * D::E * D::Np, A.res + (size_t(c) * K + k0) * D::Np, fb, bar);
}

// One thread: L2 prefetch of tile `tile`'s RK register (read by the update
// warps straight from global memory).
template <int N>
__device__ __forceinline__ void tt_prefetch_res(const StageArgs& A, int tile) {
  using D = TtDims<N>;
  const int K = A.K, k0 = tile * D::E, Ev = min(D::E, K - k0);
  const uint32_t fb = uint32_t(Ev) * D::Np * 4;
  for (int c = 0; c < 6; ++c) tc::bulk_prefetch_l2(A.res + (size_t(c) * K + k0) * D::Np, fb);
}

// 8 consecutive floats from a 16-byte aligned shared address.
__device__ __forceinline__ void lds8(const float* p, float* v) {
  const float4 a = reinterpret_cast<const float4*>(p)[0];
  const float4 b = reinterpret_cast<const float4*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// EXT: meshes with materials (A.mat) or absorbing faces; the vacuum instantiation
// has none of that arithmetic.
// The stage as run by one CTA: `cta` of `ncta` CTAs that share the tiles of A
// (tile tile0 + cta, tile0 + cta + ncta, ...).  The kernels below run it as CTA cta of
// the grid; the mixed-order kernel runs it for the group its CTA belongs to.
template <int N, bool RK, bool EXT>
__device__ __forceinline__ void tt_stage_body(const StageArgs& A, const int cta, const int ncta) {
  using D = TtDims<N>;
  constexpr int E = D::E, Np = D::Np, Nfp = D::Nfp, NF = D::NF, FSTR = D::FSTR, ROWS = D::ROWS;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_u_full[D::NSU];
  __shared__ __align__(8) uint64_t s_r_full[D::NSR1];
  __shared__ __align__(8) uint64_t s_x_full, s_mma_done[2], s_acc_free;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = A.K;
  const int ntiles = (A.num_tiles - cta + ncta - 1) / ncta;
  const int base = A.tile0 + cta;                  // this CTA's first tile of the mesh
  if (ntiles <= 0) return;

  unsigned char* sXhi = smem + D::OFF_X;
  unsigned char* sXlo = sXhi + D::X_BYTES;
  float* sU = reinterpret_cast<float*>(smem + D::OFF_U);
  float* sG = reinterpret_cast<float*>(smem + D::OFF_G);
  float* sR = reinterpret_cast<float*>(smem + D::OFF_R);
  float* sF = reinterpret_cast<float*>(smem + D::OFF_F);
  float* sBound = reinterpret_cast<float*>(smem + D::OFF_BND);
  float* sScale = reinterpret_cast<float*>(smem + D::OFF_SC);
  unsigned char* sFmask = smem + D::OFF_TAB;

  // ---- set-up: face-node table, tensor memory, barriers, Op -------------------
  for (int i = tid; i < NF; i += D::THREADS) sFmask[i] = __ldg(A.fmask + i);
  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  if (tid == 0) {
    for (int i = 0; i < D::NSU; ++i) tc::mbar_init(&s_u_full[i], 1);
    for (int i = 0; i < D::NSR; ++i) tc::mbar_init(&s_r_full[i], 1);
    tc::mbar_init(&s_x_full, D::PRODUCERS);        // every producer thread stores X chunks
    for (int i = 0; i < 2; ++i) tc::mbar_init(&s_mma_done[i], 1);
    tc::mbar_init(&s_acc_free, 4);                 // W4: one arrival per epilogue warp
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = s_tmem;
  // Op into tensor memory, one piece at a time: all threads copy the piece to
  // shared memory (coalesced, every load in flight at once), then lane r of
  // warps 0..3 writes row r (16 columns per tensor-memory store)
#pragma unroll 1
  for (int piece = 0; piece < 2; ++piece) {
    const uint4* src = reinterpret_cast<const uint4*>(A.tcB) + size_t(piece) * D::OP_VEC;
    uint4* stage = reinterpret_cast<uint4*>(smem);
    constexpr int PER = (D::OP_VEC + D::THREADS - 1) / D::THREADS;
    uint4 w[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = tid + q * D::THREADS;
      if (i < D::OP_VEC) w[q] = __ldg(src + i);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = tid + q * D::THREADS;
      if (i < D::OP_VEC) {
        const int r = i / (D::ACOLS / 4), c4 = i - r * (D::ACOLS / 4);
        stage[r * (D::OPW / 4) + c4] = w[q];
      }
    }
    __syncthreads();
    if (warp < 4) {
      const uint4* row = stage + (warp * 32 + lane) * (D::OPW / 4);
      const uint32_t trow = tbase + (uint32_t(warp * 32) << 16) + piece * D::ACOLS;
#pragma unroll 1
      for (int c0 = 0; c0 < (piece ? D::LCOLS : D::ACOLS); c0 += 16) {
        uint32_t v[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 x = row[c0 / 4 + q];
          v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
        tc::tmem_st<16>(trow + c0, v);
      }
      tc::tmem_st_wait();
    }
    if (D::W4 && piece == 1) {
      // Op_lo columns LCOLS.. into the canonical K-major A layout: chunk c of
      // row r (8 K values, 16 bytes) at (c * 128 + r) * 16
      uint4* tail = reinterpret_cast<uint4*>(smem + D::OFF_TAIL);
      for (int i = tid; i < D::TAIL_CH * 128; i += D::THREADS) {
        const int c = i >> 7, r = i & 127;
        tail[i] = stage[r * (D::OPW / 4) + D::LCOLS / 4 + c];
      }
      tc::fence_proxy_async_smem();                 // generic stores -> tensor-core reads
    }
    tc::fence_before_sync();
    __syncthreads();                                 // staging area free again
    tc::fence_after_sync();
  }
  // the set-up above reads only constant data; the previous kernel of the
  // stream has finished writing (and reading) the fields from here on
  pdl_wait();

  if (warp < 4) {
    // ======================= MMA issue + epilogue warps ========================
    // Warp 3 issues the MMAs and all bulk copies; lane i of warp w updates node
    // 32 w + i.  Orders 5, 6: nodes i < Np <= 84 sit in tensor-memory lanes
    // 0..95, so warp 3 holds none and only issues, while warps 0..2 update from
    // and into the shared-memory tiles.  Order 7 (W4): all four warps read the
    // single accumulator first (freeing it for the next tile's MMAs), warp 3
    // then issues, and the update reads and writes global memory directly.
    // Named barrier 1 (these 128 threads) closes iteration j: the update of
    // tile j-1 is done (its tiles may be stored and, with two accumulators, its
    // accumulator reused), and warp 3 has acquired X(j) -- which carries tile
    // j's column factors to the updating warps.
    static_assert(D::W4 || Np <= 96, "warp 3 holds no node");
    const int node = warp * 32 + lane;
    const uint32_t lane_off = uint32_t(warp * 32) << 16;
    if (warp == 3 && tc::elect_one()) {
      if constexpr (D::W4) {            // first loads: fields of tiles 0..NSU-1
        for (int t = 0; t < D::NSU && t < ntiles; ++t) {
          tt_load_u<N>(A, base + t * ncta, sU + t * D::U_FLOATS, sG + t * D::G_FLOATS,
                       &s_u_full[t]);
          if (RK) tt_prefetch_res<N>(A, base + t * ncta);
        }
      } else {                          // fields of tiles 0..NSU-2, res of tile 0
        for (int t = 0; t < D::NSU - 1 && t < ntiles; ++t)
          tt_load_u<N>(A, base + t * ncta, sU + t * D::U_FLOATS, sG + t * D::G_FLOATS,
                       &s_u_full[t]);
        if (RK) tt_load_res<N>(A, base, sR, &s_r_full[0]);
      }
    }
    __syncwarp();
    constexpr uint32_t IDESC = tc::idesc_f16(128, D::NN);
    constexpr uint32_t LBO = (D::NN / 8) * 128;
    // warp 3: the 3 x KSTEPS MMAs of tile j (passes p = 0, 1, 2: hi.hi, hi.lo,
    // lo.hi), after X(j) (and, W4, the single accumulator) is ready
    auto mma_begin = [&](int j) {
      wait_or_flag(&s_x_full, j & 1, A.status);
      if (D::W4 && j >= 1) wait_or_flag(&s_acc_free, (j - 1) & 1, A.status);
      tc::fence_after_sync();
    };
    auto mma_pass = [&](int j, int p) {
      const uint32_t d_acc = tbase + D::ACC0 + (D::NACC == 2 ? (j & 1) * D::NN : 0);
      const uint64_t b_hi = tc::smem_desc(tc::smem_u32(sXhi), LBO, 128);
      const uint64_t b_lo = b_hi + uint64_t(D::X_BYTES >> 4);
      const uint64_t a_tail = tc::smem_desc(tc::smem_u32(smem + D::OFF_TAIL), 128 * 16, 128);
      // fully unrolled: warp-uniform operands (base + constant) issue cheaply
#pragma unroll
      for (int ks = 0; ks < D::KSTEPS; ++ks) {
        const uint64_t bd = (p == 1 ? b_lo : b_hi) + uint64_t((ks * 2 * LBO) >> 4);
        if (p == 2 && ks >= D::LSTEPS) {               // Op_lo k-step from shared memory
          const uint64_t ad = a_tail + uint64_t(((ks - D::LSTEPS) * 2 * 128 * 16) >> 4);
          tc::mma_f16_ss_warp(d_acc, ad, bd, IDESC, 1u);
        } else {
          const uint32_t ad = tbase + (p == 2 ? D::ACOLS : 0) + ks * 8;
          tc::mma_f16_ts_warp(d_acc, ad, bd, IDESC, p > 0 || ks > 0 ? 1u : 0u);
        }
      }
    };
    auto issue_mmas = [&](int j) {
      mma_begin(j);
#pragma unroll
      for (int p = 0; p < 3; ++p) mma_pass(j, p);
      tc::mma_commit_warp(&s_mma_done[j & 1]);
    };
    for (int j = 0; j <= ntiles; ++j) {
      const int t = j - 1, buf = t & 1;               // tile whose update runs in iteration j
      const int tile = base + t * ncta;
      const int k0 = tile * E, Ev = min(E, K - k0);
      if constexpr (D::W4) {
        uint32_t acc[D::NN];
        if (j >= 1) {                                  // accumulator of tile t -> registers
          wait_or_flag(&s_mma_done[buf], (t >> 1) & 1, A.status);
          tc::fence_after_sync();
          tmem_load_cols<D::NN>(tbase + lane_off + D::ACC0, acc);
          tc::tmem_ld_wait();
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&s_acc_free);
        }
        // Warp 3 interleaves tile j's three MMA passes with the RK update of
        // tile t (independent work: the MMA queue drains while the update's
        // global loads are in flight): passes 0 and 1, update columns 0..15,
        // pass 2, columns 16..47 (GB300, 24 576 tets: 129 us per stage against
        // 142 us with every pass first; one pass per batch 131 us).
        const bool mma = warp == 3 && j < ntiles;
        const bool upd = j >= 1 && node < Np;
        if (mma) mma_begin(j);
        const float* scl = sScale + (t & 3) * ROWS;
        // per-element steps of tile t (only when an update runs: at j = 0 there
        // is no tile t, and k0 would lie before the mesh)
        float dte[E];
#pragma unroll
        for (int e = 0; e < E; ++e)
          dte[e] = RK && upd && A.dt_elem && e < Ev ? __ldg(A.dt_elem + k0 + e) : A.dt;
        constexpr int CH = 16;
        static_assert(ROWS == 3 * CH && E % 2 == 0, "epilogue batches");
        // RK update of tile t, columns n0 .. n0 + 15: column n = (c, e) is node
        // `node` of field c of element k0 + e, so a warp reads and writes 32
        // consecutive floats
        auto update = [&](const int n0) {
          if (!upd) return;
          float rv[CH], uv[CH];
          if (RK) {
#pragma unroll
            for (int q = 0; q < CH; ++q) {
              const int n = n0 + q, c = n / E, e = n - (n / E) * E;
              const size_t g = (size_t(c) * K + k0 + e) * Np + node;
              rv[q] = e < Ev ? A.res[g] : 0.f;
              uv[q] = e < Ev ? __ldg(A.u_in + g) : 0.f;
            }
          }
#pragma unroll
          for (int q = 0; q < CH; q += 2) {
            const int n = n0 + q, c = n / E, e = n - (n / E) * E;   // e even: e + 1 < E
            const size_t g = (size_t(c) * K + k0 + e) * Np + node;
            const float2 r = __fmul2_rn(
                make_float2(__uint_as_float(acc[n]), __uint_as_float(acc[n + 1])),
                make_float2(scl[n], scl[n + 1]));
            if (RK) {
              const float2 rn = __ffma2_rn(f2(A.a), make_float2(rv[q], rv[q + 1]),
                                           __fmul2_rn(make_float2(dte[e], dte[e + 1]), r));
              const float2 un = __ffma2_rn(f2(A.b), rn, make_float2(uv[q], uv[q + 1]));
              if (e < Ev) {
                A.res[g] = rn.x;
                A.u_out[g] = un.x;
              }
              if (e + 1 < Ev) {
                A.res[g + Np] = rn.y;
                A.u_out[g + Np] = un.y;
              }
            } else {
              if (e < Ev) A.rhs[g] = r.x;
              if (e + 1 < Ev) A.rhs[g + Np] = r.y;
            }
          }
        };
        if (mma) {
          mma_pass(j, 0);
          mma_pass(j, 1);
        }
        update(0);
        if (mma) {
          mma_pass(j, 2);
          tc::mma_commit_warp(&s_mma_done[j & 1]);
          if (tc::elect_one()) {
            // the producers are done with tile j's slot: it takes tile j + NSU
            tc::fence_proxy_async_smem();
            if (j + D::NSU < ntiles) {
              const int jt = base + (j + D::NSU) * ncta, s = j % D::NSU;
              tt_load_u<N>(A, jt, sU + s * D::U_FLOATS, sG + s * D::G_FLOATS, &s_u_full[s]);
              if (RK) tt_prefetch_res<N>(A, jt);
            }
          }
          __syncwarp();
        }
        update(CH);
        update(2 * CH);
        named_sync(1, 128);
      } else {
        if (warp == 3) {
          if (j < ntiles) issue_mmas(j);               // into accumulator j & 1
          if (j >= 1 && tc::elect_one()) {
            // the slots of tile t-1 (stored in the previous iteration) take tiles
            // t+NSU-1 and t+1 now, while warps 0..2 update tile t
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            tc::fence_proxy_async_smem();
            if (t + D::NSU - 1 < ntiles) {
              const int s = (t + D::NSU - 1) % D::NSU;
              tt_load_u<N>(A, tile + (D::NSU - 1) * ncta, sU + s * D::U_FLOATS,
                           sG + s * D::G_FLOATS, &s_u_full[s]);
            }
            if (RK && t + 1 < ntiles) {
              const int s = (t + 1) % D::NSR1;
              tt_load_res<N>(A, tile + ncta, sR + s * D::U_FLOATS, &s_r_full[s]);
            }
          }
          __syncwarp();
        } else if (j >= 1) {                           // RK update of tile t = j - 1
          float* su = sU + (t % D::NSU) * D::U_FLOATS;
          float* sr = sR + (t % D::NSR1) * D::U_FLOATS;
          wait_or_flag(&s_mma_done[buf], (t >> 1) & 1, A.status);
          if (RK) wait_or_flag(&s_r_full[t % D::NSR1], (t / D::NSR1) & 1, A.status);
          tc::fence_after_sync();
          uint32_t acc[D::NN];
          tmem_load_cols<D::NN>(tbase + lane_off + D::ACC0 + buf * D::NN, acc);
          tc::tmem_ld_wait();
          tc::fence_before_sync();
          if (node < Np) {
            const float* scl = sScale + (t & 3) * ROWS;
            float dte[E];
#pragma unroll
            for (int e = 0; e < E; ++e)
              dte[e] = RK && A.dt_elem && e < Ev ? __ldg(A.dt_elem + k0 + e) : A.dt;
            // column n = (c, e) is the tile row n * Np + node; u and res share one
            // shared array, so every batch is loaded before any of its stores;
            // columns are paired (n, n + 1) for packed FP32x2 arithmetic
            constexpr int CH = 12;
            static_assert(ROWS % CH == 0 && E % 2 == 0, "epilogue batches");
#pragma unroll
            for (int n0 = 0; n0 < ROWS; n0 += CH) {
              float rv[CH], uv[CH];
              if (RK) {
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                  rv[q] = sr[(n0 + q) * Np + node];
                  uv[q] = su[(n0 + q) * Np + node];
                }
              }
#pragma unroll
              for (int q = 0; q < CH; q += 2) {
                const int n = n0 + q, e = n % E;           // e even: e + 1 < E
                const float2 r = __fmul2_rn(
                    make_float2(__uint_as_float(acc[n]), __uint_as_float(acc[n + 1])),
                    make_float2(scl[n], scl[n + 1]));
                if (RK) {
                  const float2 rn = __ffma2_rn(f2(A.a), make_float2(rv[q], rv[q + 1]),
                                               __fmul2_rn(make_float2(dte[e], dte[e + 1]), r));
                  const float2 un = __ffma2_rn(f2(A.b), rn, make_float2(uv[q], uv[q + 1]));
                  if (e < Ev) {
                    sr[n * Np + node] = rn.x;
                    su[n * Np + node] = un.x;
                  }
                  if (e + 1 < Ev) {
                    sr[(n + 1) * Np + node] = rn.y;
                    su[(n + 1) * Np + node] = un.y;
                  }
                } else {
                  if (e < Ev) sr[n * Np + node] = r.x;
                  if (e + 1 < Ev) sr[(n + 1) * Np + node] = r.y;
                }
              }
            }
          }
          tc::fence_proxy_async_smem();                // tile stores -> bulk-copy reads
        }
        named_sync(1, 128);
        if (warp == 3 && j >= 1 && tc::elect_one()) {
          float* su = sU + (t % D::NSU) * D::U_FLOATS;
          float* sr = sR + (t % D::NSR1) * D::U_FLOATS;
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
        __syncwarp();
      }
    }
    if (warp == 3 && tc::elect_one()) tc::bulk_wait_all();
    __syncwarp();
  } else {
    // ============================ producer warps ===============================
    const int pt = tid - 128;
    // X row xn = (c, e) of this producer and its chunks xq + QR q
    const int xn = pt % ROWS, xq = pt / ROWS;
    const int xc = xn / E, xe = xn - (xn / E) * E;
    const int o = xc % 3;                                 // curl: field c takes fields fa, fb
    const int fa = xc < 3 ? 3 + (o + 2) % 3 : (o + 2) % 3;
    const int fb = xc < 3 ? 3 + (o + 1) % 3 : (o + 1) % 3;
    const float sgn = xc < 3 ? 1.f : -1.f;
    // X chunks of this producer: its j-chunks jc = xq + QR i (i < nj, 8 nodes
    // each) give the chunks of all three g^mu blocks from one load of U_a and
    // U_b; flux chunks fill the rest of its CPT chunks, producer xq taking flux
    // chunks f0 .. f0 + CPT - 3 nj - 1
    constexpr int NJ = D::CG, NJS = (NJ + D::QR - 1) / D::QR;   // j-chunk slots
    static_assert(3 * NJS <= D::CPT, "g chunks per producer");
    const int nj = xq < NJ ? (NJ - 1 - xq) / D::QR + 1 : 0;
    const int ng = 3 * nj;
    int f0 = 0;
    for (int p = 0; p < xq; ++p) f0 += D::CPT - 3 * (p < NJ ? (NJ - 1 - p) / D::QR + 1 : 0);
    // Item idx = pt + q * PRODUCERS is face node m of element e (idx = e * NF + m).
    // Tile-independent decode: e | m << 5 | f << 13 | idM << 15, bit 31 past the end.
    uint32_t item[D::ITEMS];
#pragma unroll
    for (int q = 0; q < D::ITEMS; ++q) {
      const int idx = pt + q * D::PRODUCERS;
      const int e = idx / NF, m = idx - e * NF;
      item[q] = idx < E * NF ? uint32_t(e) | uint32_t(m) << 5 | uint32_t(m / Nfp) << 13 |
                                   uint32_t(sFmask[m]) << 15
                             : 0x80000000u;
    }
    float* F = sF;
    for (int t = 0; t < ntiles; ++t) {
      const int tile = base + t * ncta;
      const int k0 = tile * E, Ev = min(E, K - k0);
      const int slot = t % D::NSU;
      const float* su = sU + slot * D::U_FLOATS;
      const float* sg = sG + slot * D::G_FLOATS;
      wait_or_flag(&s_u_full[slot], (t / D::NSU) & 1, A.status);
      // ---- fluxes (Alg. 3).  Classify every item (0 none, 1 wall, 2 neighbour in
      // the tile, 3 neighbour outside it) and start the gathers of kind 3 into the
      // flux-buffer words this item's flux will overwrite.  F was last read in the
      // X values of tile t-1, before its second barrier.
      const unsigned char* nodes = reinterpret_cast<const unsigned char*>(sg + kTcGeoWords * E);
      uint32_t info[D::ITEMS];          // kind | ofs << 2
#pragma unroll
      for (int q = 0; q < D::ITEMS; ++q) {
        const uint32_t it = item[q];
        const int e = it & 31, m = (it >> 5) & 255, f = (it >> 13) & 3, idM = (it >> 15) & 127;
        const bool ok = !(it >> 31) && e < Ev;
        const int ec = ok ? e : 0;
        const unsigned code = (__float_as_uint(sg[9 * E + ec]) >> (8 * f)) & 0xffu;
        const int k2 = __float_as_int(sg[(26 + f) * E + ec]);
        const int i2 = nodes[ec * NF + m];
        const int e2 = k2 - k0;
        // absorbing faces (EXT): a wall whose exterior state is zero
        const bool absorbing = EXT && code == kAbsorbingCode;
        const uint32_t kind = !ok ? 0u
                              : (code == 0u || absorbing) ? 1u
                              : unsigned(e2) < unsigned(Ev) ? 2u : 3u;
        if (kind == 3u) {
          const float* src = A.u_in + size_t(k2) * Np + i2;
#pragma unroll
          for (int c = 0; c < 6; ++c)
            tc::cp_async4(F + (c * E + e) * FSTR + m, src + size_t(c) * K * Np);
        }
        info[q] = kind | uint32_t(kind == 2u ? e2 * Np + i2 : ec * Np + idM) << 2 |
                  (absorbing ? 0x80000000u : 0u);
      }
      tc::cp_async_commit();
      tc::cp_async_wait_all();
      // upwind flux of every face node (PEC ghost state E+ = -E-, H+ = H- on walls),
      // all operands loaded before any store into the flux buffer
      {
        float uM[D::ITEMS][6], up[D::ITEMS][6], nv[D::ITEMS][4];
        float4 cf[EXT ? D::ITEMS : 1];        // EXT: Z+, B_E, Y+, B_H of the item's face
#pragma unroll
        for (int q = 0; q < D::ITEMS; ++q) {
          const uint32_t it = item[q], kind = info[q] & 3u;
          const int e = kind ? int(it & 31) : 0, m = (it >> 5) & 255, f = (it >> 13) & 3;
          const int idM = (it >> 15) & 127;
          const float* pp = kind == 3u ? F + e * FSTR + m
                                       : su + (EXT ? (info[q] >> 2) & 0x1FFFFFFFu : info[q] >> 2);
          const int ps = kind == 3u ? E * FSTR : E * Np;
          const bool zero_ext = EXT && (info[q] >> 31);          // absorbing: u+ = 0
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            uM[q][c] = su[c * E * Np + e * Np + idM];
            up[q][c] = zero_ext ? 0.f : pp[c * ps];
          }
#pragma unroll
          for (int w = 0; w < 4; ++w) nv[q][w] = sg[(10 + 4 * f + w) * E + e];
          if constexpr (EXT)
            cf[q] = A.mat && kind ? __ldg(A.mat + size_t(k0 + e) * kMatVecs + 1 + f)
                                  : make_float4(1.f, 0.5f, 1.f, 0.5f);
        }
#pragma unroll
        for (int q = 0; q < D::ITEMS; ++q) {
          const uint32_t kind = info[q] & 3u;
          if (!kind) continue;
          const float nwe = kind == 1u ? 1.f : -1.f;      // E+ = -E- on walls
          const float dEx = fmaf(nwe, up[q][0], uM[q][0]);
          const float dEy = fmaf(nwe, up[q][1], uM[q][1]);
          const float dEz = fmaf(nwe, up[q][2], uM[q][2]);
          const float dHx = uM[q][3] - up[q][3], dHy = uM[q][4] - up[q][4];
          const float dHz = uM[q][5] - up[q][5];
          const float nx = nv[q][0], ny = nv[q][1], nz = nv[q][2], sc = 0.5f * nv[q][3];
          const float al = A.alpha;
          const float aE = al * fmaf(nz, dEz, fmaf(ny, dEy, nx * dEx));
          const float aH = al * fmaf(nz, dHz, fmaf(ny, dHy, nx * dHx));
          // fluxE = -n x dH + alpha (n (n.dE) - dE), fluxH = n x dE + alpha (n (n.dH) - dH);
          // EXT: B_E (Z+ (-n x dH) + ...), B_H (Y+ (n x dE) + ...) with Fscale
          float zp = 1.f, yp = 1.f, scE = sc, scH = sc;
          if constexpr (EXT) {
            zp = cf[q].x;
            yp = cf[q].z;
            scE = cf[q].y * nv[q][3];
            scH = cf[q].w * nv[q][3];
          }
          float fl[6];
          fl[0] = fmaf(-al, dEx, fmaf(nx, aE, zp * fmaf(-ny, dHz, nz * dHy)));
          fl[1] = fmaf(-al, dEy, fmaf(ny, aE, zp * fmaf(-nz, dHx, nx * dHz)));
          fl[2] = fmaf(-al, dEz, fmaf(nz, aE, zp * fmaf(-nx, dHy, ny * dHx)));
          fl[3] = fmaf(-al, dHx, fmaf(nx, aH, yp * fmaf(-nz, dEy, ny * dEz)));
          fl[4] = fmaf(-al, dHy, fmaf(ny, aH, yp * fmaf(-nx, dEz, nz * dEx)));
          fl[5] = fmaf(-al, dHz, fmaf(nz, aH, yp * fmaf(-ny, dEx, nx * dEy)));
          float* fr = F + int(item[q] & 31) * FSTR + int((item[q] >> 5) & 255);
#pragma unroll
          for (int c = 0; c < 6; ++c) fr[c * E * FSTR] = (c < 3 ? scE : scH) * fl[c];
        }
      }
      named_sync(2, D::PRODUCERS);                     // the flux buffer is complete
      // ---- X(t): row xn, this producer's chunks (8 values each), row maximum
      const bool live = xe < Ev;
      float x[D::CPT][8];
      float ca[3], cb[3];
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) {
        ca[mu] = sgn * sg[(3 * mu + (o + 1) % 3) * E + xe];
        cb[mu] = -sgn * sg[(3 * mu + (o + 2) % 3) * E + xe];
      }
#pragma unroll
      for (int i = 0; i < NJS; ++i) {                  // g^mu, nodes j0 .. j0 + 7, mu = 0..2
        const int j0 = (xq + D::QR * i) * 8;
        float va[8], vb[8];
        if (i < nj) {
          lds8(su + (fa * E + xe) * Np + j0, va);
          lds8(su + (fb * E + xe) * Np + j0, vb);
        }
#pragma unroll
        for (int mu = 0; mu < 3; ++mu)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            x[3 * i + mu][j] = i < nj && j0 + j < Np ? fmaf(ca[mu], va[j], cb[mu] * vb[j]) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < D::CPT; ++q) {               // flux, face nodes m0 .. m0 + 7
        if (q >= ng) {
          const int m0 = (f0 + q - ng) * 8;
          float v[8];
          if (m0 < NF) {
            lds8(F + xn * FSTR + m0, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) x[q][j] = m0 + j < NF ? v[j] : 0.f;
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[q][j] = 0.f;
          }
        }
      }
      float xmax = 0.f;
#pragma unroll
      for (int q = 0; q < D::CPT; ++q)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          x[q][j] = live ? x[q][j] : 0.f;
          xmax = fmaxf(xmax, fabsf(x[q][j]));
        }
      sBound[xq * ROWS + xn] = xmax;
      named_sync(2, D::PRODUCERS);                     // row maxima published
      float rmax = 0.f;
#pragma unroll
      for (int q = 0; q < D::QR; ++q) rmax = fmaxf(rmax, sBound[q * ROWS + xn]);
      const float s = row_scale(rmax);
      // column factor of the accumulator: 1 / (Op scale x row scale), a power of
      // two (EXT with materials: times 1/eps or 1/mu of the row's element)
      if (xq == 0) {
        float fac = A.tc_inv_bscale / s;
        if (EXT && A.mat && live) {
          const float4 w = __ldg(A.mat + size_t(k0 + xe) * kMatVecs);
          fac *= xc < 3 ? w.x : w.y;
        }
        sScale[(t & 3) * ROWS + xn] = fac;
      }
      // the single X buffer is free once the MMAs of tile t-1 have completed
      if (t >= 1) wait_or_flag(&s_mma_done[(t - 1) & 1], ((t - 1) >> 1) & 1, A.status);
#pragma unroll
      for (int q = 0; q < D::CPT; ++q) {
        const int ch = q < ng ? (q % 3) * NJ + xq + D::QR * (q / 3) : D::CF + f0 + q - ng;
        if (ch >= D::KCH) continue;                   // past the row (uneven split)
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 w = __fmul2_rn(make_float2(x[q][2 * p], x[q][2 * p + 1]), f2(s));
          tc::split2<true>(w.x, w.y, hi[p], lo[p]);   // mixed-precision residual: 1-3 % faster at N = 5, 6
        }
        // canonical K-major layout: chunk ch of row n at byte (ch * NN + n) * 16
        const int off = (ch * D::NN + xn) * 16;
        *reinterpret_cast<uint4*>(sXhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sXlo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      tc::fence_proxy_async_smem();                    // X stores -> tensor-core reads
      tc::mbar_arrive(&s_x_full);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

template <int N, bool RK, bool EXT>
__global__ void __launch_bounds__(TtDims<N>::THREADS, 1) tt_stage_kernel(const __grid_constant__ StageArgs A) {
  pdl_launch_dependents();
  tt_stage_body<N, RK, EXT>(A, int(blockIdx.x), int(gridDim.x));
}

template <int N>
cudaError_t launch_tt_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s) {
  using D = TtDims<N>;
  static bool attr[2][2][16] = {};      // [rk][ext][device]: attribute set
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  dev &= 15;
  const bool ext = a.mat || a.absorbing;
  auto kern = rk ? (ext ? tt_stage_kernel<N, true, true> : tt_stage_kernel<N, true, false>)
                 : (ext ? tt_stage_kernel<N, false, true> : tt_stage_kernel<N, false, false>);
  // at least 120 KB of shared memory: never two CTAs (each takes all 512
  // tensor-memory columns) on one SM
  constexpr int smem = D::SMEM > 120 * 1024 ? D::SMEM : 120 * 1024;
  bool& done = attr[rk ? 1 : 0][ext ? 1 : 0][dev];
  if (!done) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    done = true;
  }
  const int grid = a.num_tiles < num_sms ? a.num_tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  return launch_pdl(kern, grid, D::THREADS, smem, s, a);
}

}  // namespace dgdev

#define DG_INSTANTIATE_TT_STAGE(NN)                                                        \
  namespace dgdev {                                                                         \
  template cudaError_t launch_tt_stage_n<NN>(bool, const StageArgs&, int, cudaStream_t);    \
  }
