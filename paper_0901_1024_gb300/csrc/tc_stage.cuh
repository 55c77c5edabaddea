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
// One persistent CTA per SM (all 512 tensor-memory columns), two warp groups
// working on different tiles at once, linked by mbarriers:
//   * producer warps (16): together they compute the fluxes of tile t (flux
//     extraction, Alg. 3 of the paper; up to 2 face nodes per thread; at N = 4
//     the face nodes of the tile's last 3 elements are done one tile earlier by
//     epilogue warps 1..3 into a small parity-buffered flux buffer): neighbour
//     values outside the tile arrive by 4-byte cp.async copies into the flux
//     buffer, every face node's upwind flux (PEC ghost state on walls) is
//     written to a shared [row][m] buffer; then they build the A rows of tile t
//     in tensor memory (tcgen05.st), per lane quarter roles 0 and 1 the two
//     halves of the node range of the g^mu blocks (they do not read the flux
//     buffer: they signal it with bar.arrive and go on) and roles 2 and 3 the
//     two halves of the flux block (bar.sync: after every flux is stored), with
//     one power-of-two scale per row (published by a barrier of all producers)
//     and the FP16 hi/lo split;
//   * MMA/epilogue warps (4): warp 0 issues the 3 x K/16 MMAs of tile t into a
//     double-buffered FP32 accumulator (elect.sync, commit to an mbarrier) and
//     all bulk copies; all four then read tile t-1's accumulator rows
//     (tcgen05.ld), unscale them and apply the LSERK4 update
//     res <- a res + dt rhs, u <- u + b res in place in shared memory, and
//     bulk copies write u_out and res back.
// Fields and geometry arrive by bulk copies four tiles ahead into a 5-slot
// ring; the RK register one tile ahead into a 2-slot ring.
#pragma once

#include <cuda_runtime.h>

#include "device.h"
#include "launch.cuh"
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
  static constexpr int KF = KT - KG;                  // flux part (with padding)
  static constexpr int KSTEPS = KT / 16;
  static constexpr int ACOLS = KT / 2;                // tensor-memory columns per A piece
  static constexpr int NN = (Np + 15) & ~15;          // MMA N
  static constexpr int BUF_COLS = 256;                // columns per pipeline buffer
  static_assert(2 * ACOLS + NN <= BUF_COLS, "tensor-memory buffer overflow");
  static constexpr int COLS_G = KB / 2;               // columns of one mu block
  static constexpr int COLS_F = KF / 2;               // columns of the flux block
  // FP16 split residual by mixed-precision FMAs (fewer instructions: 1-1.5 %
  // faster at N = 2, 3; 2.5 % slower at N = 4, where the kernel sits at its
  // register cap)
  static constexpr bool MIXED_SPLIT = N != 4;
  static constexpr int FSTR = NF + 2;                // flux row stride: 8-byte pair reads of
                                                      // a warp's 32 rows are conflict-free
  static constexpr int THREADS = 640;                 // 4 epilogue + 16 producer warps
  static constexpr int PRODUCERS = 512;
  // Flux items (face nodes): the producers take elements 0 .. E0-1 in at most
  // two rounds; the face nodes of elements E0 .. E-1 are computed one tile
  // ahead by epilogue warps 1..3 (warp 0 issues the MMAs), which otherwise
  // wait for A.
  static constexpr int E0 = 2 * PRODUCERS / NF < E ? 2 * PRODUCERS / NF : E;
  static constexpr int ITEMS = (E0 * NF + PRODUCERS - 1) / PRODUCERS;  // flux items per producer
  static constexpr int EPI = (E - E0) * NF;              // face nodes of the epilogue threads
  static constexpr int EITEMS = EPI ? (EPI + 95) / 96 : 1;   // per thread of warps 1..3
  static constexpr int FCOUNT = PRODUCERS + (EPI ? 128 : 0);  // threads at the flux barrier
  static constexpr int NSU = 5, NSR = 2;              // ring slots: fields+geometry, RK register
  // shared memory (bytes)
  static constexpr int U_FLOATS = 6 * E * Np;         // one tile of one state array
  static constexpr int G_FLOATS = tc_geo_floats(N);  // word-major [w][E], node bytes
  static constexpr int F_FLOATS = ROWS * FSTR;
  static constexpr int B_BYTES = NN * KT * 2;         // one FP16 piece
  static constexpr int TAB_BYTES = (4 * Nfp + 15) & ~15;
  static constexpr int OFF_B = 0;                     // 2 pieces
  static constexpr int OFF_U = OFF_B + 2 * B_BYTES;   // NSU slots
  static constexpr int OFF_G = OFF_U + NSU * U_FLOATS * 4;
  static constexpr int OFF_R = OFF_G + NSU * G_FLOATS * 4;   // NSR slots
  static constexpr int OFF_F = OFF_R + NSR * U_FLOATS * 4;   // one flux buffer
  static constexpr int F2_FLOATS = 6 * (E - E0) * FSTR;      // epilogue-computed flux rows
  static constexpr int OFF_F2 = OFF_F + F_FLOATS * 4;         // [2 tiles][6][E - E0][FSTR]
  static constexpr int OFF_BND = OFF_F2 + 2 * F2_FLOATS * 4;  // [2 tiles][4 roles][128] row bounds
  static constexpr int OFF_SC = OFF_BND + 2 * 4 * 128 * 4;   // [4][128] row scales
  static constexpr int OFF_TAB = OFF_SC + 4 * 128 * 4;
  static constexpr int SMEM = OFF_TAB + TAB_BYTES;
  static_assert((U_FLOATS * 4) % 16 == 0 && (E * Np * 4) % 16 == 0, "bulk-copy alignment");
  static_assert(OFF_U % 16 == 0 && OFF_R % 16 == 0 && OFF_G % 16 == 0 && OFF_F % 16 == 0 &&
                OFF_TAB % 16 == 0, "alignment");
  static_assert((G_FLOATS * 4) % 16 == 0, "geometry block must be a 16-byte multiple");
  static_assert(SMEM <= 226 * 1024, "shared memory budget");
};

static_assert(tc_b_bytes(4) == 2 * TcDims<4>::B_BYTES, "B buffer size formula");
static_assert(TcDims<1>::FSTR % 4 == 2 && TcDims<4>::FSTR % 4 == 2, "flux row stride");
static_assert(TcDims<4>::G_FLOATS == kTcGeoWords * kTcTileElems + kTcTileElems * TcDims<4>::NF / 4,
              "geometry block size");

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

// Columns [C0, C0 + NC) of one row: column p holds the pair val(p) (a float2 of
// values 2p, 2p + 1), split into FP16 hi/lo and stored 8 columns at a time
// (pairs are produced only as they are stored, so few registers are live).
template <int NC, int C0 = 0, bool MIXED = false, typename Val>
__device__ __forceinline__ void split_store_fn(const Val& val, uint32_t t_hi, uint32_t t_lo) {
  constexpr int CH = NC < 8 ? NC : 8;
  uint32_t hi[CH], lo[CH];
#pragma unroll
  for (int p = 0; p < CH; ++p) {
    const float2 v = val(C0 + p);
    tc::split2<MIXED>(v.x, v.y, hi[p], lo[p]);
  }
  tmem_store_cols<CH>(t_hi + C0, hi);
  tmem_store_cols<CH>(t_lo + C0, lo);
  if constexpr (NC > CH) split_store_fn<NC - CH, C0 + CH, MIXED>(val, t_hi, t_lo);
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

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
    static_assert(NC == 0, "accumulator columns must be a multiple of 4");
  }
}

// Power-of-two scale bringing the largest |value| of a row to [2^14, 2^15).
__device__ __forceinline__ float row_scale(float rmax) {
  const int ex = int((__float_as_uint(rmax) >> 23) & 0xff);
  return ex == 0 ? 1.f : __uint_as_float(uint32_t(max(1, min(254, 268 - ex))) << 23);
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}
// Signal a named barrier without waiting (producer side of bar.arrive / bar.sync).
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

// Polls of a bounded mbarrier wait.  A poll that finds the phase incomplete
// suspends for the hardware's time limit, measured at ~4 us on GB300 (the
// self-test of dg_check_wait_timeout), so 2^18 polls give up after about a
// second; the pipeline's real waits last microseconds.
constexpr uint32_t kWaitLimit = 1u << 18;

// Bounded mbarrier wait; on timeout records the failure in *status.
__device__ __forceinline__ void wait_or_flag(uint64_t* bar, uint32_t parity, int* status,
                                             uint32_t limit = kWaitLimit) {
  if (!tc::mbar_wait_bounded(bar, parity, limit) && status) atomicExch(status, 1);
}

// One thread: bulk copies of tile `tile`'s fields and geometry block.
template <int N>
__device__ __forceinline__ void tc_load_u(const StageArgs& A, int tile, float* su, float* sg,
                                          uint64_t* bar) {
  using D = TcDims<N>;
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
__device__ __forceinline__ void tc_load_res(const StageArgs& A, int tile, float* sr, uint64_t* bar) {
  using D = TcDims<N>;
  const int K = A.K, k0 = tile * D::E, Ev = min(D::E, K - k0);
  const uint32_t fb = uint32_t(Ev) * D::Np * 4;
  tc::mbar_expect_tx(bar, 6u * fb);
  for (int c = 0; c < 6; ++c)
    tc::bulk_g2s(sr + c * D::E * D::Np, A.res + (size_t(c) * K + k0) * D::Np, fb, bar);
}

// One g-block builder row (a producer thread of role 0 or 1) of tile t.
struct GRow {
  const float* su;
  const float* sg;
  float* sBound;
  float* sScale;
  int t, row, rc, re, o, fa, fb;
  float sgn;
  bool live;
  uint32_t a_hi, a_lo;
  uint64_t* mma_done;
  int* status;
};

// Node pairs [P0, P0 + NPH) of the three g^mu blocks of one A row: loads that
// part of the two curl fields, publishes its bound on |g| and, after the flux
// bound, splits g^mu = sign (r_mu,a U_a - r_mu,b U_b) into tensor memory.
template <int N, int P0, int NPH>
__device__ __forceinline__ void build_g_half(const GRow& g, int role) {
  using D = TcDims<N>;
  constexpr int E = D::E, Np = D::Np;
  float2 ua[NPH], ub[NPH];
  float umax = 0.f;
  const float* pa = g.su + (g.fa * E + g.re) * Np;
  const float* pb = g.su + (g.fb * E + g.re) * Np;
#pragma unroll
  for (int i = 0; i < NPH; ++i) {
    const int j = 2 * (P0 + i);
    ua[i].x = g.live ? pa[j] : 0.f;
    ub[i].x = g.live ? pb[j] : 0.f;
    ua[i].y = g.live && j + 1 < Np ? pa[j + 1] : 0.f;
    ub[i].y = g.live && j + 1 < Np ? pb[j + 1] : 0.f;
    umax = fmaxf(umax, fmaxf(fmaxf(fabsf(ua[i].x), fabsf(ua[i].y)),
                             fmaxf(fabsf(ub[i].x), fabsf(ub[i].y))));
  }
  float cmax = 0.f;
  if (g.live) {
#pragma unroll
    for (int mu = 0; mu < 3; ++mu)
      cmax = fmaxf(cmax, fabsf(g.sg[(3 * mu + (g.o + 1) % 3) * E + g.re]) +
                             fabsf(g.sg[(3 * mu + (g.o + 2) % 3) * E + g.re]));
  }
  // |g^mu| <= (|r_mu,a| + |r_mu,b|) max(max|U_a|, max|U_b|) over this node range;
  // bounds of tiles t and t+1 live in different halves (a thread reads tile t's
  // before it arrives at tile t+1's barrier, which precedes tile t+2's writes)
  float* bnd = g.sBound + (g.t & 1) * 512;
  bnd[role * 128 + g.row] = cmax * umax;
  named_sync(2, D::PRODUCERS);            // row bounds published
  const float s = row_scale(fmaxf(fmaxf(bnd[g.row], bnd[128 + g.row]),
                                  fmaxf(bnd[256 + g.row], bnd[384 + g.row])));
  // A[buf] is free once the MMAs of tile t-2 have completed
  if (g.t >= 2) wait_or_flag(g.mma_done, ((g.t - 2) >> 1) & 1, g.status);
  tc::fence_after_sync();
  if (role == 0) g.sScale[(g.t & 3) * 128 + g.row] = s;
  // the scale goes on the fields, not on the metric terms: s may be as large
  // as 2^127 for a row of tiny values, while |U s| < 2^15 / (|r_a| + |r_b|)
#pragma unroll
  for (int i = 0; i < NPH; ++i) {
    ua[i] = __fmul2_rn(ua[i], f2(s));
    ub[i] = __fmul2_rn(ub[i], f2(s));
  }
#pragma unroll 1
  for (int mu = 0; mu < 3; ++mu) {
    const float ca = g.live ? g.sgn * g.sg[(3 * mu + (g.o + 1) % 3) * E + g.re] : 0.f;
    const float cb = g.live ? -g.sgn * g.sg[(3 * mu + (g.o + 2) % 3) * E + g.re] : 0.f;
    split_store_fn<NPH, P0, D::MIXED_SPLIT>(
        [&](int p) { return __ffma2_rn(f2(ca), ua[p - P0], __fmul2_rn(f2(cb), ub[p - P0])); },
        g.a_hi + mu * D::COLS_G, g.a_lo + mu * D::COLS_G);
  }
}

// One flux-block builder row (a producer thread of role 2 or 3) of tile t.
struct FRow {
  const float* frow;      // the row's flux values in the flux buffer
  float* sBound;
  int t, row;
  bool live;
  uint32_t a_hi, a_lo;    // tensor-memory columns of the flux block
  uint64_t* mma_done;
  int* status;
};

// Columns [P0, P0 + NPH) of the flux block of one A row: loads those flux values
// (8-byte pairs), publishes their maximum, and after the barrier splits them,
// scaled by the row's power of two, into tensor memory.
template <int N, int P0, int NPH>
__device__ __forceinline__ void build_flux_half(const FRow& g, int role) {
  using D = TcDims<N>;
  constexpr int NF = D::NF;
  const float2* frow = reinterpret_cast<const float2*>(g.frow);
  float2 w[NPH];
  float fmax = 0.f;
#pragma unroll
  for (int i = 0; i < NPH; ++i) {
    w[i] = (g.live && 2 * (P0 + i) < NF) ? frow[P0 + i] : make_float2(0.f, 0.f);
    fmax = fmaxf(fmax, fmaxf(fabsf(w[i].x), fabsf(w[i].y)));
  }
  float* bnd = g.sBound + (g.t & 1) * 512;
  bnd[role * 128 + g.row] = fmax;
  named_sync(2, D::PRODUCERS);                     // row bounds published
  const float s = row_scale(fmaxf(fmaxf(bnd[g.row], bnd[128 + g.row]),
                                  fmaxf(bnd[256 + g.row], bnd[384 + g.row])));
  // A[buf] is free once the MMAs of tile t-2 have completed
  if (g.t >= 2) wait_or_flag(g.mma_done, ((g.t - 2) >> 1) & 1, g.status);
  tc::fence_after_sync();
  split_store_fn<NPH, P0, D::MIXED_SPLIT>([&](int p) { return __fmul2_rn(w[p - P0], f2(s)); }, g.a_hi, g.a_lo);
}

// Decode of flux item idx = e * NF + m (face node m of element e), for idx <
// `elems` * NF: e | m << 5 | f << 12 | idM << 14 (f the face, idM the element's
// node there); bit 31 set past the end.
template <int N>
__device__ __forceinline__ uint32_t tc_item(int idx, int elems, const unsigned char* sFmask) {
  using D = TcDims<N>;
  const int e = idx / D::NF, m = idx - e * D::NF;
  return idx < elems * D::NF ? uint32_t(e) | uint32_t(m) << 5 | uint32_t(m / D::Nfp) << 12 |
                                   uint32_t(sFmask[m]) << 14
                             : 0x80000000u;
}

// Flux extraction (Alg. 3) of the face nodes `item` (decoded e | m << 5 | f << 12 |
// idM << 14, bit 31: none) of the tile starting at element k0 with Ev valid
// elements, fields su and geometry sg in shared memory: classify, gather the
// neighbour values outside the tile, form the upwind fluxes (PEC ghost state on
// walls, zero exterior state on absorbing faces) and store them at
// dst + (c * CS + e - E0) * FSTR + m for field c of element e (E0 <= e < E0 + CS).
template <int N, bool EXT, int NI>
__device__ __forceinline__ void tc_flux_items(const uint32_t (&item)[NI], const StageArgs& A,
                                              int k0, int Ev, const float* su, const float* sg,
                                              float* dst, int CS, int E0) {
  using D = TcDims<N>;
  constexpr int E = D::E, Np = D::Np, NF = D::NF, FSTR = D::FSTR;
  const int K = A.K;
  const unsigned char* nodes = reinterpret_cast<const unsigned char*>(sg + kTcGeoWords * E);
  // Classify every item (0 none, 1 wall, 2 neighbour in the tile, 3 neighbour
  // outside it) and start the gathers of kind 3: the six neighbour values go by
  // 4-byte asynchronous copies into the destination words this item's flux will
  // overwrite (no registers, no extra space).
  uint32_t info[NI];                // kind | ofs << 2
#pragma unroll
  for (int q = 0; q < NI; ++q) {
    const uint32_t it = item[q];
    const int e = it & 31, m = (it >> 5) & 127, f = (it >> 12) & 3, idM = (it >> 14) & 63;
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
        tc::cp_async4(dst + (c * CS + e - E0) * FSTR + m, src + size_t(c) * K * Np);
    }
    info[q] = kind | uint32_t(kind == 2u ? e2 * Np + i2 : ec * Np + idM) << 2 |
              (absorbing ? 0x80000000u : 0u);
  }
  tc::cp_async_commit();
  tc::cp_async_wait_all();
  // upwind flux of every face node (PEC ghost state E+ = -E-, H+ = H- on walls):
  // every item's operands are loaded before any store into the flux buffer,
  // then items are processed two at a time in packed FP32x2 arithmetic
  {
    constexpr int NQ = (NI + 1) & ~1;
    float uM[NQ][6], up[NQ][6], nv[NQ][4];
    float4 cf[EXT ? NQ : 1];          // EXT: Z+, B_E, Y+, B_H of the item's face
    uint32_t kinds[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (q >= NI) {
        kinds[q] = 0u;
#pragma unroll
        for (int c = 0; c < 6; ++c) uM[q][c] = up[q][c] = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) nv[q][w] = 0.f;
        if constexpr (EXT) cf[q] = make_float4(1.f, 0.5f, 1.f, 0.5f);
        continue;
      }
      const uint32_t it = item[q], kind = info[q] & 3u;
      kinds[q] = kind;
      const int e = kind ? int(it & 31) : 0, m = (it >> 5) & 127, f = (it >> 12) & 3;
      const int idM = (it >> 14) & 63;
      const float* pp = kind == 3u ? dst + (e - E0) * FSTR + m
                                   : su + (EXT ? (info[q] >> 2) & 0x1FFFFFFFu : info[q] >> 2);
      const int ps = kind == 3u ? CS * FSTR : E * Np;
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
    const float2 m1 = f2(-1.f), nal = f2(-A.alpha), al = f2(A.alpha);
#pragma unroll
    for (int q = 0; q < NQ; q += 2) {
      const int r = q + 1;
      auto P = [&](const float (*v)[6], int c) { return make_float2(v[q][c], v[r][c]); };
      const float2 nwe = make_float2(kinds[q] == 1u ? 1.f : -1.f, kinds[r] == 1u ? 1.f : -1.f);
      const float2 dEx = __ffma2_rn(nwe, P(up, 0), P(uM, 0));
      const float2 dEy = __ffma2_rn(nwe, P(up, 1), P(uM, 1));
      const float2 dEz = __ffma2_rn(nwe, P(up, 2), P(uM, 2));
      const float2 dHx = __ffma2_rn(m1, P(up, 3), P(uM, 3));
      const float2 dHy = __ffma2_rn(m1, P(up, 4), P(uM, 4));
      const float2 dHz = __ffma2_rn(m1, P(up, 5), P(uM, 5));
      const float2 nx = make_float2(nv[q][0], nv[r][0]), ny = make_float2(nv[q][1], nv[r][1]);
      const float2 nz = make_float2(nv[q][2], nv[r][2]);
      const float2 sc = __fmul2_rn(f2(0.5f), make_float2(nv[q][3], nv[r][3]));
      // EXT: B_E (Z+ (-n x dH) + ...), B_H (Y+ (n x dE) + ...) with Fscale
      float2 zp = f2(1.f), yp = f2(1.f), scE = sc, scH = sc;
      if constexpr (EXT) {
        zp = make_float2(cf[q].x, cf[r].x);
        yp = make_float2(cf[q].z, cf[r].z);
        scE = __fmul2_rn(make_float2(cf[q].y, cf[r].y), make_float2(nv[q][3], nv[r][3]));
        scH = __fmul2_rn(make_float2(cf[q].w, cf[r].w), make_float2(nv[q][3], nv[r][3]));
      }
      const float2 mx = __fmul2_rn(m1, nx), my = __fmul2_rn(m1, ny), mz = __fmul2_rn(m1, nz);
      const float2 aE = __fmul2_rn(al, __ffma2_rn(nz, dEz, __ffma2_rn(ny, dEy, __fmul2_rn(nx, dEx))));
      const float2 aH = __fmul2_rn(al, __ffma2_rn(nz, dHz, __ffma2_rn(ny, dHy, __fmul2_rn(nx, dHx))));
      // fluxE = -n x dH + alpha (n (n.dE) - dE), fluxH = n x dE + alpha (n (n.dH) - dH)
      float2 fl[6];
      if constexpr (!EXT) {
        fl[0] = __ffma2_rn(nal, dEx, __ffma2_rn(nx, aE, __ffma2_rn(my, dHz, __fmul2_rn(nz, dHy))));
        fl[1] = __ffma2_rn(nal, dEy, __ffma2_rn(ny, aE, __ffma2_rn(mz, dHx, __fmul2_rn(nx, dHz))));
        fl[2] = __ffma2_rn(nal, dEz, __ffma2_rn(nz, aE, __ffma2_rn(mx, dHy, __fmul2_rn(ny, dHx))));
        fl[3] = __ffma2_rn(nal, dHx, __ffma2_rn(nx, aH, __ffma2_rn(mz, dEy, __fmul2_rn(ny, dEz))));
        fl[4] = __ffma2_rn(nal, dHy, __ffma2_rn(ny, aH, __ffma2_rn(mx, dEz, __fmul2_rn(nz, dEx))));
        fl[5] = __ffma2_rn(nal, dHz, __ffma2_rn(nz, aH, __ffma2_rn(my, dEx, __fmul2_rn(nx, dEy))));
      } else {
        fl[0] = __ffma2_rn(nal, dEx, __ffma2_rn(nx, aE, __fmul2_rn(zp, __ffma2_rn(my, dHz, __fmul2_rn(nz, dHy)))));
        fl[1] = __ffma2_rn(nal, dEy, __ffma2_rn(ny, aE, __fmul2_rn(zp, __ffma2_rn(mz, dHx, __fmul2_rn(nx, dHz)))));
        fl[2] = __ffma2_rn(nal, dEz, __ffma2_rn(nz, aE, __fmul2_rn(zp, __ffma2_rn(mx, dHy, __fmul2_rn(ny, dHx)))));
        fl[3] = __ffma2_rn(nal, dHx, __ffma2_rn(nx, aH, __fmul2_rn(yp, __ffma2_rn(mz, dEy, __fmul2_rn(ny, dEz)))));
        fl[4] = __ffma2_rn(nal, dHy, __ffma2_rn(ny, aH, __fmul2_rn(yp, __ffma2_rn(mx, dEz, __fmul2_rn(nz, dEx)))));
        fl[5] = __ffma2_rn(nal, dHz, __ffma2_rn(nz, aH, __fmul2_rn(yp, __ffma2_rn(my, dEx, __fmul2_rn(nx, dEy)))));
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) fl[c] = __fmul2_rn(c < 3 ? scE : scH, fl[c]);
      if (kinds[q]) {
        float* fr = dst + (int(item[q] & 31) - E0) * FSTR + int((item[q] >> 5) & 127);
#pragma unroll
        for (int c = 0; c < 6; ++c) fr[c * CS * FSTR] = fl[c].x;
      }
      if (r < NI && kinds[r]) {
        float* fr = dst + (int(item[r < NI ? r : 0] & 31) - E0) * FSTR +
                    int((item[r < NI ? r : 0] >> 5) & 127);
#pragma unroll
        for (int c = 0; c < 6; ++c) fr[c * CS * FSTR] = fl[c].y;
      }
    }
  }
}

// EXT: meshes with materials (A.mat) or absorbing faces; the vacuum instantiation
// has none of that arithmetic.
// The stage as run by one CTA: `cta` of `ncta` CTAs that share the tiles of A
// (tile tile0 + cta, tile0 + cta + ncta, ...).  The kernels below run it as CTA cta of
// the grid; the mixed-order kernel runs it for the group its CTA belongs to.
template <int N, bool RK, bool EXT>
__device__ __forceinline__ void tc_stage_body(const StageArgs& A, const int cta, const int ncta) {
  using D = TcDims<N>;
  constexpr int E = D::E, Np = D::Np, Nfp = D::Nfp, FSTR = D::FSTR;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_u_full[D::NSU];
  __shared__ __align__(8) uint64_t s_r_full[D::NSR];
  __shared__ __align__(8) uint64_t s_a_full[2], s_mma_done[2];
  __shared__ __align__(8) uint64_t s_b_full;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = A.K;
  const int ntiles = (A.num_tiles - cta + ncta - 1) / ncta;
  const int base = A.tile0 + cta;                  // this CTA's first tile of the mesh
  if (ntiles <= 0) return;

  float* sU = reinterpret_cast<float*>(smem + D::OFF_U);
  float* sG = reinterpret_cast<float*>(smem + D::OFF_G);
  float* sR = reinterpret_cast<float*>(smem + D::OFF_R);
  float* sF = reinterpret_cast<float*>(smem + D::OFF_F);
  float* sScale = reinterpret_cast<float*>(smem + D::OFF_SC);
  float* sBound = reinterpret_cast<float*>(smem + D::OFF_BND);
  float* sF2 = reinterpret_cast<float*>(smem + D::OFF_F2);
  unsigned char* sFmask = smem + D::OFF_TAB;

  // ---- set-up: B pieces (one bulk copy, constant data: it may overlap the
  // previous kernel), face-node table, tensor memory, barriers ----------------
  for (int i = tid; i < 4 * Nfp; i += D::THREADS) sFmask[i] = __ldg(A.fmask + i);
  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  if (tid == 0) {
    tc::mbar_init(&s_b_full, 1);
    for (int i = 0; i < D::NSU; ++i) tc::mbar_init(&s_u_full[i], 1);
    for (int i = 0; i < D::NSR; ++i) tc::mbar_init(&s_r_full[i], 1);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&s_a_full[i], D::PRODUCERS);  // every producer thread stores A columns
      tc::mbar_init(&s_mma_done[i], 1);
    }
    tc::fence_mbar_init();
    tc::mbar_expect_tx(&s_b_full, 2u * D::B_BYTES);
    tc::bulk_g2s(smem + D::OFF_B, A.tcB, 2u * D::B_BYTES, &s_b_full);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = s_tmem;
  // the previous kernel of the stream has finished writing (and reading) the fields
  pdl_wait();

  if (warp < 4) {
    // ======================= MMA issue + epilogue warps ========================
    const int row = warp * 32 + lane;
    const int rc = row / E, re = row - (row / E) * E;
    const uint32_t lane_off = uint32_t(warp * 32) << 16;
    if (warp == 0 && tc::elect_one()) {   // first loads: fields of tiles 0..NSU-2, res of tile 0
      for (int t = 0; t < D::NSU - 1 && t < ntiles; ++t)
        tc_load_u<N>(A, base + t * ncta, sU + t * D::U_FLOATS, sG + t * D::G_FLOATS,
                     &s_u_full[t]);
      if (RK) tc_load_res<N>(A, base, sR, &s_r_full[0]);
    }
    __syncwarp();
    // Flux items of elements E0 .. E-1 (warps 1..3), computed one tile ahead
    // into the buffer of that tile's parity (tile 0 now, tile j+1 in iteration
    // j), then signalled at the flux barrier of that tile by all four warps.
    // The buffer of parity t & 1 was last read by the flux-block builders of
    // tile t-2, before A(t-2).
    uint32_t eitem[D::EITEMS];
#pragma unroll
    for (int q = 0; q < D::EITEMS; ++q)
      eitem[q] = tc_item<N>(D::E0 * D::NF + (tid - 32) + 96 * q, E, sFmask);
    auto epilogue_fluxes = [&](int t) {
      if (warp != 0) {
        const int slot = t % D::NSU;
        const int k0t = (base + t * ncta) * E, Evt = min(E, K - k0t);
        wait_or_flag(&s_u_full[slot], (t / D::NSU) & 1, A.status);
        tc_flux_items<N, EXT, D::EITEMS>(eitem, A, k0t, Evt, sU + slot * D::U_FLOATS,
                                         sG + slot * D::G_FLOATS, sF2 + (t & 1) * D::F2_FLOATS,
                                         E - D::E0, D::E0);
      }
      named_arrive(3 + (t & 1), D::FCOUNT);
    };
    if constexpr (D::EPI > 0) epilogue_fluxes(0);
    constexpr uint32_t IDESC = tc::idesc_f16(128, D::NN);
    constexpr uint32_t LBO = (D::NN / 8) * 128;
    for (int j = 0; j <= ntiles; ++j) {
      if (j < ntiles) {
        // every epilogue warp observes A(j) complete (this also publishes tile j's
        // row scales) before the MMAs start, so no waiter can fall a phase behind
        wait_or_flag(&s_a_full[j & 1], (j >> 1) & 1, A.status);
        named_sync(1, 128);
      }
      if (j < ntiles && warp == 0) {                 // MMAs of tile j
        const int buf = j & 1;
        if (j == 0) wait_or_flag(&s_b_full, 0, A.status);   // B pieces in shared memory
        tc::fence_after_sync();
        const uint32_t d_acc = tbase + buf * D::BUF_COLS + 2 * D::ACOLS;
        const uint32_t a_base = tbase + buf * D::BUF_COLS;
        const uint64_t b_hi = tc::smem_desc(tc::smem_u32(smem + D::OFF_B), LBO, 128);
        const uint64_t b_lo = b_hi + uint64_t(D::B_BYTES >> 4);
#pragma unroll
        for (int i = 0; i < 3 * D::KSTEPS; ++i) {
          const int p = i / D::KSTEPS, ks = i - p * D::KSTEPS;   // passes: hi.hi, hi.lo, lo.hi
          const uint64_t bd = (p == 1 ? b_lo : b_hi) + uint64_t((ks * 2 * LBO) >> 4);
          const uint32_t ad = a_base + (p == 2 ? D::ACOLS : 0) + ks * 8;
          tc::mma_f16_ts_warp(d_acc, ad, bd, IDESC, i > 0 ? 1u : 0u);
        }
        tc::mma_commit_warp(&s_mma_done[buf]);
        __syncwarp();
      }
      if constexpr (D::EPI > 0) {
        if (j + 1 < ntiles) epilogue_fluxes(j + 1);
      }
      if (j >= 1) {                                  // epilogue of tile t = j - 1
        const int t = j - 1, buf = t & 1;
        const int tile = base + t * ncta;
        const int k0 = tile * E, Ev = min(E, K - k0);
        float* su = sU + (t % D::NSU) * D::U_FLOATS;
        float* sr = sR + (t % D::NSR) * D::U_FLOATS;
        if (warp == 0 && tc::elect_one()) {
          // the slots of tile t-1 (its stores were issued one round ago) take
          // tiles t+NSU-1 and t+1 now, before this tile's update
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          tc::fence_proxy_async_smem();
          if (t + D::NSU - 1 < ntiles) {
            const int s = (t + D::NSU - 1) % D::NSU;
            tc_load_u<N>(A, tile + (D::NSU - 1) * ncta, sU + s * D::U_FLOATS,
                         sG + s * D::G_FLOATS, &s_u_full[s]);
          }
          if (RK && t + 1 < ntiles) {
            const int s = (t + 1) % D::NSR;
            tc_load_res<N>(A, tile + ncta, sR + s * D::U_FLOATS, &s_r_full[s]);
          }
        }
        __syncwarp();
        wait_or_flag(&s_mma_done[buf], (t >> 1) & 1, A.status);
        if (RK) wait_or_flag(&s_r_full[t % D::NSR], (t / D::NSR) & 1, A.status);
        tc::fence_after_sync();
        uint32_t acc[D::NN];
        tmem_load_cols<D::NN>(tbase + lane_off + buf * D::BUF_COLS + 2 * D::ACOLS, acc);
        tc::tmem_ld_wait();
        tc::fence_before_sync();
        if (row < D::ROWS && re < Ev) {
          float inv = A.tc_inv_bscale / sScale[(t & 3) * 128 + row];
          if (EXT && A.mat) {                  // rhs_E / eps, rhs_H / mu
            const float4 w = __ldg(A.mat + size_t(k0 + re) * kMatVecs);
            inv *= rc < 3 ? w.x : w.y;
          }
          const float dte = RK && A.dt_elem ? __ldg(A.dt_elem + k0 + re) : A.dt;
          float* pr = sr + (rc * E + re) * Np;
          float* pu = su + (rc * E + re) * Np;
          // u and res share one shared array, so every batch is loaded before any
          // of its stores (the compiler cannot move loads across them)
          constexpr int CH = 12;
#pragma unroll
          for (int i0 = 0; i0 < Np; i0 += CH) {
            float rv[CH], uv[CH];
            if (RK) {
#pragma unroll
              for (int i = 0; i < CH; ++i)
                if (i0 + i < Np) {
                  rv[i] = pr[i0 + i];
                  uv[i] = pu[i0 + i];
                }
            }
#pragma unroll
            for (int i = 0; i < CH; i += 2) {
              if (i0 + i >= Np) break;
              // pair (i, i + 1) in packed FP32x2; a lone last node pairs with itself
              const int i1 = i0 + i + 1 < Np ? i + 1 : i;
              const float2 r = __fmul2_rn(
                  make_float2(__uint_as_float(acc[i0 + i]), __uint_as_float(acc[i0 + i1])), f2(inv));
              if (RK) {
                const float2 rn = __ffma2_rn(f2(A.a), make_float2(rv[i], rv[i1]),
                                             __fmul2_rn(f2(dte), r));
                const float2 un = __ffma2_rn(f2(A.b), rn, make_float2(uv[i], uv[i1]));
                pr[i0 + i] = rn.x;
                pu[i0 + i] = un.x;
                if (i1 != i) {
                  pr[i0 + i1] = rn.y;
                  pu[i0 + i1] = un.y;
                }
              } else {
                pr[i0 + i] = r.x;
                if (i1 != i) pr[i0 + i1] = r.y;
              }
            }
          }
        }
        tc::fence_proxy_async_smem();
        named_sync(1, 128);
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
        __syncwarp();
      }
    }
    if (warp == 0 && tc::elect_one()) tc::bulk_wait_all();
    __syncwarp();
  } else {
    // ============================ producer warps ===============================
    // Warps 4..19 compute the fluxes of tile t together, then build its A rows:
    // per tensor-memory lane quarter, roles 0 and 1 (warps 4-7, 8-11) the first
    // and second half of the node range of the three g blocks, roles 2 and 3
    // (warps 12-15, 16-19) the first and second half of the flux block.
    const int pt = tid - 128;
    const int role = (warp - 4) >> 2, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int rc = row / E, re = row - (row / E) * E;
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    const int o = rc % 3;                                  // curl: field c takes fields fa, fb
    const int fa = rc < 3 ? 3 + (o + 2) % 3 : (o + 2) % 3;
    const int fb = rc < 3 ? 3 + (o + 1) % 3 : (o + 1) % 3;
    const float sgn = rc < 3 ? 1.f : -1.f;
    // Item idx = pt + q * PRODUCERS is face node m of element e (idx = e * NF + m), so
    // a warp's items are consecutive face nodes of one or two elements (e < E0).
    uint32_t item[D::ITEMS];
#pragma unroll
    for (int q = 0; q < D::ITEMS; ++q) item[q] = tc_item<N>(pt + q * D::PRODUCERS, D::E0, sFmask);
    for (int t = 0; t < ntiles; ++t) {
      const int tile = base + t * ncta;
      const int k0 = tile * E, Ev = min(E, K - k0);
      const int slot = t % D::NSU, buf = t & 1;
      const float* su = sU + slot * D::U_FLOATS;
      const float* sg = sG + slot * D::G_FLOATS;
      float* F = sF;
      wait_or_flag(&s_u_full[slot], (t / D::NSU) & 1, A.status);
      // ---- fluxes (Alg. 3) of elements 0 .. E0-1 (the epilogue warps did the
      // rest one tile ahead).  F was last read in the build of tile t-1, before
      // its barrier.
      tc_flux_items<N, EXT, D::ITEMS>(item, A, k0, Ev, su, sg, F, E, 0);
      // The flux buffer is complete once every producer has stored its items:
      // roles 2 and 3 (which read it) wait for that; roles 0 and 1 only signal
      // and go on with the g blocks.
      // (barriers 3 and 4 alternate by tile, so the epilogue threads' arrivals
      // for tile t+1 never meet tile t's)
      if (role < 2) named_arrive(3 + (t & 1), D::FCOUNT);
      else named_sync(3 + (t & 1), D::FCOUNT);
      // ---- A rows of tile t
      const bool live = row < D::ROWS && re < Ev;
      const uint32_t a_hi = tbase + lane_off + buf * D::BUF_COLS;
      const uint32_t a_lo = a_hi + D::ACOLS;
      if (role >= 2) {
        // roles 2 and 3: the first and second half of the flux block's columns
        constexpr int HC = (D::COLS_F + 1) / 2;
        // flux rows of elements >= E0 are in the epilogue threads' buffer
        const float* frow = re < D::E0 ? F + (rc * E + re) * FSTR
                                       : sF2 + (t & 1) * D::F2_FLOATS +
                                             (rc * (E - D::E0) + re - D::E0) * FSTR;
        const FRow fr{frow, sBound, t, row, live, a_hi + 3 * D::COLS_G,
                      a_lo + 3 * D::COLS_G, &s_mma_done[buf], A.status};
        if (role == 2)
          build_flux_half<N, 0, HC>(fr, 2);
        else
          build_flux_half<N, HC, D::COLS_F - HC>(fr, 3);
      } else {
        // roles 0 and 1 split the node range: node pairs [0, H) and [H, KB/2) of
        // all three g blocks, each loading only its half of the two curl fields
        constexpr int H = (D::KB / 2 + 1) / 2;
        const GRow gr{su, sg, sBound, sScale, t, row, rc, re, o, fa, fb, sgn, live, a_hi, a_lo,
                      &s_mma_done[buf], A.status};
        if (role == 0)
          build_g_half<N, 0, H>(gr, 0);
        else
          build_g_half<N, H, D::KB / 2 - H>(gr, 1);
      }
      tc::tmem_st_wait();
      tc::fence_before_sync();
      tc::mbar_arrive(&s_a_full[buf]);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

template <int N, bool RK, bool EXT>
__global__ void __launch_bounds__(TcDims<N>::THREADS, 1) tc_stage_kernel(const __grid_constant__ StageArgs A) {
  pdl_launch_dependents();
  tc_stage_body<N, RK, EXT>(A, int(blockIdx.x), int(gridDim.x));
}

template <int N>
cudaError_t launch_tc_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s) {
  using D = TcDims<N>;
  static bool attr[2][2][16] = {};      // [rk][ext][device]: attribute set
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  dev &= 15;
  const bool ext = a.mat || a.absorbing;
  auto kern = rk ? (ext ? tc_stage_kernel<N, true, true> : tc_stage_kernel<N, true, false>)
                 : (ext ? tc_stage_kernel<N, false, true> : tc_stage_kernel<N, false, false>);
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

#define DG_INSTANTIATE_TC_STAGE(NN)                                                        \
  namespace dgdev {                                                                         \
  template cudaError_t launch_tc_stage_n<NN>(bool, const StageArgs&, int, cudaStream_t);    \
  }
