// Device-side data of a mesh and the kernel launch interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dgdev {

// Per-element geometry record, 32 words (128 bytes), one per tetrahedron:
//   [0..8]   rx ry rz sx sy sz tx ty tz   (dr_mu/dx_nu, Eq. dg-reference-matrices)
//   [9]      J
//   [10]     neighbour codes, byte f = (g*6 + sigma) + 1 of face f, 0 = wall
//   [11]     unused
//   [12+4f .. 15+4f]  nx ny nz Fscale of face f
//   [28+f]   neighbour element of face f (int32; itself on a wall)
constexpr int kGeoWords = 32;
// Neighbour code byte of a characteristic absorbing boundary face (0: perfect
// conductor, 1..24: interior face).
constexpr unsigned kAbsorbingCode = 0xFFu;
// Optional material record, 5 float4 per tetrahedron (meshes with materials):
//   [0]      1/eps, 1/mu, eps, mu
//   [1 + f]  Z+, B_E, Y+, B_H of face f: the flux of Section 6 is
//            B_E (Z+ (-n x dH) + alpha (n (n.dE) - dE)) for E and
//            B_H (Y+ ( n x dE) + alpha (n (n.dH) - dH)) for H (d = u- - u+),
//            B_E = 1/(Z- + Z+), B_H = 1/(Y- + Y+), Z+ / Y+ the neighbour's
//            impedance / admittance (the element's own on boundary faces);
//            vacuum: 1, 1/2, 1, 1/2.
constexpr int kMatVecs = 5;

// Stage-kernel tiling per order N: tile of E tetrahedra, G row groups (threads
// = E * G).  Shape 0 (the default) chosen so a thread holds at most 7 rows and
// the shared tiles of one CTA stay near 100 KB (sizes measured fastest on the
// order sweep's meshes of ~1.7e7 DOFs); shape 1 halves the elements per tile (twice the CTAs of a small mesh, half the shared tiles) with the
// same rows per thread.  The autotuner of the serving loop picks per order
// and size (dg_set_stage_shape).
constexpr int kStageShapes = 2;
__host__ __device__ constexpr int stage_tile_elems(int N, int shape = 0) {
  // N = 1: 16 per tile by default (measured 16 % faster than 32 on 705 894 tets)
  return shape == 0 ? (N == 1 ? 16 : N <= 5 ? 32 : N == 6 ? 12 : N == 7 ? 16 : 8)  // N = 6: room for its operators
                    : (N == 1 ? 8 : N <= 5 ? 16 : N == 6 ? 6 : N == 7 ? 8 : 4);
}

struct StageArgs {
  const float* u_in;       // [6][K][Np]
  float* u_out;            // [6][K][Np] (RK mode)
  float* res;              // [6][K][Np] (RK mode, in/out)
  float* rhs;              // [6][K][Np] (RHS mode)
  const float4* geo;       // [K][8] float4
  const float4* D4;        // [Np][Np] (Dr, Ds, Dt, 0)
  const float4* LIFT4;     // [Np][4*Nfp/4]
  const unsigned char* fmask;  // [4][Nfp]
  const unsigned char* perm;   // [4][24][Nfp]
  int K;
  int num_tiles;           // tiles of this launch: tile0, tile0 + 1, ..., tile0 + num_tiles - 1
  int tile0;               // first tile (0: the whole mesh; dg_rk_stage_range: a sub-range)
  float a, b, dt, alpha;
  const float* dt_elem;    // RK mode: per-element time step [K], or null for dt
  const float4* mat;       // [K][kMatVecs] material record, or null (vacuum)
  // tensor-core path only
  const float* tcgeo;       // per tile: [kTcGeoWords][tc_tile_elems(N)] word-major geometry
  int tc_geo_stride;        // floats per tile block
  const void* tcB;          // FP16 [Dr Ds Dt LIFT] hi/lo pieces: orders <= 4 in the canonical
                            // K-major shared-memory layout, orders 5..7 as tensor-memory rows
  float tc_inv_bscale;      // 1 / (power-of-two scale applied to [Dr Ds Dt LIFT])
  int* status;              // set to 1 if an MMA completion wait timed out
  int absorbing;            // 1 if any boundary face is absorbing (code kAbsorbingCode)
};

// Tensor-core stage: elements per tile.  Orders <= 4: 6 * 20 = 120 of the 128
// MMA rows (fields are the A operand); orders 5..7: 6 * 8 = 48 MMA columns
// (fields are the B operand, the operator sits in tensor memory).
constexpr int kTcTileElems = 20;
constexpr int kTtTileElems = 8;
__host__ __device__ constexpr int tc_tile_elems(int N) { return N <= 4 ? kTcTileElems : kTtTileElems; }
// Word-major geometry for the tensor-core stage: words 0..8 metric, 9 packed
// neighbour codes, 10 + 4f .. 13 + 4f normal and Fscale of face f, 26 + f
// neighbour element of face f.
constexpr int kTcGeoWords = 30;
constexpr int kTcMaxOrder = 7;
// Floats of one tile's geometry block: kTcGeoWords x E words, then E * 4 Nfp
// neighbour-node bytes (a multiple of 16 bytes), E = tc_tile_elems(N).
__host__ __device__ constexpr int tc_geo_floats(int N) {
  return kTcGeoWords * tc_tile_elems(N) + tc_tile_elems(N) * 4 * ((N + 1) * (N + 2) / 2) / 4;
}
// Orders 5..7: [Dr Ds Dt LIFT] columns (K) with each derivative block padded to
// whole 8-value chunks, and tensor-memory columns of one FP16 operator piece.
__host__ __device__ constexpr int tt_kb(int N) { return (((N + 1) * (N + 2) * (N + 3) / 6) + 7) & ~7; }
__host__ __device__ constexpr int tt_kt(int N) { return (3 * tt_kb(N) + 4 * ((N + 1) * (N + 2) / 2) + 15) & ~15; }
__host__ __device__ constexpr int tt_acols(int N) { return tt_kt(N) / 2; }
// Bytes of the prepared B buffer for order N (two FP16 pieces of NN x KT).
__host__ __device__ constexpr int tc_b_bytes(int N) {
  return 2 * 2 * ((((N + 1) * (N + 2) * (N + 3) / 6) + 15) & ~15) *
         ((3 * ((((N + 1) * (N + 2) * (N + 3) / 6) + 1) & ~1) + 4 * ((N + 1) * (N + 2) / 2) + 15) & ~15);
}

// One launch over the packs of several meshes (a group per mesh): the grid's
// CTAs are split among the groups, CTAs [first, first + count) running group g
// (its mesh, its order, its fields) as a persistent stage of `count` CTAs.
constexpr int kMaxMixedGroups = 8;
struct MixedGroup {
  StageArgs a;
  int N;
  int ext;                 // 1: materials or absorbing faces (the EXT instantiation)
  int first, count;
};
struct MixedArgs {
  MixedGroup g[kMaxMixedGroups];
  int ngroups;
};
// Fused RK stages of groups of orders 1..4 (tensor cores, one 640-thread CTA
// per SM) or of orders 5, 6 (tensor cores, operator in tensor memory); order 7
// always launches alone.
cudaError_t launch_tc_mixed(const MixedArgs& m, int grid, cudaStream_t s);
cudaError_t launch_tt_mixed(const MixedArgs& m, int grid, cudaStream_t s);

// Launches one RK stage (rk = true: res <- a res + dt rhs, u_out <- u_in + b res)
// or one bare right-hand-side evaluation (rk = false: rhs <- rhs(u_in)).
cudaError_t launch_stage(int N, bool rk, const StageArgs& a, int num_sms, cudaStream_t s,
                         int shape = 0);
cudaError_t launch_tc_stage(int N, bool rk, const StageArgs& a, int num_sms, cudaStream_t s);
// One warp waits (bounded by `polls`) on an mbarrier nothing arrives at: the
// timeout sets *status as in the tensor-core stages; *ns = the wait's duration.
cudaError_t launch_wait_selftest(int* status, uint32_t polls, unsigned long long* ns,
                                 cudaStream_t s);

struct EnergyArgs {
  const float* u;      // [6][K][Np]
  const float* M;      // [Np][Np]
  const float4* geo;   // for J
  int K, Np;
  double* partials;    // [grid]
  double* result;      // [1]
  int k0, k1;          // elements k0 <= k < k1 (0, K: the whole mesh)
  const float4* mat;   // material record (E rows weighted by eps, H rows by mu), or null
};
int energy_grid(int num_sms);
cudaError_t launch_energy_partials(const EnergyArgs& a, int grid, cudaStream_t s);
cudaError_t launch_energy_final(const EnergyArgs& a, int grid, cudaStream_t s);

}  // namespace dgdev
