// Internal host-side data structures of the DG Maxwell library.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dg.h"

namespace dg {

constexpr int kMaxOrder = 9;

inline int np_of(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
inline int nfp_of(int N) { return (N + 1) * (N + 2) / 2; }

// Local vertex numbers of each face, in face order (f0: t=-1, f1: s=-1,
// f2: r+s+t=-1, f3: r=-1 on the reference element).
extern const int kFaceVerts[4][3];

// Reference-element operators of order N, FP64 (Section 2).
struct RefOps {
  int N = 0, Np = 0, Nfp = 0;
  std::vector<double> r, s, t;   // Warp & Blend nodes
  std::vector<int> Fmask;        // [4][Nfp] node index of each face node, ascending
  std::vector<double> Dr, Ds, Dt;  // [Np][Np]
  std::vector<double> M;         // [Np][Np] mass matrix
  std::vector<double> LIFT;      // [Np][4*Nfp]
  // perm[((f*4 + g)*6 + sigma)*Nfp + j]: local node index, in the neighbour,
  // of face node j of my face f when the neighbour sees it as its face g with
  // vertex permutation sigma (see face_sigma()).
  std::vector<int> perm;
};

// Builds every reference operator for order N (1..kMaxOrder).
bool build_ref_ops(int N, RefOps& ops, std::string& err);

// The six permutations of (0,1,2), in lexicographic order.
extern const int kPerm3[6][3];

}  // namespace dg

namespace dgdev {
struct DeviceState;
void destroy_device_state(DeviceState*);
}

struct dg_mesh {
  int64_t nv = 0, K = 0;
  std::vector<double> verts;      // [nv][3]
  std::vector<int32_t> tets;      // [K][4], orientation-corrected
  // element geometry (order independent), FP64
  std::vector<double> metric;     // [9][K]: rx ry rz sx sy sz tx ty tz
  std::vector<double> J;          // [K]
  std::vector<double> normals;    // [3][K][4]
  std::vector<double> Fscale;     // [K][4]
  // element connectivity: neighbour element and code g*6+sigma (-1: wall)
  std::vector<int32_t> nbr_elem;  // [K][4]
  std::vector<int32_t> nbr_code;  // [K][4]
  // order dependent
  int N = 0;
  dg::RefOps ops;
  double dt_cfl = 0.0;
  double alpha = 1.0;
  // materials and boundary kinds (empty: vacuum, every boundary face PEC)
  std::vector<double> eps, mu;    // [K]
  std::vector<int8_t> bc;         // [K][4], DG_BC_* (read on boundary faces)
  dgdev::DeviceState* dev = nullptr;
  int64_t last_launches = 0;
  bool trace = false;
  int stage_impl = DG_STAGE_AUTO;
  int stage_shape = 0;            // FP32 stage tile shape (dg_set_stage_shape)
  double energy_check = -1.0;     // dg_step_host energy-growth limit (< 0: off)
};

namespace dg {
// dt_cfl of the current order: min over k, f of sqrt(eps_k mu_k) / Fscale_kf, times 2 / (N + 1)^2
void update_dt_cfl(dg_mesh* m);
// true when the mesh has materials or absorbing boundary faces
bool has_materials_or_absorbing(const dg_mesh* m);
// mesh.cpp
int mesh_build(dg_mesh* m, const double* verts, int64_t nv, const int32_t* tets, int64_t K,
               std::string& err);
// capi.cpp: sets the message returned by dg_last_error() on this thread
void set_error(const std::string& msg);
// perm[i] = element placed at position i by the greedy partition (Alg. 2).
void greedy_partition_order(const std::vector<int32_t>& nbr, int64_t K, int64_t block,
                            int64_t* perm);
// device.cu (stream = cudaStream_t)
int device_rhs(dg_mesh* m, const float* u, float* rhs, void* stream, std::string& err);
// k1 >= 0: only the elements [k0, k1), whole tiles of the stage kernel that runs
int device_stage(dg_mesh* m, const float* u_in, float* u_out, float* res, int stage, double dt,
                 const float* dt_elem, void* stream, std::string& err, int64_t k0 = 0,
                 int64_t k1 = -1);
// tetrahedra per tile of the stage kernel these buffers would run
int device_wait_selftest(dg_mesh* m, uint32_t polls, double* seconds, std::string& err);
int device_stage_tile(dg_mesh* m, const float* u_in, const float* u_out, const float* res,
                      int* tile, std::string& err);
int device_step(dg_mesh* m, float* u, float* res, double dt, int nsteps, void* stream,
                std::string& err);
int device_stage_multi(dg_mesh* const* ms, int n, const float* const* u_in, float* const* u_out,
                       float* const* res, const float* const* dt_elem, int stage, double dt,
                       const double* tile_cost, void* stream, std::string& err);
int device_energy(dg_mesh* m, const float* u, double* out, void* stream, std::string& err);
int device_energy_range(dg_mesh* m, const float* u, int64_t k0, int64_t k1, double* out,
                        void* stream, std::string& err);
int device_step_host(dg_mesh* m, float* u, float* res, double dt, int nsteps, double* energy,
                     void* stream, std::string& err);
int device_trace_reset(dg_mesh* m, int reserve, std::string& err);
// Device copies of M, the geometry records and the material records (null in
// vacuum) if the mesh is resident on the current device at its current order
// (no allocation), else DG_ERR_STATE.
int device_resident(const dg_mesh* m, const float** M, const void** geo, const void** mat,
                    int64_t* K, int* Np, std::string& err);
int device_trace_read(dg_mesh* m, double* ms, int32_t* kind, int64_t cap, int64_t* count,
                      std::string& err);
// Calls launch(ctx) (which launches one kernel on `stream` and returns its
// cudaError_t as an int); while tracing is on, brackets it with a pair of
// events recorded under `kind` (the record of dg_trace_read).
int trace_launch(dg_mesh* m, void* stream, int kind, int (*launch)(void*), void* ctx);
}  // namespace dg
