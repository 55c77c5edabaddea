// C ABI entry points (include/dg.h): argument checking, error reporting and
// dispatch to the host setup (refelem.cpp, mesh.cpp) and device code (device.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "device.h"
#include "dg_internal.h"

namespace {

thread_local std::string g_error;

int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

int check_mesh(const dg_mesh* m, bool need_order) {
  if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
  if (need_order && m->N == 0) return fail(DG_ERR_STATE, "dg_set_order() has not been called");
  return DG_OK;
}

}  // namespace

namespace dg {
void set_error(const std::string& msg) { g_error = msg; }
}  // namespace dg

namespace dg {
void update_dt_cfl(dg_mesh* m) {
  if (m->N == 0) return;
  double mn = INFINITY;
  for (int64_t k = 0; k < m->K; ++k) {
    const double slow = m->eps.empty() ? 1.0 : std::sqrt(m->eps[k] * m->mu[k]);
    for (int f = 0; f < 4; ++f) mn = std::fmin(mn, slow / m->Fscale[4 * k + f]);
  }
  m->dt_cfl = mn * 2.0 / ((m->N + 1.0) * (m->N + 1.0));
}

bool has_materials_or_absorbing(const dg_mesh* m) {
  if (!m->eps.empty()) return true;
  for (int8_t b : m->bc)
    if (b == DG_BC_ABSORBING) return true;
  return false;
}
}  // namespace dg

// Drops the device copy of the mesh; the next device call rebuilds it.
static void invalidate_device(dg_mesh* m) {
  if (m->dev) {
    dgdev::destroy_device_state(m->dev);
    m->dev = nullptr;
  }
}

extern "C" {

const char* dg_last_error(void) { return g_error.c_str(); }

int dg_mesh_create(const double* verts, int64_t nv, const int32_t* tets, int64_t K,
                   dg_mesh** out) {
  if (!out) return fail(DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!verts || !tets) return fail(DG_ERR_ARG, "verts or tets is NULL");
  if (nv < 4 || K < 1) return fail(DG_ERR_ARG, "need nv >= 4 and K >= 1");
  if (K >= (int64_t(1) << 31) / 220) return fail(DG_ERR_ARG, "K too large for 32-bit node ids");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  std::string err;
  int rc;
  try {
    rc = dg::mesh_build(m, verts, nv, tets, K, err);
  } catch (const std::bad_alloc&) {
    rc = DG_ERR_OOM;
    err = "host allocation failed";
  }
  if (rc != DG_OK) {
    delete m;
    return fail(rc, err);
  }
  *out = m;
  return DG_OK;
}

int dg_set_order(dg_mesh* m, int N) {
  if (int rc = check_mesh(m, false)) return rc;
  if (N < 1 || N > dg::kMaxOrder) return fail(DG_ERR_ORDER, "order N must be in 1..9");
  std::string err;
  // the reference operators depend on N only: built once per order and copied
  static std::mutex ops_mutex;
  static std::map<int, dg::RefOps> ops_cache;
  try {
    std::lock_guard<std::mutex> lock(ops_mutex);
    auto it = ops_cache.find(N);
    if (it == ops_cache.end()) {
      dg::RefOps ops;
      if (!dg::build_ref_ops(N, ops, err)) return fail(DG_ERR_ORDER, err);
      it = ops_cache.emplace(N, std::move(ops)).first;
    }
    m->ops = it->second;
  } catch (const std::bad_alloc&) {
    return fail(DG_ERR_OOM, "host allocation failed");
  }
  m->N = N;
  dg::update_dt_cfl(m);
  return DG_OK;
}

int dg_set_materials(dg_mesh* m, const double* eps, const double* mu) {
  if (int rc = check_mesh(m, false)) return rc;
  const int64_t K = m->K;
  for (const double* a : {eps, mu})
    if (a)
      for (int64_t k = 0; k < K; ++k)
        if (!std::isfinite(a[k]) || a[k] <= 0.0)
          return fail(DG_ERR_ARG, "eps and mu must be finite and > 0 (element " +
                                      std::to_string(k) + ")");
  try {
    if (!eps && !mu) {
      m->eps.clear();
      m->mu.clear();
    } else {
      m->eps.assign(K, 1.0);
      m->mu.assign(K, 1.0);
      if (eps) std::copy(eps, eps + K, m->eps.begin());
      if (mu) std::copy(mu, mu + K, m->mu.begin());
    }
  } catch (const std::bad_alloc&) {
    return fail(DG_ERR_OOM, "host allocation failed");
  }
  dg::update_dt_cfl(m);
  invalidate_device(m);
  return DG_OK;
}

int dg_set_boundary(dg_mesh* m, const int8_t* kind) {
  if (int rc = check_mesh(m, false)) return rc;
  const int64_t K = m->K;
  if (kind)
    for (int64_t i = 0; i < 4 * K; ++i)
      if (kind[i] != DG_BC_PEC && kind[i] != DG_BC_ABSORBING)
        return fail(DG_ERR_ARG, "boundary kind must be DG_BC_PEC or DG_BC_ABSORBING");
  try {
    if (kind) m->bc.assign(kind, kind + 4 * K);
    else m->bc.clear();
  } catch (const std::bad_alloc&) {
    return fail(DG_ERR_OOM, "host allocation failed");
  }
  invalidate_device(m);
  return DG_OK;
}

int dg_mesh_pack(const dg_mesh* const* meshes, int count, dg_mesh** out) {
  if (!out) return fail(DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!meshes || count < 1) return fail(DG_ERR_ARG, "need at least one mesh");
  int64_t K = 0, nv = 0;
  for (int i = 0; i < count; ++i) {
    if (int rc = check_mesh(meshes[i], true)) return rc;
    if (meshes[i]->N != meshes[0]->N) return fail(DG_ERR_ARG, "meshes of different orders");
    if (meshes[i]->alpha != meshes[0]->alpha) return fail(DG_ERR_ARG, "meshes with different fluxes");
    K += meshes[i]->K;
    nv += meshes[i]->nv;
  }
  if (K >= (int64_t(1) << 31) / 220) return fail(DG_ERR_ARG, "K too large for 32-bit node ids");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  try {
    m->K = K;
    m->nv = nv;
    m->N = meshes[0]->N;
    m->ops = meshes[0]->ops;
    m->alpha = meshes[0]->alpha;
    m->dt_cfl = INFINITY;
    m->verts.reserve(3 * nv);
    m->tets.reserve(4 * K);
    m->metric.assign(9 * K, 0.0);
    m->normals.assign(3 * 4 * K, 0.0);
    int64_t k0 = 0, v0 = 0;
    for (int i = 0; i < count; ++i) {
      const dg_mesh* s = meshes[i];
      const int64_t Ks = s->K;
      m->verts.insert(m->verts.end(), s->verts.begin(), s->verts.end());
      for (int32_t v : s->tets) m->tets.push_back(static_cast<int32_t>(v + v0));
      for (int a = 0; a < 9; ++a)
        std::copy(s->metric.begin() + a * Ks, s->metric.begin() + (a + 1) * Ks,
                  m->metric.begin() + a * K + k0);
      m->J.insert(m->J.end(), s->J.begin(), s->J.end());
      for (int d = 0; d < 3; ++d)
        std::copy(s->normals.begin() + d * Ks * 4, s->normals.begin() + (d + 1) * Ks * 4,
                  m->normals.begin() + (d * K + k0) * 4);
      m->Fscale.insert(m->Fscale.end(), s->Fscale.begin(), s->Fscale.end());
      for (int32_t e : s->nbr_elem) m->nbr_elem.push_back(static_cast<int32_t>(e + k0));
      m->nbr_code.insert(m->nbr_code.end(), s->nbr_code.begin(), s->nbr_code.end());
      m->dt_cfl = std::fmin(m->dt_cfl, s->dt_cfl);
      // materials and boundary kinds: the parts' own, defaults where a part has none
      const bool any_mat = [&] {
        for (int q = 0; q < count; ++q) if (!meshes[q]->eps.empty()) return true;
        return false;
      }();
      const bool any_bc = [&] {
        for (int q = 0; q < count; ++q) if (!meshes[q]->bc.empty()) return true;
        return false;
      }();
      if (any_mat) {
        if (s->eps.empty()) {
          m->eps.insert(m->eps.end(), Ks, 1.0);
          m->mu.insert(m->mu.end(), Ks, 1.0);
        } else {
          m->eps.insert(m->eps.end(), s->eps.begin(), s->eps.end());
          m->mu.insert(m->mu.end(), s->mu.begin(), s->mu.end());
        }
      }
      if (any_bc) {
        if (s->bc.empty()) m->bc.insert(m->bc.end(), 4 * Ks, int8_t(DG_BC_PEC));
        else m->bc.insert(m->bc.end(), s->bc.begin(), s->bc.end());
      }
      k0 += Ks;
      v0 += s->nv;
    }
  } catch (const std::bad_alloc&) {
    delete m;
    return fail(DG_ERR_OOM, "host allocation failed");
  }
  *out = m;
  return DG_OK;
}

int dg_info(const dg_mesh* m, int64_t* K, int* Np, int* Nfp, double* dt_cfl) {
  if (int rc = check_mesh(m, true)) return rc;
  if (K) *K = m->K;
  if (Np) *Np = m->ops.Np;
  if (Nfp) *Nfp = m->ops.Nfp;
  if (dt_cfl) *dt_cfl = m->dt_cfl;
  return DG_OK;
}

int dg_nodes(const dg_mesh* m, double* xyz) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!xyz) return fail(DG_ERR_ARG, "xyz is NULL");
  const int64_t K = m->K;
  const int Np = m->ops.Np;
  for (int64_t k = 0; k < K; ++k) {
    const int32_t* tv = &m->tets[4 * k];
    for (int i = 0; i < Np; ++i) {
      const double r = m->ops.r[i], s = m->ops.s[i], t = m->ops.t[i];
      const double w[4] = {-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2};
      for (int d = 0; d < 3; ++d) {
        double x = 0.0;
        for (int a = 0; a < 4; ++a) x += w[a] * m->verts[3 * tv[a] + d];
        xyz[(d * K + k) * Np + i] = x;
      }
    }
  }
  return DG_OK;
}

int dg_get_connectivity(const dg_mesh* m, int32_t* vmapM, int32_t* vmapP) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!vmapM || !vmapP) return fail(DG_ERR_ARG, "vmapM or vmapP is NULL");
  const int Np = m->ops.Np, Nfp = m->ops.Nfp;
  for (int64_t k = 0; k < m->K; ++k)
    for (int f = 0; f < 4; ++f)
      for (int j = 0; j < Nfp; ++j) {
        const int64_t idx = (k * 4 + f) * Nfp + j;
        const int32_t me = static_cast<int32_t>(k * Np + m->ops.Fmask[f * Nfp + j]);
        vmapM[idx] = me;
        const int code = m->nbr_code[4 * k + f];
        if (code < 0) {
          vmapP[idx] = me;
        } else {
          const int64_t k2 = m->nbr_elem[4 * k + f];
          vmapP[idx] = static_cast<int32_t>(k2 * Np + m->ops.perm[(f * 24 + code) * Nfp + j]);
        }
      }
  return DG_OK;
}

int dg_partition_order(const dg_mesh* m, int64_t block, int64_t* perm) {
  if (int rc = check_mesh(m, false)) return rc;
  if (!perm) return fail(DG_ERR_ARG, "perm is NULL");
  if (block < 1) return fail(DG_ERR_ARG, "block must be at least 1");
  dg::greedy_partition_order(m->nbr_elem, m->K, block, perm);
  return DG_OK;
}

int dg_get_operators(const dg_mesh* m, double* Dr, double* Ds, double* Dt, double* M,
                     double* LIFT) {
  if (int rc = check_mesh(m, true)) return rc;
  const size_t nn = m->ops.Dr.size() * sizeof(double);
  if (Dr) std::memcpy(Dr, m->ops.Dr.data(), nn);
  if (Ds) std::memcpy(Ds, m->ops.Ds.data(), nn);
  if (Dt) std::memcpy(Dt, m->ops.Dt.data(), nn);
  if (M) std::memcpy(M, m->ops.M.data(), nn);
  if (LIFT) std::memcpy(LIFT, m->ops.LIFT.data(), m->ops.LIFT.size() * sizeof(double));
  return DG_OK;
}

int dg_get_geometry(const dg_mesh* m, double* metric, double* J, double* normals,
                    double* Fscale) {
  if (int rc = check_mesh(m, false)) return rc;
  if (metric) std::memcpy(metric, m->metric.data(), m->metric.size() * sizeof(double));
  if (J) std::memcpy(J, m->J.data(), m->J.size() * sizeof(double));
  if (normals) std::memcpy(normals, m->normals.data(), m->normals.size() * sizeof(double));
  if (Fscale) std::memcpy(Fscale, m->Fscale.data(), m->Fscale.size() * sizeof(double));
  return DG_OK;
}

int dg_set_flux(dg_mesh* m, double alpha) {
  if (int rc = check_mesh(m, false)) return rc;
  if (!std::isfinite(alpha) || alpha < 0.0) return fail(DG_ERR_ARG, "alpha must be finite and >= 0");
  m->alpha = alpha;
  return DG_OK;
}

int dg_set_energy_check(dg_mesh* m, double max_growth) {
  if (int rc = check_mesh(m, false)) return rc;
  if (std::isnan(max_growth)) return fail(DG_ERR_ARG, "max_growth is NaN");
  m->energy_check = max_growth;
  return DG_OK;
}

int dg_set_stage_shape(dg_mesh* m, int shape) {
  if (int rc = check_mesh(m, false)) return rc;
  if (shape < 0 || shape >= dgdev::kStageShapes) return fail(DG_ERR_ARG, "unknown stage shape");
  m->stage_shape = shape;
  return DG_OK;
}

int dg_set_stage_impl(dg_mesh* m, int impl) {
  if (int rc = check_mesh(m, false)) return rc;
  if (impl != DG_STAGE_AUTO && impl != DG_STAGE_FP32 && impl != DG_STAGE_TC)
    return fail(DG_ERR_ARG, "unknown stage implementation");
  m->stage_impl = impl;
  return DG_OK;
}

int dg_rhs(dg_mesh* m, const float* u, float* rhs, void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u || !rhs) return fail(DG_ERR_ARG, "u or rhs is NULL");
  if (u == rhs) return fail(DG_ERR_ARG, "rhs must not alias u");
  std::string err;
  if (int rc = dg::device_rhs(m, u, rhs, stream, err)) return fail(rc, err);
  return DG_OK;
}

int dg_step(dg_mesh* m, float* u, float* res, double dt, int nsteps, void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u || !res) return fail(DG_ERR_ARG, "u or res is NULL");
  if (u == res) return fail(DG_ERR_ARG, "res must not alias u");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be positive and finite");
  if (nsteps < 0) return fail(DG_ERR_ARG, "nsteps must be >= 0");
  std::string err;
  if (int rc = dg::device_step(m, u, res, dt, nsteps, stream, err)) return fail(rc, err);
  return DG_OK;
}

int dg_rk_stage(dg_mesh* m, const float* u_in, float* u_out, float* res, int stage, double dt,
                void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u_in || !u_out || !res) return fail(DG_ERR_ARG, "u_in, u_out or res is NULL");
  if (u_in == u_out || res == u_in || res == u_out)
    return fail(DG_ERR_ARG, "u_in, u_out and res must be three different buffers");
  if (stage < 0 || stage > 4) return fail(DG_ERR_ARG, "stage must be 0..4");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be positive and finite");
  std::string err;
  if (int rc = dg::device_stage(m, u_in, u_out, res, stage, dt, nullptr, stream, err))
    return fail(rc, err);
  return DG_OK;
}

int dg_rk_stage_range(dg_mesh* m, const float* u_in, float* u_out, float* res, int stage,
                      double dt, int64_t k0, int64_t k1, void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u_in || !u_out || !res) return fail(DG_ERR_ARG, "u_in, u_out or res is NULL");
  if (u_in == u_out || res == u_in || res == u_out)
    return fail(DG_ERR_ARG, "u_in, u_out and res must be three different buffers");
  if (stage < 0 || stage > 4) return fail(DG_ERR_ARG, "stage must be 0..4");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be positive and finite");
  if (k0 < 0 || k1 <= k0 || k1 > m->K) return fail(DG_ERR_ARG, "need 0 <= k0 < k1 <= K");
  std::string err;
  if (int rc = dg::device_stage(m, u_in, u_out, res, stage, dt, nullptr, stream, err, k0, k1))
    return fail(rc, err);
  return DG_OK;
}

int dg_check_wait_timeout(dg_mesh* m, uint32_t polls, double* seconds) {
  if (int rc = check_mesh(m, true)) return rc;
  if (polls < 1 || polls > (1u << 24)) return fail(DG_ERR_ARG, "polls outside 1 .. 2^24");
  std::string err;
  if (int rc = dg::device_wait_selftest(m, polls, seconds, err)) return fail(rc, err);
  return fail(DG_ERR_STATE, "bounded wait self-test: the wait did not time out");
}

int dg_stage_tile(dg_mesh* m, const float* u_in, const float* u_out, const float* res, int* tile) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!tile) return fail(DG_ERR_ARG, "tile is NULL");
  std::string err;
  if (int rc = dg::device_stage_tile(m, u_in, u_out, res, tile, err)) return fail(rc, err);
  return DG_OK;
}

int dg_rk_stage_elem(dg_mesh* m, const float* u_in, float* u_out, float* res, int stage,
                     const float* dt_elem, void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u_in || !u_out || !res || !dt_elem)
    return fail(DG_ERR_ARG, "u_in, u_out, res or dt_elem is NULL");
  if (u_in == u_out || res == u_in || res == u_out)
    return fail(DG_ERR_ARG, "u_in, u_out and res must be three different buffers");
  if (stage < 0 || stage > 4) return fail(DG_ERR_ARG, "stage must be 0..4");
  std::string err;
  if (int rc = dg::device_stage(m, u_in, u_out, res, stage, 1.0, dt_elem, stream, err))
    return fail(rc, err);
  return DG_OK;
}

int dg_rk_stage_multi(dg_mesh* const* meshes, int n, const float* const* u_in,
                      float* const* u_out, float* const* res, const float* const* dt_elem,
                      int stage, double dt, const double* tile_cost, void* stream) {
  if (!meshes || n < 1 || !u_in || !u_out || !res)
    return fail(DG_ERR_ARG, "meshes, u_in, u_out or res is NULL, or n < 1");
  if (stage < 0 || stage > 4) return fail(DG_ERR_ARG, "stage must be 0..4");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be positive and finite");
  for (int i = 0; i < n; ++i) {
    if (int rc = check_mesh(meshes[i], true)) return rc;
    if (!u_in[i] || !u_out[i] || !res[i])
      return fail(DG_ERR_ARG, "u_in, u_out or res of mesh " + std::to_string(i) + " is NULL");
    if (u_in[i] == u_out[i] || res[i] == u_in[i] || res[i] == u_out[i])
      return fail(DG_ERR_ARG, "u_in, u_out and res must be three different buffers");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) return fail(DG_ERR_ARG, "a mesh appears twice");
  }
  std::string err;
  if (int rc = dg::device_stage_multi(meshes, n, u_in, u_out, res, dt_elem, stage, dt, tile_cost,
                                      stream, err))
    return fail(rc, err);
  return DG_OK;
}

int dg_energy_range(dg_mesh* m, const float* u, int64_t k0, int64_t k1, double* out,
                    void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u || !out) return fail(DG_ERR_ARG, "u or out is NULL");
  if (k0 < 0 || k1 <= k0 || k1 > m->K) return fail(DG_ERR_ARG, "need 0 <= k0 < k1 <= K");
  std::string err;
  if (int rc = dg::device_energy_range(m, u, k0, k1, out, stream, err)) return fail(rc, err);
  return DG_OK;
}

int dg_energy(dg_mesh* m, const float* u, double* out, void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u || !out) return fail(DG_ERR_ARG, "u or out is NULL");
  std::string err;
  if (int rc = dg::device_energy(m, u, out, stream, err)) return fail(rc, err);
  return DG_OK;
}

int dg_step_host(dg_mesh* m, float* u, float* res, double dt, int nsteps, double* energy,
                 void* stream) {
  if (int rc = check_mesh(m, true)) return rc;
  if (!u) return fail(DG_ERR_ARG, "u is NULL");
  if (u == res) return fail(DG_ERR_ARG, "res must not alias u");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be positive and finite");
  if (nsteps < 0) return fail(DG_ERR_ARG, "nsteps must be >= 0");
  std::string err;
  if (int rc = dg::device_step_host(m, u, res, dt, nsteps, energy, stream, err)) return fail(rc, err);
  return DG_OK;
}

int64_t dg_last_launch_count(const dg_mesh* m) { return m ? m->last_launches : 0; }

int dg_trace_enable(dg_mesh* m, int n) {
  if (int rc = check_mesh(m, false)) return rc;
  if (n < 0) return fail(DG_ERR_ARG, "n must be >= 0");
  m->trace = n > 0;
  if (n == 0) return DG_OK;
  if (int rc = check_mesh(m, true)) return rc;
  std::string err;
  if (int rc = dg::device_trace_reset(m, n, err)) return fail(rc, err);
  return DG_OK;
}

int dg_trace_read(dg_mesh* m, double* ms, int32_t* kind, int64_t cap, int64_t* count) {
  if (int rc = check_mesh(m, false)) return rc;
  if (!count || (cap > 0 && !ms) || cap < 0) return fail(DG_ERR_ARG, "bad output arguments");
  std::string err;
  if (int rc = dg::device_trace_read(m, ms, kind, cap, count, err)) return fail(rc, err);
  return DG_OK;
}

void dg_mesh_destroy(dg_mesh* m) {
  if (!m) return;
  dgdev::destroy_device_state(m->dev);
  delete m;
}

}  // extern "C"
