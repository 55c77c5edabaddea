// Mesh validation, element geometry and element connectivity, FP64, host.
//
// Section 2 (Eq. dg-reference-matrices): each tetrahedron is the affine image
// x = v0 + [v1-v0, v2-v0, v3-v0] ((r,s,t)+1)/2 of the reference element, so
// J = det(dx/dr) and the chain-rule coefficients dr_mu/dx_nu are constant per
// element.  Face normals are the reference face normals pushed through the
// inverse metric, n = (dr/dx)^T nhat / |.|, with nhat = -grad t, -grad s,
// grad(r+s+t), -grad r for faces f0..f3; the surface Jacobian of the face
// parameterisation is sJ = |(dr/dx)^T nhat| J, so the lifting scale is
// Fscale = sJ/J.  Faces are matched across elements by sorting their vertex
// triples (the face-pair information of Section 5.2); an unmatched face is a
// perfectly conducting wall.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>

#include "dg_internal.h"

namespace dg {

int mesh_build(dg_mesh* m, const double* verts, int64_t nv, const int32_t* tets, int64_t K,
               std::string& err) {
  m->nv = nv;
  m->K = K;
  m->verts.assign(verts, verts + 3 * nv);
  m->tets.assign(tets, tets + 4 * K);
  double scale = 0.0;
  for (int64_t i = 0; i < 3 * nv; ++i) {
    if (!std::isfinite(verts[i])) { err = "non-finite vertex coordinate"; return DG_ERR_ARG; }
    scale = std::max(scale, std::fabs(verts[i]));
  }
  m->metric.assign(9 * K, 0.0);
  m->J.assign(K, 0.0);
  m->normals.assign(3 * 4 * K, 0.0);
  m->Fscale.assign(4 * K, 0.0);

  for (int64_t k = 0; k < K; ++k) {
    int32_t* tv = &m->tets[4 * k];
    for (int a = 0; a < 4; ++a)
      if (tv[a] < 0 || tv[a] >= nv) {
        err = "tetrahedron " + std::to_string(k) + " has a vertex index out of range";
        return DG_ERR_MESH;
      }
    double xr[3][3];  // xr[d][mu] = d x_d / d r_mu
    auto fill = [&]() {
      for (int mu = 0; mu < 3; ++mu)
        for (int d = 0; d < 3; ++d)
          xr[d][mu] = 0.5 * (verts[3 * tv[mu + 1] + d] - verts[3 * tv[0] + d]);
    };
    fill();
    auto det3 = [&]() {
      return xr[0][0] * (xr[1][1] * xr[2][2] - xr[1][2] * xr[2][1]) -
             xr[0][1] * (xr[1][0] * xr[2][2] - xr[1][2] * xr[2][0]) +
             xr[0][2] * (xr[1][0] * xr[2][1] - xr[1][1] * xr[2][0]);
    };
    double J = det3();
    if (!(std::fabs(J) > 1e-14 * scale * scale * scale) ) {
      err = "tetrahedron " + std::to_string(k) + " is degenerate (zero volume)";
      return DG_ERR_MESH;
    }
    if (J < 0) {  // orientation: swap the last two vertices
      std::swap(tv[2], tv[3]);
      fill();
      J = det3();
    }
    m->J[k] = J;
    // inverse metric: row mu of (dx/dr)^-1 = grad r_mu
    double G[3][3];
    for (int mu = 0; mu < 3; ++mu)
      for (int d = 0; d < 3; ++d) {
        const int a1 = (d + 1) % 3, a2 = (d + 2) % 3, b1 = (mu + 1) % 3, b2 = (mu + 2) % 3;
        G[mu][d] = (xr[a1][b1] * xr[a2][b2] - xr[a1][b2] * xr[a2][b1]) / J;
      }
    for (int mu = 0; mu < 3; ++mu)
      for (int d = 0; d < 3; ++d) m->metric[(3 * mu + d) * K + k] = G[mu][d];
    // faces: nhat = -grad t, -grad s, grad r + grad s + grad t, -grad r
    for (int f = 0; f < 4; ++f) {
      double n[3];
      for (int d = 0; d < 3; ++d) {
        if (f == 0) n[d] = -G[2][d];
        else if (f == 1) n[d] = -G[1][d];
        else if (f == 2) n[d] = G[0][d] + G[1][d] + G[2][d];
        else n[d] = -G[0][d];
      }
      const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int d = 0; d < 3; ++d) m->normals[(d * K + k) * 4 + f] = n[d] / len;
      m->Fscale[k * 4 + f] = len;  // sJ / J
    }
  }

  // face matching by sorted vertex triples
  struct FaceKey { std::array<int32_t, 3> v; int64_t kf; };
  std::vector<FaceKey> keys(4 * K);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      std::array<int32_t, 3> v = {m->tets[4 * k + kFaceVerts[f][0]], m->tets[4 * k + kFaceVerts[f][1]],
                                  m->tets[4 * k + kFaceVerts[f][2]]};
      std::sort(v.begin(), v.end());
      keys[4 * k + f] = {v, 4 * k + f};
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey& a, const FaceKey& b) {
    return a.v != b.v ? a.v < b.v : a.kf < b.kf;
  });
  m->nbr_elem.assign(4 * K, 0);
  m->nbr_code.assign(4 * K, -1);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) m->nbr_elem[4 * k + f] = static_cast<int32_t>(k);
  for (size_t a = 0; a < keys.size();) {
    size_t b = a + 1;
    while (b < keys.size() && keys[b].v == keys[a].v) ++b;
    if (b - a > 2) { err = "a face is shared by more than two tetrahedra"; return DG_ERR_MESH; }
    if (b - a == 2) {
      for (int side = 0; side < 2; ++side) {
        const int64_t me = keys[a + side].kf, other = keys[a + 1 - side].kf;
        const int64_t k1 = me / 4, k2 = other / 4;
        const int f1 = static_cast<int>(me % 4), f2 = static_cast<int>(other % 4);
        if (k1 == k2) { err = "a tetrahedron shares a face with itself"; return DG_ERR_MESH; }
        // sigma: my face vertex p is the neighbour's face vertex sigma(p)
        int q[3];
        for (int p = 0; p < 3; ++p) {
          q[p] = -1;
          for (int c = 0; c < 3; ++c)
            if (m->tets[4 * k2 + kFaceVerts[f2][c]] == m->tets[4 * k1 + kFaceVerts[f1][p]]) q[p] = c;
        }
        int sg = -1;
        for (int s = 0; s < 6; ++s)
          if (kPerm3[s][0] == q[0] && kPerm3[s][1] == q[1] && kPerm3[s][2] == q[2]) sg = s;
        if (sg < 0) { err = "inconsistent face vertices"; return DG_ERR_MESH; }
        m->nbr_elem[me] = static_cast<int32_t>(k2);
        m->nbr_code[me] = f2 * 6 + sg;
      }
    }
    a = b;
  }
  return DG_OK;
}

}  // namespace dg
