// Reference-element operators of the nodal DG method on tetrahedra, FP64, host.
//
// Section 2 of the paper: the solution on each element is a polynomial of
// total degree N represented by its values at Np interpolation nodes
// (Warburton's explicit Warp & Blend nodes); the method needs the reference
// mass matrix M, the differentiation matrices D^r, D^s, D^t (Eq.
// dg-global-matrices with D = M^-1 S) and the lifting matrix
// LIFT = M^-1 [M^A1 .. M^A4] (Fig. lifting-matrix).  They are built here from
// an orthonormal (Koornwinder-Dubiner) basis psi_n of P_N on the reference
// tetrahedron: with V_in = psi_n(x_i),
//     M = (V V^T)^-1,   D^r = V_r V^-1,   M^A_f = (V_f V_f^T)^-1 on face f
// (V_f the 2-D orthonormal Vandermonde of the face nodes), LIFT = V V^T E.
#include <cmath>
#include <cstdio>
#include <algorithm>

#include "dg_internal.h"

namespace dg {

const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

namespace {

// ---------------------------------------------------------------- Jacobi ---
// Orthonormal Jacobi polynomial P_n^(a,b)(x) on [-1,1], weight (1-x)^a (1+x)^b,
// by the three-term recurrence of the orthonormal family.
double jacobi(int n, double a, double b, double x) {
  const double g0 = std::pow(2.0, a + b + 1) / (a + b + 1) * std::tgamma(a + 1) *
                    std::tgamma(b + 1) / std::tgamma(a + b + 1);
  double p0 = 1.0 / std::sqrt(g0);
  if (n == 0) return p0;
  const double g1 = (a + 1) * (b + 1) / (a + b + 3) * g0;
  double p1 = ((a + b + 2) * x / 2 + (a - b) / 2) / std::sqrt(g1);
  if (n == 1) return p1;
  double aold = 2.0 / (2 + a + b) * std::sqrt((a + 1) * (b + 1) / (a + b + 3));
  for (int i = 1; i < n; ++i) {
    const double h = 2.0 * i + a + b;
    const double anew = 2.0 / (h + 2) *
        std::sqrt((i + 1) * (i + 1 + a + b) * (i + 1 + a) * (i + 1 + b) / ((h + 1) * (h + 3)));
    const double bnew = -(a * a - b * b) / (h * (h + 2));
    const double p2 = ((x - bnew) * p1 - aold * p0) / anew;
    p0 = p1;
    p1 = p2;
    aold = anew;
  }
  return p1;
}

// d/dx of the orthonormal P_n^(a,b): sqrt(n (n+a+b+1)) P_{n-1}^(a+1,b+1).
double djacobi(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + a + b + 1)) * jacobi(n - 1, a + 1, b + 1, x);
}

// Gauss-Lobatto-Legendre points: -1, the zeros of P_{n-1}^(1,1), +1.
std::vector<double> lgl(int n) {
  std::vector<double> x(n + 1);
  x[0] = -1.0;
  x[n] = 1.0;
  for (int k = 1; k < n; ++k) {
    double z = -std::cos(M_PI * k / n);
    for (int it = 0; it < 100; ++it) {
      const double f = jacobi(n - 1, 1, 1, z), df = djacobi(n - 1, 1, 1, z);
      const double dz = f / df;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[k] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

// ------------------------------------------------------- Warp & Blend nodes ---
// 1-D warp: equidistant->LGL displacement interpolated on the equidistant
// points, divided by (1 - x^2); zero at the end points.
double warp1d(int N, const std::vector<double>& disp, double x) {
  double w = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double xi = -1.0 + 2.0 * i / N;
    double l = 1.0;
    for (int j = 0; j <= N; ++j)
      if (j != i) l *= (x - (-1.0 + 2.0 * j / N)) / (xi - (-1.0 + 2.0 * j / N));
    w += disp[i] * l;
  }
  if (std::fabs(x) < 1.0 - 1e-10) return w / (1.0 - x * x);
  return 0.0;
}

// In-plane displacement of a point with barycentric (l1,l2,l3) on an
// equilateral triangle with vertices (0,2/sqrt3), (-1,-1/sqrt3), (1,-1/sqrt3).
void face_shift(int N, double alpha, const std::vector<double>& disp, double l1, double l2,
                double l3, double* dx, double* dy) {
  const double w1 = 4 * l2 * l3 * warp1d(N, disp, l3 - l2) * (1 + (alpha * l1) * (alpha * l1));
  const double w2 = 4 * l1 * l3 * warp1d(N, disp, l1 - l3) * (1 + (alpha * l2) * (alpha * l2));
  const double w3 = 4 * l1 * l2 * warp1d(N, disp, l2 - l1) * (1 + (alpha * l3) * (alpha * l3));
  *dx = w1 + std::cos(2 * M_PI / 3) * w2 + std::cos(4 * M_PI / 3) * w3;
  *dy = std::sin(2 * M_PI / 3) * w2 + std::sin(4 * M_PI / 3) * w3;
}

// Blend parameter per order (Warburton 2006), orders 1..15.
const double kAlpha[15] = {0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577,
                           1.1603, 1.10153, 0.6080, 0.4523, 0.8856, 0.8717, 0.9655};

void nodes3d(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& t) {
  const double alpha = kAlpha[N - 1];
  const double q3 = std::sqrt(3.0), q6 = std::sqrt(6.0);
  const double V[4][3] = {{-1, -1 / q3, -1 / q6}, {1, -1 / q3, -1 / q6},
                          {0, 2 / q3, -1 / q6}, {0, 0, 3 / q6}};
  // face frames: t1 along the face edge, t2 in-plane towards the third vertex
  double T1[4][3], T2[4][3];
  const int e1[4][2] = {{0, 1}, {0, 1}, {1, 2}, {0, 2}};   // t1 = V[b]-V[a]
  const int apex[4] = {2, 3, 3, 3};                         // t2 = V[apex]-mid
  for (int f = 0; f < 4; ++f) {
    double n1 = 0, n2 = 0;
    for (int d = 0; d < 3; ++d) {
      T1[f][d] = V[e1[f][1]][d] - V[e1[f][0]][d];
      T2[f][d] = V[apex[f]][d] - 0.5 * (V[e1[f][0]][d] + V[e1[f][1]][d]);
      n1 += T1[f][d] * T1[f][d];
      n2 += T2[f][d] * T2[f][d];
    }
    for (int d = 0; d < 3; ++d) { T1[f][d] /= std::sqrt(n1); T2[f][d] /= std::sqrt(n2); }
  }
  const std::vector<double> g = lgl(N);
  std::vector<double> disp(N + 1);
  for (int i = 0; i <= N; ++i) disp[i] = g[i] - (-1.0 + 2.0 * i / N);

  // inverse of the equilateral->reference affine map
  double A[3][3];
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) A[d][c] = 0.5 * (V[c + 1][d] - V[0][d]);
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  double Ai[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
      Ai[i][j] = (A[i1][j1] * A[i2][j2] - A[i1][j2] * A[i2][j1]) / det;
    }
  double c0[3];
  for (int d = 0; d < 3; ++d) c0[d] = 0.5 * (V[1][d] + V[2][d] + V[3][d] - V[0][d]);

  r.clear(); s.clear(); t.clear();
  const double tol = 1e-10;
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N - k; ++j)
      for (int i = 0; i <= N - k - j; ++i) {
        const double r0 = -1.0 + 2.0 * i / N, s0 = -1.0 + 2.0 * j / N, t0 = -1.0 + 2.0 * k / N;
        // barycentric: L[0..3] for vertices v1..v4 of the reference element
        const double L[4] = {-(1 + r0 + s0 + t0) / 2, (1 + r0) / 2, (1 + s0) / 2, (1 + t0) / 2};
        double X[3];
        for (int d = 0; d < 3; ++d)
          X[d] = L[0] * V[0][d] + L[1] * V[1][d] + L[2] * V[2][d] + L[3] * V[3][d];
        // face f: (La opposite vertex, Lb apex, Lc, Ld along the edge)
        const double Lf[4][4] = {{L[3], L[2], L[0], L[1]},
                                 {L[2], L[3], L[0], L[1]},
                                 {L[0], L[3], L[1], L[2]},
                                 {L[1], L[3], L[0], L[2]}};
        double sh[3] = {0, 0, 0};
        for (int f = 0; f < 4; ++f) {
          const double La = Lf[f][0], Lb = Lf[f][1], Lc = Lf[f][2], Ld = Lf[f][3];
          double wx, wy;
          face_shift(N, alpha, disp, Lb, Lc, Ld, &wx, &wy);
          double blend = Lb * Lc * Ld;
          const double den = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La);
          if (den > tol) blend = (1 + (alpha * La) * (alpha * La)) * blend / den;
          const int npos = (Lb > tol) + (Lc > tol) + (Ld > tol);
          if (La < tol && npos < 3) {
            for (int d = 0; d < 3; ++d) sh[d] = wx * T1[f][d] + wy * T2[f][d];
          } else {
            for (int d = 0; d < 3; ++d) sh[d] += blend * (wx * T1[f][d] + wy * T2[f][d]);
          }
        }
        double y[3];
        for (int d = 0; d < 3; ++d) y[d] = X[d] + sh[d] - c0[d];
        double rst[3];
        for (int a = 0; a < 3; ++a) rst[a] = Ai[a][0] * y[0] + Ai[a][1] * y[1] + Ai[a][2] * y[2];
        r.push_back(rst[0]);
        s.push_back(rst[1]);
        t.push_back(rst[2]);
      }
}

// ---------------------------------------------------- orthonormal bases ---
void basis3d(int N, double r, double s, double t, double* v, double* vr, double* vs,
             double* vt) {
  const double a = (std::fabs(s + t) > 1e-12) ? 2 * (1 + r) / (-s - t) - 1 : -1.0;
  const double b = (std::fabs(1 - t) > 1e-12) ? 2 * (1 + s) / (1 - t) - 1 : -1.0;
  const double c = t;
  const double C = 2.0 * std::sqrt(2.0);
  auto pw = [](double x, int e) { return e >= 0 ? std::pow(x, e) : 0.0; };
  int n = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k, ++n) {
        const double f = jacobi(i, 0, 0, a), df = djacobi(i, 0, 0, a);
        const double g = jacobi(j, 2 * i + 1, 0, b), dg = djacobi(j, 2 * i + 1, 0, b);
        const double h = jacobi(k, 2 * i + 2 * j + 2, 0, c);
        const double dh = djacobi(k, 2 * i + 2 * j + 2, 0, c);
        const double ob = 1 - b, oc = 1 - c;
        v[n] = C * f * g * pw(ob, i) * h * pw(oc, i + j);
        // chain rule through the collapsed coordinates, singular factors cancelled
        vr[n] = 4 * C * df * g * pw(ob, i - 1) * h * pw(oc, i + j - 1);
        const double ta = 2 * C * (1 + a) * df * g * pw(ob, i - 1) * h * pw(oc, i + j - 1);
        const double gb = dg * pw(ob, i) - i * g * pw(ob, i - 1);
        const double hc = dh * pw(oc, i + j) - (i + j) * h * pw(oc, i + j - 1);
        vs[n] = ta + 2 * C * f * gb * h * pw(oc, i + j - 1);
        vt[n] = ta + C * f * gb * (1 + b) * h * pw(oc, i + j - 1) + C * f * g * pw(ob, i) * hc;
      }
}

void basis2d(int N, double p, double q, double* v) {
  const double a = (std::fabs(1 - q) > 1e-12) ? 2 * (1 + p) / (1 - q) - 1 : -1.0;
  const double b = q;
  int n = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j, ++n)
      v[n] = std::sqrt(2.0) * jacobi(i, 0, 0, a) * jacobi(j, 2 * i + 1, 0, b) *
             std::pow(1 - b, i);
}

// ------------------------------------------------------------- dense LA ---
// In-place inverse of the n x n row-major matrix A by Gauss-Jordan with
// partial pivoting.  Returns false if A is numerically singular.
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[i * n + c]) > std::fabs(A[p * n + c])) p = i;
    if (std::fabs(A[p * n + c]) < 1e-300) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) { std::swap(A[p * n + j], A[c * n + j]); std::swap(I[p * n + j], I[c * n + j]); }
    const double d = 1.0 / A[c * n + c];
    for (int j = 0; j < n; ++j) { A[c * n + j] *= d; I[c * n + j] *= d; }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = A[i * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[c * n + j]; I[i * n + j] -= f * I[c * n + j]; }
    }
  }
  A.swap(I);
  return true;
}

void matmul(const std::vector<double>& A, const std::vector<double>& B, std::vector<double>& C,
            int n, int k, int m) {  // C[n][m] = A[n][k] B[k][m]
  C.assign(static_cast<size_t>(n) * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[i * k + l];
      for (int j = 0; j < m; ++j) C[i * m + j] += a * B[l * m + j];
    }
}

}  // namespace

bool build_ref_ops(int N, RefOps& o, std::string& err) {
  if (N < 1 || N > kMaxOrder) { err = "order must be in 1..9"; return false; }
  o = RefOps();
  o.N = N;
  o.Np = np_of(N);
  o.Nfp = nfp_of(N);
  const int Np = o.Np, Nfp = o.Nfp;
  nodes3d(N, o.r, o.s, o.t);
  if (static_cast<int>(o.r.size()) != Np) { err = "node count mismatch"; return false; }

  // face node lists
  o.Fmask.assign(4 * Nfp, -1);
  for (int f = 0; f < 4; ++f) {
    int c = 0;
    for (int i = 0; i < Np; ++i) {
      const double v = f == 0 ? 1 + o.t[i] : f == 1 ? 1 + o.s[i]
                     : f == 2 ? 1 + o.r[i] + o.s[i] + o.t[i] : 1 + o.r[i];
      if (std::fabs(v) < 1e-10) {
        if (c >= Nfp) { err = "too many face nodes"; return false; }
        o.Fmask[f * Nfp + c++] = i;
      }
    }
    if (c != Nfp) { err = "face node count mismatch"; return false; }
  }

  // Vandermonde matrices
  std::vector<double> V(Np * Np), Vr(Np * Np), Vs(Np * Np), Vt(Np * Np);
  for (int i = 0; i < Np; ++i)
    basis3d(N, o.r[i], o.s[i], o.t[i], &V[i * Np], &Vr[i * Np], &Vs[i * Np], &Vt[i * Np]);
  std::vector<double> Vinv = V;
  if (!invert(Vinv, Np)) { err = "singular Vandermonde"; return false; }
  matmul(Vr, Vinv, o.Dr, Np, Np, Np);
  matmul(Vs, Vinv, o.Ds, Np, Np, Np);
  matmul(Vt, Vinv, o.Dt, Np, Np, Np);
  // M^-1 = V V^T
  std::vector<double> VT(Np * Np), Minv;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) VT[j * Np + i] = V[i * Np + j];
  matmul(V, VT, Minv, Np, Np, Np);
  o.M = Minv;
  if (!invert(o.M, Np)) { err = "singular mass matrix"; return false; }

  // face mass matrices and E = [M^A_1 .. M^A_4] embedded in volume rows
  const int NF = 4 * Nfp;
  std::vector<double> E(static_cast<size_t>(Np) * NF, 0.0);
  for (int f = 0; f < 4; ++f) {
    std::vector<double> V2(Nfp * Nfp), V2T(Nfp * Nfp), MA;
    for (int j = 0; j < Nfp; ++j) {
      const int i = o.Fmask[f * Nfp + j];
      double p, q;
      if (f == 0) { p = o.r[i]; q = o.s[i]; }
      else if (f == 1) { p = o.r[i]; q = o.t[i]; }
      else { p = o.s[i]; q = o.t[i]; }
      basis2d(N, p, q, &V2[j * Nfp]);
    }
    for (int i = 0; i < Nfp; ++i)
      for (int j = 0; j < Nfp; ++j) V2T[j * Nfp + i] = V2[i * Nfp + j];
    matmul(V2, V2T, MA, Nfp, Nfp, Nfp);
    if (!invert(MA, Nfp)) { err = "singular face mass"; return false; }
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b)
        E[static_cast<size_t>(o.Fmask[f * Nfp + a]) * NF + f * Nfp + b] = MA[a * Nfp + b];
  }
  matmul(Minv, E, o.LIFT, Np, Np, NF);

  // face-node permutations between neighbours (barycentric matching)
  o.perm.assign(4 * 4 * 6 * Nfp, -1);
  auto bary = [&](int i, int v) {
    switch (v) {
      case 0: return -(1 + o.r[i] + o.s[i] + o.t[i]) / 2;
      case 1: return (1 + o.r[i]) / 2;
      case 2: return (1 + o.s[i]) / 2;
      default: return (1 + o.t[i]) / 2;
    }
  };
  for (int f = 0; f < 4; ++f)
    for (int g = 0; g < 4; ++g)
      for (int sg = 0; sg < 6; ++sg)
        for (int j = 0; j < Nfp; ++j) {
          const int i = o.Fmask[f * Nfp + j];
          int found = -1;
          for (int jj = 0; jj < Nfp && found < 0; ++jj) {
            const int i2 = o.Fmask[g * Nfp + jj];
            double d = 0;
            for (int p = 0; p < 3; ++p)
              d = std::max(d, std::fabs(bary(i, kFaceVerts[f][p]) -
                                        bary(i2, kFaceVerts[g][kPerm3[sg][p]])));
            if (d < 1e-10) found = i2;
          }
          if (found < 0) { err = "face node permutation not found"; return false; }
          o.perm[((f * 4 + g) * 6 + sg) * Nfp + j] = found;
        }
  return true;
}

}  // namespace dg
