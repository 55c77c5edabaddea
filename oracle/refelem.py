"""Reference tetrahedron: nodes, Lagrange-basis matrices (oracle, FP64).

Test infrastructure only (see the package docstring).

Reference element I = {(r,s,t): r,s,t >= -1, r+s+t <= -1} with vertices
v1=(-1,-1,-1), v2=(1,-1,-1), v3=(-1,1,-1), v4=(-1,-1,1) and faces, in this
fixed order,
  f0: t = -1        (v1 v2 v3)
  f1: s = -1        (v1 v2 v4)
  f2: r + s + t = -1 (v2 v3 v4)
  f3: r = -1        (v1 v3 v4)

The matrices follow their integral definitions (Section 2, Eq.
dg-global-matrices, written on the reference element as in Eq.
dg-reference-matrices):
  M_ij   = int_I l_i l_j
  S^r_ij = int_I l_i d_r l_j,     D^r = M^-1 S^r    (likewise s, t)
  M^A_ij = int_A l_i l_j dA        (A a face, measured in the face's own
                                    2-D parameter triangle of area 2)
  LIFT   = M^-1 [M^A1 ... M^A4]    (Fig. lifting-matrix)
computed by exact Gauss quadrature on collapsed coordinates.  The nodal
(Lagrange) basis l_i at the interpolation nodes is represented through an
orthonormal basis of P_N (the total-degree polynomials), l = (basis) @ V^-1;
the matrices do not depend on that choice, only their conditioning does.

Nodes: Warburton's explicit Warp & Blend construction (the node set the paper
uses, ref. "warburton_explicit_2006" in Section 2) with its optimised blend
parameter alpha per order.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from numpy.polynomial import legendre as npleg
import scipy.special as sps

# Vertex indices of each face (0-based local vertex numbers), in face order.
FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))

# Warp & Blend blend parameter alpha for the tetrahedron, orders 1..15
# (Warburton 2006, optimised for the Lebesgue constant).
WB_ALPHA = (0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603,
            1.10153, 0.6080, 0.4523, 0.8856, 0.8717, 0.9655)


def dof_counts(N: int):
    """(Np, Nfp, Nf*Nfp) for order N on tetrahedra (Fig. dof-counts)."""
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    return Np, Nfp, 4 * Nfp


# ----------------------------------------------------------------------------
# 1-D building blocks
# ----------------------------------------------------------------------------
def lgl_points(n: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre points on [-1,1]: +-1 and the roots of P_n'."""
    if n < 1:
        raise ValueError("n >= 1")
    if n == 1:
        return np.array([-1.0, 1.0])
    inner = npleg.Legendre.basis(n).deriv().roots().real
    return np.concatenate([[-1.0], np.sort(inner), [1.0]])


def _warp_1d(N: int, x: np.ndarray) -> np.ndarray:
    """Warp function of the Warp & Blend construction.

    The displacement from N+1 equidistant points to the N+1 LGL points,
    interpolated by the equidistant Lagrange polynomial and divided by the
    edge blend (1 - x^2); set to zero at the end points x = +-1.
    """
    xeq = np.linspace(-1.0, 1.0, N + 1)
    disp = lgl_points(N) - xeq
    x = np.asarray(x, dtype=np.float64)
    w = np.zeros_like(x)
    for i in range(N + 1):
        li = np.ones_like(x)
        for j in range(N + 1):
            if j != i:
                li = li * (x - xeq[j]) / (xeq[i] - xeq[j])
        w = w + disp[i] * li
    inside = np.abs(x) < 1.0 - 1e-10
    out = np.zeros_like(x)
    out[inside] = w[inside] / (1.0 - x[inside] ** 2)
    return out


def _face_shift(N, alpha, L1, L2, L3):
    """In-plane Warp & Blend displacement on an equilateral triangle.

    L1, L2, L3 are barycentric coordinates of the triangle whose vertices sit
    at (0, 2/sqrt3), (-1, -1/sqrt3), (1, -1/sqrt3) respectively.  Each edge
    contributes its blended 1-D warp along the edge direction.
    """
    w1 = 4.0 * L2 * L3 * _warp_1d(N, L3 - L2) * (1.0 + (alpha * L1) ** 2)
    w2 = 4.0 * L1 * L3 * _warp_1d(N, L1 - L3) * (1.0 + (alpha * L2) ** 2)
    w3 = 4.0 * L1 * L2 * _warp_1d(N, L2 - L1) * (1.0 + (alpha * L3) ** 2)
    c2, s2 = math.cos(2 * math.pi / 3), math.sin(2 * math.pi / 3)
    c4, s4 = math.cos(4 * math.pi / 3), math.sin(4 * math.pi / 3)
    dx = w1 + c2 * w2 + c4 * w3
    dy = s2 * w2 + s4 * w3
    return dx, dy


def equispaced_nodes(N: int):
    """Equispaced nodes on I, t index outermost, then s, r fastest."""
    r, s, t = [], [], []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - k - j):
                r.append(-1.0 + 2.0 * i / N)
                s.append(-1.0 + 2.0 * j / N)
                t.append(-1.0 + 2.0 * k / N)
    return np.array(r), np.array(s), np.array(t)


def warp_blend_nodes(N: int):
    """Warp & Blend interpolation nodes on I (same order as equispaced_nodes).

    The equispaced nodes are placed on an equilateral tetrahedron; each face
    adds its in-plane warp (edges move to LGL points, face interiors follow
    the blended 2-D warp), scaled into the interior by the face blend
    (1 + (alpha La)^2) Lb Lc Ld / ((Lb + La/2)(Lc + La/2)(Ld + La/2)), with
    La the barycentric coordinate of the vertex opposite the face.  Nodes on
    the edges take the pure face warp.  The result is mapped back to I.
    """
    if N == 0:
        return np.array([-0.5]), np.array([-0.5]), np.array([-0.5])
    alpha = WB_ALPHA[N - 1] if N <= 15 else 1.0
    r, s, t = equispaced_nodes(N)
    # barycentric coordinates
    L1 = (1.0 + t) / 2
    L2 = (1.0 + s) / 2
    L3 = -(1.0 + r + s + t) / 2
    L4 = (1.0 + r) / 2
    q3 = math.sqrt(3.0)
    q6 = math.sqrt(6.0)
    v1 = np.array([-1.0, -1.0 / q3, -1.0 / q6])
    v2 = np.array([1.0, -1.0 / q3, -1.0 / q6])
    v3 = np.array([0.0, 2.0 / q3, -1.0 / q6])
    v4 = np.array([0.0, 0.0, 3.0 / q6])
    # face tangent frames (t1 along the edge Lc->Ld, t2 towards Lb)
    t1 = np.array([v2 - v1, v2 - v1, v3 - v2, v3 - v1])
    t2 = np.array([v3 - 0.5 * (v1 + v2), v4 - 0.5 * (v1 + v2),
                   v4 - 0.5 * (v2 + v3), v4 - 0.5 * (v1 + v3)])
    t1 = t1 / np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = t2 / np.linalg.norm(t2, axis=1, keepdims=True)
    X = (np.outer(L3, v1) + np.outer(L4, v2) + np.outer(L2, v3) + np.outer(L1, v4))
    shift = np.zeros_like(X)
    tol = 1e-10
    faces = ((L1, L2, L3, L4), (L2, L1, L3, L4), (L3, L1, L4, L2), (L4, L1, L3, L2))
    for f, (La, Lb, Lc, Ld) in enumerate(faces):
        wx, wy = _face_shift(N, alpha, Lb, Lc, Ld)
        blend = Lb * Lc * Ld
        denom = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La)
        ok = denom > tol
        blend = np.where(ok, (1.0 + (alpha * La) ** 2) * blend / np.where(ok, denom, 1.0), blend)
        shift += np.outer(blend * wx, t1[f]) + np.outer(blend * wy, t2[f])
        on_edge = (La < tol) & (((Lb > tol).astype(int) + (Lc > tol) + (Ld > tol)) < 3)
        shift[on_edge] = np.outer(wx[on_edge], t1[f]) + np.outer(wy[on_edge], t2[f])
    X = X + shift
    # equilateral -> reference: X = v1 + A [(r+1)/2... ] solved linearly
    A = np.column_stack([0.5 * (v2 - v1), 0.5 * (v3 - v1), 0.5 * (v4 - v1)])
    rhs = X.T - 0.5 * (v2 + v3 + v4 - v1)[:, None]
    rst = np.linalg.solve(A, rhs)
    return rst[0], rst[1], rst[2]


# ----------------------------------------------------------------------------
# basis and quadrature
# ----------------------------------------------------------------------------
def basis_indices(N: int):
    """Index triples (i, j, k), i+j+k <= N, of the orthonormal basis."""
    return [(i, j, k) for i in range(N + 1) for j in range(N + 1 - i)
            for k in range(N + 1 - i - j)]


def _jacobi(n, al, be, x):
    """Orthonormal Jacobi polynomial on [-1,1] with weight (1-x)^al (1+x)^be."""
    h = (2.0 ** (al + be + 1) / (2 * n + al + be + 1) * math.gamma(n + al + 1)
         * math.gamma(n + be + 1) / (math.gamma(n + al + be + 1) * math.factorial(n)))
    return sps.eval_jacobi(n, al, be, x) / math.sqrt(h)


def _djacobi(n, al, be, x):
    """Derivative of _jacobi(n, al, be, .)."""
    if n == 0:
        return np.zeros_like(x)
    h = (2.0 ** (al + be + 1) / (2 * n + al + be + 1) * math.gamma(n + al + 1)
         * math.gamma(n + be + 1) / (math.gamma(n + al + be + 1) * math.factorial(n)))
    return 0.5 * (n + al + be + 1) * sps.eval_jacobi(n - 1, al + 1, be + 1, x) / math.sqrt(h)


def collapsed_coordinates(r, s, t):
    """(a, b, c) with r = (1+a)(1-b)(1-c)/4 - 1, s = (1+b)(1-c)/2 - 1, c = t.

    On the singular edge/vertex the undetermined coordinate is set to -1.
    """
    a = np.where(np.abs(s + t) > 1e-12, 2 * (1 + r) / np.where(np.abs(s + t) > 1e-12, -s - t, 1.0) - 1, -1.0)
    b = np.where(np.abs(1 - t) > 1e-12, 2 * (1 + s) / np.where(np.abs(1 - t) > 1e-12, 1 - t, 1.0) - 1, -1.0)
    return a, b, np.asarray(t, dtype=np.float64)


def _pw(x, e):
    return x ** e if e >= 0 else np.zeros_like(x)


def orthonormal_vandermonde(N, r, s, t):
    """Orthonormal (Koornwinder-Dubiner) basis on I and its r, s, t derivatives.

    psi_ijk = 2 sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i P_k^(2i+2j+2,0)(c) (1-c)^(i+j)
    in collapsed coordinates; int_I psi_ijk psi_lmn = delta.  The gradient is
    the chain rule through (a, b, c) with the (1-b), (1-c) factors cancelled
    analytically, so it is finite on the collapsed edge and vertex.
    """
    a, b, c = collapsed_coordinates(np.asarray(r, float), np.asarray(s, float), np.asarray(t, float))
    C = 2.0 * math.sqrt(2.0)
    idx = basis_indices(N)
    V = np.empty((len(a), len(idx)))
    Vr, Vs, Vt = np.empty_like(V), np.empty_like(V), np.empty_like(V)
    for n, (i, j, k) in enumerate(idx):
        f, df = _jacobi(i, 0, 0, a), _djacobi(i, 0, 0, a)
        g, dg = _jacobi(j, 2 * i + 1, 0, b), _djacobi(j, 2 * i + 1, 0, b)
        h, dh = _jacobi(k, 2 * i + 2 * j + 2, 0, c), _djacobi(k, 2 * i + 2 * j + 2, 0, c)
        ob, oc = 1 - b, 1 - c
        V[:, n] = C * f * g * ob ** i * h * oc ** (i + j)
        # d psi / dr = psi_a * 4 / ((1-b)(1-c))
        Vr[:, n] = 4 * C * df * g * _pw(ob, i - 1) * h * _pw(oc, i + j - 1)
        # shared pieces
        ta = 2 * C * (1 + a) * df * g * _pw(ob, i - 1) * h * _pw(oc, i + j - 1)
        gb = dg * ob ** i - i * g * _pw(ob, i - 1)       # d/db [g (1-b)^i]
        # d psi / ds = psi_a 2(1+a)/((1-b)(1-c)) + psi_b 2/(1-c)
        Vs[:, n] = ta + 2 * C * f * gb * h * _pw(oc, i + j - 1)
        # d psi / dt = psi_a 2(1+a)/((1-b)(1-c)) + psi_b (1+b)/(1-c) + psi_c
        hc = dh * oc ** (i + j) - (i + j) * h * _pw(oc, i + j - 1)   # d/dc [h (1-c)^(i+j)]
        Vt[:, n] = ta + C * f * gb * (1 + b) * h * _pw(oc, i + j - 1) + C * f * g * ob ** i * hc
    return V, Vr, Vs, Vt


def tet_quadrature(n: int):
    """Collapsed (Duffy) Gauss-Legendre rule on I, exact for degree 2n-3.

    Unit simplex x = u, y = (1-u) v, z = (1-u)(1-v) w, Jacobian (1-u)^2 (1-v),
    then (r,s,t) = 2(x,y,z) - 1 (Jacobian 8).  Weights sum to vol(I) = 4/3.
    """
    g, w = npleg.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    U, Vv, Ww = np.meshgrid(g, g, g, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    x = U
    y = (1 - U) * Vv
    z = (1 - U) * (1 - Vv) * Ww
    wt = WU * WV * WW * (1 - U) ** 2 * (1 - Vv) * 8.0
    return (2 * x.ravel() - 1, 2 * y.ravel() - 1, 2 * z.ravel() - 1, wt.ravel())


def tri_quadrature(n: int):
    """Collapsed Gauss-Legendre rule on {p,q >= -1, p+q <= 0} (area 2)."""
    g, w = npleg.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    U, Vv = np.meshgrid(g, g, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    x = U
    y = (1 - U) * Vv
    wt = WU * WV * (1 - U) * 4.0
    return 2 * x.ravel() - 1, 2 * y.ravel() - 1, wt.ravel()


def face_points(f: int, p: np.ndarray, q: np.ndarray):
    """Points of face f of I given by the face's 2-D parameters (p, q)."""
    m1 = -np.ones_like(p)
    if f == 0:
        return p, q, m1
    if f == 1:
        return p, m1, q
    if f == 2:
        return p, q, -1.0 - p - q
    return m1, p, q


# ----------------------------------------------------------------------------
# reference element
# ----------------------------------------------------------------------------
class RefElement:
    """All reference-element data for order N (FP64).

    Attributes: N, Np, Nfp, r, s, t (nodes), Fmask (4, Nfp) node indices of
    each face in ascending order, V (orthonormal-basis Vandermonde), Dr, Ds, Dt, M,
    Minv, face_mass (4, Nfp, Nfp), LIFT (Np, 4 Nfp).
    """

    def __init__(self, N: int):
        if not (1 <= N <= 15):
            raise ValueError("order N must be in 1..15")
        self.N = N
        self.Np, self.Nfp, _ = dof_counts(N)
        self.r, self.s, self.t = warp_blend_nodes(N)
        r, s, t = self.r, self.s, self.t
        assert len(r) == self.Np
        tol = 1e-10
        on_face = (np.abs(1 + t) < tol, np.abs(1 + s) < tol,
                   np.abs(1 + r + s + t) < tol, np.abs(1 + r) < tol)
        self.Fmask = np.array([np.nonzero(m)[0] for m in on_face])
        assert self.Fmask.shape == (4, self.Nfp)

        V, Vr, Vs, Vt = orthonormal_vandermonde(N, r, s, t)
        self.V = V
        Vinv = np.linalg.inv(V)
        # D^mu = (derivative of basis at nodes) V^-1: the exact derivative of
        # the degree-N interpolant, which equals M^-1 S^mu.
        self.Dr = Vr @ Vinv
        self.Ds = Vs @ Vinv
        self.Dt = Vt @ Vinv

        # mass matrix: exact quadrature of the Lagrange products
        qr, qs, qt, qw = tet_quadrature(N + 2)
        Lq = orthonormal_vandermonde(N, qr, qs, qt)[0] @ Vinv  # l_j(x_q)
        self.M = Lq.T @ (qw[:, None] * Lq)
        self.Minv = np.linalg.inv(self.M)
        # stiffness matrices from their definition, kept for the identity
        # checks D = M^-1 S
        Lr = orthonormal_vandermonde(N, qr, qs, qt)
        self.S = tuple(Lq.T @ (qw[:, None] * (Lx @ Vinv)) for Lx in Lr[1:])

        # face mass matrices: the volume Lagrange functions restricted to a
        # face are the face Lagrange functions of the face nodes
        pp, pq, pw = tri_quadrature(N + 1)
        self.face_mass = np.empty((4, self.Nfp, self.Nfp))
        E = np.zeros((self.Np, 4 * self.Nfp))
        for f in range(4):
            fr, fs, ft = face_points(f, pp, pq)
            Lf = orthonormal_vandermonde(N, fr, fs, ft)[0] @ Vinv
            Mf_full = Lf.T @ (pw[:, None] * Lf)           # Np x Np
            fm = self.Fmask[f]
            self.face_mass[f] = Mf_full[np.ix_(fm, fm)]
            E[:, f * self.Nfp:(f + 1) * self.Nfp] = Mf_full[:, fm]
        self.E = E
        self.LIFT = self.Minv @ E


@functools.lru_cache(maxsize=None)
def ref_element(N: int) -> RefElement:
    return RefElement(N)
