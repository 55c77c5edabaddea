"""Per-element geometry and face connectivity (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2 (Eq. dg-reference-matrices): every tetrahedron D_k is the image of
the reference element under an affine map Psi_k,
    x = 1/2 ( -(r+s+t+1) x1 + (1+r) x2 + (1+s) x3 + (1+t) x4 ),
so d x / d(r,s,t) = [x2-x1, x3-x1, x4-x1] / 2 is constant per element,
J_k = det of it, and the chain-rule coefficients d r_mu / d x_nu are the
entries of its inverse.  Elements with a negative determinant have their last
two vertices swapped before anything else is computed.

Face data are computed here directly from the physical face triangle (not
through the metric terms): the outward unit normal is the normalised cross
product of two face edges, oriented away from the opposite vertex, and the
surface Jacobian sJ = area / 2 (the face parameter triangle has area 2), so
Fscale = sJ / J.

Connectivity (the face index lists of Section 5.2): faces are matched by their
sorted global vertex triples; for every face node of element k the matching
node of the neighbour is the one at the same physical point (brute force over
the face's nodes).  Global node ids are k*Np + i, ordered over (k, face f,
face node j in ascending Fmask order).  Boundary faces (perfect conductor
walls) have vmapP = vmapM.
"""
from __future__ import annotations

import numpy as np

from .refelem import FACE_VERTS, ref_element

# vertex opposite each face
_OPPOSITE = (3, 2, 0, 1)


class MeshError(ValueError):
    pass


class Mesh:
    """Geometry + connectivity of a tetrahedral mesh at order N."""


def build_mesh(verts, tets, N: int) -> Mesh:
    verts = np.asarray(verts, dtype=np.float64)
    tets = np.array(tets, dtype=np.int64)
    if verts.ndim != 2 or verts.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4:
        raise MeshError("bad shapes")
    if tets.size and (tets.min() < 0 or tets.max() >= len(verts)):
        raise MeshError("vertex index out of range")
    ref = ref_element(N)
    K = len(tets)
    m = Mesh()
    m.N, m.K, m.Np, m.Nfp = N, K, ref.Np, ref.Nfp
    m.ref = ref

    # orientation: positive determinant, else swap the last two vertices
    X = verts[tets]                                   # (K, 4, 3)
    A = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2) / 2
    det = np.linalg.det(A)
    if np.any(np.abs(det) < 1e-14 * np.max(np.abs(X)) ** 3 + 1e-300):
        raise MeshError("degenerate tetrahedron")
    neg = det < 0
    tets[neg] = tets[neg][:, [0, 1, 3, 2]]
    X = verts[tets]
    A = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2) / 2
    m.tets = tets
    m.J = np.linalg.det(A)                              # (K,)
    assert np.all(m.J > 0)
    inv = np.linalg.inv(A)                              # rows: grad r, grad s, grad t
    m.rx, m.ry, m.rz = inv[:, 0, 0], inv[:, 0, 1], inv[:, 0, 2]
    m.sx, m.sy, m.sz = inv[:, 1, 0], inv[:, 1, 1], inv[:, 1, 2]
    m.tx, m.ty, m.tz = inv[:, 2, 0], inv[:, 2, 1], inv[:, 2, 2]

    # physical node coordinates, shape (K, Np)
    r, s, t = ref.r, ref.s, ref.t
    lam = np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2])  # (4, Np)
    xyz = np.einsum("vi,kvd->dki", lam, X)
    m.x, m.y, m.z = xyz[0], xyz[1], xyz[2]

    # face normals and scalings from the physical triangles
    nrm = np.empty((K, 4, 3))
    area = np.empty((K, 4))
    for f, (a, b, c) in enumerate(FACE_VERTS):
        cr = np.cross(X[:, b] - X[:, a], X[:, c] - X[:, a])
        ln = np.linalg.norm(cr, axis=1)
        n = cr / ln[:, None]
        out = np.einsum("kd,kd->k", n, X[:, a] - X[:, _OPPOSITE[f]])
        n[out < 0] *= -1
        nrm[:, f] = n
        area[:, f] = ln / 2
    m.nx, m.ny, m.nz = nrm[..., 0], nrm[..., 1], nrm[..., 2]   # (K, 4)
    m.sJ = area / 2
    m.Fscale = m.sJ / m.J[:, None]

    # connectivity
    Np, Nfp = ref.Np, ref.Nfp
    faces = {}
    for k in range(K):
        for f, fv in enumerate(FACE_VERTS):
            key = tuple(sorted(int(tets[k, v]) for v in fv))
            faces.setdefault(key, []).append((k, f))
    EToE = np.tile(np.arange(K)[:, None], (1, 4))
    EToF = np.tile(np.arange(4)[None, :], (K, 1))
    for key, lst in faces.items():
        if len(lst) > 2:
            raise MeshError("face shared by more than two tetrahedra")
        if len(lst) == 2:
            (k1, f1), (k2, f2) = lst
            EToE[k1, f1], EToF[k1, f1] = k2, f2
            EToE[k2, f2], EToF[k2, f2] = k1, f1
    m.EToE, m.EToF = EToE, EToF

    vmapM = np.empty((K, 4, Nfp), dtype=np.int64)
    vmapP = np.empty((K, 4, Nfp), dtype=np.int64)
    h = np.min(np.linalg.norm(X[:, 1] - X[:, 0], axis=1))
    tol = 1e-8 * h
    for k in range(K):
        for f in range(4):
            idM = ref.Fmask[f]
            vmapM[k, f] = k * Np + idM
            k2, f2 = EToE[k, f], EToF[k, f]
            if k2 == k and f2 == f:
                vmapP[k, f] = vmapM[k, f]
                continue
            idP = ref.Fmask[f2]
            pM = np.stack([m.x[k, idM], m.y[k, idM], m.z[k, idM]], axis=1)
            pP = np.stack([m.x[k2, idP], m.y[k2, idP], m.z[k2, idP]], axis=1)
            d = np.linalg.norm(pM[:, None, :] - pP[None, :, :], axis=2)
            j2 = np.argmin(d, axis=1)
            if np.any(d[np.arange(Nfp), j2] > tol):
                raise MeshError("non-conforming face (face nodes do not match)")
            vmapP[k, f] = k2 * Np + idP[j2]
    m.vmapM = vmapM.reshape(-1)
    m.vmapP = vmapP.reshape(-1)
    m.boundary = (EToE == np.arange(K)[:, None]) & (EToF == np.arange(4)[None, :])
    return m
