"""Seeded synthetic inputs for the DG Maxwell hot path.

This module is shared by the tests, the benchmark and the oracle's callers.  It
holds no part of the discretisation itself: it builds tetrahedral meshes of the
cube [-1,1]^3 (vertex coordinates + connectivity) and evaluates closed-form
initial fields at caller-supplied points.  Every random number comes from a
numpy PCG64 generator with an explicit seed.

The paper's own meshes (TetGen cavity meshes, an aircraft surface mesh) are not
available; these meshes stand in for them with the same element counts and
orders (Section 6 of the paper: cavity eigenmode accuracy test, N=1..9, K from
a few hundred to ~80 000 tetrahedra).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "kuhn_box_mesh",
    "cavity_mode",
    "cavity_omega",
    "gaussian_pulse",
    "pulse_center",
    "random_fields",
    "WORKLOADS",
]


def kuhn_box_mesh(n: int, jitter: float = 0.0, seed: int = 0):
    """Cube [-1,1]^3 cut into n^3 hexahedra, each split into 6 Kuhn tetrahedra.

    Hex (i,j,k) with corner v0 = (i,j,k)*h - 1, h = 2/n, is split along its main
    diagonal into the 6 tetrahedra (v0, v0+e_a, v0+e_a+e_b, v0+(1,1,1)) over the
    6 permutations (a,b,c) of the axes, in itertools order.  The split is
    face-conforming across hexes.  Hexes are numbered i fastest, then j, then k;
    the 6 tetrahedra of a hex are consecutive.  Vertex (i,j,k) has index
    i + (n+1)*(j + (n+1)*k).

    Jitter: every vertex coordinate that does not lie on a boundary plane of the
    cube is moved by U[-jitter*h, +jitter*h] (PCG64(seed)), so the domain stays
    exactly [-1,1]^3.  For jitter <= 0.15 no tetrahedron can invert (the
    smallest Kuhn height is h/sqrt(2) > 2*sqrt(3)*0.15*h).

    Returns (verts float64 [nv,3], tets int32 [6 n^3, 4]).  Tetrahedra are
    returned with the vertex order above; about half of them are negatively
    oriented, which the solver must handle.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 2.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h - 1.0
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    if jitter:
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-jitter * h, jitter * h, size=verts.shape)
        on_bnd = (np.abs(np.abs(verts) - 1.0) < 1e-12)
        d[on_bnd] = 0.0
        verts = verts + d

    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    unit = np.eye(3, dtype=np.int64)
    perms = list(itertools.permutations(range(3)))
    tets = np.empty((6 * n ** 3, 4), dtype=np.int64)
    c = 0
    for k in range(n):
        for j in range(n):
            for i in range(n):
                v0 = np.array([i, j, k])
                for (a, b, _) in perms:
                    p1 = v0 + unit[a]
                    p2 = p1 + unit[b]
                    p3 = v0 + 1
                    tets[c] = [vid(*v0), vid(*p1), vid(*p2), vid(*p3)]
                    c += 1
    return verts, tets.astype(np.int32)


# PEC cavity [-1,1]^3, mode (1,1,1): k = pi/2 on every axis.
_KWAVE = math.pi / 2.0
_AMP = np.array([1.0, 1.0, -2.0])  # A . k = 0  (divergence free)


def cavity_omega() -> float:
    """Angular frequency of the (1,1,1) mode of the cavity [-1,1]^3 (eps = mu = 1)."""
    return _KWAVE * math.sqrt(3.0)


def cavity_mode(x, y, z, t: float = 0.0):
    """Exact (1,1,1) eigenmode of the perfectly conducting cube [-1,1]^3.

    With S_a = sin(k(a+1)), C_a = cos(k(a+1)), k = pi/2, A = (1,1,-2):
      E(t) = (A_x C_x S_y S_z, A_y S_x C_y S_z, A_z S_x S_y C_z) cos(w t)
      H(t) = -(curl E_hat / w) sin(w t),  w = k sqrt(3)
    Tangential E vanishes on every wall; div E = 0; it solves
    dE/dt = curl H, dH/dt = -curl E.  Returns a (6, *x.shape) array
    (Ex, Ey, Ez, Hx, Hy, Hz).
    """
    k = _KWAVE
    w = cavity_omega()
    Sx, Sy, Sz = np.sin(k * (x + 1)), np.sin(k * (y + 1)), np.sin(k * (z + 1))
    Cx, Cy, Cz = np.cos(k * (x + 1)), np.cos(k * (y + 1)), np.cos(k * (z + 1))
    Ax, Ay, Az = _AMP
    ct, st = math.cos(w * t), math.sin(w * t)
    Ex = Ax * Cx * Sy * Sz * ct
    Ey = Ay * Sx * Cy * Sz * ct
    Ez = Az * Sx * Sy * Cz * ct
    cx = k * (Az - Ay) * Sx * Cy * Cz
    cy = k * (Ax - Az) * Cx * Sy * Cz
    cz = k * (Ay - Ax) * Cx * Cy * Sz
    Hx, Hy, Hz = -cx * st / w, -cy * st / w, -cz * st / w
    return np.stack([Ex, Ey, Ez, Hx, Hy, Hz])


def pulse_center(seed: int = 1):
    """Pulse centre ~ U[-0.5, 0.5]^3 from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-0.5, 0.5, size=3)


def gaussian_pulse(x, y, z, width: float = 0.2, center=(0.0, 0.0, 0.0)):
    """E_z = exp(-|x - c|^2 / width^2), all other fields zero; shape (6, *x.shape)."""
    cx, cy, cz = center
    r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
    out = np.zeros((6,) + np.shape(x))
    out[2] = np.exp(-r2 / width ** 2)
    return out


def random_fields(K: int, Np: int, seed: int = 0):
    """Independent N(0,1) nodal values, shape (6, K, Np), float64, PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((6, K, Np))


# Named workloads (sizes follow the paper's Maxwell experiments, Section 6).
WORKLOADS = {
    # FP64 golden run: N=3 on 4^3 hexes x 6 = 384 tets, jitter 0.1h, cavity mode, 10 steps.
    "cavity_n4_N3": dict(n=4, N=3, jitter=0.10, seed=0, init="cavity", steps=10),
    # Throughput run: N=4 on 24^3 hexes x 6 = 82 944 tets, jitter 0.15h, Gaussian E_z pulse, 100 steps.
    "pulse_n24_N4": dict(n=24, N=4, jitter=0.15, seed=0, init="pulse", width=0.2, pulse_seed=1, steps=100),
    # Higher order: N=6 on 16^3 x 6 = 24 576 tets, cavity mode, 200 steps.
    "cavity_n16_N6": dict(n=16, N=6, jitter=0.10, seed=0, init="cavity", steps=200),
    # Highest order of the served stream: N=7 on 16^3 x 6 = 24 576 tets, Gaussian pulse.
    "pulse_n16_N7": dict(n=16, N=7, jitter=0.15, seed=0, init="pulse", width=0.2, pulse_seed=1,
                         steps=20),
}
