"""Pins for the oracle's geometry and connectivity (CPU only)."""
import numpy as np
import pytest

import oracle
from oracle.mesh import MeshError
from oracle.refelem import FACE_VERTS
from workloads import kuhn_box_mesh


@pytest.fixture(scope="module")
def mesh3():
    verts, tets = kuhn_box_mesh(3, 0.15, 0)
    return oracle.build_mesh(verts, tets, 3), verts


def test_kuhn_mesh_shape_and_domain():
    verts, tets = kuhn_box_mesh(4, 0.1, 0)
    assert verts.shape == (125, 3) and tets.shape == (384, 4)
    assert np.all(np.abs(verts) <= 1 + 1e-15)
    # boundary vertices stay on their planes
    corners = np.all(np.abs(np.abs(verts) - 1) < 1e-15, axis=1)
    assert corners.sum() == 8


def test_volumes_and_jacobians(mesh3):
    m, verts = mesh3
    X = verts[m.tets]
    vol = np.abs(np.einsum("kd,kd->k", X[:, 1] - X[:, 0],
                           np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6
    assert np.all(m.J > 0)
    assert np.allclose(m.J, vol / (4 / 3), rtol=1e-13)
    # the jittered tets still fill the cube [-1,1]^3 exactly
    assert abs(np.sum(m.J) * 4 / 3 - 8.0) < 1e-12


def test_metric_is_inverse_jacobian(mesh3):
    m, verts = mesh3
    X = verts[m.tets]
    xr = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2) / 2
    G = np.stack([np.stack([m.rx, m.ry, m.rz], 1), np.stack([m.sx, m.sy, m.sz], 1),
                  np.stack([m.tx, m.ty, m.tz], 1)], 1)
    assert np.allclose(np.einsum("kij,kjl->kil", G, xr), np.eye(3)[None], atol=1e-12)


def test_face_geometry(mesh3):
    m, verts = mesh3
    X = verts[m.tets]
    n = np.stack([m.nx, m.ny, m.nz], axis=2)
    assert np.allclose(np.linalg.norm(n, axis=2), 1)
    area = 2 * m.sJ
    # closed surface: sum_f area_f n_f = 0
    assert np.abs(np.einsum("kf,kfd->kd", area, n)).max() < 1e-13
    # outward: n points from the element centroid to the face centroid
    cen = X.mean(1)
    for f, fv in enumerate(FACE_VERTS):
        fc = X[:, list(fv)].mean(1)
        assert np.all(np.einsum("kd,kd->k", n[:, f], fc - cen) > 0)
    assert np.allclose(m.Fscale, m.sJ / m.J[:, None])
    # boundary faces lie on the cube walls: normals are +-axis vectors, total area 24
    bn = n[m.boundary]
    assert np.allclose(np.sort(np.abs(bn), axis=1), [0, 0, 1], atol=1e-12)
    assert abs(area[m.boundary].sum() - 24.0) < 1e-12
    assert m.boundary.sum() == 2 * 6 * 3 ** 2


@pytest.mark.parametrize("N", [1, 2, 4])
def test_connectivity_invariants(N):
    verts, tets = kuhn_box_mesh(2, 0.1, 1)
    m = oracle.build_mesh(verts, tets, N)
    K, Np, Nfp = m.K, m.Np, m.Nfp
    vM, vP = m.vmapM, m.vmapP
    assert vM.shape == (K * 4 * Nfp,)
    assert np.array_equal(vM.reshape(K, 4, Nfp)[:, :, 0] // Np, np.tile(np.arange(K)[:, None], (1, 4)))
    x, y, z = m.x.ravel(), m.y.ravel(), m.z.ravel()
    d = np.sqrt((x[vM] - x[vP]) ** 2 + (y[vM] - y[vP]) ** 2 + (z[vM] - z[vP]) ** 2)
    assert d.max() < 1e-12
    # vmapP is an involution on face nodes: following it twice returns home
    interior = ~np.repeat(m.boundary.ravel(), Nfp)
    for i in np.nonzero(interior)[0]:
        # the neighbour's node may sit on several faces; take the entry on the matched face
        k2 = vP[i] // Np
        f2 = m.EToF[vM[i] // Np, (i // Nfp) % 4]
        block = np.arange((k2 * 4 + f2) * Nfp, (k2 * 4 + f2 + 1) * Nfp)
        j = block[vM[block] == vP[i]][0]
        assert vP[j] == vM[i]
    # face count: interior faces pair up
    nb = m.boundary.sum()
    assert (4 * K - nb) % 2 == 0 and nb == 2 * 6 * 4


def test_two_tet_connectivity_by_hand():
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], float)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    m = oracle.build_mesh(verts, tets, 1)
    # the shared triangle (1,2,3) is face f2 of tet 0 and face f0 of tet 1
    assert m.EToE[0, 2] == 1 and m.EToF[0, 2] == 0
    assert m.EToE[1, 0] == 0 and m.EToF[1, 0] == 2
    assert m.boundary.sum() == 6
    # N=1 nodes are the vertices; tet-0 face f2 nodes 1,2,3 = global vertices 1,2,3
    # = tet-1 local vertices 0,1,2 = tet-1 nodes 0,1,2 (global ids 4,5,6)
    vP = m.vmapP.reshape(2, 4, 3)
    assert list(vP[0, 2]) == [4, 5, 6]
    assert list(vP[1, 0]) == [1, 2, 3]
    assert list(vP[0, 0]) == list(m.vmapM.reshape(2, 4, 3)[0, 0])


def test_orientation_fix_swaps_last_two_vertices():
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    m = oracle.build_mesh(verts, np.array([[0, 1, 3, 2]]), 2)
    assert list(m.tets[0]) == [0, 1, 2, 3]
    assert m.J[0] > 0


def test_bad_meshes_raise():
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [-1, -1, -1]], float)
    with pytest.raises(MeshError):
        oracle.build_mesh(verts, np.array([[0, 1, 2, 7]]), 1)
    with pytest.raises(MeshError):  # flat tet
        oracle.build_mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float),
                          np.array([[0, 1, 2, 3]]), 1)
    with pytest.raises(MeshError):  # face (0,1,2) shared by three tets
        oracle.build_mesh(verts, np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]]), 1)
