"""C-ABI library on the CPU: it loads, exports every declared symbol, and its
host-side setup (nodes, operators, geometry, connectivity, CFL step, error
codes) matches the oracle.  No device computation is called here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from workloads import kuhn_box_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def dg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as pkg
    return pkg


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "dg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(dg):
    lib = C.CDLL(dg.library_path())
    names = _declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_0901_1024_gb300._capi import SIGNATURES
    assert sorted(SIGNATURES) == names


@pytest.mark.parametrize("N", range(1, 10))
def test_operators_and_nodes_match_oracle(dg, N):
    verts, tets = kuhn_box_mesh(1, 0.1, 0)
    m = dg.Mesh(verts, tets, N)
    ref = oracle.ref_element(N)
    assert (m.Np, m.Nfp) == (ref.Np, ref.Nfp)
    ops = m.operators()
    tol = 1e-12 * N ** 2
    for name, want in (("Dr", ref.Dr), ("Ds", ref.Ds), ("Dt", ref.Dt), ("LIFT", ref.LIFT)):
        assert np.abs(ops[name] - want).max() < tol * max(1, np.abs(want).max()), name
    assert np.abs(ops["M"] - ref.M).max() < 1e-13 * N
    om = oracle.build_mesh(verts, tets, N)
    xyz = m.nodes()
    assert np.abs(xyz - np.stack([om.x, om.y, om.z])).max() < 1e-13


@pytest.mark.parametrize("n,N,jit,seed", [(2, 1, 0.1, 0), (2, 2, 0.15, 3), (3, 3, 0.1, 1), (2, 4, 0.15, 2),
                                          (1, 7, 0.1, 5), (1, 9, 0.0, 0)])
def test_connectivity_bit_exact(dg, n, N, jit, seed):
    verts, tets = kuhn_box_mesh(n, jit, seed)
    # shuffle the element order and the vertex order inside each tetrahedron
    rng = np.random.default_rng(seed)
    tets = tets[rng.permutation(len(tets))]
    tets = np.array([t[rng.permutation(4)] for t in tets], dtype=np.int32)
    m = dg.Mesh(verts, tets, N)
    om = oracle.build_mesh(verts, tets, N)
    vM, vP = m.connectivity()
    assert np.array_equal(vM, om.vmapM.astype(np.int32))
    assert np.array_equal(vP, om.vmapP.astype(np.int32))


def test_geometry_and_cfl_match_oracle(dg):
    verts, tets = kuhn_box_mesh(3, 0.15, 4)
    m = dg.Mesh(verts, tets, 4)
    om = oracle.build_mesh(verts, tets, 4)
    g = m.geometry()
    want = np.stack([om.rx, om.ry, om.rz, om.sx, om.sy, om.sz, om.tx, om.ty, om.tz])
    assert np.abs(g["metric"] - want).max() < 1e-11 * np.abs(want).max()
    assert np.allclose(g["J"], om.J, rtol=1e-13)
    assert np.abs(g["normals"] - np.stack([om.nx, om.ny, om.nz])).max() < 1e-13
    assert np.allclose(g["Fscale"], om.Fscale, rtol=1e-13)
    assert abs(m.dt_cfl - oracle.cfl_dt(om)) < 1e-15 * m.dt_cfl * 10


def test_error_codes(dg):
    from paper_0901_1024_gb300 import DGError
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [-1, -1, -1]], float)
    with pytest.raises(DGError) as ei:
        dg.Mesh(verts, np.array([[0, 1, 2, 7]]))
    assert ei.value.code == -2
    with pytest.raises(DGError) as ei:       # zero volume
        dg.Mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float), np.array([[0, 1, 2, 3]]))
    assert ei.value.code == -2
    with pytest.raises(DGError) as ei:       # face shared by three tets
        dg.Mesh(verts, np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]]))
    assert ei.value.code == -2
    m = dg.Mesh(verts[:5], np.array([[0, 1, 2, 3], [1, 2, 3, 4]]))
    with pytest.raises(DGError) as ei:
        m.set_order(10)
    assert ei.value.code == -3
    with pytest.raises(DGError) as ei:
        m.set_order(0)
    assert ei.value.code == -3
    lib = dg.load()
    assert lib.dg_info(m._h, None, None, None, None) == -7      # no order yet
    assert lib.dg_rhs(m._h, None, None, None) == -7
    m.set_order(2)
    assert lib.dg_rhs(m._h, None, None, None) == -1
    assert lib.dg_step(m._h, C.c_void_p(16), C.c_void_p(32), C.c_double(-1.0), 1, None) == -1
    assert lib.dg_step(m._h, C.c_void_p(16), C.c_void_p(16), C.c_double(1.0), 1, None) == -1
    assert lib.dg_set_flux(m._h, C.c_double(float("nan"))) == -1
    assert b"dt must be" in lib.dg_last_error() or b"alpha" in lib.dg_last_error()
    assert lib.dg_mesh_create(None, 0, None, 0, None) == -1
    assert lib.dg_check_wait_timeout(m._h, 0, None) == -1          # polls outside 1 .. 2^24
    assert lib.dg_check_wait_timeout(m._h, (1 << 24) + 1, None) == -1
    assert b"polls" in lib.dg_last_error()
    lib.dg_mesh_destroy(None)


def test_two_tet_connectivity_matches_hand_count(dg):
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], float)
    m = dg.Mesh(verts, np.array([[0, 1, 2, 3], [1, 2, 3, 4]]), 1)
    vM, vP = m.connectivity()
    vP = vP.reshape(2, 4, 3)
    assert list(vP[0, 2]) == [4, 5, 6] and list(vP[1, 0]) == [1, 2, 3]
    assert (vP.reshape(-1) != vM).sum() == 6


@pytest.mark.parametrize("n,block,seed", [(3, 20, 1), (4, 20, 2), (4, 7, 3), (2, 1, 4), (3, 1000, 5)])
def test_partition_order_matches_oracle(dg, n, block, seed):
    """dg_partition_order (C++) against the oracle's greedy partition: the same
    permutation, element for element, on randomly renumbered box meshes."""
    from oracle.partition import partition_order
    verts, tets = kuhn_box_mesh(n, 0.1, seed)
    tets = tets[np.random.Generator(np.random.PCG64(seed)).permutation(len(tets))]
    mesh = dg.Mesh(verts, tets, 1)
    got = mesh.partition_order(block)
    want = partition_order(oracle.build_mesh(verts, tets, 1).EToE, block)
    assert got.dtype == np.int64 and np.array_equal(got, want)


def test_partition_order_errors(dg):
    from paper_0901_1024_gb300._capi import load
    verts, tets = kuhn_box_mesh(1, 0.0, 0)
    mesh = dg.Mesh(verts, tets, 1)
    lib = load()
    perm = np.empty(mesh.K, np.int64)
    ptr = perm.ctypes.data_as(C.POINTER(C.c_int64))
    assert lib.dg_partition_order(mesh._h, 0, ptr) == -1
    assert lib.dg_partition_order(mesh._h, 20, None) == -1
    assert lib.dg_partition_order(None, 20, ptr) == -1
    assert lib.dg_partition_order(mesh._h, 4, ptr) == 0
    assert sorted(perm) == list(range(mesh.K))


def test_materials_and_boundary_host_side(dg):
    """dg_set_materials / dg_set_boundary: validation, dt_cfl with materials
    against the oracle, reset by NULL, and packing keeps each part's materials
    (its dt_cfl is the smallest part's)."""
    from paper_0901_1024_gb300 import DGError
    verts, tets = kuhn_box_mesh(2, 0.15, 8)
    m = dg.Mesh(verts, tets, 3)
    om = oracle.build_mesh(verts, tets, 3)
    vac = m.dt_cfl
    rng = np.random.default_rng(5)
    eps, mu = rng.uniform(0.5, 4.0, m.K), rng.uniform(0.5, 3.0, m.K)
    m.set_materials(eps, mu)
    want = oracle.maxwell.cfl_dt(om, 1.0, eps, mu)
    assert abs(m.dt_cfl - want) < 1e-14 * want
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        e2 = eps.copy()
        e2[3] = bad
        with pytest.raises(DGError) as ei:
            m.set_materials(e2, mu)
        assert ei.value.code == -1
    assert abs(m.dt_cfl - want) < 1e-14 * want       # a rejected call changes nothing
    m.set_materials(None, None)
    assert m.dt_cfl == vac
    m.set_materials(eps)                              # mu = 1
    assert abs(m.dt_cfl - oracle.maxwell.cfl_dt(om, 1.0, eps, np.ones(m.K))) < 1e-14 * m.dt_cfl
    kind = np.zeros((m.K, 4), np.int8)
    kind[0, 0] = 2
    with pytest.raises(DGError) as ei:
        m.set_boundary(kind)
    assert ei.value.code == -1
    with pytest.raises(ValueError):
        m.set_boundary(np.zeros((m.K, 3), np.int8))
    kind[0, 0] = 1
    m.set_boundary(kind)
    m.set_boundary(None)
    lib = dg.load()
    assert lib.dg_set_materials(None, None, None) == -1
    assert lib.dg_set_boundary(None, None) == -1
    b = dg.Mesh(verts, tets, 3)
    p = dg.Mesh.pack([m, b])
    assert p.dt_cfl == min(m.dt_cfl, b.dt_cfl)
