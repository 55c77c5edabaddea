"""GPU parity with materials (per-element eps, mu) and absorbing boundaries:
the CUDA path through the C ABI against the FP64 oracle.  Tolerances as for
the vacuum operator: 1e-5 (one RHS), 1e-4 (steps), 1e-6 (energy)."""
import numpy as np
import pytest

import oracle
from workloads import kuhn_box_mesh, random_fields

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-5
STEP_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as dg
    return torch, dg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _materials(K, seed):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.5, 4.0, K)
    mu = rng.uniform(0.5, 3.0, K)
    bc = rng.integers(0, 2, (K, 4)).astype(np.int8)
    return eps, mu, bc


def _setup(dg, verts, tets, N, seed, with_eps=True, with_bc=True):
    mesh, om = dg.Mesh(verts, tets, N), oracle.build_mesh(verts, tets, N)
    eps, mu, bc = _materials(om.K, seed)
    if not with_eps:
        eps = mu = None
    if not with_bc:
        bc = None
    mesh.set_materials(eps, mu)
    mesh.set_boundary(bc)
    return mesh, om, eps, mu, bc


def _kinds(mesh):
    _, kinds = mesh.trace_read()
    return set(int(k) for k in kinds)


FP32, TC = 1, 2


@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("impl", [FP32, TC])
@pytest.mark.parametrize("what", ["materials_and_absorbing", "absorbing_only"])
def test_rhs_parity_materials(env, N, impl, what):
    """Random eps, mu per element and a random mix of perfect-conductor and
    absorbing boundary faces on both stage implementations (the tensor-core
    request runs the tensor cores up to N = 6 and the FP32 kernel above);
    K = 162 (156 for the order <= 4 tensor cores, whose bulk copies need
    K Np % 4 == 0): ragged last tiles of 20 and of 8 elements."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.15, 60 + N)
    if impl == TC and N <= 4:
        tets = tets[:156]
    mesh, om, eps, mu, bc = _setup(dg, verts, tets, N, N, with_eps=what != "absorbing_only")
    u32 = random_fields(om.K, om.Np, 70 + N).astype(np.float32)
    u32[:, ::5] *= 1e-4                                 # rows of different scales
    mesh.set_stage_impl(impl)
    mesh.trace_enable(4)
    u = torch.from_numpy(u32).cuda()
    out = torch.full_like(u, float("nan"))
    mesh.rhs(u, out)
    torch.cuda.synchronize()
    tc_ran = impl == TC and N <= 7 and (om.K * om.Np) % 4 == 0
    assert _kinds(mesh) == ({5} if tc_ran else {1})
    want = oracle.rhs(om, u32.astype(np.float64), 1.0, eps, mu, bc)
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel(got, want) < RHS_TOL


@pytest.mark.parametrize("N", [1, 4, 7])
def test_rhs_parity_materials_fp32_tile_shape_1(env, N):
    """The FP32 stage in tile shape 1 (half the tetrahedra per tile) with random
    eps, mu and absorbing faces: K = 162, ragged last tiles."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.15, 80 + N)
    mesh, om, eps, mu, bc = _setup(dg, verts, tets, N, 90 + N)
    u32 = random_fields(om.K, om.Np, 95 + N).astype(np.float32)
    mesh.set_stage_impl(FP32)
    mesh.set_stage_shape(1)
    u = torch.from_numpy(u32).cuda()
    out = torch.full_like(u, float("nan"))
    mesh.rhs(u, out)
    torch.cuda.synchronize()
    mesh.set_stage_shape(0)
    want = oracle.rhs(om, u32.astype(np.float64), 1.0, eps, mu, bc)
    assert rel(out.cpu().numpy(), want) < RHS_TOL


@pytest.mark.parametrize("alpha", [1.0, 0.0])
@pytest.mark.parametrize("impl,N", [(FP32, 3), (TC, 3), (TC, 6)])
def test_step_parity_materials(env, alpha, impl, N):
    """20 LSERK4 steps with materials and absorbing faces, upwind and central."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(2, 0.1, 3)
    mesh, om, eps, mu, bc = _setup(dg, verts, tets, N, 11)
    mesh.set_flux(alpha)
    mesh.set_stage_impl(impl)
    u0 = random_fields(om.K, om.Np, 12).astype(np.float32)
    dt = mesh.dt_cfl
    assert dt == pytest.approx(oracle.maxwell.cfl_dt(om, 1.0, eps, mu), rel=1e-14)
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.trace_enable(200)
    mesh.step(u, res, dt, 20)
    torch.cuda.synchronize()
    assert _kinds(mesh) == ({4} if impl == TC else {0})
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), dt, 20, alpha=alpha, eps=eps, mu=mu, bc=bc)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL


def test_tensor_cores_agree_with_fp32_on_a_large_material_mesh(env):
    """N = 4, K = 10 368 (several tiles per CTA): the tensor-core and FP32
    stages agree on a mesh with materials and absorbing faces."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(12, 0.15, 9)
    mesh = dg.Mesh(verts, tets, 4)
    eps, mu, bc = _materials(mesh.K, 41)
    mesh.set_materials(eps, mu)
    mesh.set_boundary(bc)
    u0 = random_fields(mesh.K, mesh.Np, 42).astype(np.float32)
    out = []
    for impl in (TC, FP32):
        mesh.set_stage_impl(impl)
        u = torch.from_numpy(u0).cuda()
        res = torch.zeros_like(u)
        mesh.step(u, res, mesh.dt_cfl, 2)
        out.append(u.cpu().numpy())
    assert np.isfinite(out[0]).all()
    assert rel(out[0], out[1].astype(np.float64)) < RHS_TOL


@pytest.mark.parametrize("N", [2, 5, 6, 7, 9])
def test_energy_parity_materials(env, N):
    """Energy weighted by eps (E) and mu (H): the row-staged kernel (N = 2, 5),
    the shared-memory triangle kernel (N = 6, 7, 9) and the allocation-free
    entry point."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.15, 2)
    mesh, om, eps, mu, _ = _setup(dg, verts, tets, N, 21, with_bc=False)
    u32 = random_fields(om.K, om.Np, 22).astype(np.float32)
    u = torch.from_numpy(u32).cuda()
    want = oracle.energy(om, u32.astype(np.float64), eps, mu)
    assert abs(mesh.energy(u) - want) < 1e-6 * want
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    mesh.energy_noalloc(u, out)
    torch.cuda.synchronize()
    assert abs(float(out.item()) - want) < 1e-6 * want


def test_packed_mesh_with_materials_matches_its_parts(env):
    """dg_mesh_pack of a mesh with materials and absorbing faces and a mesh
    given eps = mu = 1 explicitly (the pack fills 1 for parts without
    materials): a packed stage is bit for bit each part's own stage."""
    torch, dg = env
    va, ta = kuhn_box_mesh(2, 0.1, 1)
    vb, tb = kuhn_box_mesh(2, 0.15, 2)
    a, _, _, _, _ = _setup(dg, va, ta, 3, 31)
    b = dg.Mesh(vb, tb, 3)
    b.set_materials(np.ones(b.K), np.ones(b.K))
    p = dg.Mesh.pack([a, b])
    u0 = random_fields(p.K, p.Np, 32).astype(np.float32)
    dt = min(a.dt_cfl, b.dt_cfl)
    outs = []
    for m, sl in ((a, slice(0, a.K)), (b, slice(a.K, p.K))):
        u = torch.from_numpy(np.ascontiguousarray(u0[:, sl])).cuda()
        w, r = torch.empty_like(u), torch.zeros_like(u)
        m.rk_stage(u, w, r, 1, dt)
        outs.append(w.cpu().numpy())
    u = torch.from_numpy(u0).cuda()
    w, r = torch.empty_like(u), torch.zeros_like(u)
    p.rk_stage(u, w, r, 1, dt)
    torch.cuda.synchronize()
    assert np.array_equal(w.cpu().numpy(), np.concatenate(outs, axis=1))


@pytest.mark.parametrize("N", [4, 6])
def test_vacuum_then_material_mesh_in_one_process(env, N):
    """The vacuum and the material instantiation of a tensor-core stage
    launched one after the other (each sets up its own launch attributes),
    then the vacuum one again."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(2, 0.1, 8)
    vac, om = dg.Mesh(verts, tets, N), oracle.build_mesh(verts, tets, N)
    mat, _, eps, mu, bc = _setup(dg, verts, tets, N, 51)
    u32 = random_fields(om.K, om.Np, 52).astype(np.float32)
    u = torch.from_numpy(u32).cuda()
    for mesh, kw in ((vac, {}), (mat, dict(eps=eps, mu=mu, bc=bc)), (vac, {})):
        mesh.set_stage_impl(TC)
        mesh.trace_enable(2)
        out = torch.full_like(u, float("nan"))
        mesh.rhs(u, out)
        torch.cuda.synchronize()
        assert _kinds(mesh) == {5}
        assert rel(out.cpu().numpy(), oracle.rhs(om, u32.astype(np.float64), 1.0, **kw)) < RHS_TOL
