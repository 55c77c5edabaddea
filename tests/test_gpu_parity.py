"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 over all 6*K*Np nodal values): 1e-5 for one FP32
right-hand side, 1e-4 after 100 LSERK4 steps, 1e-6 for the energy.
"""
import numpy as np
import pytest

import oracle
from workloads import cavity_mode, gaussian_pulse, kuhn_box_mesh, pulse_center, random_fields

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


def _setup(dg, verts, tets, N):
    return dg.Mesh(verts, tets, N), oracle.build_mesh(verts, tets, N)


FP32, TC = 1, 2     # stage implementations (dg_set_stage_impl)


def _gpu_rhs(torch, mesh, u32, alpha=None, impl=None):
    if alpha is not None:
        mesh.set_flux(alpha)
    if impl is not None:
        mesh.set_stage_impl(impl)
    u = torch.from_numpy(u32).cuda()
    out = torch.full_like(u, float("nan"))
    mesh.rhs(u, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("N", range(1, 10))
def test_rhs_parity_all_orders(env, N):
    torch, dg = env
    n = 3 if N <= 4 else 2
    verts, tets = kuhn_box_mesh(n, 0.15, N)          # K = 162 or 48: ragged last tile
    mesh, om = _setup(dg, verts, tets, N)
    u32 = random_fields(om.K, om.Np, 10 + N).astype(np.float32)
    got = _gpu_rhs(torch, mesh, u32)
    want = oracle.rhs(om, u32.astype(np.float64))
    assert np.isfinite(got).all()
    assert rel(got, want) < RHS_TOL


def _stage_kinds(mesh):
    _, kinds = mesh.trace_read()
    return set(int(k) for k in kinds)


@pytest.mark.parametrize("impl", [FP32, TC])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_rhs_parity_both_implementations(env, N, impl):
    """Orders 1..4 run on the tensor cores by default; both paths must match.
    K = 384 = 19 full tiles of 20 + a ragged tile of 4."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(4, 0.15, 20 + N)
    mesh, om = _setup(dg, verts, tets, N)
    u32 = random_fields(om.K, om.Np, 30 + N).astype(np.float32)
    u32[:, ::7] *= 1e-6                                  # rows with very different scales
    mesh.trace_enable(4)
    got = _gpu_rhs(torch, mesh, u32, impl=impl)
    assert _stage_kinds(mesh) == ({5} if impl == TC else {1})
    assert rel(got, oracle.rhs(om, u32.astype(np.float64))) < RHS_TOL


@pytest.mark.parametrize("N", [5, 6, 7])
def test_tc_operator_in_tensor_memory_rhs_parity(env, N):
    """Orders 5..7 on the tensor cores (operator in tensor memory, tiles of 8;
    order 7 with the update straight to global memory): K = 162 = 20 tiles + a
    ragged tile of 2, rows of very different scales."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.15, 40 + N)
    mesh, om = _setup(dg, verts, tets, N)
    u32 = random_fields(om.K, om.Np, 50 + N).astype(np.float32)
    u32[:, ::7] *= 1e-6
    mesh.trace_enable(4)
    got = _gpu_rhs(torch, mesh, u32, impl=TC)
    mesh.set_stage_impl(0)
    assert _stage_kinds(mesh) == {5}
    assert np.isfinite(got).all()
    assert rel(got, oracle.rhs(om, u32.astype(np.float64))) < RHS_TOL


@pytest.mark.parametrize("N", [5, 6])
def test_tc_operator_in_tensor_memory_step_parity(env, N):
    """20 LSERK4 steps of the cavity mode on the tensor cores at orders 5, 6."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(2, 0.1, 0)
    mesh, om = _setup(dg, verts, tets, N)
    mesh.set_stage_impl(TC)
    u0 = cavity_mode(om.x, om.y, om.z, 0.0).astype(np.float32)
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.trace_enable(200)
    mesh.step(u, res, mesh.dt_cfl, 20)
    torch.cuda.synchronize()
    mesh.set_stage_impl(0)
    assert _stage_kinds(mesh) == {4}
    ue, re_ = oracle.lserk4_run(om, u0.astype(np.float64), mesh.dt_cfl, 20)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL
    assert rel(res.cpu().numpy(), re_) < 10 * STEP_TOL


def test_tc_operator_in_tensor_memory_several_tiles_per_cta(env):
    """N = 6, K = 3 072 = 384 tiles of 8: every persistent CTA runs its
    pipeline over two or three tiles; two steps against the oracle."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(8, 0.15, 5)
    mesh, om = _setup(dg, verts, tets, 6)
    mesh.set_stage_impl(TC)
    u0 = random_fields(om.K, om.Np, 43).astype(np.float32)
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.trace_enable(10)
    mesh.step(u, res, mesh.dt_cfl, 2)
    torch.cuda.synchronize()
    mesh.set_stage_impl(0)
    assert _stage_kinds(mesh) == {4}
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), mesh.dt_cfl, 2)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL


@pytest.mark.parametrize("N", [5, 6])
def test_tc_operator_in_tensor_memory_every_magnitude(env, N):
    """Per-element magnitudes from zero through 1e-37 to 1e20: finite, and each
    magnitude class within the one-RHS tolerance."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(4, 0.15, 6)
    mesh, om = _setup(dg, verts, tets, N)
    rng = np.random.Generator(np.random.PCG64(33))
    scales = np.array([0.0, 1e-37, 1e-30, 1e-3, 1.0, 1e20])
    cls = rng.integers(0, len(scales), om.K)
    u32 = (random_fields(om.K, om.Np, 34) * scales[cls][None, :, None]).astype(np.float32)
    got = _gpu_rhs(torch, mesh, u32, impl=TC)
    mesh.set_stage_impl(0)
    want = oracle.rhs(om, u32.astype(np.float64))
    assert np.isfinite(got).all()
    for k in range(len(scales)):
        sel = cls == k
        if np.any(want[:, sel]):
            assert rel(got[:, sel], want[:, sel]) < RHS_TOL, scales[k]


def test_tc_operator_in_tensor_memory_full_size_n6(env):
    """The N = 6 workload (16^3 x 6 = 24 576 tets, cavity mode plus noise):
    tensor-core and FP32 stages agree everywhere after one step, and sampled
    elements match the oracle on a 5-ring patch."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(16, 0.15, 0)
    mesh = dg.Mesh(verts, tets, 6)
    x = mesh.nodes()
    u0 = (cavity_mode(x[0], x[1], x[2], 0.0) +
          1e-3 * random_fields(mesh.K, mesh.Np, 12)).astype(np.float32)
    out = []
    for impl in (TC, FP32):
        mesh.set_stage_impl(impl)
        u = torch.from_numpy(u0).cuda()
        res = torch.zeros_like(u)
        mesh.step(u, res, mesh.dt_cfl, 1)
        out.append(u.cpu().numpy())
    mesh.set_stage_impl(0)
    assert np.isfinite(out[0]).all()
    assert rel(out[0], out[1].astype(np.float64)) < RHS_TOL
    seeds = np.array([mesh.K // 2 + 3, 6 * (16 * 16 * 8 + 16 * 5 + 7) + 2])
    patch = _vertex_rings(tets, seeds, 5)
    om = _oracle_on_patch(verts, tets, patch, 6)
    ue, _ = oracle.lserk4_run(om, u0[:, patch].astype(np.float64), mesh.dt_cfl, 1)
    pos = np.searchsorted(patch, seeds)
    assert rel(out[0][:, seeds], ue[:, pos]) < RHS_TOL


def test_tc_falls_back_when_tiles_are_not_aligned(env):
    """K * Np not a multiple of 4 (K = 162, N = 4): the FP32 kernel runs."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.15, 2)
    mesh, om = _setup(dg, verts, tets, 4)
    u32 = random_fields(om.K, om.Np, 8).astype(np.float32)
    mesh.trace_enable(4)
    got = _gpu_rhs(torch, mesh, u32, impl=TC)
    assert _stage_kinds(mesh) == {1}
    assert rel(got, oracle.rhs(om, u32.astype(np.float64))) < RHS_TOL


@pytest.mark.parametrize("impl", [FP32, TC])
def test_step_parity_both_implementations(env, impl):
    torch, dg = env
    verts, tets = kuhn_box_mesh(2, 0.1, 0)
    mesh, om = _setup(dg, verts, tets, 4)
    mesh.set_stage_impl(impl)
    u0 = cavity_mode(om.x, om.y, om.z, 0.0).astype(np.float32)
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.trace_enable(500)
    mesh.step(u, res, mesh.dt_cfl, 100)
    torch.cuda.synchronize()
    assert _stage_kinds(mesh) == ({4} if impl == TC else {0})
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), mesh.dt_cfl, 100)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL


def test_step_parity_several_tiles_per_cta(env):
    """K = 10 368 tets = 519 tiles of 20: every persistent CTA of the
    tensor-core stage runs its tile pipeline over several tiles (the smaller
    meshes give each CTA one tile)."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(12, 0.15, 5)
    mesh, om = _setup(dg, verts, tets, 4)
    mesh.set_stage_impl(TC)
    u0 = random_fields(om.K, om.Np, 41).astype(np.float32)
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.trace_enable(10)
    mesh.step(u, res, mesh.dt_cfl, 2)
    torch.cuda.synchronize()
    assert _stage_kinds(mesh) == {4}
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), mesh.dt_cfl, 2)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL


@pytest.mark.parametrize("impl", [FP32, TC])
def test_partition_renumbering_is_exact(env, impl):
    """A randomly numbered mesh and its dg_partition_order renumbering give the
    same right-hand side and LSERK4 steps, bit for bit up to the renumbering:
    every element's arithmetic is unchanged, only where its neighbours' values
    come from (inside the tile or gathered) differs."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(6, 0.15, 8)
    tets = tets[np.random.Generator(np.random.PCG64(12)).permutation(len(tets))]
    a = dg.Mesh(verts, tets, 4)
    perm = a.partition_order(20)
    b = dg.Mesh(verts, tets[perm], 4)
    u = random_fields(a.K, a.Np, 13).astype(np.float32)
    ra = _gpu_rhs(torch, a, u, impl=impl)
    rb = _gpu_rhs(torch, b, np.ascontiguousarray(u[:, perm]), impl=impl)
    assert np.array_equal(rb, ra[:, perm])
    ua, ub = torch.from_numpy(u).cuda(), torch.from_numpy(np.ascontiguousarray(u[:, perm])).cuda()
    res_a, res_b = torch.zeros_like(ua), torch.zeros_like(ub)
    a.step(ua, res_a, a.dt_cfl, 2)
    b.step(ub, res_b, a.dt_cfl, 2)
    assert np.array_equal(ub.cpu().numpy(), ua.cpu().numpy()[:, perm])
    assert abs(a.energy(ua) - b.energy(ub)) <= 1e-12 * a.energy(ua)
    a.set_stage_impl(0)
    b.set_stage_impl(0)


def test_tc_rows_of_every_magnitude(env):
    """Per-element magnitudes from exact zero through 1e-37 (the row scale hits
    its 2^127 clamp) to 1e20, several tiles per CTA: every value finite and each
    magnitude class within the one-RHS tolerance of the oracle."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(12, 0.15, 6)
    mesh, om = _setup(dg, verts, tets, 4)
    rng = np.random.Generator(np.random.PCG64(31))
    scales = np.array([0.0, 1e-37, 1e-30, 1e-3, 1.0, 1e20])
    cls = rng.integers(0, len(scales), om.K)
    u32 = (random_fields(om.K, om.Np, 32) * scales[cls][None, :, None]).astype(np.float32)
    mesh.trace_enable(4)
    got = _gpu_rhs(torch, mesh, u32, impl=TC)
    assert _stage_kinds(mesh) == {5}
    mesh.set_stage_impl(0)
    want = oracle.rhs(om, u32.astype(np.float64))
    assert np.isfinite(got).all()
    for k in range(len(scales)):
        sel = cls == k
        if np.any(want[:, sel]):
            assert rel(got[:, sel], want[:, sel]) < RHS_TOL, scales[k]


@pytest.mark.parametrize("N", [2, 4, 6])
def test_rhs_parity_smooth_fields_and_central_flux(env, N):
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.1, 2)
    mesh, om = _setup(dg, verts, tets, N)
    u32 = cavity_mode(om.x, om.y, om.z, 0.0).astype(np.float32)
    u32[3:] = gaussian_pulse(om.x, om.y, om.z, 0.4, (0.1, -0.2, 0.3))[2]
    for alpha in (1.0, 0.0):
        got = _gpu_rhs(torch, mesh, u32, alpha)
        want = oracle.rhs(om, u32.astype(np.float64), alpha=alpha)
        assert rel(got, want) < RHS_TOL


@pytest.mark.parametrize("case", ["single_tet", "two_tets", "one_tile_plus_one", "all_wall_hex"])
def test_rhs_edge_cases(env, case):
    torch, dg = env
    if case == "single_tet":
        verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
        tets = np.array([[0, 1, 3, 2]])                  # negatively oriented: swapped internally
    elif case == "two_tets":
        verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.9, 1.1, 1.2]], float)
        tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    elif case == "one_tile_plus_one":                   # 33 elements: full tile + 1
        verts, tets = kuhn_box_mesh(2, 0.1, 7)
        tets = tets[:33]
    else:                                                # 6 tets, every tet has wall faces
        verts, tets = kuhn_box_mesh(1, 0.0, 0)
    for N in (1, 4, 9):
        mesh, om = _setup(dg, verts, tets, N)
        u32 = random_fields(om.K, om.Np, N).astype(np.float32)
        got = _gpu_rhs(torch, mesh, u32)
        assert rel(got, oracle.rhs(om, u32.astype(np.float64))) < RHS_TOL


@pytest.mark.parametrize("N", [1, 3, 5])
def test_step_parity_100_steps(env, N):
    torch, dg = env
    verts, tets = kuhn_box_mesh(2, 0.1, 0)
    mesh, om = _setup(dg, verts, tets, N)
    u0 = cavity_mode(om.x, om.y, om.z, 0.0).astype(np.float32)
    dt = mesh.dt_cfl
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.step(u, res, dt, 100)
    torch.cuda.synchronize()
    ue, re_ = oracle.lserk4_run(om, u0.astype(np.float64), dt, 100)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL
    assert rel(res.cpu().numpy(), re_) < 10 * STEP_TOL


def test_golden_cavity_run_fp64_config(env):
    """N=3 on 4^3 x 6 = 384 jittered tets, cavity mode, 10 LSERK4 steps at the CFL step."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(4, 0.1, 0)
    mesh, om = _setup(dg, verts, tets, 3)
    u0 = cavity_mode(om.x, om.y, om.z, 0.0).astype(np.float32)
    dt = mesh.dt_cfl
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    e0 = mesh.energy(u)
    for _ in range(10):                       # 10 calls of one step (odd stage count each)
        mesh.step(u, res, dt, 1)
    e1 = mesh.energy(u)
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), dt, 10)
    assert rel(u.cpu().numpy(), ue) < STEP_TOL
    assert abs(e1 - oracle.energy(om, ue)) < 1e-6 * oracle.energy(om, ue)
    assert e1 <= e0 * (1 + 1e-6)


@pytest.mark.parametrize("N,n", [(N, 2) for N in range(1, 10)] + [(4, 6), (6, 5), (7, 5), (8, 4)])
def test_energy_parity(env, N, n):
    """Every order (1, 2, 3, 5: row-staged kernel; 4, 6..9: the weighted upper
    triangle of M in shared memory, 512 / 512 / 256 / 128 / 32 rows per pass);
    n = 6, 5 and 4 give 7776, 4500 and 2304 field rows: many passes with a
    ragged last one."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(n, 0.15, 1)
    mesh, om = _setup(dg, verts, tets, N)
    u32 = random_fields(om.K, om.Np, 3).astype(np.float32)
    e = mesh.energy(torch.from_numpy(u32).cuda())
    eo = oracle.energy(om, u32.astype(np.float64))
    assert abs(e - eo) < 1e-6 * eo


def test_step_host_matches_device_step(env):
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.1, 0)
    mesh = dg.Mesh(verts, tets, 4)
    x = mesh.nodes()
    u0 = cavity_mode(x[0], x[1], x[2], 0.0).astype(np.float32)
    uh, rh = u0.copy(), np.zeros_like(u0)
    eh = mesh.step_host(uh, rh, mesh.dt_cfl, 3)
    ud, rd = torch.from_numpy(u0).cuda(), torch.zeros(u0.shape, device="cuda")
    mesh.step(ud, rd, mesh.dt_cfl, 3)
    torch.cuda.synchronize()
    assert np.array_equal(uh, ud.cpu().numpy()) and np.array_equal(rh, rd.cpu().numpy())
    assert abs(eh - mesh.energy(ud)) <= 1e-12 * eh
    # without a host RK register only u crosses the bus; the steps are the same,
    # and a garbage register left in the library's buffer does not leak in
    uh2 = u0.copy()
    mesh.step_host(uh2, np.full_like(u0, 1e30), mesh.dt_cfl, 1, with_energy=False)
    uh2 = u0.copy()
    eh2 = mesh.step_host(uh2, None, mesh.dt_cfl, 3)
    assert np.array_equal(uh2, uh) and eh2 == eh


def test_step_is_deterministic_and_resumable(env):
    """Checkpoint/resume: 2+3 steps bit-identical to 5 steps."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.1, 0)
    mesh = dg.Mesh(verts, tets, 3)
    u0 = torch.from_numpy(random_fields(mesh.K, mesh.Np, 4).astype(np.float32)).cuda()
    a, ra = u0.clone(), torch.zeros_like(u0)
    mesh.step(a, ra, mesh.dt_cfl, 5)
    b, rb = u0.clone(), torch.zeros_like(u0)
    mesh.step(b, rb, mesh.dt_cfl, 2)
    b2, rb2 = b.cpu().clone(), rb.cpu().clone()          # host checkpoint
    b.copy_(b2.cuda()); rb.copy_(rb2.cuda())
    mesh.step(b, rb, mesh.dt_cfl, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(ra, rb)


# ---------------------------------------------------------------------------
# full-size workload (N=4, 24^3 x 6 = 82 944 tets), sampled against the oracle
# ---------------------------------------------------------------------------
def _vertex_rings(tets, seeds, rings):
    """Tetrahedra within `rings` vertex-adjacency steps of the seed elements."""
    sel = np.zeros(len(tets), bool)
    sel[seeds] = True
    for _ in range(rings):
        vs = np.unique(tets[sel])
        sel |= np.isin(tets, vs).any(axis=1)
    return np.nonzero(sel)[0]


def _oracle_on_patch(verts, tets, patch, N):
    return oracle.build_mesh(verts, tets[patch], N)


@pytest.fixture(scope="module")
def full(env):
    torch, dg = env
    verts, tets = kuhn_box_mesh(24, 0.15, 0)
    mesh = dg.Mesh(verts, tets, 4)
    x = mesh.nodes()
    u0 = gaussian_pulse(x[0], x[1], x[2], 0.2, pulse_center(1)).astype(np.float32)
    u0 += 1e-3 * random_fields(mesh.K, mesh.Np, 9).astype(np.float32)   # exercise every field
    return verts, tets, mesh, u0


def test_full_size_rhs_sampled(env, full):
    torch, dg = env
    verts, tets, mesh, u0 = full
    got = _gpu_rhs(torch, mesh, u0)
    rng = np.random.default_rng(0)
    seeds = np.concatenate([[0, 1, mesh.K - 1], rng.integers(0, mesh.K, 29)])
    patch = _vertex_rings(tets, seeds, 1)
    om = _oracle_on_patch(verts, tets, patch, 4)
    want = oracle.rhs(om, u0[:, patch].astype(np.float64))
    pos = np.searchsorted(patch, seeds)
    assert rel(got[:, seeds], want[:, pos]) < RHS_TOL


def test_full_size_tc_matches_fp32_everywhere(env, full):
    """Every value at full size: tensor-core and FP32 paths agree (each is
    within 1e-5 of the oracle, so they agree within 2e-5)."""
    torch, dg = env
    verts, tets, mesh, u0 = full
    mesh.trace_enable(4)
    a = _gpu_rhs(torch, mesh, u0, impl=TC)
    assert _stage_kinds(mesh) == {5}
    b = _gpu_rhs(torch, mesh, u0, impl=FP32)
    mesh.set_stage_impl(0)
    assert np.isfinite(a).all()
    assert rel(a, b.astype(np.float64)) < 2 * RHS_TOL


def test_full_size_pure_pulse_step_both_implementations(env, full):
    """The Gaussian pulse alone (H = 0, E underflowing to zero far from the
    centre), one LSERK4 step at full size: the two stage implementations agree
    everywhere and every value stays finite."""
    torch, dg = env
    verts, tets, mesh, _ = full
    x = mesh.nodes()
    u0 = gaussian_pulse(x[0], x[1], x[2], 0.2, pulse_center(1)).astype(np.float32)
    out = []
    for impl in (TC, FP32):
        mesh.set_stage_impl(impl)
        u = torch.from_numpy(u0).cuda()
        res = torch.zeros_like(u)
        mesh.step(u, res, mesh.dt_cfl, 1)
        out.append(u.cpu().numpy())
    mesh.set_stage_impl(0)
    assert np.isfinite(out[0]).all()
    assert rel(out[0], out[1].astype(np.float64)) < RHS_TOL


def test_full_size_step_sampled(env, full):
    """One LSERK4 step (5 stages) at full size: the centre of a 5-ring patch
    depends only on patch data, so the oracle on the patch is exact there."""
    torch, dg = env
    verts, tets, mesh, u0 = full
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    e0 = mesh.energy(u)
    mesh.step(u, res, mesh.dt_cfl, 1)
    got = u.cpu().numpy()
    e1 = mesh.energy(u)
    assert e1 <= e0 * (1 + 1e-6)
    seeds = np.array([mesh.K // 2 + 3, 6 * (24 * 24 * 12 + 24 * 5 + 7) + 2])
    patch = _vertex_rings(tets, seeds, 5)
    om = _oracle_on_patch(verts, tets, patch, 4)
    ue, _ = oracle.lserk4_run(om, u0[:, patch].astype(np.float64), mesh.dt_cfl, 1)
    pos = np.searchsorted(patch, seeds)
    assert rel(got[:, seeds], ue[:, pos]) < RHS_TOL


@pytest.mark.parametrize("impl,N", [(FP32, 4), (TC, 4), (TC, 6)])
def test_rk_stages_equal_a_step(env, impl, N):
    """Five dg_rk_stage calls with swapped buffers are bit-identical to dg_step."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(4, 0.1, 3)
    mesh = dg.Mesh(verts, tets, N)
    mesh.set_stage_impl(impl)
    u0 = torch.from_numpy(random_fields(mesh.K, mesh.Np, 5).astype(np.float32)).cuda()
    u, res = u0.clone(), torch.zeros_like(u0)
    mesh.step(u, res, mesh.dt_cfl, 2)
    a, b, r = u0.clone(), torch.empty_like(u0), torch.zeros_like(u0)
    for _ in range(2):
        for i in range(5):
            mesh.rk_stage(a, b, r, i, mesh.dt_cfl)
            a, b = b, a
    mesh.set_stage_impl(0)
    torch.cuda.synchronize()
    assert torch.equal(a, u) and torch.equal(r, res)   # after each swap `a` holds the state


@pytest.mark.parametrize("impl", [FP32, TC])
def test_subdomains_in_lockstep_match_the_single_mesh(env, impl):
    """Three subdomains of one mesh (domain.build_plans), each with its own
    local mesh, stepped stage by stage on one GPU with their cut-face traces
    copied between them before every stage: every owned element is bit-identical
    to the single-mesh run (the same arithmetic, only ghost-held neighbours)."""
    torch, dg = env
    from paper_0901_1024_gb300.domain import build_plans
    verts, tets = kuhn_box_mesh(6, 0.15, 4)
    glob = dg.Mesh(verts, tets, 4)
    glob.set_stage_impl(impl)
    plans = build_plans(glob, tets, 3)
    u0 = random_fields(glob.K, glob.Np, 21).astype(np.float32)
    dt = glob.dt_cfl
    ug, rg = torch.from_numpy(u0).cuda(), torch.zeros(u0.shape, device="cuda")
    glob.step(ug, rg, dt, 2)
    meshes, us, works, ress = [], [], [], []
    for p in plans:
        m = dg.Mesh(verts, p.tets, 4)
        m.set_stage_impl(impl)
        meshes.append(m)
        us.append(torch.from_numpy(np.ascontiguousarray(u0[:, np.concatenate([p.owned, p.ghosts])])).cuda())
        works.append(torch.empty_like(us[-1]))
        ress.append(torch.zeros_like(us[-1]))
    idx = [{q: torch.as_tensor(v, device="cuda") for q, v in p.send.items()} for p in plans]
    ridx = [{q: torch.as_tensor(v, device="cuda") for q, v in p.recv.items()} for p in plans]
    src, dst = us, works
    for _ in range(2):
        for i in range(5):
            for p, u in zip(plans, src):
                u[:, p.n_owned:, :] = 0
            for r, p in enumerate(plans):
                for q, ix in idx[r].items():
                    src[q].view(6, -1).index_copy_(1, ridx[q][r], src[r].view(6, -1).index_select(1, ix))
            for r, p in enumerate(plans):
                ress[r][:, p.n_owned:, :] = 0
                meshes[r].trace_enable(1)
                meshes[r].rk_stage(src[r], dst[r], ress[r], i, dt)
                assert _stage_kinds(meshes[r]) == ({4} if impl == TC else {0})
            src, dst = dst, src
    torch.cuda.synchronize()
    glob.set_stage_impl(0)
    full = ug.cpu().numpy()
    for p, u, m in zip(plans, src, meshes):
        assert p.n_local % 4 == 0
        assert np.array_equal(u.cpu().numpy()[:, :p.n_owned], full[:, p.owned])


@pytest.mark.parametrize("impl,N", [(FP32, 4), (TC, 4), (TC, 6), (FP32, 7)])
def test_overlapped_subdomains_match_the_single_mesh(env, impl, N):
    """The overlapped stage of a subdomain: plans ordered interior first
    (build_plans with the stage kernel's tile), each stage run as
    dg_rk_stage_range over the interior tiles while the ghosts still hold NaN
    (so an interior element that read a ghost would poison its result), then the
    trace copy, then the range over the remaining owned and ghost elements.
    Every owned element is bit-identical to the single-mesh run."""
    torch, dg = env
    from paper_0901_1024_gb300.domain import build_plans
    verts, tets = kuhn_box_mesh(6 if N < 7 else 4, 0.15, 4)
    glob = dg.Mesh(verts, tets, N)
    glob.set_stage_impl(impl)
    tile = glob.stage_tile()
    plans = build_plans(glob, tets, 3, tile=tile)
    u0 = random_fields(glob.K, glob.Np, 22).astype(np.float32)
    dt = glob.dt_cfl
    ug, rg = torch.from_numpy(u0).cuda(), torch.zeros(u0.shape, device="cuda")
    glob.step(ug, rg, dt, 2)
    meshes, us, works, ress = [], [], [], []
    for p in plans:
        assert 0 < p.n_interior < p.n_owned and p.n_interior % tile == 0
        m = dg.Mesh(verts, p.tets, N)
        m.set_stage_impl(impl)
        meshes.append(m)
        us.append(torch.from_numpy(np.ascontiguousarray(u0[:, np.concatenate([p.owned, p.ghosts])])).cuda())
        works.append(torch.empty_like(us[-1]))
        ress.append(torch.zeros_like(us[-1]))
        assert m.stage_tile(us[-1], works[-1], ress[-1]) == tile
    idx = [{q: torch.as_tensor(v, device="cuda") for q, v in p.send.items()} for p in plans]
    ridx = [{q: torch.as_tensor(v, device="cuda") for q, v in p.recv.items()} for p in plans]
    src, dst = us, works
    for _ in range(2):
        for i in range(5):
            for r, p in enumerate(plans):
                src[r][:, p.n_owned:, :] = float("nan")
                meshes[r].trace_enable(2)
                meshes[r].rk_stage_range(src[r], dst[r], ress[r], i, dt, 0, p.n_interior)
            for p, u in zip(plans, src):
                u[:, p.n_owned:, :] = 0
            for r, p in enumerate(plans):
                for q, ix in idx[r].items():
                    src[q].view(6, -1).index_copy_(1, ridx[q][r], src[r].view(6, -1).index_select(1, ix))
            for r, p in enumerate(plans):
                ress[r][:, p.n_owned:, :] = 0
                meshes[r].rk_stage_range(src[r], dst[r], ress[r], i, dt, p.n_interior, p.n_local)
                assert _stage_kinds(meshes[r]) == ({4} if impl == TC else {0})
            src, dst = dst, src
    torch.cuda.synchronize()
    glob.set_stage_impl(0)
    full = ug.cpu().numpy()
    for p, u in zip(plans, src):
        assert np.array_equal(u.cpu().numpy()[:, :p.n_owned], full[:, p.owned])


def test_range_stage_argument_errors(env):
    torch, dg = env
    mesh = dg.Mesh(*kuhn_box_mesh(4, 0.1, 3), 4)
    u = torch.zeros((6, mesh.K, mesh.Np), device="cuda")
    out, res = torch.empty_like(u), torch.zeros_like(u)
    E = mesh.stage_tile(u, out, res)
    assert E == 20                                            # the tensor-core tile at N = 4
    mesh.rk_stage_range(u, out, res, 0, 0.01, 0, mesh.K)     # the whole mesh
    mesh.rk_stage_range(u, out, res, 0, 0.01, E, 3 * E)
    for k0, k1 in ((-E, E), (E, E), (3, E), (0, 7), (0, mesh.K + 1), (2 * E, E)):
        with pytest.raises(dg.DGError):
            mesh.rk_stage_range(u, out, res, 0, 0.01, k0, k1)
    mesh.set_stage_impl(FP32)
    assert mesh.stage_tile() == 32                             # FP32 tile shape 0 at N = 4
    mesh.set_stage_shape(1)
    assert mesh.stage_tile() == 16
    mesh.set_stage_shape(0)
    mesh.set_stage_impl(0)


@pytest.mark.parametrize("N", [2, 4, 7])
def test_packed_mesh_stages_and_range_energies(env, N):
    """dg_mesh_pack of two meshes: a packed stage with per-element steps
    (dg_rk_stage_elem) is bit for bit each mesh's own stage with its own step,
    and dg_energy_range over each part matches that mesh's dg_energy."""
    torch, dg = env
    va, ta = kuhn_box_mesh(2, 0.1, 1)
    vb, tb = kuhn_box_mesh(2, 0.15, 2)
    a, b = dg.Mesh(va, ta, N), dg.Mesh(vb, tb, N)
    p = dg.Mesh.pack([a, b])
    assert p.K == a.K + b.K
    ua = random_fields(a.K, a.Np, 31).astype(np.float32)
    ub = random_fields(b.K, b.Np, 32).astype(np.float32)
    dta, dtb = np.float32(0.7 * a.dt_cfl), np.float32(0.4 * b.dt_cfl)
    up = torch.from_numpy(np.concatenate([ua, ub], axis=1)).cuda()
    dts = torch.from_numpy(np.concatenate([np.full(a.K, dta), np.full(b.K, dtb)])).cuda()
    out, res = torch.empty_like(up), torch.zeros_like(up)
    p.rk_stage_elem(up, out, res, 1, dts)
    want = []
    for m, u, dt in ((a, ua, dta), (b, ub, dtb)):
        x = torch.from_numpy(u).cuda()
        y, r = torch.empty_like(x), torch.zeros_like(x)
        m.rk_stage(x, y, r, 1, float(dt))
        want.append(y.cpu().numpy())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.concatenate(want, axis=1))
    ea = p.energy_range(up, 0, a.K)
    eb = p.energy_range(up, a.K, p.K)
    assert abs(ea - a.energy(torch.from_numpy(ua).cuda())) <= 1e-12 * ea
    assert abs(eb - b.energy(torch.from_numpy(ub).cuda())) <= 1e-12 * eb
    assert p.energy_range(up, 0, p.K) == p.energy(up)
