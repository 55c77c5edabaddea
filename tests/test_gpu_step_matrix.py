"""GPU parity over time: every fused RK-stage instantiation that dg_step can run,
100 LSERK4 steps against the FP64 oracle.

The fused stage kernels are template instantiations per (kernel family, order
N, materials): the right-hand-side instantiations (no RK update) are covered by
the one-RHS tests; these tests run the stage instantiations themselves, each
for 100 LSERK4 steps on a 48-tetrahedron cavity (Section 6's time stepper),
element by element against `oracle.lserk4_run` at relative L2 <= 1e-4:

  * impl: FP32 CUDA cores (all orders; tile shape 0, and shape 1 -- half the
    tetrahedra per tile -- in vacuum) and tensor cores (every order that has a
    tensor-core stage);
  * kind: vacuum, or per-element eps, mu with a random mix of perfect-conductor
    and characteristic absorbing boundary faces (the EXT instantiation).

A second group steps meshes with several tiles per persistent CTA (K >= 3 000)
for 10 steps on every tensor-core order, so each CTA's tile pipeline wraps its
rings several times.  The trace of kernel kinds proves which family ran.
"""
import numpy as np
import pytest

import oracle
from workloads import cavity_mode, kuhn_box_mesh, random_fields

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-4
FP32, TC = 1, 2
FP32_S1 = 11                                   # FP32 stage in tile shape 1 (test-local code)
KIND_FP32_STAGE, KIND_TC_STAGE = 0, 4          # dg_trace_read kinds of a fused RK stage
TC_ORDERS = range(1, 8)


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


def _cases():
    out = []
    for kind in ("vacuum", "ext"):
        for N in range(1, 10):
            out.append(pytest.param(FP32, N, kind, id=f"fp32-N{N}-{kind}"))
            if kind == "vacuum":
                out.append(pytest.param(FP32_S1, N, kind, id=f"fp32shape1-N{N}-{kind}"))
        for N in TC_ORDERS:
            out.append(pytest.param(TC, N, kind, id=f"tc-N{N}-{kind}"))
    return out


def _materials(K, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.5, 4.0, K), rng.uniform(0.5, 3.0, K),
            rng.integers(0, 2, (K, 4)).astype(np.int8))


def _run(torch, mesh, u0, dt, nsteps, impl):
    mesh.set_stage_shape(1 if impl == FP32_S1 else 0)
    impl = FP32 if impl == FP32_S1 else impl
    mesh.set_stage_impl(impl)
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)
    mesh.trace_enable(5 * nsteps + 5)
    mesh.step(u, res, dt, nsteps)
    torch.cuda.synchronize()
    _, kinds = mesh.trace_read()
    mesh.set_stage_impl(0)
    mesh.set_stage_shape(0)
    mesh.trace_enable(0)
    return u.cpu().numpy(), res.cpu().numpy(), set(int(k) for k in kinds)


@pytest.mark.parametrize("impl,N,kind", _cases())
def test_100_steps_every_stage_instantiation(env, impl, N, kind):
    torch, dg = env
    verts, tets = kuhn_box_mesh(2, 0.1, 3)              # K = 48: K Np % 4 == 0 at every order
    mesh, om = dg.Mesh(verts, tets, N), oracle.build_mesh(verts, tets, N)
    kw = {}
    if kind == "ext":
        eps, mu, bc = _materials(om.K, 100 + N)
        mesh.set_materials(eps, mu)
        mesh.set_boundary(bc)
        kw = dict(eps=eps, mu=mu, bc=bc)
    u0 = cavity_mode(om.x, om.y, om.z, 0.0).astype(np.float32)
    u0 += 0.05 * random_fields(om.K, om.Np, 200 + N).astype(np.float32)   # every field nonzero
    dt = mesh.dt_cfl
    got, res, kinds = _run(torch, mesh, u0, dt, 100, impl)
    assert kinds == {KIND_TC_STAGE if impl == TC else KIND_FP32_STAGE}
    ue, re_ = oracle.lserk4_run(om, u0.astype(np.float64), dt, 100, **kw)
    assert np.isfinite(got).all()
    assert rel(got, ue) < STEP_TOL
    assert rel(res, re_) < 10 * STEP_TOL


@pytest.mark.parametrize("N", TC_ORDERS)
def test_several_tiles_per_cta_10_steps(env, N):
    """K = 10 368 (orders 1..4: 519 tiles of 20) or 3 072 (orders 5..7: 384
    tiles of 8) on 152 SMs: every CTA runs two or more tiles through its rings."""
    torch, dg = env
    n = 12 if N <= 4 else 8
    verts, tets = kuhn_box_mesh(n, 0.15, 5)
    mesh, om = dg.Mesh(verts, tets, N), oracle.build_mesh(verts, tets, N)
    u0 = random_fields(om.K, om.Np, 41 + N).astype(np.float32)
    dt = mesh.dt_cfl
    got, _, kinds = _run(torch, mesh, u0, dt, 10, TC)
    assert kinds == {KIND_TC_STAGE}
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), dt, 10)
    assert np.isfinite(got).all()
    assert rel(got, ue) < STEP_TOL


@pytest.mark.parametrize("N,kind", [(5, "vacuum"), (7, "vacuum"), (7, "ext")])
def test_ragged_last_tile_10_steps(env, N, kind):
    """K = 162 = 20 tiles of 8 + a ragged tile of 2 on the operator-in-tensor-
    memory stages (order 7: the update's global stores are guarded per
    element), per-element steps included via the materials case."""
    torch, dg = env
    verts, tets = kuhn_box_mesh(3, 0.15, 60 + N)
    mesh, om = dg.Mesh(verts, tets, N), oracle.build_mesh(verts, tets, N)
    kw = {}
    if kind == "ext":
        eps, mu, bc = _materials(om.K, 300 + N)
        mesh.set_materials(eps, mu)
        mesh.set_boundary(bc)
        kw = dict(eps=eps, mu=mu, bc=bc)
    u0 = random_fields(om.K, om.Np, 70 + N).astype(np.float32)
    dt = mesh.dt_cfl
    got, _, kinds = _run(torch, mesh, u0, dt, 10, TC)
    assert kinds == {KIND_TC_STAGE}
    ue, _ = oracle.lserk4_run(om, u0.astype(np.float64), dt, 10, **kw)
    assert np.isfinite(got).all()
    assert rel(got, ue) < STEP_TOL
