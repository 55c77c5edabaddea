"""Failure detection without any GPU fault: an unstable run is reported as
DG_ERR_UNSTABLE (-6).

* dg_energy refuses a non-finite energy (fields holding NaN or Inf);
* the opt-in energy-growth check of dg_step_host (dg_set_energy_check) flags a
  time step above the stability limit: with upwind flux and perfect-conductor
  walls the discrete energy of a stable run does not grow (Section 6).

The premise of the growth test is pinned on the CPU by the oracle: on the same
48-tetrahedron mesh at N = 2 the energy decays at the CFL step and grows by
more than 10^6 in five steps at three times it.

A third failure path is a tensor-core stage whose bounded mbarrier wait runs
out (a lost MMA completion, say): dg_check_wait_timeout runs that bounded wait
on a barrier nothing arrives at, in a kernel with nothing else in flight, and
the mesh reports DG_ERR_CUDA (-4) through the same status word, then stays
usable.
"""
import numpy as np
import pytest

import oracle
from workloads import kuhn_box_mesh, random_fields

UNSTABLE, CUDA_ERR, ARG_ERR = -6, -4, -1
N = 2
FACTOR, UNSTABLE_STEPS = 3.0, 5


def _mesh_and_fields():
    verts, tets = kuhn_box_mesh(2, 0.1, 0)
    om = oracle.build_mesh(verts, tets, N)
    return verts, tets, om, random_fields(om.K, om.Np, 5)


def test_oracle_energy_decays_at_the_cfl_step_and_explodes_above_it():
    _, _, om, u0 = _mesh_and_fields()
    dt = oracle.cfl_dt(om)
    e0 = oracle.energy(om, u0)
    u, _ = oracle.lserk4_run(om, u0, dt, 30)
    assert oracle.energy(om, u) < e0
    u, _ = oracle.lserk4_run(om, u0, FACTOR * dt, UNSTABLE_STEPS)
    assert oracle.energy(om, u) > 1e6 * e0
    assert np.abs(u).max() < 1e30                      # still finite in FP32


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as dg
    return torch, dg


@pytest.mark.gpu
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_fields_are_unstable(env, bad):
    torch, dg = env
    verts, tets, om, u0 = _mesh_and_fields()
    mesh = dg.Mesh(verts, tets, N)
    u32 = u0.astype(np.float32)
    u32[4, 7, 3] = bad
    with pytest.raises(dg.DGError) as ei:
        mesh.energy(torch.from_numpy(u32).cuda())
    assert ei.value.code == UNSTABLE
    with pytest.raises(dg.DGError) as ei:
        mesh.step_host(u32.copy(), None, mesh.dt_cfl, 1)
    assert ei.value.code == UNSTABLE
    # the library stays usable: a finite state afterwards is fine
    assert mesh.energy(torch.from_numpy(u0.astype(np.float32)).cuda()) > 0


@pytest.mark.gpu
def test_energy_growth_check_flags_a_too_large_step(env):
    torch, dg = env
    verts, tets, om, u0 = _mesh_and_fields()
    mesh = dg.Mesh(verts, tets, N)
    u32 = u0.astype(np.float32)
    e0 = oracle.energy(om, u32.astype(np.float64))
    # off (the default): the unstable run completes and reports its energy
    u = u32.copy()
    e = mesh.step_host(u, None, FACTOR * mesh.dt_cfl, UNSTABLE_STEPS)
    assert e > 1e6 * e0
    mesh.set_energy_check(1e-4)
    # on, stable step: no error, the energy decays
    u = u32.copy()
    e = mesh.step_host(u, None, mesh.dt_cfl, 30)
    assert e < e0
    # on, three times the CFL step: DG_ERR_UNSTABLE, with the fields copied back
    u = u32.copy()
    with pytest.raises(dg.DGError) as ei:
        mesh.step_host(u, None, FACTOR * mesh.dt_cfl, UNSTABLE_STEPS)
    assert ei.value.code == UNSTABLE
    assert "energy grew" in str(ei.value)
    assert not np.array_equal(u, u32)
    want, _ = oracle.lserk4_run(om, u32.astype(np.float64), FACTOR * mesh.dt_cfl, UNSTABLE_STEPS)
    assert np.linalg.norm(u - want) < 1e-3 * np.linalg.norm(want)
    mesh.set_energy_check(-1.0)


@pytest.mark.gpu
@pytest.mark.parametrize("polls", [1, 1000, 100000])
def test_a_wait_that_runs_out_is_reported_and_cleared(env, polls):
    torch, dg = env
    verts, tets, om, u0 = _mesh_and_fields()
    mesh = dg.Mesh(verts, tets, N)
    rc, msg, sec = mesh.check_wait_timeout(polls)
    assert rc == CUDA_ERR and "timed out" in msg
    assert 0.0 <= sec < 5.0
    # the status word was cleared: the stage and the energy run normally after it
    u = torch.from_numpy(u0.astype(np.float32)).cuda()
    res = torch.zeros_like(u)
    mesh.step(u, res, mesh.dt_cfl, 2)
    ue, _ = oracle.lserk4_run(om, u0, mesh.dt_cfl, 2)
    assert np.linalg.norm(u.cpu().numpy() - ue) / np.linalg.norm(ue) < 1e-5
    assert mesh.energy(u) > 0
    with pytest.raises(dg.DGError) as ei:            # polls outside 1 .. 2^24
        dg.check(mesh._lib.dg_check_wait_timeout(mesh._h, 0, None), "dg_check_wait_timeout")
    assert ei.value.code == ARG_ERR
