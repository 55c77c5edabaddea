"""Domain decomposition of one mesh (paper_0901_1024_gb300/domain.py) on CPU
ranks: plan invariants, and 2- and 3-rank gloo runs whose per-rank stage is the
FP64 oracle's LSERK4 stage on the rank's local mesh.  After the per-stage
trace exchange every owned element must follow the single-domain oracle run.
(The CUDA path runs the same stepping loop with dg_rk_stage on each rank's
GPU; the multi-rank exchange itself is exercised here, on CPU ranks.)"""
import os
import socket

import numpy as np
import pytest

import oracle
from workloads import kuhn_box_mesh, random_fields

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


@pytest.fixture(scope="module")
def dg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as pkg
    return pkg


def _mesh(dg, n=3, N=2, seed=3):
    verts, tets = kuhn_box_mesh(n, 0.1, seed)
    tets = tets[np.random.Generator(np.random.PCG64(seed)).permutation(len(tets))]
    return verts, tets, dg.Mesh(verts, tets, N)


@pytest.mark.parametrize("n,world", [(2, 7), (2, 9), (2, 13)])
def test_padding_falls_back_to_far_elements_and_never_touches_owned(dg, n, world):
    """Meshes so small that a rank's owned elements and ghosts are nearly the
    whole mesh: padding takes the lowest-numbered free element (the fallback
    when no free neighbour of a ghost is left); no padding element shares a
    face with an owned element of its rank."""
    from paper_0901_1024_gb300.domain import build_plans
    verts, tets, mesh = _mesh(dg, n=n)
    plans = build_plans(mesh, tets, world)
    K, Np = mesh.K, mesh.Np
    vM, vP = mesh.connectivity()
    nb = {}
    for a, b in zip(vM // Np, vP // Np):
        if a != b:
            nb.setdefault(int(a), set()).add(int(b))
    fell_back = False
    for p in plans:
        mine = set(p.owned.tolist())
        needed = set().union(*(nb.get(k, set()) for k in p.owned)) - mine
        pads = [int(g) for g in p.ghosts if int(g) not in needed]
        for q in pads:
            assert not nb.get(q, set()) & mine
        near = set().union(*(nb.get(g, set()) for g in needed)) if needed else set()
        fell_back |= any(q not in near for q in pads)
        assert p.n_local % 4 == 0 or p.n_local == K
    assert fell_back


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_plans_cover_the_mesh_and_match_pairwise(dg, world):
    from paper_0901_1024_gb300.domain import build_plans
    verts, tets, mesh = _mesh(dg)
    plans = build_plans(mesh, tets, world)
    K, Np = mesh.K, mesh.Np
    owned = np.concatenate([p.owned for p in plans])
    assert sorted(owned) == list(range(K))
    vM, vP = mesh.connectivity()
    nb = {}
    for a, b in zip(vM // Np, vP // Np):
        nb.setdefault(int(a), set()).add(int(b))
    for p in plans:
        mine = set(p.owned.tolist())
        assert not mine & set(p.ghosts.tolist())
        assert np.array_equal(p.tets, tets[np.concatenate([p.owned, p.ghosts])])
        needed = set().union(*(nb[k] for k in p.owned)) - mine
        traced = {int(g) // Np for idx in p.recv.values() for g in
                  np.concatenate([p.owned, p.ghosts])[idx // Np] * Np}
        assert traced == needed <= set(p.ghosts.tolist())
        assert p.n_local % 4 == 0 or p.n_local == K       # padded for bulk copies
        assert len(p.ghosts) - len(needed) < 4
        local = np.concatenate([p.owned, p.ghosts])
        for q, idx in p.send.items():
            back = plans[q].recv[p.rank]
            glob_send = local[idx // Np] * Np + idx % Np
            ql = np.concatenate([plans[q].owned, plans[q].ghosts])
            glob_recv = ql[back // Np] * Np + back % Np
            assert np.array_equal(glob_send, glob_recv)
            assert np.all(idx // Np < p.n_owned) and np.all(back // Np >= plans[q].n_owned)
    if world == 1:
        assert len(plans[0].ghosts) == 0 and not plans[0].send


@pytest.mark.parametrize("world,tile", [(2, 4), (3, 8), (4, 4)])
def test_interior_first_plans(dg, world, tile):
    """With a tile, the first n_interior owned elements (a multiple of the tile)
    have no face to an element the rank does not own; the plans still cover the
    mesh and their exchanges still match (same checks as without a tile)."""
    from paper_0901_1024_gb300.domain import build_plans
    verts, tets, mesh = _mesh(dg)
    plans = build_plans(mesh, tets, world, tile=tile)
    K, Np = mesh.K, mesh.Np
    assert sorted(np.concatenate([p.owned for p in plans])) == list(range(K))
    vM, vP = mesh.connectivity()
    nb = {}
    for a, b in zip(vM // Np, vP // Np):
        nb.setdefault(int(a), set()).add(int(b))
    for p in plans:
        mine = set(p.owned.tolist())
        assert p.n_interior % tile == 0 and 0 < p.n_interior <= p.n_owned
        for k in p.owned[:p.n_interior]:
            assert nb[int(k)] <= mine
        for q, idx in p.send.items():
            assert np.all(idx // Np >= p.n_interior)       # only boundary elements send


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nsteps, q, tile=None):
    import torch.distributed as dist
    import __graft_entry__  # noqa: F401  (library already built by the parent)
    import paper_0901_1024_gb300 as dgp
    from paper_0901_1024_gb300.domain import (TraceExchange, build_plans, owned_energy, run_steps,
                                              run_steps_overlapped)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    verts, tets, mesh = _mesh(dgp)
    plan = build_plans(mesh, tets, world, tile=tile)[rank]
    om_glob = oracle.build_mesh(verts, tets, 2)
    om = oracle.build_mesh(verts, plan.tets, 2)
    a, b, _ = oracle.lserk4_coefficients()

    def stage(src, dst, res, i, dt):
        un, rn = oracle.stage_update(src.numpy(), res.numpy(), oracle.rhs(om, src.numpy()),
                                     a[i], b[i], dt)
        dst.copy_(torch.from_numpy(un))
        res.copy_(torch.from_numpy(rn))

    u0 = random_fields(mesh.K, mesh.Np, 17)
    local = np.concatenate([plan.owned, plan.ghosts])
    u = torch.from_numpy(np.ascontiguousarray(u0[:, local]))
    res, work = torch.zeros_like(u), torch.zeros_like(u)
    dt = oracle.cfl_dt(om_glob)

    def stage_range(src, dst, res, i, dt, k0, k1):
        # the whole local right-hand side, the update of elements [k0, k1) only
        # (the interior's runs before the ghosts are written: it must not read them)
        un, rn = oracle.stage_update(src.numpy(), res.numpy(), oracle.rhs(om, src.numpy()),
                                     a[i], b[i], dt)
        dst[:, k0:k1] = torch.from_numpy(un[:, k0:k1])
        res[:, k0:k1] = torch.from_numpy(rn[:, k0:k1])

    if tile:
        run_steps_overlapped(TraceExchange(dist, plan, "cpu"), stage_range, u, res, work, dt, nsteps)
    else:
        run_steps(TraceExchange(dist, plan, "cpu"), stage, u, res, work, dt, nsteps)
    e = owned_energy(dist, plan, lambda v: oracle.energy(om, v.numpy()), u)
    ug, _ = oracle.lserk4_run(om_glob, u0, dt, nsteps)
    err = float(np.abs(u.numpy()[:, :plan.n_owned] - ug[:, plan.owned]).max() / np.abs(ug).max())
    q.put((rank, err, e, oracle.energy(om_glob, ug), len(plan.ghosts), plan.n_interior))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,tile", [(2, None), (3, None), (4, 4), (3, 8)])
def test_ranks_follow_the_single_domain_oracle(dg, world, tile):
    """tile: the stage overlaps the trace exchange (interior tiles first); with
    4 ranks the blocks are uneven (162 = 3 x 41 + 39 tetrahedra)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, 2, q, tile))
             for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, e, e_ref, n_ghost, n_int in got:
        assert n_ghost > 0
        if tile:
            assert n_int > 0 and n_int % tile == 0
        assert err < 1e-13, (rank, err)
        assert abs(e - e_ref) <= 1e-12 * e_ref
