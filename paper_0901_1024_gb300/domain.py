"""Element domain decomposition of one mesh over several ranks.

The elements are numbered by the greedy partition of Section 5.2 (Algorithm 2,
`dg_partition_order`) in blocks of ceil(K / ranks); rank r owns block r, a
face-connected piece of the mesh.  Its local mesh is its owned elements (in
that numbering) followed by one layer of ghost elements, the face neighbours it
does not own (plus up to three zero padding elements, so that the tensor-core
stage's bulk-copy alignment holds).  A ghost's other faces are walls in the
local mesh, so the ordinary single-mesh kernels run unchanged on it.

Once per RK stage, before the flux step, every rank sends the face traces
(6 fields x Nfp face nodes) of its elements across each cut face to the rank
that holds them as ghosts; the receiver zeroes its ghost elements and writes
the traces into their face nodes.  With a stage tile given, a rank's owned
elements are numbered interior first (no face to a ghost), so the stage can
run on the whole tiles of the interior while the traces are in flight
(`run_steps_overlapped`: sends and receives posted, interior tiles launched,
traces written, then the remaining tiles).  Owned elements then read exactly the face
values a single-domain run would, and their results are identical; the ghost
rows' results are discarded.  Communication is point-to-point only
(torch.distributed batched send/recv: gloo on CPU, NCCL on GPU, no
multicast); the energy is the only reduction (a sum over ranks of the owned
elements' energies).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class RankPlan:
    """What one rank holds and exchanges.  Node lists are flat indices into a
    field's [K_local * Np] block; send[p] and the peer's recv[rank] list the
    same nodes in the same order."""
    rank: int
    world: int
    Np: int
    owned: np.ndarray             # global element ids, local positions 0..n_owned-1
                                  # (interior first when the plan has a tile)
    ghosts: np.ndarray            # global element ids, local positions n_owned.. (traced
                                  # ghosts first, then zero padding elements)
    tets: np.ndarray              # local mesh: tets of owned then ghost elements
    send: dict = field(default_factory=dict)   # peer -> local flat node indices
    recv: dict = field(default_factory=dict)   # peer -> local flat node indices
    n_interior: int = 0           # owned elements [0, n_interior): whole tiles with no
                                  # face to a ghost (0 without a tile)

    @property
    def n_owned(self):
        return len(self.owned)

    @property
    def n_local(self):
        return len(self.owned) + len(self.ghosts)


def build_plans(mesh, tets, world: int, align: int = 4, tile: int | None = None):
    """Plans of all `world` ranks for the global mesh `mesh` (a Mesh built from
    `tets`; only its host-side connectivity is used).

    Each local mesh is padded with extra ghost elements (face neighbours of its
    ghosts where possible) until its element count is a multiple of `align`:
    the tensor-core stage moves tiles with bulk copies and needs K * Np to be a
    multiple of 4.  Padding elements receive no traces and stay zero.

    tile: the stage kernel's tetrahedra per tile (Mesh.stage_tile); then each
    rank's owned elements are numbered interior first and n_interior is the
    largest multiple of `tile` not above the interior count."""
    tets = np.asarray(tets)
    K, Np = mesh.K, mesh.Np
    if world < 1 or world > K:
        raise ValueError("need 1 <= world <= K")
    perm = mesh.partition_order(-(-K // world))
    block = -(-K // world)
    owner = np.empty(K, np.int64)
    owner[perm] = np.arange(K) // block
    vM, vP = mesh.connectivity()
    kM, kP = vM // Np, vP // Np
    cut = owner[kM] != owner[kP]
    # (receiving rank, global node of the neighbour) for every face node of a cut face
    need = {}
    for r_recv, g in zip(owner[kM[cut]], vP[cut]):
        need.setdefault(int(r_recv), set()).add(int(g))
    plans = []
    local_pos = []
    nbr = {}
    for a, b in zip(kM, kP):
        if a != b:
            nbr.setdefault(int(a), set()).add(int(b))
    for r in range(world):
        owned = perm[r * block:(r + 1) * block]
        n_interior = 0
        if tile:
            mine = set(owned.tolist())
            inner = np.array([not (nbr.get(int(k), set()) - mine) for k in owned], bool)
            owned = np.concatenate([owned[inner], owned[~inner]])
            n_interior = int(inner.sum()) // tile * tile
        ghost_set = {int(g) // Np for g in need.get(r, ())}
        local = set(owned.tolist()) | ghost_set
        pad = []
        while align > 1 and (len(local) + len(pad)) % align and len(local) + len(pad) < K:
            taken = local | set(pad)
            cand = sorted(set().union(*(nbr.get(g, set()) for g in sorted(ghost_set | set(pad))))
                          - taken) if ghost_set or pad else []
            pad.append(cand[0] if cand else min(set(range(K)) - taken))
        # every face neighbour of an owned element is owned or a traced ghost, so
        # a padding element (taken from outside both) never touches an owned
        # element: owned elements read no untraced (zero) values
        owned_set = set(owned.tolist())
        assert all(not (nbr.get(q, set()) & owned_set) for q in pad), "pad next to an owned element"
        ghosts = np.array(sorted(ghost_set) + pad, dtype=np.int64)
        plan = RankPlan(r, world, Np, owned, ghosts, tets[np.concatenate([owned, ghosts])],
                        n_interior=n_interior)
        pos = np.full(K, -1, np.int64)
        pos[plan.owned] = np.arange(plan.n_owned)
        pos[plan.ghosts] = plan.n_owned + np.arange(len(plan.ghosts))
        plans.append(plan)
        local_pos.append(pos)
    for r_recv in range(world):
        by_sender = {}
        for g in sorted(need.get(r_recv, ())):
            by_sender.setdefault(int(owner[g // Np]), []).append(g)
        for r_send, nodes in by_sender.items():
            nodes = np.array(nodes, dtype=np.int64)
            k, i = nodes // Np, nodes % Np
            plans[r_send].send[r_recv] = local_pos[r_send][k] * Np + i
            plans[r_recv].recv[r_send] = local_pos[r_recv][k] * Np + i
    return plans


class TraceExchange:
    """Per-stage exchange of cut-face traces for one rank's field tensor
    u[6][K_local][Np] (any dtype, on the device the process group uses)."""

    def __init__(self, dist, plan: RankPlan, device):
        import torch
        self.dist, self.plan = dist, plan
        self.peers = sorted(set(plan.send) | set(plan.recv))
        self.send = {p: torch.as_tensor(plan.send[p], device=device) for p in plan.send}
        self.recv = {p: torch.as_tensor(plan.recv[p], device=device) for p in plan.recv}

    def __call__(self, u):
        self.finish(u, self.start(u))

    def start(self, u):
        """Post the sends of u's cut-face traces and the receives of the ghosts'
        (reads owned elements only); returns the pending exchange."""
        import torch
        flat = u.view(6, -1)
        ops, bufs = [], {}
        for p in self.peers:
            if p in self.send:
                ops.append(self.dist.P2POp(self.dist.isend,
                                           flat.index_select(1, self.send[p]).contiguous(), p))
            if p in self.recv:
                bufs[p] = torch.empty((6, len(self.recv[p])), dtype=u.dtype, device=u.device)
                ops.append(self.dist.P2POp(self.dist.irecv, bufs[p], p))
        reqs = self.dist.batch_isend_irecv(ops) if ops else []
        return reqs, bufs

    def finish(self, u, pending):
        """Wait for the exchange, zero the ghost elements and write the traces."""
        reqs, bufs = pending
        for req in reqs:
            req.wait()
        u[:, self.plan.n_owned:, :] = 0
        flat = u.view(6, -1)
        for p, b in bufs.items():
            flat.index_copy_(1, self.recv[p], b)


def run_steps(exchange, stage, u, res, work, dt: float, nsteps: int):
    """nsteps LSERK4 steps of one rank: before each of the 5 stages the ghost
    traces are refreshed, then stage(u_in, u_out, res, i, dt) runs (for the
    CUDA path `Mesh.rk_stage`).  `work` is a buffer like u; the state ends in
    u.  Ghost rows of res are zeroed with the ghosts so they stay finite."""
    n0 = exchange.plan.n_owned
    src, dst = u, work
    for _ in range(nsteps):
        for i in range(5):
            exchange(src)
            res[:, n0:, :] = 0
            stage(src, dst, res, i, dt)
            src, dst = dst, src
    if src is not u:
        u.copy_(src)
    return u


def run_steps_overlapped(exchange, stage_range, u, res, work, dt: float, nsteps: int):
    """As run_steps, with each stage split in two: the exchange is posted, the
    stage runs on the interior tiles [0, n_interior) (no face to a ghost, so it
    reads no ghost value), the traces are written, then the stage runs on
    [n_interior, n_local).  stage_range(u_in, u_out, res, i, dt, k0, k1) runs
    one stage on elements [k0, k1) (for the CUDA path Mesh.rk_stage_range).
    Every element gets the same result as with run_steps."""
    plan = exchange.plan
    n0, n_int, n_loc = plan.n_owned, plan.n_interior, plan.n_local
    src, dst = u, work
    for _ in range(nsteps):
        for i in range(5):
            pending = exchange.start(src)
            if n_int:
                stage_range(src, dst, res, i, dt, 0, n_int)
            exchange.finish(src, pending)
            res[:, n0:, :] = 0
            stage_range(src, dst, res, i, dt, n_int, n_loc)
            src, dst = dst, src
    if src is not u:
        u.copy_(src)
    return u


def owned_energy(dist, plan: RankPlan, energy_fn, u):
    """Sum over ranks of energy_fn(u with ghost rows zeroed)."""
    import torch
    v = u.clone()
    v[:, plan.n_owned:, :] = 0
    e = torch.tensor([float(energy_fn(v))], dtype=torch.float64, device=u.device)
    if dist is not None:
        dist.all_reduce(e)
    return float(e.item())
