"""Serving many Maxwell solves on one GPU with continuous batching.

A request is a mesh (vertices, tetrahedra), an order N, an end time T and
initial fields.  It is admitted as soon as it has arrived and the HBM budget
holds its fields; admitted solves stay on the device until they finish.  Every
iteration advances all live solves by one LSERK4 step together: the solves of
one order share a packed element table (`dg_mesh_pack`: their meshes side by
side as separate components) and one fused stage launch per RK stage, every
element stepping with its own solve's time step (`dg_rk_stage_elem`).  A
finished solve leaves the pack (its fields are copied out and its energy is
reduced on the device); the next iteration's packs include whatever arrived
meanwhile.  Optionally a step of a pack is captured in a CUDA graph and
replayed, and the stage implementation of a pack (tensor cores or FP32 CUDA
cores) is picked per (N, K) by timing both.

Every solve's result is the same alone and in the mix: a packed element
performs exactly its own solve's arithmetic (the stage kernels treat elements
independently apart from their face neighbours, which belong to the same
solve), so the fields agree bit for bit with a lone run on the same stage
implementation.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import Mesh

_RK_STAGES = 5


@dataclass
class Request:
    rid: int
    verts: np.ndarray
    tets: np.ndarray
    N: int
    T: float                       # end time; dt = T / ceil(T / dt_cfl)
    init: object                   # init(xyz[3][K][Np]) -> fields [6][K][Np]
    arrival: float = 0.0           # seconds after the start of the run


@dataclass
class Result:
    rid: int
    K: int
    N: int
    steps: int
    dt: float
    energy: float
    fields: np.ndarray | None
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self):
        return self.finished - self.arrival


def solve_bytes(K: int, Np: int) -> int:
    """Device bytes one solve holds in a pack: u, res and the ping-pong copy
    (FP32 [6][K][Np] each), its time steps and its share of the packed
    geometry (records, tiled tensor-core blocks, per-node neighbour bytes)."""
    return 3 * 24 * K * Np + 4 * K + 128 * K + 180 * K + 4 * K * Np


def carry_bytes(K: int, Np: int) -> int:
    """Transient device bytes of one solve while its pack is rebuilt: the copy
    of its u and res (FP32 [6][K][Np] each) carried into the new pack."""
    return 2 * 24 * K * Np


class _Live:
    def __init__(self, req: Request, now: float):
        self.req = req
        self.mesh = Mesh(req.verts, req.tets, req.N)
        self.K, self.Np = self.mesh.K, self.mesh.Np
        self.steps = max(1, math.ceil(req.T / self.mesh.dt_cfl - 1e-12))
        self.dt = req.T / self.steps
        self.done = 0
        self.admitted = now
        self.u0 = np.ascontiguousarray(req.init(self.mesh.nodes()), dtype=np.float32)
        self.offset = 0
        self.finished = False
        self.bytes = solve_bytes(self.K, self.Np)
        self.carry = carry_bytes(self.K, self.Np)


class _Pack:
    """The live solves of one order, packed; fields in state = (u, res, work)."""

    def __init__(self, torch, N, solves, old, padding, impl, graphs, stream, shape=0):
        self.N, self.solves = N, list(solves)
        self.alive = len(self.solves)
        self.built_at = 0
        meshes = [s.mesh for s in self.solves]
        Np = meshes[0].Np
        K = sum(m.K for m in meshes)
        npad = 0
        while (K + npad) * Np % 4:
            npad += 1
        self.mesh = Mesh.pack(meshes + [padding] * npad)
        self.mesh.set_stage_impl(impl)
        self.mesh.set_stage_shape(shape)
        self.impl, self.shape = impl, shape
        self.K, self.Np = self.mesh.K, Np
        dev = "cuda"
        shape = (6, self.K, Np)
        self.u = torch.zeros(shape, device=dev)
        self.res = torch.zeros(shape, device=dev)
        self.work = torch.empty(shape, device=dev)
        dts = np.ones(self.K, np.float32)
        off = 0
        for s in self.solves:
            sl = slice(off, off + s.K)
            src = old.get(id(s)) if old else None
            if src is not None:
                self.u[:, sl].copy_(src[0])
                self.res[:, sl].copy_(src[1])
            else:
                self.u[:, sl].copy_(torch.from_numpy(s.u0).to(dev, non_blocking=True))
            s.offset = off
            dts[sl] = np.float32(s.dt)
            off += s.K
        self.dt_elem = torch.from_numpy(dts).to(dev)
        self.stream = stream
        self.graphs = None
        self.parity = 0
        if graphs:
            self._capture(torch)

    def _stages(self, src, dst):
        for i in range(_RK_STAGES):
            self.mesh.rk_stage_elem(src, dst, self.res, i, self.dt_elem, stream=self.stream)
            src, dst = dst, src

    def _capture(self, torch):
        # warm-up outside capture (device buffers and kernel attributes are set
        # up on first use), on scratch copies so that the state is untouched
        u, r = self.u.clone(), self.res.clone()
        w = torch.empty_like(u)
        for i in range(_RK_STAGES):
            self.mesh.rk_stage_elem(u, w, r, i, self.dt_elem, stream=self.stream)
            u, w = w, u
        torch.cuda.current_stream().wait_stream(self.stream)
        self.graphs = []
        for src, dst in ((self.u, self.work), (self.work, self.u)):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                self._stages(src, dst)
            self.graphs.append(g)

    def state(self):
        return self.u if self.parity == 0 else self.work

    def set_parity(self, parity):
        """Put the state in the buffer of `parity` (0: u, 1: work) by swapping the
        two tensors, so packs stepped together share one ping-pong parity."""
        if parity != self.parity:
            self.u, self.work = self.work, self.u
            self.parity = parity

    def buffers(self):
        """(source, destination) of the next stage."""
        return (self.u, self.work) if self.parity == 0 else (self.work, self.u)

    def release(self):
        """Drop the pack's graphs, fields and packed mesh (device memory goes
        back to the caching allocator at once, before the next pack is built)."""
        self.graphs = None
        self.u = self.res = self.work = self.dt_elem = None
        if self.mesh is not None:
            self.mesh.close()
            self.mesh = None

    def step(self):
        if self.graphs:
            self.graphs[self.parity].replay()
        elif self.parity == 0:
            self._stages(self.u, self.work)
        else:
            self._stages(self.work, self.u)
        self.parity ^= 1


class Server:
    """Continuous-batching request loop (see the module docstring).

    The autotuner's choices (stage implementation per order, decade of K and
    device) are kept for the life of the process, shared by every Server.

    hbm_budget : bytes of device memory the live solves may hold, including
                 the transient copies of a pack rebuild: a solve is admitted
                 only while the bytes of every admitted solve (solve_bytes)
                 plus the carried copies of all of them (carry_bytes) fit, which
                 bounds the peak of any rebuild (the old pack is released
                 before tuning or allocating the new one).  stats["model_peak"]
                 is the largest total of that accounting during the run.
    batch      : pack the solves of one order into one stage launch; False
                 steps every live solve with its own launches (same arithmetic).
    graphs     : replay each pack's step from a CUDA graph.
    autotune   : pick each pack's stage implementation by timing; else `impl`.
    keep_fields: return every solve's final fields (host FP32) in its Result.
    rebuild_every: steps a pack runs before waiting solves may join it.
    dead_fraction: share of a pack's elements held by finished solves (which
                 keep stepping, unread) at which an aged pack is rebuilt
                 without them.  On GB300, 200-request stream: 1.0 (only when
                 every solve is done) 2.12 solves/s, 0.5 3.19, 0.3 3.49, 0.15
                 3.62 (64 pack builds, 5.6 s of host time).
    mixed      : (with batch) advance all packs, of every order, with one
                 dg_rk_stage_multi call per RK stage -- one shared persistent
                 launch for orders 1..4 and one for 5, 6 -- its CTAs split by
                 the tuned cost of a tile of each pack; graphs capture the five
                 shared stages of the current set of packs.  Off by default:
                 on GB300 different orders side by side in one grid measured
                 12 % slower than one launch per order (packs of one order
                 gain 10 %), see the benchmark's serve mode.
    """

    def __init__(self, hbm_budget: float = 150e9, batch: bool = True, graphs: bool = True,
                 autotune: bool = True, impl: int = Mesh.STAGE_AUTO, keep_fields: bool = True,
                 rebuild_every: int = 32, mixed: bool = False, dead_fraction: float = 0.15):
        import torch
        self.torch = torch
        self.budget, self.batch, self.graphs = hbm_budget, batch, graphs
        self.mixed = mixed and batch
        self._gparity = 0              # ping-pong parity shared by the packs (mixed)
        self._gcache = {}              # (pack ids, parity) -> captured graph, or None: seen once
        self.rebuild_every = rebuild_every
        self.dead_fraction = dead_fraction
        self.autotune, self.impl, self.keep = autotune, impl, keep_fields
        self.stream = torch.cuda.Stream()
        self._padding = {}
        # host seconds per phase of the last run: admitting (mesh setup),
        # packing (pack build, device setup, graph capture, tuning), stepping,
        # retiring (energy, copy-out); and how many packs were built
        self.stats = {}

    _tuned = {}                        # (device, N, decade of K) -> (stage implementation, tile shape)
    _cost = {}                         # (device, N, decade of K) -> ms per tile on one SM

    # ---- stage implementation per (N, K) ---------------------------------
    def _pad_mesh(self, N):
        if N not in self._padding:
            v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64)
            self._padding[N] = Mesh(v, np.array([[0, 1, 2, 3]]), N)
        return self._padding[N]

    def _tune_key(self, N, solves):
        K = sum(s.K for s in solves)
        return (self.torch.cuda.current_device(), N,
                min(3, int(math.log10(max(K, 1))) - 2))     # <1e3, <1e4, <1e5, more

    def _time_impl(self, N, solves, impl, shape=0):
        """Milliseconds of 3 steps of a scratch pack of `solves` on `impl` with
        tile shape `shape`; the pack is released before returning."""
        torch = self.torch
        self._charge(sum(s.bytes for s in solves))
        p = _Pack(torch, N, solves, None, self._pad_mesh(N), impl, False, self.stream, shape)
        for _ in range(2):                       # warm-up
            p.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(3):
            p.step()
        e1.record(self.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if impl == Mesh.STAGE_TC and N <= 7:
            # one tile's cost on one SM: stage time x CTAs in use / tiles
            tiles = -(-p.K // (20 if N <= 4 else 8))
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            self._cost[self._tune_key(N, solves)] = ms / 15 * min(tiles, sms) / tiles
        p.release()
        self._charge(-sum(s.bytes for s in solves))
        return ms

    def _choose_impl(self, N, solves):
        """(stage implementation, FP32 tile shape) of a pack: without autotuning
        the server's `impl` and the default shape; with it, the fastest of the
        tensor-core stage (orders <= 7) and the FP32 stage in each tile shape,
        timed on a scratch pack once per (device, order, decade of K)."""
        if not self.autotune:
            return self.impl, 0
        key = self._tune_key(N, solves)
        if key not in self._tuned:
            cands = [(Mesh.STAGE_FP32, 0), (Mesh.STAGE_FP32, 1)]
            if N <= 7:
                cands.insert(0, (Mesh.STAGE_TC, 0))
            times = {c: self._time_impl(N, solves, *c) for c in cands}
            self._tuned[key] = min(times, key=times.get)
        return self._tuned[key]

    @classmethod
    def tuned_choices(cls):
        """The autotuner's picks so far: "device/N/decade" -> "tc" or "fp32/shape"."""
        names = {Mesh.STAGE_TC: "tc", Mesh.STAGE_FP32: "fp32", Mesh.STAGE_AUTO: "auto"}
        return {f"{d}/{N}/{k}": (names[i] if i == Mesh.STAGE_TC else f"{names[i]}/{sh}")
                for (d, N, k), (i, sh) in sorted(cls._tuned.items())}

    # ---- device-memory accounting (a model of what the loop allocates) ------
    def _charge(self, nbytes):
        m = self.stats
        m["model_now"] = m.get("model_now", 0) + nbytes
        m["model_peak"] = max(m.get("model_peak", 0), m["model_now"])

    # ---- pack rebuilds -------------------------------------------------------
    def _carry(self, old, members):
        """Copies of (u, res) of the old pack's solves that go on in `members`."""
        state = old.state()
        carry = {}
        for s in old.solves:
            if s in members:
                sl = slice(s.offset, s.offset + s.K)
                carry[id(s)] = (state[:, sl].clone(), old.res[:, sl].clone())
                self._charge(s.carry)
        return carry

    def _release(self, pack):
        pack.release()
        self._charge(-sum(s.bytes for s in pack.solves))

    def _new_pack(self, N, members, carry, impl):
        self._charge(sum(s.bytes for s in members))
        impl, shape = impl
        p = _Pack(self.torch, N, members, carry, self._pad_mesh(N), impl,
                  self.graphs and not self.mixed, self.stream, shape)
        if self.mixed:
            p.set_parity(self._gparity)
            p.cost = self._cost.get(self._tune_key(N, members))
        return p

    # ---- all packs in shared launches ------------------------------------------
    def _stages_mixed(self, packs, par):
        meshes = [p.mesh for p in packs]
        bufs = [p.buffers() for p in packs]
        src, dst = [b[0] for b in bufs], [b[1] for b in bufs]
        res = [p.res for p in packs]
        dts = [p.dt_elem for p in packs]
        costs = None
        if all(getattr(p, "cost", None) for p in packs):
            costs = [p.cost for p in packs]
        for i in range(_RK_STAGES):
            Mesh.rk_stage_multi(meshes, src, dst, res, i, dt_elem=dts, tile_cost=costs,
                                stream=self.stream)
            src, dst = dst, src

    def _step_mixed(self, packs):
        """One LSERK4 step of every pack: five dg_rk_stage_multi calls, replayed
        from a graph once the same set of packs is stepped a second time."""
        torch = self.torch
        key = (tuple(id(p) for p in packs), self._gparity)
        g = self._gcache.get(key, False)
        if g is False or not self.graphs:
            if self.graphs:
                # a new set of packs: forget the graphs of earlier sets
                self._gcache = {k: v for k, v in self._gcache.items() if k[0] == key[0]}
                self._gcache[key] = None
            self._stages_mixed(packs, self._gparity)
        elif g is None:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                self._stages_mixed(packs, self._gparity)
            self._gcache[key] = g
            g.replay()
        else:
            g.replay()
        for p in packs:
            p.parity ^= 1
        self._gparity ^= 1

    def _build(self, N, members, old, st):
        """A pack of `members` (live solves of order N), continuing from the
        old pack's state for those that were in it.  The carried copies are
        taken first, then the old pack is released, then the implementation is
        tuned (scratch packs, one at a time) and the new pack allocated: the
        peak is the admitted solves' bytes plus the carried copies."""
        carry = {}
        if old is not None:
            carry = self._carry(old, members)
            self._release(old)
        impl = self._choose_impl(N, members)
        p = self._new_pack(N, members, carry, impl)
        for s in members:
            if id(s) in carry:
                self._charge(-s.carry)
        carry.clear()
        p.built_at = st["iterations"]
        st["packs_built"] += 1
        return p

    def _admit(self, req, now):
        return _Live(req, now)

    def _retire(self, p, s, now):
        state = p.state()
        sl = slice(s.offset, s.offset + s.K)
        energy = p.mesh.energy_range(state, s.offset, s.offset + s.K, stream=self.stream)
        fields = state[:, sl].cpu().numpy() if self.keep else None
        return Result(s.req.rid, s.K, s.req.N, s.steps, s.dt, energy, fields, s.req.arrival,
                      s.admitted, now())

    def _device_context(self):
        return self.torch.cuda.stream(self.stream)

    def _dead_weight(self, pack) -> bool:
        """Finished solves hold at least `dead_fraction` of the pack's elements
        (they keep stepping, unread, until a rebuild drops them)."""
        dead = sum(s.K for s in pack.solves if s.finished)
        return dead > 0 and dead >= self.dead_fraction * sum(s.K for s in pack.solves)

    def run(self, requests, max_iterations: int | None = None):
        """Serve `requests` (arriving at their `arrival` times) to completion;
        returns their Results in rid order.

        A pack of order N is rebuilt when solves of that order wait to join it
        and it has run at least `rebuild_every` steps since it was built (at once
        when there is no pack), or, after as many steps, when finished solves
        hold `dead_fraction` of its elements.  A
        finished solve's fields and energy are taken at its last step; its
        elements keep stepping, unread, until its pack is rebuilt; a pack with
        no unfinished solve is dropped at the start of the next iteration.
        `max_iterations` bounds the loop (RuntimeError when exceeded)."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        waiting, packs, results = [], [], []
        held = 0                      # bytes of every admitted solve not yet released
        reserve = 0                   # their carried copies during a rebuild
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        st = self.stats = dict(admit_s=0.0, pack_s=0.0, step_s=0.0, retire_s=0.0, packs_built=0,
                               iterations=0, model_now=0, model_peak=0)
        every = self.rebuild_every if self.batch else 0
        while pending or waiting or packs:
            if max_iterations is not None and st["iterations"] > max_iterations:
                raise RuntimeError("serve loop exceeded max_iterations")
            for p in [p for p in packs if not p.alive]:     # finished packs free their memory
                packs.remove(p)
                self._release(p)
                held -= sum(s.bytes for s in p.solves)
                reserve -= sum(s.carry for s in p.solves)
            while pending and pending[0].arrival <= now():
                req = pending[0]
                Np = (req.N + 1) * (req.N + 2) * (req.N + 3) // 6
                need = solve_bytes(len(req.tets), Np) + carry_bytes(len(req.tets), Np)
                if held > 0 and held + reserve + need > self.budget:
                    break                                # first come, first served
                pending.pop(0)
                ta = time.perf_counter()
                s = self._admit(req, now())
                st["admit_s"] += time.perf_counter() - ta
                waiting.append(s)
                held += s.bytes
                reserve += s.carry
            if not waiting and not packs:
                if not pending:
                    break                                # the last packs just finished
                time.sleep(max(0.0, pending[0].arrival - now()))
                continue
            with self._device_context():
                tp = time.perf_counter()
                it = st["iterations"]
                if self.batch:
                    for N in sorted({s.req.N for s in waiting} | {p.N for p in packs}):
                        old = next((p for p in packs if p.N == N), None)
                        new = [s for s in waiting if s.req.N == N]
                        aged = old is not None and it - old.built_at >= every
                        if old is not None and not new and not (aged and self._dead_weight(old)):
                            continue
                        if old is not None and new and not aged:
                            continue
                        keep = [s for s in old.solves if not s.finished] if old is not None else []
                        if old is not None:
                            packs.remove(old)
                        packs.append(self._build(N, keep + new, old, st))
                        if old is not None:                  # released by the rebuild
                            held -= sum(s.bytes for s in old.solves if s.finished)
                            reserve -= sum(s.carry for s in old.solves if s.finished)
                        waiting = [s for s in waiting if s.req.N != N]
                else:
                    for s in waiting:
                        packs.append(self._build(s.req.N, [s], None, st))
                    waiting = []
                ts = time.perf_counter()
                st["pack_s"] += ts - tp
                if self.mixed and packs:
                    self._step_mixed(packs)
                else:
                    for p in packs:
                        p.step()
                st["iterations"] += 1
                tr = time.perf_counter()
                st["step_s"] += tr - ts
                for p in packs:
                    for s in p.solves:
                        if s.finished:
                            continue
                        s.done += 1
                        if s.done < s.steps:
                            continue
                        results.append(self._retire(p, s, now))
                        s.finished = True
                        p.alive -= 1
                st["retire_s"] += time.perf_counter() - tr
        return sorted(results, key=lambda r: r.rid)


def run_alone(req: Request, impl: int = Mesh.STAGE_AUTO):
    """Reference: one solve by itself with scalar-step stages (dg_rk_stage);
    returns (fields, energy, steps, dt)."""
    import torch
    s = _Live(req, 0.0)
    s.mesh.set_stage_impl(impl)
    u = torch.from_numpy(s.u0).cuda()
    w, r = torch.empty_like(u), torch.zeros_like(u)
    for _ in range(s.steps):
        for i in range(_RK_STAGES):
            s.mesh.rk_stage(u, w, r, i, float(np.float32(s.dt)))
            u, w = w, u
    return u.cpu().numpy(), s.mesh.energy(u), s.steps, s.dt
