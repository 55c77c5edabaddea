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
        self.bytes = solve_bytes(self.K, self.Np)


class _Pack:
    """The live solves of one order, packed; fields in state = (u, res, work)."""

    def __init__(self, torch, N, solves, old, padding, impl, graphs, stream):
        self.N, self.solves = N, list(solves)
        meshes = [s.mesh for s in self.solves]
        Np = meshes[0].Np
        K = sum(m.K for m in meshes)
        npad = 0
        while (K + npad) * Np % 4:
            npad += 1
        self.mesh = Mesh.pack(meshes + [padding] * npad)
        self.mesh.set_stage_impl(impl)
        self.impl = impl
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

    hbm_budget : bytes of device memory the live solves may hold.
    batch      : pack the solves of one order into one stage launch; False
                 steps every live solve with its own launches (same arithmetic).
    graphs     : replay each pack's step from a CUDA graph.
    autotune   : pick each pack's stage implementation by timing; else `impl`.
    keep_fields: return every solve's final fields (host FP32) in its Result.
    """

    def __init__(self, hbm_budget: float = 150e9, batch: bool = True, graphs: bool = True,
                 autotune: bool = True, impl: int = Mesh.STAGE_AUTO, keep_fields: bool = True):
        import torch
        self.torch = torch
        self.budget, self.batch, self.graphs = hbm_budget, batch, graphs
        self.autotune, self.impl, self.keep = autotune, impl, keep_fields
        self.stream = torch.cuda.Stream()
        self._padding = {}
        self._tuned = {}

    # ---- stage implementation per (N, K) ---------------------------------
    def _pad_mesh(self, N):
        if N not in self._padding:
            v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64)
            self._padding[N] = Mesh(v, np.array([[0, 1, 2, 3]]), N)
        return self._padding[N]

    def _choose_impl(self, N, solves):
        if not self.autotune:
            return self.impl
        if N > 4:
            return Mesh.STAGE_FP32
        K = sum(s.K for s in solves)
        key = (N, int(round(math.log2(max(K, 1)) * 2)))
        if key not in self._tuned:
            torch = self.torch
            times = {}
            for impl in (Mesh.STAGE_TC, Mesh.STAGE_FP32):
                p = _Pack(torch, N, solves, None, self._pad_mesh(N), impl, False, self.stream)
                for _ in range(2):                       # warm-up
                    p.step()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                for _ in range(3):
                    p.step()
                e1.record(self.stream)
                e1.synchronize()
                times[impl] = e0.elapsed_time(e1)
            self._tuned[key] = min(times, key=times.get)
        return self._tuned[key]

    # ---- the loop ----------------------------------------------------------
    def run(self, requests):
        torch = self.torch
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        live, packs, results = [], {}, []
        held = 0
        t0 = time.perf_counter()
        dirty = set()
        while pending or live:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                req = pending[0]
                need = solve_bytes(len(req.tets), (req.N + 1) * (req.N + 2) * (req.N + 3) // 6)
                if live and held + need > self.budget:
                    break                                # first come, first served
                pending.pop(0)
                s = _Live(req, time.perf_counter() - t0)
                live.append(s)
                held += s.bytes
                dirty.add(req.N)
            if not live:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
                continue
            with torch.cuda.stream(self.stream):
                for N in sorted(dirty):
                    members = [s for s in live if s.req.N == N]
                    old = packs.pop(N, None)
                    carry = {}
                    for op in (old if isinstance(old, list) else [old] if old else []):
                        st = op.state()
                        for s in op.solves:
                            if s in members:
                                sl = slice(s.offset, s.offset + s.K)
                                carry[id(s)] = (st[:, sl].clone(), op.res[:, sl].clone())
                    if not members:
                        continue
                    groups = [members] if self.batch else [[s] for s in members]
                    built = []
                    for g in groups:
                        impl = self._choose_impl(N, g)
                        built.append(_Pack(torch, N, g, carry, self._pad_mesh(N), impl,
                                           self.graphs, self.stream))
                    packs[N] = built[0] if self.batch else built
                dirty.clear()
                all_packs = [p for v in packs.values() for p in (v if isinstance(v, list) else [v])]
                for p in all_packs:
                    p.step()
                finished = []
                for p in all_packs:
                    for s in p.solves:
                        s.done += 1
                        if s.done == s.steps:
                            finished.append((p, s))
                for p, s in finished:
                    st = p.state()
                    sl = slice(s.offset, s.offset + s.K)
                    tmp = torch.zeros_like(st)
                    tmp[:, sl].copy_(st[:, sl])
                    energy = p.mesh.energy(tmp, stream=self.stream)
                    fields = st[:, sl].cpu().numpy() if self.keep else None
                    results.append(Result(s.req.rid, s.K, s.req.N, s.steps, s.dt, energy, fields,
                                          s.req.arrival, s.admitted, time.perf_counter() - t0))
                    live.remove(s)
                    held -= s.bytes
                    dirty.add(s.req.N)
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
