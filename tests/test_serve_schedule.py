"""Scheduling logic of the serving loop (serve.Server.run) on the CPU: the
real loop with fake solves and packs (no GPU), bounded by max_iterations so
that a scheduling bug fails instead of hanging.  Checks completion, exact step
counts, budget-limited one-at-a-time admission, rebuild pacing and per-solve
packs."""
import contextlib

import numpy as np
import pytest

from paper_0901_1024_gb300 import serve


class FakeLive:
    def __init__(self, req, now):
        self.req, self.K, self.steps, self.dt = req, len(req.tets), int(req.T), 1.0
        self.done, self.admitted, self.offset, self.finished = 0, now, 0, False
        self.stepped = 0
        Np = (req.N + 1) * (req.N + 2) * (req.N + 3) // 6
        self.bytes = serve.solve_bytes(self.K, Np)
        self.carry = serve.carry_bytes(self.K, Np)


class FakePack:
    def __init__(self, N, solves, built_at):
        self.N, self.solves, self.alive, self.built_at = N, list(solves), len(solves), built_at

    def step(self):
        for s in self.solves:
            if not s.finished:
                s.stepped += 1

    def state(self):
        return None

    def release(self):
        self.released = True


class FakeServer(serve.Server):
    def __init__(self, budget=1e18, batch=True, rebuild_every=4, dead_fraction=0.5):
        self.budget, self.batch, self.rebuild_every = budget, batch, rebuild_every
        self.dead_fraction = dead_fraction
        self.graphs, self.autotune, self.keep, self.mixed = False, False, False, False
        self.stats, self.live_log = {}, []

    def _admit(self, req, now):
        return FakeLive(req, now)

    def _build(self, N, members, old, st):
        assert members and all(s.req.N == N and not s.finished for s in members)
        st["packs_built"] += 1
        self.live_log.append(len(members))
        return FakePack(N, members, st["iterations"])

    def _release(self, pack):
        pack.release()

    def _retire(self, p, s, now):
        assert s.stepped == s.steps
        return serve.Result(s.req.rid, s.K, s.req.N, s.steps, s.dt, 0.0, None, s.req.arrival,
                            s.admitted, now())

    def _device_context(self):
        return contextlib.nullcontext()


def requests(count=20, seed=0, spread=0.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for rid in range(count):
        K = int(rng.integers(6, 60))
        out.append(serve.Request(rid, None, np.zeros((K, 4)), int(rng.integers(1, 4)),
                                 float(rng.integers(1, 15)), None, arrival=spread * rid))
    return out


@pytest.mark.parametrize("batch,every", [(True, 1), (True, 4), (True, 50), (False, 0)])
def test_every_solve_finishes_with_its_step_count(batch, every):
    reqs = requests()
    res = FakeServer(batch=batch, rebuild_every=every).run(reqs, max_iterations=10_000)
    assert [r.rid for r in res] == list(range(len(reqs)))
    assert all(r.steps == int(q.T) for r, q in zip(res, reqs))


def test_small_budget_admits_one_solve_at_a_time():
    srv = FakeServer(budget=1.0)
    res = sorted(srv.run(requests(8), max_iterations=10_000), key=lambda r: r.admitted)
    for a, b in zip(res, res[1:]):
        assert b.admitted >= a.finished
    assert max(srv.live_log) == 1


def test_arrivals_in_the_future_are_waited_for():
    res = FakeServer().run(requests(5, spread=0.002), max_iterations=10_000)
    assert all(r.admitted >= r.arrival for r in res)


def test_rebuilds_are_paced_and_unbatched_packs_are_per_solve():
    paced = FakeServer(rebuild_every=8)
    paced.run(requests(30), max_iterations=10_000)
    eager = FakeServer(rebuild_every=1)
    eager.run(requests(30), max_iterations=10_000)
    assert paced.stats["packs_built"] <= eager.stats["packs_built"]
    single = FakeServer(batch=False)
    single.run(requests(12), max_iterations=10_000)
    assert single.stats["packs_built"] == 12 and max(single.live_log) == 1


def test_loop_bound_raises():
    with pytest.raises(RuntimeError):
        FakeServer().run(requests(3), max_iterations=1)


class LedgerServer(FakeServer):
    """The real rebuild sequence (Server._build: carry, release the old pack,
    tune on scratch packs, allocate the new pack) and the real device-memory
    accounting, with packs that hold no memory: only the accounting runs."""
    _build = serve.Server._build
    _release = serve.Server._release

    def __init__(self, budget, rebuild_every=2):
        super().__init__(budget=budget, rebuild_every=rebuild_every)
        self.carried = 0

    def _carry(self, old, members):
        carry = {}
        for s in old.solves:
            if s in members:
                carry[id(s)] = None
                self._charge(s.carry)
                self.carried += 1
        return carry

    def _choose_impl(self, N, solves):
        for _ in range(2):                     # two scratch packs, one at a time
            self._charge(sum(s.bytes for s in solves))
            self._charge(-sum(s.bytes for s in solves))
        return 0

    def _new_pack(self, N, members, carry, impl):
        self._charge(sum(s.bytes for s in members))
        self.live_log.append(len(members))
        return FakePack(N, members, 0)


@pytest.mark.parametrize("every", [1, 2, 8])
def test_rebuild_peak_stays_within_the_budget(every):
    """Admissions as budget frees up join live packs, so packs are rebuilt while they hold carried
    solves; the accounted device bytes (admitted solves, the carried copies of
    a rebuild, the tuner's scratch packs) never exceed the budget, although
    several solves are live at once."""
    reqs = requests(40, seed=3)
    per = [serve.solve_bytes(len(q.tets), (q.N + 1) * (q.N + 2) * (q.N + 3) // 6) +
           serve.carry_bytes(len(q.tets), (q.N + 1) * (q.N + 2) * (q.N + 3) // 6) for q in reqs]
    budget = 4 * max(per)
    srv = LedgerServer(budget, rebuild_every=every)
    res = srv.run(reqs, max_iterations=100_000)
    assert [r.rid for r in res] == list(range(len(reqs)))
    assert srv.carried > 0 and max(srv.live_log) > 1
    assert 0 < srv.stats["model_peak"] <= budget
    assert srv.stats["model_now"] == 0                # everything released at the end


@pytest.mark.parametrize("frac", [0.2, 0.5, 1.0])
def test_dead_weight_rebuilds(frac):
    """A pack is rebuilt without its finished solves once they hold `frac` of
    its elements (after rebuild_every steps); every solve still finishes with
    its exact step count, and a lower threshold never builds fewer packs."""
    reqs = requests(count=30, seed=3)
    srv = FakeServer(rebuild_every=2, dead_fraction=frac)
    res = srv.run(reqs, max_iterations=10_000)
    assert sorted(r.rid for r in res) == list(range(30))
    base = FakeServer(rebuild_every=2, dead_fraction=1.0)
    base.run(requests(count=30, seed=3), max_iterations=10_000)
    assert srv.stats["packs_built"] >= base.stats["packs_built"]


def test_dead_weight_counts_elements_not_solves():
    srv = FakeServer(dead_fraction=0.5)
    small = [FakeLive(serve.Request(i, None, np.zeros((10, 4)), 2, 3.0, None), 0.0) for i in range(3)]
    big = FakeLive(serve.Request(9, None, np.zeros((100, 4)), 2, 3.0, None), 0.0)
    p = FakePack(2, small + [big], 0)
    for s in small:
        s.finished = True                     # 3 of 4 solves, 30 of 130 elements
    assert not srv._dead_weight(p)
    big.finished, small[0].finished = True, False
    assert srv._dead_weight(p)                # 120 of 130 elements
