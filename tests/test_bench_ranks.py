"""Host logic of bench.py's multi-GPU path: independent replicas (the stage
does not shard), the job time is the slowest rank's, and the value counts
every replica's updates.  Run as two gloo ranks on the CPU; the reference arm
prints from rank 0 only."""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    t = bench.max_over_ranks(dist, 1.5 + rank, "cpu")         # rank 1 is the slow one
    v = bench.job_value(w, 1000, 10, t)
    out.put((r, w, local, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for r, w, local, t, v in got:
        assert (w, local) == (2, r)
        assert t == 2.5                                    # the max, on every rank
        assert v == pytest.approx(2 * 1000 * 10 / 2.5)     # both replicas' updates


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
    assert bench.job_value(1, 6 * 10 * 35, 5, 0.5) == 6 * 10 * 35 * 5 / 0.5


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup = "pulse_n24_N4", 1, 3
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_all_cores_oracle_timing_sums_independent_processes():
    """The all-cores oracle baseline: two spawned processes, each stepping its
    own copy of a one-layer sample of the 384-tet cavity mesh; the value is
    the sum of their rates and the sample names the step count."""
    w, verts, tets = bench.workload_inputs("cavity_n4_N3")
    r = bench.time_oracle_all_cores(w, verts, tets, seconds=0.5, procs=2)
    assert "error" not in r, r
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0
    assert "96 tets" in r["sample"]
