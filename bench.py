"""Benchmark of the DG Maxwell hot path: LSERK4 steps of the fused RK-stage kernel.

One benchmark step = one LSERK4 time step = 5 RK stages, each a full right-
hand side (volume derivative + curl, face gather + upwind flux, LIFT) fused
with the stage update; the timed region also ends with one energy evaluation.
Metric: DOF-updates/s = 6 * K * Np per stage (six fields counted separately,
as in the paper's Fig. dofs-per-sec) / time.

Workload (default): N = 4 (Np = 35) on [-1,1]^3 cut into 24^3 hexes x 6 Kuhn
tetrahedra = 82 944 tets, interior vertices jittered by U[-0.15h, 0.15h]
(seed 0), PEC walls, Gaussian E_z pulse of width 0.2 centred at a seeded point.
Synthetic data.  u + res + the work copy are 209 MB > the 129 MB L2, so no L2
flush is needed between iterations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (weak scaling, no collective in the data path); the time is the max
over ranks.  `--impl reference` times the FP64 CPU oracle (the only reference
this method has) on a bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import WORKLOADS, gaussian_pulse, kuhn_box_mesh, pulse_center, cavity_mode  # noqa: E402

METRIC = "DOF-updates/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}


def workload_inputs(name):
    w = WORKLOADS[name]
    verts, tets = kuhn_box_mesh(w["n"], w["jitter"], w["seed"])
    return w, verts, tets


def element_order(dg, order, verts, tets, N):
    """Element numbering of the timed mesh: the workload's own (hex by hex),
    a seeded random renumbering (an unstructured generator's arbitrary order),
    or that random numbering renumbered by the greedy partition
    (dg_partition_order, blocks of 20 = the tensor-core tiles)."""
    if order == "native":
        return tets
    tets = tets[np.random.Generator(np.random.PCG64(11)).permutation(len(tets))]
    if order == "partition":
        tets = tets[dg.Mesh(verts, tets, N).partition_order(20)]
    return tets


def initial_fields(w, x):
    if w["init"] == "pulse":
        return gaussian_pulse(x[0], x[1], x[2], w["width"], pulse_center(w["pulse_seed"]))
    return cavity_mode(x[0], x[1], x[2], 0.0)


def describe(name, w, K, Np):
    return (f"{name}: N={w['N']} (Np={Np}), {w['n']}^3 hexes x 6 = {K} tets on [-1,1]^3, "
            f"jitter {w['jitter']}h (seed {w['seed']}), PEC walls, upwind flux, "
            f"{'Gaussian Ez pulse w=' + str(w['width']) if w['init'] == 'pulse' else 'cavity (1,1,1) mode'}")


def stage_bytes_per_elem(Np):
    # read u, read res, write res, write u (4 x 6 Np floats) + 132 B geometry/connectivity
    return 96 * Np + 132


def flops_per_elem_stage(N, Np, Nfp):
    # additions + multiplications (the paper's counting): derivatives, chain rule + curl,
    # flux, lifting, assembly, plus the LSERK4 update
    return 36 * Np * Np + 66 * Np + 60 * 4 * Nfp + 12 * Np * 4 * Nfp + 6 * Np + 30 * Np


def fp32_peak_tflops(sms: int, peaks: dict) -> float:
    """FP32 FMA peak in TFLOP/s: SMs (queried from the device) x 128 FP32 lanes x
    2 flop x the maximum SM clock (MEASURED_PEAKS.json, else 2070 MHz)."""
    return sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# Source files of each stage kernel family: a profile summary records the
# digest of the family it measured.
KERNEL_SOURCES = {
    "tc": ("tc_stage.cuh", "tcgen05.cuh", "launch.cuh", "device.h"),      # tensor cores, N <= 4
    "tt": ("tc_stage_t.cuh", "tc_stage.cuh", "tcgen05.cuh", "launch.cuh",
           "device.h"),                                                   # tensor cores, N = 5..7
    "fp32": ("stage_kernel.cuh", "tcgen05.cuh", "launch.cuh", "device.h"),  # CUDA cores
}


def kernel_family(N, tc_path):
    return ("tc" if N <= 4 else "tt") if tc_path else "fp32"


def kernel_source_digest(family):
    h = hashlib.sha256()
    for n in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_0901_1024_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, family):
    """DRAM bytes per stage launch from the committed ncu summary of this
    workload, if it was taken on the current source of the kernel family that
    ran (digest line), else None."""
    p = os.path.join(ROOT, "profiles", f"stage_kernel_{workload}.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    dg = re.search(r"kernel_source_digest:\s*([0-9a-f]+)", text)
    tb = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not dg or not tb or dg.group(1) != kernel_source_digest(family):
        return None
    return float(tb.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.samples = []
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), parts))

    def stop(self, t0, t1):
        if not self.p:
            return None
        time.sleep(0.12)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        rows = [(t, p) for t, p in self.samples]
        inwin = [p for t, p in rows if t0 - 0.06 <= t <= t1 + 0.06]
        busy = [p for t, p in rows if (num(p[3]) or 0) >= 50]
        use = inwin or busy or [p for _, p in rows]
        if not use:
            return None
        sm = [num(p[0]) for p in use if num(p[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in use for i in range(4) if p[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(use[0][1]), "reasons": reasons, "samples": len(use),
                "window": "timed region" if inwin else ("busy samples" if busy else "all samples")}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(dist, x, device):
    """The largest of every rank's x (x itself on one rank): the job's time is
    its slowest replica's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, dof_per_stage, stages, seconds):
    """Whole-job DOF-updates/s: every replica advances its own copy of the
    workload by `stages` stages in `seconds` (the slowest replica's time)."""
    return world * dof_per_stage * stages / seconds


def path_accuracy(mesh, w, x, u0, dt, steps=200):
    """Outside the timed region: `steps` LSERK4 steps from the initial fields on
    the default stage path and on the plain FP32 CUDA-core path; their relative
    L2 distance, and for the cavity mode each one's error against the exact
    solution at the final time."""
    import torch
    out = {"steps": steps}
    finals = {}
    for name, impl in (("default", mesh.STAGE_AUTO), ("plain_fp32", mesh.STAGE_FP32)):
        mesh.set_stage_impl(impl)
        mesh.trace_enable(5)
        u = torch.from_numpy(u0).cuda()
        r = torch.zeros_like(u)
        mesh.step(u, r, dt, steps)
        torch.cuda.synchronize()
        _, kinds = mesh.trace_read()
        mesh.trace_enable(0)
        finals[name] = u.cpu().numpy().astype(np.float64)
        out[name + "_kernel"] = "tensor cores" if 4 in set(int(k) for k in kinds) else "FP32 CUDA cores"
    mesh.set_stage_impl(mesh.STAGE_AUTO)
    ref = finals["plain_fp32"]
    out["rel_l2_default_vs_plain_fp32"] = float(np.linalg.norm(finals["default"] - ref) / np.linalg.norm(ref))
    if w["init"] == "cavity":
        exact = cavity_mode(x[0], x[1], x[2], steps * dt)
        for name, v in finals.items():
            out["rel_l2_vs_exact_" + name] = float(np.linalg.norm(v - exact) / np.linalg.norm(exact))
    return out


def run_ours(args):
    import torch
    import paper_0901_1024_gb300 as dg

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w, verts, tets = workload_inputs(args.workload)
    tets = element_order(dg, args.order, verts, tets, w["N"])
    mesh = dg.Mesh(verts, tets, w["N"])
    mesh.set_stage_impl({"auto": mesh.STAGE_AUTO, "fp32": mesh.STAGE_FP32,
                         "tc": mesh.STAGE_TC}[args.stage_kernel])
    K, Np, Nfp = mesh.K, mesh.Np, mesh.Nfp
    x = mesh.nodes()
    u0 = initial_fields(w, x).astype(np.float32)
    dt = mesh.dt_cfl
    stream = torch.cuda.current_stream()
    u = torch.from_numpy(u0).cuda()
    res = torch.zeros_like(u)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    # warm-up (also creates the work buffer and JIT-free kernels' attributes)
    mesh.step(u, res, dt, args.warmup)
    mesh.energy(u)
    # which stage kernel runs (per-launch trace of one step, outside the timed
    # region: events between launches would serialise the stage kernels, whose
    # launches otherwise overlap set-up with the previous kernel's tail)
    mesh.trace_enable(8)
    mesh.step(u, res, dt, 1)
    _, trace_kind = mesh.trace_read()
    mesh.trace_enable(0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t0 = time.time()
    e0.record(stream)
    mesh.step(u, res, dt, args.steps)
    launches = stage_launches = mesh.last_launch_count()
    em.record(stream)
    energy = mesh.energy(u)
    launches += mesh.last_launch_count()
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    ms = e0.elapsed_time(e1)
    stage_region_ms = e0.elapsed_time(em)
    ms = max_over_ranks(dist, ms, "cuda")
    if dist:
        dist.barrier()
    clocks = sampler.stop(t0, t1) if sampler else None

    dof_stage = 6 * K * Np
    value = job_value(world, dof_stage, 5 * args.steps, ms * 1e-3)
    tc_path = any(k == 4 for k in trace_kind)
    if (5 * args.steps) % 2 == 0:
        # the stage launches of the timed region, back to back on the stream
        avg_stage_s = stage_region_ms * 1e-3 / stage_launches
        avg_src = "timed region: CUDA events around the stage launches / launch count"
    else:
        # an odd stage count ends with a device copy of the state inside the
        # region; time the stages alone right after it (two steps)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        mesh.step(u, res, dt, 2)
        f1.record(stream)
        torch.cuda.synchronize()
        avg_stage_s = f0.elapsed_time(f1) * 1e-3 / 10
        avg_src = "two steps after the timed region (odd stage count inside it)"
    peaks, peaks_src = load_peaks()
    algo_bytes = stage_bytes_per_elem(Np) * K
    achieved = algo_bytes / avg_stage_s / 1e9
    traffic = profiled_traffic(args.workload, kernel_family(w["N"], tc_path))
    flops = flops_per_elem_stage(w["N"], Np, Nfp) * K
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = fp32_peak_tflops(sms, peaks)

    e2e = None
    if not args.no_e2e:
        # the step's input and result is the state u (the RK register is the
        # library's own: an LSERK4 step's result does not depend on it)
        uh = torch.from_numpy(u0.copy()).pin_memory()
        mesh.step_host(uh, None, dt, 1)                    # warm the host-path buffers
        n_e2e = max(1, min(args.steps, 20))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        for _ in range(n_e2e):
            mesh.step_host(uh, None, dt, 1, with_energy=True)
        h1 = time.perf_counter()
        el = max_over_ranks(dist, h1 - h0, "cuda")
        nbytes = u0.nbytes
        e2e = {"value": job_value(world, dof_stage, 5 * n_e2e, el), "unit": METRIC,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8,
               "steps": n_e2e, "call": "dg_step_host (pinned host u; H2D, 5 stages, D2H of u, energy)"}

    accuracy = None
    if rank == 0 and not args.no_accuracy:
        accuracy = path_accuracy(mesh, w, x, u0, dt)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(w, verts, tets, budget_s=args.cpu_budget)
        cpu["host_cores"] = usable_cores()
        cpu["blas"] = "none: the oracle's contractions are numpy.einsum loops (one thread)"
        if args.cpu_all_cores > 0:
            cpu["all_cores"] = time_oracle_all_cores(w, verts, tets, seconds=args.cpu_all_cores)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(args.workload, w, K, Np), "K": K, "N": w["N"], "Np": Np,
                       "dt": dt, "stages_per_step": 5, "energy_evals_in_timed_region": 1,
                       "l2": "inputs larger than L2 (u+res+work copy = %.0f MB > 129 MB)"
                             % (3 * u0.nbytes / 1e6),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "element_order": args.order, "stage_kernel": args.stage_kernel},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "kernel": ((f"tc_stage_kernel<N={w['N']},RK> (tcgen05, FP16x3 split)" if w["N"] <= 4
                                     else f"tt_stage_kernel<N={w['N']},RK> (tcgen05, FP16x3 split, "
                                          "operator in tensor memory)") if tc_path
                                    else f"stage_kernel<N={w['N']},RK> (FP32 CUDA cores)"),
                         "algorithmic_bytes_per_launch": algo_bytes,
                         "avg_launch_ms": avg_stage_s * 1e3, "launches_timed": stage_launches,
                         "avg_launch_source": avg_src,
                         "peak_source": f"{peaks_src} (MEASURED_PEAKS.json hbm_gbs)" if peaks_src == "measured"
                         else "fallback 6.8 TB/s"},
            "fp32_alu": {"achieved_tflops": flops / avg_stage_s / 1e12, "peak_tflops": fp32_peak,
                         "frac": flops / avg_stage_s / 1e12 / fp32_peak,
                         "peak_derivation": f"{sms} SMs (device query) x 128 FP32 lanes x 2 flop "
                                            "x sm_max_mhz"},
            "gflops": flops * 5 * args.steps / (ms * 1e-3) / 1e9 * world,
            "energy": energy,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "accuracy": accuracy,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def oracle_sample(w, verts, tets, layers):
    """The first `layers` z-layers of hexes of the workload mesh (6*n*n*layers tets)."""
    import oracle
    n = w["n"]
    Ks = 6 * n * n * layers
    om = oracle.build_mesh(verts, tets[:Ks], w["N"])
    u0 = initial_fields(w, np.stack([om.x, om.y, om.z]))
    return om, u0


def _run_oracle(om, u, budget_s, steps=None, cap=50):
    """Steps the oracle's LSERK4 from u for `steps` steps, or until about
    budget_s seconds (at most `cap` steps); returns (steps done, seconds)."""
    import oracle
    dt = oracle.cfl_dt(om)
    res = np.zeros_like(u)
    t0 = time.perf_counter()
    done = 0
    while True:
        u, res = oracle.lserk4_run(om, u, dt, 1, res)
        done += 1
        el = time.perf_counter() - t0
        if (steps and done >= steps) or (not steps and (el >= budget_s or done >= cap)):
            return done, el


def time_oracle(w, verts, tets, budget_s=15.0, layers=None, steps=None):
    """Times the FP64 oracle's LSERK4 steps on a bounded sample of the workload."""
    layers = layers or 2
    om, u = oracle_sample(w, verts, tets, layers)
    done, el = _run_oracle(om, u, budget_s, steps)
    dof = 6 * om.K * om.Np * 5 * done
    return {"value": dof / el, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{done} LSERK4 step(s) on the first {layers} z-layer(s) of hexes "
                      f"({om.K} of {len(tets)} tets) of the same mesh, FP64 NumPy oracle "
                      f"(single-threaded einsum), {el:.1f} s"}


def _oracle_process(job):
    """One process of the all-cores oracle timing: builds the sample mesh and
    steps it for about `seconds`; returns (DOF-updates, seconds taken)."""
    w, verts, tets, layers, seconds = job
    om, u = oracle_sample(w, verts, tets, layers)
    done, el = _run_oracle(om, u, seconds, cap=200)
    return 6 * om.K * om.Np * 5 * done, el


def usable_cores():
    """Cores this process may run on (its affinity mask where the OS has one)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_all_cores(w, verts, tets, seconds=10.0, layers=1, procs=None):
    """The FP64 oracle on every usable host core: one spawned process per core, each
    stepping its own copy of the same bounded sample (independent solves, as
    in the multi-GPU benchmark); the value is the sum of the processes' rates.
    A child that dies or overruns turns into an "error" entry, never a hang."""
    import concurrent.futures as cf
    import multiprocessing as mp
    procs = procs or usable_cores()
    Ks = 6 * w["n"] * w["n"] * layers
    Np = (w["N"] + 1) * (w["N"] + 2) * (w["N"] + 3) // 6
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})       # one thread per child
    ex = cf.ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn"))
    try:
        futs = [ex.submit(_oracle_process, (w, verts, tets, layers, seconds)) for _ in range(procs)]
        out = [f.result(timeout=4 * seconds + 120) for f in futs]
    except Exception as err:                         # broken pool, timeout
        for p in list(getattr(ex, "_processes", {}).values()):
            p.kill()
        ex.shutdown(wait=False, cancel_futures=True)
        return {"error": f"{type(err).__name__}: {err}"[:200], "cores": procs}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    ex.shutdown()
    steps = sum(d for d, _ in out) // (6 * Ks * Np * 5)
    return {"value": sum(d / e for d, e in out), "unit": METRIC, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes (one per host core), each stepping its own copy of the "
                      f"first {layers} z-layer(s) of hexes ({Ks} tets) for ~{seconds:.0f} s; "
                      f"{steps} LSERK4 steps in all"}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    w, verts, tets = workload_inputs(args.workload)
    import oracle
    layers = 1
    om, u = oracle_sample(w, verts, tets, layers)
    dt = oracle.cfl_dt(om)
    res = np.zeros_like(u)
    for _ in range(args.warmup):
        u, res = oracle.lserk4_run(om, u, dt, 1, res)
    t0 = time.perf_counter()
    u, res = oracle.lserk4_run(om, u, dt, args.steps, res)
    el = time.perf_counter() - t0
    e = oracle.energy(om, u)
    value = 6 * om.K * om.Np * 5 * args.steps / el
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": describe(args.workload, w, len(tets), om.Np), "K": len(tets),
                       "N": w["N"], "Np": om.Np,
                       "sample": f"first {layers} z-layer of hexes ({om.K} tets)"},
            "energy": e,
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} LSERK4 steps on {om.K} of {len(tets)} tets "
                                       "(first z-layer of hexes), FP64 NumPy oracle"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVE_SHAPE = {"n": (4, 20), "N": (1, 7), "T": (0.5, 4.0)}


def serve_requests(count, rate, seed, shape=SERVE_SHAPE):
    """Seeded request stream: Poisson arrivals at `rate` per second; box meshes
    of n^3 x 6 tets (n uniform in shape["n"], jitter 0.1h), orders N uniform in
    shape["N"], end times T uniform in shape["T"] (both ends included for
    integers), Gaussian pulse of width 0.3 at a seeded centre."""
    from paper_0901_1024_gb300.serve import Request
    rng = np.random.Generator(np.random.PCG64(seed))
    t, reqs = 0.0, []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.integers(shape["n"][0], shape["n"][1] + 1))
        N = int(rng.integers(shape["N"][0], shape["N"][1] + 1))
        T = float(rng.uniform(*shape["T"]))
        c = tuple(rng.uniform(-0.5, 0.5, 3))
        verts, tets = kuhn_box_mesh(n, 0.1, 1000 + rid)
        reqs.append(Request(rid, verts, tets, N, T,
                            lambda x, c=c: gaussian_pulse(x[0], x[1], x[2], 0.3, c), arrival=t))
    return reqs


SERVE_CONFIGS = {
    # Poisson stream of solves with n in [4, 20], N in {1..7}, T in [0.5, 4]
    "served": dict(count=32, seed=5, shape=SERVE_SHAPE),
    # 64 independent solves present at once, n in [4, 16], N in {2..6}
    "batched": dict(count=64, seed=6, shape={"n": (4, 16), "N": (2, 6), "T": (0.5, 0.5)}),
}


def run_serve(args):
    """Solves/s and latency percentiles of a request set, four ways on the same
    GPU: the continuous-batching server (one packed launch per order and stage,
    CUDA graphs, autotuned stage kernels); the same server advancing the packs
    of every order by shared launches (dg_rk_stage_multi); the per-solve form
    with the same kernels (one solve at a time, its own launches); and the plain
    per-solve form (one solve at a time on the FP32 CUDA-core stage).
    `--serve-config served` is a Poisson stream at `--rate`; `batched` releases
    all solves at once."""
    import torch
    from paper_0901_1024_gb300 import Mesh
    from paper_0901_1024_gb300.serve import Server
    cfg = SERVE_CONFIGS[args.serve_config]
    count = args.requests if args.serve_config == "served" else cfg["count"]
    rate = args.rate if args.serve_config == "served" else 1e12
    reqs = serve_requests(count, rate, cfg["seed"], cfg["shape"])
    # warm-up, as a serving process would at start-up: the same meshes released
    # together with a tiny end time set up every kernel and let the autotuner
    # pick the stage implementation of every (order, decade of K) in the set
    Server(autotune=True).run(serve_requests(count, 1e12, cfg["seed"],
                                             {**cfg["shape"], "T": (0.01, 0.01)}),
                              max_iterations=10**6)

    def summary(results, wall, srv):
        lat = np.array([r.latency for r in results])
        dofs = int(sum(6 * r.K * ((r.N + 1) * (r.N + 2) * (r.N + 3) // 6) * 5 * r.steps
                       for r in results))
        return {"solves_per_s": len(results) / wall, "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "wall_s": wall,
                "dof_updates": dofs, "dof_updates_per_s": dofs / wall, "host_phases": srv.stats}

    def timed(srv):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = srv.run(reqs, max_iterations=10**7)
        torch.cuda.synchronize()
        return res, summary(res, time.perf_counter() - t0, srv)

    served, ours = timed(Server(batch=True, graphs=not args.serve_no_graphs, autotune=True,
                                rebuild_every=args.rebuild_every, mixed=False,
                                dead_fraction=args.dead_fraction))
    shared = None
    if args.serve_shared:
        _, shared = timed(Server(batch=True, graphs=not args.serve_no_graphs, autotune=True,
                                 rebuild_every=args.rebuild_every, mixed=True,
                                 dead_fraction=args.dead_fraction))
    same, base = timed(Server(hbm_budget=1.0, batch=False, graphs=False, autotune=False))
    plain_res, plain = timed(Server(hbm_budget=1.0, batch=False, graphs=False, autotune=False,
                                    impl=Mesh.STAGE_FP32))

    def worst(a_list, b_list):
        return max(float(np.linalg.norm(a.fields - b.fields) / max(np.linalg.norm(b.fields), 1e-30))
                   for a, b in zip(a_list, b_list))
    shape = cfg["shape"]
    workload = (f"{count} requests, " + (f"Poisson {rate}/s" if args.serve_config == "served"
                                          else "all released at t = 0") +
                f", box meshes n^3 x 6 with n in {shape['n'][0]}..{shape['n'][1]}, N in "
                f"{shape['N'][0]}..{shape['N'][1]}, T in [{shape['T'][0]}, {shape['T'][1]}], "
                "Gaussian pulse, jitter 0.1h, seeded")
    line = {"metric": "served solves/s", "value": ours["solves_per_s"], "unit": "solves/s",
            "higher_is_better": True, "n_gpus": 1,
            "dtype": "f32 fields (FP16x3 tensor-core contractions for N = 2..7)",
            "data": "synthetic", "mode": "serve", "serve_config": args.serve_config,
            "config": {"workload": workload,
                       "server": "continuous batching: one packed launch per RK stage and order, "
                                 "CUDA graphs, autotuned stage kernel per (N, K), HBM budget 150 GB"},
            "served": ours, "shared_launch_all_orders": shared,
            "one_at_a_time_same_kernels": base, "plain_one_at_a_time_fp32": plain,
            "speedup_of_shared_launch": (shared["solves_per_s"] / ours["solves_per_s"]
                                         if shared else None),
            "speedup_vs_same_kernels": ours["solves_per_s"] / base["solves_per_s"],
            "speedup_vs_plain": ours["solves_per_s"] / plain["solves_per_s"],
            "autotuner_choices": Server.tuned_choices(),
            "max_rel_l2_vs_same_kernels": worst(served, same),
            "max_rel_l2_vs_plain_fp32": worst(served, plain_res)}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """Roofline curve over the order: for N = 1..9 a pulse workload on a box mesh
    with n chosen so that 6 K Np is about 1.7e7, timed per stage launch (CUDA
    events around back-to-back steps, divided by the stage count) after warm-up,
    for the default stage kernel (tensor cores for N = 2..7, FP32 CUDA cores
    otherwise) and the FP32 kernel in both tile shapes."""
    import torch
    import paper_0901_1024_gb300 as dg
    peaks, _ = load_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = fp32_peak_tflops(sms, peaks)
    rows = []
    for N in range(1, 10):
        Np, Nfp = (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2
        n = max(2, round((1.7e7 / (36 * Np)) ** (1 / 3)))
        verts, tets = kuhn_box_mesh(n, 0.15, 0)
        mesh = dg.Mesh(verts, tets, N)
        x = mesh.nodes()
        u0 = gaussian_pulse(x[0], x[1], x[2], 0.2, pulse_center(1)).astype(np.float32)
        for impl, shape in ([(0, 0), (1, 0), (1, 1)] if 2 <= N <= 7 else [(0, 0), (1, 1)]):
            mesh.set_stage_impl(impl)
            mesh.set_stage_shape(shape)
            u = torch.from_numpy(u0).cuda()
            res = torch.zeros_like(u)
            mesh.step(u, res, mesh.dt_cfl, 3)
            mesh.trace_enable(8)                   # which kernel runs (one traced step)
            mesh.step(u, res, mesh.dt_cfl, 1)
            _, kinds = mesh.trace_read()
            mesh.trace_enable(0)
            steps = args.sweep_steps + args.sweep_steps % 2      # even: no copy-back inside
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record()
            mesh.step(u, res, mesh.dt_cfl, steps)
            f1.record()
            torch.cuda.synchronize()
            stage = f0.elapsed_time(f1) * 1e-3 / (5 * steps)
            K = mesh.K
            gbs = stage_bytes_per_elem(Np) * K / stage / 1e9
            tf = flops_per_elem_stage(N, Np, Nfp) * K / stage / 1e12
            rows.append({"N": N, "n": n, "K": K, "Np": Np, "dofs": 6 * K * Np,
                         "kernel": ("tensor cores (FP16x3)" if 4 in kinds
                                    else f"FP32 CUDA cores, tile shape {shape}"),
                         "stage_us": stage * 1e6, "dof_updates_per_s": 6 * K * Np / stage,
                         "hbm_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"],
                         "tflops": tf, "fp32_frac": tf / fp32_peak})
        del mesh
    print(json.dumps({"mode": "sweep", "metric": "DOF-updates/s and % HBM roofline per RK stage",
                      "unit": "DOF-updates/s", "peak_hbm_gbs": peaks["hbm_gbs"],
                      "fp32_peak_tflops": fp32_peak, "steps": args.sweep_steps, "orders": rows}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pulse_n24_N4", choices=sorted(WORKLOADS))
    ap.add_argument("--order", default="native", choices=["native", "shuffled", "partition"],
                    help="element numbering of the timed mesh (see element_order)")
    ap.add_argument("--mode", default="stage", choices=["stage", "serve", "sweep"],
                    help="stage: the RK-stage benchmark (default); serve: the request-stream "
                         "benchmark; sweep: stage throughput for N = 1..9")
    ap.add_argument("--sweep-steps", type=int, default=20)
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--rebuild-every", type=int, default=32,
                    help="serve mode: steps a pack runs before waiting solves join it")
    ap.add_argument("--serve-no-graphs", action="store_true")
    ap.add_argument("--dead-fraction", type=float, default=0.15,
                    help="serve: rebuild an aged pack once finished solves hold this share of it")
    ap.add_argument("--serve-shared", action="store_true",
                    help="serve mode: also time the server with shared launches of all orders")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--serve-config", default="served", choices=sorted(SERVE_CONFIGS),
                    help="request set of --mode serve: a Poisson stream, or solves released together")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stage-kernel", default="auto", choices=["auto", "fp32", "tc"],
                    help="stage implementation of the timed run (auto: the library's default per order)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the 200-step comparison of the default and the plain FP32 path")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-all-cores", type=float, default=10.0,
                    help="seconds of the all-cores oracle timing (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)          # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
