"""The benchmark's roofline arithmetic (host only): algorithmic bytes and
flops per element and RK stage, built here from their parts, and the
per-order table they give (bytes / flops per element for N = 1..9, and
289.6 MB per stage on the 82 944-tet N = 4 workload)."""
import os
import re

import pytest

import bench


def _dofs(N):
    return (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2


def test_bytes_per_element_from_the_arrays_a_stage_streams():
    f32, i32 = 4, 4
    for N in range(1, 10):
        Np, _ = _dofs(N)
        fields = 4 * 6 * Np * f32          # read u, read res, write res, write u
        geometry = (9 + 4 * (3 + 1)) * f32 + 4 * 2 * i32   # metric, 4 x (normal, Fscale), 4 x (neighbour, code)
        assert bench.stage_bytes_per_elem(Np) == fields + geometry


def test_flops_per_element_from_the_steps_of_the_method():
    """Additions and multiplications, as the paper counts them."""
    for N in range(1, 10):
        Np, Nfp = _dofs(N)
        nf = 4 * Nfp
        derivatives = 3 * 6 * Np * 2 * Np      # Dr, Ds, Dt on six fields
        chain_rule = 12 * Np * 5               # 12 physical derivatives, 3 products + 2 sums each
        curl = 6 * Np                          # one difference per curl component
        flux = 60 * nf                         # upwind flux per face node (R11)
        lift = 6 * Np * 2 * nf                 # LIFT on six fields
        assembly = 6 * Np                      # volume + surface
        rk = 6 * Np * 5                        # res = a res + dt rhs, u += b res
        want = derivatives + chain_rule + curl + flux + lift + assembly + rk
        assert bench.flops_per_elem_stage(N, Np, Nfp) == want


@pytest.mark.parametrize("N,bytes_,flops", [
    (1, 516, 2280), (2, 1092, 8940), (3, 2052, 28440), (4, 3492, 76470), (5, 5508, 180096),
    (6, 8196, 382200), (7, 11652, 746640), (8, 15972, 1364130), (9, 21252, 2358840)])
def test_per_order_table(N, bytes_, flops):
    Np, Nfp = _dofs(N)
    assert bench.stage_bytes_per_elem(Np) == bytes_
    assert bench.flops_per_elem_stage(N, Np, Nfp) == flops


def test_headline_workload_bytes():
    Np, _ = _dofs(4)
    assert bench.stage_bytes_per_elem(Np) * 82944 == 289_640_448


@pytest.mark.parametrize("workload,family", [("pulse_n24_N4", "tc"), ("cavity_n16_N6", "tt"),
                                             ("pulse_n16_N7", "tt")])
def test_stage_profiles_are_machine_readable(workload, family):
    """The committed ncu summary of each benchmark workload carries the source
    digest of the kernel family it measured and the DRAM bytes per launch; the
    bench reports those bytes only while the digest matches the source."""
    text = open(os.path.join(bench.ROOT, "profiles", f"stage_kernel_{workload}.md")).read()
    digest = re.search(r"kernel_source_digest:\s*([0-9a-f]{16})\b", text)
    traffic = re.search(r"dram_bytes_per_launch:\s*([0-9]+)\b", text)
    assert digest and traffic and int(traffic.group(1)) > 0
    got = bench.profiled_traffic(workload, family)
    fresh = digest.group(1) == bench.kernel_source_digest(family)
    assert got == (float(traffic.group(1)) if fresh else None)


def test_kernel_family_of_each_stage_path():
    assert [bench.kernel_family(N, True) for N in range(1, 8)] == ["tc"] * 4 + ["tt"] * 3
    assert {bench.kernel_family(N, False) for N in range(1, 10)} == {"fp32"}
    for files in bench.KERNEL_SOURCES.values():
        for f in files:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_0901_1024_gb300", "csrc", f))
