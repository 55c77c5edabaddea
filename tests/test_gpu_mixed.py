"""dg_rk_stage_multi: one persistent launch per RK stage over the packed meshes
of several orders (the batched form of the paper's element-local stage).

Every mesh's fields must be bit for bit those of its own per-mesh stage
(dg_rk_stage_elem / dg_rk_stage): a packed element does the same arithmetic
whichever CTA of the shared grid runs it.  Orders 1..4 share one launch, 5..6
another, the rest (order 7 here: the tensor-core kernel with part of its
operator in shared memory) launch alone; the trace shows it.
"""
import numpy as np
import pytest

from workloads import kuhn_box_mesh, random_fields

pytestmark = pytest.mark.gpu

KIND_FP32_STAGE, KIND_MIXED = 0, 6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as dg
    return torch, dg


def _meshes(dg, spec):
    """spec: (order, n, seed, materials) per mesh; each a pack of two jittered
    box meshes (two solves side by side, as the serving loop builds them; K =
    12 n^3 keeps K Np a multiple of 4, which the tensor-core stages need)."""
    out = []
    for N, n, seed, mat in spec:
        a = dg.Mesh(*kuhn_box_mesh(n, 0.1, seed), N)
        b = dg.Mesh(*kuhn_box_mesh(n, 0.15, seed + 1), N)
        if mat:
            rng = np.random.default_rng(seed)
            a.set_materials(rng.uniform(0.5, 3.0, a.K), rng.uniform(0.5, 3.0, a.K))
            b.set_materials(np.ones(b.K), np.ones(b.K))
        p = dg.Mesh.pack([a, b])
        if N == 1:
            p.set_stage_impl(p.STAGE_TC)           # order 1 runs on CUDA cores by default
        out.append(p)
    return out


def _state(torch, meshes, seed):
    us, ress, dts = [], [], []
    for i, m in enumerate(meshes):
        us.append(torch.from_numpy(random_fields(m.K, m.Np, seed + i).astype(np.float32)).cuda())
        ress.append(torch.from_numpy(0.01 * random_fields(m.K, m.Np, 50 + seed + i)
                                     .astype(np.float32)).cuda())
        dts.append(torch.full((m.K,), 0.5 * m.dt_cfl, dtype=torch.float32, device="cuda"))
    return us, ress, dts


SPEC = [(1, 3, 1, False), (2, 4, 2, False), (3, 3, 3, True), (4, 4, 4, False),
        (5, 3, 5, False), (6, 2, 6, True), (7, 2, 7, False)]


@pytest.mark.parametrize("costs", ["default", "skewed"])
def test_mixed_stage_is_bit_identical_to_per_mesh_stages(env, costs):
    torch, dg = env
    meshes = _meshes(dg, SPEC)
    us, ress, dts = _state(torch, meshes, 10)
    want = []
    for m, u, r, dt in zip(meshes, us, ress, dts):
        out, rr = torch.empty_like(u), r.clone()
        m.rk_stage_elem(u, out, rr, 2, dt)
        want.append((out, rr))
    outs = [torch.empty_like(u) for u in us]
    rr = [r.clone() for r in ress]
    tile_cost = None if costs == "default" else [1.0, 9.0, 0.2, 3.0, 5.0, 0.5, 1.0]
    meshes[0].trace_enable(16)
    dg.Mesh.rk_stage_multi(meshes, us, outs, rr, 2, dt_elem=dts, tile_cost=tile_cost)
    torch.cuda.synchronize()
    _, kinds = meshes[0].trace_read()
    meshes[0].trace_enable(0)
    assert sorted(int(k) for k in kinds) == [KIND_MIXED, KIND_MIXED]   # orders 1..4, then 5..6
    assert meshes[0].last_launch_count() == 3                           # + order 7 on its own
    for (o, r), (wo, wr) in zip(zip(outs, rr), want):
        assert torch.equal(o, wo) and torch.equal(r, wr)


def test_mixed_steps_match_per_mesh_steps(env):
    """Three LSERK4 steps (15 shared launches, buffers swapped after each stage)
    with a scalar step: every mesh bit-identical to its own dg_rk_stage run."""
    torch, dg = env
    meshes = _meshes(dg, SPEC[1:6])
    us, _, _ = _state(torch, meshes, 20)
    dt = min(m.dt_cfl for m in meshes)
    ref = []
    for m, u in zip(meshes, us):
        a, b, r = u.clone(), torch.empty_like(u), torch.zeros_like(u)
        for _ in range(3):
            for i in range(5):
                m.rk_stage(a, b, r, i, dt)
                a, b = b, a
        ref.append((a, r))
    a = [u.clone() for u in us]
    b = [torch.empty_like(u) for u in us]
    r = [torch.zeros_like(u) for u in us]
    for _ in range(3):
        for i in range(5):
            dg.Mesh.rk_stage_multi(meshes, a, b, r, i, dt)
            a, b = b, a
    torch.cuda.synchronize()
    for x, rx, (wa, wr) in zip(a, r, ref):
        assert torch.equal(x, wa) and torch.equal(rx, wr)


def test_more_meshes_than_one_launch_holds(env):
    """Ten order-2 packs: two shared launches (8 + 2 groups), same results."""
    torch, dg = env
    meshes = _meshes(dg, [(2, 2 + (i % 3), 30 + i, False) for i in range(10)])
    us, ress, dts = _state(torch, meshes, 40)
    want = []
    for m, u, r, dt in zip(meshes, us, ress, dts):
        out, rr = torch.empty_like(u), r.clone()
        m.rk_stage_elem(u, out, rr, 4, dt)
        want.append((out, rr))
    outs = [torch.empty_like(u) for u in us]
    rr = [r.clone() for r in ress]
    dg.Mesh.rk_stage_multi(meshes, us, outs, rr, 4, dt_elem=dts)
    torch.cuda.synchronize()
    assert meshes[0].last_launch_count() == 2
    for (o, r), (wo, wr) in zip(zip(outs, rr), want):
        assert torch.equal(o, wo) and torch.equal(r, wr)


def test_mixed_stage_argument_errors(env):
    torch, dg = env
    meshes = _meshes(dg, [(2, 2, 1, False), (3, 2, 2, False)])
    us, ress, _ = _state(torch, meshes, 5)
    with pytest.raises(dg.DGError):                       # a mesh twice
        dg.Mesh.rk_stage_multi([meshes[0], meshes[0]], us, [torch.empty_like(u) for u in us],
                               ress, 0, 0.01)
    with pytest.raises(dg.DGError):                       # stage out of range
        dg.Mesh.rk_stage_multi(meshes, us, [torch.empty_like(u) for u in us], ress, 5, 0.01)
    with pytest.raises(dg.DGError):                       # u_out aliases u_in
        dg.Mesh.rk_stage_multi(meshes, us, us, ress, 0, 0.01)
