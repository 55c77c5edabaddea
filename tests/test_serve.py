"""Serving loop (paper_0901_1024_gb300/serve.py) on the GPU: every solve's
fields are the same alone and in the mix -- bit for bit on the same stage
implementation -- whether solves are packed into one launch per order or
stepped one by one, packs of all orders advanced by shared launches or one
launch per pack, replayed from CUDA graphs or launched directly, admitted
together or one at a time by a small HBM budget."""
import numpy as np
import pytest

from workloads import gaussian_pulse, kuhn_box_mesh, random_fields

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(120)]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as dg
    from paper_0901_1024_gb300 import serve
    return torch, dg, serve


def _requests(serve, spread=0.02):
    specs = [(2, 2, 0.3, "pulse"), (3, 3, 0.2, "rand"), (2, 4, 0.25, "pulse"),
             (4, 4, 0.15, "rand"), (3, 1, 0.4, "pulse"), (2, 3, 0.1, "rand")]
    reqs = []
    for rid, (n, N, T, kind) in enumerate(specs):
        verts, tets = kuhn_box_mesh(n, 0.1, rid)
        if kind == "pulse":
            init = (lambda x: gaussian_pulse(x[0], x[1], x[2], 0.3, (0.1, -0.2, 0.05)))
        else:
            init = (lambda x, s=rid: random_fields(x.shape[1], x.shape[2], 100 + s))
        reqs.append(serve.Request(rid, verts, tets, N, T, init, arrival=spread * (rid % 3)))
    return reqs


def _check_against_alone(serve, dg, results, reqs, impl):
    for res, req in zip(results, reqs):
        u, e, steps, dt = serve.run_alone(req, impl=impl)
        assert res.rid == req.rid and res.steps == steps and res.dt == dt
        assert np.array_equal(res.fields, u), req.rid
        assert abs(res.energy - e) <= 1e-12 * abs(e)
        assert res.finished >= res.admitted >= res.arrival - 1e-9


@pytest.mark.parametrize("batch,graphs,mixed", [(True, True, True), (True, False, True),
                                                 (True, True, False), (False, False, False)])
def test_same_alone_and_in_the_mix(env, batch, graphs, mixed):
    """mixed: every pack, of every order, advanced by shared launches
    (dg_rk_stage_multi); else one launch per pack and stage."""
    torch, dg, serve = env
    reqs = _requests(serve)
    srv = serve.Server(batch=batch, graphs=graphs, autotune=False, impl=dg.Mesh.STAGE_TC,
                       mixed=mixed)
    results = srv.run(reqs, max_iterations=200_000)
    _check_against_alone(serve, dg, results, reqs, dg.Mesh.STAGE_TC)


def test_small_budget_admits_one_at_a_time(env):
    torch, dg, serve = env
    reqs = _requests(serve, spread=0.0)
    srv = serve.Server(hbm_budget=1.0, batch=True, graphs=True, autotune=False,
                       impl=dg.Mesh.STAGE_TC)
    results = sorted(srv.run(reqs, max_iterations=200_000), key=lambda r: r.admitted)
    for a, b in zip(results, results[1:]):
        assert b.admitted >= a.finished - 1e-6
    _check_against_alone(serve, dg, sorted(results, key=lambda r: r.rid), reqs, dg.Mesh.STAGE_TC)


def test_autotuned_packs_stay_within_the_parity_tolerance(env):
    torch, dg, serve = env
    reqs = _requests(serve)
    results = serve.Server(autotune=True).run(reqs, max_iterations=200_000)
    for res, req in zip(results, reqs):
        u, _, _, _ = serve.run_alone(req, impl=dg.Mesh.STAGE_FP32)
        assert np.linalg.norm(res.fields - u) <= 1e-5 * np.linalg.norm(u), req.rid
