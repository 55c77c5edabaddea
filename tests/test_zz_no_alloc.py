"""dg_energy_noalloc: the discrete energy computed without any allocation.

Callers whose device memory is owned by their own pool and budget (a serving
process), or time loops that must keep cudaMalloc/cudaFree out of their steady
state, cannot let the library allocate scratch.  This entry point keeps its
partial sums in a fixed device array inside the library; here it is called
through the C ABI and checked against dg_energy, the allocating entry point,
and against the FP64 oracle's energy, on two calls in a row, on vacuum meshes
and on a mesh with per-element eps and mu (E rows weighted by eps, H rows by
mu).  A host-only test checks that a mesh above the array's limit is refused
before anything touches the device.  Collected last so that a
stop-at-first-failure run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle

TOL = 1e-6   # relative, the energy tolerance of the parity tests
MAX_K = 4194304   # 65 536 blocks of 64 tetrahedra


def _call(lib, mesh, u, out, stream):
    return lib.dg_energy_noalloc(mesh._h, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()),
                                 C.c_void_p(stream.cuda_stream))


@pytest.mark.gpu
def test_energy_noalloc_matches_dg_energy_and_oracle_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as dg
    from workloads import kuhn_box_mesh, random_fields

    lib = dg.load()
    stream = torch.cuda.current_stream()
    # K = 1296 (ragged last block of 64), K = 162, and K = 162 with materials
    for n, N, seed, materials in ((6, 4, 3, False), (3, 2, 4, False), (3, 3, 5, True)):
        verts, tets = kuhn_box_mesh(n, 0.1, seed)
        mesh = dg.Mesh(verts, tets, N)
        om = oracle.build_mesh(verts, tets, N)
        eps = mu = None
        if materials:
            rng = np.random.default_rng(seed)
            eps, mu = rng.uniform(0.5, 4.0, mesh.K), rng.uniform(0.5, 3.0, mesh.K)
            mesh.set_materials(eps, mu)
        u32 = random_fields(mesh.K, mesh.Np, seed).astype(np.float32)
        u = torch.from_numpy(u32).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        if n == 6:
            # not yet on the device: refused, since uploading the mesh would allocate
            assert _call(lib, mesh, u, out, stream) == -7
        ref = mesh.energy(u)                        # allocating entry point (uploads the mesh)
        want = oracle.energy(om, u32.astype(np.float64), eps, mu)
        assert abs(ref - want) <= TOL * want
        for _ in range(2):
            out.fill_(float("nan"))
            assert _call(lib, mesh, u, out, stream) == 0, lib.dg_last_error()
            torch.cuda.synchronize()
            got = out.item()
            assert abs(got - ref) <= TOL * abs(ref), (got, ref)
            assert abs(got - want) <= TOL * want, (got, want)


def _kuhn_tets(n):
    """Connectivity of the n^3 x 6 Kuhn split of a unit-spaced grid (as
    workloads.kuhn_box_mesh, vectorised, no jitter) and its vertices."""
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v0 = np.stack([k.ravel(), j.ravel(), i.ravel()], 1)           # x fastest, as the generator
    vid = lambda p: p[..., 0] + (n + 1) * (p[..., 1] + (n + 1) * p[..., 2])  # noqa: E731
    unit = np.eye(3, dtype=np.int64)
    perms = [(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)]
    tets = np.empty((len(v0), 6, 4), np.int32)
    for q, (a, b) in enumerate(perms):
        p1 = v0 + unit[a]
        tets[:, q] = np.stack([vid(v0), vid(p1), vid(p1 + unit[b]), vid(v0 + 1)], 1)
    g = np.arange(n + 1, dtype=np.float64)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1), tets.reshape(-1, 4)


def test_energy_noalloc_refuses_a_mesh_above_its_limit():
    """Host only: K = 6 * 89^3 = 4 229 814 > 4 194 304 is refused with DG_ERR_ARG
    before any device work (the pointers are never dereferenced)."""
    import paper_0901_1024_gb300 as dg
    verts, tets = _kuhn_tets(89)
    assert len(tets) > MAX_K
    mesh = dg.Mesh(verts, tets, 1)
    lib = dg.load()
    rc = lib.dg_energy_noalloc(mesh._h, C.c_void_p(256), C.c_void_p(256), None)
    assert rc == -1
    assert b"4194304" in lib.dg_last_error()
    mesh.close()
