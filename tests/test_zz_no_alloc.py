"""dg_energy_noalloc: the discrete energy computed without any allocation.

Callers whose device memory is owned by their own pool and budget (a serving
process), or time loops that must keep cudaMalloc/cudaFree out of their steady
state, cannot let the library allocate scratch.  This entry point keeps its
partial sums in a fixed device array inside the library; here it is called
through the C ABI and checked against dg_energy, the allocating entry point,
on two calls in a row.  Collected last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6   # relative, the energy tolerance of the parity tests


def _call(lib, mesh, u, out, stream):
    return lib.dg_energy_noalloc(mesh._h, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()),
                                 C.c_void_p(stream.cuda_stream))


def test_energy_noalloc_matches_dg_energy_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0901_1024_gb300 as dg
    from workloads import kuhn_box_mesh, random_fields

    lib = dg.load()
    stream = torch.cuda.current_stream()
    for n, N, seed in ((6, 4, 3), (3, 2, 4)):      # K = 1296 (ragged last block), K = 162
        verts, tets = kuhn_box_mesh(n, 0.1, seed)
        mesh = dg.Mesh(verts, tets, N)
        u = torch.from_numpy(random_fields(mesh.K, mesh.Np, seed).astype(np.float32)).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        if n == 6:
            # not yet on the device: refused, since uploading the mesh would allocate
            assert _call(lib, mesh, u, out, stream) == -7
        ref = mesh.energy(u)                        # allocating entry point (uploads the mesh)
        for _ in range(2):
            out.fill_(float("nan"))
            assert _call(lib, mesh, u, out, stream) == 0, lib.dg_last_error()
            torch.cuda.synchronize()
            got = out.item()
            assert abs(got - ref) <= TOL * abs(ref), (got, ref)
