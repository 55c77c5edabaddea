"""GB300 nodal DG Maxwell solver: thin Python binding over libdg.so (include/dg.h).

Every computation runs inside the C/CUDA library; this module only marshals
arguments (NumPy arrays for host data, torch CUDA tensors or raw device
pointers for fields) and turns error codes into exceptions.  There is no
Python or CPU fallback: if libdg.so is missing, importing `Mesh` works but the
first call raises ImportError.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._capi import DGError, check, library_path, load  # noqa: F401

__all__ = ["Mesh", "DGError", "load", "library_path"]


def _dptr(a: np.ndarray, dtype):
    assert a.dtype == dtype and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _devptr(x):
    if isinstance(x, int):
        return C.c_void_p(x)
    assert x.is_cuda and x.is_contiguous(), "fields must be contiguous CUDA tensors"
    import torch
    assert x.dtype == torch.float32, "fields must be float32"
    return C.c_void_p(x.data_ptr())


def _devptr_any(x):
    if isinstance(x, int):
        return C.c_void_p(x)
    assert x.is_cuda and x.is_contiguous()
    return C.c_void_p(x.data_ptr())


class Mesh:
    """A tetrahedral mesh with its DG operators (owns a dg_mesh*)."""

    def __init__(self, verts, tets, N: int | None = None):
        self._lib = load()
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        if verts.ndim != 2 or verts.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4:
            raise ValueError("verts must be [nv,3] and tets [K,4]")
        h = C.c_void_p()
        check(self._lib.dg_mesh_create(_dptr(verts, np.float64), len(verts),
                                       _dptr(tets, np.int32), len(tets), C.byref(h)),
              "dg_mesh_create")
        self._h = h
        self.N = None
        if N is not None:
            self.set_order(N)

    @classmethod
    def pack(cls, meshes):
        """dg_mesh_pack: one mesh made of `meshes` (same order) side by side;
        element k of meshes[i] becomes k + sum of the earlier meshes' K."""
        lib = load()
        arr = (C.c_void_p * len(meshes))(*[m._h.value for m in meshes])
        h = C.c_void_p()
        check(lib.dg_mesh_pack(arr, len(meshes), C.byref(h)), "dg_mesh_pack")
        self = cls.__new__(cls)
        self._lib, self._h = lib, h
        return self._read_info(meshes[0].N)

    def _read_info(self, N):
        self.N = int(N)
        K, Np, Nfp, dt = C.c_int64(), C.c_int(), C.c_int(), C.c_double()
        check(self._lib.dg_info(self._h, C.byref(K), C.byref(Np), C.byref(Nfp), C.byref(dt)),
              "dg_info")
        self.K, self.Np, self.Nfp, self.dt_cfl = K.value, Np.value, Nfp.value, dt.value
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.dg_mesh_destroy(h)
            self._h = None

    close = __del__

    # ---- host setup -------------------------------------------------------
    def set_order(self, N: int):
        check(self._lib.dg_set_order(self._h, int(N)), "dg_set_order")
        return self._read_info(N)

    def set_flux(self, alpha: float):
        check(self._lib.dg_set_flux(self._h, float(alpha)), "dg_set_flux")

    def set_materials(self, eps=None, mu=None):
        """Per-element permittivity and permeability (K values > 0 each; None: 1).
        The stage then uses the impedance-weighted upwind flux; dt_cfl and the
        energy follow the materials."""
        e = None if eps is None else np.ascontiguousarray(eps, np.float64)
        m = None if mu is None else np.ascontiguousarray(mu, np.float64)
        for a in (e, m):
            if a is not None and a.shape != (self.K,):
                raise ValueError("eps and mu need one value per element")
        check(self._lib.dg_set_materials(self._h, None if e is None else _dptr(e, np.float64),
                                         None if m is None else _dptr(m, np.float64)),
              "dg_set_materials")
        self._read_info(self.N)

    BC_PEC, BC_ABSORBING = 0, 1

    def set_boundary(self, kind=None):
        """Boundary kind of every face, (K, 4) array of BC_PEC / BC_ABSORBING
        (read on boundary faces only; faces numbered as the normals of
        dg_get_geometry); None: every boundary face a perfect conductor."""
        k = None if kind is None else np.ascontiguousarray(kind, np.int8)
        if k is not None and k.shape != (self.K, 4):
            raise ValueError("kind needs shape (K, 4)")
        check(self._lib.dg_set_boundary(self._h, None if k is None else k.ctypes.data),
              "dg_set_boundary")

    STAGE_AUTO, STAGE_FP32, STAGE_TC = 0, 1, 2

    def set_stage_impl(self, impl: int):
        """0 = auto (tensor cores for N = 2..6), 1 = FP32 CUDA cores, 2 = tensor cores."""
        check(self._lib.dg_set_stage_impl(self._h, int(impl)), "dg_set_stage_impl")

    def set_stage_shape(self, shape: int):
        """dg_set_stage_shape: FP32 stage tile shape, 0 (default) or 1 (half the
        tetrahedra per tile)."""
        check(self._lib.dg_set_stage_shape(self._h, int(shape)), "dg_set_stage_shape")

    def set_energy_check(self, max_growth: float):
        """dg_set_energy_check: step_host fails with DG_ERR_UNSTABLE when the
        energy grows by more than the factor 1 + max_growth (< 0: off)."""
        check(self._lib.dg_set_energy_check(self._h, float(max_growth)), "dg_set_energy_check")

    def nodes(self) -> np.ndarray:
        out = np.empty((3, self.K, self.Np), np.float64)
        check(self._lib.dg_nodes(self._h, _dptr(out, np.float64)), "dg_nodes")
        return out

    def connectivity(self):
        n = self.K * 4 * self.Nfp
        vM, vP = np.empty(n, np.int32), np.empty(n, np.int32)
        check(self._lib.dg_get_connectivity(self._h, _dptr(vM, np.int32), _dptr(vP, np.int32)),
              "dg_get_connectivity")
        return vM, vP

    def partition_order(self, block: int = 20):
        """Greedy partition numbering (dg_partition_order): perm[i] is the
        current index of the element to place at position i; renumber with
        tets[perm] and u[:, perm]."""
        perm = np.empty(self.K, np.int64)
        check(self._lib.dg_partition_order(self._h, int(block), _dptr(perm, np.int64)),
              "dg_partition_order")
        return perm

    def operators(self):
        Np, NF = self.Np, 4 * self.Nfp
        Dr, Ds, Dt, M = (np.empty((Np, Np)) for _ in range(4))
        L = np.empty((Np, NF))
        check(self._lib.dg_get_operators(self._h, *(_dptr(a, np.float64) for a in (Dr, Ds, Dt, M, L))),
              "dg_get_operators")
        return dict(Dr=Dr, Ds=Ds, Dt=Dt, M=M, LIFT=L)

    def geometry(self):
        K = self.K
        metric, J, n, Fs = np.empty((9, K)), np.empty(K), np.empty((3, K, 4)), np.empty((K, 4))
        check(self._lib.dg_get_geometry(self._h, *(_dptr(a, np.float64) for a in (metric, J, n, Fs))),
              "dg_get_geometry")
        return dict(metric=metric, J=J, normals=n, Fscale=Fs)

    # ---- device calls -----------------------------------------------------
    def rhs(self, u, out, stream=None):
        check(self._lib.dg_rhs(self._h, _devptr(u), _devptr(out), _stream_handle(stream)), "dg_rhs")
        return out

    def step(self, u, res, dt: float, nsteps: int, stream=None):
        check(self._lib.dg_step(self._h, _devptr(u), _devptr(res), float(dt), int(nsteps),
                                _stream_handle(stream)), "dg_step")

    def rk_stage(self, u_in, u_out, res, stage: int, dt: float, stream=None):
        """One LSERK4 stage (dg_rk_stage): res <- a_i res + dt rhs(u_in),
        u_out <- u_in + b_i res."""
        check(self._lib.dg_rk_stage(self._h, _devptr(u_in), _devptr(u_out), _devptr(res),
                                    int(stage), float(dt), _stream_handle(stream)), "dg_rk_stage")

    def rk_stage_range(self, u_in, u_out, res, stage: int, dt: float, k0: int, k1: int,
                       stream=None):
        """dg_rk_stage_range: one LSERK4 stage for the elements [k0, k1) only (tile
        boundaries of `stage_tile`, or k1 = K)."""
        check(self._lib.dg_rk_stage_range(self._h, _devptr(u_in), _devptr(u_out), _devptr(res),
                                          int(stage), float(dt), int(k0), int(k1),
                                          _stream_handle(stream)), "dg_rk_stage_range")

    def check_wait_timeout(self, polls: int):
        """dg_check_wait_timeout: (status code, message, seconds) of the stage
        kernels' bounded wait run out on purpose (expected: DG_ERR_CUDA)."""
        sec = C.c_double(-1.0)
        rc = self._lib.dg_check_wait_timeout(self._h, int(polls), C.byref(sec))
        msg = self._lib.dg_last_error().decode() if rc else ""
        return rc, msg, sec.value

    def stage_tile(self, u_in=None, u_out=None, res=None) -> int:
        """dg_stage_tile: tetrahedra per tile of the stage kernel these buffers run
        (None: aligned buffers)."""
        t = C.c_int()
        ptr = lambda x: None if x is None else _devptr(x)  # noqa: E731
        check(self._lib.dg_stage_tile(self._h, ptr(u_in), ptr(u_out), ptr(res), C.byref(t)),
              "dg_stage_tile")
        return t.value

    def rk_stage_elem(self, u_in, u_out, res, stage: int, dt_elem, stream=None):
        """dg_rk_stage_elem: one LSERK4 stage with the per-element steps dt_elem
        (a device FP32 tensor of K entries)."""
        check(self._lib.dg_rk_stage_elem(self._h, _devptr(u_in), _devptr(u_out), _devptr(res),
                                         int(stage), _devptr(dt_elem), _stream_handle(stream)),
              "dg_rk_stage_elem")

    @staticmethod
    def rk_stage_multi(meshes, u_in, u_out, res, stage: int, dt: float = 1.0, dt_elem=None,
                       tile_cost=None, stream=None):
        """dg_rk_stage_multi: one LSERK4 stage of several meshes in shared
        launches (orders 1..4 in one, 5..6 in another); dt_elem is a list of
        device FP32 step tensors (or None entries / None: the scalar dt) and
        tile_cost a list of per-mesh tile costs (None: library defaults)."""
        lib = load()
        n = len(meshes)
        arr = lambda xs: (C.c_void_p * n)(*[None if x is None else _devptr_any(x).value for x in xs])  # noqa: E731
        hs = (C.c_void_p * n)(*[m._h.value for m in meshes])
        dts = None if dt_elem is None else arr(dt_elem)
        costs = None if tile_cost is None else (C.c_double * n)(*[float(c) for c in tile_cost])
        for xs in (u_in, u_out, res):
            for x in xs:
                _devptr(x)
        check(lib.dg_rk_stage_multi(hs, n, arr(u_in), arr(u_out), arr(res), dts, int(stage),
                                    float(dt), costs, _stream_handle(stream)), "dg_rk_stage_multi")

    def energy(self, u, stream=None) -> float:
        out = C.c_double()
        check(self._lib.dg_energy(self._h, _devptr(u), C.byref(out), _stream_handle(stream)),
              "dg_energy")
        return out.value

    def energy_range(self, u, k0: int, k1: int, stream=None) -> float:
        """dg_energy_range: the energy of elements k0 <= k < k1."""
        out = C.c_double()
        check(self._lib.dg_energy_range(self._h, _devptr(u), int(k0), int(k1), C.byref(out),
                                        _stream_handle(stream)), "dg_energy_range")
        return out.value

    def energy_noalloc(self, u, out, stream=None):
        """Energy into the device double `out` (a CUDA tensor or pointer); allocates nothing."""
        check(self._lib.dg_energy_noalloc(self._h, _devptr(u), _devptr_any(out),
                                          _stream_handle(stream)), "dg_energy_noalloc")
        return out

    def step_host(self, u_host, res_host, dt: float, nsteps: int, with_energy=True, stream=None):
        """u_host, res_host: host float32 buffers (NumPy arrays or pinned CPU
        tensors); res_host may be None (only u crosses the bus)."""
        def hptr(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float32 and a.flags.c_contiguous
                return C.c_void_p(a.ctypes.data)
            assert (not a.is_cuda) and a.is_contiguous()
            return C.c_void_p(a.data_ptr())
        e = C.c_double()
        check(self._lib.dg_step_host(self._h, hptr(u_host), hptr(res_host), float(dt), int(nsteps),
                                     C.byref(e) if with_energy else None, _stream_handle(stream)),
              "dg_step_host")
        return e.value if with_energy else None

    def last_launch_count(self) -> int:
        return int(self._lib.dg_last_launch_count(self._h))

    def trace_enable(self, n: int):
        """Clear the launch trace and reserve n launches (n = 0: tracing off)."""
        check(self._lib.dg_trace_enable(self._h, int(n)), "dg_trace_enable")

    def trace_read(self):
        """(durations in ms, kernel kinds) of the launches traced so far."""
        cnt = C.c_int64()
        check(self._lib.dg_trace_read(self._h, None, None, 0, C.byref(cnt)), "dg_trace_read")
        ms, kind = np.empty(cnt.value), np.empty(cnt.value, np.int32)
        check(self._lib.dg_trace_read(self._h, _dptr(ms, np.float64), _dptr(kind, np.int32),
                                      cnt.value, C.byref(cnt)), "dg_trace_read")
        return ms, kind
