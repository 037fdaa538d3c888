"""Python binding of libmcsteklov (the B300 Monte Carlo DtN / Steklov library).

Argument marshalling only: every step runs in the library's CUDA kernels,
declared in include/mcsteklov.h.  PyTorch provides device memory and the
current CUDA stream.  There is no CPU fallback: importing this module loads
the compiled library and raises if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

__all__ = ["lib", "Mesh", "default_params", "vertex_rows", "closest_points", "philox_words", "estimate_dtn",
           "workspace_size", "steklov_modes", "tc_symm_product", "MCSError", "Batch", "sample_rows", "sample_rows_batched",
           "estimate_dtn_noalloc", "dense_hist"]

_LIB_PATH = _build.LIB


class MCSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mcsteklov status {status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("cap_deg", C.c_double), ("bisect_iters", C.c_int), ("kappa", C.c_double),
                ("max_steps", C.c_int), ("rho_min_factor", C.c_double), ("prec", C.c_int), ("domain", C.c_int),
                ("origin_auto", C.c_int), ("origin", C.c_double * 3), ("killing_walks", C.c_longlong),
                ("seed", C.c_uint64), ("walks_per_row", C.c_int), ("blocks_per_sm", C.c_int),
                ("threads_per_block", C.c_int), ("timing", C.c_int), ("count_work", C.c_int),
                ("queue_order", C.c_int), ("bvh_layout", C.c_int), ("lanes_per_query", C.c_int),
                ("start_mode", C.c_int), ("inset", C.c_double)]


class Rows(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("pos", C.c_void_p), ("nrm", C.c_void_p), ("area", C.c_void_p),
                ("tri2bin", C.c_void_p)]


class Outputs(C.Structure):
    _fields_ = [("hist_bin", C.c_void_p), ("hist_cnt", C.c_void_p), ("hist_nnz", C.c_void_p),
                ("Lambda", C.c_void_p), ("omega", C.c_void_p), ("H0", C.c_void_p), ("exit_tri", C.c_void_p),
                ("Lambda32", C.c_void_p), ("exit_bary", C.c_void_p), ("walk_w", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("walks", C.c_longlong), ("steps", C.c_longlong), ("capped", C.c_longlong), ("lost", C.c_longlong),
                ("discarded_rows", C.c_longlong), ("killing_steps", C.c_longlong),
                ("killing_capped", C.c_longlong), ("origin", C.c_double * 3), ("rmax", C.c_double),
                ("device_error", C.c_int), ("phase_ms", C.c_float * 4), ("nodes_visited", C.c_longlong),
                ("tris_tested", C.c_longlong)]


class BatchItem(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("rows", Rows), ("domain", C.c_int), ("origin_auto", C.c_int),
                ("origin", C.c_double * 3), ("seed", C.c_uint64), ("out", Outputs)]


class SampleItem(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("n", C.c_int), ("sel", C.c_void_p), ("pos", C.c_void_p), ("nrm", C.c_void_p),
                ("area", C.c_void_p), ("tri2bin", C.c_void_p), ("orient_gap", C.c_void_p)]


class TuneTrial(C.Structure):
    _fields_ = [("threads_per_block", C.c_int), ("blocks_per_sm", C.c_int), ("queue_order", C.c_int),
                ("bvh_layout", C.c_int), ("lanes_per_query", C.c_int), ("ms", C.c_float)]


class EigParams(C.Structure):
    _fields_ = [("degree", C.c_int), ("max_iters", C.c_int), ("tol", C.c_double), ("product", C.c_int)]


class EigStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("block", C.c_int), ("tc_products", C.c_int),
                ("upper_bound", C.c_double), ("max_residual", C.c_double), ("device_error", C.c_int),
                ("product", C.c_int), ("nnz", C.c_longlong), ("jacobi_sweeps", C.c_int)]


_lib = None


def lib():
    """Load libmcsteklov.so (built in-tree by ``build.py``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libmcsteklov.so not found at {_LIB_PATH}: run paper_2606_05581_b300/build.py")
        L = C.CDLL(_LIB_PATH)
        vp, i32, i64, u64, u32, dbl = C.c_void_p, C.c_int, C.c_longlong, C.c_uint64, C.c_uint32, C.c_double
        L.mcs_last_error.restype = C.c_char_p
        L.mcs_version.restype = C.c_char_p
        L.mcs_launch_count.restype = C.c_ulonglong
        L.mcs_default_params.argtypes = [C.POINTER(Params)]
        L.mcs_build_bvh.argtypes = [vp, i32, vp, i32, vp, C.POINTER(vp)]
        L.mcs_build_bvh_batched.argtypes = [i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(vp), C.POINTER(i32), vp,
                                            C.POINTER(vp)]
        L.mcs_mesh_destroy.argtypes = [vp]
        L.mcs_mesh_nv.argtypes = [vp]
        L.mcs_mesh_nf.argtypes = [vp]
        L.mcs_mesh_build_wide.argtypes = [vp, vp]
        L.mcs_mesh_has_wide.argtypes = [vp]
        L.mcs_vertex_rows.argtypes = [vp, vp, vp, vp, vp]
        L.mcs_closest_points.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp]
        L.mcs_estimate_workspace_size.argtypes = [vp, i32, i32, i64]
        L.mcs_estimate_workspace_size.restype = C.c_size_t
        L.mcs_estimate_dtn.argtypes = [vp, C.POINTER(Rows), C.POINTER(Params), C.POINTER(Outputs), vp, C.c_size_t,
                                       C.POINTER(Stats), vp]
        L.mcs_philox_words.argtypes = [u64, u64, u32, u32, u32, u32, vp, vp]
        L.mcs_probe_l2_read.argtypes = [vp, C.c_size_t, i32, vp, vp]
        L.mcs_probe_fma32.argtypes = [i32, vp, vp]
        L.mcs_probe_fma64.argtypes = [i32, vp, vp]
        L.mcs_probe_threads.restype = i64
        L.mcs_sample_rows_workspace_size.argtypes = [vp, i32]
        L.mcs_sample_rows_workspace_size.restype = C.c_size_t
        L.mcs_sample_rows.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, C.c_size_t, vp]
        L.mcs_sample_rows_batched_workspace_size.argtypes = [C.POINTER(SampleItem), i32]
        L.mcs_sample_rows_batched_workspace_size.restype = C.c_size_t
        L.mcs_sample_rows_batched.argtypes = [C.POINTER(SampleItem), i32, i32, vp, C.c_size_t, vp]
        L.mcs_estimate_dtn_noalloc_capacity.restype = C.c_size_t
        L.mcs_estimate_dtn_noalloc.argtypes = [vp, C.POINTER(Rows), C.POINTER(Params), C.POINTER(Outputs),
                                               C.POINTER(Stats), vp]
        L.mcs_estimate_batched_workspace_size.argtypes = [C.POINTER(BatchItem), i32, i32]
        L.mcs_estimate_batched_workspace_size.restype = C.c_size_t
        L.mcs_estimate_batched.argtypes = [C.POINTER(BatchItem), i32, C.POINTER(Params), vp, C.c_size_t,
                                           C.POINTER(Stats), C.POINTER(Stats), vp]
        L.mcs_graph_create.argtypes = [C.POINTER(BatchItem), i32, C.POINTER(Params), vp, C.c_size_t, C.POINTER(vp)]
        L.mcs_graph_launch.argtypes = [vp, vp]
        L.mcs_graph_stats.argtypes = [vp, C.POINTER(Stats), C.POINTER(Stats), vp]
        L.mcs_graph_nodes.argtypes = [vp]
        L.mcs_graph_nodes.restype = C.c_size_t
        L.mcs_graph_destroy.argtypes = [vp]
        L.mcs_autotune_walks.argtypes = [C.POINTER(BatchItem), i32, C.POINTER(Params), vp, C.c_size_t, dbl,
                                         C.POINTER(Params), C.POINTER(TuneTrial), i32, C.POINTER(i32), vp]
        L.mcs_default_eig_params.argtypes = [C.POINTER(EigParams)]
        L.mcs_steklov_workspace_size.argtypes = [i32, i32]
        L.mcs_steklov_workspace_size.restype = C.c_size_t
        L.mcs_steklov_modes.argtypes = [vp, vp, i32, i32, vp, vp, vp, C.c_size_t, C.POINTER(EigParams),
                                        C.POINTER(EigStats), vp]
        L.mcs_cotan_laplacian.argtypes = [vp, vp, vp]
        L.mcs_galerkin_workspace_size.argtypes = [vp, i32, i32]
        L.mcs_galerkin_workspace_size.restype = C.c_size_t
        L.mcs_galerkin_dtn.argtypes = [vp, C.POINTER(Rows), vp, vp, vp, vp, vp, i32, i32, i32, C.POINTER(C.c_double),
                                       vp, i64, vp, i32, vp, vp, vp, C.c_size_t, vp]
        L.mcs_galerkin_modes.argtypes = [vp, i32, i32, vp, i32, vp, vp, vp, vp]
        L.mcs_steklov_heat_workspace_size.argtypes = [i32, i32, i32]
        L.mcs_steklov_heat_workspace_size.restype = C.c_size_t
        L.mcs_steklov_heat.argtypes = [vp, vp, vp, i32, i32, vp, i32, vp, i32, vp, vp, C.c_size_t, vp]
        L.mcs_hks.argtypes = [vp, vp, i32, i32, vp, i32, vp, vp]
        L.mcs_galerkin_project_workspace_size.argtypes = [i32, i32]
        L.mcs_galerkin_project_workspace_size.restype = C.c_size_t
        L.mcs_galerkin_project.argtypes = [vp, vp, i32, i32, vp, vp, C.c_size_t, vp]
        L.mcs_points_workspace_size.argtypes = [i32]
        L.mcs_points_workspace_size.restype = C.c_size_t
        L.mcs_point_knn.argtypes = [vp, vp, i32, vp, vp, i32, i32, dbl, dbl, i32, vp, vp, vp, vp, C.c_size_t, vp]
        L.mcs_point_laplacian.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, C.c_size_t, vp]
        L.mcs_point_galerkin_lambda.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32, i32, C.POINTER(C.c_double), vp,
                                                i64, i32, dbl, dbl, vp, vp, C.c_size_t, vp]
        L.mcs_tc_symm_product_workspace_size.argtypes = [i32, i32]
        L.mcs_tc_symm_product_workspace_size.restype = C.c_size_t
        L.mcs_tc_symm_product.argtypes = [vp, vp, i32, i32, vp, vp, C.c_size_t, vp]
        _lib = L
    return _lib


def launch_count() -> int:
    """Library kernels enqueued since load (instrumentation)."""
    return int(lib().mcs_launch_count())


def _check(status):
    if status < 0:
        raise MCSError(status, lib().mcs_last_error().decode())
    return status


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def default_params(**kw) -> Params:
    p = Params()
    lib().mcs_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "origin":
            p.origin_auto = 0
            for i in range(3):
                p.origin[i] = float(v[i])
        else:
            setattr(p, k, v)
    return p


def _mesh_arrays(V, F):
    V = V if isinstance(V, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(V, np.float64))
    F = F if isinstance(F, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(F, np.int32))
    return V.to(torch.float64).contiguous(), F.to(torch.int32).contiguous()


def build_meshes(pairs) -> "list[Mesh]":
    """Many meshes, [(V, F), ...], built by mcs_build_bvh_batched: every
    build enqueued before one synchronisation."""
    arrs = [_mesh_arrays(V, F) for V, F in pairs]
    n = len(arrs)
    Vp = (C.c_void_p * n)(*[V.data_ptr() for V, _ in arrs])
    Fp = (C.c_void_p * n)(*[F.data_ptr() for _, F in arrs])
    nv = (C.c_int * n)(*[int(V.shape[0]) for V, _ in arrs])
    nf = (C.c_int * n)(*[int(F.shape[0]) for _, F in arrs])
    out = (C.c_void_p * n)()
    _check(lib().mcs_build_bvh_batched(n, Vp, nv, Fp, nf, _stream(), out))
    return [Mesh._adopt(C.c_void_p(out[i]), V, F) for i, (V, F) in enumerate(arrs)]


class Mesh:
    """A mesh on the device with its BVH (owned by the library)."""

    def __init__(self, V, F):
        V, F = _mesh_arrays(V, F)
        self._keep = (V, F)
        h = C.c_void_p()
        _check(lib().mcs_build_bvh(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _stream(), C.byref(h)))
        self.handle = h
        self.nv = int(V.shape[0])
        self.nf = int(F.shape[0])

    @classmethod
    def _adopt(cls, handle, V, F):
        obj = cls.__new__(cls)
        obj._keep = (V, F)
        obj.handle = handle
        obj.nv = int(V.shape[0])
        obj.nf = int(F.shape[0])
        return obj

    def build_wide(self):
        """Build the 4-wide BVH (bvh_layout 4) of this mesh."""
        _check(lib().mcs_mesh_build_wide(self.handle, _stream()))
        return self

    def close(self):
        if self.handle:
            lib().mcs_mesh_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vertex_rows(mesh: Mesh):
    dev = torch.device("cuda")
    pos = torch.empty((mesh.nv, 3), dtype=torch.float64, device=dev)
    nrm = torch.empty_like(pos)
    area = torch.empty(mesh.nv, dtype=torch.float64, device=dev)
    _check(lib().mcs_vertex_rows(mesh.handle, _ptr(pos), _ptr(nrm), _ptr(area), _stream()))
    return dict(pos=pos, nrm=nrm, area=area, tri2bin=None)


def sample_rows(mesh: Mesh, n: int, orient: "bool | int" = True, workspace: "Workspace | None" = None):
    """Farthest-point sample rows with Voronoi areas and oriented face normals
    (orient: 0 none; 3 hierarchical winding numbers with brute force where the
    certified bound does not decide; 2 brute force for every row; 1 / True
    the first for faces x rows >= 2^28, else the second)."""
    dev = torch.device("cuda")
    sel = torch.empty(n, dtype=torch.int32, device=dev)
    pos = torch.empty((n, 3), dtype=torch.float64, device=dev)
    nrm = torch.empty((n, 3), dtype=torch.float64, device=dev)
    area = torch.empty(n, dtype=torch.float64, device=dev)
    t2b = torch.empty(mesh.nf, dtype=torch.int32, device=dev)
    gap = torch.empty(n, dtype=torch.float32, device=dev)
    nb = int(lib().mcs_sample_rows_workspace_size(mesh.handle, n))
    ws = (workspace or Workspace()).get(nb)
    _check(lib().mcs_sample_rows(mesh.handle, n, int(orient), _ptr(sel), _ptr(pos), _ptr(nrm), _ptr(area), _ptr(t2b),
                                 _ptr(gap), C.c_void_p(_aligned_ptr(ws)), nb, _stream()))
    return dict(pos=pos, nrm=nrm, area=area, tri2bin=t2b, sel=sel, gap=gap)


def sample_rows_batched(meshes: list, n: int, orient: bool = True) -> list:
    """Farthest-point sample rows of many meshes, their sampling in one launch."""
    dev = torch.device("cuda")
    outs = []
    arr = (SampleItem * len(meshes))()
    for i, mesh in enumerate(meshes):
        o = dict(sel=torch.empty(n, dtype=torch.int32, device=dev),
                 pos=torch.empty((n, 3), dtype=torch.float64, device=dev),
                 nrm=torch.empty((n, 3), dtype=torch.float64, device=dev),
                 area=torch.empty(n, dtype=torch.float64, device=dev),
                 tri2bin=torch.empty(mesh.nf, dtype=torch.int32, device=dev),
                 gap=torch.empty(n, dtype=torch.float32, device=dev))
        arr[i] = SampleItem(mesh.handle, n, o["sel"].data_ptr(), o["pos"].data_ptr(), o["nrm"].data_ptr(),
                            o["area"].data_ptr(), o["tri2bin"].data_ptr(), o["gap"].data_ptr())
        outs.append(o)
    nb = int(lib().mcs_sample_rows_batched_workspace_size(arr, len(meshes)))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    _check(lib().mcs_sample_rows_batched(arr, len(meshes), int(orient), C.c_void_p(_aligned_ptr(ws)), nb, _stream()))
    return outs


def closest_points(mesh: Mesh, P: torch.Tensor, prec: int = 64, layout: int = 2):
    P = P.to(device="cuda", dtype=torch.float64).contiguous()
    n = P.shape[0]
    d2 = torch.empty(n, dtype=torch.float64, device="cuda")
    tri = torch.empty(n, dtype=torch.int32, device="cuda")
    bary = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    _check(lib().mcs_closest_points(mesh.handle, _ptr(P), n, prec, layout, _ptr(d2), _ptr(tri), _ptr(bary),
                                    _stream()))
    return d2, tri, bary


def philox_words(start: int, n: int, c2: int, c3: int, key: int) -> torch.Tensor:
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    _check(lib().mcs_philox_words(start, n, c2, c3, key & 0xFFFFFFFF, key >> 32, _ptr(out), _stream()))
    return out


def probe_peaks(l2_sizes_mib=(8, 16, 32, 64, 96), pass_bytes: int = 8 << 30) -> dict:
    """Ceilings of the running GPU for the walk kernel's roofline, each the
    best of 3 event-timed calls of the library's probes: L2 read bandwidth
    (GB/s; L1-bypassing loads over device buffers below the L2 size, the best
    size taken) and FP32 / FP64 fused multiply-add instruction rates (T
    instructions/s)."""
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.int64, device=dev)

    def best(fn, k=3):
        fn()
        out = []
        for _ in range(k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b) / 1e3)
        return min(out)

    l2 = {}
    for mib in l2_sizes_mib:
        buf = torch.ones(mib << 20, dtype=torch.uint8, device=dev)
        reps = max(1, pass_bytes // buf.numel())
        t = best(lambda: _check(lib().mcs_probe_l2_read(_ptr(buf), buf.numel(), reps, _ptr(sink), _stream())))
        l2[mib] = buf.numel() * reps / t / 1e9
        del buf
    th = int(lib().mcs_probe_threads())
    o32 = torch.zeros(1, dtype=torch.float32, device=dev)
    o64 = torch.zeros(1, dtype=torch.float64, device=dev)
    i32, i64 = 16384, 256
    t32 = best(lambda: _check(lib().mcs_probe_fma32(i32, _ptr(o32), _stream())))
    t64 = best(lambda: _check(lib().mcs_probe_fma64(i64, _ptr(o64), _stream())))
    return {"l2_read_gbs": max(l2.values()), "l2_read_gbs_by_mib": l2,
            "fp32_fma_tinst_s": th * 8 * i32 / t32 / 1e12, "fp64_fma_tinst_s": th * 8 * i64 / t64 / 1e12,
            "probe_threads": th}


def workspace_size(mesh: Mesh, n_rows: int, walks: int, killing_walks: int = 0) -> int:
    return int(lib().mcs_estimate_workspace_size(mesh.handle, n_rows, walks, killing_walks))


class Workspace:
    """Caller-owned device scratch for estimate_dtn, grown on demand."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes + 256:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        return self.buf


def _aligned_ptr(buf: torch.Tensor) -> int:
    p = buf.data_ptr()
    return (p + 255) & ~255


_OUT_KEYS = ("hist_bin", "hist_cnt", "hist_nnz", "Lambda", "omega", "H0", "exit_tri", "Lambda32", "exit_bary",
             "walk_w")


def _alloc_outputs(R: int, W: int, dev, assemble: bool, record_exits: bool, fp32_copy: bool = False,
                   record_bary: bool = False) -> dict:
    cap = min(W, R)
    return dict(hist_bin=torch.empty(R * cap, dtype=torch.int32, device=dev),
                hist_cnt=torch.empty(R * cap, dtype=torch.int32, device=dev),
                hist_nnz=torch.empty(R, dtype=torch.int32, device=dev),
                omega=torch.empty(R, dtype=torch.float64, device=dev),
                H0=torch.empty(R, dtype=torch.int32, device=dev),
                Lambda=torch.empty((R, R), dtype=torch.float64, device=dev) if assemble else None,
                exit_tri=torch.empty((R, W), dtype=torch.int32, device=dev) if record_exits else None,
                Lambda32=torch.empty((R, R), dtype=torch.float32, device=dev) if (assemble and fp32_copy) else None,
                exit_bary=torch.empty((R, W, 3), dtype=torch.float64, device=dev) if record_bary else None,
                walk_w=torch.empty((R, W), dtype=torch.float64, device=dev) if record_bary else None)


def _rows_struct(rows: dict) -> Rows:
    t2b = rows.get("tri2bin")
    return Rows(int(rows["pos"].shape[0]), rows["pos"].data_ptr(), rows["nrm"].data_ptr(), rows["area"].data_ptr(),
                None if t2b is None else t2b.data_ptr())


def _outputs_struct(o: dict) -> Outputs:
    return Outputs(*[None if o.get(k) is None else o[k].data_ptr() for k in _OUT_KEYS])


def _stats_dict(st: Stats) -> dict:
    return {k: (list(getattr(st, k)) if k in ("origin", "phase_ms") else getattr(st, k)) for k, _ in Stats._fields_}


def estimate_dtn(mesh: Mesh, rows: dict, params: Params, assemble: bool = True, want_stats: bool = True,
                 record_exits: bool = False, workspace: Workspace | None = None, outputs: dict | None = None,
                 fp32_copy: bool = False, record_bary: bool = False):
    """Run the DtN estimator; returns a dict of device tensors (+ stats).
    record_exits / record_bary: also each walk's exit triangle / exit barycentrics."""
    pos = rows["pos"]
    R = int(pos.shape[0])
    W = int(params.walks_per_row)
    cap = min(W, R)
    o = outputs or _alloc_outputs(R, W, pos.device, assemble, record_exits, fp32_copy, record_bary)
    rs = _rows_struct(rows)
    out = _outputs_struct(o)
    nbytes = workspace_size(mesh, R, W, params.killing_walks)
    ws = (workspace or Workspace()).get(nbytes)
    st = Stats()
    status = _check(lib().mcs_estimate_dtn(mesh.handle, C.byref(rs), C.byref(params), C.byref(out),
                                           C.c_void_p(_aligned_ptr(ws)), nbytes, C.byref(st) if want_stats else None,
                                           _stream()))
    res = dict(o)
    res["cap"] = cap
    res["walks"] = W
    res["status"] = status
    res["_ws"] = ws
    if want_stats:
        res["stats"] = _stats_dict(st)
    return res


class Batch:
    """Many meshes in one persistent walk launch (mcs_estimate_batched).

    ``items``: list of dicts with keys mesh (Mesh), rows (dict of device
    tensors as for estimate_dtn), domain (0 interior, 1 exterior), seed and
    optionally origin (exterior inversion centre; automatic otherwise).
    Outputs are allocated per mesh (``self.outputs[i]``) unless given."""

    def __init__(self, items: list, params: Params, assemble: bool = True, record_exits: bool = False,
                 outputs: list | None = None):
        self.params = params
        self.items = items
        W = int(params.walks_per_row)
        self.outputs = outputs or [_alloc_outputs(int(it["rows"]["pos"].shape[0]), W, it["rows"]["pos"].device,
                                                  assemble, record_exits) for it in items]
        arr = (BatchItem * len(items))()
        for i, it in enumerate(items):
            b = arr[i]
            b.mesh = it["mesh"].handle
            b.rows = _rows_struct(it["rows"])
            b.domain = int(it.get("domain", 0))
            org = it.get("origin")
            b.origin_auto = 1 if org is None else 0
            if org is not None:
                for k in range(3):
                    b.origin[k] = float(org[k])
            b.seed = int(it.get("seed", 0))
            b.out = _outputs_struct(self.outputs[i])
        self._arr = arr
        self.nbytes = int(lib().mcs_estimate_batched_workspace_size(arr, len(items), W))
        self._ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        self.ws_ptr = C.c_void_p(_aligned_ptr(self._ws))
        self.graph = None

    def __len__(self):
        return len(self.items)

    def run(self, params: Params | None = None, want_stats: bool = True, check: bool = True):
        """Enqueue the batch; returns (status, total stats, per-mesh stats) when
        want_stats (check=False: an error status is returned, not raised)."""
        p = params or self.params
        n = len(self.items)
        tot = Stats()
        per = (Stats * n)()
        status = lib().mcs_estimate_batched(self._arr, n, C.byref(p), self.ws_ptr, self.nbytes,
                                            C.byref(tot) if want_stats else None, per if want_stats else None,
                                            _stream())
        if check:
            _check(status)
        if not want_stats:
            return status, None, None
        t = _stats_dict(tot)
        if status < 0:
            t["error"] = lib().mcs_last_error().decode()
        return status, t, [_stats_dict(per[i]) for i in range(n)]

    def autotune(self, sample_fraction: float = 1.0 / 64, max_trials: int = 32):
        """Time the walk launch on a sample for candidate launch shapes and queue orders;
        sets and returns the tuned params and the trial list."""
        n = len(self.items)
        tuned = Params()
        trials = (TuneTrial * max_trials)()
        nt = C.c_int(0)
        _check(lib().mcs_autotune_walks(self._arr, n, C.byref(self.params), self.ws_ptr, self.nbytes,
                                        float(sample_fraction), C.byref(tuned), trials, max_trials, C.byref(nt),
                                        _stream()))
        self.params = tuned
        self.close_graph()
        out = [dict(threads_per_block=t.threads_per_block, blocks_per_sm=t.blocks_per_sm,
                    queue_order=t.queue_order, bvh_layout=t.bvh_layout, lanes_per_query=t.lanes_per_query,
                    ms=t.ms)
               for t in trials[:min(nt.value, max_trials)]]
        return tuned, out

    def capture(self):
        """Capture the batch into a CUDA graph (mcs_graph_create)."""
        self.close_graph()
        h = C.c_void_p()
        _check(lib().mcs_graph_create(self._arr, len(self.items), C.byref(self.params), self.ws_ptr, self.nbytes,
                                      C.byref(h)))
        self.graph = h
        return int(lib().mcs_graph_nodes(h))

    def launch(self):
        if not self.graph:
            self.capture()
        _check(lib().mcs_graph_launch(self.graph, _stream()))

    def graph_stats(self, check: bool = True):
        """(status, total stats, per-mesh stats) of the last replay; check=False
        returns an error status (and its message as 'error' in the totals)
        instead of raising."""
        n = len(self.items)
        tot = Stats()
        per = (Stats * n)()
        status = lib().mcs_graph_stats(self.graph, C.byref(tot), per, _stream())
        if check:
            _check(status)
        t = _stats_dict(tot)
        if status < 0:
            t["error"] = lib().mcs_last_error().decode()
        return status, t, [_stats_dict(per[i]) for i in range(n)]

    def close_graph(self):
        if self.graph:
            lib().mcs_graph_destroy(self.graph)
            self.graph = None

    def result(self, i: int) -> dict:
        """Per-mesh outputs in the layout estimate_dtn returns."""
        R = int(self.items[i]["rows"]["pos"].shape[0])
        W = int(self.params.walks_per_row)
        res = dict(self.outputs[i])
        res["cap"] = min(W, R)
        res["walks"] = W
        return res

    def __del__(self):
        try:
            self.close_graph()
        except Exception:
            pass


def dense_hist(res: dict, R: int) -> torch.Tensor:
    """Padded CSR -> dense R x R int32 hit counts (for tests and small cases)."""
    cap = res["cap"]
    nnz = res["hist_nnz"].long()
    idx = torch.arange(cap, device=nnz.device)[None, :] < nnz[:, None]
    rows = torch.arange(R, device=nnz.device)[:, None].expand(R, cap)[idx]
    bins = res["hist_bin"].view(R, cap)[idx].long()
    cnts = res["hist_cnt"].view(R, cap)[idx]
    H = torch.zeros((R, R), dtype=torch.int32, device=nnz.device)
    H[rows, bins] = cnts
    return H


def default_eig_params(**kw) -> EigParams:
    p = EigParams()
    lib().mcs_default_eig_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def steklov_modes(Lambda: torch.Tensor, mass: torch.Tensor, k: int, params: EigParams | None = None,
                  vectors: bool = True, workspace: Workspace | None = None):
    """Smallest k eigenpairs of Lambda psi = lambda M psi; returns (evals, evecs, stats)."""
    n = int(Lambda.shape[0])
    L = Lambda.contiguous()
    M = mass.to(torch.float64).contiguous()
    ev = torch.empty(k, dtype=torch.float64, device=L.device)
    X = torch.empty((n, k), dtype=torch.float64, device=L.device) if vectors else None
    nb = int(lib().mcs_steklov_workspace_size(n, k))
    ws = (workspace or Workspace()).get(nb)
    st = EigStats()
    status = _check(lib().mcs_steklov_modes(_ptr(L), _ptr(M), n, k, _ptr(ev), _ptr(X), C.c_void_p(_aligned_ptr(ws)),
                                            nb, C.byref(params) if params is not None else None, C.byref(st),
                                            _stream()))
    stats = {f: getattr(st, f) for f, _ in EigStats._fields_}
    stats["status"] = status
    return ev, X, stats


def cotan_laplacian(mesh: Mesh) -> torch.Tensor:
    """Dense cotangent Laplacian of the mesh (nv x nv FP64, device)."""
    L = torch.empty((mesh.nv, mesh.nv), dtype=torch.float64, device="cuda")
    _check(lib().mcs_cotan_laplacian(mesh.handle, _ptr(L), _stream()))
    return L


def galerkin_dtn(mesh: Mesh, rows: dict, res: dict, Phi: torch.Tensor, exterior: bool = False,
                 killing_walks: int = 0, want_lambda: bool = False, workspace: "Workspace | None" = None,
                 start_mode: int = 0):
    """Galerkin estimate S = Phi^T Lambda_bary Phi (K x K) from an estimate
    recorded with record_exits and record_bary; rows as given to that
    estimate (sample rows: their "sel" faces are the row points' faces).
    start_mode: that of the estimate (1: per-walk weights; 2: the naive
    form).  Returns S, or (S, Lambda_bary) with want_lambda."""
    P = Phi.to(torch.float64).contiguous()
    K = int(P.shape[1])
    S = torch.empty((K, K), dtype=torch.float64, device=P.device)
    Lb = torch.empty((mesh.nv, mesh.nv), dtype=torch.float64, device=P.device) if want_lambda else None
    rs = _rows_struct(rows)
    sel = rows.get("sel") if rows.get("tri2bin") is not None else None
    origin = (C.c_double * 3)(*res["stats"]["origin"])
    nb = int(lib().mcs_galerkin_workspace_size(mesh.handle, K, 0 if want_lambda else 1))
    if nb == 0:
        raise MCSError("galerkin_dtn: K must be a multiple of 16 in [16, 160]")
    ws = (workspace or Workspace()).get(nb)
    H0 = res.get("H0") if (exterior and killing_walks > 0) else None
    ww = res.get("walk_w") if start_mode == 1 else None
    form = 1 if start_mode == 2 else 0
    _check(lib().mcs_galerkin_dtn(mesh.handle, C.byref(rs), _ptr(sel), _ptr(res["omega"]), _ptr(res["exit_tri"]),
                                  _ptr(res["exit_bary"]), _ptr(ww), form, int(res["walks"]), int(exterior), origin,
                                  _ptr(H0),
                                  int(killing_walks), _ptr(P), K, _ptr(S), _ptr(Lb), C.c_void_p(_aligned_ptr(ws)), nb,
                                  _stream()))
    return (S, Lb) if want_lambda else S


def galerkin_modes(S: torch.Tensor, k: int, Phi: "torch.Tensor | None" = None):
    """Eigenpairs of the K x K Galerkin matrix: (evals K ascending, coeffs K x K,
    psi = Phi coeffs[:, :k] or None)."""
    S = S.to(torch.float64).contiguous()
    K = int(S.shape[0])
    ev = torch.empty(K, dtype=torch.float64, device=S.device)
    Cm = torch.empty((K, K), dtype=torch.float64, device=S.device)
    psi = None
    n = 0
    if Phi is not None:
        Phi = Phi.to(torch.float64).contiguous()
        n = int(Phi.shape[0])
        psi = torch.empty((n, k), dtype=torch.float64, device=S.device)
    _check(lib().mcs_galerkin_modes(_ptr(S), K, k, _ptr(Phi), n, _ptr(ev), _ptr(Cm), _ptr(psi), _stream()))
    return ev, Cm, psi


def galerkin_project(Lam: torch.Tensor, Phi: torch.Tensor, workspace: "Workspace | None" = None) -> torch.Tensor:
    """S = Phi^T Lam Phi (K x K FP64) for a symmetric n x n Lam (tensor-core product)."""
    Lam = Lam.to(torch.float64).contiguous()
    P = Phi.to(torch.float64).contiguous()
    n, K = int(P.shape[0]), int(P.shape[1])
    S = torch.empty((K, K), dtype=torch.float64, device=P.device)
    nb = int(lib().mcs_galerkin_project_workspace_size(n, K))
    if nb == 0:
        raise MCSError("galerkin_project: need n >= 16 and K a multiple of 16 in [16, 160]")
    ws = (workspace or Workspace()).get(nb)
    _check(lib().mcs_galerkin_project(_ptr(Lam), _ptr(P), n, K, _ptr(S), C.c_void_p(_aligned_ptr(ws)), nb,
                                      _stream()))
    return S


# point-based Galerkin basis (Sec. 4.4; appendix "Point-based k-NN Interpolator")
KNN_K, KNN_SIGMA, KNN_TAU = 8, 0.025, 0.8


def _points_ws(n: int, workspace):
    nb = int(lib().mcs_points_workspace_size(n))
    return nb, (workspace or Workspace()).get(nb)


def point_knn(P: torch.Tensor, NP: "torch.Tensor | None", Q: torch.Tensor, NQ: "torch.Tensor | None" = None,
              k: int = KNN_K, sigma: float = KNN_SIGMA, tau_n: float = KNN_TAU, exclude_self: bool = False,
              weights: bool = True, workspace: "Workspace | None" = None):
    """The k nearest points of P to each query of Q (exact FP64 distances, ties
    by index) and, with weights, the bilateral interpolation weights (needs the
    point normals NP and query normals NQ).  Returns (idx, w or None, d2)."""
    P = P.to(torch.float64).contiguous()
    Q = Q.to(torch.float64).contiguous()
    n, nq = int(P.shape[0]), int(Q.shape[0])
    dev = P.device
    idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float64, device=dev)
    w = torch.empty((nq, k), dtype=torch.float64, device=dev) if weights else None
    NPc = NP.to(torch.float64).contiguous() if NP is not None else None
    NQc = NQ.to(torch.float64).contiguous() if NQ is not None else None
    nb, ws = _points_ws(n, workspace)
    _check(lib().mcs_point_knn(_ptr(P), _ptr(NPc), n, _ptr(Q), _ptr(NQc), nq, k, float(sigma), float(tau_n),
                               int(exclude_self), _ptr(idx), _ptr(w), _ptr(d2), C.c_void_p(_aligned_ptr(ws)), nb,
                               _stream()))
    return idx, w, d2


def point_laplacian(P: torch.Tensor, NP: torch.Tensor, k_nbr: int = 16, workspace: "Workspace | None" = None):
    """Point-cloud Laplacian from local tangent-plane Voronoi cells (dense
    n x n FP64).  Returns (L, cell_area, nbr, nbr_w)."""
    P = P.to(torch.float64).contiguous()
    NP = NP.to(torch.float64).contiguous()
    n = int(P.shape[0])
    dev = P.device
    L = torch.empty((n, n), dtype=torch.float64, device=dev)
    area = torch.empty(n, dtype=torch.float64, device=dev)
    nbr = torch.empty((n, k_nbr), dtype=torch.int32, device=dev)
    nbw = torch.empty((n, k_nbr), dtype=torch.float64, device=dev)
    nb, ws = _points_ws(n, workspace)
    _check(lib().mcs_point_laplacian(_ptr(P), _ptr(NP), n, k_nbr, _ptr(L), _ptr(area), _ptr(nbr), _ptr(nbw),
                                     C.c_void_p(_aligned_ptr(ws)), nb, _stream()))
    return L, area, nbr, nbw


def point_basis(rows: dict, K: int, k_nbr: int = 16, workspace: "Workspace | None" = None):
    """The point-based Galerkin basis: the K lowest generalised eigenvectors of
    the point-cloud Laplacian with the rows' areas as the mass (M-orthonormal,
    n x K).  Returns (Phi, evals, eig stats)."""
    L, _, _, _ = point_laplacian(rows["pos"], rows["nrm"], k_nbr, workspace)
    ev, Phi, st = steklov_modes(L, rows["area"], K)
    return Phi, ev, st


def point_galerkin_lambda(mesh: Mesh, rows: dict, res: dict, exterior: bool = False, killing_walks: int = 0,
                          k: int = KNN_K, sigma: float = KNN_SIGMA, tau_n: float = KNN_TAU,
                          workspace: "Workspace | None" = None) -> torch.Tensor:
    """Point-basis Galerkin matrix (n_rows x n_rows FP64) of an estimate whose
    rows are the points (recorded with record_exits and record_bary)."""
    P = rows["pos"].to(torch.float64).contiguous()
    NP = rows["nrm"].to(torch.float64).contiguous()
    n = int(P.shape[0])
    Lp = torch.empty((n, n), dtype=torch.float64, device=P.device)
    origin = (C.c_double * 3)(*res["stats"]["origin"])
    H0 = res.get("H0") if (exterior and killing_walks > 0) else None
    nb, ws = _points_ws(n, workspace)
    _check(lib().mcs_point_galerkin_lambda(mesh.handle, _ptr(P), _ptr(NP), n, _ptr(res["omega"]),
                                           _ptr(res["exit_tri"]), _ptr(res["exit_bary"]), int(res["walks"]),
                                           int(exterior), origin, _ptr(H0), int(killing_walks), k, float(sigma),
                                           float(tau_n), _ptr(Lp), C.c_void_p(_aligned_ptr(ws)), nb, _stream()))
    return Lp


def steklov_heat(evals: torch.Tensor, evecs: torch.Tensor, mass: torch.Tensor, u0: torch.Tensor,
                 times, workspace: "Workspace | None" = None) -> torch.Tensor:
    """Steklov heat u_t = sum_j exp(-lambda_j t) <u0, psi_j>_M psi_j for each time
    (u0: n or n x c); returns nt x n (x c) FP64 on the device."""
    dev = evecs.device
    ev = evals.to(device=dev, dtype=torch.float64).contiguous()
    X = evecs.to(torch.float64).contiguous()
    n, k = int(X.shape[0]), int(X.shape[1])
    M = mass.to(device=dev, dtype=torch.float64).contiguous()
    vec = u0.dim() == 1
    U = u0.to(device=dev, dtype=torch.float64).reshape(n, -1).contiguous()
    c = int(U.shape[1])
    T = torch.as_tensor(times, dtype=torch.float64).reshape(-1).to(dev).contiguous()
    nt = int(T.shape[0])
    out = torch.empty((nt, n, c), dtype=torch.float64, device=dev)
    nb = int(lib().mcs_steklov_heat_workspace_size(n, k, c))
    ws = (workspace or Workspace()).get(nb)
    _check(lib().mcs_steklov_heat(_ptr(ev), _ptr(X), _ptr(M), n, k, _ptr(U), c, _ptr(T), nt, _ptr(out),
                                  C.c_void_p(_aligned_ptr(ws)), nb, _stream()))
    return out[:, :, 0] if vec else out


def hks(evals: torch.Tensor, evecs: torch.Tensor, times) -> torch.Tensor:
    """Heat kernel signature sum_j exp(-lambda_j t) psi_j(x)^2; returns nt x n FP64 on the device."""
    dev = evecs.device
    ev = evals.to(device=dev, dtype=torch.float64).contiguous()
    X = evecs.to(torch.float64).contiguous()
    n, k = int(X.shape[0]), int(X.shape[1])
    T = torch.as_tensor(times, dtype=torch.float64).reshape(-1).to(dev).contiguous()
    out = torch.empty((int(T.shape[0]), n), dtype=torch.float64, device=dev)
    _check(lib().mcs_hks(_ptr(ev), _ptr(X), n, k, _ptr(T), int(T.shape[0]), _ptr(out), _stream()))
    return out


def tc_symm_product(A: torch.Tensor, Xt: torch.Tensor) -> torch.Tensor:
    """Test hook: (A X)^T via the tensor-core split product (A symmetric n x n, Xt m x n)."""
    n, m = int(A.shape[0]), int(Xt.shape[0])
    A = A.to(torch.float64).contiguous()
    Xt = Xt.to(torch.float64).contiguous()
    Zt = torch.empty_like(Xt)
    nb = int(lib().mcs_tc_symm_product_workspace_size(n, m))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=A.device)
    _check(lib().mcs_tc_symm_product(_ptr(A), _ptr(Xt), n, m, _ptr(Zt), C.c_void_p(_aligned_ptr(ws)), nb, _stream()))
    return Zt


def estimate_dtn_noalloc(mesh: Mesh, rows: dict, params: Params, outputs: dict):
    """The estimate with the library's fixed device scratch (no allocation in
    the call); ``outputs`` holds caller-allocated device tensors named as in
    estimate_dtn.  Returns the stats dict."""
    rs = _rows_struct(rows)
    out = _outputs_struct(outputs)
    st = Stats()
    _check(lib().mcs_estimate_dtn_noalloc(mesh.handle, C.byref(rs), C.byref(params), C.byref(out), C.byref(st),
                                          _stream()))
    return _stats_dict(st)
