"""GB300 collision-affording point tree (CAPT) library: Python binding of the C ABI.

Every function here has the name of the C entry point it calls (include/capt.h) and
only marshals arguments: numpy arrays for host inputs, torch CUDA tensors for device
buffers, torch's current stream by default.  All work runs in libcapt.so (host C++ and
sm_103a kernels); there is no Python or CPU fallback, and loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB, build

__all__ = [
    "build", "CaptError", "capt_build", "capt_build_threads", "sfc_filter", "capt_stats", "capt_export",
    "capt_upload", "capt_query_spheres", "capt_query_configs", "capt_query_configs_host",
    "capt_count_config_work", "capt_query_leaves", "capt_device_status", "capt_set_launch_cfg",
    "capt_get_launch_cfg", "capt_autotune_configs", "capt_validate_edges", "capt_edge_plan_create",
    "capt_edge_plan_launch", "capt_edge_plan_info", "capt_edge_plan_free", "capt_clearance_fwd",
    "capt_clearance_bwd", "capt_free", "capt_last_error", "make_arm", "CaptTree", "EdgePlan",
    "capt_validate_edges_static", "CAPT_STATIC_MAX_EDGES", "capt_build_device", "capt_query_joint_configs",
    "capt_autotune_joint_configs", "CAPT_KERNEL_JOINTS", "sfc_filter_device", "capt_autotune_spheres",
    "capt_morton_order", "capt_build_frame_device", "capt_compact", "CAPT_SCAN_SETS", "CAPT_SCAN_CHUNKED",
    "capt_count_sphere_work", "capt_count_clearance_work", "capt_build_grid", "capt_grid_export",
    "capt_build_near_lists", "capt_autotune_clearance", "capt_edge_plan_work", "CAPT_SCAN_COMPACT", "STATUS", "CAPT_STAGE_GLOBAL", "CAPT_STAGE_SMEM", "CAPT_KERNEL_SPHERES", "CAPT_KERNEL_CONFIGS",
    "CAPT_KERNEL_EDGES", "CAPT_KERNEL_CLEARANCE", "CAPT_EDGES_PERSISTENT", "CAPT_EDGES_PER_EDGE",
    "EXPORTED_SYMBOLS",
]

STATUS = {0: "CAPT_OK", -1: "CAPT_E_ARG", -2: "CAPT_E_RANGE", -3: "CAPT_E_NONFINITE", -4: "CAPT_E_NOMEM",
          -5: "CAPT_E_CUDA", -6: "CAPT_E_TIMEOUT", -7: "CAPT_E_BOUNDS", -8: "CAPT_E_STATE"}
CAPT_STAGE_GLOBAL, CAPT_STAGE_SMEM = 0, 1
CAPT_SCAN_SETS, CAPT_SCAN_CHUNKED, CAPT_SCAN_COMPACT = 0, 1, 2
CAPT_KERNEL_SPHERES, CAPT_KERNEL_CONFIGS, CAPT_KERNEL_EDGES, CAPT_KERNEL_CLEARANCE, CAPT_KERNEL_JOINTS = 0, 1, 2, 3, 4
CAPT_EDGES_PERSISTENT, CAPT_EDGES_PER_EDGE = 0, 1
MAX_JOINTS, MAX_SPHERES = 16, 64

# every extern "C" symbol declared in include/capt.h
EXPORTED_SYMBOLS = [
    "capt_build", "capt_build_threads", "sfc_filter", "capt_stats", "capt_export", "capt_free", "capt_last_error",
    "capt_upload", "capt_query_spheres", "capt_query_configs", "capt_query_configs_host", "capt_count_config_work",
    "capt_query_leaves", "capt_device_status", "capt_set_launch_cfg", "capt_get_launch_cfg",
    "capt_autotune_configs", "capt_validate_edges", "capt_edge_plan_create", "capt_edge_plan_launch",
    "capt_edge_plan_info", "capt_edge_plan_free", "capt_clearance_fwd", "capt_clearance_bwd",
    "capt_validate_edges_static", "capt_build_device", "capt_query_joint_configs", "capt_autotune_joint_configs",
    "sfc_filter_device", "capt_autotune_spheres", "capt_morton_order", "capt_build_frame_device", "capt_compact",
    "capt_count_sphere_work", "capt_count_clearance_work", "capt_build_grid", "capt_grid_export",
    "capt_build_near_lists", "capt_autotune_clearance", "capt_edge_plan_work",
]
CAPT_STATIC_MAX_EDGES = 65536


class CaptError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Stats(C.Structure):
    _fields_ = [("n_points", C.c_uint64), ("n_leaves", C.c_uint64), ("depth", C.c_uint32),
                ("max_set", C.c_uint32), ("total_afforded", C.c_uint64), ("total_blocks", C.c_uint64),
                ("pruned_leaves", C.c_uint64), ("empty_leaves", C.c_uint64), ("device_bytes", C.c_uint64),
                ("build_ms", C.c_double), ("r_min", C.c_float), ("r_max", C.c_float), ("device", C.c_int32),
                ("build_threads", C.c_int32), ("compact_chunks", C.c_uint64), ("compact_entries", C.c_uint64),
                ("compact_bytes", C.c_uint64), ("full_dropped", C.c_int32), ("reserved", C.c_int32),
                ("scratch_bytes", C.c_uint64), ("grid_dims", C.c_uint32 * 3), ("grid_cell", C.c_float),
                ("near_entries", C.c_uint64), ("near_bytes", C.c_uint64), ("near_fallback_cells", C.c_uint64)]


class _LaunchCfg(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("spheres_per_lane", C.c_int32), ("staging", C.c_int32),
                ("chunk", C.c_int32), ("prefetch", C.c_int32), ("grid", C.c_int32)]


class _Arm(C.Structure):
    _fields_ = [("n_joints", C.c_int32), ("n_spheres", C.c_int32), ("base", C.c_float * 3),
                ("axis", C.c_int32 * MAX_JOINTS), ("link", (C.c_float * 3) * MAX_JOINTS),
                ("sphere_link", C.c_int32 * MAX_SPHERES), ("sphere_offset", (C.c_float * 3) * MAX_SPHERES),
                ("sphere_radius", C.c_float * MAX_SPHERES)]


class _GridInfo(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("cell", C.c_float), ("inv_cell", C.c_float), ("unit", C.c_float),
                ("dims", C.c_int32 * 3), ("cells", C.c_uint32)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # CAPT_LIBRARY names another build of the same library (a test variant, see
    # _build.VARIANTS); by default the in-tree libcapt.so
    lib = os.environ.get("CAPT_LIBRARY") or LIB
    if not os.path.exists(lib):
        raise ImportError(f"libcapt.so is not built ({lib}); run paper_2406_02807_gb300.build()")
    L = C.CDLL(lib)
    P, SZ, I, F = C.c_void_p, C.c_size_t, C.c_int, C.c_float
    sig = {
        "capt_build": [P, SZ, F, F, C.POINTER(P)],
        "capt_build_threads": [P, SZ, F, F, I, C.POINTER(P)],
        "sfc_filter": [P, SZ, F, P, C.POINTER(SZ)],
        "sfc_filter_device": [P, SZ, F, P, C.POINTER(SZ), P],
        "capt_morton_order": [P, SZ, P],
        "capt_stats": [P, C.POINTER(_Stats)],
        "capt_export": [P, P, P, P, P],
        "capt_upload": [P, I, P],
        "capt_compact": [P, I, P],
        "capt_build_device": [P, SZ, F, F, P, C.POINTER(P)],
        "capt_build_frame_device": [P, SZ, F, F, F, P, C.POINTER(SZ), P, C.POINTER(P)],
        "capt_query_spheres": [P, P, P, SZ, P, P],
        "capt_query_configs": [P, P, P, SZ, I, P, P],
        "capt_query_configs_host": [P, P, P, SZ, I, P, P],
        "capt_count_config_work": [P, P, P, SZ, I, P, P],
        "capt_count_sphere_work": [P, P, P, SZ, P, P],
        "capt_count_clearance_work": [P, P, SZ, P, P],
        "capt_build_grid": [P, C.c_uint64, P],
        "capt_build_near_lists": [P, P],
        "capt_edge_plan_work": [P, C.POINTER(C.c_uint64)],
        "capt_grid_export": [P, C.POINTER(_GridInfo), P],
        "capt_query_leaves": [P, P, SZ, P, P],
        "capt_device_status": [P, P],
        "capt_set_launch_cfg": [P, I, C.POINTER(_LaunchCfg)],
        "capt_get_launch_cfg": [P, I, C.POINTER(_LaunchCfg)],
        "capt_autotune_configs": [P, P, P, SZ, I, P, P, C.POINTER(_LaunchCfg), C.POINTER(F)],
        "capt_autotune_spheres": [P, P, P, SZ, P, P, C.POINTER(_LaunchCfg), C.POINTER(F)],
        "capt_validate_edges": [P, C.POINTER(_Arm), P, P, P, SZ, P, I, P],
        "capt_validate_edges_static": [P, C.POINTER(_Arm), P, P, P, SZ, P, P],
        "capt_query_joint_configs": [P, C.POINTER(_Arm), P, SZ, P, P],
        "capt_autotune_joint_configs": [P, C.POINTER(_Arm), P, SZ, P, P, C.POINTER(_LaunchCfg), C.POINTER(F)],
        "capt_edge_plan_create": [P, C.POINTER(_Arm), P, P, P, SZ, P, C.POINTER(_LaunchCfg), P, C.POINTER(P)],
        "capt_edge_plan_launch": [P, P],
        "capt_edge_plan_info": [P, C.POINTER(_LaunchCfg), C.POINTER(F)],
        "capt_clearance_fwd": [P, P, P, SZ, I, I, F, P, P, P, P],
        "capt_autotune_clearance": [P, P, P, SZ, I, I, F, P, P, P, P, C.POINTER(_LaunchCfg), C.POINTER(F)],
        "capt_clearance_bwd": [P, P, P, P, P, P, SZ, I, I, F, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.capt_free.argtypes = [P]
    L.capt_free.restype = None
    L.capt_edge_plan_free.argtypes = [P]
    L.capt_edge_plan_free.restype = None
    L.capt_last_error.argtypes = []
    L.capt_last_error.restype = C.c_char_p
    _lib = L
    return L


def capt_last_error() -> str:
    return _load().capt_last_error().decode()


def _check(rc: int, where: str):
    if rc != 0:
        raise CaptError(rc, where, capt_last_error())


# ---------------------------------------------------------------------------- marshalling

def _host_f32(a, cols=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a.size else C.c_void_p(0)


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _numel(t, n, name):
    """A caller-passed buffer must hold exactly n elements: the C ABI receives only its
    base address, so a shorter one would be written past its end on the device."""
    if t is not None and t.numel() != n:
        raise ValueError(f"{name} must hold {n} elements, got {t.numel()}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class CaptTree:
    """Owning handle of a capt_tree (freed with capt_free)."""

    def __init__(self, handle: C.c_void_p):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            try:
                _load().capt_free(self.h)
            except Exception:
                pass
            self.h = C.c_void_p(0)

    @property
    def _as_parameter_(self):
        return self.h


# ----------------------------------------------------------------------------- host side

def capt_build(points, r_min: float, r_max: float) -> CaptTree:
    p = _host_f32(points, 3)
    h = C.c_void_p()
    _check(_load().capt_build(_ptr(p), p.shape[0], float(r_min), float(r_max), C.byref(h)), "capt_build")
    return CaptTree(h)


def capt_build_threads(points, r_min: float, r_max: float, n_threads: int) -> CaptTree:
    p = _host_f32(points, 3)
    h = C.c_void_p()
    _check(_load().capt_build_threads(_ptr(p), p.shape[0], float(r_min), float(r_max), int(n_threads), C.byref(h)),
           "capt_build_threads")
    return CaptTree(h)


def sfc_filter(points, min_spacing: float) -> np.ndarray:
    p = _host_f32(points, 3)
    out = np.zeros(max(p.shape[0], 1), np.uint32)
    n = C.c_size_t(0)
    _check(_load().sfc_filter(_ptr(p), p.shape[0], float(min_spacing), _ptr(out), C.byref(n)), "sfc_filter")
    return out[: n.value].copy()


def capt_morton_order(points) -> np.ndarray:
    """Permutation of the points along a Z-order curve (x most significant, ties by
    index); points[order] gives spatially tight affordance-set chunks."""
    p = _host_f32(points, 3)
    out = np.zeros(max(p.shape[0], 1), np.uint32)
    _check(_load().capt_morton_order(_ptr(p), p.shape[0], _ptr(out)), "capt_morton_order")
    return out[: p.shape[0]].copy()


def sfc_filter_device(points, min_spacing: float, stream=None):
    """Alg. 2 on the GPU: points is a float32 CUDA tensor [n, 3]; returns the kept
    indices (int32 CUDA tensor, last pass's curve order), equal to sfc_filter's."""
    import torch
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be [n, 3]")
    n = points.shape[0]
    kept = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    p = _dev(points, torch.float32, "points") if n else C.c_void_p(0)
    cnt = C.c_size_t(0)
    _check(_load().sfc_filter_device(p, n, float(min_spacing), _dev(kept, torch.int32, "kept"), C.byref(cnt),
                                     _stream(stream)), "sfc_filter_device")
    return kept[: cnt.value]


def capt_stats(tree: CaptTree) -> dict:
    s = _Stats()
    _check(_load().capt_stats(tree.h, C.byref(s)), "capt_stats")
    return {k: (list(getattr(s, k)) if k == "grid_dims" else getattr(s, k)) for k, _ in _Stats._fields_}


def capt_export(tree: CaptTree) -> dict:
    st = capt_stats(tree)
    N, tot = st["n_leaves"], st["total_afforded"]
    T = np.zeros(max(N - 1, 0), np.float32)
    sb = np.zeros(N + 1, np.uint64)
    si = np.zeros(tot, np.uint32)
    aabb = np.zeros((N, 6), np.float32)
    _check(_load().capt_export(tree.h, _ptr(T), _ptr(sb), _ptr(si), _ptr(aabb)), "capt_export")
    return dict(T=T, set_begin=sb, set_idx=si, aabb=aabb)


def capt_free(tree: CaptTree):
    if tree.h.value:
        _load().capt_free(tree.h)
        tree.h = C.c_void_p(0)


# --------------------------------------------------------------------------- device side

def capt_build_device(points, r_min: float, r_max: float, stream=None) -> CaptTree:
    """Build on the GPU from a contiguous float32 CUDA tensor [n, 3] on the current
    device; the tree comes back uploaded to that device."""
    import torch
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be [n, 3]")
    p = _dev(points, torch.float32, "points") if points.shape[0] else C.c_void_p(0)
    h = C.c_void_p()
    _check(_load().capt_build_device(p, points.shape[0], float(r_min), float(r_max), _stream(stream), C.byref(h)),
           "capt_build_device")
    return CaptTree(h)


def capt_build_frame_device(points, r_filter: float, r_min: float, r_max: float, stream=None):
    """Filter (Alg. 2) and build (Alg. 1) on the GPU in one call from a float32 CUDA
    tensor [n, 3]; returns (tree, kept) with kept the int32 indices of the points the tree
    holds, in its order."""
    import torch
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be [n, 3]")
    n = points.shape[0]
    kept = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    p = _dev(points, torch.float32, "points") if n else C.c_void_p(0)
    h = C.c_void_p()
    m = C.c_size_t(0)
    _check(_load().capt_build_frame_device(p, n, float(r_filter), float(r_min), float(r_max),
                                           _dev(kept, torch.int32, "kept"), C.byref(m), _stream(stream), C.byref(h)),
           "capt_build_frame_device")
    return CaptTree(h), kept[: m.value]


def capt_upload(tree: CaptTree, device: int = 0, stream=None):
    _check(_load().capt_upload(tree.h, int(device), _stream(stream)), "capt_upload")


def capt_build_grid(tree: CaptTree, max_cells: int = 0, stream=None):
    """Build (or rebuild) the tree's distance-bound grid on its device (at most max_cells
    cells; 0 = the library's default); configuration queries use it with grid = 1."""
    _check(_load().capt_build_grid(tree.h, int(max_cells), _stream(stream)), "capt_build_grid")


def capt_grid_export(tree: CaptTree):
    """(shape dict, cells uint8 [n2, n1, n0, 2] = {lower, upper} bound) of the tree's
    distance-bound grid, or (None, None) without one."""
    info = _GridInfo()
    _check(_load().capt_grid_export(tree.h, C.byref(info), None), "capt_grid_export")
    if info.cells == 0:
        return None, None
    cells = np.zeros(2 * info.cells, np.uint8)
    _check(_load().capt_grid_export(tree.h, C.byref(info), _ptr(cells)), "capt_grid_export")
    shape = dict(origin=np.array(info.origin, np.float32), cell=np.float32(info.cell),
                 inv_cell=np.float32(info.inv_cell), unit=np.float32(info.unit), dims=tuple(info.dims))
    n0, n1, n2 = shape["dims"]
    return shape, cells.reshape(n2, n1, n0, 2)


def capt_build_near_lists(tree: CaptTree, stream=None):
    """Build the clearance's nearest-candidate lists over the tree's distance-bound grid
    (capt_build_grid first; tree with r_min = 0); capt_clearance_fwd uses them with
    grid = 1 (the clearance default)."""
    _check(_load().capt_build_near_lists(tree.h, _stream(stream)), "capt_build_near_lists")


def capt_compact(tree: CaptTree, drop_full: bool = False, stream=None):
    """Build the tree's compact (de-duplicated) sets on its device; drop_full frees the
    replicated device sets afterwards."""
    _check(_load().capt_compact(tree.h, 1 if drop_full else 0, _stream(stream)), "capt_compact")


def capt_query_spheres(tree: CaptTree, centers, radii, flags=None, stream=None):
    import torch
    m = centers.shape[0]
    if centers.dim() != 2 or centers.shape[1] != 3 or radii.shape != (m,):
        raise ValueError("centers must be [m, 3] and radii [m]")
    _numel(flags, m, "flags")
    if flags is None:
        flags = torch.empty(m, dtype=torch.uint8, device=centers.device)
    _check(_load().capt_query_spheres(tree.h, _dev(centers, torch.float32, "centers"),
                                      _dev(radii, torch.float32, "radii"), m,
                                      _dev(flags, torch.uint8, "flags"), _stream(stream)), "capt_query_spheres")
    return flags


def capt_query_configs(tree: CaptTree, centers, radii, flags=None, stream=None):
    import torch
    if centers.dim() != 3 or centers.shape[2] != 3:
        raise ValueError("centers must be [C, S, 3]")
    Cn, S = centers.shape[0], centers.shape[1]
    if radii.shape != (S,):
        raise ValueError("radii must be [S]")
    _numel(flags, Cn, "flags")
    if flags is None:
        flags = torch.empty(Cn, dtype=torch.uint8, device=centers.device)
    _check(_load().capt_query_configs(tree.h, _dev(centers, torch.float32, "centers"),
                                      _dev(radii, torch.float32, "radii"), Cn, S,
                                      _dev(flags, torch.uint8, "flags"), _stream(stream)), "capt_query_configs")
    return flags


def capt_query_configs_host(tree: CaptTree, centers, radii, flags=None, stream=None):
    """Host arrays (numpy or CPU tensors, ideally pinned) in, host flags out."""
    import torch
    if isinstance(centers, torch.Tensor):
        if centers.is_cuda or centers.dtype != torch.float32 or not centers.is_contiguous():
            raise TypeError("centers must be a contiguous float32 CPU tensor")
        Cn, S = centers.shape[0], centers.shape[1]
        cp = C.c_void_p(centers.data_ptr())
    else:
        centers = _host_f32(centers)
        Cn, S = centers.shape[0], centers.shape[1]
        cp = _ptr(centers)
    r = np.ascontiguousarray(radii.cpu().numpy() if isinstance(radii, torch.Tensor) else radii, np.float32)
    if centers.ndim != 3 or centers.shape[2] != 3 or r.shape != (S,):
        raise ValueError("centers must be [C, S, 3] and radii [S]")
    if flags is not None and (flags.size if isinstance(flags, np.ndarray) else flags.numel()) != Cn:
        raise ValueError(f"flags must hold {Cn} elements")
    if isinstance(flags, torch.Tensor) and (flags.is_cuda or flags.dtype != torch.uint8 or not flags.is_contiguous()):
        raise TypeError("flags must be a contiguous uint8 CPU tensor")
    if isinstance(flags, np.ndarray) and (flags.dtype != np.uint8 or not flags.flags.c_contiguous):
        raise TypeError("flags must be a contiguous uint8 array")
    if flags is None:
        flags = np.zeros(Cn, np.uint8)
    fp = C.c_void_p(flags.data_ptr()) if isinstance(flags, torch.Tensor) else _ptr(flags)
    _check(_load().capt_query_configs_host(tree.h, cp, _ptr(r), Cn, S, fp, _stream(stream)), "capt_query_configs_host")
    return flags


def capt_count_config_work(tree: CaptTree, centers, radii, stream=None):
    import torch
    if centers.dim() != 3 or centers.shape[2] != 3 or radii.shape != (centers.shape[1],):
        raise ValueError("centers must be [C, S, 3] and radii [S]")
    Cn, S = centers.shape[0], centers.shape[1]
    counts = torch.zeros(8, dtype=torch.int64, device=centers.device)
    _check(_load().capt_count_config_work(tree.h, _dev(centers, torch.float32, "centers"),
                                          _dev(radii, torch.float32, "radii"), Cn, S,
                                          _dev(counts, torch.int64, "counts"), _stream(stream)),
           "capt_count_config_work")
    return counts


def capt_count_sphere_work(tree: CaptTree, centers, radii, stream=None):
    """The eight work counters of capt_count_config_work for sphere queries [m, 3] with
    radii [m]."""
    import torch
    if centers.dim() != 2 or centers.shape[1] != 3 or radii.shape != (centers.shape[0],):
        raise ValueError("centers must be [m, 3] and radii [m]")
    counts = torch.zeros(8, dtype=torch.int64, device=centers.device)
    _check(_load().capt_count_sphere_work(tree.h, _dev(centers, torch.float32, "centers"),
                                          _dev(radii, torch.float32, "radii"), centers.shape[0],
                                          _dev(counts, torch.int64, "counts"), _stream(stream)),
           "capt_count_sphere_work")
    return counts


def capt_count_clearance_work(tree: CaptTree, centers, stream=None):
    """[spheres, near the cloud box, passing the leaf box, points scanned, blocks scanned,
    answered by a nearest-candidate list, list entries scanned, fallback spheres] of
    capt_clearance_fwd on centres [..., 3]."""
    import torch
    if centers.shape[-1] != 3:
        raise ValueError("centers must end in a dimension of 3")
    m = centers.numel() // 3
    counts = torch.zeros(8, dtype=torch.int64, device=centers.device)
    _check(_load().capt_count_clearance_work(tree.h, _dev(centers, torch.float32, "centers"), m,
                                             _dev(counts, torch.int64, "counts"), _stream(stream)),
           "capt_count_clearance_work")
    return counts


def capt_query_leaves(tree: CaptTree, centers, leaves=None, stream=None):
    import torch
    if centers.dim() != 2 or centers.shape[1] != 3:
        raise ValueError("centers must be [m, 3]")
    m = centers.shape[0]
    _numel(leaves, m, "leaves")
    if leaves is None:
        leaves = torch.empty(m, dtype=torch.int32, device=centers.device)
    _check(_load().capt_query_leaves(tree.h, _dev(centers, torch.float32, "centers"), m,
                                     _dev(leaves, torch.int32, "leaves"), _stream(stream)), "capt_query_leaves")
    return leaves


def capt_device_status(tree: CaptTree, stream=None) -> int:
    """Returns the status code (0 = no latched device error); does not raise."""
    return int(_load().capt_device_status(tree.h, _stream(stream)))


def capt_set_launch_cfg(tree: CaptTree, kernel: int, warps_per_block: int, spheres_per_lane: int, staging: int,
                        chunk: int = 0, prefetch: int = 0, grid: int = 0):
    c = _LaunchCfg(warps_per_block, spheres_per_lane, staging, chunk, prefetch, grid)
    _check(_load().capt_set_launch_cfg(tree.h, int(kernel), C.byref(c)), "capt_set_launch_cfg")


def capt_get_launch_cfg(tree: CaptTree, kernel: int) -> dict:
    c = _LaunchCfg()
    _check(_load().capt_get_launch_cfg(tree.h, int(kernel), C.byref(c)), "capt_get_launch_cfg")
    return {k: getattr(c, k) for k, _ in _LaunchCfg._fields_}


def capt_autotune_configs(tree: CaptTree, centers, radii, flags=None, stream=None):
    import torch
    if centers.dim() != 3 or centers.shape[2] != 3 or radii.shape != (centers.shape[1],):
        raise ValueError("centers must be [C, S, 3] and radii [S]")
    Cn, S = centers.shape[0], centers.shape[1]
    _numel(flags, Cn, "flags")
    if flags is None:
        flags = torch.empty(Cn, dtype=torch.uint8, device=centers.device)
    c = _LaunchCfg()
    ms = C.c_float()
    _check(_load().capt_autotune_configs(tree.h, _dev(centers, torch.float32, "centers"),
                                         _dev(radii, torch.float32, "radii"), Cn, S,
                                         _dev(flags, torch.uint8, "flags"), _stream(stream), C.byref(c),
                                         C.byref(ms)), "capt_autotune_configs")
    return {k: getattr(c, k) for k, _ in _LaunchCfg._fields_}, ms.value


def capt_autotune_spheres(tree: CaptTree, centers, radii, flags=None, stream=None):
    import torch
    m = centers.shape[0]
    if centers.dim() != 2 or centers.shape[1] != 3 or radii.shape != (m,):
        raise ValueError("centers must be [m, 3] and radii [m]")
    _numel(flags, m, "flags")
    if flags is None:
        flags = torch.empty(m, dtype=torch.uint8, device=centers.device)
    c = _LaunchCfg()
    ms = C.c_float()
    _check(_load().capt_autotune_spheres(tree.h, _dev(centers, torch.float32, "centers"),
                                         _dev(radii, torch.float32, "radii"), m, _dev(flags, torch.uint8, "flags"),
                                         _stream(stream), C.byref(c), C.byref(ms)), "capt_autotune_spheres")
    return {k: getattr(c, k) for k, _ in _LaunchCfg._fields_}, ms.value


# -------------------------------------------------------------------------------- edges

def make_arm(arm) -> _Arm:
    """capt_arm from an object with base, axis, link, sphere_link, sphere_offset, sphere_radius."""
    a = _Arm()
    J, S = len(arm.axis), len(arm.sphere_radius)
    if not (1 <= J <= MAX_JOINTS and 1 <= S <= MAX_SPHERES):
        raise ValueError("arm must have 1..16 joints and 1..64 spheres")
    a.n_joints, a.n_spheres = J, S
    for i in range(3):
        a.base[i] = float(arm.base[i])
    for j in range(J):
        a.axis[j] = int(arm.axis[j])
        for i in range(3):
            a.link[j][i] = float(arm.link[j][i])
    for s in range(S):
        a.sphere_link[s] = int(arm.sphere_link[s])
        a.sphere_radius[s] = float(arm.sphere_radius[s])
        for i in range(3):
            a.sphere_offset[s][i] = float(arm.sphere_offset[s][i])
    return a


def _edge_args(tree: CaptTree, a: _Arm, qa, qb, nsteps, valid):
    """Shape and device checks of an edge batch, before any pointer crosses the C ABI
    (which sees only base addresses and E): qa, qb [E, n_joints], nsteps [E], valid
    with E elements, all on one CUDA device, the tree's when it is uploaded.  A shorter
    buffer would otherwise be read or written past its end on the device."""
    import torch
    for name, x in (("qa", qa), ("qb", qb), ("nsteps", nsteps)):
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
    if qa.dim() != 2 or qa.shape[1] != a.n_joints:
        raise ValueError(f"qa must be [E, {a.n_joints}], got {list(qa.shape)}")
    E = qa.shape[0]
    if tuple(qb.shape) != tuple(qa.shape):
        raise ValueError(f"qb must have the shape of qa {list(qa.shape)}, got {list(qb.shape)}")
    if tuple(nsteps.shape) != (E,):
        raise ValueError(f"nsteps must be [{E}], got {list(nsteps.shape)}")
    if valid is not None:
        if not isinstance(valid, torch.Tensor):
            raise TypeError("valid must be a torch tensor")
        if valid.numel() != E:
            raise ValueError(f"valid must hold {E} elements, got {valid.numel()}")
    devs = {x.device for x in (qa, qb, nsteps) + ((valid,) if valid is not None else ())}
    if len(devs) != 1:
        raise ValueError(f"qa, qb, nsteps and valid must be on one device, got {sorted(map(str, devs))}")
    d = qa.device
    if d.type == "cuda":
        td = capt_stats(tree)["device"]
        if td >= 0 and (d.index if d.index is not None else torch.cuda.current_device()) != td:
            raise ValueError(f"edge buffers are on {d}, the tree on cuda:{td}")
    return E


def capt_validate_edges(tree: CaptTree, arm, qa, qb, nsteps, valid=None, mode=CAPT_EDGES_PERSISTENT, stream=None):
    import torch
    a = arm if isinstance(arm, _Arm) else make_arm(arm)
    E = _edge_args(tree, a, qa, qb, nsteps, valid)
    if valid is None:
        valid = torch.empty(E, dtype=torch.uint8, device=qa.device)
    _check(_load().capt_validate_edges(tree.h, C.byref(a), _dev(qa, torch.float32, "qa"), _dev(qb, torch.float32, "qb"),
                                       _dev(nsteps, torch.int32, "nsteps"), E, _dev(valid, torch.uint8, "valid"),
                                       int(mode), _stream(stream)), "capt_validate_edges")
    return valid


def capt_query_joint_configs(tree: CaptTree, arm, q, flags=None, stream=None):
    """One flag per configuration given by joint angles q [C, n_joints] (float32 CUDA
    tensor); the kinematics run inside the kernel."""
    import torch
    a = arm if isinstance(arm, _Arm) else make_arm(arm)
    if q.dim() != 2 or q.shape[1] != a.n_joints:
        raise ValueError("q must be [C, n_joints]")
    Cn = q.shape[0]
    _numel(flags, Cn, "flags")
    if flags is None:
        flags = torch.empty(Cn, dtype=torch.uint8, device=q.device)
    _check(_load().capt_query_joint_configs(tree.h, C.byref(a), _dev(q, torch.float32, "q"), Cn,
                                            _dev(flags, torch.uint8, "flags"), _stream(stream)),
           "capt_query_joint_configs")
    return flags


def capt_autotune_joint_configs(tree: CaptTree, arm, q, flags=None, stream=None):
    import torch
    a = arm if isinstance(arm, _Arm) else make_arm(arm)
    if q.dim() != 2 or q.shape[1] != a.n_joints:
        raise ValueError("q must be [C, n_joints]")
    Cn = q.shape[0]
    _numel(flags, Cn, "flags")
    if flags is None:
        flags = torch.empty(Cn, dtype=torch.uint8, device=q.device)
    c = _LaunchCfg()
    ms = C.c_float()
    _check(_load().capt_autotune_joint_configs(tree.h, C.byref(a), _dev(q, torch.float32, "q"), Cn,
                                               _dev(flags, torch.uint8, "flags"), _stream(stream), C.byref(c),
                                               C.byref(ms)), "capt_autotune_joint_configs")
    return {k: getattr(c, k) for k, _ in _LaunchCfg._fields_}, ms.value


def capt_validate_edges_static(tree: CaptTree, arm, qa, qb, nsteps, valid=None, stream=None):
    """capt_validate_edges without any device allocation by the library (at most
    CAPT_STATIC_MAX_EDGES edges; calls share one scratch array, so overlapping calls
    race).  For callers that must not enter the CUDA allocator, such as a planner in a
    real-time control loop or an application whose device memory another allocator owns."""
    import torch
    a = arm if isinstance(arm, _Arm) else make_arm(arm)
    E = _edge_args(tree, a, qa, qb, nsteps, valid)
    if valid is None:
        valid = torch.empty(E, dtype=torch.uint8, device=qa.device)
    _check(_load().capt_validate_edges_static(tree.h, C.byref(a), _dev(qa, torch.float32, "qa"),
                                              _dev(qb, torch.float32, "qb"), _dev(nsteps, torch.int32, "nsteps"), E,
                                              _dev(valid, torch.uint8, "valid"), _stream(stream)),
           "capt_validate_edges_static")
    return valid


class EdgePlan:
    """Owning handle of a capt_edge_plan; keeps its buffers alive."""

    def __init__(self, handle, keep):
        self.h = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            try:
                _load().capt_edge_plan_free(self.h)
            except Exception:
                pass
            self.h = C.c_void_p(0)


def capt_edge_plan_create(tree: CaptTree, arm, qa, qb, nsteps, valid, cfg=None, stream=None) -> EdgePlan:
    import torch
    a = arm if isinstance(arm, _Arm) else make_arm(arm)
    E = _edge_args(tree, a, qa, qb, nsteps, valid)
    c = None if cfg is None else C.byref(_LaunchCfg(cfg["warps_per_block"], cfg["spheres_per_lane"], cfg["staging"],
                                                    cfg["chunk"], cfg.get("prefetch", 0), cfg.get("grid", 0)))
    h = C.c_void_p()
    _check(_load().capt_edge_plan_create(tree.h, C.byref(a), _dev(qa, torch.float32, "qa"),
                                         _dev(qb, torch.float32, "qb"), _dev(nsteps, torch.int32, "nsteps"), E,
                                         _dev(valid, torch.uint8, "valid"), c, _stream(stream), C.byref(h)),
           "capt_edge_plan_create")
    return EdgePlan(h, (tree, qa, qb, nsteps, valid))


def capt_edge_plan_launch(plan: EdgePlan, stream=None):
    _check(_load().capt_edge_plan_launch(plan.h, _stream(stream)), "capt_edge_plan_launch")


def capt_edge_plan_info(plan: EdgePlan):
    c = _LaunchCfg()
    ms = C.c_float()
    _check(_load().capt_edge_plan_info(plan.h, C.byref(c), C.byref(ms)), "capt_edge_plan_info")
    return {k: getattr(c, k) for k, _ in _LaunchCfg._fields_}, ms.value


def capt_edge_plan_work(plan: EdgePlan) -> int:
    """Configurations the plan's last launch evaluated (call after it has finished)."""
    v = C.c_uint64()
    _check(_load().capt_edge_plan_work(plan.h, C.byref(v)), "capt_edge_plan_work")
    return int(v.value)


def capt_edge_plan_free(plan: EdgePlan):
    if plan.h.value:
        _load().capt_edge_plan_free(plan.h)
        plan.h = C.c_void_p(0)


# ---------------------------------------------------------------------------- clearance

def capt_clearance_fwd(tree: CaptTree, centers, radii, margin: float, cost=None, dist=None, argmin=None,
                       stream=None):
    import torch
    if centers.dim() != 4 or centers.shape[3] != 3:
        raise ValueError("centers must be [T, W, S, 3]")
    T, W, S = centers.shape[:3]
    if radii.shape != (S,):
        raise ValueError("radii must be [S]")
    _numel(cost, T, "cost")
    _numel(dist, T * W * S, "dist")
    _numel(argmin, T * W * S, "argmin")
    dev = centers.device
    cost = torch.empty(T, dtype=torch.float32, device=dev) if cost is None else cost
    dist = torch.empty((T, W, S), dtype=torch.float32, device=dev) if dist is None else dist
    argmin = torch.empty((T, W, S), dtype=torch.int32, device=dev) if argmin is None else argmin
    _check(_load().capt_clearance_fwd(tree.h, _dev(centers, torch.float32, "centers"),
                                      _dev(radii, torch.float32, "radii"), T, W, S, float(margin),
                                      _dev(cost, torch.float32, "cost"), _dev(dist, torch.float32, "dist"),
                                      _dev(argmin, torch.int32, "argmin"), _stream(stream)), "capt_clearance_fwd")
    return cost, dist, argmin


def capt_autotune_clearance(tree: CaptTree, centers, radii, margin: float, stream=None):
    """Time the clearance forward's launch configurations on these inputs, keep the
    fastest on the tree; returns (cfg dict, best ms)."""
    import torch
    if centers.dim() != 4 or centers.shape[3] != 3:
        raise ValueError("centers must be [T, W, S, 3]")
    T, W, S = centers.shape[:3]
    if radii.shape != (S,):
        raise ValueError("radii must be [S]")
    dev = centers.device
    cost = torch.empty(T, dtype=torch.float32, device=dev)
    dist = torch.empty((T, W, S), dtype=torch.float32, device=dev)
    argmin = torch.empty((T, W, S), dtype=torch.int32, device=dev)
    best, ms = _LaunchCfg(), C.c_float()
    _check(_load().capt_autotune_clearance(tree.h, _dev(centers, torch.float32, "centers"),
                                           _dev(radii, torch.float32, "radii"), T, W, S, float(margin),
                                           _dev(cost, torch.float32, "cost"), _dev(dist, torch.float32, "dist"),
                                           _dev(argmin, torch.int32, "argmin"), _stream(stream), C.byref(best),
                                           C.byref(ms)), "capt_autotune_clearance")
    return {k: getattr(best, k) for k, _ in _LaunchCfg._fields_}, ms.value


def capt_clearance_bwd(tree: CaptTree, centers, radii, dist, argmin, grad_cost, margin: float, grad=None,
                       stream=None):
    import torch
    if centers.dim() != 4 or centers.shape[3] != 3:
        raise ValueError("centers must be [T, W, S, 3]")
    T, W, S = centers.shape[:3]
    if radii.shape != (S,):
        raise ValueError("radii must be [S]")
    _numel(dist, T * W * S, "dist")
    _numel(argmin, T * W * S, "argmin")
    _numel(grad_cost, T, "grad_cost")
    _numel(grad, T * W * S * 3, "grad")
    grad = torch.empty_like(centers) if grad is None else grad
    _check(_load().capt_clearance_bwd(tree.h, _dev(centers, torch.float32, "centers"),
                                      _dev(radii, torch.float32, "radii"), _dev(dist, torch.float32, "dist"),
                                      _dev(argmin, torch.int32, "argmin"), _dev(grad_cost, torch.float32, "grad_cost"),
                                      T, W, S, float(margin), _dev(grad, torch.float32, "grad"), _stream(stream)),
           "capt_clearance_bwd")
    return grad


from .clearance import CaptClearance  # noqa: E402  (autograd wrapper over the two calls above)

__all__.append("CaptClearance")
