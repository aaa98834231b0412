"""CPU oracle for the CAPT query path: ctypes wrappers around oracle.c.

TEST INFRASTRUCTURE ONLY: imported by tests/, by `__graft_entry__.smoke()` and by the
CPU-baseline leg of bench.py, never by the product package.  It shares no code with the
CUDA library (see the header of oracle.c for what each function computes, the passage
of the paper it follows, and what pins it).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
          "-fPIC", "-shared", "-pthread", "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, no contraction of float expressions)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


P = C.c_void_p
SZ = C.c_size_t


def _declare(L):
    L.orc_brute_flags.argtypes = [P, SZ, P, P, SZ, P, C.c_int]
    L.orc_brute_config_flags.argtypes = [P, SZ, P, P, SZ, C.c_int, P, C.c_int]
    L.orc_min_gap64.argtypes = [P, SZ, P, P, SZ, P, C.c_int]
    L.orc_nearest64.argtypes = [P, SZ, P, SZ, P, P, P, C.c_int]
    L.orc_clearance64.argtypes = [P, SZ, P, P, SZ, C.c_int, C.c_int, C.c_double, C.c_double, P, P, P, P,
                                  C.c_int]
    L.orc_capt_build.argtypes = [P, SZ, C.c_float, C.c_float, C.POINTER(C.c_void_p)]
    L.orc_capt_free.argtypes = [P]
    L.orc_capt_free.restype = None
    L.orc_capt_info.argtypes = [P, P]
    L.orc_capt_export.argtypes = [P, P, P, P, P, P, P]
    L.orc_capt_query.argtypes = [P, P, P, SZ, P, P, P]
    L.orc_capt_query_configs.argtypes = [P, P, P, SZ, C.c_int, P, P]
    L.orc_capt_nearest64.argtypes = [P, P, SZ, C.c_double, P, P]
    L.orc_morton_key.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, P]
    L.orc_morton_key.restype = C.c_uint64
    L.orc_sfc_filter.argtypes = [P, SZ, C.c_float, P, C.POINTER(C.c_size_t), P, P, P]
    L.orc_sincos32.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.orc_sincos32.restype = None
    L.orc_fk32.argtypes = [C.c_int, P, P, P, C.c_int, P, P, P, SZ, P]
    L.orc_interp32.argtypes = [C.c_int, P, P, C.c_int, P]
    L.orc_edges.argtypes = [P, P, SZ, C.c_int, P, P, P, C.c_int, P, P, P, P, P, P, SZ, P, C.c_int]


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def brute_flags(points, centers, radii, threads=None):
    """FP32 brute force, one flag per sphere (Lemma 1's right-hand side)."""
    p, c, r = _f32(points).reshape(-1, 3), _f32(centers).reshape(-1, 3), _f32(radii).reshape(-1)
    out = np.zeros(c.shape[0], np.uint8)
    _check(lib().orc_brute_flags(_ptr(p), p.shape[0], _ptr(c), _ptr(r), c.shape[0], _ptr(out),
                                 threads or default_threads()), "brute_flags")
    return out


def brute_config_flags(points, centers, radii, threads=None):
    """FP32 brute force OR-ed over the S spheres of each configuration; centers [C,S,3]."""
    p, c, r = _f32(points).reshape(-1, 3), _f32(centers), _f32(radii).reshape(-1)
    Cn, S = c.shape[0], c.shape[1]
    out = np.zeros(Cn, np.uint8)
    _check(lib().orc_brute_config_flags(_ptr(p), p.shape[0], _ptr(c), _ptr(r), Cn, S, _ptr(out),
                                        threads or default_threads()), "brute_config_flags")
    return out


def min_gap64(points, centers, radii, threads=None):
    p, c, r = _f32(points).reshape(-1, 3), _f32(centers).reshape(-1, 3), _f32(radii).reshape(-1)
    out = np.zeros(c.shape[0], np.float64)
    _check(lib().orc_min_gap64(_ptr(p), p.shape[0], _ptr(c), _ptr(r), c.shape[0], _ptr(out),
                               threads or default_threads()), "min_gap64")
    return out


def nearest64(points, centers, threads=None):
    """FP64 nearest distance, index and runner-up distance per centre."""
    p, c = _f32(points).reshape(-1, 3), _f32(centers).reshape(-1, 3)
    m = c.shape[0]
    d, i, s = np.zeros(m), np.zeros(m, np.int64), np.zeros(m)
    _check(lib().orc_nearest64(_ptr(p), p.shape[0], _ptr(c), m, _ptr(d), _ptr(i), _ptr(s),
                               threads or default_threads()), "nearest64")
    return d, i, s


def clearance64(points, centers, radii, r_max, margin, grad_cost=None, want_grad=True, threads=None):
    """FP64 hinge clearance; centers [T,W,S,3].  Returns (cost [T], d [T,W,S], grad or None)."""
    p, c, r = _f32(points).reshape(-1, 3), _f32(centers), _f32(radii).reshape(-1)
    T, W, S = c.shape[:3]
    cost, dist = np.zeros(T), np.zeros((T, W, S))
    grad = np.zeros((T, W, S, 3)) if want_grad else None
    g = None if grad_cost is None else np.ascontiguousarray(grad_cost, np.float64)
    _check(lib().orc_clearance64(_ptr(p), p.shape[0], _ptr(c), _ptr(r), T, W, S, float(r_max), float(margin),
                                 _ptr(g), _ptr(cost), _ptr(dist), _ptr(grad), threads or default_threads()),
           "clearance64")
    return cost, dist, grad


class PlainCAPT:
    """The plain recursive CAPT of Alg. 1, queried with Alg. 3."""

    def __init__(self, points, r_min, r_max):
        self.points = _f32(points).reshape(-1, 3)
        h = C.c_void_p()
        _check(lib().orc_capt_build(_ptr(self.points), self.points.shape[0], float(r_min), float(r_max),
                                    C.byref(h)), "capt_build")
        self.h = h
        info = np.zeros(5, np.int64)
        _check(lib().orc_capt_info(self.h, _ptr(info)), "capt_info")
        self.N, self.L, self.total, self.max_set, self.n_pruned = (int(v) for v in info)

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            lib().orc_capt_free(self.h)
            self.h = C.c_void_p()

    def export(self):
        N = self.N
        T = np.zeros(max(N - 1, 0), np.float32)
        sb = np.zeros(N + 1, np.int64)
        si = np.zeros(self.total, np.uint32)
        aabb = np.zeros((N, 6), np.float32)
        cell = np.zeros((N, 6), np.float64)
        pr = np.zeros(N, np.uint8)
        _check(lib().orc_capt_export(self.h, _ptr(T), _ptr(sb), _ptr(si), _ptr(aabb), _ptr(cell), _ptr(pr)),
               "capt_export")
        return dict(T=T, set_begin=sb, set_idx=si, aabb=aabb, cell=cell, pruned=pr)

    def query(self, centers, radii):
        c, r = _f32(centers).reshape(-1, 3), _f32(radii).reshape(-1)
        m = c.shape[0]
        f, leaf, ms = np.zeros(m, np.uint8), np.zeros(m, np.int64), np.zeros(m, np.int64)
        _check(lib().orc_capt_query(self.h, _ptr(c), _ptr(r), m, _ptr(f), _ptr(leaf), _ptr(ms)), "capt_query")
        return f, leaf, ms

    def query_configs(self, centers, radii):
        c, r = _f32(centers), _f32(radii).reshape(-1)
        Cn, S = c.shape[0], c.shape[1]
        f = np.zeros(Cn, np.uint8)
        counts = np.zeros(3, np.int64)
        _check(lib().orc_capt_query_configs(self.h, _ptr(c), _ptr(r), Cn, S, _ptr(f), _ptr(counts)),
               "capt_query_configs")
        return f, counts

    def nearest64(self, centers, r_max):
        c = _f32(centers).reshape(-1, 3)
        m = c.shape[0]
        d, i = np.zeros(m), np.zeros(m, np.int64)
        _check(lib().orc_capt_nearest64(self.h, _ptr(c), m, float(r_max), _ptr(d), _ptr(i)), "capt_nearest64")
        return d, i


def morton_key(q, perm):
    pa = np.ascontiguousarray(perm, np.int32)
    return int(lib().orc_morton_key(int(q[0]), int(q[1]), int(q[2]), _ptr(pa)))


def sfc_filter(points, r_filter, trace=False):
    """Plain Alg. 2.  Returns kept indices (final-pass curve order) [and the pass trace]."""
    p = _f32(points).reshape(-1, 3)
    n = p.shape[0]
    out = np.zeros(max(n, 1), np.uint32)
    nout = C.c_size_t(0)
    to = ta = tl = None
    if trace:
        to, ta, tl = np.zeros(6 * max(n, 1), np.uint32), np.zeros(6 * max(n, 1), np.uint32), np.zeros(6, np.int64)
    _check(lib().orc_sfc_filter(_ptr(p), n, float(r_filter), _ptr(out), C.byref(nout), _ptr(to), _ptr(ta),
                                _ptr(tl)), "sfc_filter")
    kept = out[: nout.value].copy()
    if not trace:
        return kept
    passes = []
    for k in range(6):
        m = int(tl[k])
        passes.append((to[k * n: k * n + m].copy(), ta[k * n: k * n + m].copy()))
    return kept, passes


def sincos32(x):
    s, c = C.c_float(), C.c_float()
    lib().orc_sincos32(float(x), C.byref(s), C.byref(c))
    return s.value, c.value


def _arm_arrays(arm):
    return dict(
        base=_f32(arm.base), axis=np.ascontiguousarray(arm.axis, np.int32), link=_f32(arm.link),
        sl=np.ascontiguousarray(arm.sphere_link, np.int32), so=_f32(arm.sphere_offset), sr=_f32(arm.sphere_radius))


def fk32(arm, q):
    """FP32 kinematics of the oracle: q [C,J] -> centres [C,S,3]."""
    a = _arm_arrays(arm)
    q = _f32(q).reshape(-1, arm.n_joints)
    out = np.zeros((q.shape[0], arm.n_spheres, 3), np.float32)
    _check(lib().orc_fk32(arm.n_joints, _ptr(a["base"]), _ptr(a["axis"]), _ptr(a["link"]), arm.n_spheres,
                          _ptr(a["sl"]), _ptr(a["so"]), _ptr(q), q.shape[0], _ptr(out)), "fk32")
    return out


def interp32(qa, qb, n):
    qa, qb = _f32(qa), _f32(qb)
    out = np.zeros((n, qa.shape[0]), np.float32)
    _check(lib().orc_interp32(qa.shape[0], _ptr(qa), _ptr(qb), n, _ptr(out)), "interp32")
    return out


def edges(arm, qa, qb, nsteps, tree: PlainCAPT | None = None, points=None, threads=None):
    """Per-edge validity (1 = no interpolated configuration collides)."""
    a = _arm_arrays(arm)
    qa, qb = _f32(qa), _f32(qb)
    ns = np.ascontiguousarray(nsteps, np.int32)
    E = ns.shape[0]
    out = np.zeros(E, np.uint8)
    p = None if points is None else _f32(points).reshape(-1, 3)
    _check(lib().orc_edges(tree.h if tree is not None else None, _ptr(p), 0 if p is None else p.shape[0],
                           arm.n_joints, _ptr(a["base"]), _ptr(a["axis"]), _ptr(a["link"]), arm.n_spheres,
                           _ptr(a["sl"]), _ptr(a["so"]), _ptr(a["sr"]), _ptr(qa), _ptr(qb), _ptr(ns), E,
                           _ptr(out), threads or default_threads()), "edges")
    return out
