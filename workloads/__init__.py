"""Seeded synthetic workloads for the collision-affording point tree (CAPT) query path.

Input generation only: point clouds, query spheres, arm configurations, edges and
trajectories, all drawn from one counter-based generator (SplitMix64, Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).  Nothing here
builds a tree, filters a cloud or tests a sphere against a point: this module holds
none of the method's arithmetic, so the CUDA library and the CPU oracle can both draw
their inputs from it without sharing any of the computation they are compared on.

The paper measures on MotionBenchMaker scenes, recorded planner queries and RealSense
frames (Sec. VI).  None of those is available, so the generators below stand in for
them with the shapes and sizes the paper uses: clouds of thousands of points sampled
on table / box / shelf surfaces, r_min = 1-2 cm and r_max = 5.5-10 cm (Sec. VI-A),
r_filter = 1-2 cm, and a 7-joint serial arm approximated by spheres (Sec. IV).

Seeds: workload `i` uses seed 1000 + i; every purpose (points, layout, noise, queries,
configurations) draws from its own stream of that seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Stream", "ArmModel", "arm_7dof", "fk_centers",
    "uniform_cloud", "tabletop_cloud", "room_cloud", "depth_frame",
    "cube_queries", "room_queries", "random_configs", "random_edges",
    "random_trajectories", "WORKLOADS",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# purpose ids: one independent stream per purpose of a seed
P_POINTS, P_LAYOUT, P_NOISE, P_QUERIES, P_CONFIGS = 1, 2, 3, 4, 5


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the published 'mix64' finaliser)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream: value i is mix64(base + (i + 1) * gamma)."""

    def __init__(self, seed: int, purpose: int):
        with np.errstate(over="ignore"):
            s = np.array([(seed & 0xFFFFFFFF) | ((purpose & 0xFFFF) << 32)], dtype=np.uint64)
            self.base = _mix64(s * _GAMMA)[0]
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + i * _GAMMA)

    def uniform01(self, n: int) -> np.ndarray:
        """float64 values that are exact float32 numbers: (u >> 40) * 2^-24, in [0, 1)."""
        return (self.u64(n) >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))

    def uniform(self, lo, hi, n: int) -> np.ndarray:
        return lo + (hi - lo) * self.uniform01(n)

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller in float64 from 53-bit uniforms."""
        m = (n + 1) // 2
        u = self.u64(2 * m)
        u1 = ((u[:m] >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / (1 << 53))  # (0, 1]
        u2 = (u[m:] >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
        return z[:n]

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive) by multiply-shift on 32 high bits."""
        span = hi - lo + 1
        u = (self.u64(n) >> np.uint64(32)).astype(np.uint64)
        return (lo + ((u * np.uint64(span)) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


# --------------------------------------------------------------------------------------
# Clouds
# --------------------------------------------------------------------------------------

def uniform_cloud(n: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1]^3, float32 [n,3]."""
    return Stream(seed, P_POINTS).uniform01(3 * n).reshape(n, 3).astype(np.float32)


def _sample_rects(rects, areas, n, st_pts):
    """Area-weighted sampling on axis-aligned rectangles.

    rects: list of (origin[3], edge_u[3], edge_v[3]); a point is origin + a*u + b*v.
    """
    areas = np.asarray(areas, dtype=np.float64)
    cdf = np.cumsum(areas) / areas.sum()
    pick = np.searchsorted(cdf, st_pts.uniform01(n), side="right")
    pick = np.minimum(pick, len(rects) - 1)
    a = st_pts.uniform01(n)
    b = st_pts.uniform01(n)
    org = np.array([r[0] for r in rects])[pick]
    eu = np.array([r[1] for r in rects])[pick]
    ev = np.array([r[2] for r in rects])[pick]
    return org + a[:, None] * eu + b[:, None] * ev


def _box_faces(lo, hi, with_bottom):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    dx, dy, dz = hi - lo
    X, Y, Z = np.eye(3)
    faces = [
        (np.array([lo[0], lo[1], hi[2]]), dx * X, dy * Y),   # top
        (np.array([lo[0], lo[1], lo[2]]), dx * X, dz * Z),   # y = lo
        (np.array([lo[0], hi[1], lo[2]]), dx * X, dz * Z),   # y = hi
        (np.array([lo[0], lo[1], lo[2]]), dy * Y, dz * Z),   # x = lo
        (np.array([hi[0], lo[1], lo[2]]), dy * Y, dz * Z),   # x = hi
    ]
    areas = [dx * dy, dx * dz, dx * dz, dy * dz, dy * dz]
    if with_bottom:
        faces.append((np.array([lo[0], lo[1], lo[2]]), dx * X, dy * Y))
        areas.append(dx * dy)
    return faces, areas


def tabletop_cloud(seed: int, n: int = 30000, sigma: float = 0.002):
    """Depth-like tabletop cloud: table top, 6 boxes, 3 vertical cylinders (surface samples).

    Table top z = 0, x in [0, 1.2], y in [-0.4, 0.4].  Boxes: sides U[0.05, 0.30], resting
    on the table, footprint inside it.  Cylinders: radius U[0.03, 0.06], height
    U[0.10, 0.30], on the table.  Samples are area-weighted over the table top and every
    face but the bottom, then perturbed by N(0, sigma^2) per coordinate.
    Returns (points float32 [n,3], layout dict).
    """
    lay = Stream(seed, P_LAYOUT)
    rects, areas = [], []
    rects.append((np.array([0.0, -0.4, 0.0]), np.array([1.2, 0, 0.0]), np.array([0, 0.8, 0.0])))
    areas.append(1.2 * 0.8)
    boxes = []
    for _ in range(6):
        sx, sy, sz = lay.uniform(0.05, 0.30, 3)
        cx = lay.uniform(sx / 2, 1.2 - sx / 2, 1)[0]
        cy = lay.uniform(-0.4 + sy / 2, 0.4 - sy / 2, 1)[0]
        lo = [cx - sx / 2, cy - sy / 2, 0.0]
        hi = [cx + sx / 2, cy + sy / 2, sz]
        boxes.append((lo, hi))
        f, a = _box_faces(lo, hi, with_bottom=False)
        rects += f
        areas += a
    cyls = []
    for _ in range(3):
        r = lay.uniform(0.03, 0.06, 1)[0]
        h = lay.uniform(0.10, 0.30, 1)[0]
        cx = lay.uniform(r, 1.2 - r, 1)[0]
        cy = lay.uniform(-0.4 + r, 0.4 - r, 1)[0]
        cyls.append((cx, cy, r, h))
    # split the sample count between rectangles and cylinders by area
    cyl_areas = [2 * math.pi * r * h + math.pi * r * r for (_, _, r, h) in cyls]
    tot = sum(areas) + sum(cyl_areas)
    st = Stream(seed, P_POINTS)
    u = st.uniform01(n)
    cdf = np.cumsum(np.array(areas + cyl_areas)) / tot
    which = np.minimum(np.searchsorted(cdf, u, side="right"), len(cdf) - 1)
    pts = np.empty((n, 3), dtype=np.float64)
    a = st.uniform01(n)
    b = st.uniform01(n)
    nr = len(rects)
    rmask = which < nr
    if rmask.any():
        idx = which[rmask]
        org = np.array([r[0] for r in rects])[idx]
        eu = np.array([r[1] for r in rects])[idx]
        ev = np.array([r[2] for r in rects])[idx]
        pts[rmask] = org + a[rmask, None] * eu + b[rmask, None] * ev
    for ci, (cx, cy, r, h) in enumerate(cyls):
        m = which == nr + ci
        if not m.any():
            continue
        aa, bb = a[m], b[m]
        side = 2 * math.pi * r * h
        top = math.pi * r * r
        on_side = aa * (side + top) < side
        th = 2 * math.pi * bb
        out = np.empty((m.sum(), 3))
        # side: angle from b, height from a rescaled
        hs = np.where(on_side, aa * (side + top) / side, 0.0) * h
        out[:, 0] = cx + r * np.cos(th)
        out[:, 1] = cy + r * np.sin(th)
        out[:, 2] = hs
        # top disc: radius sqrt-uniform from the rescaled a
        at = np.where(on_side, 0.0, (aa * (side + top) - side) / top)
        rr = r * np.sqrt(np.clip(at, 0, 1))
        out[~on_side, 0] = cx + rr[~on_side] * np.cos(th[~on_side])
        out[~on_side, 1] = cy + rr[~on_side] * np.sin(th[~on_side])
        out[~on_side, 2] = h
        pts[m] = out
    pts += sigma * Stream(seed, P_NOISE).normal(3 * n).reshape(n, 3)
    return pts.astype(np.float32), {"boxes": boxes, "cylinders": cyls}


def room_cloud(seed: int, n: int = 200000, sigma: float = 0.003):
    """Room [0,4]x[0,4]x[0,2.5]: floor + 4 walls (no ceiling) and 40 boxes (shelves).

    Box sides U[0.1, 0.6], base height U[0, 1.9], footprint inside the room; all six faces
    are sampled.  Area-weighted surface samples with N(0, sigma^2) noise.
    """
    lay = Stream(seed, P_LAYOUT)
    X, Y, Z = np.eye(3)
    rects = [
        (np.zeros(3), 4 * X, 4 * Y),                       # floor
        (np.zeros(3), 4 * X, 2.5 * Z),                     # y = 0 wall
        (np.array([0, 4.0, 0]), 4 * X, 2.5 * Z),           # y = 4 wall
        (np.zeros(3), 4 * Y, 2.5 * Z),                     # x = 0 wall
        (np.array([4.0, 0, 0]), 4 * Y, 2.5 * Z),           # x = 4 wall
    ]
    areas = [16.0, 10.0, 10.0, 10.0, 10.0]
    for _ in range(40):
        sx, sy, sz = lay.uniform(0.1, 0.6, 3)
        z0 = lay.uniform(0.0, 1.9, 1)[0]
        cx = lay.uniform(sx / 2, 4 - sx / 2, 1)[0]
        cy = lay.uniform(sy / 2, 4 - sy / 2, 1)[0]
        f, a = _box_faces([cx - sx / 2, cy - sy / 2, z0], [cx + sx / 2, cy + sy / 2, z0 + sz], True)
        rects += f
        areas += a
    pts = _sample_rects(rects, areas, n, Stream(seed, P_POINTS))
    pts += sigma * Stream(seed, P_NOISE).normal(3 * n).reshape(n, 3)
    return pts.astype(np.float32)


def depth_frame(seed: int = 1001, width: int = 640, height: int = 480, sigma: float = 0.002,
                cam=(0.6, 0.0, 0.6), target=(0.7, 0.0, 0.0), hfov_deg: float = 87.0):
    """A depth-camera frame of the tabletop scene: one point per pixel of a pinhole camera
    (640 x 480, 87 degree horizontal field of view, as a RealSense D455's depth stream)
    0.6 m above the table looking down at it, where the pixel's ray first meets the
    scene (307,200 points, the size of the paper's real-robot frames, Table III; the
    Morton filter keeps 34,892 / 15,703 / 7,900 of them at 1 / 1.5 / 2 cm).

    The scene is the tabletop layout of `tabletop_cloud(seed)` (table top, boxes,
    vertical cylinders) inside a room that catches every other ray: a floor at
    z = -0.75, a back wall at x = 2.5 and side walls at y = +-1.5 (no ceiling is needed:
    the camera looks down).  Each point is perturbed along its ray by N(0, sigma^2).
    Returns float32 [height * width, 3], row-major over the image.
    """
    _, layout = tabletop_cloud(seed, n=1)
    o = np.asarray(cam, np.float64)
    fwd = np.asarray(target, np.float64) - o
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    fx = (width / 2) / math.tan(math.radians(hfov_deg) / 2)
    u = (np.arange(width) + 0.5 - width / 2) / fx
    v = (np.arange(height) + 0.5 - height / 2) / fx
    uu, vv = np.meshgrid(u, v)
    d = fwd[None, None, :] + uu[..., None] * right[None, None, :] - vv[..., None] * up[None, None, :]
    d = d.reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        best = np.full(len(d), np.inf)

        def take(t, ok):
            t = np.where(ok & (t > 1e-9), t, np.inf)
            np.minimum(best, t, out=best)

        def plane(axis, value, lo=None, hi=None):
            t = (value - o[axis]) / d[:, axis]
            ok = np.isfinite(t)
            if lo is not None:
                p = o[None, :] + t[:, None] * d
                for a in range(3):
                    if a != axis:
                        ok &= (p[:, a] >= lo[a]) & (p[:, a] <= hi[a])
            take(t, ok)

        plane(2, 0.0, (0.0, -0.4, 0.0), (1.2, 0.4, 0.0))          # table top
        plane(2, -0.75)                                            # floor
        plane(0, 2.5)                                              # back wall
        plane(1, 1.5)
        plane(1, -1.5)                                             # side walls
        for lo, hi in layout["boxes"]:
            lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
            t0 = (lo[None, :] - o[None, :]) / d
            t1 = (hi[None, :] - o[None, :]) / d
            tn = np.max(np.minimum(t0, t1), axis=1)
            tf = np.min(np.maximum(t0, t1), axis=1)
            take(tn, tn <= tf)
        for cx, cy, r, h in layout["cylinders"]:
            ox, oy = o[0] - cx, o[1] - cy
            a = d[:, 0] ** 2 + d[:, 1] ** 2
            b = 2 * (ox * d[:, 0] + oy * d[:, 1])
            c = ox * ox + oy * oy - r * r
            disc = b * b - 4 * a * c
            t = (-b - np.sqrt(np.maximum(disc, 0.0))) / (2 * a)
            z = o[2] + t * d[:, 2]
            take(t, (disc >= 0) & (z >= 0) & (z <= h))
            t = (h - o[2]) / d[:, 2]
            px, py = o[0] + t * d[:, 0] - cx, o[1] + t * d[:, 1] - cy
            take(t, px * px + py * py <= r * r)
    t = best + sigma * Stream(seed + 4, P_NOISE).normal(len(d))
    return (o[None, :] + t[:, None] * d).astype(np.float32)


# --------------------------------------------------------------------------------------
# Query spheres
# --------------------------------------------------------------------------------------

def cube_queries(m: int, seed: int, lo=-0.1, hi=1.1, rlo=0.01, rhi=0.08):
    st = Stream(seed, P_QUERIES)
    c = st.uniform(lo, hi, 3 * m).reshape(m, 3).astype(np.float32)
    r = st.uniform(rlo, rhi, m).astype(np.float32)
    return c, r


def room_queries(m: int, seed: int, rlo=0.02, rhi=0.10):
    st = Stream(seed, P_QUERIES)
    c = np.empty((m, 3), dtype=np.float32)
    c[:, 0] = st.uniform(0.0, 4.0, m)
    c[:, 1] = st.uniform(0.0, 4.0, m)
    c[:, 2] = st.uniform(0.0, 2.5, m)
    r = st.uniform(rlo, rhi, m).astype(np.float32)
    return c, r


# --------------------------------------------------------------------------------------
# Serial arm
# --------------------------------------------------------------------------------------

@dataclass
class ArmModel:
    """A serial arm as spheres.

    Joint j rotates about its local axis `axis[j]` (0 = x, 1 = y, 2 = z) by q_j, then the
    frame translates by `link[j]` (expressed in the rotated frame).  Sphere s hangs on
    link `sphere_link[s]`: centre = origin of that link + R_link @ sphere_offset[s], with
    R_link the rotation after joint `sphere_link[s]`.
    """
    base: np.ndarray
    axis: np.ndarray
    link: np.ndarray
    sphere_link: np.ndarray
    sphere_offset: np.ndarray
    sphere_radius: np.ndarray
    joint_lo: float = -2.8
    joint_hi: float = 2.8

    @property
    def n_joints(self):
        return len(self.axis)

    @property
    def n_spheres(self):
        return len(self.sphere_radius)


def arm_7dof(n_spheres: int = 60) -> ArmModel:
    """7 revolute joints alternating local z / y; link lengths (m) along local z.

    Spheres s = 0..S-1 sit at arc length (s + 0.5)/S * sum(L) along the polyline through
    the joint origins and the tip; radius 0.08 - 0.06 * s/(S-1).
    """
    L = np.array([0.333, 0.0, 0.316, 0.0825, 0.384, 0.0, 0.107])
    axis = np.array([2, 1, 2, 1, 2, 1, 2], dtype=np.int32)
    link = np.zeros((7, 3))
    link[:, 2] = L
    cum = np.concatenate([[0.0], np.cumsum(L)])
    total = cum[-1]
    s_link = np.empty(n_spheres, dtype=np.int32)
    s_off = np.zeros((n_spheres, 3))
    for s in range(n_spheres):
        a = (s + 0.5) / n_spheres * total
        j = int(np.searchsorted(cum, a, side="right") - 1)
        j = min(j, 6)
        while L[j] == 0.0:      # arc positions never fall strictly inside a zero-length link
            j -= 1
        s_link[s] = j
        s_off[s, 2] = a - cum[j]
    rad = 0.08 - 0.06 * np.arange(n_spheres) / max(n_spheres - 1, 1)
    return ArmModel(
        base=np.array([-0.15, 0.0, 0.0], dtype=np.float32),
        axis=axis,
        link=link.astype(np.float32),
        sphere_link=s_link,
        sphere_offset=s_off.astype(np.float32),
        sphere_radius=rad.astype(np.float32),
    )


def fk_centers(arm: ArmModel, q: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """Sphere centres for configurations q [C, J]: float64 kinematics rounded to float32.

    Returns float32 [C, S, 3].  This is workload generation (the inputs of the
    configuration and trajectory queries), not the FP32 kinematics evaluated inside the
    edge validator.
    """
    q = np.asarray(q, dtype=np.float64)
    C = q.shape[0]
    out = np.empty((C, arm.n_spheres, 3), dtype=np.float32)
    base = arm.base.astype(np.float64)
    link = arm.link.astype(np.float64)
    off = arm.sphere_offset.astype(np.float64)
    for c0 in range(0, C, chunk):
        qq = q[c0:c0 + chunk]
        m = qq.shape[0]
        R = np.broadcast_to(np.eye(3), (m, 3, 3)).copy()
        p = np.broadcast_to(base, (m, 3)).copy()
        origins, frames = [], []
        for j in range(arm.n_joints):
            c, s = np.cos(qq[:, j]), np.sin(qq[:, j])
            Rot = np.zeros((m, 3, 3))
            ax = arm.axis[j]
            i1, i2 = [(1, 2), (2, 0), (0, 1)][ax]
            Rot[:, ax, ax] = 1.0
            Rot[:, i1, i1] = c
            Rot[:, i1, i2] = -s
            Rot[:, i2, i1] = s
            Rot[:, i2, i2] = c
            R = R @ Rot
            origins.append(p.copy())
            frames.append(R.copy())
            p = p + R @ link[j]
        O = np.stack(origins, 1)            # [m, J, 3]
        F = np.stack(frames, 1)             # [m, J, 3, 3]
        sl = arm.sphere_link
        cen = O[:, sl, :] + np.einsum("mjab,jb->mja", F[:, sl], off)
        out[c0:c0 + m] = cen.astype(np.float32)
    return out


def random_configs(C: int, seed: int, n_joints: int = 7, lo=-2.8, hi=2.8, first: int = 0) -> np.ndarray:
    """Configurations first .. first + C - 1 of the seed's configuration stream, so that
    disjoint ranges (one per process) are slices of one global sequence."""
    st = Stream(seed, P_CONFIGS)
    st.counter = first * n_joints
    return st.uniform(lo, hi, C * n_joints).reshape(C, n_joints).astype(np.float32)


def tabletop_scene(seed: int = 1001):
    """The tabletop cloud (30,000 points) and the arm used by every tabletop workload."""
    pts, layout = tabletop_cloud(seed)
    return pts, layout, arm_7dof()


def random_edges(E: int, seed: int, n_joints: int = 7, lo=-2.8, hi=2.8, step=0.01,
                 nmin=5, nmax=500):
    """Straight joint-space edges with uneven interpolation counts.

    n_e ~ U{nmin..nmax}; direction u with max-norm 1 (one random coordinate +-1, the
    others U[-1,1]); q_b = q_a + step * (n_e - 1) * u, so consecutive interpolated
    configurations are `step` rad apart in max-norm.  q_a is uniform over the set that
    keeps both ends inside [lo, hi]^J (equivalent to rejection sampling).
    Returns (qa float32 [E,J], qb float32 [E,J], nsteps int32 [E]).
    """
    st = Stream(seed, P_CONFIGS)
    n = st.integers(nmin, nmax, E)
    u = st.uniform(-1.0, 1.0, E * n_joints).reshape(E, n_joints)
    k = st.integers(0, n_joints - 1, E)
    sgn = np.where(st.uniform01(E) < 0.5, -1.0, 1.0)
    u[np.arange(E), k] = sgn
    delta = step * (n - 1)[:, None] * u
    qlo = np.maximum(lo, lo - delta)
    qhi = np.minimum(hi, hi - delta)
    qa = qlo + (qhi - qlo) * st.uniform01(E * n_joints).reshape(E, n_joints)
    qb = qa + delta
    return qa.astype(np.float32), qb.astype(np.float32), n.astype(np.int32)


def random_trajectories(T: int, W: int, seed: int, n_joints: int = 7, lo=-2.8, hi=2.8,
                        max_step=0.05) -> np.ndarray:
    """Random-walk trajectories: q_0 ~ U[lo,hi]^J, then steps U[-max_step, max_step]^J, clipped."""
    st = Stream(seed, P_CONFIGS)
    q = np.empty((T, W, n_joints))
    q[:, 0] = st.uniform(lo, hi, T * n_joints).reshape(T, n_joints)
    steps = st.uniform(-max_step, max_step, T * (W - 1) * n_joints).reshape(T, W - 1, n_joints)
    for w in range(1, W):
        q[:, w] = np.clip(q[:, w - 1] + steps[:, w - 1], lo, hi)
    return q.astype(np.float32)


# --------------------------------------------------------------------------------------
# The five workloads (sizes; the recipes live in the functions above)
# --------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    seed: int
    params: dict = field(default_factory=dict)


WORKLOADS = {
    "uniform2k": Workload("uniform2k", 1000, dict(n_points=2000, r_min=0.01, r_max=0.08, n_spheres=100_000)),
    "tabletop_configs": Workload("tabletop_configs", 1001, dict(n_raw=30000, sigma=0.002, r_filter=0.01,
                                                                r_min=0.02, r_max=0.08, n_configs=1 << 20)),
    "tabletop_edges": Workload("tabletop_edges", 1002, dict(n_edges=4096, r_min=0.02, r_max=0.08)),
    "tabletop_clearance": Workload("tabletop_clearance", 1003, dict(n_traj=16384, n_way=32, r_min=0.0,
                                                                    r_max=0.08, margin=0.01)),
    "room200k": Workload("room200k", 1004, dict(n_points=200_000, sigma=0.003, r_min=0.02, r_max=0.10,
                                                n_spheres=1 << 22)),
}
