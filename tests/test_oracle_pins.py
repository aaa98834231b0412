"""Pins for the CPU oracle: what the paper and the mathematics fix, independent of the
oracle's own code.  Each test names the part of the oracle it pins and the kind of
mistake it would catch.  No GPU."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_trees.json")))


def fp64_flags(points, centers, radii):
    p = points.astype(np.float64)
    out = []
    for x, r in zip(centers.astype(np.float64), radii.astype(np.float64)):
        d2 = ((p - x) ** 2).sum(1)
        out.append(d2.min() <= r * r)
    return np.array(out, np.uint8)


# ------------------------------------------------------------------ 1. brute force ----

def test_brute_boundary_is_inclusive(orc):
    """d^2 = r^2 exactly (0.75^2 + 1^2 = 1.25^2 in binary) hits; one ulp less misses."""
    p = np.zeros((1, 3), np.float32)
    c = np.array([[0.75, 1.0, 0.0], [0.75, 1.0, 0.0]], np.float32)
    r = np.array([1.25, np.nextafter(np.float32(1.25), np.float32(0))], np.float32)
    assert orc.brute_flags(p, c, r).tolist() == [1, 0]


def test_brute_uses_every_axis(orc):
    """A dropped or swapped coordinate term would flip one of these."""
    p = np.array([[0.0, 0.0, 0.0]], np.float32)
    c = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.25, 0.25, 0.25]], np.float32)
    r = np.full(4, 0.5, np.float32)
    assert orc.brute_flags(p, c, r).tolist() == [0, 0, 0, 1]
    # a point displaced along one axis only: offsets (-0.4, 0.2, 0.3) give d^2 = 0.29 <= 0.3^2? no
    p2 = np.array([[0.4, -0.2, -0.3]], np.float32)
    c2 = np.zeros((2, 3), np.float32)
    r2 = np.array([0.5, 0.6], np.float32)   # 0.25 < 0.29 < 0.36
    assert orc.brute_flags(p2, c2, r2).tolist() == [0, 1]


def test_brute_matches_fp64_up_to_rounding(orc):
    """FP32 and FP64 brute force may disagree only where |d^2 - r^2| <= 1e-6 r^2."""
    pts = W.uniform_cloud(500, 7)
    c, r = W.cube_queries(4000, 8)
    f32 = orc.brute_flags(pts, c, r)
    f64 = fp64_flags(pts, c, r)
    bad = np.nonzero(f32 != f64)[0]
    if len(bad):
        gap = orc.min_gap64(pts, c[bad], r[bad])
        assert np.all(gap <= 1e-6 * r[bad].astype(np.float64) ** 2)
    assert 0.05 < f32.mean() < 0.95


def test_brute_config_flags_is_or_over_spheres(orc):
    pts = W.uniform_cloud(300, 3)
    c, _ = W.cube_queries(50 * 7, 4)
    c = c.reshape(50, 7, 3)
    r = np.linspace(0.01, 0.05, 7).astype(np.float32)
    per = orc.brute_flags(pts, c.reshape(-1, 3), np.tile(r, 50)).reshape(50, 7)
    assert orc.brute_config_flags(pts, c, r).tolist() == per.max(1).tolist()


# ----------------------------------------------------------- 3. plain CAPT (Alg. 1/3) ----

@pytest.mark.parametrize("case", GOLD["trees"], ids=[t["name"] for t in GOLD["trees"]])
def test_capt_hand_derived_trees(orc, case):
    t = orc.PlainCAPT(np.array(case["points"], np.float32), case["r_min"], case["r_max"])
    e = t.export()
    assert e["T"].tolist() == case["T"]
    sets = [e["set_idx"][e["set_begin"][l]:e["set_begin"][l + 1]].tolist() for l in range(t.N)]
    assert sets == case["sets"]
    np.testing.assert_array_equal(e["aabb"], np.array(case["aabb"], np.float32))
    for q in case["queries"]:
        f, leaf, _ = t.query(np.array([q["center"]], np.float32), np.array([q["r"]], np.float32))
        assert (int(leaf[0]), int(f[0])) == (q["leaf"], q["flag"]), q
        assert orc.brute_flags(np.array(case["points"], np.float32), np.array([q["center"]], np.float32),
                               np.array([q["r"]], np.float32))[0] == q["flag"]


def _tiny_clouds():
    rng = np.random.default_rng(5)
    out = []
    for n in (1, 2, 3, 5, 8, 13, 31, 64):
        out.append(("uniform", n, rng.random((n, 3)).astype(np.float32)))
        # grid-aligned coordinates: many points on split planes and duplicated keys
        out.append(("grid", n, (rng.integers(0, 4, (n, 3)) * 0.25).astype(np.float32)))
    return out


@pytest.mark.parametrize("kind,n,pts", _tiny_clouds(), ids=lambda v: str(v) if not hasattr(v, "shape") else "")
def test_capt_lemma1_matches_brute_force(orc, kind, n, pts):
    """Lemma 1: for r in [r_min, r_max] the CAPT answer equals brute force, exactly."""
    r_min, r_max = 0.05, 0.3
    t = orc.PlainCAPT(pts, r_min, r_max)
    g = np.arange(-0.25, 1.26, 0.125, dtype=np.float32)        # includes every grid plane
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    c = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1).astype(np.float32)
    for r in (r_min, 0.125, 0.2, r_max):
        rr = np.full(len(c), r, np.float32)
        f, leaf, _ = t.query(c, rr)
        assert np.array_equal(f, orc.brute_flags(pts, c, rr)), r
        assert leaf.min() >= 0 and leaf.max() < t.N
    rng = np.random.default_rng(n)
    c2 = rng.uniform(-0.3, 1.3, (3000, 3)).astype(np.float32)
    r2 = rng.uniform(r_min, r_max, 3000).astype(np.float32)
    assert np.array_equal(t.query(c2, r2)[0], orc.brute_flags(pts, c2, r2))


def _check_structure(orc, pts, r_min, r_max):
    t = orc.PlainCAPT(pts, r_min, r_max)
    e = t.export()
    n = len(pts)
    N = t.N
    assert N >= max(n, 1) and (N & (N - 1)) == 0 and N < 2 * max(n, 1)
    p64 = pts.astype(np.float64)
    for l in range(N):
        s = e["set_idx"][e["set_begin"][l]:e["set_begin"][l + 1]]
        cell = e["cell"][l]
        assert np.all(np.diff(s.astype(np.int64)) > 0)           # ascending, no duplicates
        assert np.all(s < n)                                    # no pads stored
        q = np.clip(p64, cell[:3], cell[3:])
        dist2 = ((p64 - q) ** 2).sum(1)
        must = np.nonzero(dist2 <= float(r_max) ** 2)[0]
        if e["pruned"][l]:
            assert len(s) == 1
            t_ = p64[s[0]]
            corners = np.array([[cell[3 * ((k >> a) & 1) + a] for a in range(3)] for k in range(8)])
            assert np.all(np.isfinite(corners))
            assert np.all(np.sqrt(((corners - t_) ** 2).sum(1)) <= r_min)
            assert np.all(dist2[s] == 0.0)                      # the representative lies in c
        else:
            # affordance invariant: every point within r_max of the cell is stored
            assert set(must.tolist()) <= set(s.tolist()), l
        if len(s):
            np.testing.assert_array_equal(e["aabb"][l, :3], pts[s].min(0))
            np.testing.assert_array_equal(e["aabb"][l, 3:], pts[s].max(0))
    return t, e


@pytest.mark.parametrize("n,scale", [(1, 0.5), (7, 0.5), (64, 0.5), (200, 0.5), (1000, 0.5), (1000, 0.08)])
def test_capt_affordance_invariant(orc, n, scale):
    """Every point within r_max of a cell is in that cell's set (Sec. IV-A, Lemma 1 case 1);
    pruned cells lie within r_min of their representative (Alg. 1, Sec. IV-B)."""
    pts = W.uniform_cloud(n, 100 + n) * np.float32(scale)
    t, e = _check_structure(orc, pts, 0.02, 0.08)
    if scale < 0.1:
        assert t.n_pruned > 0       # the dense cloud exercises the r_min prune


def test_capt_leaf_cells_tile_space_and_contain_queries(orc):
    pts = W.uniform_cloud(300, 11)
    t = orc.PlainCAPT(pts, 0.01, 0.1)
    e = t.export()
    c, r = W.cube_queries(5000, 12)
    _, leaf, _ = t.query(c, r)
    cell = e["cell"][leaf]
    assert np.all(c >= cell[:, :3]) and np.all(c <= cell[:, 3:])
    # every representative (one real point per leaf of the first n) lies in its own cell
    assert np.isinf(e["cell"]).any()


def test_capt_empty_cloud_and_single_point(orc):
    t = orc.PlainCAPT(np.zeros((0, 3), np.float32), 0.0, 0.1)
    assert t.N == 1 and t.total == 0
    c, r = W.cube_queries(100, 1)
    assert t.query(c, r)[0].sum() == 0
    p = np.array([[0.5, 0.5, 0.5]], np.float32)
    t1 = orc.PlainCAPT(p, 0.0, 1.0)
    assert np.array_equal(t1.query(c, r)[0], orc.brute_flags(p, c, r))


def test_capt_radius_at_both_ends(orc):
    pts = W.uniform_cloud(2000, 21)
    t = orc.PlainCAPT(pts, 0.01, 0.08)
    c, _ = W.cube_queries(20000, 22)
    for rv in (0.01, 0.08):
        r = np.full(len(c), rv, np.float32)
        assert np.array_equal(t.query(c, r)[0], orc.brute_flags(pts, c, r))


def test_capt_nearest_is_exact_within_rmax(orc):
    """With r_min = 0 every leaf keeps all points within r_max of its cell, so the
    nearest point inside the set is the global nearest whenever it is <= r_max."""
    pts = W.uniform_cloud(1500, 31)
    t = orc.PlainCAPT(pts, 0.0, 0.08)
    c, _ = W.cube_queries(5000, 32)
    d_set, i_set = t.nearest64(c, 0.08)
    d_all, i_all, _ = orc.nearest64(pts, c)
    near = d_all < 0.08
    assert near.any() and (~near).any()
    np.testing.assert_array_equal(d_set[near], d_all[near])
    np.testing.assert_array_equal(i_set[near], i_all[near])
    assert np.all(d_set[~near] == 0.08) and np.all(i_set[~near] == -1)


# ----------------------------------------------------------------- 4. filter (Alg. 2) ----

def test_morton_keys_hand_computed(orc):
    for case in GOLD["morton"]["cases"]:
        assert orc.morton_key(case["q"], case["perm"]) == case["key"], case


def test_filter_on_a_line_is_greedy_spacing(orc):
    g = GOLD["filter_line"]
    x = np.array(g["points_x"], np.float32)
    pts = np.stack([x, np.full_like(x, 0.5), np.full_like(x, -1.0)], 1)
    kept = orc.sfc_filter(pts, g["r_filter"])
    assert kept.tolist() == g["kept"]
    # shuffled input order gives the same set (the curve order does not depend on it)
    perm = np.array([4, 1, 5, 0, 3, 2])
    kept2 = orc.sfc_filter(pts[perm], g["r_filter"])
    assert sorted(perm[kept2].tolist()) == g["kept"]


def test_filter_invariants(orc):
    """Output is a subset; within a pass a point is removed only when the retained
    anchor it was compared with is within r_filter (Lemma 2's premise); across the six
    passes every removed point is within 6 r_filter of the output (triangle
    inequality); consecutive output points are farther apart than r_filter."""
    pts, _ = W.tabletop_cloud(1001, n=6000)
    rf = 0.01
    kept, passes = orc.sfc_filter(pts, rf, trace=True)
    assert len(set(kept.tolist())) == len(kept) and kept.max() < len(pts)
    prev = np.arange(len(pts))
    for order, anchor in passes:
        assert sorted(order.tolist()) == sorted(prev.tolist())
        removed = order != anchor
        d = np.sqrt(((pts[order[removed]].astype(np.float64) - pts[anchor[removed]]) ** 2).sum(1))
        assert np.all(d <= rf * (1 + 1e-6))
        prev = np.unique(anchor)
        assert set(prev.tolist()) == set(order[~removed].tolist())
    assert sorted(prev.tolist()) == sorted(kept.tolist())
    gaps = np.sqrt(((pts[kept[1:]].astype(np.float64) - pts[kept[:-1]]) ** 2).sum(1))
    assert np.all(gaps > rf * (1 - 1e-6))
    dk, _, _ = orc.nearest64(pts[kept], pts)
    assert dk.max() <= 6 * rf * (1 + 1e-6)
    assert len(kept) < len(pts)


def test_filter_zero_radius_keeps_distinct_points(orc):
    pts = np.array([[0, 0, 0], [1, 1, 1], [0, 0, 0], [2, 2, 2]], np.float32)
    kept = orc.sfc_filter(pts, 0.0)
    assert sorted(pts[kept].tolist()) == [[0, 0, 0], [1, 1, 1], [2, 2, 2]]
    assert orc.sfc_filter(np.zeros((0, 3), np.float32), 0.1).tolist() == []


# ------------------------------------------------------------ 2. clearance (FP64) ----

def test_nearest_hand_case(orc):
    pts = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    d, i, s = orc.nearest64(pts, np.array([[0.25, 0, 0], [0.75, 0, 0], [0.5, 0, 0]], np.float32))
    assert d.tolist() == [0.25, 0.25, 0.5] and i.tolist() == [0, 1, 0] and s.tolist() == [0.75, 0.75, 0.5]


def test_clearance_special_cases(orc):
    pts = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    r = np.array([0.05, 0.02], np.float32)
    c = np.array([[[[0, 0, 0], [0.5, 0.5, 0.5]]]], np.float32)          # d = 0 and d > r_max
    cost, d, g = orc.clearance64(pts, c, r, 0.08, 0.01)
    assert d[0, 0].tolist() == [0.0, 0.08]
    assert np.all(g == 0.0)
    r0, r1 = (float(v) for v in r)                                    # the float32 radii
    assert cost[0] == pytest.approx((r0 + 0.01) ** 2 + max(0.0, r1 + 0.01 - 0.08) ** 2, abs=1e-15)


def test_clearance_gradient_matches_central_differences(orc):
    """d cost / d c against FP64 central differences (h = 1e-4) away from ties/kinks."""
    pts = W.uniform_cloud(400, 41) * np.float32(0.3)
    rng = np.random.default_rng(42)
    T, Wn, S = 3, 4, 5
    c = rng.uniform(-0.02, 0.32, (T, Wn, S, 3)).astype(np.float32)
    r = np.linspace(0.02, 0.08, S).astype(np.float32)
    g = rng.uniform(0.5, 2.0, T)
    r_max, margin, h = 0.08, 0.01, 1e-4
    cost, d, grad = orc.clearance64(pts, c, r, r_max, margin, grad_cost=g)
    dn, _, d2 = orc.nearest64(pts, c.reshape(-1, 3))
    checked = 0
    for k in range(T * Wn * S):
        t, s = k // (Wn * S), k % S
        ok = (d2[k] - dn[k] > 4 * h and abs(dn[k] - r_max) > 2 * h and
              abs(r[s] + margin - dn[k]) > 2 * h and dn[k] > 2 * h)
        if not ok:
            continue
        for a in range(3):
            # the oracle takes float32 centres: difference the FP64 cost in closed form
            # of the FP64 nearest distance instead, perturbing the point in FP64
            x = c.reshape(-1, 3)[k].astype(np.float64)
            vals = []
            for sgn in (+1, -1):
                y = x.copy()
                y[a] += sgn * h
                dd = np.sqrt(((pts.astype(np.float64) - y) ** 2).sum(1)).min()
                dd = min(dd, r_max)
                vals.append(g[t] * max(0.0, float(r[s]) + margin - dd) ** 2)
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grad.reshape(-1, 3)[k, a]
            assert abs(an - fd) <= 1e-3 * abs(fd) + 1e-6, (k, a, an, fd)
        checked += 1
    assert checked >= 10
    # and the cost sums the per-sphere hinge terms
    hh = np.maximum(0.0, r[None, None, :].astype(np.float64) + margin - d)
    np.testing.assert_allclose(cost, (hh ** 2).sum((1, 2)), rtol=0, atol=1e-15)


# ------------------------------------------------------------- 5. kinematics (FP32) ----

def test_sincos_against_libm():
    import oracle
    xs = np.concatenate([np.linspace(-3.2, 3.2, 4001), [0.0, math.pi / 2, -math.pi / 2, math.pi, 2.8, -2.8]])
    for x in xs.astype(np.float32):
        s, c = oracle.sincos32(float(x))
        assert abs(s - math.sin(float(x))) <= 4e-7 and abs(c - math.cos(float(x))) <= 4e-7, x
    assert oracle.sincos32(0.0) == (0.0, 1.0)


def test_fk32_hand_cases(orc):
    arm = W.arm_7dof()
    cum = np.concatenate([[0.0], np.cumsum([0.333, 0.0, 0.316, 0.0825, 0.384, 0.0, 0.107])])
    a_s = (np.arange(60) + 0.5) / 60 * cum[-1]
    cen = orc.fk32(arm, np.zeros((1, 7), np.float32))[0]
    np.testing.assert_allclose(cen[:, 0], -0.15, atol=0)
    np.testing.assert_allclose(cen[:, 1], 0.0, atol=0)
    np.testing.assert_allclose(cen[:, 2], a_s, atol=2e-7)
    # joint 1 (about y) at +pi/2 turns everything after the first link towards +x
    q = np.zeros((1, 7), np.float32)
    q[0, 1] = np.float32(math.pi / 2)
    cen = orc.fk32(arm, q)[0]
    after = a_s > 0.333
    np.testing.assert_allclose(cen[after, 0], -0.15 + (a_s[after] - 0.333), atol=1e-6)
    np.testing.assert_allclose(cen[after, 2], 0.333, atol=1e-6)
    np.testing.assert_allclose(cen[~after, 2], a_s[~after], atol=1e-6)


def test_fk32_matches_fp64_kinematics(orc):
    arm = W.arm_7dof()
    q = W.random_configs(2000, 77)
    np.testing.assert_allclose(orc.fk32(arm, q), W.fk_centers(arm, q), atol=1e-5, rtol=0)


def test_interp_endpoints(orc):
    qa = np.array([0.1, -0.2, 0.3], np.float32)
    qb = np.array([0.5, 0.2, -0.7], np.float32)
    q = orc.interp32(qa, qb, 5)
    np.testing.assert_array_equal(q[0], qa)
    np.testing.assert_allclose(q[-1], qb, atol=1e-7)
    np.testing.assert_allclose(q[2], (qa.astype(np.float64) + qb) / 2, atol=1e-7)


def test_edges_tree_equals_brute_force(orc):
    pts, _ = W.tabletop_cloud(1001, n=4000)
    arm = W.arm_7dof()
    qa, qb, ns = W.random_edges(64, 5, nmax=40)
    t = orc.PlainCAPT(pts, 0.02, 0.08)
    v_tree = orc.edges(arm, qa, qb, ns, tree=t)
    v_brute = orc.edges(arm, qa, qb, ns, points=pts)
    assert np.array_equal(v_tree, v_brute)
    assert 0 < v_tree.sum() < len(v_tree)
    # an edge is valid iff every interpolated configuration is collision-free
    for e in range(8):
        qs = orc.interp32(qa[e], qb[e], int(ns[e]))
        cen = orc.fk32(arm, qs)
        assert v_tree[e] == 1 - orc.brute_config_flags(pts, cen, arm.sphere_radius).max()
    ns0 = ns.copy()
    ns0[:4] = 0
    assert orc.edges(arm, qa, qb, ns0, tree=t)[:4].tolist() == [1, 1, 1, 1]


@pytest.mark.parametrize("case", [t for t in GOLD["trees"] if "config_queries" in t], ids=lambda t: t["name"])
def test_capt_hand_derived_work_counts(orc, case):
    """The oracle's Alg. 3 work counts (spheres examined up to each configuration's first
    hit, leaf box passes, points scanned up to the first hit), worked out by hand."""
    t = orc.PlainCAPT(np.array(case["points"], np.float32), case["r_min"], case["r_max"])
    q = case["config_queries"]
    flags, counts = t.query_configs(np.array(q["centers"], np.float32), np.array(q["radii"], np.float32))
    assert flags.tolist() == q["flags"]
    assert counts.tolist() == q["counts"]
