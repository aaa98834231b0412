"""The distance-bound grid (capt_build_grid) and the configuration query that uses it.

1. The grid's two bounds, checked directly: for sampled centres x (random in and around
   the grid box, near the cloud's points, on cell boundaries) the cell the kernels would
   pick (the same FP32 index arithmetic, in numpy) must bound the exact FP64 distance
   from x to the cloud from below, and from above where an upper bound is stored, each
   with the 9.8e-6 relative margin the exactness argument needs.
2. Flags with grid = 1 are those of the oracle, bit for bit, on every launch
   configuration, on ragged batches and sphere counts that are not multiples of 4, on
   degenerate clouds, with a coarse and a fine grid, after the replicated sets are
   dropped, and at full size."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GRID_CFGS = [(w, s, ch, pf) for w in (4, 8, 16) for s in (2, 4, 8, 16) for ch in (0, 1) for pf in (0, 1)]


@pytest.fixture(scope="module")
def torch_():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cuda(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def scene(orc, capt_lib, torch_):
    raw, _, arm = W.tabletop_scene(1001)
    kept = capt_lib.sfc_filter(raw, 0.01)
    assert np.array_equal(kept, orc.sfc_filter(raw, 0.01))
    pts = raw[kept]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_build_grid(tree)
    return dict(pts=pts, arm=arm, tree=tree)


def _cell_of(shape, x):
    """The kernels' cell of each centre: floor(fl(fl(x - origin) * inv_cell)) clamped,
    with its 'inside the grid box' flag (numpy float32 arithmetic rounds like the
    kernels' __fsub_rn / __fmul_rn)."""
    x = x.astype(np.float32)
    u = (x - shape["origin"]).astype(np.float32) * shape["inv_cell"]
    u = u.astype(np.float32)
    dims = np.array(shape["dims"])
    inside = np.all((u >= 0) & (u < dims.astype(np.float32)), axis=1)
    idx = np.minimum(np.maximum(u, 0), (dims - 1).astype(np.float32)).astype(np.int64)
    return idx, inside


def test_grid_bounds_hold(scene, capt_lib):
    from scipy.spatial import cKDTree
    pts = scene["pts"]
    shape, cells = capt_lib.capt_grid_export(scene["tree"])
    assert shape is not None and cells.shape[:3] == tuple(reversed(shape["dims"]))
    st = capt_lib.capt_stats(scene["tree"])
    assert st["grid_dims"] == list(shape["dims"]) and st["grid_cell"] == shape["cell"]
    rng = np.random.default_rng(3)
    lo = shape["origin"].astype(np.float64)
    hi = lo + np.array(shape["dims"]) * float(shape["cell"])
    xs = [rng.uniform(lo - 0.05, hi + 0.05, (100000, 3)),                          # in and around the box
          pts[rng.integers(0, len(pts), 100000)] + rng.normal(0, 0.02, (100000, 3)),   # near the cloud
          pts[rng.integers(0, len(pts), 20000)]]                                   # on the points
    # on cell boundaries (and one float step either side)
    b = rng.uniform(lo, hi, (20000, 3))
    ax = rng.integers(0, 3, 20000)
    k = rng.integers(0, np.array(shape["dims"])[ax] + 1)
    b[np.arange(20000), ax] = lo[ax] + k * float(shape["cell"])
    xs += [b, np.nextafter(b.astype(np.float32), np.float32(np.inf)), np.nextafter(b.astype(np.float32), -np.inf)]
    x = np.concatenate([a.astype(np.float32) for a in xs])
    D = cKDTree(pts.astype(np.float64)).query(x.astype(np.float64))[0]
    idx, inside = _cell_of(shape, x)
    q = cells[idx[:, 2], idx[:, 1], idx[:, 0]]
    lb = q[:, 0].astype(np.float32) * shape["unit"]
    ub = q[:, 1].astype(np.float32) * shape["unit"]
    assert np.all(lb.astype(np.float64) <= D * (1 - 9e-6)), "a lower bound exceeds the distance"
    has_ub = inside & (q[:, 1] < 255)
    assert np.all(ub[has_ub].astype(np.float64) >= D[has_ub] * (1 + 9e-6)), "an upper bound is below the distance"
    # the grid decides something: many centres near the cloud get both bounds
    assert has_ub.mean() > 0.2 and (q[:, 0] > 0).mean() > 0.2


@pytest.mark.parametrize("warps,spl,chunk,pf", GRID_CFGS)
def test_grid_configs_every_launch_cfg(scene, orc, capt_lib, torch_, warps, spl, chunk, pf):
    cen = W.fk_centers(scene["arm"], W.random_configs(3001, 1001, first=555))   # odd: ragged last tile
    r = scene["arm"].sphere_radius
    ref = orc.brute_config_flags(scene["pts"], cen, r)
    t = scene["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, warps, spl, 0, chunk, pf, 1)
    f = capt_lib.capt_query_configs(t, _cuda(torch_, cen), _cuda(torch_, r))
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, 1)
    assert np.array_equal(f.cpu().numpy(), ref)
    assert capt_lib.capt_device_status(t) == 0


@pytest.mark.parametrize("max_cells", [64, 4096, 1 << 18, 1 << 22])
@pytest.mark.parametrize("S", [1, 7, 33, 60, 64])
def test_grid_configs_sphere_counts_and_grid_sizes(scene, orc, capt_lib, torch_, max_cells, S):
    """S not a multiple of 4 takes the general stream path; coarse grids decide little,
    fine ones most."""
    pts = scene["pts"]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_build_grid(tree, max_cells)
    dims = capt_lib.capt_stats(tree)["grid_dims"]
    assert 0 < dims[0] * dims[1] * dims[2] <= max_cells
    rng = np.random.default_rng(S)
    lo, hi = pts.min(0), pts.max(0)
    C = 1537
    # each configuration a cluster of spheres (like an arm) around a centre in and around
    # the cloud's box; a quarter of the centres on cloud points
    c0 = rng.uniform(lo - 0.3, hi + 0.3, (C, 1, 3))
    k = C // 4
    c0[:k, 0] = pts[rng.integers(0, len(pts), k)]
    cen = (c0 + rng.normal(0, 0.06, (C, S, 3))).astype(np.float32)
    r = rng.uniform(0.02, 0.08, S).astype(np.float32)
    ref = orc.brute_config_flags(pts, cen, r)
    assert 0.1 < ref.mean() < 0.9
    for spl in (2, 16):
        capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 8, spl, 0, 1, 0, 1)
        f = capt_lib.capt_query_configs(tree, _cuda(torch_, cen), _cuda(torch_, r))
        assert np.array_equal(f.cpu().numpy(), ref), spl
    assert capt_lib.capt_device_status(tree) == 0


@pytest.mark.parametrize("kind", ["one", "two", "five", "duplicates", "plane", "line"])
def test_grid_degenerate_clouds(orc, capt_lib, torch_, kind):
    rng = np.random.default_rng(11)
    pts = {"one": np.array([[0.5, 0.5, 0.5]]), "two": np.array([[0.1, 0.2, 0.3], [0.15, 0.2, 0.3]]),
           "five": rng.random((5, 3)), "duplicates": np.repeat([[0.3, 0.3, 0.3]], 40, 0),
           "plane": np.c_[rng.random((500, 2)), np.zeros(500)],
           "line": np.c_[np.linspace(0, 1, 300), np.zeros(300), np.zeros(300)]}[kind].astype(np.float32)
    tree = capt_lib.capt_build(pts, 0.01, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_build_grid(tree, 1 << 16)
    S = 12
    C = 700
    cen = (pts[rng.integers(0, len(pts), (C, S))] + rng.normal(0, 0.05, (C, S, 3))).astype(np.float32)
    r = rng.uniform(0.01, 0.08, S).astype(np.float32)
    ref = orc.brute_config_flags(pts, cen, r)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 8, 4, 0, 1, 0, 1)
    f = capt_lib.capt_query_configs(tree, _cuda(torch_, cen), _cuda(torch_, r))
    assert np.array_equal(f.cpu().numpy(), ref)


def test_grid_empty_cloud_and_rebuild(orc, capt_lib, torch_):
    tree = capt_lib.capt_build(np.zeros((0, 3), np.float32), 0.01, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_build_grid(tree)
    assert capt_lib.capt_grid_export(tree) == (None, None)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 8, 4, 0, 1, 0, 1)
    f = capt_lib.capt_query_configs(tree, _cuda(torch_, np.zeros((10, 4, 3), np.float32)),
                                    _cuda(torch_, np.full(4, 0.05, np.float32)))
    assert not f.cpu().numpy().any()
    pts = W.uniform_cloud(300, 4)
    t2 = capt_lib.capt_build(pts, 0.01, 0.08)
    capt_lib.capt_upload(t2, 0)
    for cells in (1 << 12, 1 << 16, 1 << 12):   # rebuilding replaces the grid
        capt_lib.capt_build_grid(t2, cells)
        d = capt_lib.capt_stats(t2)["grid_dims"]
        assert d[0] * d[1] * d[2] <= cells
    with pytest.raises(capt_lib.CaptError):
        capt_lib.capt_build_grid(t2, 1 << 29)


def test_grid_after_dropping_the_replicated_sets(scene, orc, capt_lib, torch_):
    pts = scene["pts"]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_build_grid(tree)
    capt_lib.capt_compact(tree, drop_full=True)
    with pytest.raises(capt_lib.CaptError):
        capt_lib.capt_build_grid(tree)          # needs the replicated sets
    cen = W.fk_centers(scene["arm"], W.random_configs(2000, 1001, first=9))
    r = scene["arm"].sphere_radius
    ref = orc.brute_config_flags(pts, cen, r)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 16, 4, 0, capt_lib.CAPT_SCAN_COMPACT, 0, 1)
    f = capt_lib.capt_query_configs(tree, _cuda(torch_, cen), _cuda(torch_, r))
    assert np.array_equal(f.cpu().numpy(), ref)


def test_grid_configs_full_size(scene, orc, capt_lib, torch_):
    """1,048,576 configurations with the grid, against the oracle's plain CAPT (every flag)."""
    C = 1 << 20
    cen = W.fk_centers(scene["arm"], W.random_configs(C, 1001))
    r = scene["arm"].sphere_radius
    t = scene["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 16, 4, 0, 1, 1, 1)
    f = capt_lib.capt_query_configs(t, _cuda(torch_, cen), _cuda(torch_, r)).cpu().numpy()
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, 1)
    ref, _ = orc.PlainCAPT(scene["pts"], 0.02, 0.08).query_configs(cen, r)
    assert np.array_equal(f, ref)
    assert capt_lib.capt_device_status(t) == 0


SPHERE_CFGS = [(w, s, st, ch) for w in (4, 8, 16) for s in (1, 2, 4, 8) for st in (0, 1) for ch in (0, 1)]


@pytest.mark.parametrize("warps,spl,stage,chunk", SPHERE_CFGS)
def test_grid_spheres_every_launch_cfg(scene, orc, capt_lib, torch_, warps, spl, stage, chunk):
    """Sphere queries with the grid: ragged batch, centres in and around the cloud's box
    and on its surfaces, against FP32 brute force."""
    pts = scene["pts"]
    rng = np.random.default_rng(7)
    lo, hi = pts.min(0), pts.max(0)
    m = 20001
    c = rng.uniform(lo - 0.1, hi + 0.1, (m, 3)).astype(np.float32)
    c[: m // 2] = (pts[rng.integers(0, len(pts), m // 2)] + rng.normal(0, 0.04, (m // 2, 3))).astype(np.float32)
    r = rng.uniform(0.02, 0.08, m).astype(np.float32)
    ref = orc.brute_flags(pts, c, r)
    assert 0.1 < ref.mean() < 0.9
    t = scene["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, warps, spl, stage, chunk, 0, 1)
    f = capt_lib.capt_query_spheres(t, _cuda(torch_, c), _cuda(torch_, r))
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 1, 0)
    assert np.array_equal(f.cpu().numpy(), ref)
    assert capt_lib.capt_device_status(t) == 0


@pytest.mark.parametrize("mode", ["persistent", "per_edge", "plan", "static"])
def test_grid_edges_match_oracle(scene, orc, capt_lib, torch_, mode):
    """Edges with the grid: a sphere the grid proves colliding invalidates its edge at
    once; flags equal the oracle's interpolation + kinematics + brute force."""
    arm = scene["arm"]
    qa, qb, ns = W.random_edges(600, 1014, nmax=120)
    ref = orc.edges(arm, qa, qb, ns, points=scene["pts"])
    assert 0.05 < ref.mean() < 0.95
    t = scene["tree"]
    dqa, dqb, dns = _cuda(torch_, qa), _cuda(torch_, qb), _cuda(torch_, ns)
    valid = torch_.empty(len(ns), dtype=torch_.uint8, device="cuda")
    for warps, stage, chunk in ((8, 0, 32), (16, 1, 64), (4, 0, 128)):
        cfg = dict(warps_per_block=warps, spheres_per_lane=1, staging=stage, chunk=chunk, prefetch=0, grid=1)
        if mode == "plan":
            plan = capt_lib.capt_edge_plan_create(t, arm, dqa, dqb, dns, valid, cfg=cfg)
            capt_lib.capt_edge_plan_launch(plan)
            capt_lib.capt_edge_plan_launch(plan)
            capt_lib.capt_edge_plan_free(plan)
        else:
            capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_EDGES, warps, 1, stage, chunk, 0, 1)
            if mode == "static":
                capt_lib.capt_validate_edges_static(t, arm, dqa, dqb, dns, valid)
            else:
                capt_lib.capt_validate_edges(t, arm, dqa, dqb, dns, valid,
                                             mode=capt_lib.CAPT_EDGES_PER_EDGE if mode == "per_edge"
                                             else capt_lib.CAPT_EDGES_PERSISTENT)
        torch_.cuda.synchronize()
        assert np.array_equal(valid.cpu().numpy(), ref), (mode, warps, stage, chunk)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_EDGES, 8, 2, 1, 32)
    assert capt_lib.capt_device_status(t) == 0


@pytest.mark.parametrize("warps,stage", [(2, 0), (4, 1), (8, 0), (16, 0)])
def test_grid_joint_configs_match_oracle(scene, orc, capt_lib, torch_, warps, stage):
    arm = scene["arm"]
    q = W.random_configs(3001, 1015)
    ref = orc.brute_config_flags(scene["pts"], orc.fk32(arm, q), arm.sphere_radius)
    t = scene["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_JOINTS, warps, 1, stage, 0, 0, 1)
    f = capt_lib.capt_query_joint_configs(t, arm, _cuda(torch_, q))
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_JOINTS, 4, 1, 0, 0)
    assert np.array_equal(f.cpu().numpy(), ref)
    assert capt_lib.capt_device_status(t) == 0


def test_grid_edges_and_joints_on_compact_sets(scene, orc, capt_lib, torch_):
    """After the replicated sets are dropped the edge and joint-angle kernels scan the
    compact sets; the grid built before the drop still decides most spheres."""
    pts = scene["pts"]
    arm = scene["arm"]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_build_grid(tree)
    capt_lib.capt_compact(tree, drop_full=True)
    qa, qb, ns = W.random_edges(400, 1016, nmax=80)
    ref = orc.edges(arm, qa, qb, ns, points=pts)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_EDGES, 8, 1, 0, 32, 0, 1)
    v = capt_lib.capt_validate_edges(tree, arm, _cuda(torch_, qa), _cuda(torch_, qb), _cuda(torch_, ns))
    assert np.array_equal(v.cpu().numpy(), ref)
    q = W.random_configs(2000, 1017)
    refj = orc.brute_config_flags(pts, orc.fk32(arm, q), arm.sphere_radius)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_JOINTS, 8, 1, 0, 0, 0, 1)
    f = capt_lib.capt_query_joint_configs(tree, arm, _cuda(torch_, q))
    assert np.array_equal(f.cpu().numpy(), refj)
