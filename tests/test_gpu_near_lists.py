"""Nearest-candidate lists of the clearance (capt_build_near_lists).

With lists (launch grid = 1) a centre near the cloud is answered from its grid cell's
list instead of the descent and the full scan of its leaf set (Lemma 1, case 1).  The
lists are built so that the answer is the paper's bit for bit, so every test here
compares the two paths' distances, indices and costs for equality, and the lists' path
with the FP64 oracle within the clearance tolerance (1e-5):
  - the tabletop clearance workload, three grid sizes;
  - adversarial centres: on and around the grid's cell faces, on cloud points, at the
    r_max shell, far away, on ragged trajectories;
  - degenerate clouds (one point, duplicates, a plane, a line);
  - a coarse grid whose cells overflow the builder (fallback cells take the paper's
    path);
  - the state rules (grid first, r_min = 0, rebuilds release the lists), the work
    counters and the autotuner;
  - the full bench workload."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


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
    return dict(pts=pts, arm=arm)


def _tree(capt_lib, pts, r_max=0.08):
    t = capt_lib.capt_build(pts, 0.0, r_max)
    capt_lib.capt_upload(t, 0)
    return t


def _both(capt_lib, torch_, t, cen, r, margin=0.01):
    """(paper path, lists path) outputs [cost, dist, argmin] as numpy."""
    dc, dr = _cuda(torch_, cen), _cuda(torch_, r)
    out = []
    for grid in (0, 1):
        capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE, 8, 2, 0, 0, 0, grid)
        cost, d, am = capt_lib.capt_clearance_fwd(t, dc, dr, margin)
        out.append([x.cpu().numpy() for x in (cost, d, am)])
    assert capt_lib.capt_device_status(t) == 0
    return out


def _equal(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.ascontiguousarray(x).view(np.uint32), np.ascontiguousarray(y).view(np.uint32))


def _check_oracle(orc, pts, cen, d, am, r_max, n=20000, seed=0):
    """A sample of the lists' distances against the FP64 nearest distance (1e-5), and the
    index where the runner-up is separated."""
    c = cen.reshape(-1, 3)
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(c), min(n, len(c)), replace=False)
    dn, ni, d2 = orc.nearest64(pts, c[idx])
    d, am = d.reshape(-1)[idx], am.reshape(-1)[idx]
    assert np.abs(d - np.minimum(dn, r_max)).max() <= 1e-5
    sep = (dn < r_max - 1e-5) & (d2 - dn > 1e-5)
    assert np.array_equal(am[sep], ni[sep])
    assert np.all(am[dn >= r_max + 1e-5] == -1)


@pytest.mark.parametrize("cells", [1 << 16, 1 << 20, 1 << 24])
def test_lists_match_the_paper_path_on_the_tabletop(scene, orc, capt_lib, torch_, cells):
    t = _tree(capt_lib, scene["pts"])
    capt_lib.capt_build_grid(t, cells)
    capt_lib.capt_build_near_lists(t)
    st = capt_lib.capt_stats(t)
    assert st["near_entries"] > 0 and st["near_entries"] % 4 == 0 and st["near_bytes"] > 0
    q = W.random_trajectories(1024, 32, 1003)
    cen = W.fk_centers(scene["arm"], q.reshape(-1, 7)).reshape(1024, 32, 60, 3)
    r = scene["arm"].sphere_radius
    a, b = _both(capt_lib, torch_, t, cen, r)
    _equal(a, b)
    assert (b[1] < 0.08).sum() > 5000
    _check_oracle(orc, scene["pts"], cen, b[1], b[2], 0.08)
    # the work counters follow the lists: every near sphere either has a list or falls back
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE, 8, 2, 0, 0, 0, 1)
    g = capt_lib.capt_count_clearance_work(t, _cuda(torch_, cen)).cpu().numpy()
    assert g[5] + g[7] == g[1] and g[5] > 0
    assert g[6] % 4 == 0
    if st["near_fallback_cells"] == 0:
        assert g[7] == 0 and g[2] == g[3] == g[4] == 0
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE, 8, 2, 0, 0, 0, 0)
    g0 = capt_lib.capt_count_clearance_work(t, _cuda(torch_, cen)).cpu().numpy()
    assert g0[1] == g[1] and g0[5] == g0[6] == g0[7] == 0 and g0[3] > g[6]   # fewer entries than points


def test_lists_on_adversarial_centres(scene, orc, capt_lib, torch_):
    """Centres on the grid's cell faces and one ulp either side, on cloud points, at
    distance r_max (1 +- 1e-6) from a point, far away, and a ragged trajectory shape."""
    pts = scene["pts"]
    t = _tree(capt_lib, pts)
    capt_lib.capt_build_grid(t, 1 << 20)
    capt_lib.capt_build_near_lists(t)
    shape, _ = capt_lib.capt_grid_export(t)
    rng = np.random.default_rng(11)
    n = 20000
    org, h = shape["origin"].astype(np.float64), float(shape["cell"])
    dims = np.array(shape["dims"])
    # cell faces: coordinates org + k h exactly (in FP64, then rounded), and one ulp off
    k = rng.integers(0, dims, (n, 3))
    face = (org + k * h).astype(np.float32)
    ax = rng.integers(0, 3, n)
    jitter = rng.uniform(0, 1, (n, 3)) * h
    c1 = (org + k * h + jitter).astype(np.float32)
    c1[np.arange(n), ax] = face[np.arange(n), ax]
    c1b = c1.copy()
    c1b[np.arange(n), ax] = np.nextafter(face[np.arange(n), ax], np.float32(np.inf))
    c1c = c1.copy()
    c1c[np.arange(n), ax] = np.nextafter(face[np.arange(n), ax], np.float32(-np.inf))
    # on points, at the r_max shell, far
    c2 = pts[rng.integers(0, len(pts), n // 4)]
    u = rng.normal(size=(n // 4, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c3 = (pts[rng.integers(0, len(pts), n // 4)] + 0.08 * (1 + rng.uniform(-1e-6, 1e-6, (n // 4, 1))) * u)
    c4 = rng.uniform(-5, 5, (n // 4, 3))
    cen = np.concatenate([c1, c1b, c1c, c2, c3.astype(np.float32), c4.astype(np.float32)]).astype(np.float32)
    m = len(cen) - len(cen) % 7
    cen = cen[:m].reshape(-1, 1, 7, 3)
    r = np.full(7, 0.03, np.float32)
    a, b = _both(capt_lib, torch_, t, cen, r)
    _equal(a, b)
    _check_oracle(orc, pts, cen, b[1], b[2], 0.08, n=len(cen.reshape(-1, 3)))


@pytest.mark.parametrize("kind", ["one", "two", "duplicates", "plane", "line", "uniform"])
def test_lists_on_degenerate_clouds(orc, capt_lib, torch_, kind):
    rng = np.random.default_rng(5)
    if kind == "one":
        pts = np.array([[0.3, 0.2, 0.1]], np.float32)
    elif kind == "two":
        pts = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]], np.float32)
    elif kind == "duplicates":
        pts = np.repeat(rng.uniform(0, 0.2, (20, 3)), 30, axis=0).astype(np.float32)
    elif kind == "plane":
        pts = rng.uniform(0, 0.5, (3000, 3)).astype(np.float32)
        pts[:, 2] = 0.25
    elif kind == "line":
        pts = np.zeros((2000, 3), np.float32)
        pts[:, 0] = rng.uniform(0, 1, 2000)
    else:
        pts = W.uniform_cloud(5000, 3)
    t = _tree(capt_lib, pts)
    capt_lib.capt_build_grid(t, 1 << 18)
    capt_lib.capt_build_near_lists(t)
    lo, hi = pts.min(0) - 0.1, pts.max(0) + 0.1
    cen = rng.uniform(lo, hi, (4096, 1, 3, 3)).astype(np.float32)
    cen[:512, 0, 0] = pts[rng.integers(0, len(pts), 512)]
    r = np.full(3, 0.02, np.float32)
    a, b = _both(capt_lib, torch_, t, cen, r)
    _equal(a, b)
    _check_oracle(orc, pts, cen, b[1], b[2], 0.08)


def test_coarse_grid_falls_back_to_the_paper_path(scene, capt_lib, torch_):
    """Cells far larger than the leaves meet too many leaves or points for the builder's
    buffers: they are marked, and their centres take the paper's path."""
    t = _tree(capt_lib, scene["pts"])
    capt_lib.capt_build_grid(t, 64)
    capt_lib.capt_build_near_lists(t)
    st = capt_lib.capt_stats(t)
    assert st["near_fallback_cells"] > 0
    q = W.random_trajectories(256, 16, 1004)
    cen = W.fk_centers(scene["arm"], q.reshape(-1, 7)).reshape(256, 16, 60, 3)
    a, b = _both(capt_lib, torch_, t, cen, scene["arm"].sphere_radius)
    _equal(a, b)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE, 8, 2, 0, 0, 0, 1)
    g = capt_lib.capt_count_clearance_work(t, _cuda(torch_, cen)).cpu().numpy()
    assert g[7] > 0 and g[5] + g[7] == g[1]


def test_list_state_rules(scene, capt_lib, torch_):
    pts = scene["pts"]
    t = _tree(capt_lib, pts)
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_build_near_lists(t)                     # no grid yet
    assert e.value.status == -8
    pruned = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(pruned, 0)
    capt_lib.capt_build_grid(pruned, 1 << 16)
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_build_near_lists(pruned)                # r_min > 0
    assert e.value.status == -8
    empty = capt_lib.capt_build(np.zeros((0, 3), np.float32), 0.0, 0.08)
    capt_lib.capt_upload(empty, 0)
    capt_lib.capt_build_grid(empty, 1 << 16)
    capt_lib.capt_build_near_lists(empty)                     # nothing to list, no error
    assert capt_lib.capt_stats(empty)["near_entries"] == 0
    capt_lib.capt_build_grid(t, 1 << 16)
    capt_lib.capt_build_near_lists(t)
    assert capt_lib.capt_stats(t)["near_entries"] > 0
    capt_lib.capt_build_grid(t, 1 << 17)                      # a new grid releases the lists
    assert capt_lib.capt_stats(t)["near_entries"] == 0
    capt_lib.capt_build_near_lists(t)
    b0 = capt_lib.capt_stats(t)["device_bytes"]
    capt_lib.capt_build_near_lists(t)                         # rebuilding replaces them
    assert capt_lib.capt_stats(t)["device_bytes"] == b0
    capt_lib.capt_upload(t, 0)                                # so does a new upload
    st = capt_lib.capt_stats(t)
    assert st["near_entries"] == 0 and st["grid_dims"] == [0, 0, 0]


def test_clearance_autotuner_keeps_the_results(scene, capt_lib, torch_):
    t = _tree(capt_lib, scene["pts"])
    capt_lib.capt_build_grid(t, 1 << 20)
    capt_lib.capt_build_near_lists(t)
    q = W.random_trajectories(512, 32, 1005)
    cen = W.fk_centers(scene["arm"], q.reshape(-1, 7)).reshape(512, 32, 60, 3)
    r = scene["arm"].sphere_radius
    a, _ = _both(capt_lib, torch_, t, cen, r)
    cfg, ms = capt_lib.capt_autotune_clearance(t, _cuda(torch_, cen), _cuda(torch_, r), 0.01)
    assert ms > 0 and cfg["warps_per_block"] in (4, 8, 16) and cfg["grid"] in (0, 1)
    assert capt_lib.capt_get_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE) == cfg
    cost, d, am = capt_lib.capt_clearance_fwd(t, _cuda(torch_, cen), _cuda(torch_, r), 0.01)
    _equal(a, [x.cpu().numpy() for x in (cost, d, am)])


@pytest.mark.slow
def test_lists_full_size(scene, orc, capt_lib, torch_):
    """The bench's clearance workload (16,384 trajectories x 32 waypoints x 60 spheres)
    with the bench's grid: the two paths agree on all 31.5M spheres."""
    t = _tree(capt_lib, scene["pts"])
    capt_lib.capt_build_grid(t, 1 << 24)
    capt_lib.capt_build_near_lists(t)
    q = W.random_trajectories(16384, 32, 1003)
    cen = W.fk_centers(scene["arm"], q.reshape(-1, 7)).reshape(16384, 32, 60, 3)
    a, b = _both(capt_lib, torch_, t, cen, scene["arm"].sphere_radius)
    _equal(a, b)
    _check_oracle(orc, scene["pts"], cen, b[1], b[2], 0.08, n=30000, seed=4)


def _cost_fixed_order(d, r, margin):
    """The cost's fixed FP32 order, in numpy: per waypoint, lane l forms
    (0 + h(l)^2) + h(l + 32)^2 (absent spheres add nothing), the 32 lane terms meet in a
    butterfly (xor 16, 8, 4, 2, 1), and the waypoints are added in order."""
    f = np.float32
    T, Wn, S = d.shape
    rm = (r.astype(np.float32) + f(margin)).astype(np.float32)
    h = np.maximum(f(0), (rm[None, None, :] - d).astype(np.float32))
    sq = (h * h).astype(np.float32)
    lanes = np.zeros((T, Wn, 32), np.float32)
    lanes[..., :min(S, 32)] = (f(0) + sq[..., :min(S, 32)]).astype(np.float32)
    if S > 32:
        lanes[..., :S - 32] = (lanes[..., :S - 32] + sq[..., 32:]).astype(np.float32)
    for o in (16, 8, 4, 2, 1):
        lanes = (lanes + lanes[..., np.arange(32) ^ o]).astype(np.float32)
    acc = np.zeros(T, np.float32)
    for w in range(Wn):
        acc = (acc + lanes[:, w, 0]).astype(np.float32)
    return acc


@pytest.mark.parametrize("Wn,S", [(32, 60), (7, 33), (1024, 5), (1100, 5)])
def test_cost_is_the_fixed_order_sum(scene, capt_lib, torch_, Wn, S):
    """The trajectory cost is the fixed-order FP32 sum of its hinge terms, bit for bit,
    whether the distance kernel sums it (W <= 1024) or the separate cost kernel does,
    on both paths."""
    t = _tree(capt_lib, scene["pts"])
    capt_lib.capt_build_grid(t, 1 << 20)
    capt_lib.capt_build_near_lists(t)
    rng = np.random.default_rng(Wn + S)
    T = max(3, 4096 // Wn)
    pts = scene["pts"]
    cen = (pts[rng.integers(0, len(pts), (T, Wn, S))] + rng.normal(0, 0.04, (T, Wn, S, 3))).astype(np.float32)
    r = rng.uniform(0.02, 0.08, S).astype(np.float32)
    a, b = _both(capt_lib, torch_, t, cen, r, margin=0.01)
    _equal(a, b)
    want = _cost_fixed_order(b[1].reshape(T, Wn, S), r, 0.01)
    assert np.array_equal(b[0].view(np.uint32), want.view(np.uint32))
    assert (want > 0).mean() > 0.5


def test_lists_on_a_device_built_tree(scene, capt_lib, torch_):
    """The lists of a tree built on the device (capt_build_device) are those of the host
    build of the same points, so the two trees' clearance outputs are equal, and equal
    to the leaf-set path."""
    pts = scene["pts"]
    th = _tree(capt_lib, pts)
    td = capt_lib.capt_build_device(_cuda(torch_, pts), 0.0, 0.08)
    for t in (th, td):
        capt_lib.capt_build_grid(t, 1 << 20)
        capt_lib.capt_build_near_lists(t)
    sh, sd = capt_lib.capt_stats(th), capt_lib.capt_stats(td)
    assert sh["near_entries"] == sd["near_entries"] and sh["near_fallback_cells"] == sd["near_fallback_cells"]
    q = W.random_trajectories(256, 32, 1006)
    cen = W.fk_centers(scene["arm"], q.reshape(-1, 7)).reshape(256, 32, 60, 3)
    r = scene["arm"].sphere_radius
    a, b = _both(capt_lib, torch_, td, cen, r)
    _equal(a, b)
    _, bh = _both(capt_lib, torch_, th, cen, r)
    _equal(b, bh)
