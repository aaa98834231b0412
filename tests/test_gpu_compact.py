"""Parity of the compact (de-duplicated) affordance sets with the oracle.

capt_compact replaces every leaf's copied set by the list of 32-point chunks of the
Z-ordered cloud that hold its points; the chunks hold a superset of the set inside the
cloud, so every flag must still equal the FP32 brute force (Lemma 1).  These tests
compare the CUDA path in scan mode CAPT_SCAN_COMPACT with the oracle bit for bit, on
every launch configuration, ragged sizes, the degenerate clouds, device-built trees and
the 200,000-point room, and check the state rules of dropping the replicated sets."""
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
def uniform2k(orc, capt_lib, torch_):
    p = W.WORKLOADS["uniform2k"].params
    pts = W.uniform_cloud(p["n_points"], 1000)
    c, r = W.cube_queries(p["n_spheres"], 1000)
    tree = capt_lib.capt_build(pts, p["r_min"], p["r_max"])
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_compact(tree)
    return dict(pts=pts, c=c, r=r, tree=tree, ref=orc.brute_flags(pts, c, r), dc=_cuda(torch_, c),
                dr=_cuda(torch_, r))


@pytest.fixture(scope="module")
def tabletop(orc, capt_lib, torch_):
    raw, _, arm = W.tabletop_scene(1001)
    kept = orc.sfc_filter(raw, 0.01)
    assert np.array_equal(kept, capt_lib.sfc_filter(raw, 0.01))
    pts = raw[kept]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_compact(tree)
    cen = W.fk_centers(arm, W.random_configs(3001, 1001, first=777))   # odd count: ragged last tile
    ref, _ = orc.PlainCAPT(pts, 0.02, 0.08).query_configs(cen, arm.sphere_radius)
    return dict(pts=pts, arm=arm, tree=tree, cen=cen, ref=ref, dcen=_cuda(torch_, cen),
                dr=_cuda(torch_, arm.sphere_radius))


def test_compact_stats(uniform2k, tabletop, capt_lib):
    for w in (uniform2k, tabletop):
        s = capt_lib.capt_stats(w["tree"])
        n = len(w["pts"])
        assert s["compact_chunks"] == (n + 31) // 32
        # every non-empty set lists at least one chunk and at most one per point
        assert s["n_leaves"] - s["empty_leaves"] <= s["compact_entries"] <= s["total_afforded"]
        assert s["full_dropped"] == 0 and s["compact_bytes"] > 0


@pytest.mark.parametrize("warps,spl,stage", [(w, s, st) for w in (4, 8, 16) for s in (1, 2, 4, 8) for st in (0, 1)])
def test_spheres_compact_every_launch_cfg(uniform2k, capt_lib, torch_, warps, spl, stage):
    t = uniform2k["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, warps, spl, stage, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_spheres(t, uniform2k["dc"], uniform2k["dr"])
    assert np.array_equal(f.cpu().numpy(), uniform2k["ref"])
    assert capt_lib.capt_device_status(t) == 0


@pytest.mark.parametrize("m", [1, 31, 33, 65, 1000, 4097])
def test_spheres_compact_ragged(uniform2k, capt_lib, torch_, m):
    t = uniform2k["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 0, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_spheres(t, uniform2k["dc"][:m].contiguous(), uniform2k["dr"][:m].contiguous())
    assert np.array_equal(f.cpu().numpy(), uniform2k["ref"][:m])


def test_spheres_compact_on_points_and_planes(uniform2k, orc, capt_lib, torch_):
    """Spheres centred on cloud points, on split planes and touching points at exactly
    r: the boundary cases of the FP32 predicate."""
    pts, t = uniform2k["pts"], uniform2k["tree"]
    rng = np.random.default_rng(77)
    i = rng.integers(0, len(pts), 3000)
    c = np.concatenate([pts[i[:1000]], pts[i[1000:2000]] + np.float32([0.03, 0, 0]),
                        pts[i[2000:]] * np.float32([1, 1, 0]) + np.float32([0, 0, 0.5])]).astype(np.float32)
    r = np.concatenate([np.full(1000, 0.01), np.full(1000, 0.03), rng.uniform(0.01, 0.08, 1000)]).astype(np.float32)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 0, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_spheres(t, _cuda(torch_, c), _cuda(torch_, r))
    assert np.array_equal(f.cpu().numpy(), orc.brute_flags(pts, c, r))


@pytest.mark.parametrize("warps,spl,stage", [(w, s, st) for w in (4, 8, 16) for s in (2, 4, 8, 16) for st in (0, 1)])
def test_configs_compact_every_launch_cfg(tabletop, capt_lib, torch_, warps, spl, stage):
    t = tabletop["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, warps, spl, stage, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_configs(t, tabletop["dcen"], tabletop["dr"])
    assert np.array_equal(f.cpu().numpy(), tabletop["ref"])
    assert capt_lib.capt_device_status(t) == 0


def test_configs_compact_against_brute_force(tabletop, orc, capt_lib, torch_):
    cen = W.fk_centers(tabletop["arm"], W.random_configs(5000, 9))
    r = tabletop["arm"].sphere_radius
    t = tabletop["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_configs(t, _cuda(torch_, cen), _cuda(torch_, r))
    ref = orc.brute_config_flags(tabletop["pts"], cen, r)
    assert np.array_equal(f.cpu().numpy(), ref)
    assert 0.05 < ref.mean() < 0.95


@pytest.mark.parametrize("n", [0, 1, 2, 5, 31, 32, 33])
def test_compact_degenerate_clouds(orc, capt_lib, torch_, n):
    pts = W.uniform_cloud(n, 300 + n) if n else np.zeros((0, 3), np.float32)
    if n >= 5:
        pts[1] = pts[0]                                        # a duplicate point
    c, r = W.cube_queries(3000, 31 + n)
    tree = capt_lib.capt_build(pts, 0.01, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_compact(tree, drop_full=True)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_SPHERES, 4, 1, 0, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_spheres(tree, _cuda(torch_, c), _cuda(torch_, r))
    assert np.array_equal(f.cpu().numpy(), orc.brute_flags(pts, c, r))


def test_compact_device_built_tree(tabletop, capt_lib, torch_):
    """capt_build_device + capt_compact (the cloud is read back from the device)."""
    tree = capt_lib.capt_build_device(_cuda(torch_, tabletop["pts"]), 0.02, 0.08)
    capt_lib.capt_compact(tree)
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, capt_lib.CAPT_SCAN_COMPACT)
    f = capt_lib.capt_query_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert np.array_equal(f.cpu().numpy(), tabletop["ref"])
    s = capt_lib.capt_stats(tree)
    assert s["compact_chunks"] == (len(tabletop["pts"]) + 31) // 32


def test_drop_full_state_rules(tabletop, capt_lib, torch_):
    pts, arm = tabletop["pts"], tabletop["arm"]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    with pytest.raises(capt_lib.CaptError) as e:                 # not uploaded
        capt_lib.capt_compact(tree)
    assert e.value.status == -8
    capt_lib.capt_upload(tree, 0)
    # the compact mode needs capt_compact first
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, capt_lib.CAPT_SCAN_COMPACT)
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_query_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert e.value.status == -8
    before = capt_lib.capt_stats(tree)["device_bytes"]
    # an edge plan holds the replicated sets: dropping them is refused while it lives
    qa, qb, ns = W.random_edges(16, 5)
    valid = torch_.empty(16, dtype=torch_.uint8, device="cuda")
    plan = capt_lib.capt_edge_plan_create(tree, arm, _cuda(torch_, qa), _cuda(torch_, qb), _cuda(torch_, ns), valid,
                                          cfg=dict(warps_per_block=4, spheres_per_lane=1, staging=0, chunk=32))
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_compact(tree, drop_full=True)
    assert e.value.status == -8
    capt_lib.capt_edge_plan_free(plan)
    capt_lib.capt_compact(tree, drop_full=True)
    s = capt_lib.capt_stats(tree)
    assert s["full_dropped"] == 1 and s["device_bytes"] < before
    f = capt_lib.capt_query_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert np.array_equal(f.cpu().numpy(), tabletop["ref"])
    # the other scan modes and the calls that need the replicated sets now refuse
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, capt_lib.CAPT_SCAN_CHUNKED)
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_query_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert e.value.status == -8
    for call in (lambda: capt_lib.capt_compact(tree),
                 lambda: capt_lib.capt_clearance_fwd(tree, tabletop["dcen"][:2].reshape(1, 2, -1, 3).contiguous(),
                                                     tabletop["dr"], 0.01),
                 lambda: capt_lib.capt_count_config_work(tree, tabletop["dcen"], tabletop["dr"])):
        with pytest.raises(capt_lib.CaptError) as e:
            call()
        assert e.value.status == -8
    # the autotuner only tries what is there
    best, _ = capt_lib.capt_autotune_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert best["chunk"] == capt_lib.CAPT_SCAN_COMPACT
    f = capt_lib.capt_query_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert np.array_equal(f.cpu().numpy(), tabletop["ref"])
    # a new upload brings the replicated sets back (and releases the compact form)
    capt_lib.capt_upload(tree, 0)
    s = capt_lib.capt_stats(tree)
    assert s["full_dropped"] == 0 and s["compact_chunks"] == 0 and s["device_bytes"] == before
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, capt_lib.CAPT_SCAN_CHUNKED)
    f = capt_lib.capt_query_configs(tree, tabletop["dcen"], tabletop["dr"])
    assert np.array_equal(f.cpu().numpy(), tabletop["ref"])


def test_edges_and_joints_on_compact_sets(tabletop, orc, capt_lib, torch_):
    """With the replicated sets dropped, edge validation (persistent, per-edge, graph
    plan, allocation-free) and joint-angle configurations scan the compact sets and
    give the oracle's answers."""
    pts, arm = tabletop["pts"], tabletop["arm"]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    capt_lib.capt_compact(tree, drop_full=True)
    qa, qb, ns = W.random_edges(256, 1002)
    ref = orc.edges(arm, qa, qb, ns, points=pts)
    assert 0.05 < ref.mean() < 0.95
    dqa, dqb, dns = _cuda(torch_, qa), _cuda(torch_, qb), _cuda(torch_, ns)
    for mode in (capt_lib.CAPT_EDGES_PERSISTENT, capt_lib.CAPT_EDGES_PER_EDGE):
        v = capt_lib.capt_validate_edges(tree, arm, dqa, dqb, dns, mode=mode)
        assert np.array_equal(v.cpu().numpy(), ref)
    v = capt_lib.capt_validate_edges_static(tree, arm, dqa, dqb, dns)
    assert np.array_equal(v.cpu().numpy(), ref)
    valid = torch_.empty(256, dtype=torch_.uint8, device="cuda")
    plan = capt_lib.capt_edge_plan_create(tree, arm, dqa, dqb, dns, valid)
    capt_lib.capt_edge_plan_launch(plan)
    assert np.array_equal(valid.cpu().numpy(), ref)
    capt_lib.capt_edge_plan_free(plan)
    q = W.random_configs(3000, 4242)
    fref = orc.brute_config_flags(pts, orc.fk32(arm, q), arm.sphere_radius)
    for stage in (0, 1):
        capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_JOINTS, 4, 1, stage)
        f = capt_lib.capt_query_joint_configs(tree, arm, _cuda(torch_, q.astype(np.float32)))
        assert np.array_equal(f.cpu().numpy(), fref)
    assert capt_lib.capt_device_status(tree) == 0


@pytest.mark.slow
def test_room_compact_full_size(orc, capt_lib, torch_):
    """200,000 unfiltered points, 4,194,304 spheres: the compact sets (replicated sets
    dropped) give the oracle's plain CAPT flags, and hold the room in a small fraction
    of the replicated layout's memory."""
    p = W.WORKLOADS["room200k"].params
    pts = W.room_cloud(1004)
    c, r = W.room_queries(p["n_spheres"], 1004)
    tree = capt_lib.capt_build(pts, p["r_min"], p["r_max"])
    capt_lib.capt_upload(tree, 0)
    full = capt_lib.capt_stats(tree)["device_bytes"]
    capt_lib.capt_compact(tree, drop_full=True)
    s = capt_lib.capt_stats(tree)
    assert s["device_bytes"] * 8 < full
    ref, _, _ = orc.PlainCAPT(pts, p["r_min"], p["r_max"]).query(c, r)
    dc, dr = _cuda(torch_, c), _cuda(torch_, r)
    for spl in (1, 2):
        capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_SPHERES, 8, spl, 0, capt_lib.CAPT_SCAN_COMPACT)
        assert np.array_equal(capt_lib.capt_query_spheres(tree, dc, dr).cpu().numpy(), ref)
