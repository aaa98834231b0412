"""Parity of the GPU builder (capt_build_device) with the oracle's plain Alg. 1.

The device builder finds each leaf's set directly as the points its closed cell
affords, instead of carrying z down the recursion; the tree must still be the
oracle's bit for bit: split values, set offsets, set members in ascending index,
FP32 boxes and the prune decisions.  Queries on the device-built tree must then give
the brute-force flags and the same work counts as the oracle's sequential Alg. 3."""
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


def _same_tree(capt_lib, tree, ref):
    st = capt_lib.capt_stats(tree)
    ex = capt_lib.capt_export(tree)
    assert st["build_threads"] == 0 and st["device"] == 0
    assert np.array_equal(ex["T"].view(np.uint32), ref["T"].view(np.uint32))
    assert np.array_equal(ex["set_begin"].astype(np.int64), ref["set_begin"])
    assert np.array_equal(ex["set_idx"], ref["set_idx"])
    assert np.array_equal(ex["aabb"].view(np.uint32), ref["aabb"].view(np.uint32))
    assert st["pruned_leaves"] == int(ref["pruned"].sum())
    return st


def _build(capt_lib, torch_, pts, r_min, r_max):
    d = torch_.from_numpy(np.ascontiguousarray(pts, np.float32).reshape(-1, 3)).cuda()
    return capt_lib.capt_build_device(d, r_min, r_max)


def _signed_zero_cloud(seed):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.1, 0.1, (97, 3)).astype(np.float32)
    z[::5, 0] = 0.0
    z[1::5, 0] = -0.0
    z[2::7, 2] = -0.0
    return z


def _grid_with_duplicates():
    g = np.stack(np.meshgrid(*[np.arange(5)] * 3), -1).reshape(-1, 3).astype(np.float32) * 0.1
    return np.concatenate([g, g[:40], g[7:9]])


CASES = {
    "uniform300": (lambda: W.uniform_cloud(300, 7), 0.02, 0.2),
    "uniform2k": (lambda: W.uniform_cloud(2000, 1000), 0.01, 0.08),
    "uniform1025": (lambda: W.uniform_cloud(1025, 8), 0.01, 0.08),     # N = 2048, 1023 pads
    "dense_pruned": (lambda: W.uniform_cloud(4000, 9), 0.3, 0.35),
    "grid_duplicates": (_grid_with_duplicates, 0.05, 0.15),
    "signed_zeros": (lambda: _signed_zero_cloud(3), 0.0, 0.05),
    "r_max_zero": (lambda: W.uniform_cloud(200, 11), 0.0, 0.0),
    "one": (lambda: W.uniform_cloud(1, 12), 0.01, 0.1),
    "two": (lambda: W.uniform_cloud(2, 13), 0.01, 0.1),
    "three": (lambda: W.uniform_cloud(3, 14), 0.01, 0.1),
    "all_same_point": (lambda: np.tile(np.float32([[0.5, -0.25, 2.0]]), (70, 1)), 0.01, 0.1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_build_equals_oracle(orc, capt_lib, torch_, name):
    make, r_min, r_max = CASES[name]
    pts = make()
    ref = orc.PlainCAPT(pts, r_min, r_max).export()
    tree = _build(capt_lib, torch_, pts, r_min, r_max)
    _same_tree(capt_lib, tree, ref)


def test_device_build_empty_cloud(capt_lib, torch_):
    tree = _build(capt_lib, torch_, np.zeros((0, 3), np.float32), 0.01, 0.1)
    st = capt_lib.capt_stats(tree)
    assert st["n_points"] == 0 and st["n_leaves"] == 1 and st["total_afforded"] == 0
    c = torch_.rand(100, 3, device="cuda")
    r = torch_.full((100,), 0.05, device="cuda")
    assert int(capt_lib.capt_query_spheres(tree, c, r).sum()) == 0


def test_device_build_rejects_bad_input(capt_lib, torch_):
    bad = W.uniform_cloud(50, 1)
    bad[17, 1] = np.nan
    with pytest.raises(capt_lib.CaptError) as e:
        _build(capt_lib, torch_, bad, 0.01, 0.1)
    assert e.value.status == -3
    with pytest.raises(capt_lib.CaptError) as e:
        _build(capt_lib, torch_, W.uniform_cloud(50, 1), 0.2, 0.1)
    assert e.value.status == -2
    bad[17, 1] = np.inf
    with pytest.raises(capt_lib.CaptError) as e:
        _build(capt_lib, torch_, bad, 0.01, 0.1)
    assert e.value.status == -3


def test_device_built_tree_answers_queries(orc, capt_lib, torch_):
    """Flags equal the brute force, and the work counts equal the oracle's Alg. 3 over
    its own tree (so the device layout is the one the host upload makes)."""
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[orc.sfc_filter(raw, 0.01)]
    tree = _build(capt_lib, torch_, pts, 0.02, 0.08)
    cen = W.fk_centers(arm, W.random_configs(3000, 77))
    dc = torch_.from_numpy(cen).cuda()
    dr = torch_.from_numpy(np.ascontiguousarray(arm.sphere_radius, np.float32)).cuda()
    flags = capt_lib.capt_query_configs(tree, dc, dr).cpu().numpy()
    assert np.array_equal(flags, orc.brute_config_flags(pts, cen, arm.sphere_radius))
    g = capt_lib.capt_count_config_work(tree, dc, dr).cpu().numpy()
    _, counts = orc.PlainCAPT(pts, 0.02, 0.08).query_configs(cen, arm.sphere_radius)
    assert g[0] == counts[0] and g[2] == counts[1] and g[3] == counts[2]
    sph = torch_.from_numpy(cen.reshape(-1, 3)).cuda()
    rr = dr.repeat(cen.shape[0])
    f = capt_lib.capt_query_spheres(tree, sph, rr).cpu().numpy()
    ref = orc.brute_flags(pts, cen.reshape(-1, 3), np.tile(arm.sphere_radius, cen.shape[0]))
    assert np.array_equal(f, ref)
    assert capt_lib.capt_device_status(tree) == 0


def test_device_built_tree_reuploads(orc, capt_lib, torch_):
    """capt_upload of a device-built tree goes through its host form and answers the
    same."""
    pts = W.uniform_cloud(2000, 1000)
    c, r = W.cube_queries(20000, 1000)
    tree = _build(capt_lib, torch_, pts, 0.01, 0.08)
    dc, dr = torch_.from_numpy(c).cuda(), torch_.from_numpy(r).cuda()
    f1 = capt_lib.capt_query_spheres(tree, dc, dr).cpu().numpy()
    capt_lib.capt_upload(tree, 0)
    f2 = capt_lib.capt_query_spheres(tree, dc, dr).cpu().numpy()
    ref = orc.brute_flags(pts, c, r)
    assert np.array_equal(f1, ref) and np.array_equal(f2, ref)


def test_device_build_tabletop_full(orc, capt_lib, torch_):
    raw, _, _ = W.tabletop_scene(1001)
    pts = raw[orc.sfc_filter(raw, 0.01)]
    ref = orc.PlainCAPT(pts, 0.02, 0.08).export()
    st = _same_tree(capt_lib, _build(capt_lib, torch_, pts, 0.02, 0.08), ref)
    assert st["n_points"] == 15080 and st["total_afforded"] == ref["set_begin"][-1]
    ref0 = orc.PlainCAPT(pts, 0.0, 0.08).export()   # the clearance tree (no prune)
    _same_tree(capt_lib, _build(capt_lib, torch_, pts, 0.0, 0.08), ref0)


@pytest.mark.slow
def test_device_build_room_full(orc, capt_lib, torch_):
    p = W.WORKLOADS["room200k"].params
    pts = W.room_cloud(W.WORKLOADS["room200k"].seed, p["n_points"], p["sigma"])
    ref = orc.PlainCAPT(pts, p["r_min"], p["r_max"]).export()
    _same_tree(capt_lib, _build(capt_lib, torch_, pts, p["r_min"], p["r_max"]), ref)
