"""Parity of the GPU space-filling-curve filter (sfc_filter_device) with the oracle's
plain Alg. 2: the same kept indices in the same order, bit for bit, on the tabletop
and room clouds, uniform clouds of ragged sizes, and the degenerate cases of the
method (coincident points, points on a line, a flat axis, duplicates, signed zeros)."""
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


def _gpu_filter(capt_lib, torch_, pts, r):
    d = torch_.from_numpy(np.ascontiguousarray(pts, np.float32).reshape(-1, 3)).cuda()
    return capt_lib.sfc_filter_device(d, r).cpu().numpy().astype(np.uint32)


def _same(orc, capt_lib, torch_, pts, r):
    ref = orc.sfc_filter(pts, r)
    got = _gpu_filter(capt_lib, torch_, pts, r)
    assert np.array_equal(got, ref), (len(got), len(ref))
    return ref


def test_filter_tabletop(orc, capt_lib, torch_):
    raw, _, _ = W.tabletop_scene(1001)
    ref = _same(orc, capt_lib, torch_, raw, 0.01)
    assert len(ref) == 15080
    assert np.array_equal(ref, capt_lib.sfc_filter(raw, 0.01))


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 4095, 4096, 4097, 20000])
@pytest.mark.parametrize("r", [0.0, 0.004, 0.05])
def test_filter_uniform(orc, capt_lib, torch_, n, r):
    _same(orc, capt_lib, torch_, W.uniform_cloud(n, 50 + n), r)


def test_filter_degenerate(orc, capt_lib, torch_):
    same = np.tile(np.float32([[0.3, -1.0, 2.5]]), (700, 1))
    assert list(_same(orc, capt_lib, torch_, same, 0.01)) == [0]
    assert list(_same(orc, capt_lib, torch_, same, 0.0)) == [0]   # d^2 = 0 is not > 0
    rng = np.random.default_rng(5)
    line = np.zeros((3000, 3), np.float32)
    line[:, 0] = rng.uniform(-1, 1, 3000).astype(np.float32)
    _same(orc, capt_lib, torch_, line, 0.003)                       # two flat axes
    flat = W.uniform_cloud(5000, 6)
    flat[:, 2] = 0.25
    _same(orc, capt_lib, torch_, flat, 0.01)
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3), -1).reshape(-1, 3).astype(np.float32) * 0.01
    dup = np.concatenate([g, g[::3], g[5:40]])
    for r in (0.0, 0.01, 0.0100001, 0.015):                         # spacing equal to the grid step
        _same(orc, capt_lib, torch_, dup, r)
    z = rng.uniform(-0.01, 0.01, (900, 3)).astype(np.float32)
    z[::4, 0] = 0.0
    z[1::4, 0] = -0.0
    z[::7, 1] = -0.0
    _same(orc, capt_lib, torch_, z, 0.002)


def test_filter_room(orc, capt_lib, torch_):
    p = W.WORKLOADS["room200k"].params
    pts = W.room_cloud(W.WORKLOADS["room200k"].seed, p["n_points"], p["sigma"])
    _same(orc, capt_lib, torch_, pts, 0.02)


@pytest.mark.parametrize("rf", [0.01, 0.02])
def test_filter_depth_frame(orc, capt_lib, torch_, rf):
    """A 640 x 480 depth frame (307,200 points): device, host and oracle agree."""
    frame = W.depth_frame()
    ref = _same(orc, capt_lib, torch_, frame, rf)
    assert np.array_equal(ref, capt_lib.sfc_filter(frame, rf))


def test_filter_errors_and_empty(capt_lib, torch_):
    assert _gpu_filter(capt_lib, torch_, np.zeros((0, 3), np.float32), 0.01).size == 0
    bad = W.uniform_cloud(100, 1)
    bad[40, 2] = np.inf
    with pytest.raises(capt_lib.CaptError) as e:
        _gpu_filter(capt_lib, torch_, bad, 0.01)
    assert e.value.status == -3
    bad[40, 2] = np.nan
    with pytest.raises(capt_lib.CaptError) as e:
        _gpu_filter(capt_lib, torch_, bad, 0.01)
    assert e.value.status == -3
    for r in (-0.1, float("nan")):
        with pytest.raises(capt_lib.CaptError) as e:
            _gpu_filter(capt_lib, torch_, W.uniform_cloud(10, 2), r)
        assert e.value.status == -2


def test_filter_then_device_build(orc, capt_lib, torch_):
    """Filter and build entirely on the device: the tree equals the oracle's Alg. 1 on
    the oracle's Alg. 2 output."""
    raw, _, _ = W.tabletop_scene(1001)
    d = torch_.from_numpy(raw).cuda()
    kept = capt_lib.sfc_filter_device(d, 0.01)
    pts_d = d[kept.long()].contiguous()
    tree = capt_lib.capt_build_device(pts_d, 0.02, 0.08)
    ref = orc.PlainCAPT(raw[orc.sfc_filter(raw, 0.01)], 0.02, 0.08).export()
    ex = capt_lib.capt_export(tree)
    assert np.array_equal(ex["T"].view(np.uint32), ref["T"].view(np.uint32))
    assert np.array_equal(ex["set_idx"], ref["set_idx"])


@pytest.mark.parametrize("rf", [0.015, 0.02])
def test_frame_to_tree_in_one_call(orc, capt_lib, torch_, rf):
    """capt_build_frame_device on a 307,200-point depth frame: the kept indices are the
    oracle's Alg. 2 output and the tree is the oracle's Alg. 1 on those points."""
    frame = W.depth_frame()
    tree, kept = capt_lib.capt_build_frame_device(torch_.from_numpy(frame).cuda(), rf, 0.015, 0.08)
    ref_kept = orc.sfc_filter(frame, rf)
    assert np.array_equal(kept.cpu().numpy().astype(np.uint32), ref_kept)
    ref = orc.PlainCAPT(frame[ref_kept], 0.015, 0.08).export()
    ex = capt_lib.capt_export(tree)
    assert np.array_equal(ex["T"].view(np.uint32), ref["T"].view(np.uint32))
    assert np.array_equal(ex["set_begin"].astype(np.int64), ref["set_begin"])
    assert np.array_equal(ex["set_idx"], ref["set_idx"])
    # and it answers queries at once
    c, r = W.cube_queries(20000, 9)
    c = (c * np.float32([1.2, 0.8, 0.3]) + np.float32([0.0, -0.4, 0.0])).astype(np.float32)
    r = np.clip(r, 0.015, 0.08).astype(np.float32)
    f = capt_lib.capt_query_spheres(tree, torch_.from_numpy(c).cuda(), torch_.from_numpy(r).cuda()).cpu().numpy()
    assert np.array_equal(f, orc.brute_flags(frame[ref_kept], c, r))


def test_frame_to_tree_empty(capt_lib, torch_):
    tree, kept = capt_lib.capt_build_frame_device(torch_.empty((0, 3), dtype=torch_.float32, device="cuda"),
                                                  0.01, 0.015, 0.08)
    assert kept.numel() == 0 and capt_lib.capt_stats(tree)["n_points"] == 0
