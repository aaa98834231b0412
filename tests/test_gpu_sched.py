"""Dynamic tile scheduling of the query kernels: the warps take tiles from a work
counter of the tree's pool, zeroed before each launch after the last launch that used
the same counter has finished; a launch inside a stream capture keeps the static
schedule.  These tests run queries on several streams at once, more launches than the
pool has counters, and a captured CUDA graph, and compare every flag with the oracle."""
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


@pytest.fixture(scope="module")
def scene(orc, capt_lib, torch_):
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[orc.sfc_filter(raw, 0.01)]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    cen = W.fk_centers(arm, W.random_configs(6 * 4096, 77))
    ref = orc.brute_config_flags(pts, cen, arm.sphere_radius)
    return dict(pts=pts, arm=arm, tree=tree, cen=cen, ref=ref,
                dcen=torch_.from_numpy(cen).cuda(), dr=torch_.from_numpy(arm.sphere_radius.copy()).cuda())


def test_concurrent_streams_share_a_tree(scene, capt_lib, torch_):
    t, dcen, dr = scene["tree"], scene["dcen"], scene["dr"]
    streams = [torch_.cuda.Stream() for _ in range(3)]
    outs = []
    for k in range(6):
        s = streams[k % 3]
        with torch_.cuda.stream(s):
            outs.append(capt_lib.capt_query_configs(t, dcen[k * 4096:(k + 1) * 4096], dr))
    torch_.cuda.synchronize()
    got = np.concatenate([o.cpu().numpy() for o in outs])
    assert np.array_equal(got, scene["ref"])
    assert capt_lib.capt_device_status(t) == 0


def test_more_launches_than_counters(scene, orc, capt_lib, torch_):
    """200 launches over 4 streams (the pool has 64 counters, so each is reused)."""
    t, dcen, dr = scene["tree"], scene["dcen"], scene["dr"]
    streams = [torch_.cuda.Stream() for _ in range(4)]
    n = 200
    flags = torch_.empty((n, 512), dtype=torch_.uint8, device="cuda")
    for k in range(n):
        o = (k * 613) % (len(scene["ref"]) - 512)
        with torch_.cuda.stream(streams[k % 4]):
            capt_lib.capt_query_configs(t, dcen[o:o + 512], dr, flags[k])
    torch_.cuda.synchronize()
    f = flags.cpu().numpy()
    for k in range(n):
        o = (k * 613) % (len(scene["ref"]) - 512)
        assert np.array_equal(f[k], scene["ref"][o:o + 512]), k
    # spheres too
    c = scene["cen"].reshape(-1, 3)[:50000]
    r = np.tile(scene["arm"].sphere_radius, len(c) // 60 + 1)[:len(c)].astype(np.float32)
    dc, drs = torch_.from_numpy(c).cuda(), torch_.from_numpy(r).cuda()
    ref = orc.brute_flags(scene["pts"], c, r)
    outs = []
    for k in range(80):
        with torch_.cuda.stream(streams[k % 4]):
            outs.append(capt_lib.capt_query_spheres(t, dc, drs))
    torch_.cuda.synchronize()
    for o in outs:
        assert np.array_equal(o.cpu().numpy(), ref)


def test_captured_graph_replays_exactly(scene, capt_lib, torch_):
    """A query captured into a CUDA graph (static schedule) replays with exact flags."""
    t, dcen, dr = scene["tree"], scene["dcen"], scene["dr"]
    flags = torch_.empty(len(scene["ref"]), dtype=torch_.uint8, device="cuda")
    s = torch_.cuda.Stream()
    with torch_.cuda.stream(s):
        capt_lib.capt_query_configs(t, dcen, dr, flags)      # first launch outside the capture
    torch_.cuda.synchronize()
    g = torch_.cuda.CUDAGraph()
    with torch_.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        capt_lib.capt_query_configs(t, dcen, dr, flags)
    flags.zero_()
    for _ in range(3):
        g.replay()
    torch_.cuda.synchronize()
    assert np.array_equal(flags.cpu().numpy(), scene["ref"])


def test_joint_configs_many_streams(scene, orc, capt_lib, torch_):
    arm, t = scene["arm"], scene["tree"]
    q = W.random_configs(4096, 4243)
    ref = orc.brute_config_flags(scene["pts"], orc.fk32(arm, q), arm.sphere_radius)
    dq = torch_.from_numpy(q).cuda()
    streams = [torch_.cuda.Stream() for _ in range(3)]
    outs = []
    for k in range(90):
        with torch_.cuda.stream(streams[k % 3]):
            outs.append(capt_lib.capt_query_joint_configs(t, arm, dq))
    torch_.cuda.synchronize()
    for o in outs:
        assert np.array_equal(o.cpu().numpy(), ref)
