"""Device-side failure reporting, exercised without faulting or hanging the GPU.

1. Bounded waits.  Every wait on a bulk copy into shared memory gives up after a poll
   limit, latches CAPT_E_TIMEOUT in the tree's status word and falls back to global
   memory.  A test build of the library (its own build directory and .so) sets the
   first-wait limit to 0, so every such wait gives up at once while the copies still
   land and are drained; the queries must still give the oracle's flags, and
   capt_device_status must report the timeout.  The variant runs in a child process
   (the library is loaded once per process).
2. Oversized edge batches.  The persistent edge validator counts work items in 32-bit
   words; a batch of more than 2^31 items is refused on the device (every edge reported
   not valid, CAPT_E_BOUNDS latched) instead of wrapping the counter.  The refused
   batch does no work, so the huge step counts are never walked."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
import paper_2406_02807_gb300 as capt
import workloads as W

out = {}
raw, _, arm = W.tabletop_scene(1001)
raw = raw[:8000]
pts = raw[oracle.sfc_filter(raw, 0.01)]
tree = capt.capt_build(pts, 0.02, 0.08)
capt.capt_upload(tree, 0)
dev = torch.device("cuda:0")
# sphere queries: per-warp input copies (always used) and, with staging 1, the split array
c, r = W.cube_queries(20000, 1005)
c = c * np.array([1.3, 1.0, 0.4], np.float32) + np.array([-0.05, -0.5, -0.05], np.float32)
r = np.clip(r, 0.02, 0.08).astype(np.float32)
ref = oracle.brute_flags(pts, c, r)
dc, dr = torch.from_numpy(c).to(dev), torch.from_numpy(r).to(dev)
res = []
for staging in (0, 1):
    for spl in (1, 4):
        capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_SPHERES, 8, spl, staging, capt.CAPT_SCAN_CHUNKED)
        f = capt.capt_query_spheres(tree, dc, dr)
        torch.cuda.synchronize()
        res.append(dict(kind="spheres", staging=staging, spl=spl, equal=bool(np.array_equal(f.cpu().numpy(), ref)),
                        status=capt.capt_device_status(tree)))
# configuration queries with the split array staged
cen = W.fk_centers(arm, W.random_configs(4096, 1006))
rr = arm.sphere_radius
refc = oracle.brute_config_flags(pts, cen, rr)
dcen, drr = torch.from_numpy(cen).to(dev), torch.from_numpy(rr).to(dev)
for spl in (4, 16):
    capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_CONFIGS, 8, spl, 1, capt.CAPT_SCAN_CHUNKED)
    f = capt.capt_query_configs(tree, dcen, drr)
    torch.cuda.synchronize()
    res.append(dict(kind="configs", staging=1, spl=spl, equal=bool(np.array_equal(f.cpu().numpy(), refc)),
                    status=capt.capt_device_status(tree)))
out["runs"] = res
out["collide_fraction"] = float(ref.mean())
print("RESULT " + json.dumps(out))
"""


def test_stage_wait_timeout_is_reported_and_flags_stay_exact(capt_lib, orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02807_gb300 import _build
    lib = _build.build(variant="stage_timeout")
    env = dict(os.environ, CAPT_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT), 1)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    assert 0.0 < out["collide_fraction"] < 1.0
    for run in out["runs"]:
        assert run["equal"], run
        # every launch met a wait that gave up: the status word reports it, once read
        assert run["status"] == -6, run   # CAPT_E_TIMEOUT


def test_edge_batch_over_the_item_limit_is_refused_on_the_device(capt_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[capt_lib.sfc_filter(raw, 0.01)]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    E = 4096
    qa, qb, ns = W.random_edges(E, 1007, nmax=60)
    dqa, dqb = torch.from_numpy(qa).cuda(), torch.from_numpy(qb).cuda()
    ok = capt_lib.capt_validate_edges(tree, arm, dqa, dqb, torch.from_numpy(ns).cuda())
    torch.cuda.synchronize()
    ok = ok.cpu().numpy()
    assert capt_lib.capt_device_status(tree) == 0
    # 2^31 - 1 configurations per edge is at least 2^21 work items (items hold at most
    # 1024 configurations): 4096 edges are at least 2^33 items, beyond the 2^31 the
    # 32-bit counter takes, whatever the launch configuration
    cfg = capt_lib.capt_get_launch_cfg(tree, capt_lib.CAPT_KERNEL_EDGES)
    assert cfg["chunk"] <= 1024
    assert E * -(-(2**31 - 1) // 1024) > 2**31
    huge = torch.full((E,), 2**31 - 1, dtype=torch.int32, device="cuda")
    for kw in (dict(), dict(static=True)):
        if kw:
            v = capt_lib.capt_validate_edges_static(tree, arm, dqa, dqb, huge)
        else:
            v = capt_lib.capt_validate_edges(tree, arm, dqa, dqb, huge)
        torch.cuda.synchronize()
        assert not v.cpu().numpy().any(), "a refused batch reports every edge as not valid"
        assert capt_lib.capt_device_status(tree) == -7
        assert capt_lib.capt_device_status(tree) == 0   # read and cleared
    # the tree is still usable, and the next batch is exact again
    again = capt_lib.capt_validate_edges(tree, arm, dqa, dqb, torch.from_numpy(ns).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(again.cpu().numpy(), ok)
    assert capt_lib.capt_device_status(tree) == 0
