"""capt_validate_edges_static: edge validation for callers that cannot let the library
allocate device memory (a planner in a real-time control loop that must not enter the
CUDA allocator, or an application whose device memory another allocator owns).

It must give exactly the flags of the allocating entry point (capt_validate_edges,
persistent mode): edge flags are exact booleans, so the tolerance is equality.  Two
calls in a row check that the shared scratch array is re-initialised by every call.
This file is collected last so that a stop at its first failure has already run every
other test; it also passes alone in a fresh process (it builds what it needs)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_static_edges_match_allocating_entry_point(capt_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[capt_lib.sfc_filter(raw, 0.01)]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    qa, qb, ns = W.random_edges(2048, 1002)
    dqa, dqb, dns = (torch.from_numpy(a).cuda() for a in (qa, qb, ns))
    ref = capt_lib.capt_validate_edges(tree, arm, dqa, dqb, dns, mode=capt_lib.CAPT_EDGES_PERSISTENT)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert 0 < ref.sum() < len(ref)
    for _ in range(2):
        out = torch.full((len(ns),), 7, dtype=torch.uint8, device="cuda")
        capt_lib.capt_validate_edges_static(tree, arm, dqa, dqb, dns, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    # a different, smaller batch right after: nothing from the previous call leaks in
    sub = slice(100, 400)
    out = capt_lib.capt_validate_edges_static(tree, arm, dqa[sub].contiguous(), dqb[sub].contiguous(),
                                              dns[sub].contiguous())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref[sub])
    assert capt_lib.capt_device_status(tree) == 0


def test_static_edges_reject_batches_over_the_limit(capt_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pts = W.uniform_cloud(100, 5)
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    arm = W.arm_7dof()
    E = capt_lib.CAPT_STATIC_MAX_EDGES + 1
    q = torch.zeros((E, 7), dtype=torch.float32, device="cuda")
    ns = torch.ones(E, dtype=torch.int32, device="cuda")
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_validate_edges_static(tree, arm, q, q, ns)
    assert e.value.status == -1 and "65536" in str(e.value)


def test_static_edges_allocate_no_device_memory(capt_lib):
    """The point of the entry point: repeated calls leave the device's free memory and the
    tree's on-demand scratch exactly as they were.  The allocating entry point, called
    afterwards on the same tree, does allocate its scratch (the check can see it)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    raw, _, arm = W.tabletop_scene(1001)
    pts = raw[capt_lib.sfc_filter(raw, 0.01)]
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    qa, qb, ns = W.random_edges(1024, 1008)
    dqa, dqb, dns = (torch.from_numpy(a).cuda() for a in (qa, qb, ns))
    outs = [torch.empty(len(ns), dtype=torch.uint8, device="cuda") for _ in range(4)]
    # first call: the per-device set-up and the first launch of each kernel
    capt_lib.capt_validate_edges_static(tree, arm, dqa, dqb, dns, outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert capt_lib.capt_stats(tree)["scratch_bytes"] == 0
    for o in outs[1:]:
        capt_lib.capt_validate_edges_static(tree, arm, dqa, dqb, dns, o)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert capt_lib.capt_stats(tree)["scratch_bytes"] == 0
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ref = capt_lib.capt_validate_edges(tree, arm, dqa, dqb, dns)
    torch.cuda.synchronize()
    assert capt_lib.capt_stats(tree)["scratch_bytes"] > 0
    assert torch.equal(ref, outs[0])
