"""Host side of the product library against the oracle (no GPU): the optimised C++
builder must produce the oracle's plain Alg. 1 tree (same T, same sets, same boxes),
the C++ filter the oracle's plain Alg. 2 output, and the C ABI must export every
symbol include/capt.h declares and reject bad arguments without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sets(sb, si, N):
    return [si[int(sb[l]):int(sb[l + 1])] for l in range(N)]


def _compare_trees(orc, capt, pts, r_min, r_max, threads=0):
    ref = orc.PlainCAPT(pts, r_min, r_max)
    t = capt.capt_build_threads(pts, r_min, r_max, threads)
    st = capt.capt_stats(t)
    assert st["n_leaves"] == ref.N and st["depth"] == ref.L
    assert st["total_afforded"] == ref.total and st["max_set"] == ref.max_set
    assert st["pruned_leaves"] == ref.n_pruned
    a, b = capt.capt_export(t), ref.export()
    np.testing.assert_array_equal(a["T"], b["T"])
    np.testing.assert_array_equal(a["set_begin"].astype(np.int64), b["set_begin"])
    np.testing.assert_array_equal(a["set_idx"], b["set_idx"])
    np.testing.assert_array_equal(a["aabb"], b["aabb"])
    return t, st


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 17, 64, 100, 1000])
def test_builder_equals_plain_capt_uniform(orc, capt_lib, n):
    pts = W.uniform_cloud(n, 300 + n)
    _compare_trees(orc, capt_lib, pts, 0.01, 0.08)
    _compare_trees(orc, capt_lib, pts, 0.0, 0.2)


def test_builder_equals_plain_capt_grid_duplicates(orc, capt_lib):
    rng = np.random.default_rng(9)
    pts = (rng.integers(0, 5, (300, 3)) * 0.125).astype(np.float32)   # many ties and plane points
    _compare_trees(orc, capt_lib, pts, 0.02, 0.3)
    _compare_trees(orc, capt_lib, pts, 0.0, 0.125)


def test_builder_dense_prunes_like_oracle(orc, capt_lib):
    pts = W.uniform_cloud(1500, 77) * np.float32(0.08)
    _, st = _compare_trees(orc, capt_lib, pts, 0.02, 0.08)
    assert st["pruned_leaves"] > 0


@pytest.mark.parametrize("threads", [1, 2, 8])
def test_builder_threads_do_not_change_the_tree(orc, capt_lib, threads):
    pts, _ = W.tabletop_cloud(1001, n=5000)
    _compare_trees(orc, capt_lib, pts, 0.02, 0.08, threads)


def test_builder_rejects_bad_input(capt_lib):
    pts = W.uniform_cloud(10, 1)
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_build(pts, 0.1, 0.05)
    assert e.value.status == -2
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_build(bad, 0.0, 0.05)
    assert e.value.status == -3
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_build(pts, -0.1, 0.05)
    assert e.value.status == -2


@pytest.mark.parametrize("n,rf", [(0, 0.1), (1, 0.1), (6, 0.4), (3000, 0.01), (30000, 0.01), (20000, 0.0)])
def test_filter_equals_plain_alg2(orc, capt_lib, n, rf):
    if n == 6:
        x = np.array([0.0, 0.3, 0.5, 1.2, 1.25, 2.0], np.float32)
        pts = np.stack([x, np.zeros_like(x), np.zeros_like(x)], 1)
    else:
        pts, _ = W.tabletop_cloud(1001, n=max(n, 1))
        pts = pts[:n]
    if rf == 0.0:
        pts = np.concatenate([pts, pts[::7]])          # exact duplicates
    a = capt_lib.sfc_filter(pts, rf)
    b = orc.sfc_filter(pts, rf)
    np.testing.assert_array_equal(a, b)


def test_filter_rejects_nonfinite(capt_lib):
    pts = W.uniform_cloud(10, 2)
    pts[4, 0] = np.inf
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.sfc_filter(pts, 0.1)
    assert e.value.status == -3


def test_header_symbols_are_exported(capt_lib):
    hdr = open(os.path.join(ROOT, "include", "capt.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", hdr, re.M))
    assert declared == set(capt_lib.EXPORTED_SYMBOLS)
    lib = ctypes.CDLL(capt_lib._build.LIB)
    for name in declared:
        assert hasattr(lib, name), name


def test_device_calls_reject_unuploaded_tree_without_gpu(capt_lib):
    """Host-side argument checks run before any CUDA call."""
    t = capt_lib.capt_build(W.uniform_cloud(50, 3), 0.01, 0.08)
    L = capt_lib._load()
    rc = L.capt_query_spheres(t.h, None, None, 10, None, None)
    assert rc == -8                                    # CAPT_E_STATE: not uploaded
    assert "not uploaded" in capt_lib.capt_last_error()
    rc = L.capt_query_spheres(None, None, None, 10, None, None)
    assert rc == -1
    st = capt_lib.capt_stats(t)
    assert st["device"] == -1 and st["device_bytes"] == 0


def test_compact_rejects_unuploaded_tree_without_gpu(capt_lib):
    """capt_compact needs the uploaded sets; its checks run before any CUDA call."""
    t = capt_lib.capt_build(W.uniform_cloud(50, 3), 0.01, 0.08)
    L = capt_lib._load()
    assert L.capt_compact(t.h, 0, None) == -8                     # not uploaded
    assert L.capt_compact(None, 0, None) == -1
    st = capt_lib.capt_stats(t)
    assert st["compact_chunks"] == st["compact_entries"] == st["compact_bytes"] == st["full_dropped"] == 0
    assert ctypes.sizeof(capt_lib._Stats) == 168                  # the C struct's size


def test_joint_and_filter_calls_reject_bad_arguments_without_gpu(capt_lib):
    """capt_query_joint_configs and sfc_filter_device check their arguments on the host
    before any CUDA call."""
    t = capt_lib.capt_build(W.uniform_cloud(50, 3), 0.01, 0.08)
    L = capt_lib._load()
    arm = capt_lib.make_arm(W.arm_7dof())
    assert L.capt_query_joint_configs(t.h, ctypes.byref(arm), None, 10, None, None) == -8   # not uploaded
    assert L.capt_query_joint_configs(None, ctypes.byref(arm), None, 10, None, None) == -1
    n = ctypes.c_size_t(7)
    assert L.sfc_filter_device(None, 10, 0.01, None, ctypes.byref(n), None) == -1      # NULL points
    assert L.sfc_filter_device(None, 0, -1.0, None, ctypes.byref(n), None) == -2       # negative spacing
    assert L.sfc_filter_device(None, 0, 0.01, None, ctypes.byref(n), None) == 0 and n.value == 0
    assert L.sfc_filter_device(None, 0, 0.01, None, None, None) == -1


def test_morton_order_follows_the_oracles_curve(orc, capt_lib):
    """capt_morton_order is a permutation along the oracle's Z-order key (21 bits per axis
    over the bounding box, x most significant), ties in ascending index."""
    pts = W.uniform_cloud(3000, 21)
    pts[100:140] = pts[7]                          # coincident points: ties
    pts[200:260, 2] = 0.5                          # a plane: equal z
    order = capt_lib.capt_morton_order(pts)
    assert sorted(order.tolist()) == list(range(len(pts)))
    p64 = pts.astype(np.float64)
    lo, hi = p64.min(0), p64.max(0)
    q = np.minimum(2 ** 21 - 1, np.floor((p64 - lo) / (hi - lo) * 2097152.0)).astype(np.int64)
    keys = np.array([orc.morton_key(q[i], (0, 1, 2)) for i in order], dtype=np.uint64)
    assert np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(order[1:][same] > order[:-1][same])
    assert capt_lib.capt_morton_order(np.zeros((0, 3), np.float32)).size == 0
    bad = pts.copy()
    bad[5, 0] = np.nan
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_morton_order(bad)
    assert e.value.status == -3


def test_depth_frame_is_a_full_deterministic_frame():
    f = W.depth_frame()
    assert f.shape == (640 * 480, 3) and f.dtype == np.float32 and np.all(np.isfinite(f))
    assert np.array_equal(f, W.depth_frame())
    # the camera looks down at the table: most pixels see the table top or what is on it
    assert ((f[:, 2] > -0.01) & (f[:, 0] >= -0.01) & (f[:, 0] <= 1.21)).mean() > 0.5


def test_edge_and_query_bindings_reject_mismatched_buffers_without_gpu(capt_lib):
    """The C ABI receives base addresses and counts only, so the binding must refuse
    buffers whose shapes disagree before any pointer reaches a kernel."""
    import torch
    pts = W.uniform_cloud(64, 7)
    tree = capt_lib.capt_build(pts, 0.02, 0.08)
    arm = W.arm_7dof()
    E = 8
    qa = torch.zeros((E, 7))
    ns = torch.ones(E, dtype=torch.int32)
    bad = [
        dict(qa=torch.zeros((E, 6)), qb=torch.zeros((E, 6)), nsteps=ns, valid=None),      # wrong joint count
        dict(qa=qa, qb=torch.zeros((E - 1, 7)), nsteps=ns, valid=None),                  # shorter qb
        dict(qa=qa, qb=qa, nsteps=torch.ones(E - 1, dtype=torch.int32), valid=None),     # shorter nsteps
        dict(qa=qa, qb=qa, nsteps=ns, valid=torch.ones(E - 2, dtype=torch.uint8)),       # shorter valid
        dict(qa=torch.zeros(E * 7), qb=torch.zeros(E * 7), nsteps=ns, valid=None),        # flat qa
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            capt_lib.capt_validate_edges(tree, arm, kw["qa"], kw["qb"], kw["nsteps"], kw["valid"])
        with pytest.raises(ValueError):
            capt_lib.capt_validate_edges_static(tree, arm, kw["qa"], kw["qb"], kw["nsteps"], kw["valid"])
        with pytest.raises(ValueError):
            capt_lib.capt_edge_plan_create(tree, arm, kw["qa"], kw["qb"], kw["nsteps"],
                                           kw["valid"] if kw["valid"] is not None else torch.ones(E, dtype=torch.uint8))
    # outputs of the other queries
    c = torch.zeros((5, 60, 3))
    r = torch.ones(60)
    with pytest.raises(ValueError):
        capt_lib.capt_query_configs(tree, c, r, torch.zeros(4, dtype=torch.uint8))
    with pytest.raises(ValueError):
        capt_lib.capt_query_configs(tree, c, torch.ones(59))
    with pytest.raises(ValueError):
        capt_lib.capt_query_spheres(tree, torch.zeros((5, 3)), torch.ones(5), torch.zeros(6, dtype=torch.uint8))
    with pytest.raises(ValueError):
        capt_lib.capt_query_joint_configs(tree, arm, torch.zeros((5, 7)), torch.zeros(3, dtype=torch.uint8))
    with pytest.raises(ValueError):
        capt_lib.capt_query_leaves(tree, torch.zeros((5, 3)), torch.zeros(4, dtype=torch.int32))
    with pytest.raises(ValueError):
        capt_lib.capt_query_configs_host(tree, np.zeros((5, 60, 3), np.float32), np.ones(60, np.float32),
                                         np.zeros(4, np.uint8))
    cc = torch.zeros((2, 3, 60, 3))
    with pytest.raises(ValueError):
        capt_lib.capt_clearance_fwd(tree, cc, r, 0.01, dist=torch.zeros(2 * 3 * 60 - 1))
    with pytest.raises(ValueError):
        capt_lib.capt_clearance_bwd(tree, cc, r, torch.zeros(360), torch.zeros(360, dtype=torch.int32),
                                    torch.ones(3), 0.01)


def test_binding_structs_match_the_c_header(capt_lib, tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's sizes and field
    offsets (a mismatch would make every call read or write the wrong bytes)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"capt_tree_stats": capt_lib._Stats, "capt_launch_cfg": capt_lib._LaunchCfg, "capt_arm": capt_lib._Arm,
               "capt_grid_info": capt_lib._GridInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "capt.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_near_lists_and_clearance_autotuner_reject_bad_state_without_gpu(capt_lib):
    """capt_build_near_lists and capt_autotune_clearance check the tree and their
    arguments on the host before any CUDA call."""
    t = capt_lib.capt_build(W.uniform_cloud(50, 3), 0.0, 0.08)
    L = capt_lib._load()
    assert L.capt_build_near_lists(t.h, None) == -8               # not uploaded
    assert L.capt_build_near_lists(None, None) == -1
    cfg, ms = capt_lib._LaunchCfg(), ctypes.c_float()
    assert L.capt_autotune_clearance(t.h, None, None, 1, 1, 1, 0.01, None, None, None, None,
                                     ctypes.byref(cfg), ctypes.byref(ms)) == -8
    assert L.capt_autotune_clearance(None, None, None, 1, 1, 1, 0.01, None, None, None, None,
                                     ctypes.byref(cfg), ctypes.byref(ms)) == -1
    st = capt_lib.capt_stats(t)
    assert st["near_entries"] == st["near_bytes"] == st["near_fallback_cells"] == 0
    # the clearance launch defaults to the lists (used once they exist)
    assert capt_lib.capt_get_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE)["grid"] == 1
