"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Flags are compared bit for bit: Lemma 1 makes the CAPT answer equal to the FP32 brute
force over the cloud, and the kernels evaluate the same FP32 expression.  Clearance is
compared with the FP64 oracle within 1e-5 absolute, gradients within 1e-3 relative.
The oracle never sees an output of the CUDA path: both sides get the same seeded
inputs and, where a cloud is filtered first, each side filters with its own Alg. 2
(the two outputs are checked equal before use)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ALL_CFGS = [(w, s, st, ch) for w in (4, 8, 16) for s in (1, 2, 4, 8) for st in (0, 1) for ch in (0, 1)]


@pytest.fixture(scope="module")
def torch_():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cuda(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.fixture(scope="module")
def uniform2k(orc, capt_lib, torch_):
    p = W.WORKLOADS["uniform2k"].params
    pts = W.uniform_cloud(p["n_points"], 1000)
    c, r = W.cube_queries(p["n_spheres"], 1000)
    tree = capt_lib.capt_build(pts, p["r_min"], p["r_max"])
    capt_lib.capt_upload(tree, 0)
    ref = orc.brute_flags(pts, c, r)
    return dict(pts=pts, c=c, r=r, tree=tree, ref=ref, dc=_cuda(torch_, c), dr=_cuda(torch_, r))


@pytest.fixture(scope="module")
def tabletop(orc, capt_lib, torch_):
    raw, _, arm = W.tabletop_scene(1001)
    k_gpu = capt_lib.sfc_filter(raw, 0.01)
    k_orc = orc.sfc_filter(raw, 0.01)
    assert np.array_equal(k_gpu, k_orc)
    pts_gpu, pts_orc = raw[k_gpu], raw[k_orc]
    tree = capt_lib.capt_build(pts_gpu, 0.02, 0.08)
    capt_lib.capt_upload(tree, 0)
    ctree = capt_lib.capt_build(pts_gpu, 0.0, 0.08)
    capt_lib.capt_upload(ctree, 0)
    return dict(pts=pts_orc, pts_gpu=pts_gpu, arm=arm, tree=tree, ctree=ctree,
                oracle_tree=orc.PlainCAPT(pts_orc, 0.02, 0.08))


# --------------------------------------------------------------------- sphere queries

def test_spheres_uniform2k_bit_exact(uniform2k, capt_lib, torch_):
    f = capt_lib.capt_query_spheres(uniform2k["tree"], uniform2k["dc"], uniform2k["dr"])
    torch_.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), uniform2k["ref"])
    assert 0.05 < uniform2k["ref"].mean() < 0.95
    assert capt_lib.capt_device_status(uniform2k["tree"]) == 0


@pytest.mark.parametrize("warps,spl,stage,chunked", ALL_CFGS)
def test_spheres_every_launch_cfg(uniform2k, capt_lib, torch_, warps, spl, stage, chunked):
    t = uniform2k["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, warps, spl, stage, chunked)
    f = capt_lib.capt_query_spheres(t, uniform2k["dc"], uniform2k["dr"])
    assert np.array_equal(f.cpu().numpy(), uniform2k["ref"])
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 1)


def test_spheres_autotune_keeps_results(uniform2k, capt_lib, torch_):
    t = uniform2k["tree"]
    cfg, ms = capt_lib.capt_autotune_spheres(t, uniform2k["dc"], uniform2k["dr"])
    assert ms > 0 and cfg["chunk"] in (0, 1)
    f = capt_lib.capt_query_spheres(t, uniform2k["dc"], uniform2k["dr"])
    assert np.array_equal(f.cpu().numpy(), uniform2k["ref"])
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 1)


@pytest.mark.parametrize("m", [1, 31, 33, 64, 65, 127, 1000, 4097])
def test_spheres_ragged_tails(uniform2k, capt_lib, torch_, m):
    f = capt_lib.capt_query_spheres(uniform2k["tree"], uniform2k["dc"][:m].contiguous(),
                                    uniform2k["dr"][:m].contiguous())
    assert np.array_equal(f.cpu().numpy(), uniform2k["ref"][:m])


def test_spheres_radius_at_both_ends(uniform2k, orc, capt_lib, torch_):
    c = uniform2k["c"][:20000]
    for rv in (0.01, 0.08):
        r = np.full(len(c), rv, np.float32)
        f = capt_lib.capt_query_spheres(uniform2k["tree"], _cuda(torch_, c), _cuda(torch_, r))
        assert np.array_equal(f.cpu().numpy(), orc.brute_flags(uniform2k["pts"], c, r))


def test_spheres_on_points_and_planes(uniform2k, orc, capt_lib, torch_):
    """Centres exactly on cloud points, on split planes and far outside the cloud."""
    pts = uniform2k["pts"]
    T = capt_lib.capt_export(uniform2k["tree"])["T"]
    rng = np.random.default_rng(3)
    on_pts = pts[rng.integers(0, len(pts), 500)]
    planes = rng.uniform(0, 1, (len(T), 3)).astype(np.float32)
    ax = np.arange(len(T))
    depth = np.floor(np.log2(ax + 1)).astype(int) % 3
    planes[ax, depth] = T                              # the splitting coordinate sits on T_i
    far = np.array([[1e6, 1e6, 1e6], [-1e30, 0.5, 0.5], [0.5, 3e38, -3e38]], np.float32)
    c = np.concatenate([on_pts, planes, far]).astype(np.float32)
    r = rng.uniform(0.01, 0.08, len(c)).astype(np.float32)
    f = capt_lib.capt_query_spheres(uniform2k["tree"], _cuda(torch_, c), _cuda(torch_, r))
    assert np.array_equal(f.cpu().numpy(), orc.brute_flags(pts, c, r))
    assert f.cpu().numpy()[:500].all()


def test_leaves_match_oracle_descent(uniform2k, orc, capt_lib, torch_):
    ot = orc.PlainCAPT(uniform2k["pts"], 0.01, 0.08)
    _, leaf, _ = ot.query(uniform2k["c"], uniform2k["r"])
    g = capt_lib.capt_query_leaves(uniform2k["tree"], uniform2k["dc"])
    assert np.array_equal(g.cpu().numpy().astype(np.int64), leaf)


@pytest.mark.parametrize("n", [0, 1, 2, 5])
def test_degenerate_clouds(orc, capt_lib, torch_, n):
    pts = W.uniform_cloud(n, 50 + n)
    c, r = W.cube_queries(3000, 51)
    tree = capt_lib.capt_build(pts, 0.01, 0.08)
    capt_lib.capt_upload(tree, 0)
    for stage in (0, 1):
        capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, stage)
        f = capt_lib.capt_query_spheres(tree, _cuda(torch_, c), _cuda(torch_, r))
        assert np.array_equal(f.cpu().numpy(), orc.brute_flags(pts, c, r))


def test_empty_query_is_noop(uniform2k, capt_lib, torch_):
    e = torch_.empty((0, 3), dtype=torch_.float32, device="cuda")
    f = capt_lib.capt_query_spheres(uniform2k["tree"], e, torch_.empty(0, device="cuda"))
    assert f.numel() == 0


# ------------------------------------------------------------------ configuration queries

def _configs(tabletop, C, seed=1001, first=0):
    q = W.random_configs(C, seed, first=first)
    return W.fk_centers(tabletop["arm"], q)


def test_configs_bit_exact_against_brute_force(tabletop, orc, capt_lib, torch_):
    cen = _configs(tabletop, 6000)
    r = tabletop["arm"].sphere_radius
    ref = orc.brute_config_flags(tabletop["pts"], cen, r)
    f = capt_lib.capt_query_configs(tabletop["tree"], _cuda(torch_, cen), _cuda(torch_, r))
    assert np.array_equal(f.cpu().numpy(), ref)
    assert 0.05 < ref.mean() < 0.95


@pytest.mark.parametrize("warps,spl,stage,chunked",
                         [(w, s, st, ch) for w in (4, 8, 16) for s in (2, 4, 8, 16) for st in (0, 1) for ch in (0, 1)])
def test_configs_every_launch_cfg(tabletop, orc, capt_lib, torch_, warps, spl, stage, chunked):
    cen = _configs(tabletop, 3001, first=777)                    # odd count: ragged last tile
    r = tabletop["arm"].sphere_radius
    ref, _ = tabletop["oracle_tree"].query_configs(cen, r)
    t = tabletop["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, warps, spl, stage, chunked)
    f = capt_lib.capt_query_configs(t, _cuda(torch_, cen), _cuda(torch_, r))
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, 1)
    assert np.array_equal(f.cpu().numpy(), ref)


@pytest.mark.parametrize("S", [1, 7, 32, 33, 64])
def test_configs_sphere_counts(tabletop, orc, capt_lib, torch_, S):
    arm = W.arm_7dof(S)
    q = W.random_configs(1500, 4242)
    cen = W.fk_centers(arm, q)
    ref = orc.brute_config_flags(tabletop["pts"], cen, arm.sphere_radius)
    f = capt_lib.capt_query_configs(tabletop["tree"], _cuda(torch_, cen), _cuda(torch_, arm.sphere_radius))
    assert np.array_equal(f.cpu().numpy(), ref)


def test_work_counters_match_oracle(tabletop, capt_lib, torch_):
    """Spheres examined, leaf-box passes and points scanned equal the oracle's Alg. 3
    counts; the root box count is the FP32 box test against the cloud's bounds."""
    cen = _configs(tabletop, 4000, first=99)
    r = tabletop["arm"].sphere_radius
    flags, counts = tabletop["oracle_tree"].query_configs(cen, r)
    g = capt_lib.capt_count_config_work(tabletop["tree"], _cuda(torch_, cen), _cuda(torch_, r)).cpu().numpy()
    assert [g[0], g[2], g[3]] == counts.tolist()
    pts = tabletop["pts"]
    lo, hi = pts.min(0), pts.max(0)
    d = (cen - np.clip(cen, lo, hi)).astype(np.float32)
    q = d * d
    near = ((q[..., 0] + q[..., 1]) + q[..., 2]) <= (r * r)[None, :]
    # spheres examined: all S of a free configuration, up to the first hit otherwise
    assert g[1] <= near.sum() and g[1] >= near[flags == 0].sum()


def test_sphere_work_counters_match_oracle(uniform2k, orc, capt_lib, torch_):
    """Per-sphere counts (each sphere its own radius) against the oracle's plain Alg. 3:
    every sphere examined, a sphere passing its leaf box scans at least one point, and
    the points scanned up to the first hit add up."""
    ot = orc.PlainCAPT(uniform2k["pts"], 0.01, 0.08)
    f, _, ms = ot.query(uniform2k["c"], uniform2k["r"])
    g = capt_lib.capt_count_sphere_work(uniform2k["tree"], uniform2k["dc"], uniform2k["dr"]).cpu().numpy()
    assert g[0] == len(ms)
    assert g[2] == int((ms > 0).sum())
    assert g[3] == int(ms.sum())
    assert g[5] <= g[3] and g[4] >= g[2]
    assert g[6] == g[7] == 0
    # with the grid every sphere that reaches the cloud's box is looked up, and the
    # decided ones never descend
    t = uniform2k["tree"]
    capt_lib.capt_build_grid(t, 1 << 16)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 1, 0, 0, 1)
    h = capt_lib.capt_count_sphere_work(t, uniform2k["dc"], uniform2k["dr"]).cpu().numpy()
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 1, 0)
    assert h[0] == g[0] and h[1] == g[1] and h[6] == g[1]
    assert 0 < h[7] <= h[6] and h[2] <= g[2] and h[3] <= g[3]
    assert capt_lib.capt_device_status(t) == 0


def test_clearance_work_counters_match_oracle_tree(tabletop, orc, capt_lib, torch_):
    """Clearance work (full-set scans within r_max) counted from the oracle's own tree:
    its leaves (Alg. 3 descent), its leaf boxes and set sizes, the FP32 box expression."""
    arm = tabletop["arm"]
    q = W.random_trajectories(64, 8, 1011)
    c = W.fk_centers(arm, q.reshape(-1, 7)).reshape(-1, 3)
    pts = tabletop["pts"]
    ot = orc.PlainCAPT(pts, 0.0, 0.08)
    _, leaf, _ = ot.query(c, np.full(len(c), 0.08, np.float32))
    ex = ot.export()
    cnt = np.diff(ex["set_begin"].astype(np.int64))
    aabb = ex["aabb"].reshape(-1, 6)

    def box_d2(x, lo, hi):
        g = (x - np.minimum(np.maximum(x, lo), hi)).astype(np.float32)
        q2 = g * g
        return (q2[:, 0] + q2[:, 1]) + q2[:, 2]

    r2 = np.float32(0.08) * np.float32(0.08)
    near = box_d2(c, pts.min(0), pts.max(0)) <= r2
    lb = aabb[leaf]
    ok = near & (cnt[leaf] > 0) & (box_d2(c, lb[:, :3], lb[:, 3:]) <= r2)
    want = [len(c), int(near.sum()), int(ok.sum()), int(cnt[leaf][ok].sum()), int(((cnt[leaf][ok] + 3) // 4).sum())]
    g = capt_lib.capt_count_clearance_work(tabletop["ctree"], _cuda(torch_, c)).cpu().numpy()
    assert g.tolist() == want + [0, 0, 0]   # no nearest-candidate lists on this tree
    assert want[2] > 0


def _chunk_model_counts(ex, pts, cen, r, L):
    """Chunked-scan work counted sequentially in FP32 from the oracle's tree: the block
    layout (each set from a 4-point block boundary, sets in leaf order), boxes of chunks
    of 8 consecutive blocks, then per configuration, sphere by sphere until the first
    hit: chunk boxes tested and points scanned in the chunks whose box the sphere
    reaches."""
    T, sb, si, aabb = ex["T"], ex["set_begin"].astype(np.int64), ex["set_idx"], ex["aabb"].reshape(-1, 6)
    N = len(sb) - 1
    cnt = np.diff(sb)
    fb = np.concatenate([[0], np.cumsum((cnt + 3) // 4)]).astype(np.int64)
    slots = np.full((int(fb[-1]) * 4 + 32, 3), np.inf, np.float32)
    for leaf in range(N):
        if cnt[leaf]:
            slots[fb[leaf] * 4: fb[leaf] * 4 + cnt[leaf]] = pts[si[sb[leaf]:sb[leaf + 1]]]
    nch = (max(int(fb[-1]), 1) + 7) // 8
    ch = slots[: nch * 32].reshape(nch, 32, 3)
    fin = np.isfinite(ch)
    clo, chi = np.where(fin, ch, np.inf).min(1), np.where(fin, ch, -np.inf).max(1)
    lo, hi = pts.min(0), pts.max(0)

    def bd2(x, a, b):
        d = (x - np.clip(x, a, b)).astype(np.float32)
        q = d * d
        return (q[0] + q[1]) + q[2]

    def d2(x, P):
        d = (x[None, :] - P).astype(np.float32)
        q = d * d
        return (q[:, 0] + q[:, 1]) + q[:, 2]

    nbox = ncpts = 0
    r2 = (r * r).astype(np.float32)
    for c in range(cen.shape[0]):
        for s in range(cen.shape[1]):
            x = cen[c, s]
            if not bd2(x, lo, hi) <= r2[s]:
                continue
            i = 0
            for l in range(L):
                i = 2 * i + 1 + int(x[l % 3] > T[i])
            leaf = i - (N - 1)
            if cnt[leaf] == 0 or not bd2(x, aabb[leaf, :3], aabb[leaf, 3:]) <= r2[s]:
                continue
            b0, b1 = int(fb[leaf]), int(fb[leaf + 1])
            hit = False
            for k in range(b0 // 8, (b1 - 1) // 8 + 1):
                nbox += 1
                if not bd2(x, clo[k], chi[k]) <= r2[s]:
                    continue
                j0, j1 = max(b0, 8 * k) * 4, min(b1 * 4, (k + 1) * 32, b0 * 4 + int(cnt[leaf]))
                h = np.nonzero(d2(x, slots[j0:j1]) <= r2[s])[0]
                if len(h):
                    ncpts += int(h[0]) + 1
                    hit = True
                    break
                ncpts += j1 - j0
            if hit:
                break
    return nbox, ncpts


def test_chunk_work_counters_match_model(tabletop, capt_lib, torch_):
    """The chunk counters of capt_count_config_work equal a sequential FP32 count over
    the oracle's tree, and the chunked walk finds exactly the plain walk's hits (the
    device status stays clean)."""
    cen = _configs(tabletop, 300, first=4321)
    r = tabletop["arm"].sphere_radius
    g = capt_lib.capt_count_config_work(tabletop["tree"], _cuda(torch_, cen), _cuda(torch_, r)).cpu().numpy()
    ex = tabletop["oracle_tree"].export()
    L = capt_lib.capt_stats(tabletop["tree"])["depth"]
    assert (int(g[4]), int(g[5])) == _chunk_model_counts(ex, tabletop["pts"], cen, r, L)
    assert g[5] < g[3] and g[4] > 0
    assert capt_lib.capt_device_status(tabletop["tree"]) == 0


def test_host_buffer_pipeline_matches_device_path(tabletop, capt_lib, torch_):
    cen = _configs(tabletop, 140_000, first=5)                   # three chunks, ragged last
    r = tabletop["arm"].sphere_radius
    dev = capt_lib.capt_query_configs(tabletop["tree"], _cuda(torch_, cen), _cuda(torch_, r)).cpu().numpy()
    pinned = torch_.from_numpy(cen).pin_memory()
    host = capt_lib.capt_query_configs_host(tabletop["tree"], pinned, r)   # read in place, flags copied
    assert np.array_equal(host, dev)
    pflags = torch_.full((len(cen),), 7, dtype=torch_.uint8).pin_memory()
    capt_lib.capt_query_configs_host(tabletop["tree"], pinned, r, pflags)  # both in place
    assert np.array_equal(pflags.numpy(), dev)
    host2 = capt_lib.capt_query_configs_host(tabletop["tree"], cen, r)   # pageable: chunked copies
    assert np.array_equal(host2, dev)


@pytest.mark.slow
def test_configs_full_size(tabletop, orc, capt_lib, torch_):
    """1,048,576 configurations: every flag against the oracle's plain CAPT, and a
    sample of 4096 against FP32 brute force."""
    C = 1 << 20
    cen = _configs(tabletop, C)
    r = tabletop["arm"].sphere_radius
    dc = _cuda(torch_, cen)
    capt_lib.capt_autotune_configs(tabletop["tree"], dc, _cuda(torch_, r))
    f = capt_lib.capt_query_configs(tabletop["tree"], dc, _cuda(torch_, r)).cpu().numpy()
    ref, _ = tabletop["oracle_tree"].query_configs(cen, r)
    assert np.array_equal(f, ref)
    idx = np.random.default_rng(0).choice(C, 4096, replace=False)
    assert np.array_equal(f[idx], orc.brute_config_flags(tabletop["pts"], cen[idx], r))


# -------------------------------------------------------------------------------- edges

@pytest.fixture(scope="module")
def edges(tabletop, orc, torch_):
    qa, qb, ns = W.random_edges(4096, 1002)
    ref = orc.edges(tabletop["arm"], qa, qb, ns, tree=tabletop["oracle_tree"])
    return dict(qa=qa, qb=qb, ns=ns, ref=ref, dqa=_cuda(torch_, qa), dqb=_cuda(torch_, qb), dns=_cuda(torch_, ns))


def test_edge_oracle_sample_against_brute_force(tabletop, edges, orc):
    sel = np.arange(0, 4096, 64)
    v = orc.edges(tabletop["arm"], edges["qa"][sel], edges["qb"][sel], edges["ns"][sel], points=tabletop["pts"])
    assert np.array_equal(v, edges["ref"][sel])


@pytest.mark.parametrize("mode", [0, 1])
def test_edges_modes_bit_exact(tabletop, edges, capt_lib, torch_, mode):
    v = capt_lib.capt_validate_edges(tabletop["tree"], tabletop["arm"], edges["dqa"], edges["dqb"], edges["dns"],
                                     mode=mode)
    assert np.array_equal(v.cpu().numpy(), edges["ref"])
    assert 0.05 < edges["ref"].mean() < 0.95


@pytest.mark.parametrize("warps,spl,stage,chunk", [(4, 2, 0, 1), (8, 4, 1, 8), (16, 2, 1, 32), (8, 4, 0, 1024)])
def test_edge_plan_graph_bit_exact(tabletop, edges, capt_lib, torch_, warps, spl, stage, chunk):
    valid = torch_.full((4096,), 7, dtype=torch_.uint8, device="cuda")
    plan = capt_lib.capt_edge_plan_create(tabletop["tree"], tabletop["arm"], edges["dqa"], edges["dqb"],
                                          edges["dns"], valid, cfg=dict(warps_per_block=warps, spheres_per_lane=spl,
                                                                         staging=stage, chunk=chunk))
    for _ in range(2):                                # replays reset their own state
        capt_lib.capt_edge_plan_launch(plan)
        torch_.cuda.synchronize()
        assert np.array_equal(valid.cpu().numpy(), edges["ref"])


def test_edge_plan_autotuned(tabletop, edges, capt_lib, torch_):
    valid = torch_.empty(4096, dtype=torch_.uint8, device="cuda")
    plan = capt_lib.capt_edge_plan_create(tabletop["tree"], tabletop["arm"], edges["dqa"], edges["dqb"],
                                          edges["dns"], valid)
    capt_lib.capt_edge_plan_launch(plan)
    torch_.cuda.synchronize()
    assert np.array_equal(valid.cpu().numpy(), edges["ref"])
    cfg, ms = capt_lib.capt_edge_plan_info(plan)
    assert ms > 0 and cfg["chunk"] in (32, 64, 128)


def test_edges_degenerate_counts(tabletop, orc, capt_lib, torch_):
    qa, qb, ns = W.random_edges(300, 77, nmax=40)
    ns = ns.copy()
    ns[:10] = 0
    ns[10:20] = 1
    ns[20:30] = 2
    ref = orc.edges(tabletop["arm"], qa, qb, ns, tree=tabletop["oracle_tree"])
    for mode in (0, 1):
        v = capt_lib.capt_validate_edges(tabletop["tree"], tabletop["arm"], _cuda(torch_, qa), _cuda(torch_, qb),
                                         _cuda(torch_, ns), mode=mode)
        assert np.array_equal(v.cpu().numpy(), ref)


def test_kernel_kinematics_match_oracle_fk(tabletop, orc, capt_lib, torch_):
    """An edge of one configuration is valid iff that configuration (oracle FP32 FK,
    oracle brute force) is free: checks the in-kernel kinematics bit-exactly on the
    sphere flags over thousands of single configurations."""
    q = W.random_configs(5000, 31337)
    ns = np.ones(len(q), np.int32)
    cen = orc.fk32(tabletop["arm"], q)
    ref = 1 - orc.brute_config_flags(tabletop["pts"], cen, tabletop["arm"].sphere_radius)
    v = capt_lib.capt_validate_edges(tabletop["tree"], tabletop["arm"], _cuda(torch_, q), _cuda(torch_, q),
                                     _cuda(torch_, ns))
    assert np.array_equal(v.cpu().numpy(), ref)


# ---------------------------------------------------------------------------- clearance

def _traj(tabletop, T, W_, seed=1003):
    q = W.random_trajectories(T, W_, seed)
    return W.fk_centers(tabletop["arm"], q.reshape(-1, 7)).reshape(T, W_, -1, 3)


def test_clearance_forward_against_fp64(tabletop, orc, capt_lib, torch_):
    cen = _traj(tabletop, 96, 32)
    r = tabletop["arm"].sphere_radius
    cost, d, am = capt_lib.capt_clearance_fwd(tabletop["ctree"], _cuda(torch_, cen), _cuda(torch_, r), 0.01)
    cost, d, am = cost.cpu().numpy(), d.cpu().numpy(), am.cpu().numpy()
    ocost, od, _ = orc.clearance64(tabletop["pts"], cen, r, 0.08, 0.01, want_grad=False)
    assert np.abs(d - od).max() <= 1e-5
    near = od < 0.08 - 1e-5
    assert near.sum() > 1000                 # random arm postures: a few percent of spheres near the cloud
    dn, idx, d2 = orc.nearest64(tabletop["pts"], cen.reshape(-1, 3))
    sep = (d2 - dn > 1e-5).reshape(d.shape) & near
    assert np.array_equal(am[sep], idx.reshape(d.shape)[sep])
    assert np.all(am[od >= 0.08 + 1e-5] == -1)
    h = np.maximum(0.0, r[None, None, :].astype(np.float64) + 0.01 - od)
    bound = (2 * h * np.abs(d - od) + (d - od) ** 2).sum((1, 2)) + 1e-6 * ocost + 1e-9
    assert np.all(np.abs(cost - ocost) <= bound)


def test_clearance_cost_is_reproducible(tabletop, capt_lib, torch_):
    cen = _cuda(torch_, _traj(tabletop, 64, 32, seed=5))
    r = _cuda(torch_, tabletop["arm"].sphere_radius)
    a = capt_lib.capt_clearance_fwd(tabletop["ctree"], cen, r, 0.01)[0].cpu().numpy()
    for w in (1, 4, 16):
        capt_lib.capt_set_launch_cfg(tabletop["ctree"], capt_lib.CAPT_KERNEL_CLEARANCE, w, 2, w % 2)
        b = capt_lib.capt_clearance_fwd(tabletop["ctree"], cen, r, 0.01)[0].cpu().numpy()
        assert np.array_equal(a, b)
    capt_lib.capt_set_launch_cfg(tabletop["ctree"], capt_lib.CAPT_KERNEL_CLEARANCE, 16, 2, 0)


def test_clearance_backward_against_oracle_and_fd(tabletop, orc, capt_lib, torch_):
    import paper_2406_02807_gb300 as capt
    T, W_ = 48, 32
    cen = _traj(tabletop, T, W_, seed=11)
    r = tabletop["arm"].sphere_radius
    g = np.random.default_rng(1).uniform(0.5, 2.0, T)
    x = _cuda(torch_, cen).requires_grad_(True)
    cost, _, _ = capt.CaptClearance.apply(tabletop["ctree"], x, _cuda(torch_, r), 0.01)
    cost.backward(_cuda(torch_, g.astype(np.float32)))
    grad = x.grad.cpu().numpy().astype(np.float64)
    _, _, ograd = orc.clearance64(tabletop["pts"], cen, r, 0.08, 0.01, grad_cost=g)
    dn, _, d2 = orc.nearest64(tabletop["pts"], cen.reshape(-1, 3))
    hgap = 1e-4
    rr = np.tile(r, T * W_).astype(np.float64)
    away = ((d2 - dn > 4 * hgap) & (np.abs(dn - 0.08) > 2 * hgap) & (np.abs(rr + 0.01 - dn) > 2 * hgap)
            & (dn > 2 * hgap))
    gg, og = grad.reshape(-1, 3)[away], ograd.reshape(-1, 3)[away]
    assert np.all(np.abs(gg - og) <= 1e-3 * np.abs(og) + 1e-6)
    active = np.nonzero(away & (np.abs(ograd.reshape(-1, 3)).sum(1) > 0))[0]
    assert len(active) >= 256
    sample = np.random.default_rng(2).choice(active, 256, replace=False)
    pts64 = tabletop["pts"].astype(np.float64)
    for k in sample:
        t, s = k // (W_ * 60), k % 60
        for a in range(3):
            vals = []
            for sgn in (1, -1):
                y = cen.reshape(-1, 3)[k].astype(np.float64)
                y[a] += sgn * hgap
                dd = min(np.sqrt(((pts64 - y) ** 2).sum(1)).min(), 0.08)
                vals.append(g[t] * max(0.0, float(r[s]) + 0.01 - dd) ** 2)
            fd = (vals[0] - vals[1]) / (2 * hgap)
            assert abs(grad.reshape(-1, 3)[k, a] - fd) <= 1e-3 * abs(fd) + 1e-6


@pytest.mark.slow
def test_clearance_full_size(tabletop, orc, capt_lib, torch_):
    """The full clearance workload (16,384 trajectories x 32 waypoints x 60 spheres) in
    the bench's launch configuration: distances of 30,000 sampled spheres within 1e-5 of
    the FP64 nearest distance, their argmin where the runner-up is separated, and the
    cost and analytic gradient of 48 sampled trajectories against the FP64 oracle."""
    import paper_2406_02807_gb300 as capt
    T, W_ = 16384, 32
    cen = _traj(tabletop, T, W_)
    r = tabletop["arm"].sphere_radius
    x = _cuda(torch_, cen).requires_grad_(True)
    cost, d, am = capt.CaptClearance.apply(tabletop["ctree"], x, _cuda(torch_, r), 0.01)
    cost.sum().backward()
    d, am = d.detach().cpu().numpy().reshape(-1), am.cpu().numpy().reshape(-1)
    rng = np.random.default_rng(3)
    idx = rng.choice(d.size, 30000, replace=False)
    dn, ni, d2 = orc.nearest64(tabletop["pts"], cen.reshape(-1, 3)[idx])
    od = np.minimum(dn, 0.08)
    assert np.abs(d[idx] - od).max() <= 1e-5
    near = dn < 0.08 - 1e-5
    assert near.sum() > 500
    sep = near & (d2 - dn > 1e-5)
    assert np.array_equal(am[idx][sep], ni[sep])
    assert np.all(am[idx][dn >= 0.08 + 1e-5] == -1)
    tr = rng.choice(T, 48, replace=False)
    ocost, odist, ograd = orc.clearance64(tabletop["pts"], cen[tr], r, 0.08, 0.01)
    c_gpu = cost.detach().cpu().numpy()[tr]
    dd = d.reshape(T, W_, -1)[tr]
    h = np.maximum(0.0, r[None, None, :].astype(np.float64) + 0.01 - odist)
    bound = (2 * h * np.abs(dd - odist) + (dd - odist) ** 2).sum((1, 2)) + 1e-6 * ocost + 1e-9
    assert np.all(np.abs(c_gpu - ocost) <= bound)
    g = x.grad.cpu().numpy()[tr].astype(np.float64).reshape(-1, 3)
    dn2, _, d22 = orc.nearest64(tabletop["pts"], cen[tr].reshape(-1, 3))
    hgap = 1e-4
    rr = np.tile(r, len(tr) * W_).astype(np.float64)
    away = ((d22 - dn2 > 4 * hgap) & (np.abs(dn2 - 0.08) > 2 * hgap) & (np.abs(rr + 0.01 - dn2) > 2 * hgap)
            & (dn2 > 2 * hgap))
    og = ograd.reshape(-1, 3)
    assert np.all(np.abs(g[away] - og[away]) <= 1e-3 * np.abs(og[away]) + 1e-6)


def test_clearance_rejects_pruned_tree(tabletop, capt_lib, torch_):
    cen = _cuda(torch_, _traj(tabletop, 2, 2))
    with pytest.raises(capt_lib.CaptError) as e:
        capt_lib.capt_clearance_fwd(tabletop["tree"], cen, _cuda(torch_, tabletop["arm"].sphere_radius), 0.01)
    assert e.value.status == -8


# ------------------------------------------------------------------------ large cloud

@pytest.mark.slow
def test_room_full_size(orc, capt_lib, torch_):
    """200,000-point room, 4,194,304 spheres: every flag against the oracle's plain
    CAPT (built by the oracle), a sample of 20,000 against FP32 brute force."""
    p = W.WORKLOADS["room200k"].params
    pts = W.room_cloud(1004)
    c, r = W.room_queries(p["n_spheres"], 1004)
    tree = capt_lib.capt_build(pts, p["r_min"], p["r_max"])
    capt_lib.capt_upload(tree, 0)
    f = capt_lib.capt_query_spheres(tree, _cuda(torch_, c), _cuda(torch_, r)).cpu().numpy()
    ot = orc.PlainCAPT(pts, p["r_min"], p["r_max"])
    ref, _, _ = ot.query(c, r)
    assert np.array_equal(f, ref)
    idx = np.random.default_rng(0).choice(len(c), 20000, replace=False)
    assert np.array_equal(f[idx], orc.brute_flags(pts, c[idx], r[idx]))
    capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 0, 1)   # chunked scan
    assert np.array_equal(capt_lib.capt_query_spheres(tree, _cuda(torch_, c), _cuda(torch_, r)).cpu().numpy(), ref)
    # the same cloud relabelled along the Z-order curve: the same point set, so the same
    # flags, with either scan
    order = capt_lib.capt_morton_order(pts)
    ts = capt_lib.capt_build(pts[order], p["r_min"], p["r_max"])
    capt_lib.capt_upload(ts, 0)
    for chunked in (0, 1):
        capt_lib.capt_set_launch_cfg(ts, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 0, chunked)
        assert np.array_equal(capt_lib.capt_query_spheres(ts, _cuda(torch_, c), _cuda(torch_, r)).cpu().numpy(), ref)
    # with the distance-bound grid most spheres are decided before any descent: the same
    # flags, with either scan
    capt_lib.capt_build_grid(tree)
    for chunked in (0, 1):
        capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_SPHERES, 8, 2, 0, chunked, 0, 1)
        assert np.array_equal(capt_lib.capt_query_spheres(tree, _cuda(torch_, c), _cuda(torch_, r)).cpu().numpy(), ref)
    assert capt_lib.capt_device_status(tree) == 0


@pytest.mark.parametrize("pf", [1, 2, 4])
@pytest.mark.parametrize("spl", [2, 16])
def test_configs_l2_lookahead(tabletop, orc, capt_lib, torch_, pf, spl):
    """The L2 lookahead of the centre stream changes no flag (ragged batch)."""
    cen = _configs(tabletop, 2999, first=123)
    r = tabletop["arm"].sphere_radius
    ref, _ = tabletop["oracle_tree"].query_configs(cen, r)
    t = tabletop["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 8, spl, 0, 1, pf, 0)
    f = capt_lib.capt_query_configs(t, _cuda(torch_, cen), _cuda(torch_, r))
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 4, 8, 0, 1)
    assert np.array_equal(f.cpu().numpy(), ref)


def test_edge_plan_counts_the_configurations_it_evaluates(orc, capt_lib, torch_):
    """With the cloud out of the arm's reach every edge is valid, so every configuration
    is evaluated and the plan's count is exactly the sum of n_e; with a cloud in reach it
    is at most that (work items already running when their edge is found to collide
    finish their pass; a small batch starts every item at once)."""
    arm = W.arm_7dof()
    qa, qb, ns = W.random_edges(300, 1021, nmax=90)
    far = (W.uniform_cloud(500, 21) + np.float32(10.0)).astype(np.float32)
    for pts, all_valid in ((far, True), (W.tabletop_scene(1001)[0][:8000], False)):
        t = capt_lib.capt_build(pts, 0.02, 0.08)
        capt_lib.capt_upload(t, 0)
        valid = torch_.empty(len(ns), dtype=torch_.uint8, device="cuda")
        plan = capt_lib.capt_edge_plan_create(t, arm, _cuda(torch_, qa), _cuda(torch_, qb), _cuda(torch_, ns), valid,
                                              cfg=dict(warps_per_block=8, spheres_per_lane=1, staging=0, chunk=32))
        capt_lib.capt_edge_plan_launch(plan)
        torch_.cuda.synchronize()
        n = capt_lib.capt_edge_plan_work(plan)
        v = valid.cpu().numpy()
        assert np.array_equal(v, orc.edges(arm, qa, qb, ns, points=pts))
        if all_valid:
            assert v.all() and n == int(np.maximum(ns, 0).sum())
        else:
            assert not v.all() and 0 < n <= int(np.maximum(ns, 0).sum())
        capt_lib.capt_edge_plan_free(plan)
