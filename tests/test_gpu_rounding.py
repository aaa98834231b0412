"""The FP32 distance test is the oracle's separately rounded expression,
((px - cx)^2 + (py - cy)^2) + (pz - cz)^2 <= fl(r^2), with no fused multiply-add
anywhere (Sec. IV-D's test as the oracle states it, every operation rounded).

Adversarial spheres: each centre lies at distance R (to within 4e-7 relative) from one
point of a sparse lattice (no other point within reach), placed so that fl(R^2) falls
between the separately rounded squared distance and the once-rounded one that fused
multiply-adds give.  So every flag here flips if the products are fused into the sum
on the way.  The same spheres' clearance distances must be fl(sqrt(separately rounded
d^2)) bit for bit, on the paper's path and on the nearest-candidate lists."""
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


R = np.float32(0.05)   # every sphere's radius


def _adversarial(seed=5, want=40000):
    """(points, centres, index of each centre's point, separately rounded d^2): centres at
    distance R (1 +- 4e-7) from a lattice point, kept when the separately rounded and
    the once-rounded squared distances lie on opposite sides of fl(R^2)."""
    rng = np.random.default_rng(seed)
    g = np.arange(6, dtype=np.float32) * np.float32(0.3)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pts = (pts + rng.uniform(-0.01, 0.01, pts.shape)).astype(np.float32)
    rr = np.float32(R * R)
    cen, own, sep = [], [], []
    n = 0
    while n < want:
        k = rng.integers(0, len(pts), 1 << 16)
        u = rng.normal(size=(1 << 16, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        t = np.float64(R) * (1.0 + rng.uniform(-4e-7, 4e-7, (1 << 16, 1)))
        c = (pts[k] + t * u).astype(np.float32)
        d = (pts[k] - c).astype(np.float32)                       # p - c, rounded
        sq = (d * d).astype(np.float32)                           # each square rounded
        plain = ((sq[:, 0] + sq[:, 1]).astype(np.float32) + sq[:, 2]).astype(np.float32)
        d64 = d.astype(np.float64)
        once = (d64 * d64).sum(1).astype(np.float32)              # one rounding, as fusing gives
        keep = (plain <= rr) != (once <= rr)
        cen.append(c[keep])
        own.append(k[keep])
        sep.append(plain[keep])
        n += int(keep.sum())
    cen, own, sep = (np.concatenate(x)[:want] for x in (cen, own, sep))
    return pts, cen, own, sep


@pytest.fixture(scope="module")
def adv(capt_lib, torch_):
    pts, c, own, sep = _adversarial()
    tree = capt_lib.capt_build(pts, 0.0, 0.08)
    capt_lib.capt_upload(tree, 0)
    return dict(pts=pts, c=c, own=own, sep=sep, tree=tree)


def test_adversarial_flags_follow_the_separately_rounded_test(adv, orc):
    """The construction: the oracle's FP32 brute force gives the separately rounded
    verdict, with both verdicts well represented, and the once-rounded verdict would be
    the opposite on every sphere."""
    r = np.full(len(adv["c"]), R, np.float32)
    flags = orc.brute_flags(adv["pts"], adv["c"], r)
    assert np.array_equal(flags.astype(bool), adv["sep"] <= np.float32(R * R))
    assert 0.2 < flags.mean() < 0.8


@pytest.mark.parametrize("warps,spl,stage,chunk", [(w, s, st, ch) for w in (4, 8) for s in (1, 2, 4, 8)
                                                   for st in (0, 1) for ch in (0, 1)])
def test_sphere_queries_never_fuse(adv, orc, capt_lib, torch_, warps, spl, stage, chunk):
    t = adv["tree"]
    r = np.full(len(adv["c"]), R, np.float32)
    ref = orc.brute_flags(adv["pts"], adv["c"], r)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_SPHERES, warps, spl, stage, chunk)
    f = capt_lib.capt_query_spheres(t, _cuda(torch_, adv["c"]), _cuda(torch_, r)).cpu().numpy()
    assert np.array_equal(f, ref)
    assert capt_lib.capt_device_status(t) == 0


@pytest.mark.parametrize("S", [1, 2])
@pytest.mark.parametrize("spl,chunk,grid", [(2, 0, 0), (8, 1, 0), (16, 0, 1), (4, 1, 1)])
def test_configuration_queries_never_fuse(adv, orc, capt_lib, torch_, S, spl, chunk, grid):
    """Configurations of S spheres of radius R, with and without the grid, against the
    oracle's FP32 brute force."""
    t = adv["tree"]
    if grid:
        capt_lib.capt_build_grid(t, 1 << 20)
    c = adv["c"].reshape(-1, S, 3)
    rad = np.full(S, R, np.float32)
    ref = orc.brute_config_flags(adv["pts"], c, rad)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CONFIGS, 4, spl, 0, chunk, 0, grid)
    got = capt_lib.capt_query_configs(t, _cuda(torch_, c), _cuda(torch_, rad)).cpu().numpy()
    assert np.array_equal(got, ref)
    assert capt_lib.capt_device_status(t) == 0


def test_clearance_distances_are_the_separately_rounded_ones(adv, capt_lib, torch_):
    """d = fl(sqrt(separately rounded d^2)) to the centre's own lattice point, bit for bit,
    with the paper's path and with the nearest-candidate lists."""
    t = adv["tree"]
    c = adv["c"].reshape(-1, 1, 1, 3)
    r = np.full(1, R, np.float32)
    want = np.sqrt(adv["sep"]).astype(np.float32)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE, 16, 2, 0, 0, 0, 0)
    _, d, am = capt_lib.capt_clearance_fwd(t, _cuda(torch_, c), _cuda(torch_, r), 0.01)
    assert np.array_equal(d.cpu().numpy().ravel().view(np.uint32), want.view(np.uint32))
    assert np.array_equal(am.cpu().numpy().ravel(), adv["own"])
    capt_lib.capt_build_grid(t, 1 << 20)
    capt_lib.capt_build_near_lists(t)
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_CLEARANCE, 16, 2, 0, 0, 0, 1)
    _, d2, am2 = capt_lib.capt_clearance_fwd(t, _cuda(torch_, c), _cuda(torch_, r), 0.01)
    assert np.array_equal(d2.cpu().numpy().ravel().view(np.uint32), want.view(np.uint32))
    assert np.array_equal(am2.cpu().numpy().ravel(), adv["own"])
    assert capt_lib.capt_device_status(t) == 0


def _sep_d2(p, c):
    """The oracle's FP32 squared distance, every operation rounded (numpy float32)."""
    d = (np.asarray(p, np.float32) - np.asarray(c, np.float32)).astype(np.float32)
    sq = (d * d).astype(np.float32)
    return ((sq[..., 0] + sq[..., 1]).astype(np.float32) + sq[..., 2]).astype(np.float32)


def _boundary_cloud(orc, arm, q, seed=9):
    """One point per configuration, one FP32 rounding step inside or outside the
    boundary of one of its distal spheres (links 3 and up) and inside none of its other
    spheres, chosen so that moving that sphere's centre by one ulp per coordinate (away
    from the point, or toward it) flips the configuration's flag.  Returns the points
    and the number of configurations for which such a point was found (the others get a
    point far away)."""
    rng = np.random.default_rng(seed)
    cen = orc.fk32(arm, q)                                # [C, S, 3], the oracle's FP32 kinematics
    rad = np.asarray(arm.sphere_radius, np.float32)
    rr_all = (rad * rad).astype(np.float32)
    distal = np.nonzero(np.asarray(arm.sphere_link) >= 3)[0]
    pts, found = [], 0
    for k in range(len(cen)):
        want_in = k % 2 == 0
        best = None
        for _ in range(32):
            s = distal[rng.integers(0, len(distal))]
            c = cen[k, s]
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            p = (c.astype(np.float64) + rad[s] * (1 + 2e-6) * u).astype(np.float32)
            for _ in range(200):                          # step in until the test passes
                if _sep_d2(p, c) <= rr_all[s]:
                    break
                p = np.nextafter(p, c)
            if not want_in:                               # then one step back out
                p = np.nextafter(p, p + (p - c))
                if _sep_d2(p, c) <= rr_all[s]:
                    continue
            others = np.delete(np.arange(len(rad)), s)
            if np.any(_sep_d2(p, cen[k, others]) <= rr_all[others]):
                continue                                  # inside another sphere: no teeth
            moved = np.nextafter(c, c + (c - p)) if want_in else np.nextafter(c, p)
            if (_sep_d2(p, moved) <= rr_all[s]) == want_in:
                continue                                  # a one-ulp move does not flip it
            best = p
            break
        if best is None:
            best = np.full(3, 50.0, np.float32)           # far from everything
        else:
            found += 1
        pts.append(best)
    return np.array(pts, np.float32), found


def test_joint_angle_kinematics_never_fuse(orc, capt_lib, torch_):
    """The joint-angle kernel's kinematics are the oracle's separately rounded FP32 ones:
    on clouds whose points sit on sphere boundaries, where a centre off by one ulp flips
    the configuration, its flags are the oracle's, with and without the grid, and so are
    the edge validator's (edges of one configuration).  Batches of four configurations
    turned a quarter turn apart at the base, one point each, so that a point meets only
    its own configuration."""
    arm = W.arm_7dof()
    rad = np.asarray(arm.sphere_radius, np.float32)
    rng = np.random.default_rng(33)
    n_hang = n_all = 0
    for b in range(48):
        q = W.random_configs(4, 100 + b).astype(np.float32)
        q[:, 0] = (np.arange(4) * (np.pi / 2) + rng.uniform(-0.2, 0.2, 4)).astype(np.float32)
        p, found = _boundary_cloud(orc, arm, q, seed=200 + b)
        n_hang += found
        n_all += len(q)
        ref = orc.brute_config_flags(p, orc.fk32(arm, q), rad)
        tree = capt_lib.capt_build(p, 0.0, float(rad.max()))
        capt_lib.capt_upload(tree, 0)
        qd = _cuda(torch_, q)
        ones = _cuda(torch_, np.ones(len(q), np.int32))
        for grid in (0, 1):
            if grid:
                capt_lib.capt_build_grid(tree, 1 << 16)
            capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_JOINTS, 4, 1, 0, 0, 0, grid)
            f = capt_lib.capt_query_joint_configs(tree, arm, qd).cpu().numpy()
            assert np.array_equal(f, ref)
            capt_lib.capt_set_launch_cfg(tree, capt_lib.CAPT_KERNEL_EDGES, 8, 2, 0, 32, 0, grid)
            v = capt_lib.capt_validate_edges(tree, arm, qd, qd, ones).cpu().numpy()
            assert np.array_equal(v, 1 - ref)
        assert capt_lib.capt_device_status(tree) == 0
        capt_lib.capt_free(tree)
    assert n_hang > 0.5 * n_all                           # the test has teeth
