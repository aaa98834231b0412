"""Parity of capt_query_joint_configs (configurations given by joint angles, kinematics
inside the kernel) with the oracle: the oracle's own FP32 kinematics gives the sphere
centres, and its FP32 brute force or its plain CAPT (Alg. 1 + Alg. 3) gives the flags.
Flags are compared bit for bit."""
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
    return dict(pts=pts, arm=arm, tree=tree, oracle_tree=orc.PlainCAPT(pts, 0.02, 0.08))


def _q(torch_, q):
    return torch_.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()


def test_joint_configs_against_brute_force(scene, orc, capt_lib, torch_):
    q = W.random_configs(6000, 4242)
    ref = orc.brute_config_flags(scene["pts"], orc.fk32(scene["arm"], q), scene["arm"].sphere_radius)
    f = capt_lib.capt_query_joint_configs(scene["tree"], scene["arm"], _q(torch_, q)).cpu().numpy()
    assert np.array_equal(f, ref)
    assert 0.05 < ref.mean() < 0.95
    assert capt_lib.capt_device_status(scene["tree"]) == 0


@pytest.mark.parametrize("warps,stage", [(w, st) for w in (1, 2, 4, 8, 16) for st in (0, 1)])
def test_joint_configs_every_launch_cfg(scene, orc, capt_lib, torch_, warps, stage):
    q = W.random_configs(2049, 99, first=5)          # ragged last pass of 32
    ref, _ = scene["oracle_tree"].query_configs(orc.fk32(scene["arm"], q), scene["arm"].sphere_radius)
    t = scene["tree"]
    capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_JOINTS, warps, 1, stage)
    try:
        f = capt_lib.capt_query_joint_configs(t, scene["arm"], _q(torch_, q)).cpu().numpy()
    finally:
        capt_lib.capt_set_launch_cfg(t, capt_lib.CAPT_KERNEL_JOINTS, 4, 1, 0)
    assert np.array_equal(f, ref)


def _long_arm():
    """16 joints (the most an arm may have), one sphere per link."""
    from types import SimpleNamespace
    J = 16
    return SimpleNamespace(base=[-0.05, 0.0, 0.06], axis=[2 if j % 2 == 0 else 1 for j in range(J)],
                           link=[[0.0, 0.0, 0.05]] * J, sphere_link=list(range(J)),
                           sphere_offset=[[0.0, 0.0, 0.025]] * J, sphere_radius=[0.03] * J, n_joints=J, n_spheres=J)


def test_joint_configs_long_arm(scene, orc, capt_lib, torch_):
    """A 16-joint arm with one sphere per link, against the oracle's kinematics and
    brute force."""
    arm = _long_arm()
    q = W.random_configs(3000, 17, n_joints=16)
    f = capt_lib.capt_query_joint_configs(scene["tree"], arm, _q(torch_, q)).cpu().numpy()
    ref = orc.brute_config_flags(scene["pts"], orc.fk32(arm, q), np.float32(arm.sphere_radius))
    assert np.array_equal(f, ref)
    assert 0.05 < ref.mean() < 0.95


@pytest.mark.parametrize("C", [1, 31, 32, 33, 95, 1000])
def test_joint_configs_ragged_counts(scene, orc, capt_lib, torch_, C):
    q = W.random_configs(C, 7, first=123)
    ref = orc.brute_config_flags(scene["pts"], orc.fk32(scene["arm"], q), scene["arm"].sphere_radius)
    flags = torch_.full((C + 8,), 7, dtype=torch_.uint8, device="cuda")
    capt_lib.capt_query_joint_configs(scene["tree"], scene["arm"], _q(torch_, q), flags[:C])
    out = flags.cpu().numpy()
    assert np.array_equal(out[:C], ref)
    assert np.all(out[C:] == 7)                       # nothing written past the end


def test_joint_configs_degenerate(scene, orc, capt_lib, torch_):
    arm = scene["arm"]
    # all-zero configuration (the arm straight up), and joint limits exactly
    q = np.zeros((3, 7), np.float32)
    q[1] = 2.8
    q[2] = -2.8
    ref = orc.brute_config_flags(scene["pts"], orc.fk32(arm, q), arm.sphere_radius)
    assert np.array_equal(capt_lib.capt_query_joint_configs(scene["tree"], arm, _q(torch_, q)).cpu().numpy(), ref)
    # zero configurations: a no-op
    empty = torch_.empty((0, 7), dtype=torch_.float32, device="cuda")
    assert capt_lib.capt_query_joint_configs(scene["tree"], arm, empty).numel() == 0
    # an empty cloud never collides
    et = capt_lib.capt_build(np.zeros((0, 3), np.float32), 0.02, 0.08)
    capt_lib.capt_upload(et, 0)
    q = W.random_configs(100, 3)
    assert int(capt_lib.capt_query_joint_configs(et, arm, _q(torch_, q)).sum()) == 0
    with pytest.raises(ValueError):
        capt_lib.capt_query_joint_configs(scene["tree"], arm, _q(torch_, q[:, :6]))


def test_joint_configs_autotune_keeps_results(scene, orc, capt_lib, torch_):
    q = W.random_configs(20000, 555)
    dq = _q(torch_, q)
    cfg, ms = capt_lib.capt_autotune_joint_configs(scene["tree"], scene["arm"], dq)
    assert ms > 0 and cfg["warps_per_block"] in (2, 4, 8, 16)
    f = capt_lib.capt_query_joint_configs(scene["tree"], scene["arm"], dq).cpu().numpy()
    ref, _ = scene["oracle_tree"].query_configs(orc.fk32(scene["arm"], q), scene["arm"].sphere_radius)
    assert np.array_equal(f, ref)


def test_joint_configs_full_size(scene, orc, capt_lib, torch_):
    """1,048,576 configurations, the tabletop workload's size: every flag against the
    oracle's plain CAPT over the oracle's FP32 kinematics, and 4096 sampled against its
    FP32 brute force."""
    C = 1 << 20
    q = W.random_configs(C, 1001)
    cen = orc.fk32(scene["arm"], q)
    r = scene["arm"].sphere_radius
    f = capt_lib.capt_query_joint_configs(scene["tree"], scene["arm"], _q(torch_, q)).cpu().numpy()
    ref, _ = scene["oracle_tree"].query_configs(cen, r)
    assert np.array_equal(f, ref)
    idx = np.random.default_rng(1).choice(C, 4096, replace=False)
    assert np.array_equal(f[idx], orc.brute_config_flags(scene["pts"], cen[idx], r))
