#!/usr/bin/env python
"""Throughput of the CAPT configuration query on GB300 (one JSON line on rank 0).

Workload (timed): the tabletop scene (30,000 surface points, Morton-order filter at
1 cm, CAPT with r_min = 0.02, r_max = 0.08) and 1,048,576 configurations per GPU of a
7-joint arm with 60 spheres; one step = one capt_query_configs over all of them, the
centres (755 MB, larger than L2) already in HBM.  Metric: sphere queries per second
(configurations x 60 / time; a configuration stops at its first colliding sphere).
Also reported: the same through the host-buffer entry point (e2e), edges validated per
second (4,096 edges, persistent graph launch vs one launch per edge), the roofline of
the query kernel and the oracle timed on the host cores.

Each further workload of the method (clearance forward and backward, the large room
cloud with replicated and compact sets, the small uniform cloud) is timed in the same
run under "workloads", with its own roofline and an oracle parity sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--all]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "sphere-vs-cloud CAPT queries/sec (configuration queries, flags bit-exact)"
UNIT = "sphere queries/s"
SPHERES = 60
R_MIN, R_MAX, R_FILTER = 0.02, 0.08, 0.01
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) per launch of the configuration-query kernel from an ncu
# capture, keyed by the hash of the kernel source it was taken on (null when stale).
TRAFFIC = {"87fc78282cd4552d": 805148672 + 4087296}   # k_configs_grid<32, 0>, tabletop, 1M configurations
HBM_FALLBACK_GBS = 6800.0   # used only when MEASURED_PEAKS.json is absent
PARITY_SAMPLE = 32768       # configurations of the timed run checked against the oracle
GRID_CELLS = 1 << 24        # cells of the distance-bound grid of the tabletop tree (32 MB)
# FP32 operations per configuration evaluated by the kernels that run the arm's
# kinematics, counted from their code: per joint 3 (interpolation) + 30 (sin and cos)
# + 12 (rotation) + 18 (translation); per sphere 18 (placement) + 14 (box test); per link
# 32 for the edge kernel's cull.  Spheres of culled links and of configurations resolved
# early are counted too, so the ALU fractions below are upper bounds.
JOINT_OPS_PER_CFG = 7 * (3 + 30 + 12 + 18) + 60 * (18 + 14)
EDGE_OPS_PER_CFG = JOINT_OPS_PER_CFG + 7 * 32
EDGE_OPS_NOTE = ("issue-bound kinematics: ops = configurations the launch evaluated (counted on the device) x "
                 f"{EDGE_OPS_PER_CFG} FP32 operations each (interpolation, sin/cos, rotations, translations, link "
                 "culls, 60 sphere placements and box tests); an upper bound")
JOINT_OPS_NOTE = (f"issue-bound kinematics: ops = configurations x {JOINT_OPS_PER_CFG} FP32 operations each "
                  "(sin/cos, rotations, translations, 60 sphere placements and box tests); an upper bound")


def hbm_peak():
    """Measured copy bandwidth of this machine's GB300 (GB/s) and where it came from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback (no MEASURED_PEAKS.json)"


# Profiling mode (--profile NAME): the workload, its kernel and the fixed launch
# configuration used (warps per block, spheres per lane, staging, scan, prefetch, grid).
PROFILES = {
    "configs": ("tabletop, 1,048,576 configurations x 60 spheres, grid of 2^24 cells", "k_configs_grid",
                (16, 16, 0, 0, 1, 1)),
    "configs_nogrid": ("tabletop, 1,048,576 configurations x 60 spheres, no grid", "k_configs", (4, 4, 0, 1, 0, 0)),
    "room": ("room, 200,000 points, 4,194,304 spheres, grid of 2^24 cells", "k_spheres", (8, 2, 0, 0, 0, 1)),
    "clearance": ("tabletop, 16,384 x 32 x 60 spheres, r_min = 0, the paper's path", "k_clearance_dist",
                  (16, 2, 0, 0, 0, 0)),
    "clearance_lists": ("tabletop, 16,384 x 32 x 60 spheres, r_min = 0, nearest-candidate lists over a grid of "
                        "2^24 cells", "k_clearance_dist", (8, 2, 0, 0, 0, 1)),
    "near_lists": ("tabletop, r_min = 0, nearest-candidate lists over a grid of 2^24 cells (the builder)",
                   "k_near_lists", (8, 2, 0, 0, 0, 1)),
    "edges": ("tabletop, 4,096 edges (1,038,247 configurations), grid of 2^24 cells", "k_edges_persistent",
              (4, 1, 0, 64, 0, 1)),
    "joints": ("tabletop, 1,048,576 configurations by joint angles, grid of 2^24 cells", "k_joint_configs",
               (8, 1, 0, 0, 0, 1)),
}


def run_profile(args):
    """Set up one workload, then launch only the kernel under study: --warmup launches,
    then --steps launches (an ncu capture skips the first with -s and takes one with -c)."""
    import torch
    import paper_2406_02807_gb300 as capt
    capt.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    _, _, cfg = PROFILES[args.profile]
    name = args.profile
    if name == "room":
        pr = W.room_cloud(1004)
        tree = capt.capt_build(pr, 0.02, 0.10)
        capt.capt_upload(tree, 0)
        capt.capt_build_grid(tree, GRID_CELLS)
        cr, rr = W.room_queries(1 << 22, 1004)
        dc, dr = torch.from_numpy(cr).to(dev), torch.from_numpy(rr).to(dev)
        f = torch.empty(1 << 22, dtype=torch.uint8, device=dev)
        capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_SPHERES, *cfg)
        step = lambda: capt.capt_query_spheres(tree, dc, dr, f)   # noqa: E731
    else:
        raw, _, arm = W.tabletop_scene(1001)
        pts = raw[capt.sfc_filter(raw, R_FILTER)]
        if name in ("clearance", "clearance_lists", "near_lists"):
            tree = capt.capt_build(pts, 0.0, R_MAX)
            capt.capt_upload(tree, 0)
            if cfg[5]:
                capt.capt_build_grid(tree, GRID_CELLS)
                capt.capt_build_near_lists(tree)
            q = W.random_trajectories(16384, 32, 1003)
            c = torch.from_numpy(W.fk_centers(arm, q.reshape(-1, 7)).reshape(16384, 32, SPHERES, 3)).to(dev)
            r = torch.from_numpy(arm.sphere_radius.copy()).to(dev)
            capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_CLEARANCE, *cfg)
            cost = torch.empty(16384, dtype=torch.float32, device=dev)
            d = torch.empty((16384, 32, SPHERES), dtype=torch.float32, device=dev)
            am = torch.empty((16384, 32, SPHERES), dtype=torch.int32, device=dev)
            step = lambda: capt.capt_clearance_fwd(tree, c, r, 0.01, cost, d, am)   # noqa: E731
            if name == "near_lists":
                step = lambda: capt.capt_build_near_lists(tree)   # noqa: E731
        else:
            tree = capt.capt_build(pts, R_MIN, R_MAX)
            capt.capt_upload(tree, 0)
            if cfg[5]:
                capt.capt_build_grid(tree, GRID_CELLS)
            if name == "edges":
                qa, qb, ns = W.random_edges(4096, 1002)
                dqa, dqb, dns = (torch.from_numpy(a).to(dev) for a in (qa, qb, ns))
                v = torch.empty(4096, dtype=torch.uint8, device=dev)
                capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_EDGES, *cfg)
                step = lambda: capt.capt_validate_edges(tree, arm, dqa, dqb, dns, v)   # noqa: E731
            elif name == "joints":
                dq = torch.from_numpy(W.random_configs(1 << 20, 1001)).to(dev)
                f = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
                capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_JOINTS, *cfg)
                step = lambda: capt.capt_query_joint_configs(tree, arm, dq, f)   # noqa: E731
            else:
                cen = torch.from_numpy(W.fk_centers(arm, W.random_configs(1 << 20, 1001))).to(dev)
                r = torch.from_numpy(arm.sphere_radius.copy()).to(dev)
                f = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
                capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_CONFIGS, *cfg)
                step = lambda: capt.capt_query_configs(tree, cen, r, f)   # noqa: E731
    torch.cuda.synchronize()
    for _ in range(args.warmup + args.steps):
        step()
    torch.cuda.synchronize()
    print(json.dumps({"profile": name, "workload": PROFILES[name][0], "kernel": PROFILES[name][1],
                      "launch_cfg": list(cfg), "launches": args.warmup + args.steps,
                      "device_status": capt.capt_device_status(tree)}), flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--configs", type=int, default=1 << 20, help="configurations per GPU")
    ap.add_argument("--all", action="store_true", help="also time the clearance and the other clouds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the clearance, room and uniform-cloud workloads of the default run")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the configuration query (for profiling); the JSON line lacks e2e and the rest")
    ap.add_argument("--profile", choices=sorted(PROFILES),
                    help="for ncu: set up one workload, then launch only its kernel, --warmup times and then "
                         "--steps times, with the fixed launch configuration listed in PROFILES")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(k)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def keep_busy(torch, step, seconds):
    """Run `step` back to back (untimed) for about `seconds`."""
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for _ in range(8):
            step()
        torch.cuda.synchronize()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def src_hash(*names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2406_02807_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def tabletop_tree(capt, with_device=True):
    raw, _, arm = W.tabletop_scene(1001)
    t0 = time.perf_counter()
    kept = capt.sfc_filter(raw, R_FILTER)
    filt_ms = (time.perf_counter() - t0) * 1e3
    pts = raw[kept]
    t0 = time.perf_counter()
    tree1 = capt.capt_build_threads(pts, R_MIN, R_MAX, 1)
    build1_ms = (time.perf_counter() - t0) * 1e3
    del tree1
    tree = capt.capt_build(pts, R_MIN, R_MAX)
    st = capt.capt_stats(tree)
    dev_ms = device_build_ms(capt, pts, R_MIN, R_MAX) if with_device else float("nan")
    dev_filt_ms = device_filter_ms(capt, raw, R_FILTER) if with_device else float("nan")
    return raw, pts, arm, tree, dict(filter_ms=round(filt_ms, 3), build_ms_1thread=round(build1_ms, 3),
                                     build_ms=round(st["build_ms"], 3), build_threads=st["build_threads"],
                                     device_build_ms=round(dev_ms, 3), device_filter_ms=round(dev_filt_ms, 3),
                                     n_points=int(st["n_points"]), n_leaves=int(st["n_leaves"]),
                                     mean_set=round(st["total_afforded"] / st["n_leaves"], 2),
                                     max_set=int(st["max_set"]))


def device_build_ms(capt, pts, r_min, r_max, reps=5):
    """Median wall time of capt_build_device (points already on the device; the call
    returns once the tree is complete), after one untimed call."""
    import torch
    d = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    capt.capt_build_device(d, r_min, r_max)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = capt.capt_build_device(d, r_min, r_max)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
        del t
    return statistics.median(ts)


def host_filter_ms(capt, raw, r, reps=3):
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        capt.sfc_filter(raw, r)
        ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts)


def frame_to_tree_ms(capt, d_points, rf, r_min, r_max, reps=3):
    """Median wall time of capt_build_frame_device (filter + gather + build in one call,
    points already on the device), after one untimed call."""
    import torch
    capt.capt_build_frame_device(d_points, rf, r_min, r_max)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        capt.capt_build_frame_device(d_points, rf, r_min, r_max)
        ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts)


def device_filter_ms(capt, raw, r, reps=5):
    """Median wall time of sfc_filter_device (points already on the device; the call
    returns with the kept count on the host), after one untimed call."""
    import torch
    d = torch.from_numpy(np.ascontiguousarray(raw, np.float32)).cuda()
    capt.sfc_filter_device(d, r)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        capt.sfc_filter_device(d, r)
        ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts)


def time_events(torch, fn, steps, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def time_events_flushed(torch, fn, steps, stream, flush):
    """Mean device time of fn over `steps` calls, each timed alone with CUDA events
    after a write of `flush` (a buffer larger than L2), so no call finds the previous
    call's inputs in L2."""
    total = 0.0
    for _ in range(steps):
        flush.add_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def cpu_baseline(pts, arm, sample_cfgs):
    """The oracle as it stands: FP32 brute force on all host cores, plus its plain CAPT
    single-threaded (the paper's setting: one CPU thread).  Also returns the brute-force
    flags of the sample (the first configurations of the timed workload)."""
    import oracle
    cores = oracle.default_threads()
    cen = W.fk_centers(arm, W.random_configs(sample_cfgs, 1001))
    t0 = time.perf_counter()
    ref_flags = oracle.brute_config_flags(pts, cen, arm.sphere_radius, threads=cores)
    dt = time.perf_counter() - t0
    ot = oracle.PlainCAPT(pts, R_MIN, R_MAX)
    n2 = 2 * sample_cfgs
    cen2 = W.fk_centers(arm, W.random_configs(n2, 1001))
    t0 = time.perf_counter()
    _, counts = ot.query_configs(cen2, arm.sphere_radius)
    dt2 = time.perf_counter() - t0
    return {"value": sample_cfgs * SPHERES / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP32 brute force over all {len(pts)} points for the first {sample_cfgs} configurations "
                      f"of the workload, {cores} threads ({dt:.1f} s wall, {dt * cores:.0f} core-seconds)",
            "plain_capt_1thread": {"ns_per_sphere_query_examined": dt2 * 1e9 / max(int(counts[0]), 1),
                                   "sphere_queries_per_s": n2 * SPHERES / dt2,
                                   "sample": f"{n2} configurations, 1 thread ({dt2:.1f} s)"}}, ref_flags


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    raw, _, arm = W.tabletop_scene(1001)
    kept = oracle.sfc_filter(raw, R_FILTER)
    pts = raw[kept]
    sample = 4096
    cores = oracle.default_threads()
    cen = W.fk_centers(arm, W.random_configs(sample, 1001))
    for _ in range(args.warmup):
        oracle.brute_config_flags(pts, cen, arm.sphere_radius, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.brute_config_flags(pts, cen, arm.sphere_radius, threads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    v = sample * SPHERES / dt
    print(json.dumps({
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
        "config": {"workload": "tabletop_configs", "n_points": int(len(pts)), "spheres_per_config": SPHERES,
                   "configs_per_step": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} configurations per step, FP32 brute force, {cores} threads"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.profile:
        run_profile(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import paper_2406_02807_gb300 as capt
    from paper_2406_02807_gb300.shard import max_over_ranks, weak_slice
    capt.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    raw, pts, arm, tree, host = tabletop_tree(capt, with_device=not args.headline_only)
    capt.capt_upload(tree, local)
    C = args.configs
    first, _ = weak_slice(C, rank)          # this rank's own configurations (weak scaling)
    q = W.random_configs(C, 1001, first=first)
    cen_host = torch.from_numpy(W.fk_centers(arm, q)).pin_memory()
    cen = cen_host.to(dev, non_blocking=False)
    r_host = torch.from_numpy(arm.sphere_radius.copy())
    r = r_host.to(dev)
    flags = torch.empty(C, dtype=torch.uint8, device=dev)

    # the distance-bound grid (one-time per tree, like the upload): spheres that reach the
    # cloud's box are decided by their cell where it can tell, the rest descend
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    capt.capt_build_grid(tree, GRID_CELLS)
    grid_ms = (time.perf_counter() - t0) * 1e3
    gst = capt.capt_stats(tree)
    host["grid_build_ms"] = round(grid_ms, 3)
    host["grid"] = {"dims": gst["grid_dims"], "cell_m": gst["grid_cell"], "bytes": 2 * int(np.prod(gst["grid_dims"]))}
    tuned, tuned_ms = capt.capt_autotune_configs(tree, cen, r, flags)
    counts = capt.capt_count_config_work(tree, cen, r).cpu().numpy().astype(np.int64)
    L = capt.capt_stats(tree)["depth"]
    # FP32 operations per launch of the method as the kernel runs it: a root box test
    # for every examined sphere (15), a grid lookup for the near ones when the grid is on
    # (about 20), a descent and leaf box test for the near ones the grid leaves undecided
    # (L + 15), a box test per chunk walked (15) and 9 per point scanned in the chunks
    # that pass; on-chip bytes likewise (12 per centre, 2 per grid cell, 32 per leaf
    # record, 4 per split, 32 per chunk box, 12 per point)
    ops_per_launch, bytes_per_launch = sphere_ops(counts, L, chunked=tuned["chunk"] != capt.CAPT_SCAN_SETS,
                                                  in_bytes=12)
    # DRAM bytes the step must move: every centre once, the flags, the radii
    hbm_bytes = C * SPHERES * 12 + C + SPHERES * 4

    def step():
        capt.capt_query_configs(tree, cen, r, flags)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # the timed region lasts milliseconds and nvidia-smi samples every 100 ms: the same
    # steps run untimed for a few hundred ms on both sides of it, so that every clock
    # sample is taken under this load
    clocks = Clocks(local)
    clocks.start()
    keep_busy(torch, step, 0.4)
    if pg:
        pg.barrier()
    ms = time_events(torch, step, args.steps, stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    keep_busy(torch, step, 0.3)
    clk = clocks.stop()
    if pg:
        ms = max_over_ranks(ms, pg, dev)
    value = world * C * SPHERES / (ms / 1e3)
    collide = float(flags.float().mean().item())
    flags_host = flags[:PARITY_SAMPLE].cpu().numpy()

    sec = None if args.headline_only else secondary(capt, torch, dev, stream, tree, arm, q, cen, cen_host, r_host,
                                                    flags, C, args, pg)

    out = None
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        peak_tops = sms * 128 * SM_MAX_MHZ * 1e6 / 1e12
        achieved = ops_per_launch / (ms / 1e3) / 1e12
        peak_gbs, peak_src = hbm_peak()
        achieved_gbs = hbm_bytes / (ms / 1e3) / 1e9
        h = src_hash("kernels_query.cu", "scan.cuh", "device_common.cuh", "capt_internal.h")
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "tabletop_configs", "cloud": f"30,000-point tabletop, Morton filter at 1 cm -> "
                                                                f"{len(pts)} points", "configs_per_gpu": C,
                       "spheres_per_config": SPHERES, "r_min": R_MIN, "r_max": R_MAX,
                       "l2": "inputs larger than L2 (755 MB of centres per step); the tree stays resident by design",
                       "parallelism": f"replicas x{world}, configurations sharded by rank", "launch_cfg": tuned},
            "ns_per_sphere_query": 1e9 / value * world,
            "configs_per_s": world * C / (ms / 1e3),
            "collision_fraction": collide,
            # the binding floor is HBM: reading the centres once takes longer than the
            # method's FP32 work at the ALU peak
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                         "frac": achieved_gbs / peak_gbs, "traffic": TRAFFIC.get(h),
                         "peak_basis": peak_src, "algorithmic_bytes_per_launch": hbm_bytes,
                         "hbm_floor_ms": hbm_bytes / (peak_gbs * 1e9) * 1e3,
                         "alu": {"achieved": achieved, "peak": peak_tops, "unit": "TFLOP/s",
                                 "frac": achieved / peak_tops, "floor_ms": ops_per_launch / (peak_tops * 1e12) * 1e3,
                                 "peak_basis": f"{sms} SMs x 128 FP32 lanes x {SM_MAX_MHZ:.0f} MHz "
                                               f"(no FMA on this path)"},
                         "ops_per_launch": ops_per_launch,
                         "work": {"spheres_examined": int(counts[0]), "near_cloud_box": int(counts[1]),
                                  "leaf_box_pass": int(counts[2]), "chunk_boxes": int(counts[4]),
                                  "points_scanned": int(counts[5]), "points_scanned_alg3_alone": int(counts[3]),
                                  "grid_lookups": int(counts[6]), "decided_by_grid": int(counts[7]), "depth": L},
                         "l1_bytes_per_launch": bytes_per_launch,
                         "l1_frac": bytes_per_launch / (ms / 1e3) / (sms * 128 * SM_MAX_MHZ * 1e6)},
            "host": host,
            "gpu_launches": args.steps,
            "clocks": clk,
        }
        if sec:
            out.update(sec)
        if not args.headline_only and not args.no_workloads:
            # the other workloads of the paper's method, each timed on the device with its
            # own roofline (rank 0 only; the other ranks wait at the closing barrier)
            out["workloads"] = {
                "clearance": bench_clearance(capt, torch, dev, stream, pts, arm, max(args.steps // 2, 5), sms),
                "room200k": bench_room(capt, torch, dev, stream, max(args.steps // 2, 5), sms),
                "uniform2k": bench_uniform(capt, torch, dev, stream, args.steps, sms),
            }
        if args.all:
            out["extra"] = extra_workloads(capt, torch, dev, stream, pts, arm, args)
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"], ref = cpu_baseline(pts, arm, PARITY_SAMPLE)
            # the timed run's own flags against the oracle's brute force on the sample
            got = flags_host[:PARITY_SAMPLE]
            out["parity_sample_equal"] = bool(np.array_equal(got, ref))
            out["parity_sample"] = (f"flags of configurations 0..{PARITY_SAMPLE - 1} of the timed run vs the "
                                    f"oracle's FP32 brute force over all {len(pts)} points")
        print(json.dumps(out), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def secondary(capt, torch, dev, stream, tree, arm, q, cen, cen_host, r_host, flags, C, args, pg):
    """The host-buffer (e2e) run of the headline, edges (persistent graph vs per edge)
    and the joint-angle configuration query, as extra keys of the JSON line."""
    from paper_2406_02807_gb300.shard import max_over_ranks
    world = pg.get_world_size() if pg else 1
    # end to end through the host-buffer entry point (copies inside the timed region)
    h_flags = torch.empty(C, dtype=torch.uint8).pin_memory()
    capt.capt_query_configs_host(tree, cen_host, r_host, h_flags)
    e2e_steps = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        capt.capt_query_configs_host(tree, cen_host, r_host, h_flags)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if pg:
        e2e_s = max_over_ranks(e2e_s, pg, dev)
    e2e_ok = bool(torch.equal(h_flags, flags.cpu()))
    # the host link's ceiling on this machine: plain page-locked copies of the same centres
    # (one NUMA node holds every host core and the GPU's affinity here)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    link = {}
    for name, fn in (("h2d", lambda: cen.copy_(cen_host, non_blocking=True)),
                     ("d2h", lambda: cen_host.copy_(cen, non_blocking=True))):
        fn()
        best = 0.0
        for _ in range(3):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            best = max(best, cen_host.numel() * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
        link[name + "_GBps"] = best

    # batched edge validation: persistent graph launch vs one launch per edge
    qa, qb, ns = W.random_edges(4096, 1002)
    dqa, dqb, dns = (torch.from_numpy(a).to(dev) for a in (qa, qb, ns))
    valid = torch.empty(4096, dtype=torch.uint8, device=dev)
    plan = capt.capt_edge_plan_create(tree, arm, dqa, dqb, dns, valid)
    ecfg, _ = capt.capt_edge_plan_info(plan)
    for _ in range(3):
        capt.capt_edge_plan_launch(plan)
    edge_ms = time_events(torch, lambda: capt.capt_edge_plan_launch(plan), max(args.steps, 5), stream)
    torch.cuda.synchronize()
    evaluated = capt.capt_edge_plan_work(plan)
    v_plan = valid.clone()
    valid2 = torch.empty_like(valid)
    capt.capt_set_launch_cfg(tree, capt.CAPT_KERNEL_EDGES, ecfg["warps_per_block"], ecfg["spheres_per_lane"],
                             0, ecfg["chunk"])
    capt.capt_validate_edges(tree, arm, dqa, dqb, dns, valid2, mode=capt.CAPT_EDGES_PER_EDGE)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_edge_steps = 3
    for _ in range(per_edge_steps):
        capt.capt_validate_edges(tree, arm, dqa, dqb, dns, valid2, mode=capt.CAPT_EDGES_PER_EDGE)
    torch.cuda.synchronize()
    per_edge_ms = (time.perf_counter() - t0) * 1e3 / per_edge_steps
    edges_equal = bool(torch.equal(v_plan, valid2))

    # the same configurations given by joint angles: kinematics inside the kernel, so
    # the 755 MB of centres never exist (29 MB of joint angles instead; L2 flushed
    # before every timed call because they would fit in it)
    dq = torch.from_numpy(q).to(dev)
    jflags = torch.empty(C, dtype=torch.uint8, device=dev)
    jcfg, _ = capt.capt_autotune_joint_configs(tree, arm, dq, jflags)
    flush = torch.zeros(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(3):
        capt.capt_query_joint_configs(tree, arm, dq, jflags)
    joint_ms = time_events_flushed(torch, lambda: capt.capt_query_joint_configs(tree, arm, dq, jflags), args.steps,
                                   stream, flush)
    del flush
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    return {
        "e2e": {"value": world * C * SPHERES / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": C * SPHERES * 12 + SPHERES * 4, "d2h_bytes_per_step": C,
                "flags_equal_device_path": e2e_ok,
                "link": dict(link, frac_of_h2d=(C * SPHERES * 12 / e2e_s / 1e9) / max(link["h2d_GBps"], 1e-9),
                             note="plain page-locked copies of the same 755 MB of centres, best of 3")},
        "edges": {"edges": 4096, "configs": int(ns.sum()), "persistent_graph_ms": edge_ms,
                  "edges_per_s_persistent": 4096 / (edge_ms / 1e3), "per_edge_launch_ms": per_edge_ms,
                  "edges_per_s_per_edge": 4096 / (per_edge_ms / 1e3), "valid_fraction": float(valid2.float().mean()),
                  "equal_results": edges_equal, "launch_cfg": ecfg, "configs_evaluated": evaluated,
                  "roofline": roof(edge_ms, int(qa.nbytes + qb.nbytes + ns.nbytes + 4096), evaluated * EDGE_OPS_PER_CFG,
                                   None, sms, note=EDGE_OPS_NOTE)},
        "joint_configs": {"configs": C, "ms": joint_ms, "configs_per_s": world * C / (joint_ms / 1e3),
                          "sphere_queries_per_s": world * C * SPHERES / (joint_ms / 1e3),
                          "collision_fraction": float(jflags.float().mean().item()), "launch_cfg": jcfg,
                          "input_bytes": int(q.nbytes), "l2": "flushed before every timed call",
                          "roofline": roof(joint_ms, int(q.nbytes) + C, C * JOINT_OPS_PER_CFG, None, sms,
                                           note=JOINT_OPS_NOTE)},
    }


def roof(ms, hbm_bytes, ops, l1_bytes, sms, note=None):
    """Both floors of a launch (or step): DRAM bytes against the measured copy bandwidth,
    FP32 operations against the ALU peak (no FMA on this path), the on-chip bytes
    beside them.  `bound` names the floor that is higher, the roofline that binds."""
    peak_gbs, peak_src = hbm_peak()
    peak_tops = sms * 128 * SM_MAX_MHZ * 1e6 / 1e12
    t = ms / 1e3
    hbm = {"achieved": hbm_bytes / t / 1e9, "peak": peak_gbs, "unit": "GB/s", "frac": hbm_bytes / t / 1e9 / peak_gbs,
           "floor_ms": hbm_bytes / (peak_gbs * 1e9) * 1e3, "bytes": int(hbm_bytes), "peak_basis": peak_src}
    alu = {"achieved": ops / t / 1e12, "peak": peak_tops, "unit": "TFLOP/s", "frac": ops / t / 1e12 / peak_tops,
           "floor_ms": ops / (peak_tops * 1e12) * 1e3, "ops": int(ops),
           "peak_basis": f"{sms} SMs x 128 FP32 lanes x {SM_MAX_MHZ:.0f} MHz"}
    out = {"bound": "hbm" if hbm["floor_ms"] >= alu["floor_ms"] else "alu"}
    top = hbm if out["bound"] == "hbm" else alu
    out.update({k: top[k] for k in ("achieved", "peak", "unit", "frac")})
    out["hbm"], out["alu"] = hbm, alu
    if l1_bytes is not None:
        out["l1_bytes"] = int(l1_bytes)
        out["l1_frac"] = l1_bytes / t / (sms * 128 * SM_MAX_MHZ * 1e6)
    if note:
        out["note"] = note
    return out


def sphere_ops(counts, L, chunked=True, in_bytes=16):
    """FP32 operations and on-chip bytes of a sphere query launch from its work counts:
    a root box test per sphere (15 ops, 16 bytes in), a descent and leaf box test per
    near sphere (L + 15 ops, 32 + 4 L bytes), then either the chunk walk (15 ops and 32
    bytes per chunk box, 9 ops and 12 bytes per point scanned) or Alg. 3's plain scan
    (9 ops and 12 bytes per point)."""
    c = [int(x) for x in counts] + [0] * (8 - len(counts))
    # with the distance-bound grid: a lookup (about 20 operations, 2 bytes) per sphere
    # that reaches the cloud's box, and only the undecided ones descend
    desc = c[1] - c[7]
    ops = c[0] * 15 + c[6] * 20 + desc * (L + 15)
    byt = c[0] * in_bytes + c[6] * 2 + desc * (32 + 4 * L)
    if chunked:
        return ops + c[4] * 15 + c[5] * 9, byt + c[4] * 32 + c[5] * 12
    return ops + c[3] * 9, byt + c[3] * 12


def bench_clearance(capt, torch, dev, stream, pts, arm, steps, sms):
    """The differentiable clearance workload: 16,384 trajectories x 32 waypoints x 60
    spheres, forward (distances, argmin, hinge cost) and backward, inputs (377 MB of
    centres) larger than L2.  The forward runs on the nearest-candidate lists (built
    over the distance-bound grid, build times reported) in the launch configuration the
    autotuner picks; the paper's path (descent and full set scan) is timed beside it."""
    import oracle
    ctree = capt.capt_build(pts, 0.0, R_MAX)
    capt.capt_upload(ctree, dev.index)
    T, Wn = 16384, 32
    q = W.random_trajectories(T, Wn, 1003)
    c_host = W.fk_centers(arm, q.reshape(-1, 7)).reshape(T, Wn, SPHERES, 3)
    c = torch.from_numpy(c_host).to(dev)
    r = torch.from_numpy(arm.sphere_radius.copy()).to(dev)
    g = torch.ones(T, device=dev)
    m = T * Wn * SPHERES
    L = capt.capt_stats(ctree)["depth"]
    cost, d, am = capt.capt_clearance_fwd(ctree, c, r, 0.01)
    grad = torch.empty_like(c)

    def run_fwd():
        return time_events(torch, lambda: capt.capt_clearance_fwd(ctree, c, r, 0.01, cost, d, am), steps, stream)

    # the paper's path: every near sphere descends and scans its leaf set
    capt.capt_set_launch_cfg(ctree, capt.CAPT_KERNEL_CLEARANCE, 16, 2, 0, 0, 0, 0)
    for _ in range(3):
        capt.capt_clearance_fwd(ctree, c, r, 0.01, cost, d, am)
    paper_ms = run_fwd()
    d_paper, am_paper = d.clone(), am.clone()
    paper_counts = [int(x) for x in capt.capt_count_clearance_work(ctree, c).cpu().numpy()]
    # the nearest-candidate lists
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    capt.capt_build_grid(ctree, GRID_CELLS)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    capt.capt_build_near_lists(ctree)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    st = capt.capt_stats(ctree)
    cfg, _ = capt.capt_autotune_clearance(ctree, c, r, 0.01)
    for _ in range(3):
        capt.capt_clearance_fwd(ctree, c, r, 0.01, cost, d, am)
        capt.capt_clearance_bwd(ctree, c, r, d, am, g, 0.01, grad)
    fwd_ms = run_fwd()
    bwd_ms = time_events(torch, lambda: capt.capt_clearance_bwd(ctree, c, r, d, am, g, 0.01, grad), steps, stream)
    same = bool(torch.equal(d, d_paper)) and bool(torch.equal(am, am_paper))
    counts = [int(x) for x in capt.capt_count_clearance_work(ctree, c).cpu().numpy()]
    # per sphere a box test (15 ops, 12 bytes); per near sphere with a list a cell lookup
    # (about 12 ops, 8 bytes) and 9 ops per list entry (4 + 16 bytes); per fallback sphere
    # a descent and leaf box test (L + 15 ops) and 9 ops per point of its set
    ops = counts[0] * 15 + counts[5] * 12 + counts[6] * 9 + counts[7] * (L + 15) + counts[3] * 9
    l1 = counts[0] * 12 + counts[5] * 8 + counts[6] * 20 + counts[7] * (32 + 4 * L) + counts[4] * 48
    paper_ops = paper_counts[0] * 15 + paper_counts[1] * (L + 15) + paper_counts[3] * 9
    paper_l1 = paper_counts[0] * 12 + paper_counts[1] * (32 + 4 * L) + paper_counts[4] * 48
    fwd_bytes = m * (12 + 4 + 4) + T * 4          # centres in; distance and argmin out; cost
    bwd_bytes = m * (12 + 4 + 4 + 12) + T * 4      # centres, distance, argmin in; gradient out
    # parity sample: the first 8 trajectories against the oracle's FP64 nearest distance
    k = 8
    ocost, od, _ = oracle.clearance64(pts, c_host[:k], arm.sphere_radius, R_MAX, 0.01, want_grad=False)
    derr = float(np.abs(d[:k].cpu().numpy().astype(np.float64) - od).max())
    cerr = float(np.abs(cost[:k].cpu().numpy().astype(np.float64) - ocost).max())
    return {"trajectories": T, "waypoints": Wn, "spheres": m, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
            "fwd_spheres_per_s": m / (fwd_ms / 1e3), "fwd_bwd_spheres_per_s": m / ((fwd_ms + bwd_ms) / 1e3),
            "launch_cfg": cfg,
            "near_lists": {"grid_cells": int(np.prod(st["grid_dims"])), "grid_build_ms": (t1 - t0) * 1e3,
                           "lists_build_ms": (t2 - t1) * 1e3, "entries": st["near_entries"],
                           "bytes": st["near_bytes"], "fallback_cells": st["near_fallback_cells"],
                           "same_as_paper_path": same},
            "paper_path": {"fwd_ms": paper_ms, "fwd_spheres_per_s": m / (paper_ms / 1e3),
                           "roofline": roof(paper_ms, fwd_bytes, paper_ops, paper_l1, sms),
                           "points_scanned": paper_counts[3], "points_per_sphere": paper_counts[3] / m},
            "work": {"spheres": counts[0], "near_cloud_box": counts[1], "answered_by_lists": counts[5],
                     "list_entries": counts[6], "fallback_spheres": counts[7],
                     "entries_per_list_sphere": counts[6] / max(counts[5], 1)},
            "roofline_fwd": roof(fwd_ms, fwd_bytes, ops, l1, sms),
            "roofline_bwd": roof(bwd_ms, bwd_bytes, m * 12, None, sms),
            "l2": "inputs larger than L2 (377 MB of centres)",
            "parity_sample": {"trajectories": k, "max_abs_dist_err_vs_fp64": derr, "max_abs_cost_err_vs_fp64": cerr,
                              "within_1e-5": derr <= 1e-5}}


def bench_spheres(capt, torch, dev, stream, tree, c_host, r_host, steps, sms, parity_n, pts):
    """One sphere-query workload on an uploaded tree: autotuned launch, device time with
    L2 flushed before every call, work counts, roofline and an oracle parity sample."""
    import oracle
    m = len(c_host)
    dc, dr = torch.from_numpy(c_host).to(dev), torch.from_numpy(r_host).to(dev)
    fl = torch.empty(m, dtype=torch.uint8, device=dev)
    cfg, _ = capt.capt_autotune_spheres(tree, dc, dr, fl)
    st = capt.capt_stats(tree)
    counts = None if st["full_dropped"] else capt.capt_count_sphere_work(tree, dc, dr).cpu().numpy()
    flush = torch.zeros(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(3):
        capt.capt_query_spheres(tree, dc, dr, fl)
    ms = time_events_flushed(torch, lambda: capt.capt_query_spheres(tree, dc, dr, fl), steps, stream, flush)
    del flush
    got = fl.cpu().numpy()
    k = min(parity_n, m)
    ref = oracle.brute_flags(pts, c_host[:k], r_host[:k], threads=oracle.default_threads())
    out = {"spheres": m, "ms": ms, "sphere_queries_per_s": m / (ms / 1e3), "launch_cfg": cfg,
           "collision_fraction": float(got.mean()), "tree_device_bytes": int(st["device_bytes"]),
           "l2": "flushed before every timed call", "parity_sample_equal": bool(np.array_equal(got[:k], ref)),
           "parity_sample": f"first {k} spheres vs the oracle's FP32 brute force over all {len(pts)} points"}
    if counts is not None:
        ops, l1 = sphere_ops(counts, st["depth"], chunked=cfg["chunk"] != capt.CAPT_SCAN_SETS)
        out["work"] = {"spheres": int(counts[0]), "near_cloud_box": int(counts[1]), "leaf_box_pass": int(counts[2]),
                       "points_scanned_alg3": int(counts[3]), "chunk_boxes": int(counts[4]),
                       "points_scanned_chunked": int(counts[5]), "grid_lookups": int(counts[6]),
                       "decided_by_grid": int(counts[7])}
        out["roofline"] = roof(ms, m * 17, ops, l1, sms)
    return out, got


def bench_uniform(capt, torch, dev, stream, steps, sms):
    """The small uniform workload: 2,000 points in the unit cube, 100,000 spheres."""
    pu = W.uniform_cloud(2000, 1000)
    cu, ru = W.cube_queries(100_000, 1000)
    tu = capt.capt_build(pu, 0.01, 0.08)
    capt.capt_upload(tu, dev.index)
    capt.capt_build_grid(tu, 1 << 20)
    out, _ = bench_spheres(capt, torch, dev, stream, tu, cu, ru, steps, sms, 100_000, pu)
    out["roofline"]["note"] = ("one launch of ~10 us: launch and tail latency dominate; both floors are far "
                               "below the measured time")
    return out


def bench_room(capt, torch, dev, stream, steps, sms):
    """The large room cloud: 200,000 unfiltered points, 4,194,304 spheres, host build
    timed, then the same queries on the compact (de-duplicated) sets."""
    pr = W.room_cloud(1004)
    t0 = time.perf_counter()
    tr = capt.capt_build(pr, 0.02, 0.10)
    build_ms = (time.perf_counter() - t0) * 1e3
    st = capt.capt_stats(tr)
    capt.capt_upload(tr, dev.index)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    capt.capt_build_grid(tr, GRID_CELLS)
    grid_ms = (time.perf_counter() - t0) * 1e3
    cr, rr = W.room_queries(1 << 22, 1004)
    rep, f_rep = bench_spheres(capt, torch, dev, stream, tr, cr, rr, steps, sms, 8192, pr)
    gst = capt.capt_stats(tr)
    rep.update({"host_build_ms": build_ms, "host_build_threads": int(st["build_threads"]), "grid_build_ms": grid_ms,
                "grid": {"dims": gst["grid_dims"], "cell_m": gst["grid_cell"]},
                "total_afforded": int(st["total_afforded"]), "max_set": int(st["max_set"]),
                "mean_set": st["total_afforded"] / st["n_leaves"]})
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    capt.capt_compact(tr, drop_full=True)
    torch.cuda.synchronize(dev)
    cms = (time.perf_counter() - t0) * 1e3
    comp, f_comp = bench_spheres(capt, torch, dev, stream, tr, cr, rr, steps, sms, 8192, pr)
    # the compact sets' scan has no work counter; the bytes floor is the same
    comp["roofline"] = roof(comp["ms"], (1 << 22) * 17, 0, None, sms,
                            note="HBM floor of the sphere inputs and flags only; the scan work is not counted "
                                 "for the compact sets")
    comp.update({"compact_ms": cms, "compact_entries": int(capt.capt_stats(tr)["compact_entries"]),
                 "flags_equal_replicated": bool(np.array_equal(f_rep, f_comp))})
    return {"replicated": rep, "compact": comp}


def extra_workloads(capt, torch, dev, stream, pts, arm, args):
    res = {}
    # depth frame -> tree, host and device (the paper's Table III setting: a 640 x 480
    # frame of 307,200 points, r_filter 1 / 1.5 / 2 cm, r_min 1.5 cm, r_max 8 cm)
    frame = W.depth_frame()
    df = torch.from_numpy(frame).to(dev)
    rows = []
    for rf in (0.01, 0.015, 0.02):
        kept = capt.sfc_filter(frame, rf)
        t0 = time.perf_counter()
        tr_h = capt.capt_build(frame[kept], 0.015, 0.08)
        hb = (time.perf_counter() - t0) * 1e3
        kd = capt.sfc_filter_device(df, rf)
        same = bool(np.array_equal(kd.cpu().numpy().astype(np.uint32), kept))
        rows.append({"r_filter": rf, "kept": int(len(kept)), "host_filter_ms": host_filter_ms(capt, frame, rf),
                     "host_build_ms": hb, "device_filter_ms": device_filter_ms(capt, frame, rf, reps=3),
                     "device_build_ms": device_build_ms(capt, frame[kept], 0.015, 0.08, reps=3),
                     "device_filter_equals_host": same,
                     "device_frame_to_tree_ms": frame_to_tree_ms(capt, df, rf, 0.015, 0.08),
                     "total_afforded": int(capt.capt_stats(tr_h)["total_afforded"])})
    res["depth_frame_to_tree"] = {"points": int(len(frame)), "rows": rows}
    # room: filter at 2 cm (host and device), device build; the cloud relabelled along
    # the Z-order curve (same point set, same flags)
    pr = W.room_cloud(1004)
    res["room_filter_2cm"] = {"points": len(pr), "host_ms": host_filter_ms(capt, pr, 0.02),
                              "device_ms": device_filter_ms(capt, pr, 0.02, reps=3)}
    res["room_device_build_ms"] = device_build_ms(capt, pr, 0.02, 0.10, reps=3)
    order = capt.capt_morton_order(pr)
    ts = capt.capt_build(pr[order], 0.02, 0.10)
    capt.capt_upload(ts, dev.index)
    cr, rr = W.room_queries(1 << 22, 1004)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    res["room200k_zorder"], _ = bench_spheres(capt, torch, dev, stream, ts, cr, rr, 10, sms, 4096, pr[order])
    return res


if __name__ == "__main__":
    main()
