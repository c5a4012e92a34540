#!/usr/bin/env python
"""Throughput of the batched Active-SLAM environment step on GB300.

Workload (default): 750 envs, each a 256x256 grid at 0.05 m with 20-40
rectangles and 5-15 discs, 360 beams over 360 deg, 12 m range, Gaussian range
noise sigma = 0.01 m, int16 log-odds, 1000 steps of random (v, w) actions
and a synthetic uncertainty signal U_t (composite reward, Eq. 7-17).

A "step" is one call of the whole path (action integration, raycast, log-odds
update, reward, observation) for all envs: two kernel launches (sensing,
which also integrates the actions, then the persistent update; one for the
3-D variant).  Inputs (all steps' actions and U_t) are resident in HBM
before timing; L2 is flushed (256 MiB write) between timed steps, each step
is timed with its own CUDA event pair on the launching stream, and the
library's own events time each kernel in a separate pass.

The default line also carries `batched_4096`: the batched uneven form
(4096 envs, map sides {128,256,384,512}, beams {180,360,720}), autotuned,
timed both as plain launches and as replays of the captured CUDA graph, with
its step's algorithmic bytes against the measured HBM peak; and
`cpu_baseline`: the oracle on one thread and with a step's envs spread over
every host core.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the job holds N x 750 envs and every rank steps its
contiguous, cost-balanced share (weak scaling, no collective on the data
path); the max over ranks of the timed total is used.
`--impl reference` times the CPU oracle (the plain C definition of the
method) on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s and ray-cells/s at 750/4096 envs on 1 GB300; % of HBM roofline"
UNIT = "env-steps/s"
WORKLOAD = dict(workload="paper_scale: 750 envs x 256^2 cells @0.05 m, 360 beams, 12 m, sigma 0.01 m",
                envs=750, map_side=256, beams=360, res_m=0.05, r_max_m=12.0, noise_sigma_m=0.01,
                reward="composite Eq. 7-17", steps_of_actions="random (v,w)",
                l2="flushed (256 MiB write) between timed steps")
KERNEL_SOURCES = {"2d": ["paper_2603_25834_gb300/csrc/step2d.cu",
                         "paper_2603_25834_gb300/csrc/walk2d.cuh",
                         "paper_2603_25834_gb300/csrc/aslam_internal.cuh",
                         "paper_2603_25834_gb300/csrc/env_common.cuh",
                         "include/aslam.h"],
                  "3d": ["paper_2603_25834_gb300/csrc/step3d.cu",
                         "paper_2603_25834_gb300/csrc/aslam_internal.cuh",
                         "paper_2603_25834_gb300/csrc/env_common.cuh",
                         "include/aslam.h"]}


def traffic_file(kernel, workload):
    return os.path.join(ROOT, "profiles", "%s_%s_traffic.json" % (kernel.replace("_kernel", ""),
                                                                   workload))


def strip_comments(src):
    """C/C++ source without its comments and blank lines (string and
    character literals kept), so that a comment edit leaves the hash of an
    unchanged kernel alone."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(l.rstrip() for l in "".join(out).splitlines() if l.strip())


def kernel_hash(dims="2d"):
    """The kernel sources' hash (comments removed): a traffic record taken
    with another hash describes other code and is not reported."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[dims]:
        with open(os.path.join(ROOT, f)) as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(inputs, n_envs, steps, threads=1, seed_actions=2026):
    """Env-steps/s of the CPU oracle on the first n_envs envs, its step's
    independent envs spread over `threads` host threads (OpenMP)."""
    import oracle
    from paper_2603_25834_gb300 import synth
    used = oracle.set_threads(threads)
    try:
        sub = synth.subset(inputs, list(range(n_envs)))
        ob = oracle.OracleBatch2D(sub, r_max=12.0, sigma=0.01)
        acts = synth.random_actions(steps, n_envs, seed_actions)
        u = synth.random_uncertainty(steps, n_envs, seed_actions + 1)
        t0 = time.perf_counter()
        rc = 0
        for s in range(steps):
            o = ob.step(acts[s], u[s])
            rc += int(o["ray_cells"].sum())
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return n_envs * steps / dt, rc / dt, dt, used


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2603_25834_gb300 import synth
    import oracle
    # bounded sample of the same workload: four envs per host core per step,
    # the step's envs spread over every core (OpenMP)
    cores = host_cores()
    used = oracle.set_threads(cores)
    n_sample = 4 * used
    inp = synth.paper_scale(E=n_sample)
    ob = oracle.OracleBatch2D(inp, r_max=12.0, sigma=0.01)
    total = args.warmup + args.steps
    acts = synth.random_actions(total, n_sample, 2026)
    u = synth.random_uncertainty(total, n_sample, 2027)
    for s in range(args.warmup):
        ob.step(acts[s], u[s])
    t0 = time.perf_counter()
    rc = 0
    for s in range(args.warmup, total):
        rc += int(ob.step(acts[s], u[s])["ray_cells"].sum())
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    val = n_sample * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i16+f32", "data": "synthetic", "config": WORKLOAD,
        "ray_cells_per_s": rc / dt,
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": "%d of the 750 envs per step (4 per core), %d steps, the envs "
                                   "of a step spread over %d threads" % (n_sample, args.steps, used)},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def timed_steps(batch, acts, uu, W, K, reward, obs, flush, stream, dev, counters=None,
                clocks=None):
    """K steps (after W untimed ones), each timed with its own CUDA event pair
    on the launching stream, L2 flushed before each; returns the summed ms.
    `counters` (ray_cells, gt_cells device views and accumulators) sums the
    exact cell counts of every timed step on the device."""
    for s in range(W):
        batch.step_fused(acts[s], uu[s], reward, obs)
    starts = [torch_event() for _ in range(K)]
    ends = [torch_event() for _ in range(K)]
    torch_sync(dev)
    if clocks is not None:
        clocks.start()
        time.sleep(0.1)
    for k in range(K):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        batch.step_fused(acts[W + k], uu[W + k], reward, obs)
        ends[k].record(stream)
        if counters is not None:
            rc, gc, rc_acc, gc_acc = counters
            rc_acc += rc.sum()
            gc_acc += gc.sum()
    torch_sync(dev)
    clk = clocks.stop() if clocks is not None else None
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), clk


def graph_steps(batch, acts, uu, W, n, reward, obs, flush, dev):
    """Capture one step into a CUDA graph and time n replays (inputs copied
    into the captured buffers before each, outside the timed region)."""
    import torch
    gstream = torch.cuda.Stream(dev)
    abuf = acts[0].clone()
    ubuf = uu[0].clone()
    with torch.cuda.stream(gstream):
        batch.capture_graph(abuf, ubuf, reward, obs, stream=gstream)
    torch_sync(dev)
    tot = 0.0
    with torch.cuda.stream(gstream):
        for k in range(n):
            abuf.copy_(acts[W + k])
            ubuf.copy_(uu[W + k])
            flush.fill_(k & 0xFF)
            e0, e1 = torch_event(), torch_event()
            e0.record(gstream)
            batch.graph_step(stream=gstream)
            e1.record(gstream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
    torch_sync(dev)
    return tot / n


def kernel_split(batch, acts, uu, W, n, reward, obs, flush, dev):
    """Per-kernel device time from the library's own events (a separate pass:
    the events between kernels serialise them)."""
    batch.profile_begin(n)
    for k in range(n):
        flush.fill_(k & 0xFF)
        batch.step_fused(acts[W + k], uu[W + k], reward, obs)
    torch_sync(dev)
    return batch.profile_end()


def torch_event():
    import torch
    return torch.cuda.Event(enable_timing=True)


def torch_sync(dev):
    import torch
    torch.cuda.synchronize(dev)


def step_kernel_bytes(E, b_max, Bsum, rc_step, gt_step):
    """Algorithmic bytes of one 2-D step per kernel and in total (per-unit
    figures x units of one launch): each cell an update walk visits is an
    int16 read + write (4 B); each ground-truth cell a sensing walk visits is
    1 bit of the packed world (1/8 B); per beam a 4 B range and a 4 B walk
    code written by the sensing and read by the update; per env the
    observation row (b_max + 2) x 4 B and 24 B of pose, action and reward,
    and 96 B of integration state and the start-of-step header."""
    io_env = E * (b_max + 2) * 4 + E * 24
    kb = {"sense2d_kernel": gt_step / 8 + Bsum * 8 + E * 96,
          "update2d_kernel": rc_step * 4 + Bsum * 4 + io_env}
    step = rc_step * 4 + gt_step / 8 + Bsum * 4 + io_env
    return kb, step


def batched_record(args, world, rank, dev, peak):
    """The batched uneven form at its full size (4096 envs per GPU, map sides
    {128, 256, 384, 512}, beams {180, 360, 720}): the persistent update launch
    and the captured CUDA graph of the whole step, autotuned, each timed over
    K steps; the step's ray-cell bytes against the HBM peak."""
    import torch
    from paper_2603_25834_gb300 import aslam, shard, synth
    E_all = 4096 * world
    side, nb = synth.uneven_shapes(E_all)
    lo, hi = shard.env_range(shard.env_cost(side, side, nb), world, rank)
    inp = synth.uneven(E=E_all, envs=range(lo, hi))
    E = hi - lo
    batch = aslam.Batch2D(inp, device=dev, reward_mode=aslam.REWARD_COMPOSITE, r_max_m=12.0,
                          noise_sigma_m=0.01, env_base=lo)
    tuned = batch.autotune()
    K, W = args.steps, args.warmup
    acts = torch.from_numpy(synth.random_actions(K + W, E_all, 7)[:, lo:hi].copy()).to(dev)
    uu = torch.from_numpy(synth.random_uncertainty(K + W, E_all, 8)[:, lo:hi].copy()).to(dev)
    reward = torch.empty(E, device=dev)
    obs = torch.empty(E, batch.b_max + 2, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = batch.state()
    rc_acc = torch.zeros((), dtype=torch.int64, device=dev)
    gc_acc = torch.zeros((), dtype=torch.int64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    plain_ms, _ = timed_steps(batch, acts, uu, W, K, reward, obs, flush, stream, dev,
                              counters=(st["ray_cells"], st["gt_cells"], rc_acc, gc_acc))
    plain_ms = shard.max_over_ranks(plain_ms, dev) / K
    rc_step = int(rc_acc.item()) / K
    gt_step = int(gc_acc.item()) / K
    Kg = min(K, 200)
    g_ms = shard.max_over_ranks(graph_steps(batch, acts, uu, W, Kg, reward, obs, flush, dev), dev)
    kms, ns = kernel_split(batch, acts, uu, W, min(K, 100), reward, obs, flush, dev)
    kb, step_b = step_kernel_bytes(E, batch.b_max, int(batch.ray_off[-1]), rc_step, gt_step)
    batch.sync_status()
    rc_all = shard.sum_over_ranks(rc_step, dev)
    step_all = shard.sum_over_ranks(step_b, dev)
    kernels = {k: {"ms_per_launch": v / ns,
                   "achieved_gbs": kb[k] / (v / ns / 1e3) / 1e9 if k in kb else None,
                   "frac": kb[k] / (v / ns / 1e3) / 1e9 / peak if k in kb else None}
               for k, v in kms.items()}
    del batch
    return {
        "workload": "uneven: %d envs per GPU, sides {128,256,384,512} @0.05 m, beams "
                    "{180,360,720}, 12 m, sigma 0.01 m, composite reward" % E,
        "envs": E_all, "mean_beams": float(nb.mean()),
        "mean_cells": float((side.astype(np.int64) ** 2).mean()),
        "autotuned": {"threads_per_cta": tuned[0], "window_cells": tuned[1]},
        "ray_cells_per_step": rc_all, "bytes_per_step": step_all,
        "graph": {"ms_per_step": g_ms, "value": E_all / (g_ms / 1e3), "unit": UNIT,
                  "ray_cells_per_s": rc_all / (g_ms / 1e3),
                  "achieved_gbs": step_all / (g_ms / 1e3) / 1e9,
                  "frac": step_all / (g_ms / 1e3) / 1e9 / peak, "steps": Kg},
        "plain": {"ms_per_step": plain_ms, "value": E_all / (plain_ms / 1e3), "unit": UNIT,
                  "ray_cells_per_s": rc_all / (plain_ms / 1e3),
                  "achieved_gbs": step_all / (plain_ms / 1e3) / 1e9,
                  "frac": step_all / (plain_ms / 1e3) / 1e9 / peak, "steps": K},
        "kernels": kernels,
        "frac_target": 0.5,
        "note": "frac = the step's algorithmic bytes (4 B per ray cell, 1/8 B per ground-truth "
                "cell, ranges, observation, pose/action/reward) / step time / measured hbm_gbs",
        "l2": "flushed (256 MiB write) between timed steps",
    }


def bench_diff(args):
    """Differentiable form: 1024 envs x 256^2 fp32 log-odds, 360 beams x 64
    samples of 0.05 m; a step is one Gauss-Newton correction (5 iterations)
    of every env from N(0, 5 cm, 0.02 rad) perturbed poses."""
    import torch
    from paper_2603_25834_gb300 import soft, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    E, W, B, K, iters = 1024, 256, 360, 64, 5
    inp = synth.paper_scale(E=E, W=W, B=8, seed=synth.BASE_SEED + 300_000)
    L = torch.from_numpy(synth.logodds_maps(inp)).to(dev)
    true = torch.from_numpy(np.ascontiguousarray(inp.spawn[:, 0, :])).to(dev)
    cfg = soft.soft_config(E, W, W, B, K)
    z = soft.soft_range_fwd(cfg, L, true)
    steps, warm = args.steps if args.steps != 1000 else 50, args.warmup
    starts = [torch.from_numpy(synth.perturb_poses(inp.spawn[:, 0, :], 90 + k)).to(dev)
              for k in range(steps + warm)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for k in range(warm):
        soft.gn_correct(cfg, L, starts[k], z, iters)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, n):
        tot = 0.0
        for k in range(n):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / n

    clocks = ClockSampler(dev.index)
    torch.cuda.synchronize(dev)
    clocks.start()
    ms_gn = timed(lambda k: soft.gn_correct(cfg, L, starts[warm + k], z, iters), steps)
    clk = clocks.stop()
    ms_fwd = timed(lambda k: soft.soft_range_fwd(cfg, L, starts[k]), min(steps, 20))
    gr = torch.ones(E, B, device=dev)
    gmap = torch.zeros_like(L)
    ms_bwd = timed(lambda k: soft.soft_range_bwd(cfg, L, starts[k], gr), min(steps, 20))
    # FP32 operations per sample in the forward-mode sweep, counted from the
    # kernel source: bilinear 34, sigmoid 5, tangents and accumulators 35.
    flops = float(E) * B * K * (iters + 1) * 74
    peak_fp32 = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = flops / (ms_gn / 1e3) / 1e12
    pg, cov, u = soft.gn_correct(cfg, L, starts[0], z, iters)
    conv = float(((pg - true).abs() < 2e-3).all(dim=1).float().mean())
    line = {
        "metric": "env Gauss-Newton corrections/s (differentiable form)",
        "value": E / (ms_gn / 1e3), "unit": "env-GN-steps/s", "n_gpus": 1, "steps": steps,
        "warmup": warm, "ms_per_step": ms_gn, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "diff: 1024 envs x 256^2 fp32 log-odds, 360 beams x 64 samples "
                               "@0.05 m, 5 GN iterations from N(0, 5 cm, 0.02 rad)",
                   "l2": "flushed (256 MiB write) between timed steps",
                   "converged_frac": conv},
        "soft_fwd_ms": ms_fwd, "soft_bwd_ms": ms_bwd,
        "rays_per_s_gn": E * B * (iters + 1) / (ms_gn / 1e3),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                     "frac": achieved / peak_fp32, "traffic": None,
                     "peak_kind": "nominal FP32 FMA rate: 152 SMs x 128 lanes x 2 x 2.07 GHz",
                     "kernel": "gn_kernel"},
        "gpu_launches": steps, "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def bench_csm(args):
    """Batched correlative scan matching (Sec. III-D) of 750 paper-scale envs
    whose maps were built by 30 plain steps, from predicted poses perturbed
    by N(0, 6 cm, 6 cm, 0.02 rad), 11 x 11 x 11 candidates."""
    import torch
    from paper_2603_25834_gb300 import aslam, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    E, n_xy, n_th = args.envs, 5, 5
    inp = synth.paper_scale(E=E)
    batch = aslam.Batch2D(inp, device=dev, r_max_m=12.0, noise_sigma_m=0.01)
    acts = torch.from_numpy(synth.random_actions(30, E, 7)).to(dev)
    for s in range(30):
        batch.step(acts[s])
    st = batch.state()
    true = torch.stack([st["x"], st["y"], st["th"]], dim=1).cpu().numpy()
    steps = args.steps if args.steps != 1000 else 200
    preds = [torch.from_numpy(synth.perturb_poses(true, 100 + k, sigma=(0.06, 0.06, 0.02))
                              .astype(np.float32)).to(dev) for k in range(steps + args.warmup)]
    for k in range(args.warmup):
        batch.csm(preds[k], n_xy=n_xy, n_th=n_th)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(dev.index)
    torch.cuda.synchronize(dev)
    clocks.start()
    tot = 0.0
    for k in range(steps):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.csm(preds[args.warmup + k], n_xy=n_xy, n_th=n_th)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = tot / steps
    z = st["z"].cpu().numpy()
    n_ret = int((z < 12.0).sum())
    cand = (2 * n_xy + 1) ** 2 * (2 * n_th + 1)
    lookups = float(n_ret) * cand
    # integer operations per lookup, counted from the kernel source: two
    # adds for the shifted cell, two compares, the index, the load, the add
    ops = lookups * 7
    peak = 152 * 128 * 2.07e9 / 1e12
    achieved = ops / (ms / 1e3) / 1e12
    line = {
        "metric": "env scan matches/s (batched correlative scan matching)",
        "value": E / (ms / 1e3), "unit": "env-matches/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i16/u8+i32", "data": "synthetic",
        "config": {"workload": "csm: %d envs x 256^2 maps after 30 steps, 360 beams, 11x11 cells "
                               "x 11 rotations of 0.01 rad" % E,
                   "l2": "flushed (256 MiB write) between timed calls"},
        "lookups_per_s": lookups / (ms / 1e3),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_kind": "nominal 32-bit integer lane rate: 152 SMs x 128 lanes x 2.07 GHz",
                     "kernel": "csm2d_kernel"},
        "gpu_launches": steps, "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_scale",
                    choices=["paper_scale", "paper_sensor", "uneven", "diff", "3d", "csm"])
    ap.add_argument("--envs", type=int, default=750)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 4096-env batched record of the default workload")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: default/tuned)")
    ap.add_argument("--window", type=int, default=0, help="shared window side (0: default/tuned)")
    ap.add_argument("--u-mode", default="caller",
                    choices=["caller", "scanmatch", "fixedlag", "fixedlag_weighted", "fixedlag_gn",
                             "fixedlag_weighted_gn"],
                    help="U_t from the caller (a synthetic signal), the in-step scan-match "
                         "covariance, or the in-step SLAM backbone (CSM + fixed-lag window; "
                         "_weighted: confidence-weighted map update)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "diff":
        return bench_diff(args)
    if args.workload == "csm":
        return bench_csm(args)

    import torch
    import torch.distributed as dist
    from paper_2603_25834_gb300 import aslam, shard, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)

    # Weak scaling: E envs per GPU, world * E in the whole job; each rank
    # builds and steps its contiguous, cost-balanced share of the global set
    # (env_base = first global index keeps every env's noise stream).
    cfg_kw = dict(r_max_m=12.0, noise_sigma_m=0.01)
    if args.workload == "3d":
        E_all = (args.envs if args.envs != 750 else 512) * world
        lo, hi = shard.env_range(np.ones(E_all, np.int64), world, rank)
        inp = synth.voxel_batch(E=E_all, envs=range(lo, hi))
        cfg_kw = dict(r_max_m=20.0, noise_sigma_m=0.01, n_rings=16)
        workload = dict(workload="3d: %d envs per GPU x 128x128x32 voxels @0.1 m (floor, boxes, "
                                 "pillars), 16 rings x 512 azimuths over +-15 deg at 0.5 m, 20 m, "
                                 "sigma 0.01 m, CUDA graph" % (E_all // world),
                        envs=E_all, res_m=0.1, r_max_m=20.0, noise_sigma_m=0.01,
                        reward="composite Eq. 7-17", l2="flushed (256 MiB write) between timed steps")
    elif args.workload == "uneven":
        E_all = (args.envs if args.envs != 750 else 4096) * world
        side, nb = synth.uneven_shapes(E_all)
        lo, hi = shard.env_range(shard.env_cost(side, side, nb), world, rank)
        inp = synth.uneven(E=E_all, envs=range(lo, hi))
        workload = dict(workload="uneven: %d envs per GPU, sides {128,256,384,512} @0.05 m, beams "
                                 "{180,360,720}, 12 m, sigma 0.01 m, persistent launch, CUDA graph"
                                 % (E_all // world),
                        envs=E_all, res_m=0.05, r_max_m=12.0, noise_sigma_m=0.01,
                        reward="composite Eq. 7-17", l2="flushed (256 MiB write) between timed steps",
                        mean_beams=float(nb.mean()),
                        mean_cells=float((side.astype(np.int64) ** 2).mean()))
    elif args.workload == "paper_sensor":
        # the paper's LiDAR (Sec. IV-A): 128 rays over the front 180 degrees,
        # 0.1-10 m, two decimal places; v in (0, 0.4) (Eq. 4)
        E_all = args.envs * world
        lo, hi = shard.env_range(np.ones(E_all, np.int64), world, rank)
        inp = synth.paper_scale(E=E_all, B=128, envs=range(lo, hi))
        cfg_kw = dict(r_max_m=10.0, noise_sigma_m=0.01, fov_rad=math.pi, r_min_m=0.1,
                      range_decimals=2, v_max=0.4)
        workload = dict(workload="paper_sensor: %d envs per GPU x 256^2 cells @0.05 m, 128 beams "
                                 "over the front 180 deg, 0.1-10 m, 2 decimals, sigma 0.01 m, "
                                 "v <= 0.4 m/s" % (E_all // world),
                        envs=E_all, res_m=0.05, r_max_m=10.0, r_min_m=0.1, range_decimals=2,
                        noise_sigma_m=0.01, reward="composite Eq. 7-17",
                        l2="flushed (256 MiB write) between timed steps")
    else:
        E_all = args.envs * world
        lo, hi = shard.env_range(np.ones(E_all, np.int64), world, rank)
        inp = synth.paper_scale(E=E_all, envs=range(lo, hi))
        workload = dict(WORKLOAD, envs=E_all)
    E = hi - lo
    cfg_kw["env_base"] = lo
    if args.u_mode != "caller" and args.workload == "3d":
        raise SystemExit("an in-step --u-mode is 2-D only")
    if args.u_mode == "scanmatch":
        cfg_kw["u_mode"] = aslam.U_SCANMATCH
        workload = dict(workload,
                        u_t="in-step scan-match covariance (64 samples of one cell, Eq. 5-6)")
    elif args.u_mode.startswith("fixedlag"):
        cfg_kw["u_mode"] = aslam.U_FIXEDLAG
        cfg_kw["slam_weighted_update"] = int(args.u_mode.startswith("fixedlag_weighted"))
        cfg_kw["slam_gn_iters"] = 2 if args.u_mode.endswith("_gn") else 0
        workload = dict(workload,
                        u_t="in-step SLAM backbone: CSM 11x11x11%s + 8-pose fixed-lag window, "
                            "3 GN iterations (Eq. 5-6)%s"
                            % (" + 2 scan-to-map Gauss-Newton steps of the soft range model"
                               if args.u_mode.endswith("_gn") else "",
                               ", confidence-weighted map update"
                               if args.u_mode.startswith("fixedlag_weighted") else ""))
    batch = aslam.Batch2D(inp, device=dev, reward_mode=aslam.REWARD_COMPOSITE,
                          threads_per_cta=args.threads, window_cells=args.window, **cfg_kw)
    tuned = None
    if not args.no_autotune and not args.threads and not args.window:
        tuned = batch.autotune()
    K, W = args.steps, args.warmup
    v_max = cfg_kw.get("v_max", 0.5)
    acts = torch.from_numpy(synth.random_actions(K + W, E_all, 7, v_max=v_max)[:, lo:hi].copy()).to(dev)
    uu = torch.from_numpy(synth.random_uncertainty(K + W, E_all, 8)[:, lo:hi].copy()).to(dev)
    reward = torch.empty(E, device=dev)
    obs = torch.empty(E, batch.b_max + 2, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc_acc = torch.zeros((), dtype=torch.int64, device=dev)
    gc_acc = torch.zeros((), dtype=torch.int64, device=dev)
    st = batch.state()
    clocks = ClockSampler(dev.index)
    if world > 1:
        dist.barrier()
    total_ms, clk = timed_steps(batch, acts, uu, W, K, reward, obs, flush, stream, dev,
                                counters=(st["ray_cells"], st["gt_cells"], rc_acc, gc_acc),
                                clocks=clocks)
    if world > 1:
        dist.barrier()
    kernel_ms, prof_steps = kernel_split(batch, acts, uu, W, min(K, 100), reward, obs, flush, dev)
    ray_cells = int(rc_acc.item())
    gt_cells = int(gc_acc.item())
    total_ms_max = shard.max_over_ranks(total_ms, dev)
    batch.sync_status()

    # ---- graph-captured replay of the same step (reported beside) ----
    gk = min(K, 200)
    g_ms = graph_steps(batch, acts, uu, W, gk, reward, obs, flush, dev)

    # ---- end to end through the public API with host buffers ----
    K2 = min(args.e2e_steps, K)
    h_acts = torch.from_numpy(synth.random_actions(K2, E_all, 17, v_max=v_max)[:, lo:hi].copy()).pin_memory()
    h_u = torch.from_numpy(synth.random_uncertainty(K2, E_all, 18)[:, lo:hi].copy()).pin_memory()
    h_rew = torch.empty(K2, E).pin_memory()
    h_obs = torch.empty(K2, E, batch.b_max + 2).pin_memory()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e2e_ms = 0.0
    for k in range(K2):
        flush.fill_(k & 0xFF)
        e0, e1 = torch_event(), torch_event()
        e0.record(stream)
        # the C-ABI call with host buffers: copies in, step, copies out
        batch.step_host(h_acts[k], h_u[k], h_rew[k], h_obs[k], stream=stream)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = shard.max_over_ranks(e2e_ms, dev)
    h2d = shard.sum_over_ranks(E * 2 * 4 + E * 4, dev)
    d2h = shard.sum_over_ranks(E * 4 + E * (batch.b_max + 2) * 4, dev)
    ray_cells_all = shard.sum_over_ranks(ray_cells, dev)
    b_max, Bsum, n_cells = batch.b_max, int(batch.ray_off[-1]), int(batch.map_off[-1])
    del batch
    peak, peak_kind = measured_peaks()

    # ---- the batched uneven form at 4096 envs per GPU, beside the headline ----
    batched = None
    if args.workload == "paper_scale" and not args.no_batched and args.u_mode == "caller":
        batched = batched_record(args, world, rank, dev, peak)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    value = E_all * K / (total_ms_max / 1e3)
    ms_step = total_ms_max / K
    rc_step, gt_step = ray_cells / K, gt_cells / K
    dims = "3d" if args.workload == "3d" else "2d"
    if dims == "3d":
        io_env = E * (b_max + 2) * 4 + E * 24
        kbytes = {"step3d_kernel": rc_step * 4 + gt_step / 8 + Bsum * 4 + io_env}
        step_bytes = kbytes["step3d_kernel"]
    else:
        kbytes, step_bytes = step_kernel_bytes(E, b_max, Bsum, rc_step, gt_step)
        if args.u_mode == "scanmatch":
            # the belief read once per env, the covariance read and written, U written
            kbytes["uq2d_kernel"] = 2 * n_cells + E * (96 + 4)
    kern = max((k for k in kernel_ms if k in kbytes), key=kernel_ms.get)
    k_ms = kernel_ms[kern] / prof_steps
    achieved = kbytes[kern] / (k_ms / 1e3) / 1e9
    kernels = {k: {"ms_per_launch": v / prof_steps, "share": v / sum(kernel_ms.values()),
                   "alg_bytes_per_launch": kbytes.get(k),
                   "achieved_gbs": (kbytes[k] / (v / prof_steps / 1e3) / 1e9
                                    if k in kbytes else None)}
               for k, v in kernel_ms.items()}
    traffic = None
    issue = None
    tf = traffic_file(kern, args.workload)
    if os.path.exists(tf):
        with open(tf) as fh:
            tr = json.load(fh)
        if tr.get("kernel_hash") == kernel_hash(dims) and tr.get("envs") == E:
            traffic = tr.get("dram_bytes_per_launch")
            if tr.get("warp_inst_per_launch"):
                # the kernel's warp instructions (ncu) over the live launch
                # time, against one instruction per scheduler per clock
                n_inst = float(tr["warp_inst_per_launch"])
                mhz = (clk or {}).get("sm_max_mhz") or 2070.0
                ipeak = 152 * 4 * mhz * 1e6
                issue = {"warp_inst_per_launch": n_inst, "achieved": n_inst / (k_ms / 1e3),
                         "peak": ipeak, "unit": "warp-inst/s",
                         "frac": n_inst / (k_ms / 1e3) / ipeak,
                         "peak_kind": "152 SMs x 4 schedulers x max SM clock"}
    cpu = None
    if not args.no_cpu_baseline and args.workload == "paper_scale":
        # the oracle on a bounded sample of the same workload: one thread, and
        # the step's envs spread over every host core (OpenMP)
        n_s, steps_s = 48, 60
        rate1, rcs1, dt1, _ = oracle_rate(inp, n_s, steps_s, threads=1)
        cores = host_cores()
        n_m, steps_m = min(E, 16 * cores), 30
        rate_m, rcs_m, dt_m, used = oracle_rate(inp, n_m, steps_m, threads=cores)
        cpu = {"value": rate_m, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": "first %d of the %d envs x %d steps (%.1f s), the envs of a step spread "
                         "over %d threads; oracle ray-cells/s %.3g" % (n_m, E, steps_m, dt_m, used,
                                                                       rcs_m),
               "nproc": cores,
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": "first %d envs x %d steps (%.1f s); oracle ray-cells/s "
                                           "%.3g" % (n_s, steps_s, dt1, rcs1)}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i16+f32", "data": "synthetic",
        "config": dict(workload, autotuned=({"threads_per_cta": tuned[0], "window_cells": tuned[1]}
                                            if tuned else None)),
        "ray_cells_per_s": ray_cells_all / (total_ms_max / 1e3),
        "ray_cells_per_step": ray_cells / K,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind + " hbm_gbs (STREAM-style copy)",
                     "bytes_per_launch": kbytes[kern], "ms_per_launch": k_ms, "kernel": kern,
                     "issue": issue},
        "kernels": kernels,
        "kernel_pass": {"steps": prof_steps,
                        "note": "per-kernel CUDA events in a separate pass; they serialise "
                                "the kernels, so their sum exceeds the timed step"},
        "step_roofline": {"bytes_per_step": step_bytes,
                          "achieved": step_bytes / (ms_step / 1e3) / 1e9,
                          "frac": step_bytes / (ms_step / 1e3) / 1e9 / peak},
        "batched_4096": batched,
        "cpu_baseline": cpu,
        "e2e": {"value": E_all * K2 / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "aslam_step_host on page-locked host buffers: the step's kernels read the "
                        "actions and U and write the reward and observation through the buffers' "
                        "device mapping (NVLink-C2C), inside the timed region"},
        "graph": {"value": E_all / (g_ms / 1e3), "unit": UNIT, "steps": gk,
                  "ms_per_step": g_ms},
        "gpu_launches": K * len(kernel_ms),
        "clocks": clk,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
