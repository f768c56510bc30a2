#!/usr/bin/env python
"""Benchmark of the batched push-rollout path (one JSON line on stdout, rank 0).

Workload: 4096 independent cluttered scenes with uneven box counts (n ~ U{5..40},
half extents U[0.01, 0.04] m, mu U[0.3, 0.8], yaw U[0, pi/2), clutter density
U[0.2, 0.6]), one random valid first push per environment, then two device-sampled
pushes (depth 3), 240 substeps of 1/240 s per push, 10 PGS iterations.  A step is one
batched rollout of all environments.  Metric: simulated environment-substeps per second
(env-steps/s).

  value   device-resident inputs (scene store loaded once; environment ids, first pushes
          and seeds in device memory), timed with CUDA events on the launching stream;
          the L2 cache is flushed (256 MB write) before every step.
  e2e     the same metric through the C ABI from host buffers: scenes loaded, batch
          submitted, results copied back and memory released inside the timed region.
  roofline  the rollout kernel against the FP32 CUDA-core peak (ALU bound).
  cpu_baseline  the FP64 CPU oracle on the host cores, on a bounded sample.

--impl reference times the FP64 CPU oracle (a plain sequential restatement of the method,
the comparison arm) on the same workload and metric.  Under torchrun each rank runs its own 4096-environment workload on
its own GPU (weak scaling, no data-path collective).
"""
import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM traffic of one rollout-kernel launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), valid only for the kernel source it was measured on.
TRAFFIC = {"source_sha": "f79caa85e37b8739", "bytes_per_launch": 118213120,
           "note": "ncu dram bytes (read 21.36 MB + write 96.85 MB) of one launch of the benchmark "
                   "workload itself (4096 scenes, depth 3) in the 32,2,0 launch shape, single-pass capture"}


def measured_hbm_gbs():
    """Measured copy bandwidth of the B300s (MEASURED_PEAKS.json), else the
    recipe's fallback of 6400 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0


def _code_only(src: bytes) -> bytes:
    """Source with // comments and blank lines removed (comment edits change no kernel)."""
    out = []
    for line in src.decode().splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return "\n".join(out).encode()


def kernel_source_sha():
    """Hash of the rollout kernel's device code: the three device headers and the marked
    rollout section of the engine source (host code and other kernels excluded), with
    comments stripped."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_06649_b300", "csrc")
    for f in ("pmbs_exact.cuh", "pmbs_collide.cuh", "pmbs_warp.cuh"):
        h.update(_code_only(open(os.path.join(csrc, f), "rb").read()))
    eng = open(os.path.join(csrc, "pmbs_engine.cu"), "rb").read()
    a = eng.index(b"// ---- rollout device code begins")
    b = eng.index(b"// ---- rollout device code ends")
    h.update(_code_only(eng[a:b]))
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--depth", type=int, default=3)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=768)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="time the default launch shape")
    ap.add_argument("--no-heightmaps", action="store_true")
    ap.add_argument("--no-phases", action="store_true", help="skip the per-phase cycle split")
    ap.add_argument("--cylinders", type=int, default=1, help="also time the cylinder workload (0 = skip)")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape 'lanes,warps_per_block,smem_manifolds' instead of autotuning")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="served-load run length (0 = skip)")
    ap.add_argument("--plan-seeds", type=int, default=10, help="planning scenes per method (0 = skip)")
    ap.add_argument("--arena-gb", type=float, default=8.0, help="device arena of the timed engine")
    ap.add_argument("--plan-tmax", type=float, default=2.0, help="PMBS planning budget per action (s)")
    ap.add_argument("--serial-budgets", default="1,4", help="serial MCTS budgets per action (s), ascending")
    ap.add_argument("--plan-c", default="1.4", help="UCB exploration constants of the planning run")
    ap.add_argument("--planning-study", action="store_true",
                    help="only the planning episodes (--plan-seeds, --plan-c, budgets); one JSON line")
    ap.add_argument("--cpu-config2", action="store_true",
                    help="only the FP64 oracle on the fixed 1024 x 15-box workload in full; one JSON line")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOAD = "uneven rollout: {envs} scenes x U{{5..40}} boxes, depth {depth} x 240 substeps"
METRIC = "env-steps/s at 4096 uneven envs"


class ClockSampler:
    """nvidia-smi SM clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(scenes, pushes, seeds, depth, sample, label):
    import oracle
    from paper_2207_06649_b300 import scenegen as sg
    n = min(sample, scenes.n_scenes)
    sub = scenes.gather(range(n))
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    r = oracle.rollout(sub.box_offset, sg.state13(sub), sub.half, sub.mass, sub.mu, sub.target, pushes[:n], depth,
                       seeds[:n], threads=cores)
    dt = time.perf_counter() - t
    es = int(r.steps.sum())
    return {"value": es / dt, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n} of the {label} environments ({es} env-steps, FP64, {cores} threads, "
                      f"{dt:.1f} s)"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    from paper_2207_06649_b300 import scenegen as sg
    scenes, pushes, seeds = sg.config_uneven(seed=args.seed, n_envs=args.envs)
    per_step = min(args.cpu_sample, scenes.n_scenes)
    for _ in range(args.warmup):
        cpu_baseline(scenes, pushes, seeds, args.depth, max(8, per_step // 8), "workload's")
    vals, t_total, es_total = [], 0.0, 0
    for _ in range(args.steps):
        b = cpu_baseline(scenes, pushes, seeds, args.depth, per_step, "workload's")
        vals.append(b)
    v = float(np.mean([b["value"] for b in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(envs=args.envs, depth=args.depth), "envs": args.envs, "depth": args.depth,
                       "per_step_sample": per_step},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"], "value": v,
                             "unit": "env-steps/s"},
            "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_run(pmbs, sg, dev_index, seconds, rate, seed=5, planners=64, pool=None, eng=None):
    """Served rollouts: `planners` threads submit batches of log-uniform size in [32, 2048]
    at Poisson times (aggregate `rate` batches/s) over device-resident scenes of 5-40
    boxes, depth 3; returns offered and achieved load and latency percentiles."""
    import threading
    scenes, pushes = pool
    ids = eng.load(scenes)
    sv = pmbs.Server(eng, n_streams=8, max_inflight=64)
    tickets, lock = [], threading.Lock()
    t0 = time.perf_counter()

    def planner(pid):
        rng = np.random.default_rng(seed * 1000 + pid)
        t = t0
        while True:
            t += rng.exponential(planners / rate)
            if t > t0 + seconds:
                break
            dt = t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            n = int(round(np.exp(rng.uniform(np.log(32), np.log(2048)))))
            pick = rng.integers(0, scenes.n_scenes, size=n)
            sd = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
            tk = sv.submit(ids[pick], pushes[pick], 3, sd)
            with lock:
                tickets.append(tk)

    th = [threading.Thread(target=planner, args=(i,)) for i in range(planners)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for tk in list(tickets):
        sv.wait(tk)
    st = sv.stats()
    sv.close()
    eng.free_scenes(ids)
    return {"offered_batches_per_s": rate, "submitted": len(tickets), "window_s": seconds,
            "achieved_batches_per_s": st["completed"] / st["span_s"] if st["span_s"] else None,
            "env_steps_per_s": st["env_steps"] / st["span_s"] if st["span_s"] else None,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "peak_arena_gb": st["peak_bytes"] / 2 ** 30}


def hard_planning_scenes(pmbs, sg, eng, count, max_seed=200):
    """Planning scenes whose target no single push frees: the target starts not graspable
    and none of the root's expansion candidates (16 contour points around every box
    within 0.1 m of the target) makes it graspable after one push (one batched depth-1
    rollout on the engine).  Returns [(seed, scene, candidates)], seeds in order."""
    from paper_2207_06649_b300 import planner as P
    out, rejected = [], {"graspable_at_start": 0, "one_push": 0}
    for sd in range(max_seed):
        if len(out) >= count:
            break
        sc = sg.config_planning(sd)
        st = sg.state13(sc)
        be = P.GpuBackend(eng, sc.half, sc.mass, sc.mu)
        if be.graspable(st, sc.half, 0):
            rejected["graspable_at_start"] += 1
            continue
        cand = P.contour_candidates(st, sc.half, 0)
        h = be.load_state(st, sc.half, 0)
        r = be.rollout(np.full(len(cand), h, np.int32), cand, 1, np.zeros(len(cand), np.uint64))
        be.release([h] + list(r["child_handles"]))
        if np.any(r["cost"] == 1):
            rejected["one_push"] += 1
            continue
        out.append((sd, sc, len(cand)))
    return out, rejected


def planning_run(pmbs, sg, local, seeds, tmax, serial_budgets, n_envs=512, c=1.4, max_actions=16):
    """Full planning episodes on buried-target 30-box scenes that no single push solves:
    PMBS with n_envs rollouts per iteration vs serial MCTS (one rollout per iteration) on
    the same engine, each given a planning budget per action; reports actions to
    retrieval (pushes + grasp) with their distribution, completion within max_actions,
    planning seconds per action, and the serial budget at which serial MCTS first
    matches PMBS's mean actions (equal solution cost)."""
    from paper_2207_06649_b300 import planner as P
    eng = pmbs.Engine(device=local, mem_budget_bytes=4 << 30)
    scenes, rejected = hard_planning_scenes(pmbs, sg, eng, seeds)
    methods = [("pmbs", n_envs, tmax)] + [("serial", 1, b) for b in serial_budgets]
    res = {}
    for name, ne, budget in methods:
        acts, done, plan, iters = [], 0, [], []
        for sd, sc, _ in scenes:
            be = P.GpuBackend(eng, sc.half, sc.mass, sc.mu)
            st = sg.state13(sc)
            ep = P.run_episode(be, st, sc.half, 0,
                               lambda: P.Planner(be, sc.half, 0, n_envs=ne, c=c, t_max=budget, seed=sd),
                               max_actions=max_actions)
            acts.append(ep["actions"])
            done += int(ep["success"])
            plan.extend(ep["plan_s"])
        key = f"{name}_{budget:g}s" if name == "serial" else f"pmbs_{ne}envs_{budget:g}s"
        res[key] = {"episodes": len(acts), "actions_mean": float(np.mean(acts)) if acts else None,
                    "actions": [int(a) for a in acts],
                    "completion": done / max(1, len(acts)),
                    "plan_s_per_action": float(np.mean(plan)) if plan else None,
                    "plan_s_total_mean": float(np.sum(plan) / max(1, len(acts)))}
    eng.close()
    pm = res[f"pmbs_{n_envs}envs_{tmax:g}s"]
    equal = None
    for b in serial_budgets:
        r = res[f"serial_{b:g}s"]
        if r["actions_mean"] is not None and pm["actions_mean"] is not None and \
                r["actions_mean"] <= pm["actions_mean"] + 1e-9:
            equal = {"serial_budget_s": b, "serial_plan_s_total_mean": r["plan_s_total_mean"],
                     "pmbs_plan_s_total_mean": pm["plan_s_total_mean"],
                     "speedup": r["plan_s_total_mean"] / max(pm["plan_s_total_mean"], 1e-9)}
            break
    return {"scenes": [sd for sd, _, _ in scenes], "rejected": rejected,
            "root_candidates": [k for _, _, k in scenes], "by_method": res,
            "equal_cost": equal if equal else "no serial budget reached PMBS's mean actions"}


def run_ours(args):
    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2207_06649_b300 import flops, multigpu, pmbs, scenegen as sg

    scenes, pushes, seeds = sg.config_uneven(seed=multigpu.rank_seed(args.seed, rank), n_envs=args.envs)
    stream = torch.cuda.current_stream()
    eng = pmbs.Engine(device=local, mem_budget_bytes=int(args.arena_gb * 2 ** 30), max_envs=max(args.envs, 1),
                      stream=pmbs.C.c_void_p(stream.cuda_stream))
    ids = eng.load(scenes)
    d_ids = torch.from_numpy(ids.astype(np.int32)).to(dev)
    d_push = torch.from_numpy(pushes.astype(np.float32)).to(dev)
    d_seed = torch.from_numpy(seeds.view(np.int64)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def one_step():
        b = eng.rollout_pushes_device(args.envs, d_ids.data_ptr(), d_push.data_ptr(), args.depth, d_seed.data_ptr())
        eng.step(b, 0)
        return b

    # launch shape picked by the library's autotuner on this workload (untimed)
    tuned = None
    rollout_launches = 1
    if args.shape:
        g_, w_, m_ = (int(x) for x in args.shape.split(","))
        eng.set_launch_shape(g_, w_, -1, m_)
        tuned = {"lanes_per_env": g_, "warps_per_block": w_, "smem_manifolds": m_, "fixed": True}
    elif not args.no_autotune:
        tuned = eng.autotune(ids, pushes, args.depth, seeds, substeps=240)
        k = tuned.get("substeps_per_launch", 0)
        rollout_launches = 1 if k <= 0 else -(-args.depth * 240 // k)

    # warm-up (untimed); the first batch also gives the per-step work counts
    batches = []
    for w in range(max(args.warmup, 1)):
        flush.zero_()
        batches.append(one_step())
    torch.cuda.synchronize()
    st, steps = eng.query_states(batches[0])
    env_steps = int(steps.sum())
    ev = eng.query_events(batches[0])
    flops_per_launch = flops.algorithmic_flops(ev, pmbs.EVENT_NAMES)
    flops_phases = flops.flops_by_phase(ev, pmbs.EVENT_NAMES)
    boxes = scenes.counts()
    for b in batches:
        eng.release_batch(b)
    batches = []

    # timed region
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0.record()
        for i in range(args.steps):
            flush.zero_()
            k0[i].record()
            batches.append(one_step())
            k1[i].record()
        t1.record()
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    elapsed = t0.elapsed_time(t1) / 1e3
    step_ms = [a.elapsed_time(b) for a, b in zip(k0, k1)]
    kernel_s = float(np.mean(step_ms)) / 1e3
    for b in batches:
        eng.release_batch(b)
    elapsed, total_env_steps = multigpu.reduce_job(elapsed, env_steps * args.steps, device=dev)
    value = total_env_steps / elapsed

    # per-phase split of the warps' cycles (library phase timers, one untimed launch of the
    # same batch in the same launch shape)
    phase = None
    if not args.no_phases:
        teng = pmbs.Engine(device=local, mem_budget_bytes=int(args.arena_gb * 2 ** 30), max_envs=max(args.envs, 1),
                           stream=pmbs.C.c_void_p(stream.cuda_stream), phase_timers=1)
        if tuned is not None:
            teng.set_launch_shape(tuned["lanes_per_env"], tuned["warps_per_block"], -1, tuned["smem_manifolds"])
        tids = teng.load(scenes)
        tb = teng.rollout_pushes(tids, pushes, args.depth, seeds)
        teng.step(tb, 0)
        cyc = teng.query_phase_cycles(tb).astype(np.float64)
        teng.release_batch(tb)
        teng.close()
        tot = cyc.sum(0)
        phase = {"cycles_share": {n: float(v / tot.sum()) for n, v in zip(pmbs.PHASE_NAMES, tot)},
                 "cycles_per_env_step": float(tot.sum() / max(env_steps, 1)),
                 "source": "pmbs_query_phase_cycles on one untimed launch of the same batch (phase_timers=1)"}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_off, h_pose, h_vel = pin(scenes.box_offset), pin(scenes.pose), pin(scenes.vel)
        h_half, h_mass, h_mu, h_tgt = pin(scenes.half), pin(scenes.mass), pin(scenes.mu), pin(scenes.target)
        h_push, h_seed = pin(pushes.astype(np.float32)), pin(seeds)
        h2d = sum(a.nbytes for a in (h_off, h_pose, h_vel, h_half, h_mass, h_mu, h_tgt, h_push, h_seed)) + 4 * args.envs
        d2h = 9 * args.envs

        def e2e_step():
            sid = eng.load_scenes(h_off, h_pose, h_half, h_mass, h_mu, h_tgt, vel=h_vel)
            b = eng.rollout_pushes(sid, h_push, args.depth, h_seed)
            eng.step(b, 0)
            r = eng.query_cost(b)
            eng.release_batch(b)
            eng.free_scenes(sid)
            return r

        for _ in range(max(1, args.warmup - 1)):
            e2e_step()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        te = time.perf_counter() - ts
        e2e = {"value": env_steps * args.steps * ws / te, "unit": "env-steps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # top-down workspace heightmaps of the workload's final states (device entry point),
    # timed with CUDA events on the engine's stream; output-write bound (83 KB per map)
    heightmaps = None
    if not args.no_heightmaps:
        d_off = torch.from_numpy(scenes.box_offset.astype(np.int32)).to(dev)
        d_st = torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(dev)
        d_half = torch.from_numpy(np.ascontiguousarray(scenes.half, np.float32)).to(dev)
        d_hm = torch.empty((args.envs, 144, 144), dtype=torch.float32, device=dev)
        render = lambda: eng.render_heightmaps_device(args.envs, d_off.data_ptr(), d_st.data_ptr(),
                                                      d_half.data_ptr(), d_hm.data_ptr())
        for _ in range(3):
            render()
        h0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        h1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            h0[i].record()
            render()
            h1[i].record()
        torch.cuda.synchronize()
        hm_s = float(np.mean([a.elapsed_time(b) for a, b in zip(h0, h1)])) / 1e3
        out_bytes = 4.0 * 144 * 144 * args.envs
        in_bytes = float(boxes.sum()) * (52 + 12) + 4.0 * (args.envs + 1)
        hbm = measured_hbm_gbs()
        heightmaps = {"maps": args.envs, "cells": "144 x 144 x 2 mm", "ms": hm_s * 1e3,
                      "maps_per_s": args.envs / hm_s, "bytes_per_launch": out_bytes + in_bytes,
                      "achieved_gbs": (out_bytes + in_bytes) / hm_s / 1e9, "peak_gbs": hbm,
                      "frac": (out_bytes + in_bytes) / hm_s / 1e9 / hbm if hbm else None,
                      "kernel": "heightmap_kernel"}

    # the same workload with cylinders (30 % of the objects, every target): the rollout
    # kernel built with the cylinder contact paths, autotuned, timed like the main line
    cylinders = None
    if args.cylinders and ws == 1:
        cs, cp, cd = sg.config_cylinders(seed=args.seed + 2, n_envs=args.envs)
        cids = eng.load(cs)
        if not args.no_autotune:
            ctuned = eng.autotune(cids, cp, args.depth, cd, substeps=240)
        c_steps = None
        cms = []
        for i in range(args.warmup + args.steps):
            cb = eng.rollout_pushes(cids, cp, args.depth, cd)
            flush.zero_()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            eng.step(cb, 0)
            c1.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                cms.append(c0.elapsed_time(c1))
            if c_steps is None:
                c_steps = int(eng.query_states(cb)[1].sum())
            eng.release_batch(cb)
        eng.free_scenes(cids)
        cms_mean = float(np.mean(cms))
        cylinders = {"workload": f"{args.envs} scenes x U{{5..40}} objects, 30 % cylinders (16-gon prisms), "
                                 f"cylinder targets, depth {args.depth} x 240 substeps",
                     "cylinder_fraction": float(sg.is_cylinder(cs.half).mean()),
                     "env_steps_per_step": c_steps, "ms_per_step": cms_mean,
                     "value": c_steps / (cms_mean / 1e3), "unit": "env-steps/s",
                     "launch_shape": ctuned if not args.no_autotune else "default",
                     "kernel": "rollout_kernel (cylinder contact paths compiled in)"}

    serving = None
    if args.serve_seconds > 0 and ws == 1:
        pool_sc, pool_pu, _ = sg.config_uneven(seed=args.seed + 7, n_envs=512)
        seng = pmbs.Engine(device=local, mem_budget_bytes=16 << 30, max_envs=4096)
        sweep = [serving_run(pmbs, sg, local, args.serve_seconds, rate, seed=5 + i, pool=(pool_sc, pool_pu), eng=seng)
                 for i, rate in enumerate((50.0, 100.0, 150.0, 200.0))]
        full = sweep[-1]
        # sustainable rate: what the device completed under overload, with 20 % headroom
        rate = max(1.0, 0.8 * (full["achieved_batches_per_s"] or 1.0))
        sus = serving_run(pmbs, sg, local, args.serve_seconds * 2, rate, seed=9, pool=(pool_sc, pool_pu), eng=seng)
        seng.close()
        serving = {"config": "64 planners, batches log-uniform 32..2048 envs, Poisson arrivals, 5-40 boxes, "
                             "depth 3, 16 GB arena, continuous batching on 8 streams",
                   "offered_load_sweep": sweep, "at_200_per_s": full, "sustainable": sus}
    planning = None
    if args.plan_seeds > 0 and ws == 1:
        budgets = [float(x) for x in args.serial_budgets.split(",") if x]
        planning = {"config": "30-box clutter, target buried on 16 rays within 0.03 m and freed by no single "
                              "push, UCB c=1.4, gamma 0.8, d_T 7 + d_s 3, expansion candidates 16 contour points "
                              "per box within 0.1 m, completion within 16 actions",
                    "seeds": args.plan_seeds,
                    "results": planning_run(pmbs, sg, local, args.plan_seeds, args.plan_tmax, budgets)}
    peak_fma = eng.fp32_peak()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    max_mhz = clocks["sm_max_mhz"] or 2032.0
    peak = flops.fp32_peak_tflops(sms, max_mhz)
    achieved = flops_per_launch / kernel_s / 1e12
    solve = None
    if phase is not None:
        # the contact solve's own rate: its algorithmic flops over the share of the launch
        # its warps spent in it
        sh = phase["cycles_share"]["contact_solve"]
        rate = flops_phases["contact_solve"] / (kernel_s * sh) / 1e12
        solve = {"achieved": rate, "frac": rate / peak, "cycles_share": sh,
                 "flops_per_launch": flops_phases["contact_solve"]}
    sha = kernel_source_sha()
    default_workload = (args.envs, args.depth, args.seed) == (4096, 3, 3)
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["source_sha"] == sha and default_workload else None
    state_bytes = float(boxes.sum()) * (72 + 52 + 52) + args.envs * (28 + 64 + 13)
    line = {
        "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(envs=args.envs, depth=args.depth), "envs": args.envs, "boxes_per_env_mean": float(boxes.mean()),
                   "boxes_per_env_range": [int(boxes.min()), int(boxes.max())], "depth": args.depth,
                   "substeps_per_push": 240, "pgs_iters": 10, "env_steps_per_step": env_steps,
                   "box_steps_per_s": value * float(boxes.mean()),
                   "l2": "flushed before every step (256 MB device write)",
                   "parallelism": f"one environment per warp, persistent launch; {ws} GPU(s), weak scaling",
                   "launch_shape": tuned if tuned is not None else "default",
                   "step_ms_best": float(np.min(step_ms)), "step_ms_median": float(np.median(step_ms)),
                   "env_steps_per_s_best": env_steps / (float(np.min(step_ms)) / 1e3)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "rollout_kernel", "kernel_ms": kernel_s * 1e3,
                     "flops_per_launch": flops_per_launch, "flops_by_phase": flops_phases,
                     "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                     "fma_probe_tflops": peak_fma,
                     "hbm_achieved_gbs": state_bytes / kernel_s / 1e9,
                     "contact_solve": solve},
        "phases": phase,
        "clocks": clocks,
        "e2e": e2e,
        "serving": serving,
        "heightmaps": heightmaps,
        "cylinders": cylinders,
        "planning": planning,
        # per timed step: the batch set-up kernel and the rollout launch(es) of the tiling
        "gpu_launches": args.steps * (1 + rollout_launches),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scenes, pushes, seeds, args.depth, args.cpu_sample, "workload's")
    eng.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def planning_study(args):
    """Planning episodes alone: for every UCB constant, PMBS and the serial budgets."""
    from paper_2207_06649_b300 import pmbs, scenegen as sg
    budgets = [float(x) for x in args.serial_budgets.split(",") if x]
    out = {"study": "planning", "seeds": args.plan_seeds, "pmbs_budget_s": args.plan_tmax,
           "config": "30-box clutter, target buried on 16 rays within 0.03 m, gamma 0.8, d_T 7 + d_s 3, "
                     "512 rollouts per PMBS iteration, expansion candidates 16 contour points per box "
                     "within 0.1 m, completion within 16 actions", "by_c": {}}
    for c in [float(x) for x in args.plan_c.split(",") if x]:
        out["by_c"][f"{c:g}"] = planning_run(pmbs, sg, 0, args.plan_seeds, args.plan_tmax, budgets, c=c)
    print(json.dumps(out), flush=True)


def cpu_config2(args):
    """The FP64 oracle on the fixed workload (1024 clones of one 15-box scene, depth 3)
    in full, one thread per host core."""
    import oracle
    from paper_2207_06649_b300 import scenegen as sg
    oracle.build()
    sc, pushes, seeds = sg.config_fixed()
    envs = sc.gather([0] * len(pushes))
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    r = oracle.rollout(envs.box_offset, sg.state13(envs), envs.half, envs.mass, envs.mu, envs.target, pushes,
                       depth=3, seeds=seeds, threads=cores)
    dt = time.perf_counter() - t
    es = int(r.steps.sum())
    bs = int(sum(r.steps[e] * (envs.box_offset[e + 1] - envs.box_offset[e]) for e in range(len(pushes))))
    print(json.dumps({"study": "cpu_baseline_config2", "kind": "oracle", "cores": cores, "seconds": dt,
                      "env_steps": es, "env_steps_per_s": es / dt, "box_steps_per_s": bs / dt,
                      "workload": "1024 clones of one 15-box scene, 1024 first pushes, depth 3 x 240 substeps",
                      "invalid_starts": int(np.sum((r.flags & 2) != 0))}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.planning_study:
        planning_study(a)
    elif a.cpu_config2:
        cpu_config2(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
