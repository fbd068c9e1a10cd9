#!/usr/bin/env python3
"""Benchmark: SMMO parallel_do on Wa-Tor 2048x2048 (thesis Sec. 7.6).

One bench step = one Wa-Tor iteration: the fish phase and the shark phase,
each a parallel_do of prepare and of update over all live agents of the
class (4 enumeration kernels + 4 method kernels, with device new/delete).
The metric is object-updates/s: objects visited by the parallel_do launches
of the timed steps divided by their device time.  Timed steps start from the
seeded initial state (step 1, 2, ...); the L2 cache (129 MB) is flushed by a
256 MiB write before every timed step, outside the timed interval, since the
simulation's working set (~60-120 MB) would otherwise stay L2-resident.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl smmo|reference]

--impl reference times the CPU oracle (plain single-threaded C) on the same
workload and metric.  Under torchrun every rank runs an independent replica
(the workload does not shard; see the design notes); value = objects of all
ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W_SIDE = 2048
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
SEED = 1
CONFIG_STEPS = 500
FLUSH_BYTES = 256 << 20
# Algorithmic bytes per visited object for each method kernel (bytes the
# method must read or write for that object: its own SOA fields plus the
# cell words it touches; the request atomics count 8 read + 8 write).
BYTES_PER_OBJECT = {
    "fish_prepare": 4 + 2 + 2 + 4 + 4 * 4 + 16,      # cell, age r/w, target, 4 occ, req RMW
    "fish_update": 4 + 4 + 8 + 4 + 4 + 2 + 4,        # cell, target, req, occ[tgt], cell w, age, occ[old]
    "shark_prepare": 4 + 4 + 4 + 4 + 4 * 4 + 4 * 4 + 16,  # cell, age, energy r/w, target, occ, types, req
    "shark_update": 4 + 2 + 4 + 8 + 4 + 4 + 4 + 2 + 4,
}
# a species' prepare and update fused into one launch (the phased Wa-Tor
# step kernels) move the bytes of both
BYTES_PER_OBJECT["fish_step"] = BYTES_PER_OBJECT["fish_prepare"] + BYTES_PER_OBJECT["fish_update"]
BYTES_PER_OBJECT["shark_step"] = BYTES_PER_OBJECT["shark_prepare"] + BYTES_PER_OBJECT["shark_update"]
PHASES = ["life_cand_prepare", "life_alive_prepare", "life_cand_update", "life_alive_update",
          "fish_prepare", "fish_update", "shark_prepare", "shark_update"]
# phase names when each species runs as one fused launch (phases 5 and 7 empty)
PHASES_FUSED = PHASES[:4] + ["fish_step", "", "shark_step", ""]
STEP_KERNELS = {"four_do_alls": 0, "phased1": 1, "phased2": 2, "four_do_alls_queued": 4, "phased2_queued": 6,
                "four_do_alls_marked": 8, "four_do_alls_marked_queued": 12}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "wator_2048_fish_update_traffic.txt")  # JSON
# Sources of the Wa-Tor kernels: the allocator and do-all core, the
# cellular helpers, the fused phases, and the Wa-Tor methods and their
# variants (world_wator.cuh, world_modes.cu, world_phased.cu), so that
# changes elsewhere keep a traffic capture valid.
KERNEL_SOURCES = ["paper_1908_05845_gb300/csrc/smmo_core.cuh", "paper_1908_05845_gb300/csrc/grid_common.cuh",
                  "paper_1908_05845_gb300/csrc/phased.cuh", "paper_1908_05845_gb300/csrc/levels.cuh",
                  "paper_1908_05845_gb300/csrc/world_wator.cuh", "paper_1908_05845_gb300/csrc/world_modes.cu",
                  "paper_1908_05845_gb300/csrc/world_phased.cu"]


def kernel_hash(read=lambda f: open(os.path.join(ROOT, f), "rb").read()) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(read(f))
    return h.hexdigest()[:16]


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the
    timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        """Starts sampling every 50 ms and returns once the first sample is
        in (nvidia-smi takes a while to start), so that the samples kept,
        those after this call, lie inside the timed region."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.first = len(self.lines)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples taken during the timed region; the one just before it if
        # the region was shorter than the sampling interval
        kept = self.lines[self.first:] or self.lines[max(0, self.first - 1):self.first]
        for ln in kept:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_over_ranks(t_local: float, objects: int, allocfree: int, device):
    """Whole-job figures of the replicas: the largest timed interval over
    the ranks and the objects (and allocations + frees) of all ranks."""
    import torch
    import torch.distributed as dist
    v = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    o = torch.tensor([objects, allocfree], dtype=torch.float64, device=device)
    dist.all_reduce(o)
    return float(v.item()), int(o[0].item()), int(o[1].item())


def host_info() -> dict:
    """The host the CPU legs ran on: logical CPUs, architecture and the
    processor's model name (from lscpu, when it is there)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model}


def replica_seed(rank: int) -> int:
    """Seed of rank `rank`'s independent replica."""
    return SEED + rank


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ reference arm
def oracle_sample(steps: int, t0: int = 0, state=None):
    """Times the oracle for `steps` Wa-Tor steps; returns (updates, seconds,
    final state)."""
    import oracle
    from paper_1908_05845_gb300 import inputs
    if state is None:
        state = inputs.wator_initial(W_SIDE, W_SIDE, SEED)
    k, a, e = state
    F0, S0 = int((k == 1).sum()), int((k == 2).sum())
    t = time.perf_counter()
    k2, a2, e2, cnt = oracle.wator_run(W_SIDE, W_SIDE, SEED, k, a, e, steps, t0=t0)
    dt = time.perf_counter() - t
    F = np.concatenate([[F0], cnt[:-1, 0]])
    S = np.concatenate([[S0], cnt[:-1, 1]])
    return int(np.sum(2 * F + 2 * S)), dt, (k2, a2, e2)


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    state = None
    t0 = 0
    if args.warmup:
        _, _, state = oracle_sample(args.warmup, 0, state)
        t0 = args.warmup
    # timed steps start again from the initial state so they cover the same
    # iterations as the GPU arm
    upd, dt, _ = oracle_sample(args.steps, 0, None)
    value = upd / dt
    line = {
        "impl": "reference", "metric": "object-updates/s", "value": value, "unit": "object-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32/int16", "data": "synthetic (seeded Philox)",
        "config": {"workload": "wator_2048x2048", "W": W_SIDE, "H": W_SIDE, "seed": SEED,
                   "steps_in_config": CONFIG_STEPS, "instances": 1},
        "cpu_baseline": {"value": value, "unit": "object-updates/s", "cores": 1, "kind": "oracle", "host": host_info(),
                         "sample": "Wa-Tor 2048x2048 steps 1..%d from the seeded initial state, "
                                   "single-threaded C oracle" % args.steps},
        "e2e": {"value": value, "unit": "object-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU arm
def run_gpu(args, ws, rank, local):
    import torch
    from paper_1908_05845_gb300 import inputs, smmo
    from paper_1908_05845_gb300.workloads import WaTor, heap_bytes_for

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        smmo.lib()
    except smmo.SmmoError:
        from paper_1908_05845_gb300 import build
        build.build()
    seed = replica_seed(rank)  # independent replicas
    k0, a0, e0 = inputs.wator_initial(W_SIDE, W_SIDE, seed)
    hb = heap_bytes_for(W_SIDE * W_SIDE, 1.0)
    stream = torch.cuda.current_stream()
    # warm-up on its own world (same seed)
    mode = STEP_KERNELS[args.step_kernels]
    fused = (mode & 3) != 0
    warm = WaTor(W_SIDE, W_SIDE, seed, k0, a0, e0, heap_bytes=hb, step_kernels=mode)
    if args.warmup:
        warm.step_profiled(args.warmup)
    warm.sync()
    warm.close()
    del warm
    sim = WaTor(W_SIDE, W_SIDE, seed, k0, a0, e0, heap_bytes=hb, step_kernels=mode)
    fish_cls, shark_cls = sim.class_ids["Fish"], sim.class_ids["Shark"]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    phase_ms = np.zeros(16)
    step_ms = 0.0
    launches = 0
    objs_phase = np.zeros(8)
    F = int((k0 == 1).sum())
    S = int((k0 == 2).sum())
    enum0, alloc0, free0 = sim.heap.counters()
    ac0 = sim.heap.alloc_counters()
    blocks0 = ac0["enumerated_blocks"]
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        ph, sm, la = sim.step_profiled(1)
        phase_ms += np.array(ph)
        step_ms += sm
        launches += la
        objs_phase[4] += F
        objs_phase[5] += F
        objs_phase[6] += S
        objs_phase[7] += S
        st = sim.heap.stats()
        F, S = st["live_objects"][fish_cls], st["live_objects"][shark_cls]
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    enum1, alloc1, free1 = sim.heap.counters()
    ac1 = sim.heap.alloc_counters()
    blocks1 = ac1["enumerated_blocks"]
    sim.sync()
    objects = enum1 - enum0
    assert objects == int(objs_phase.sum()), (objects, objs_phase.sum())
    allocfree = (alloc1 - alloc0) + (free1 - free0)
    t_local = step_ms / 1e3
    t_max, objects_all, allocfree_all = t_local, objects, allocfree
    if ws > 1:
        t_max, objects_all, allocfree_all = reduce_over_ranks(t_local, objects, allocfree, "cuda")
    value = objects_all / t_max

    # roofline of the dominant kernel
    names = PHASES_FUSED if fused else PHASES
    meth = phase_ms[1::2]
    dom = int(np.argmax(meth))
    name = names[dom]
    peaks = load_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    bytes_dom = BYTES_PER_OBJECT.get(name, 0) * objs_phase[dom]
    achieved = bytes_dom / (meth[dom] / 1e3) / 1e9 if meth[dom] > 0 else 0.0
    n_launch_dom = args.steps
    traffic = None
    try:
        tr = json.load(open(TRAFFIC_FILE))
        if tr.get("kernel_hash") == kernel_hash() and tr.get("phase") == name:
            # per launch at the captured case, scaled by objects per launch
            traffic = tr["dram_bytes_per_object"] * objs_phase[dom] / n_launch_dom
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "kernel": "do_all<%s>" % name,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                "bytes_per_object": BYTES_PER_OBJECT.get(name, 0),
                "objects_per_launch": objs_phase[dom] / n_launch_dom,
                "avg_launch_us": 1e3 * meth[dom] / n_launch_dom,
                # the same against the nominal HBM3e bandwidth (7.9 TB/s)
                "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS}

    # the whole step: every do-all's objects x its bytes per object, a
    # 16-byte bitmap read-modify-write per device new or delete, and 24
    # bytes (bitmap word read, entry written) per enumerated block
    step_bytes = (sum(BYTES_PER_OBJECT.get(names[p], 0) * objs_phase[p] for p in range(8))
                  + 16 * allocfree + 24 * (blocks1 - blocks0))
    step_achieved = step_bytes / t_local / 1e9
    step_roofline = {"bound": "hbm", "achieved": step_achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": step_achieved / hbm_peak, "bytes_per_step": step_bytes / args.steps,
                     "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": step_achieved / NOMINAL_HBM_GBS}

    cpu = None
    e2e = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle runs the timed steps themselves when they are few
        # enough (then the timed run's end state is compared with it)
        csteps = args.steps if args.steps <= 100 else args.cpu_steps
        upd, dt, want = oracle_sample(csteps)
        cpu = {"value": upd / dt, "unit": "object-updates/s", "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": "Wa-Tor 2048x2048 steps 1..%d (single-threaded C oracle, %.1f s)"
                         % (csteps, dt)}
        if csteps == args.steps and seed == SEED:
            got = sim.read()
            parity = {"value": bool(all(np.array_equal(g, w) for g, w in zip(got, want))),
                      "steps": args.steps,
                      "compared": "kind, age and energy of all %d cells after the timed steps, against the "
                                  "oracle's run of the same steps" % (W_SIDE * W_SIDE)}
    if rank == 0 and not args.no_e2e:
        e2e = run_e2e(args, seed, hb)
    sim.close()
    compared = None
    if rank == 0 and ws == 1 and not args.no_secondary:
        compared = compare_step_kernels(args, seed, hb, (k0, a0, e0), flush)
    secondary = {}
    if rank == 0 and ws == 1 and not args.no_secondary:
        secondary["batched_speedup_vs_per_instance"] = secondary_batched(args)
        secondary["adjoint_over_forward"] = secondary_adjoint(args)

    if rank == 0:
        line = {
            "metric": "object-updates/s", "value": value, "unit": "object-updates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/int16", "data": "synthetic (seeded Philox)",
            "config": {"workload": "wator_2048x2048", "W": W_SIDE, "H": W_SIDE, "seed": SEED,
                       "steps_in_config": CONFIG_STEPS, "instances_per_gpu": 1,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed (256 MiB write) before every timed step"},
            "alloc_free_per_s": allocfree_all / t_max,
            "roofline": roofline,
            "step_roofline": step_roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            # allocator events per step (warp-cache refills, blocks taken
            # from the free bitmap, reservations that found a full block...)
            "alloc_events_per_step": {k: (ac1[k] - ac0[k]) / args.steps for k in ac1},
            "phase_ms_per_step": {names[p]: {"enumerate": phase_ms[2 * p] / args.steps,
                                             "method": phase_ms[2 * p + 1] / args.steps}
                                  for p in range(4, 8) if names[p]},
            "step_kernels": args.step_kernels,
            "step_kernels_compared": compared,
            "parity_bit_exact": parity,
        }
        line.update(secondary)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def compare_step_kernels(args, seed, hb, init, flush, steps: int = 20):
    """ms per step of the same Wa-Tor run (seeded start, L2 flushed before
    every step, CUDA events around each step) in each step-kernel mode: the
    four do-alls, each species' prepare and update fused into one launch
    with one or two units per warp round, and either with the creations
    queued for a launch of their own."""
    import torch
    from paper_1908_05845_gb300.workloads import WaTor
    out = {}
    steps = min(steps, args.steps)
    for name, mode in STEP_KERNELS.items():
        w = WaTor(W_SIDE, W_SIDE, seed, *init, heap_bytes=hb, step_kernels=mode)
        total = 0.0
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            _, sm, _ = w.step_profiled(1)
            total += sm
        got = w.read() if seed == SEED else None
        w.sync()
        w.close()
        out[name] = {"ms_per_step": total / steps, "steps": steps}
        if got is not None:
            out[name]["state"] = got
    # the modes must agree cell for cell
    states = [v.pop("state") for v in out.values() if "state" in v]
    same = all(all(np.array_equal(a, b) for a, b in zip(states[0], st)) for st in states[1:])
    return {"modes": out, "identical_results": bool(same) if states else None}


def secondary_batched(args, n_inst: int = 64, steps: int = 10, warm: int = 3):
    """Batched heap against one launch sequence per instance, on the first
    n_inst instances of the batched recipe (sides 64..1021, log-uniform),
    default heap configuration: device ms per step of one captured graph
    over all instances, and of every instance stepped on a heap of its
    own (same instance numbers, so both simulate the same thing)."""
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import World, heap_bytes_for
    kinds, sides, init = inputs.batched_initial(SEED, n_inst)
    offs = np.concatenate([[0], np.cumsum(sides.astype(np.int64) ** 2)])
    total = int(offs[-1])
    stream = torch.cuda.Stream()
    clocks = ClockSampler(torch.cuda.current_device())
    with torch.cuda.stream(stream):
        w = World(kinds, sides, sides, SEED, *init, heap_bytes=heap_bytes_for(total), stream=stream)
        w.step(warm)
        w.capture(1)
        e0 = w.heap.counters()[0]
        a, b = _events(stream)
        torch.cuda.synchronize()
        clocks.start()
        a.record(stream)
        for _ in range(steps):
            w.replay()
        b.record(stream)
        b.synchronize()
        t_b = a.elapsed_time(b)
        objs_b = w.heap.counters()[0] - e0
        w.sync()
        w.close()
        worlds = [World([kinds[i]], [sides[i]], [sides[i]], SEED, *(x[offs[i]:offs[i + 1]] for x in init),
                        heap_bytes=heap_bytes_for(int(sides[i]) ** 2), stream=stream, inst_ids=[i])
                  for i in range(n_inst)]
        for x in worlds:
            x.step(warm)
        e0 = sum(x.heap.counters()[0] for x in worlds)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            for x in worlds:
                x.step(1)
        b.record(stream)
        b.synchronize()
        t_p = a.elapsed_time(b)
        clk = clocks.stop()
        objs_p = sum(x.heap.counters()[0] for x in worlds) - e0
        for x in worlds:
            x.close()
    return {"value": (objs_b / t_b) / (objs_p / t_p), "instances": n_inst, "cells": total, "steps": steps,
            "batched_ms_per_step": t_b / steps, "per_instance_ms_per_step": t_p / steps,
            "batched_object_updates_per_s": objs_b / t_b * 1e3,
            "per_instance_object_updates_per_s": objs_p / t_p * 1e3,
            "objects_equal": bool(objs_b == objs_p), "config": "default heap configuration (not tuned)",
            "clocks": clk}


def secondary_adjoint(args, n: int = 65536, steps: int = 50, ckpt: int = 10):
    """Cost of the n-body adjoint against its forward run (no merging,
    65,536 bodies, 50 steps, checkpoints every 10): device time of the
    checkpointed forward and of the reverse sweep (which recomputes each
    segment), per step."""
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.nbody import NBody
    st = inputs.nbody_initial(n, SEED)
    stream = torch.cuda.Stream()
    clocks = ClockSampler(torch.cuda.current_device())
    with torch.cuda.stream(stream):
        w = NBody(st, merge=False, stream=stream)
        a, b = _events(stream)
        torch.cuda.synchronize()
        clocks.start()
        a.record(stream)
        w.forward_ckpt(steps, ckpt)
        b.record(stream)
        b.synchronize()
        t_f = a.elapsed_time(b)
        a.record(stream)
        w.backward()
        b.record(stream)
        b.synchronize()
        t_b = a.elapsed_time(b)
        clk = clocks.stop()
        w.close()
    return {"value": t_b / t_f, "bodies": n, "steps": steps, "checkpoint_every": ckpt,
            "forward_ms_per_step": t_f / steps, "backward_ms_per_step": t_b / steps, "clocks": clk}


def run_e2e(args, seed, hb):
    """Same metric through the public API from host memory: pinned initial
    state copied in, world created, K steps each followed by a read-back of
    the device counters, final per-cell state copied out."""
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import WaTor
    k0, a0, e0 = inputs.wator_initial(W_SIDE, W_SIDE, seed)
    hk = torch.from_numpy(k0).pin_memory()
    ha = torch.from_numpy(a0).pin_memory()
    he = torch.from_numpy(e0).pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    dk, da, de = (x.to("cuda", non_blocking=True) for x in (hk, ha, he))
    sim = WaTor(W_SIDE, W_SIDE, seed, dk, da, de, heap_bytes=hb)
    e_start, _, _ = sim.heap.counters()
    for _ in range(args.steps):
        sim.step(1)
        sim.heap.counters()
    k, a, e = sim.read()
    e_end, _, _ = sim.heap.counters()
    dt = time.perf_counter() - t
    sim.close()
    h2d = hk.numel() + 2 * ha.numel() + 2 * he.numel()
    d2h = k.nbytes + a.nbytes + e.nbytes
    ctr = 8 * 40 * 32
    return {"value": (e_end - e_start) / dt, "unit": "object-updates/s",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps + ctr,
            "seconds": dt, "includes": "H2D of initial state, world setup, K steps with a "
                                       "counter read-back each, D2H of final state"}


# ------------------------------------------------------------ other workloads
def _events(stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    return a, b


def batched_init(seed, n):
    from paper_1908_05845_gb300 import inputs
    return inputs.batched_initial(seed, n)


def batched_parity_sample(kinds, sides, k_want=16):
    """Instances whose end state the batched bench compares with the
    oracle: the 8 largest and the rest spread evenly over the sizes."""
    order = np.argsort(-sides.astype(np.int64), kind="stable")
    big = [int(i) for i in order[:8]]
    rest = order[8:]
    spread = [int(rest[j]) for j in np.linspace(0, len(rest) - 1, max(0, k_want - 8)).round().astype(int)] if len(rest) else []
    return sorted(set(big + spread))


def run_batched(args):
    """256 Life/Wa-Tor instances (sides log-uniform 64..1024) on one heap,
    one step = one captured CUDA graph (one parallel_do per class per phase
    over all instances), against the same instances on separate heaps stepped
    one instance at a time (plain launches, and one graph per instance)."""
    import torch
    from paper_1908_05845_gb300 import autotune, smmo
    from paper_1908_05845_gb300.workloads import World, heap_bytes_for
    n_inst = args.instances
    kinds, sides, init = batched_init(SEED, n_inst)
    total = int(np.sum(sides.astype(np.int64) ** 2))
    offs = np.concatenate([[0], np.cumsum(sides.astype(np.int64) ** 2)])
    # tuned on the full set of instances (a sample of them ranked the
    # launch shapes differently from the full world)
    cfg, _ = autotune.tune("batched_life_wator_%d" % n_inst, kinds, sides, SEED, init, steps=10, warm=3,
                           use_cache=not args.retune)
    stream = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(stream):
        # batched: one heap, one graph per step
        w = World(kinds, sides, sides, SEED, *init, config=smmo.default_config(**cfg),
                  heap_bytes=heap_bytes_for(total), stream=stream)
        w.step(args.warmup)
        w.capture(1)
        e0 = w.heap.counters()[0]
        a, b = _events(stream)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            w.replay()
        b.record(stream)
        b.synchronize()
        t_b = a.elapsed_time(b) / 1e3
        objs = w.heap.counters()[0] - e0
        w.sync()
        k_gpu, a_gpu, e_gpu, s_gpu, err = w.export()
        res["batched"] = objs / t_b
        steps_done = args.warmup + args.steps
        w.close()
        # per-instance heaps
        worlds = []
        for i in range(n_inst):
            sl = slice(offs[i], offs[i + 1])
            worlds.append(World([kinds[i]], [sides[i]], [sides[i]], SEED, *(x[sl] for x in init),
                                config=smmo.default_config(**cfg),
                                heap_bytes=heap_bytes_for(int(sides[i]) ** 2), stream=stream, inst_ids=[i]))
        # every per-instance world draws with its instance's number, so both
        # arms simulate the same instances
        for x in worlds:
            x.step(args.warmup)
        e0 = sum(x.heap.counters()[0] for x in worlds)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            for x in worlds:
                x.step(1)
        b.record(stream)
        b.synchronize()
        t_p = a.elapsed_time(b) / 1e3
        objs_p = sum(x.heap.counters()[0] for x in worlds) - e0
        res["per_instance_launches"] = objs_p / t_p
        for x in worlds:
            x.capture(1)
        e0 = sum(x.heap.counters()[0] for x in worlds)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            for x in worlds:
                x.replay()
        b.record(stream)
        b.synchronize()
        t_g = a.elapsed_time(b) / 1e3
        objs_g = sum(x.heap.counters()[0] for x in worlds) - e0
        res["per_instance_graphs"] = objs_g / t_g
        for x in worlds:
            x.close()
    # parity of a sample of instances against the oracle (a spawned pool:
    # the CUDA context exists already)
    import multiprocessing as mp
    import oracle
    from paper_1908_05845_gb300.workloads import LIFE
    checked = []
    jobs = []
    for i in batched_parity_sample(kinds, sides):
        sl = slice(offs[i], offs[i + 1])
        jobs.append((i, int(kinds[i]), int(sides[i]), SEED, *(x[sl] for x in init), steps_done))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        for i, wk, wa, we, ws in pool.imap_unordered(oracle.batched_instance_run, jobs):
            sl = slice(offs[i], offs[i + 1])
            if kinds[i] == LIFE:
                ok = np.array_equal(k_gpu[sl], wk) and np.array_equal(s_gpu[sl], ws)
            else:
                ok = np.array_equal(k_gpu[sl], wk) and np.array_equal(a_gpu[sl], wa) and np.array_equal(e_gpu[sl], we)
            checked.append({"instance": i, "side": int(sides[i]), "kind": "life" if kinds[i] == LIFE else "wator",
                            "bit_exact": bool(ok)})
    checked.sort(key=lambda r: -r["side"])
    line = {"metric": "object-updates/s", "value": res["batched"], "unit": "object-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_b / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/int16",
            "data": "synthetic (seeded Philox)",
            "config": {"workload": "batched_%d_instances" % n_inst, "cells": total,
                       "life_instances": int((kinds == LIFE).sum()), "tuned": cfg,
                       "l2": "working set larger than L2"},
            "per_instance_launches": res["per_instance_launches"],
            "per_instance_graphs": res["per_instance_graphs"],
            "speedup_vs_per_instance_launches": res["batched"] / res["per_instance_launches"],
            "speedup_vs_per_instance_graphs": res["batched"] / res["per_instance_graphs"],
            "export_errors": int(err), "parity_sample": checked}
    print(json.dumps(line), flush=True)
    return 0


def run_gol(args):
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import Life
    k, s = inputs.gol_initial(256, 256, SEED)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        w = Life(256, 256, k, s, stream=stream)
        w.capture(1)
        e0 = w.heap.counters()[0]
        a, b = _events(stream)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            w.replay()
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        objs = w.heap.counters()[0] - e0
        w.sync()
    print(json.dumps({"metric": "object-updates/s", "value": objs / t, "unit": "object-updates/s",
                      "ms_per_step": 1e3 * t / args.steps, "steps": args.steps,
                      "config": {"workload": "life_256x256", "graph": "one CUDA graph per generation"}}),
          flush=True)
    return 0


def run_generation(args):
    """The generation application (Sec. 7.8: Life objects with the Burst
    rule, a dead cell blocked for 255 generations) on a 1024 x 1024 torus
    from 30 % alive, 500 generations as one captured graph per generation;
    once plain and once with compact(n = 2) of Alive and Candidate every 50
    generations (the thesis' defragmentation experiment for this
    application).  Both runs are checked cell for cell against the oracle."""
    import torch
    import oracle
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import Generation
    W = H = 1024
    T = args.gen_steps
    k0, s0 = inputs.gol_initial(W, H, SEED, p=(3, 10))
    t0 = time.time()
    ok_, os_, ob, cnt = oracle.gen_run(W, H, k0, s0, np.zeros(W * H, np.uint16), T, oracle.BURST)
    cpu_s = time.time() - t0
    out = {}
    stream = torch.cuda.Stream()
    for label, every in (("plain", 0), ("compact_every_50", 50)):
        with torch.cuda.stream(stream):
            g = Generation(W, H, k0, s0, stream=stream)
            A, C = g.class_ids["Alive"], g.class_ids["Candidate"]
            g.capture(1)
            a, b = _events(stream)
            c0, c1 = _events(stream)
            e0 = g.heap.counters()[0]
            t_compact = 0.0
            peak_blocks = 0
            torch.cuda.synchronize()
            a.record(stream)
            for t in range(T):
                g.replay()
                if every and (t + 1) % every == 0:
                    c0.record(stream)
                    g.heap.compact(A, n=2, k1=0)
                    g.heap.compact(C, n=2, k1=0)
                    c1.record(stream)
                    c1.synchronize()
                    t_compact += c0.elapsed_time(c1)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            objs = g.heap.counters()[0] - e0
            st = g.heap.stats()
            k, s_, bl = g.read()
            g.close()
        out[label] = {"ms_per_generation": ms / T, "object_updates_per_s": objs / (ms / 1e3),
                      "compaction_ms_total": t_compact,
                      "alive_blocks_end": st["blocks"][A], "candidate_blocks_end": st["blocks"][C],
                      "fragmentation_alive_end": st["fragmentation"][A],
                      "fragmentation_candidate_end": st["fragmentation"][C],
                      "bit_exact": bool(np.array_equal(k, ok_) and np.array_equal(s_, os_)
                                        and np.array_equal(bl, ob))}
    p, c = out["plain"], out["compact_every_50"]
    line = {"metric": "object-updates/s", "value": p["object_updates_per_s"], "unit": "object-updates/s",
            "ms_per_step": p["ms_per_generation"], "steps": T, "higher_is_better": True,
            "dtype": "int32/u16", "data": "synthetic (seeded Philox)",
            "config": {"workload": "generation_burst_1024x1024", "rule": "0235678/3468, blocked 255",
                       "initial_alive": 0.3},
            "runs": out,
            "compaction_speedup": p["ms_per_generation"] / c["ms_per_generation"],
            # every object is visited by two of the four do-alls per generation
            "cpu_baseline": {"value": 2.0 * float(np.sum(cnt[:, :3])) / cpu_s, "unit": "object-updates/s",
                             "cores": 1, "kind": "oracle", "host": host_info(),
                             "sample": "all %d generations (%.1f s)" % (T, cpu_s)}}
    print(json.dumps(line), flush=True)
    return 0 if (p["bit_exact"] and c["bit_exact"]) else 1


def run_bh(args):
    """2-D Barnes-Hut with a dynamic quad tree (Sec. 7.3): 65,536 bodies,
    100 steps (tree summaries, forces, update, removal, reinsertion with
    device new of tree nodes, collapse with device delete).  Parity: a
    separate 10-step run against the oracle at full size."""
    import torch
    import oracle
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import BarnesHut
    N = args.bh_bodies
    P = dict(G=1e-5, eps=1e-2, dt=1e-3, theta=0.5)
    st = inputs.bh_initial(N, SEED)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = BarnesHut(st, stream=stream, **P)
        sim.step(args.warmup)
        e0, a0, f0 = sim.heap.counters()
        l0 = sim.levels()
        a, b = _events(stream)
        torch.cuda.synchronize()
        a.record(stream)
        sim.step(args.steps)
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        e1, a1, f1 = sim.heap.counters()
        l1 = sim.levels()
        _, nodes = sim.read()
        sim.sync()
        sim.close()
        chk = BarnesHut(st, stream=stream, **P)
        chk.step(10)
        got, _ = chk.read()
        chk.close()
    # independent repetitions of the timed run: the device error word of
    # each (a bounded wait that gave up records its site in the detail)
    repeats = []
    for r in range(args.bh_repeat):
        with torch.cuda.stream(stream):
            code, detail = 0, 0
            try:
                rs = BarnesHut(st, stream=stream, **P)
                rs.step(args.warmup + args.steps)
                code, detail = rs.heap.sync(raise_on_error=False)
            except Exception as ex:  # a step that reported an error
                code, detail = rs.heap.sync(raise_on_error=False)
                code = code or getattr(ex, "status", -99)
            rs.close()
        repeats.append({"run": r, "status": int(code), "detail": hex(int(detail))})
    t0 = time.time()
    want, _ = oracle.bh_run(st, 10, **P)
    cpu_s = time.time() - t0
    exact = all(np.array_equal(got[k], want[k]) for k in ("x", "y", "vx", "vy"))
    print(json.dumps({"metric": "bodies/s", "value": N * args.steps / t, "unit": "body-steps/s",
                      "ms_per_step": 1e3 * t / args.steps, "steps": args.steps, "dtype": "f32",
                      "higher_is_better": True, "data": "synthetic (seeded Philox)",
                      "config": {"workload": "barnes_hut_2d_%d" % N, **P},
                      "object_updates_per_s": (e1 - e0) / t,
                      "tree_node_news_per_step": (a1 - a0) / args.steps,
                      "tree_node_deletes_per_step": (f1 - f0) / args.steps,
                      "tree_traversals_per_step": (l1 - l0) / args.steps, "tree_nodes_end": nodes,
                      "parity_10_steps_bit_exact": bool(exact),
                      "repeated_runs": {"runs": len(repeats), "steps_each": args.warmup + args.steps,
                                        "errors": [x for x in repeats if x["status"]]},
                      "cpu_baseline": {"value": N * 10 / cpu_s, "unit": "body-steps/s", "cores": 1,
                                       "kind": "oracle", "host": host_info(), "sample": "10 steps (%.1f s)" % cpu_s}}), flush=True)
    return 0 if exact else 1


def run_bfs(args):
    """Frontier BFS (Sec. 4.3) on a 1043 x 1043 road grid (1,087,849
    vertices, about 3.08 M directed edges: the size of the thesis'
    Pennsylvania road network), one parallel_do_and_reduce per level.
    Timed: the whole search from vertex 0 (best of `reps`); checked against
    the oracle."""
    import torch
    import oracle
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import Bfs
    side = 1043
    rp, col = inputs.road_grid(side, SEED)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = Bfs(rp, col, stream=stream)
        g.run(0, check_every=args.bfs_check)  # warm-up
        a, b = _events(stream)
        best = None
        for _ in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a.record(stream)
            lv = g.run(0, check_every=args.bfs_check)
            b.record(stream)
            b.synchronize()
            wall = time.perf_counter() - t0
            ms = a.elapsed_time(b)
            best = (ms, wall, lv) if best is None or ms < best[0] else best
        d = g.distances()
        g.close()
    t0 = time.time()
    want, wl = oracle.bfs(rp, col, 0)
    cpu_s = time.time() - t0
    ms, wall, lv = best
    edges = int(len(col))
    print(json.dumps({"metric": "traversed edges/s", "value": edges / (ms / 1e3), "unit": "edges/s",
                      "ms_per_search": ms, "wall_ms_per_search": 1e3 * wall, "levels": lv,
                      "ms_per_level": ms / lv, "higher_is_better": True, "dtype": "int32",
                      "data": "synthetic (seeded Philox)",
                      "config": {"workload": "bfs_road_grid_%dx%d" % (side, side), "vertices": side * side,
                                 "directed_edges": edges, "check_every": args.bfs_check},
                      "bit_exact": bool(np.array_equal(d, want) and lv == wl),
                      "cpu_baseline": {"value": edges / cpu_s, "unit": "edges/s", "cores": 1, "kind": "oracle", "host": host_info(),
                                       "sample": "one full search (%.3f s)" % cpu_s}}), flush=True)
    return 0 if np.array_equal(d, want) else 1


def run_structure(args):
    """The spring mesh of Sec. 7.4 (a tensile test of a composite: anchor
    nodes along the bottom row, pull nodes along the top row) on a
    256 x 8192 brick-wall mesh (2,097,152 nodes, about 2.8 M springs;
    --struct-cols narrows it for small profiler captures):
    iterations of pull, 40 compute steps (Spring::compute_force with
    breaking, Node::update) and the BFS removal of parts cut off from the
    anchors.  Timed: `struct_iters` iterations, plain and with compaction of
    Spring and Node (n = 10) every 50 iterations (the thesis' CompactGpu
    setting for this application); the removal alone on the final state.
    Parity: 3 iterations against the oracle at full size (--no-parity skips
    it, for profiler captures)."""
    import torch
    import oracle
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import Structure
    rows, cols, T = 256, args.struct_cols, args.struct_iters
    g = inputs.structure_mesh(rows, cols, SEED)
    stream = torch.cuda.Stream()
    a, b = _events(stream)
    out = {}
    for label, every in (("plain", 0), ("compact_every_50", 50)):
        with torch.cuda.stream(stream):
            sim = Structure(g, stream=stream)
            sim.step(args.warmup)
            e0, a0, f0 = sim.heap.counters()
            c0 = sim.counters()
            ids = sim.class_ids
            t_compact, done = 0.0, 0
            torch.cuda.synchronize()
            a.record(stream)
            while done < T:
                k = min(T - done, every) if every else T
                sim.step(k)
                done += k
                if every and done % every == 0 and done < T:
                    for cname in ("Spring", "Node"):
                        cs = sim.heap.compact(ids[cname], 10, 0)
                        t_compact += cs["scan_ms"] + cs["copy_ms"] + cs["state_ms"] + cs["rewrite_ms"]
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            e1, a1, f1 = sim.heap.counters()
            c1 = sim.counters()
            st = sim.heap.stats()
            # the removal phase alone on the final state
            torch.cuda.synchronize()
            a.record(stream)
            sim.step(5, 4)
            b.record(stream)
            b.synchronize()
            ms_remove = a.elapsed_time(b) / 5
            assert sim.heap.check() == 0
            sim.sync()
            sim.close()
        out[label] = {"ms_per_iteration": ms / T, "object_updates_per_s": (e1 - e0) / (ms / 1e3),
                      "removal_ms_per_iteration": ms_remove, "compaction_ms_total": t_compact,
                      "springs_broken": c1["broken"] - c0["broken"],
                      "nodes_deleted": c1["nodes_deleted"] - c0["nodes_deleted"],
                      "frees_per_s": (f1 - f0) / (ms / 1e3),
                      "bfs_levels_per_iteration": (c1["bfs_levels"] - c0["bfs_levels"]) / T,
                      "node_blocks_end": st["blocks"][ids["Node"]],
                      "spring_blocks_end": st["blocks"][ids["Spring"]],
                      "fragmentation_node_end": st["fragmentation"][ids["Node"]],
                      "fragmentation_spring_end": st["fragmentation"][ids["Spring"]]}
    # parity at full size: 3 iterations
    exact, cpu = None, None
    if not args.no_parity:
        with torch.cuda.stream(stream):
            chk = Structure(g, stream=stream)
            chk.step(3)
            got = chk.read()
            chk.close()
        t0 = time.time()
        want, oc = oracle.structure_run(g, 3)
        cpu_s = time.time() - t0
        alive = want["nalive"].astype(bool)
        exact = bool(np.array_equal(got["nalive"].astype(bool), alive)
                     and np.array_equal(got["salive"].astype(bool), want["salive"].astype(bool))
                     and all(np.array_equal(got[k][alive], want[k][alive])
                             for k in ("x", "y", "nspr", "dist", "slot")))
        # oracle object-updates: per iteration every spring and node twice per
        # compute step plus one node visit per BFS level
        n_obj = len(g["kind"]) + len(g["p1"])
        ou = 3 * (2 * 40 * n_obj) + int(oc[:, 4].sum()) * len(g["kind"])
        cpu = {"value": ou / cpu_s, "unit": "object-updates/s", "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": "3 iterations (%.1f s)" % cpu_s}
    p, c = out["plain"], out["compact_every_50"]
    print(json.dumps({"metric": "object-updates/s", "value": p["object_updates_per_s"], "unit": "object-updates/s",
                      "ms_per_step": p["ms_per_iteration"], "steps": T, "higher_is_better": True, "dtype": "f32",
                      "data": "synthetic (seeded Philox)",
                      "config": {"workload": "structure_%dx%d" % (rows, cols), "nodes": len(g["kind"]),
                                 "springs": len(g["p1"]), "substeps": 40, "dt": 0.05, "damping": 0.01},
                      "runs": out, "compaction_speedup": p["ms_per_iteration"] / c["ms_per_iteration"],
                      "parity_3_iterations_bit_exact": exact, "cpu_baseline": cpu}), flush=True)
    return 0 if exact in (True, None) else 1


def run_wator_compact(args):
    """CompactGpu on Wa-Tor (Sec. 6.4's wa-tor experiment): the 2048 x 2048
    world for 500 steps, plain, with compact(n = 10, k1 = 16) of Fish and
    Shark every 50 steps (and with n = 2), and with the "after massive
    deallocations" policy (Sec. 6.3.8: n = 10, checked every 10 steps, k2 =
    5 % of the heap's blocks).  L2 is not flushed between steps here: the
    runs are compared with each other.
    Reported per run: ms per step (compaction included), compaction time,
    the largest and the final number of allocated Fish + Shark blocks (the
    memory footprint; sampled every 10 steps outside the timed intervals),
    and whether the final world equals the plain run's (placement does not
    change the results)."""
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import WaTor, heap_bytes_for
    W = W_SIDE
    T = 500
    k0, a0, e0 = inputs.wator_initial(W, W, SEED)
    stream = torch.cuda.Stream()
    a, b = _events(stream)
    out, ref = {}, None
    for label, n in (("plain", 0), ("compact_every_50", 10), ("compact_every_50_n2", 2),
                     ("compact_after_massive_deallocations", 10)):
        with torch.cuda.stream(stream):
            sim = WaTor(W, W, SEED, k0, a0, e0, heap_bytes=heap_bytes_for(W * W, 1.0), stream=stream)
            F, S = sim.class_ids["Fish"], sim.class_ids["Shark"]
            ms, t_compact, runs, passes, peak, blocks = 0.0, 0.0, 0, 0, 0, []
            for t0 in range(0, T, 10):
                torch.cuda.synchronize()
                a.record(stream)
                sim.step(10)
                done = t0 + 10
                for cls in (F, S):
                    cs = None
                    if label.startswith("compact_every_50") and done % 50 == 0:
                        cs = sim.heap.compact(cls, n=n, k1=16)
                    elif label == "compact_after_massive_deallocations":
                        ran, cs = sim.heap.compact_if(cls, n=n, k1=16, k2_fraction=0.05)
                        cs = cs if ran else None
                    if cs is not None:
                        runs += 1
                        passes += cs["passes"]
                        t_compact += cs["scan_ms"] + cs["copy_ms"] + cs["state_ms"] + cs["rewrite_ms"]
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
                st = sim.heap.stats()
                nb = st["blocks"][F] + st["blocks"][S]
                blocks.append(nb)
                peak = max(peak, nb)
            world = sim.read()
            sim.sync()
            sim.close()
        same = True
        if ref is None:
            ref = world
        else:
            same = all(np.array_equal(x, y) for x, y in zip(world, ref))
        out[label] = {"n": n, "ms_per_step": ms / T, "compactions": runs, "passes": passes,
                      "compaction_ms_total": t_compact,
                      "peak_blocks": peak, "final_blocks": blocks[-1],
                      "mean_blocks": float(np.mean(blocks)), "world_equals_plain": bool(same)}
    p = out["plain"]
    for k, v in out.items():
        v["slowdown_vs_plain"] = v["ms_per_step"] / p["ms_per_step"]
        v["peak_memory_vs_plain"] = v["peak_blocks"] / p["peak_blocks"]
    print(json.dumps({"metric": "ms/step", "value": p["ms_per_step"], "unit": "ms", "higher_is_better": False,
                      "steps": T, "dtype": "int32/int16", "data": "synthetic (seeded Philox)",
                      "config": {"workload": "wator_%dx%d_compaction" % (W, W), "n": 10, "k1": 16,
                                 "k2_fraction": 0.05},
                      "runs": out}), flush=True)
    return 0 if all(v["world_equals_plain"] for v in out.values()) else 1


def run_nbody_compact(args):
    """CompactGpu on the n-body simulation with collisions (the thesis'
    "collision" benchmark, Sec. 6.4): 65,536 bodies, 600 steps of force,
    update and merge (merged bodies are deleted, so the body blocks empty
    out), plain and with compact of the Body class every 50 steps at n = 10
    and n = 36.  Reported per run: ms per step (compaction included), the
    force pass of the last 50 steps, live bodies and Body blocks at the end;
    the final state must equal the plain run's (forces are summed in id
    order, so placement never changes a result)."""
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.nbody import NBody
    N, T = 65536, 600
    st = inputs.nbody_initial(N, SEED)
    stream = torch.cuda.Stream()
    a, b = _events(stream)
    out, ref = {}, None
    for label, n in (("plain", 0), ("compact_every_50_n10", 10), ("compact_every_50_n36", 36)):
        with torch.cuda.stream(stream):
            w = NBody(st, merge_r=1e-2, stream=stream)
            body = w.heap.class_id("Body")
            ms, ms_last, t_compact, runs = 0.0, 0.0, 0.0, 0
            for t0 in range(0, T, 50):
                torch.cuda.synchronize()
                a.record(stream)
                w.step(50)
                if n and t0 + 50 < T:
                    cs = w.heap.compact(body, n=n, k1=0)
                    t_compact += cs["scan_ms"] + cs["copy_ms"] + cs["state_ms"] + cs["rewrite_ms"]
                    runs += 1
                b.record(stream)
                b.synchronize()
                dt = a.elapsed_time(b)
                ms += dt
                if t0 + 50 == T:
                    ms_last = dt / 50
            hs = w.heap.stats()
            got, merges = w.read()
            w.close()
        live = got["live"].astype(bool)
        same = True
        if ref is None:
            ref = got
        else:
            same = bool(np.array_equal(live, ref["live"].astype(bool))
                        and all(np.array_equal(got[k][live], ref[k][live]) for k in ("x", "y", "z", "vx", "vy", "vz", "m")))
        out[label] = {"n": n, "ms_per_step": ms / T, "ms_per_step_last_50": ms_last, "compactions": runs,
                      "compaction_ms_total": t_compact, "merges": int(merges), "live_end": int(live.sum()),
                      "body_blocks_end": hs["blocks"][body], "fragmentation_end": hs["fragmentation"][body],
                      "state_equals_plain": same}
    p = out["plain"]
    for v in out.values():
        v["speedup_vs_plain"] = p["ms_per_step"] / v["ms_per_step"]
    print(json.dumps({"metric": "ms/step", "value": p["ms_per_step"], "unit": "ms", "higher_is_better": False,
                      "steps": T, "dtype": "f32", "data": "synthetic (seeded Philox)",
                      "config": {"workload": "nbody_65536_collision_compaction", "merge_r": 1e-2},
                      "runs": out}), flush=True)
    return 0 if all(v["state_equals_plain"] for v in out.values()) else 1


def run_nasch(args):
    import torch
    from paper_1908_05845_gb300 import inputs
    from paper_1908_05845_gb300.workloads import Traffic
    g = inputs.nasch_graph(SEED)
    v = inputs.nasch_cars(g, SEED)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        w = Traffic(g, SEED, v, stream=stream)
        w.step(args.warmup)
        e0, a0, f0 = w.heap.counters()
        a, b = _events(stream)
        torch.cuda.synchronize()
        a.record(stream)
        w.step(args.steps)
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        e1, a1, f1 = w.heap.counters()
        w.sync()
    # the same graph with traffic controllers (lights, smart lights, yield)
    kind = inputs.nasch_controllers(g, SEED)
    with torch.cuda.stream(stream):
        w = Traffic(g, SEED, v, stream=stream)
        w.set_controllers(kind, phase_len=8, lookahead=5)
        w.step(args.warmup)
        ce0 = w.heap.counters()[0]
        torch.cuda.synchronize()
        a.record(stream)
        w.step(args.steps)
        b.record(stream)
        b.synchronize()
        tc = a.elapsed_time(b) / 1e3
        ce1 = w.heap.counters()[0]
        w.sync()
    print(json.dumps({"metric": "object-updates/s", "value": (e1 - e0) / t, "unit": "object-updates/s",
                      "alloc_free_per_s": ((a1 - a0) + (f1 - f0)) / t, "ms_per_step": 1e3 * t / args.steps,
                      "steps": args.steps, "config": {"workload": "nasch_2000_streets", "cells": g["num_cells"],
                                                      "cars": int((v >= 0).sum())},
                      "controllers": {"ms_per_step": 1e3 * tc / args.steps, "object_updates_per_s": (ce1 - ce0) / tc,
                                      "guarded_streets": int((kind >= 0).sum()),
                                      "kinds": {"light": int((kind == 0).sum()), "smart": int((kind == 1).sum()),
                                                "yield": int((kind == 2).sum())}}}), flush=True)
    return 0


def run_nbody(args):
    import torch
    from paper_1908_05845_gb300 import inputs, smmo
    from paper_1908_05845_gb300.nbody import NBody
    N = 65536
    st = inputs.nbody_initial(N, SEED)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        w = NBody(st, stream=stream)
        w.step(args.warmup)
        p0 = w.pairs()
        a, b = _events(stream)
        torch.cuda.synchronize()
        a.record(stream)
        w.step(args.steps)
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        pairs = float(w.pairs() - p0)  # live x live per step: merged bodies drop out
        got, merges = w.read()
        live = int(got["live"].sum())
        w.close()
        # adjoint cost: forward with checkpoints vs reverse sweep (50 steps)
        w = NBody(st, merge=False, stream=stream)
        a.record(stream)
        w.forward_ckpt(50, 10)
        b.record(stream)
        b.synchronize()
        t_f = a.elapsed_time(b) / 1e3
        a.record(stream)
        w.backward()
        b.record(stream)
        b.synchronize()
        t_b = a.elapsed_time(b) / 1e3
        w.close()
    # ALU roofline of the force pass (no-merge forward with checkpoints,
    # which is the force kernel plus an O(N) drift): 19 FP32 operations per
    # pair (3 sub, 3 fused multiply-adds for |r|^2 + eps^2, 1 mul, 1 sqrt,
    # 1 div, 1 mul for the weight, 3 fused multiply-adds for the sum; a
    # fused multiply-add counts as two) against the measured fused
    # multiply-add rate of this GPU (two operations per lane and clock)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = (load_peaks() or {}).get("sm_max_mhz", 2070.0)
    derived_tflops = props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12
    fma = ctypes.c_double()
    smmo.check(smmo.lib().smmo_measure_fma_peak(8192, ctypes.byref(fma), smmo._stream(None)), "fma_peak")
    peak_tflops = fma.value / 1e12
    ops = ctypes.c_double()
    smmo.check(smmo.lib().smmo_measure_fp32_peak(8192, ctypes.byref(ops), smmo._stream(None)), "fp32_peak")
    mufu = ctypes.c_double()
    smmo.check(smmo.lib().smmo_measure_mufu_peak(4096, ctypes.byref(mufu), smmo._stream(None)), "mufu_peak")
    fwd_pairs_per_s = float(N) * N * 50 / t_f
    ach_tflops = fwd_pairs_per_s * 19 / 1e12
    print(json.dumps({"metric": "pair-interactions/s", "value": pairs / t, "unit": "pairs/s",
                      "ms_per_step": 1e3 * t / args.steps, "steps": args.steps, "merges": merges,
                      "live_after": live, "adjoint_backward_over_forward": t_b / t_f,
                      "forward_ckpt_ms_per_step": 1e3 * t_f / 50, "backward_ms_per_step": 1e3 * t_b / 50,
                      "dtype": "f32",
                      "roofline": {"bound": "alu", "achieved": ach_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                                   "frac": ach_tflops / peak_tflops, "traffic": None, "kernel": "k_force",
                                   "flops_per_pair": 19,
                                   "peak_source": "measured: FP32 fused multiply-add chains on every SM "
                                                  "(smmo_measure_fma_peak, two operations each)",
                                   "peak_derived": derived_tflops,
                                   # the FP32 instruction rate (one multiply or add per lane and clock)
                                   "fp32_instr_peak_per_s": ops.value,
                                   # the two hardware approximations per pair against the
                                   # special-function pipe's measured rate
                                   "mufu_peak_per_s": mufu.value,
                                   "mufu_frac": fwd_pairs_per_s * 2 / mufu.value if mufu.value else None,
                                   "peak_derived_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz"
                                                          % (props.multi_processor_count, mhz)},
                      "config": {"workload": "nbody_65536_merge",
                                 "note": "force O(N^2), merge search on a uniform grid"}}),
          flush=True)
    return 0


def run_alloc(args):
    """Raw allocation throughput (the thesis' Linux-scalability experiment,
    Sec. 5.6.4): 16,384 threads each allocate n objects of a 64-byte class
    inside one do-all, then every object deletes itself in a second do-all.
    One heap serves every n; its block count is the smallest that holds the
    spawners plus 16,384 x n_max objects in full blocks (heap sized for 100 %
    at n_max = 1024: 1 GiB of object data).  Reported per n: allocations/s
    and frees/s (best of --reps), objects created, and the heap utilisation
    they reach (bytes of live objects over the bytes of the blocks the
    objects may use); at n_max, allocations that find no room leave the
    device error SMMO_E_DEVICE_OOM, and the utilisation says how far the
    allocator got."""
    import torch
    from paper_1908_05845_gb300 import smmo
    threads = 16384
    ns = [int(x) for x in args.alloc_n.split(",")]
    n_max = max(ns)
    cfg = smmo.default_config(block_data_bytes=64 * 64)  # 64 objects of 64 bytes per block

    def make(nbytes):
        h = smmo.Heap(nbytes, cfg)
        D = h.register("Spawner", [("v", smmo.I32)])
        O = h.register("Obj", [("w", smmo.I32, 16)])
        h.freeze()
        return h, D, O

    # smallest buffer whose block count holds the spawners and n_max objects per thread
    spawner_blocks = -(-threads // 64)
    want = spawner_blocks + threads * n_max // 64
    lo, hi = want * 4096, want * 4400 + (64 << 20)
    while hi - lo > 4096:
        mid = (lo + hi) // 2 // 256 * 256
        h, _, _ = make(mid)
        m = h.stats()["num_blocks"]
        h.close()
        del h
        if m >= want:
            hi = mid
        else:
            lo = mid
    h, D, O = make(hi)
    M = h.stats()["num_blocks"]
    h.bulk_new(D, threads, [torch.arange(threads, dtype=torch.int32, device="cuda")])
    obj_capacity = (M - spawner_blocks) * 64
    a, b = _events(None)
    st = torch.cuda.current_stream()
    rows = []
    for n in ns:
        best_a = best_f = None
        live = 0
        oom = False
        for rep in range(args.reps):
            torch.cuda.synchronize()
            a.record(st)
            h.parallel_do(D, "test.alloc_k", smmo.AllocKArgs(O, n, 0, 1, 0, 1))
            b.record(st)
            b.synchronize()
            ta = a.elapsed_time(b) / 1e3
            code, _ = h.sync(raise_on_error=False)
            oom = oom or code == -3  # SMMO_E_DEVICE_OOM
            live = h.stats()["live_objects"][O]
            a.record(st)
            h.parallel_do(O, "test.free_self_if", smmo.FreeSelfIfArgs(0, 0, 0))
            b.record(st)
            b.synchronize()
            tf = a.elapsed_time(b) / 1e3
            h.sync()
            best_a = ta if best_a is None else min(best_a, ta)
            best_f = tf if best_f is None else min(best_f, tf)
        stt = h.stats()
        rows.append({"n": n, "allocs_per_s": live / best_a, "frees_per_s": live / best_f,
                     "alloc_plus_free_per_s": 2 * live / (best_a + best_f),
                     "alloc_ms": 1e3 * best_a, "free_ms": 1e3 * best_f, "objects": live,
                     "requested": threads * n, "utilisation": live / obj_capacity, "device_oom": oom,
                     "live_after_free": stt["live_objects"][O], "free_blocks_after": stt["free_blocks"]})
    h.close()
    print(json.dumps({"metric": "allocations/s", "workload": "alloc_16384_threads_64B",
                      "heap": {"num_blocks": M, "object_blocks": M - spawner_blocks,
                               "object_bytes": obj_capacity * 64,
                               "sized_for": "100 %% at n = %d" % n_max},
                      "thesis_context": "Sec. 5.6.4 (TITAN Xp, 1 GiB heap): utilisation DynaSOAr 96.9 %, "
                                        "BitmapAlloc 98.4 %, Halloc and mallocMC at most 49.8 %",
                      "rows": rows}), flush=True)
    return 0


def run_compact(args):
    """The thesis' synthetic defragmentation benchmark (Sec. 6.4): two
    classes of 32,768,000 objects of 32 bytes pointing at each other at
    random, 60 % of the first class deleted, then one compact(A, n=3, k1=0)
    (all passes).  Timed with CUDA events around the call and per phase
    inside it; the relocation is verified afterwards at full size."""
    import torch
    from paper_1908_05845_gb300.workloads import CompactSynthetic
    n = args.compact_objects
    t0 = time.time()
    w = CompactSynthetic(n, seed=SEED)
    setup_s = time.time() - t0
    h = w.heap
    st0 = h.stats()
    a, b = _events(None)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a.record(stream)
    st = h.compact(w.A, n=3, k1=0)
    b.record(stream)
    b.synchronize()
    total_ms = a.elapsed_time(b)
    st1 = h.stats()
    ver = w.verify()
    obj = 32
    moved, rew, passes = st["objects_moved"], st["pointers_rewritten"], st["passes"]
    # algorithmic bytes: copy = read + write of each moved object and its
    # forwarding handle; rewrite (once, after all passes) = every B
    # reference read plus a forwarding read and a write per rewritten one
    copy_bytes = moved * (2 * obj + 4)
    rewrite_bytes = n * 4 + rew * 8
    hbm = (load_peaks() or {}).get("hbm_gbs")
    copy_gbs = copy_bytes / (st["copy_ms"] * 1e6) if st["copy_ms"] else None
    rew_gbs = rewrite_bytes / (st["rewrite_ms"] * 1e6) if st["rewrite_ms"] else None
    dom = "rewrite" if st["rewrite_ms"] >= st["copy_ms"] else "copy"
    ach = rew_gbs if dom == "rewrite" else copy_gbs
    out = {"metric": "compaction time", "value": total_ms, "unit": "ms", "higher_is_better": False,
           "config": {"workload": "compact_synthetic_2x%d_32B_60pct_n3" % n, "objects_per_class": n,
                      "object_bytes": obj, "killed_fraction": 0.6, "n": 3, "k1": 0},
           "passes": passes, "blocks_freed": st["blocks_freed"], "objects_moved": moved,
           "pointers_rewritten": rew, "phase_ms": {k: st[k + "_ms"] for k in ("scan", "copy", "state", "rewrite")},
           "copy_gbs": copy_gbs, "rewrite_gbs": rew_gbs,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": (ach / hbm) if (ach and hbm) else None, "traffic": None, "phase": dom,
                        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
           "blocks_before": st0["blocks"][w.A], "blocks_after": st1["blocks"][w.A],
           "fragmentation_before": st0["fragmentation"][w.A], "fragmentation_after": st1["fragmentation"][w.A],
           "verify": ver, "setup_s": setup_s}
    w.close()
    print(json.dumps(out), flush=True)
    return 0 if (ver["a_objects_ok"] and ver["b_references_ok"] and ver["heap_violations"] == 0) else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=CONFIG_STEPS)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smmo", choices=["smmo", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched-vs-per-instance and adjoint-over-forward measurements")
    ap.add_argument("--workload", default="wator",
                    choices=["wator", "batched", "gol", "generation", "nasch", "nbody", "bh", "bfs", "alloc",
                             "compact", "structure", "wator_compact", "nbody_compact"])
    ap.add_argument("--bfs-check", type=int, default=1024)
    ap.add_argument("--struct-iters", type=int, default=100)
    ap.add_argument("--struct-cols", type=int, default=8192)
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--step-kernels", default="four_do_alls", choices=sorted(STEP_KERNELS),
                    help="how a Wa-Tor iteration is launched (smmo_world_set_step_kernels)")
    ap.add_argument("--bh-bodies", type=int, default=65536)
    ap.add_argument("--bh-repeat", type=int, default=0,
                    help="extra independent Barnes-Hut runs whose device error words are reported")
    ap.add_argument("--gen-steps", type=int, default=500)
    ap.add_argument("--compact-objects", type=int, default=32_768_000)
    ap.add_argument("--alloc-n", default="1,4,16,64,256,1024")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--retune", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != "wator":
        import torch
        torch.cuda.set_device(local)
        from paper_1908_05845_gb300 import smmo
        smmo.lib()
        return {"batched": run_batched, "gol": run_gol, "generation": run_generation, "nasch": run_nasch,
                "nbody": run_nbody, "bh": run_bh, "bfs": run_bfs, "structure": run_structure,
                "wator_compact": run_wator_compact, "nbody_compact": run_nbody_compact,
                "alloc": run_alloc, "compact": run_compact}[args.workload](args)
    return run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
