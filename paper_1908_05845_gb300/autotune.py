"""Autotuner for the heap's launch and layout parameters.

Searches block capacity (through the block data segment size: 320 bytes
gives the cells N_T = 32, 640 bytes N_T = 64), threads per CTA and
CTAs per SM of the persistent do-all grid over their full grid, then the
fan-out of the hierarchical bitmaps (32 or 64 bits per container) at the
best of those, by timing a few steps of a world built from the given
instances (the bench passes all of them) with CUDA events.  Results are
cached in a JSON file keyed by GPU
name, workload and a hash of the library's sources (a rebuilt library is
tuned again).  Every choice computes the same result (tested), so tuning
never changes what the simulation does.
"""
from __future__ import annotations

import glob
import hashlib
import itertools
import json
import os

import numpy as np
import torch

from . import smmo
from .workloads import World, heap_bytes_for

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune_cache.json")
SPACE = {"block_data_bytes": (320, 640), "threads_per_cta": (128, 256, 512), "ctas_per_sm": (4, 8, 16)}
# searched one at a time at the best point of SPACE
FANOUT = {"bitmap_fanout": (64, 32)}
_PKG = os.path.dirname(os.path.abspath(__file__))


def source_hash() -> str:
    """Hash of the CUDA sources and the C header the library is built from."""
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(_PKG, "csrc", "*")))
    files.append(os.path.join(os.path.dirname(_PKG), "include", "smmo.h"))
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _load():
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _key(workload: str) -> str:
    return "%s|%s|%s" % (torch.cuda.get_device_name(), workload, source_hash())


def time_world(cfg: dict, kinds, sides, seed, init, steps: int = 8, warm: int = 2) -> float:
    """Device ms per step of a world with config cfg (heap config fields)."""
    k, a, e, s = init
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        w = World(kinds, sides, sides, seed, k, a, e, s, config=smmo.default_config(**cfg),
                  heap_bytes=heap_bytes_for(int(np.sum(np.asarray(sides, np.int64) ** 2))),
                  stream=stream)
        w.step(warm)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        w.step(steps)
        t1.record(stream)
        t1.synchronize()
        ms = t0.elapsed_time(t1) / steps
        w.sync()
        w.close()
    return ms


def tune(workload: str, kinds, sides, seed, init, space=SPACE, steps: int = 8, use_cache=True,
         extra=FANOUT, warm: int = 2):
    """Best heap config (dict) for the given instance sample: the grid of
    `space`, then each parameter of `extra` in turn at the best point."""
    cache = _load()
    key = _key(workload)
    if use_cache and key in cache:
        return cache[key]["config"], cache[key].get("ms")
    best, best_ms, table = None, None, []
    for vals in itertools.product(*space.values()):
        cfg = dict(zip(space.keys(), vals))
        ms = time_world(cfg, kinds, sides, seed, init, steps, warm)
        table.append((cfg, ms))
        if best_ms is None or ms < best_ms:
            best, best_ms = cfg, ms
    for name, choices in extra.items():
        base = dict(best)
        for v in choices:
            cfg = dict(base, **{name: v})
            if v == choices[0]:  # the default, already timed as `best`
                best = cfg
                continue
            ms = time_world(cfg, kinds, sides, seed, init, steps, warm)
            table.append((cfg, ms))
            if ms < best_ms:
                best, best_ms = cfg, ms
    cache[key] = {"config": best, "ms": best_ms,
                  "table": [{"config": c, "ms": m} for c, m in table]}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1)
    return best, best_ms
