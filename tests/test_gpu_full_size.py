"""Parity at the configured sizes and lengths, element by element against
the oracle.

* Wa-Tor 2048 x 2048 (thesis Sec. 7.6), all 500 steps, compared at step 100
  (after the first shark births and the fish birth waves) and at step 500;
  the allocator's counters equal the oracle's births and deaths.
* n-body with merging (Sec. 7.1, 7.2), 65,536 bodies, 20 steps: every
  body's position, velocity and mass, the live set and the merges of every
  step (the hashed merge grid at its full bucket load).
* The batched heap: all 256 Life / Wa-Tor instances (sides 64..1021, 44.5 M
  cells) stepped together for 300 steps, three plain steps and 297 replays
  of a captured step graph; every instance equals the oracle's run of that
  instance alone.  The oracle runs the instances in a process pool started
  with "spawn" (each instance single-threaded).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.nbody import NBody  # noqa: E402
from paper_1908_05845_gb300.workloads import LIFE, WaTor, World  # noqa: E402


def test_wator_2048_all_500_steps(orc):
    W = H = 2048
    k, a, e = inputs.wator_initial(W, H, 1)
    sim = WaTor(W, H, 1, k, a, e)
    ids = sim.class_ids
    state, t = (k, a, e), 0
    births = deaths = shark_births = starved = 0
    for T in (100, 400):
        sim.step(T)
        got = sim.read()
        want = orc.wator_run(W, H, 1, *state, T, t0=t)
        for name, g, w in zip(("kind", "age", "energy"), got, want[:3]):
            assert np.array_equal(g, w), (t + T, name, int(np.sum(g != w)))
        c = want[3]
        births += c[:, 2].sum(); deaths += c[:, 3].sum()
        shark_births += c[:, 4].sum(); starved += c[:, 5].sum()
        st = sim.heap.stats()
        assert st["allocs"][ids["Fish"]] == births and st["frees"][ids["Fish"]] == deaths
        assert st["allocs"][ids["Shark"]] == shark_births and st["frees"][ids["Shark"]] == starved
        state, t = want[:3], t + T
    assert shark_births > 0 and births > 0
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()


def test_nbody_65536_with_merging_20_steps(orc):
    N, T = 65536, 20
    st0 = inputs.nbody_initial(N, 1)
    sim = NBody(st0)
    orc.set_threads(0)  # every core: receivers are independent
    want, per_step = orc.nbody_run_f32(st0, T)
    done = 0
    for t in range(T):
        sim.step(1)
        _, merges = sim.read()
        assert merges - done == per_step[t], (t, merges - done, per_step[t])
        done = merges
    got, merges = sim.read()
    assert merges == per_step.sum() > 0
    live = want["live"] == 1
    assert np.array_equal(got["live"], want["live"])
    for key in ("x", "y", "z", "vx", "vy", "vz", "m"):
        assert np.array_equal(got[key][live], want[key][live]), key
    assert sim.heap.stats()["live_objects"][0] == N - merges
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()


def test_batched_256_instances_300_steps(orc):
    seed, T = 1, 300
    kinds, sides, init = inputs.batched_initial(seed, 256)
    offs = np.concatenate([[0], np.cumsum(sides.astype(np.int64) ** 2)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        w = World(kinds, sides, sides, seed, *init, stream=stream)
        w.step(3)
        w.capture(1)
        for _ in range(T - 3):
            w.replay()
        k, a, e, s, err = w.export()
        assert err == 0
        assert w.heap.check() == 0
        w.sync()
        w.close()
    # largest instances first, so the pool finishes together
    jobs = []
    for i in np.argsort(-sides.astype(np.int64), kind="stable"):
        i = int(i)
        sl = slice(offs[i], offs[i + 1])
        jobs.append((i, int(kinds[i]), int(sides[i]), seed, *(x[sl] for x in init), T))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        for i, wk, wa, we, ws in pool.imap_unordered(orc.batched_instance_run, jobs):
            sl = slice(offs[i], offs[i + 1])
            assert np.array_equal(k[sl], wk), ("kind", i, int(sides[i]))
            if kinds[i] == LIFE:
                assert np.array_equal(s[sl], ws), ("state", i)
                assert np.array_equal(a[sl], wa), ("blocked", i)
            else:
                assert np.array_equal(a[sl], wa), ("age", i)
                assert np.array_equal(e[sl], we), ("energy", i)
