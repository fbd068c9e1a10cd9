"""Parity of the cellular workloads (object-based Life, Wa-Tor, batched
instances) against the CPU oracle: bit-exact per-cell object state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.workloads import LIFE, WATOR, Life, WaTor, World  # noqa: E402


def test_wator_small_many_seeds(orc):
    for size in (8, 16):
        for seed in range(1, 41):
            k, a, e = inputs.wator_initial(size, size, seed)
            sim = WaTor(size, size, seed, k, a, e)
            sim.step(30)
            got = sim.read()
            want = orc.wator_run(size, size, seed, k, a, e, 30)
            for g, w in zip(got, want[:3]):
                assert np.array_equal(g, w), (size, seed)
            sim.sync()
            sim.close()


@pytest.mark.parametrize("W,H,T", [(64, 48, 60), (200, 130, 40), (256, 256, 25)])
def test_wator_ragged_sizes(orc, W, H, T):
    k, a, e = inputs.wator_initial(W, H, 3)
    sim = WaTor(W, H, 3, k, a, e)
    for chunk in (1, T - 1):
        sim.step(chunk)
    got = sim.read()
    want = orc.wator_run(W, H, 3, k, a, e, T)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)
    st = sim.heap.stats()
    ids = sim.class_ids
    c = want[3]
    assert st["allocs"][ids["Fish"]] == c[:, 2].sum()
    assert st["allocs"][ids["Shark"]] == c[:, 4].sum()
    assert st["frees"][ids["Fish"]] == c[:, 3].sum()
    assert st["frees"][ids["Shark"]] == c[:, 5].sum()
    assert sim.heap.check() == 0
    sim.sync()


def test_wator_2048_sampled_steps(orc):
    """Full configured size, first steps, compared in full."""
    W = H = 2048
    k, a, e = inputs.wator_initial(W, H, 1)
    sim = WaTor(W, H, 1, k, a, e)
    sim.step(5)
    got = sim.read()
    want = orc.wator_run(W, H, 1, k, a, e, 5)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)
    sim.sync()


def test_life_small_many_seeds(orc):
    for size in (8, 16):
        for seed in range(1, 41):
            k, s = inputs.gol_initial(size, size, seed, p=(3, 10))
            sim = Life(size, size, k, s)
            sim.step(20)
            gk, gs = sim.read()
            wk, ws, _ = orc.gol_run(size, size, k, s, 20)
            assert np.array_equal(gk, wk) and np.array_equal(gs, ws), (size, seed)
            sim.close()


@pytest.mark.parametrize("W,H,T", [(256, 256, 100), (100, 77, 37)])
def test_life_parity(orc, W, H, T):
    k, s = inputs.gol_initial(W, H, 1)
    sim = Life(W, H, k, s)
    sim.step(T)
    gk, gs = sim.read()
    wk, ws, c = orc.gol_run(W, H, k, s, T)
    assert np.array_equal(gk, wk) and np.array_equal(gs, ws)
    st = sim.heap.stats()
    ids = sim.class_ids
    assert st["allocs"][ids["Alive"]] == c[:, 2].sum()
    assert st["frees"][ids["Alive"]] == c[:, 3].sum()
    assert st["allocs"][ids["Candidate"]] == c[:, 3].sum() + c[:, 4].sum()
    assert sim.heap.check() == 0
    sim.sync()


def test_life_glider_on_gpu():
    k = np.zeros(16 * 16, np.uint8)
    for y, x in [(0, 1), (1, 2), (2, 0), (2, 1), (2, 2)]:
        k[y * 16 + x] = 1
    a2 = (k == 1).reshape(16, 16)
    nb = sum(np.roll(np.roll(a2, dy, 0), dx, 1).astype(int) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy)
    k[((~a2) & (nb >= 1)).reshape(-1)] = 2
    sim = Life(16, 16, k, np.zeros(256, np.uint8))
    sim.step(4)
    gk, _ = sim.read()
    want = np.zeros((16, 16), bool)
    for y, x in [(1, 2), (2, 3), (3, 1), (3, 2), (3, 3)]:
        want[y, x] = True
    assert np.array_equal(gk.reshape(16, 16) == 1, want)


def test_batched_mixed_instances(orc):
    kinds, sides = inputs.batched_instances(5, n=12, side_min=8, ratio=8.0)
    seed = 5
    ks, ags, ens, sts = [], [], [], []
    for i, (kd, sd) in enumerate(zip(kinds, sides)):
        if kd == LIFE:
            k, s = inputs.gol_initial(sd, sd, seed, inst=i)
            a, e = np.zeros(sd * sd, np.int16), np.zeros(sd * sd, np.int16)
        else:
            k, a, e = inputs.wator_initial(sd, sd, seed, inst=i)
            s = np.zeros(sd * sd, np.uint8)
        ks.append(k.astype(np.int8)); ags.append(a); ens.append(e); sts.append(s)
    w = World(kinds, sides, sides, seed, np.concatenate(ks), np.concatenate(ags),
              np.concatenate(ens), np.concatenate(sts))
    T = 25
    w.step(T)
    k, a, e, s, err = w.export()
    assert err == 0
    for i, (kd, sd) in enumerate(zip(kinds, sides)):
        gk, ga, ge, gs = (w.split(x)[i] for x in (k, a, e, s))
        if kd == LIFE:
            wk, ws, _ = orc.gol_run(sd, sd, ks[i].astype(np.uint8), sts[i], T)
            assert np.array_equal(gk.astype(np.uint8), wk) and np.array_equal(gs, ws), i
        else:
            wk, wa, we, _ = orc.wator_run(sd, sd, seed, ks[i], ags[i], ens[i], T, inst=i)
            assert np.array_equal(gk, wk) and np.array_equal(ga, wa) and np.array_equal(ge, we), i
    assert w.heap.check() == 0
    w.sync()


def test_graph_replay_matches_plain_steps(orc):
    """A captured step replayed k times advances the simulation exactly like
    k plain steps (the step counter lives in device memory)."""
    import torch
    k, a, e = inputs.wator_initial(64, 64, 9)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = WaTor(64, 64, 9, k, a, e, stream=stream)
        sim.step(2)
        sim.capture(3)
        for _ in range(4):
            sim.replay()
        got = sim.read()
    want = orc.wator_run(64, 64, 9, k, a, e, 14)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)


def test_results_identical_for_every_tuning_choice(orc):
    from paper_1908_05845_gb300 import smmo
    kinds, sides = inputs.batched_instances(4, n=6, side_min=8, ratio=8.0)
    seed = 4
    ks, ags, ens, sts = [], [], [], []
    for i, (kd, sd) in enumerate(zip(kinds, sides)):
        if kd == LIFE:
            kk, s = inputs.gol_initial(sd, sd, seed, inst=i)
            aa, ee = np.zeros(sd * sd, np.int16), np.zeros(sd * sd, np.int16)
        else:
            kk, aa, ee = inputs.wator_initial(sd, sd, seed, inst=i)
            s = np.zeros(sd * sd, np.uint8)
        ks.append(kk.astype(np.int8)); ags.append(aa); ens.append(ee); sts.append(s)
    init = [np.concatenate(x) for x in (ks, ags, ens, sts)]
    outs = []
    for cfg in ({"block_data_bytes": 320, "threads_per_cta": 128, "ctas_per_sm": 4},
                {"block_data_bytes": 640, "threads_per_cta": 512, "ctas_per_sm": 16},
                {"block_data_bytes": 640, "threads_per_cta": 256, "ctas_per_sm": 8},
                {"block_data_bytes": 640, "threads_per_cta": 256, "ctas_per_sm": 8, "bitmap_fanout": 32},
                {"block_data_bytes": 320, "threads_per_cta": 512, "ctas_per_sm": 4, "bitmap_fanout": 32}):
        w = World(kinds, sides, sides, seed, *init, config=smmo.default_config(**cfg))
        w.step(20)
        outs.append(w.export())
        w.close()
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            assert np.array_equal(x, y)
    assert outs[0][4] == 0


@pytest.mark.parametrize("W,H,seed", [(96, 80, 1), (67, 45, 2), (130, 33, 3)])
def test_generation_burst_matches_oracle(orc, W, H, seed):
    """The generation application (Burst rule, dead cells blocked for 255
    generations) equals the oracle cell for cell (kind, is_new, blocked)
    after 300 generations, so blocked cells have expired into Candidates."""
    from paper_1908_05845_gb300.workloads import Generation
    k0, s0 = inputs.gol_initial(W, H, seed, p=(3, 10))
    g = Generation(W, H, k0, s0, seed=seed)
    g.step(300)
    k, s, b = g.read()
    assert g.heap.check() == 0
    g.close()
    ok, os_, ob, cnt = orc.gen_run(W, H, k0, s0, np.zeros(W * H, np.uint16), 300, orc.BURST)
    assert cnt[:, 5].sum() > 0 and cnt[:, 3].sum() > 0
    assert np.array_equal(k, ok) and np.array_equal(s, os_) and np.array_equal(b, ob)


def test_generation_graph_replay_and_rule_switch(orc):
    """Graph replay of the generation world matches plain steps; switching
    the rule back to Life gives Life."""
    import torch
    from paper_1908_05845_gb300.workloads import Generation
    W, H = 64, 48
    k0, s0 = inputs.gol_initial(W, H, 5, p=(3, 10))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = Generation(W, H, k0, s0, stream=stream)
        g.step(5)
        g.capture(1)
        for _ in range(20):
            g.replay()
        k, s, b = g.read()
        g.close()
    ok, os_, ob, _ = orc.gen_run(W, H, k0, s0, np.zeros(W * H, np.uint16), 25, orc.BURST)
    assert np.array_equal(k, ok) and np.array_equal(b, ob)
    g = Generation(W, H, k0, s0, rule=orc.LIFE_RULE)
    g.step(30)
    k, s, b = g.read()
    g.close()
    lk, ls, _ = orc.gol_run(W, H, k0, s0, 30)
    assert np.array_equal(k, lk) and np.array_equal(s, ls) and not b.any()


@pytest.mark.parametrize("kind", [WATOR, LIFE])
def test_thousand_small_tori_in_one_batched_world(orc, kind):
    """1,000 independent 8 x 8 and 16 x 16 tori (500 each, instance i draws
    with instance id i) stepped together in one batched heap; every one
    equals the oracle's run of that instance alone."""
    sides = np.array([8] * 500 + [16] * 500, np.int32)
    n = len(sides)
    seed = 11
    ks, ags, ens, sts = [], [], [], []
    for i, sd in enumerate(sides):
        if kind == LIFE:
            k, s = inputs.gol_initial(int(sd), int(sd), seed, inst=i, p=(3, 10))
            a, e = np.zeros(sd * sd, np.int16), np.zeros(sd * sd, np.int16)
        else:
            k, a, e = inputs.wator_initial(int(sd), int(sd), seed, inst=i)
            s = np.zeros(sd * sd, np.uint8)
        ks.append(k.astype(np.int8)); ags.append(a); ens.append(e); sts.append(s)
    w = World([kind] * n, sides, sides, seed, np.concatenate(ks), np.concatenate(ags), np.concatenate(ens),
              np.concatenate(sts))
    T = 30
    w.step(T)
    k, a, e, s, err = w.export()
    assert err == 0
    assert w.heap.check() == 0
    w.sync()
    w.close()
    for i, sd in enumerate(sides):
        gk, ga, ge, gs = (w.split(x)[i] for x in (k, a, e, s))
        sd = int(sd)
        if kind == LIFE:
            wk, ws, _ = orc.gol_run(sd, sd, ks[i].astype(np.uint8), sts[i], T)
            assert np.array_equal(gk.astype(np.uint8), wk) and np.array_equal(gs, ws), i
        else:
            wk, wa, we, _ = orc.wator_run(sd, sd, seed, ks[i], ags[i], ens[i], T, inst=i)
            assert np.array_equal(gk, wk) and np.array_equal(ga, wa) and np.array_equal(ge, we), i
