"""Wa-Tor in every step-kernel mode (four do-alls; each species' prepare and
update in one cooperative launch with the request words kept in shared
memory; creations queued for a launch of their own; updates run only on
the agents their prepare marked): bit-exact against the oracle, including
warps whose units do not all fit the shared carry, mode switches between
steps, graph replay, and batched worlds mixing Life and Wa-Tor instances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs, smmo  # noqa: E402
from paper_1908_05845_gb300.workloads import (FOUR_DO_ALLS, LIFE, MARKED, PHASED1, PHASED2, QUEUED,  # noqa: E402
                                              WATOR, WaTor, World)

MODES = [FOUR_DO_ALLS, PHASED1, PHASED2, FOUR_DO_ALLS | QUEUED, PHASED1 | QUEUED, PHASED2 | QUEUED,
         FOUR_DO_ALLS | MARKED, FOUR_DO_ALLS | MARKED | QUEUED]


@pytest.mark.parametrize("mode", MODES)
def test_small_tori_many_seeds(orc, mode):
    for size in (8, 13, 16):
        for seed in range(1, 21):
            k, a, e = inputs.wator_initial(size, size, seed)
            sim = WaTor(size, size, seed, k, a, e, step_kernels=mode)
            sim.step(30)
            got = sim.read()
            want = orc.wator_run(size, size, seed, k, a, e, 30)
            for g, w in zip(got, want[:3]):
                assert np.array_equal(g, w), (mode, size, seed)
            assert sim.heap.check() == 0
            sim.sync()
            sim.close()


@pytest.mark.parametrize("mode", MODES[1:])
@pytest.mark.parametrize("W,H,T", [(64, 48, 60), (200, 130, 40)])
def test_ragged_sizes_and_counters(orc, mode, W, H, T):
    k, a, e = inputs.wator_initial(W, H, 5)
    sim = WaTor(W, H, 5, k, a, e, step_kernels=mode)
    sim.step(T)
    got = sim.read()
    want = orc.wator_run(W, H, 5, k, a, e, T)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)
    st = sim.heap.stats()
    ids = sim.class_ids
    c = want[3]
    assert st["allocs"][ids["Fish"]] == c[:, 2].sum() and st["frees"][ids["Fish"]] == c[:, 3].sum()
    assert st["allocs"][ids["Shark"]] == c[:, 4].sum() and st["frees"][ids["Shark"]] == c[:, 5].sum()
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()


@pytest.mark.parametrize("mode", [PHASED1, PHASED2, PHASED2 | QUEUED])
def test_units_beyond_the_shared_carry(orc, mode):
    """One CTA per SM: a 1024 x 1024 torus gives every warp more units than
    the shared carry holds, so the rest go through the target field."""
    W = H = 1024
    k, a, e = inputs.wator_initial(W, H, 2)
    cfg = smmo.default_config(ctas_per_sm=1)
    sim = WaTor(W, H, 2, k, a, e, step_kernels=mode, config=cfg)
    sim.step(20)
    got = sim.read()
    want = orc.wator_run(W, H, 2, k, a, e, 20)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()


def test_modes_switch_between_steps_and_graph_replay(orc):
    W, H, seed = 300, 200, 7
    k, a, e = inputs.wator_initial(W, H, seed)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = WaTor(W, H, seed, k, a, e, stream=stream, step_kernels=FOUR_DO_ALLS)
        sim.step(3)
        sim.set_step_kernels(PHASED1)
        sim.step(4)
        sim.set_step_kernels(FOUR_DO_ALLS | QUEUED)
        sim.step(2)
        sim.set_step_kernels(FOUR_DO_ALLS | MARKED)
        sim.step(3)
        sim.set_step_kernels(PHASED2)
        sim.step(2)
        sim.capture(3)
        for _ in range(4):
            sim.replay()
        got = sim.read()
        sim.sync()
        sim.close()
    want = orc.wator_run(W, H, seed, k, a, e, 3 + 4 + 2 + 3 + 2 + 12)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)


def test_unknown_mode_is_rejected():
    k, a, e = inputs.wator_initial(16, 16, 1)
    sim = WaTor(16, 16, 1, k, a, e)
    for bad in (3, 7, 9, 10, 16, -1):
        with pytest.raises(smmo.SmmoError):
            sim.set_step_kernels(bad)
    sim.close()


@pytest.mark.parametrize("mode", [FOUR_DO_ALLS, PHASED2, FOUR_DO_ALLS | QUEUED, PHASED2 | QUEUED,
                                  FOUR_DO_ALLS | MARKED])
def test_batched_life_and_wator_in_every_mode(orc, mode):
    seed = 3
    kinds, sides, init = inputs.batched_initial(seed, 24, side_min=16, ratio=10.0)
    offs = np.concatenate([[0], np.cumsum(sides.astype(np.int64) ** 2)])
    w = World(kinds, sides, sides, seed, *init, step_kernels=mode)
    w.step(25)
    k, a, e, s, err = w.export()
    assert err == 0 and w.heap.check() == 0
    w.sync()
    w.close()
    for i in range(len(kinds)):
        sl = slice(offs[i], offs[i + 1])
        _, wk, wa, we, ws = orc.batched_instance_run((i, int(kinds[i]), int(sides[i]), seed,
                                                      *(x[sl] for x in init), 25))
        assert np.array_equal(k[sl], wk), (mode, i)
        if kinds[i] == LIFE:
            assert np.array_equal(s[sl], ws) and np.array_equal(a[sl], wa), (mode, i)
        else:
            assert kinds[i] == WATOR
            assert np.array_equal(a[sl], wa) and np.array_equal(e[sl], we), (mode, i)
