"""Pins of the Wa-Tor oracle (thesis Sec. 7.6).

Bookkeeping identities, hand-checkable histories (lone fish, lone shark,
the fish phase before the shark phase, a breeding shark,
shark next to a fish, full grid of fish) and an exhaustive check that a
contested cell goes to the requester on the lowest cell index.
"""
import itertools

import numpy as np

from paper_1908_05845_gb300 import inputs


def empty(W, H):
    return np.zeros(W * H, np.int8), np.zeros(W * H, np.int16), np.zeros(W * H, np.int16)


def test_bookkeeping_random(orc):
    for seed in (1, 2, 3):
        k, a, e = inputs.wator_initial(64, 64, seed)
        F, S = int((k == 1).sum()), int((k == 2).sum())
        k2, a2, e2, c = orc.wator_run(64, 64, seed, k, a, e, 120)
        for row in c:
            fish, sharks, fb, eaten, sb, starved = row[:6]
            assert fish == F + fb - eaten
            assert sharks == S + sb - starved
            F, S = fish, sharks
        assert (k2 == 1).sum() == F and (k2 == 2).sum() == S
        assert np.all(a2[k2 == 0] == 0) and np.all(e2[k2 != 2] == 0)
        assert np.all(e2[k2 == 2] >= 1) and np.all(e2[k2 == 2] <= 3)


def test_full_grid_of_fish_never_moves(orc):
    k = np.ones(64, np.int8)
    a = np.zeros(64, np.int16)
    k2, a2, _, c = orc.wator_run(8, 8, 5, k, a, np.zeros(64, np.int16), 7)
    assert np.all(k2 == 1) and np.all(a2 == 7)
    assert c[:, 6].sum() == 0 and c[:, 2].sum() == 0


def test_lone_fish_moves_and_breeds_at_step_4(orc):
    W = H = 16
    k, a, e = empty(W, H)
    k[5 * W + 5] = 1
    pos = 5 * W + 5
    for t in range(1, 6):
        k2, a2, e2, c = orc.wator_run(W, H, 9, k, a, e, 1, t0=t - 1)
        if t <= 4:
            assert c[0, 6] == 1  # a lone fish always has a free neighbour
        fish = np.flatnonzero(k2 == 1)
        if t < 4:
            assert fish.size == 1
            x0, y0, x1, y1 = pos % W, pos // W, fish[0] % W, fish[0] // W
            assert min(abs(x1 - x0), W - abs(x1 - x0)) + min(abs(y1 - y0), H - abs(y1 - y0)) == 1
            pos = fish[0]
        elif t == 4:
            assert fish.size == 2 and pos in fish and c[0, 2] == 1
            assert sorted(a2[fish]) == [0, 0]
        k, a, e = k2, a2, e2


def test_lone_shark_starves_at_step_3(orc):
    k, a, e = empty(16, 16)
    k[40] = 2
    e[40] = 3
    counts = []
    for t in range(3):
        k, a, e, c = orc.wator_run(16, 16, 4, k, a, e, 1, t0=t)
        counts.append(int((k == 2).sum()))
    assert counts == [1, 1, 0]


def test_shark_eats_adjacent_fish(orc):
    W = H = 8
    k, a, e = empty(W, H)
    s, f = 3 * W + 3, 3 * W + 4
    k[s], e[s], k[f] = 2, 3, 1
    k2, a2, e2, c = orc.wator_run(W, H, 1, k, a, e, 1)
    # fish moves first (to some empty cell), shark then hunts only if adjacent
    assert c[0, 3] in (0, 1)
    if c[0, 3] == 1:
        assert (k2 == 1).sum() == 0 and e2[k2 == 2][0] == 3


def test_contested_cell_exhaustive(orc):
    W = H = 5
    tgt = 2 * W + 2
    nbrs = [1 * W + 2, 2 * W + 3, 3 * W + 2, 2 * W + 1]  # up, right, down, left
    for subset in itertools.product([0, 1], repeat=4):
        if not any(subset):
            continue
        k = np.ones(W * H, np.int8)  # fill with fish so requesters see only tgt
        k[tgt] = 0
        for n, on in zip(nbrs, subset):
            if not on:
                k[n] = 0  # empty
        # non-requesting neighbour positions hold sharks with one unit of
        # energy left: they block the fish phase and starve (without moving)
        # in the shark phase, so the fish phase's outcome is what remains
        e = np.zeros(W * H, np.int16)
        for n, on in zip(nbrs, subset):
            if not on:
                k[n] = 2
                e[n] = 1
        for seed in (1, 2):
            k2, _, _, c = orc.wator_run(W, H, seed, k, np.zeros(W * H, np.int16), e, 1)
            reqs = [n for n, on in zip(nbrs, subset) if on]
            winner = min(reqs)
            assert k2[tgt] == 1
            assert k2[winner] == 0, (subset, seed)
            for r in reqs:
                if r != winner:
                    assert k2[r] == 1


def test_breed_threshold_reading(orc):
    W = H = 16
    k, a, e = empty(W, H)
    k[100] = 1
    k4, *_ = orc.wator_run(W, H, 3, k, a, e, 4)
    k4s, *_ = orc.wator_run(W, H, 3, k, a, e, 4, breed_strict=1)
    assert (k4 == 1).sum() == 2 and (k4s == 1).sum() == 1


def test_deterministic(orc):
    k, a, e = inputs.wator_initial(48, 48, 7)
    r1 = orc.wator_run(48, 48, 7, k, a, e, 40)
    r2 = orc.wator_run(48, 48, 7, k, a, e, 40)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)
    # splitting the run in two gives the same state
    m = orc.wator_run(48, 48, 7, k, a, e, 15)
    s = orc.wator_run(48, 48, 7, m[0], m[1], m[2], 25, t0=15)
    for x, y in zip(r1[:3], s[:3]):
        assert np.array_equal(x, y)


def test_fish_phase_precedes_shark_phase(orc):
    """A 3x1 torus leaves every agent one choice, so the draws do not matter:
    the fish at 0 moves to the empty cell 2 in the fish phase, then the shark
    at 1 hunts it there (Sec. 7.6: the fish phase runs before the shark
    phase, a shark prefers a neighbouring fish and is fed on eating)."""
    k = np.array([1, 2, 0], np.int8)
    a = np.zeros(3, np.int16)
    e = np.array([0, 3, 0], np.int16)
    k2, a2, e2, c = orc.wator_run(3, 1, 11, k, a, e, 1)
    assert k2.tolist() == [0, 0, 2]
    assert e2[2] == 3 and a2[2] == 1
    fish, sharks, fb, eaten, sb, starved, fmoves, smoves = c[0]
    assert (fish, sharks, fb, eaten, sb, starved, fmoves, smoves) == (0, 1, 0, 1, 0, 0, 1, 1)


def test_ripe_shark_leaves_a_fed_newborn(orc):
    """A lone shark one step short of breeding age moves and breeds: the
    newborn on the old cell starts with age 0 and a full energy reserve, the
    parent's age is reset and its energy has dropped by one."""
    W = H = 8
    k, a, e = empty(W, H)
    s = 3 * W + 3
    k[s], a[s], e[s] = 2, 11, 3
    k2, a2, e2, c = orc.wator_run(W, H, 2, k, a, e, 1)
    sharks = np.flatnonzero(k2 == 2)
    assert sharks.size == 2 and s in sharks and c[0, 4] == 1
    assert e2[s] == 3 and a2[s] == 0
    (p,) = [x for x in sharks if x != s]
    assert e2[p] == 2 and a2[p] == 0
    assert abs(p % W - s % W) + abs(p // W - s // W) == 1
