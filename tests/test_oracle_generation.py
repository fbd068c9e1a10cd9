"""Pins of the generational-automaton oracle (the thesis' "generation",
an extension of Life, Sec. 7.8).

* With the Life rule and no blocking it is the Life oracle, generation by
  generation (kind and is_new of every cell).
* It equals a textbook Generations automaton on a plain state array
  (0 dead, 1 alive, 1 + k dead and blocking for k generations; an alive
  cell with a neighbour count outside `survive` starts blocking, a blocking
  cell advances and frees its cell after `block` generations, a dead cell
  with a count in `born` becomes alive) on random tori, for short and for
  the thesis' 255-generation blocking; every dead, unblocked cell with
  an alive neighbour holds a Candidate; every counter follows from the
  state arrays before and after the generation.
* Worked cases of the Burst rule: a lone cell survives (0 is in the
  survive set); two touching cells die at once, block for exactly 255
  generations, become Candidates in the 256th and are deleted in the 257th.
"""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs

BURST_S, BURST_B = {0, 2, 3, 5, 6, 7, 8}, {3, 4, 6, 8}


def mask(ns):
    m = 0
    for n in ns:
        m |= 1 << n
    return m


def count8(a):
    return sum(np.roll(np.roll(a, dy, 0), dx, 1).astype(np.int32)
               for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy)


def textbook_step(s, S, B, block):
    """One generation of the Generations automaton with states 0 (dead),
    1 (alive), 2 .. block + 1 (dead, blocking)."""
    n = count8(s == 1)
    out = s.copy()
    alive, dead, blk = s == 1, s == 0, s >= 2
    dies = alive & ~np.isin(n, list(S))
    out[dies] = 2 if block > 0 else 0
    adv = s + 1
    adv[adv > block + 1] = 0
    out[blk] = adv[blk]
    out[dead & np.isin(n, list(B))] = 1
    return out


def objects_from_states(s):
    """Per-cell object arrays for a state array: Alive (blocked = s - 1) on
    alive and blocking cells, Candidates on dead cells with an alive
    neighbour."""
    kind = np.zeros(s.shape, np.uint8)
    kind[s >= 1] = 1
    kind[(s == 0) & (count8(s == 1) >= 1)] = 2
    blocked = np.where(s >= 1, s - 1, 0).astype(np.uint16)
    return kind.reshape(-1), np.zeros(s.size, np.uint8), blocked.reshape(-1)


def states_from_objects(kind, blocked, shape):
    s = np.where(kind == 1, 1 + blocked.astype(np.int32), 0)
    return s.reshape(shape)


def test_life_rule_without_blocking_is_the_life_oracle(orc):
    for seed in (1, 2, 3):
        k0, s0 = inputs.gol_initial(24, 20, seed)
        for T in (1, 7, 30):
            kg, sg, _ = orc.gol_run(24, 20, k0, s0, T)
            kn, sn, bn, _ = orc.gen_run(24, 20, k0, s0, np.zeros(k0.size, np.uint16), T, orc.LIFE_RULE)
            assert np.array_equal(kg, kn) and np.array_equal(sg, sn) and not bn.any()


@pytest.mark.parametrize("block", [1, 3, 17])
def test_equals_textbook_generations_automaton(orc, block):
    rng = np.random.default_rng(block)
    S, B = BURST_S, BURST_B
    for trial in range(4):
        H, W = 14 + trial, 17
        s = np.where(rng.random((H, W)) < 0.3, 1, 0)
        blk = rng.random((H, W)) < 0.1
        s[blk] = rng.integers(2, block + 2, size=int(blk.sum()))
        k, st, bl = objects_from_states(s)
        ref = s
        for t in range(1, 3 * block + 12):
            prev, kprev, n = ref, k.reshape(H, W), count8(ref == 1)
            ref = textbook_step(ref, S, B, block)
            k, st, bl, c = orc.gen_run(W, H, k, st, bl, 1, (mask(S), mask(B), block))
            got = states_from_objects(k, bl, (H, W))
            assert np.array_equal(got, ref), (block, trial, t)
            # counters from the two state arrays: populations, births,
            # deaths, expiries, and the Candidates deleted (no alive
            # neighbour) and created (on cells empty after that, next to a
            # birth)
            births = (prev == 0) & (ref == 1)
            deleted = (kprev == 2) & (n == 0)
            empty3 = (kprev == 0) | deleted
            nb8 = count8(births) >= 1
            want = [(ref == 1).sum(), (ref >= 2).sum(), (k == 2).sum(), births.sum(),
                    ((prev == 1) & (ref != 1)).sum(), (prev == block + 1).sum(),
                    (empty3 & nb8 & ~births).sum(), deleted.sum()]
            assert c[0].tolist() == [int(x) for x in want], (block, trial, t)
            # every dead unblocked cell with an alive neighbour is a Candidate
            need = (ref == 0) & (count8(ref == 1) >= 1)
            assert np.all(k.reshape(H, W)[need] == 2)


def test_burst_with_255_generation_blocking_on_a_random_torus(orc):
    rng = np.random.default_rng(7)
    H, W = 12, 13
    s = np.where(rng.random((H, W)) < 0.35, 1, 0)
    k, st, bl = objects_from_states(s)
    ref = s
    for _ in range(300):
        ref = textbook_step(ref, BURST_S, BURST_B, 255)
    k, st, bl, cnt = orc.gen_run(W, H, k, st, bl, 300, orc.BURST)
    assert np.array_equal(states_from_objects(k, bl, (H, W)), ref)
    assert cnt[:, 5].sum() > 0  # some cells were freed after blocking


def test_lone_cell_survives_under_burst(orc):
    s = np.zeros((9, 9), np.int32)
    s[4, 4] = 1
    k, st, bl = objects_from_states(s)
    k, st, bl, cnt = orc.gen_run(9, 9, k, st, bl, 10, orc.BURST)
    assert k.reshape(9, 9)[4, 4] == 1 and bl.reshape(9, 9)[4, 4] == 0
    assert (k == 2).sum() == 8 and (cnt[:, 3] == 0).all()


def test_touching_pair_blocks_for_exactly_255_generations(orc):
    s = np.zeros((11, 11), np.int32)
    s[5, 5] = s[5, 6] = 1  # one neighbour each: both die in generation 1
    k0, st0, bl0 = objects_from_states(s)

    def at(T):
        k, _, bl, _ = orc.gen_run(11, 11, k0, st0, bl0, T, orc.BURST)
        return k.reshape(11, 11), bl.reshape(11, 11)

    k, bl = at(1)
    assert k[5, 5] == k[5, 6] == 1 and bl[5, 5] == bl[5, 6] == 1
    k, bl = at(255)
    assert k[5, 5] == k[5, 6] == 1 and bl[5, 5] == bl[5, 6] == 255
    k, bl = at(256)
    assert k[5, 5] == k[5, 6] == 2  # replaced by Candidates
    k, bl = at(257)
    assert (k == 0).all()  # no alive neighbour: every Candidate deleted
