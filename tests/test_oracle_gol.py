"""Pins of the object-based Game of Life oracle (thesis Sec. 7.8).

Closed forms: the Alive set must equal dense B3/S23 on the torus; the
Candidate set must equal D_{t+1} & ({c in Cand_t: n_t(c) >= 1} | A_t |
N8(Births_{t+1})); every dead cell with an alive neighbour holds a
Candidate; is_new marks exactly this generation's births; the created,
deleted and allocator-operation counts follow from the dense boards.
"""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs


def dense_step(a):
    n = sum(np.roll(np.roll(a, dy, 0), dx, 1).astype(np.int32)
            for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy)
    return (n == 3) | (a & (n == 2)), n


def n8(mask):
    out = np.zeros_like(mask)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx or dy:
                out |= np.roll(np.roll(mask, dy, 0), dx, 1)
    return out


def from_alive(alive):
    H, W = alive.shape
    kind = np.zeros((H, W), np.uint8)
    kind[alive] = 1
    kind[(~alive) & n8(alive)] = 2
    return kind.reshape(-1), np.zeros(H * W, np.uint8)


def run(orc, alive, T):
    H, W = alive.shape
    k, s = from_alive(alive)
    k, s, c = orc.gol_run(W, H, k, s, T)
    return k.reshape(H, W), s.reshape(H, W), c


def place(H, W, cells):
    a = np.zeros((H, W), bool)
    for y, x in cells:
        a[y % H, x % W] = True
    return a


def test_blinker_period_2(orc):
    a = place(16, 16, [(5, 4), (5, 5), (5, 6)])
    k1, _, _ = run(orc, a, 1)
    assert not np.array_equal(k1 == 1, a)
    k2, _, _ = run(orc, a, 2)
    assert np.array_equal(k2 == 1, a)


def test_glider_period_4(orc):
    g = [(0, 1), (1, 2), (2, 0), (2, 1), (2, 2)]
    a = place(16, 16, g)
    k, _, _ = run(orc, a, 4)
    assert np.array_equal(k == 1, place(16, 16, [(y + 1, x + 1) for y, x in g]))
    k, _, _ = run(orc, a, 64)  # once around the 16x16 torus
    assert np.array_equal(k == 1, a)


def test_block_still(orc):
    a = place(8, 8, [(2, 2), (2, 3), (3, 2), (3, 3)])
    for T in (1, 5):
        k, s, c = run(orc, a, T)
        assert np.array_equal(k == 1, a)
        assert c[:, 2].sum() == 0 and c[:, 3].sum() == 0


def test_all_512_neighbourhoods(orc):
    for pat in range(512):
        a = np.zeros((7, 7), bool)
        for b in range(9):
            if pat >> b & 1:
                a[2 + b // 3, 2 + b % 3] = True
        centre = a[3, 3]
        n = int(a[2:5, 2:5].sum()) - int(centre)
        want = (n == 3) or (centre and n == 2)
        k, _, _ = run(orc, a, 1)
        assert (k[3, 3] == 1) == want, pat


@pytest.mark.parametrize("size", [8, 16])
def test_random_tori_vs_dense(orc, size):
    for seed in range(1, 601 if size == 8 else 401):
        kind0, state0 = inputs.gol_initial(size, size, seed, p=(3, 10))
        alive = (kind0 == 1).reshape(size, size)
        cand = (kind0 == 2).reshape(size, size)
        k, s = kind0, state0
        for t in range(6):
            k, s, c = orc.gol_run(size, size, k, s, 1)
            nxt, n = dense_step(alive)
            births = nxt & ~alive
            K = k.reshape(size, size)
            assert np.array_equal(K == 1, nxt)
            assert np.array_equal(s.reshape(size, size) == 1, births)
            dead = ~nxt
            want_cand = dead & ((cand & (n >= 1)) | alive | n8(births))
            assert np.array_equal(K == 2, want_cand)
            assert np.all((K == 2)[dead & n8(nxt)])
            assert c[0, 0] == nxt.sum() and c[0, 1] == want_cand.sum()
            assert c[0, 2] == births.sum() and c[0, 3] == (alive & ~nxt).sum()
            # candidates without an alive neighbour are deleted; the cells
            # empty after that (and after the births) that touch a birth
            # get one new Candidate each
            deleted = cand & (n == 0)
            empty3 = ~alive & ~(cand & (n >= 1))
            created = empty3 & n8(births)
            assert c[0, 4] == created.sum() and c[0, 5] == deleted.sum()
            # allocator operations: a birth and a death each delete one
            # object and create one; creations and deletions one each
            news = births.sum() + (alive & ~nxt).sum() + created.sum()
            frees = births.sum() + (alive & ~nxt).sum() + deleted.sum()
            assert c[0, 6] == news + frees
            alive, cand = nxt, K == 2


def test_population_bookkeeping_256(orc):
    kind0, state0 = inputs.gol_initial(256, 256, 1)
    k, s, c = orc.gol_run(256, 256, kind0, state0, 30)
    a_prev = int((kind0 == 1).sum())
    for row in c:
        assert row[0] == a_prev - row[3] + row[2]
        a_prev = row[0]
