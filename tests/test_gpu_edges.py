"""Degenerate inputs of every workload on the GPU, each against the oracle
(or its closed form): empty and full Wa-Tor worlds and a lone shark; an
empty and a completely alive Life board; a street graph without cars
(with and without sources); one and two bodies; a one-vertex graph; a
spring mesh of one row and one without springs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.nbody import NBody  # noqa: E402
from paper_1908_05845_gb300.workloads import Bfs, Life, Structure, Traffic, WaTor  # noqa: E402


def wator_case(orc, W, H, k, T, seed=5):
    a = np.zeros(W * H, np.int16)
    e = np.where(k == 2, 3, 0).astype(np.int16)
    sim = WaTor(W, H, seed, k, a, e)
    sim.step(T)
    got = sim.read()
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()
    want = orc.wator_run(W, H, seed, k, a, e, T)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)
    return got, want[3]


def test_wator_empty_full_and_lone_shark(orc):
    W, H = 64, 48
    got, _ = wator_case(orc, W, H, np.zeros(W * H, np.int8), 10)
    assert (got[0] == 0).all()
    # every cell a fish, no shark: nobody can move, so nobody breeds
    got, c = wator_case(orc, W, H, np.ones(W * H, np.int8), 9)
    assert (got[0] == 1).all() and (got[1] == 9).all() and c[:, 2].sum() == 0
    # a lone shark on an empty torus starves at its third step
    k = np.zeros(W * H, np.int8)
    k[W * 7 + 11] = 2
    got, c = wator_case(orc, W, H, k, 2)
    assert (got[0] == 2).sum() == 1
    got, c = wator_case(orc, W, H, k, 3)
    assert (got[0] == 0).all()


def test_life_empty_and_all_alive(orc):
    W, H = 40, 30
    for kind in (np.zeros(W * H, np.uint8), np.ones(W * H, np.uint8)):  # EMPTY, ALIVE everywhere
        s = np.zeros(W * H, np.uint8)
        sim = Life(W, H, kind, s)
        sim.step(3)
        gk, gs = sim.read()
        assert sim.heap.check() == 0
        sim.close()
        wk, ws, _ = orc.gol_run(W, H, kind, s, 3)
        assert np.array_equal(gk, wk) and np.array_equal(gs, ws)
    assert (wk != 1).all()  # eight alive neighbours each: all of them die at once


def test_traffic_without_cars(orc):
    g = inputs.nasch_graph(4, num_streets=40, n_sources=4, n_sinks=4, len_min=20, len_span=20)
    v = np.full(g["num_cells"], -1, np.int8)
    for src in (0, 1):
        gg = dict(g, sources_enabled=src)
        sim = Traffic(gg, 4, v)
        sim.step(30)
        got = sim.read()
        sim.close()
        want, _ = orc.nasch_run(gg, 4, v, 30)
        assert np.array_equal(got, want)
        assert ((got >= 0).sum() > 0) == bool(src)


@pytest.mark.parametrize("N", [1, 2])
def test_one_and_two_bodies(orc, N):
    st = inputs.nbody_initial(N, 7)
    for merge_r in (5e-3, 2.0):  # the second merges the two bodies at once
        sim = NBody(st, merge_r=merge_r)
        sim.step(5)
        got, merges = sim.read()
        sim.close()
        want, k = orc.nbody_run_f32(st, 5, merge_r=merge_r)
        assert merges == k.sum() and merges == (N - 1 if merge_r > 1 else 0)
        for key in ("x", "y", "z", "vx", "vy", "vz", "m"):
            live = np.asarray(want["live"]).astype(bool)
            assert np.array_equal(got[key][live], want[key][live]), key


def test_single_vertex_graph():
    g = Bfs(np.array([0, 0], np.int32), np.zeros(0, np.int32))
    assert g.run(0) == 1
    assert g.distances().tolist() == [0]
    g.close()


def test_structure_one_row_and_no_springs(orc):
    g = inputs.structure_mesh(1, 50, 2)  # a single row: anchor nodes only
    assert (g["kind"] == 0).all()
    sim = Structure(g)
    sim.step(3)
    got = sim.read()
    sim.close()
    want, _ = orc.structure_run(g, 3)
    assert got["nalive"].all() and want["nalive"].all()
    assert np.array_equal(got["x"], want["x"]) and np.array_equal(got["fx"], want["fx"])
    # three isolated nodes, one of each kind, no spring: the pull node moves,
    # nothing else changes, and the removal (which flags springs) keeps all
    lone = dict(kind=np.array([0, 1, 2], np.int8), x=np.array([0, 1, 2], np.float32),
                y=np.zeros(3, np.float32), vx=np.zeros(3, np.float32), vy=np.array([0, 0.5, 0], np.float32),
                m=np.ones(3, np.float32), slot=np.full((3, 3), -1, np.int32), nspr=np.zeros(3, np.int32),
                p1=np.zeros(0, np.int32), p2=np.zeros(0, np.int32), k=np.zeros(0, np.float32),
                L0=np.zeros(0, np.float32), fmax=np.zeros(0, np.float32))
    sim = Structure(lone)
    sim.step(4)
    got = sim.read()
    sim.close()
    want, _ = orc.structure_run(lone, 4)
    assert got["nalive"].all() and want["nalive"].all()
    for k in ("x", "y", "vx", "vy"):
        assert np.array_equal(got[k], np.where(lone["kind"] == 0, 0, want[k]) if k in ("vx", "vy") else want[k]), k
    assert got["y"][1] > 0 and got["dist"].tolist() == [0, 2**31 - 1, 2**31 - 1]
