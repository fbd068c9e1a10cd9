"""Barnes-Hut with a dynamic quad tree on the GPU (thesis Sec. 7.3) against
the oracle: positions and velocities bit-exact after several steps (the
tree after every collapse is the region quad tree, so thread timing cannot
change the result); the tree-node count equals the oracle's region tree;
heap invariants hold while tree nodes are created and deleted."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.workloads import BarnesHut  # noqa: E402

P = dict(G=1e-3, eps=1e-2, dt=1e-3, theta=0.5)


@pytest.mark.parametrize("N,T,seed", [(1, 3, 1), (2, 5, 1), (257, 10, 2), (3000, 15, 3)])
def test_bit_exact_against_oracle(orc, N, T, seed):
    st = inputs.bh_initial(N, seed)
    sim = BarnesHut(st, **P)
    sim.step(T)
    got, nodes = sim.read()
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()
    want, cnt = orc.bh_run(st, T, **P)
    for k in ("x", "y", "vx", "vy", "m"):
        assert np.array_equal(got[k], want[k]), (k, N, T)
    assert nodes == orc.bh_build(want["x"], want["y"])[0]


def test_theta_zero_and_fast_moving_bodies(orc):
    """theta 0 (every tree node opened) and bodies that cross many squares
    and bounce: still bit-exact, tree still the region tree."""
    st = inputs.bh_initial(800, 4)
    st["vx"] = st["vx"] * 300.0
    st["vy"] = st["vy"] * 300.0
    p = dict(P, theta=0.0, dt=1e-2)
    sim = BarnesHut(st, **p)
    sim.step(12)
    got, nodes = sim.read()
    assert sim.heap.check() == 0
    sim.close()
    want, _ = orc.bh_run(st, 12, **p)
    for k in ("x", "y", "vx", "vy"):
        assert np.array_equal(got[k], want[k]), k
    assert nodes == orc.bh_build(want["x"], want["y"])[0]


def test_clustered_bodies_contended_insertion(orc):
    """20,000 bodies in a 2^-6-wide square: every insertion descends the
    same six levels and competes for the same slots; the tree and the
    trajectory still equal the oracle's.  (Positions are distinct: the
    square holds 2^36 representable points.)"""
    st = inputs.bh_initial(20000, 6)
    st["x"] = (0.5 + st["x"] * 2.0 ** -6).astype(np.float32)
    st["y"] = (0.25 + st["y"] * 2.0 ** -6).astype(np.float32)
    assert len(set(zip(st["x"].tolist(), st["y"].tolist()))) == 20000
    p = dict(P, G=1e-9, dt=1e-4)
    sim = BarnesHut(st, **p)
    sim.step(4)
    got, nodes = sim.read()
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()
    want, _ = orc.bh_run(st, 4, **p)
    for k in ("x", "y", "vx", "vy"):
        assert np.array_equal(got[k], want[k]), k
    assert nodes == orc.bh_build(want["x"], want["y"])[0]


def test_midlines_walls_and_a_large_theta(orc):
    """Boundary cases, bit-exact against the oracle: bodies on the exact
    midlines of squares at several depths (half-open squares); a theta so
    large that only a body's own ancestors are opened; bodies that cross
    the low walls; one that lands exactly on 1 and is clamped below it."""
    g = np.array([0.5, 0.25, 0.75, 0.375, 0.625, 0.125, 0.875], np.float32)
    xs, ys = np.meshgrid(g, g)
    rng = np.random.default_rng(3)
    st = dict(x=xs.reshape(-1), y=ys.reshape(-1), vx=(rng.standard_normal(49) * 1e-3).astype(np.float32),
              vy=(rng.standard_normal(49) * 1e-3).astype(np.float32), m=np.ones(49, np.float32))
    three = dict(x=np.array([0.05, 0.45, 0.9], np.float32), y=np.array([0.05, 0.45, 0.9], np.float32),
                 vx=np.zeros(3, np.float32), vy=np.zeros(3, np.float32), m=np.ones(3, np.float32))
    walls = dict(x=np.array([0.004, 0.6], np.float32), y=np.array([0.003, 0.7], np.float32),
                 vx=np.array([-1.0, 0.2], np.float32), vy=np.array([-0.5, 0.1], np.float32),
                 m=np.ones(2, np.float32))
    land = dict(x=np.array([0.5], np.float32), y=np.array([0.25], np.float32), vx=np.array([0.5], np.float32),
                vy=np.zeros(1, np.float32), m=np.ones(1, np.float32))
    for state, p, T in ((st, P, 8), (st, dict(P, theta=10.0), 8), (three, dict(P, theta=10.0), 5),
                        (walls, dict(P, dt=1e-2), 3), (land, dict(P, dt=1.0), 2)):
        sim = BarnesHut(state, **p)
        sim.step(T)
        got, nodes = sim.read()
        assert sim.heap.check() == 0
        sim.close()
        want, _ = orc.bh_run(state, T, **p)
        for k in ("x", "y", "vx", "vy"):
            assert np.array_equal(got[k], want[k]), (k, len(state["x"]), p)
        assert nodes == orc.bh_build(want["x"], want["y"])[0]
