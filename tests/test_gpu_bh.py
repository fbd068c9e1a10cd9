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
