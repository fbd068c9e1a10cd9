"""The spring mesh of thesis Sec. 7.4 on the GPU against the oracle: node
positions, velocities, spring arrays, spring forces, BFS distances and the
sets of live nodes and springs bit-exact after iterations with cracks and
removals (every deletion is decided by FP32 values computed in a fixed
order, so thread timing cannot change the result); each phase on its own;
heap invariants while springs and nodes are deleted; the full-size mesh."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.workloads import Structure  # noqa: E402

NODE_KEYS = ("x", "y", "vx", "vy", "nspr", "dist", "slot")


def compare(got, want, g, check_dist=True):
    alive = want["nalive"].astype(bool)
    assert np.array_equal(got["nalive"].astype(bool), alive)
    assert np.array_equal(got["salive"].astype(bool), want["salive"].astype(bool))
    for k in NODE_KEYS:
        if k == "dist" and not check_dist:
            continue
        w = want[k][alive]
        if k in ("vx", "vy"):  # anchors export 0
            w = np.where(g["kind"][alive] == 0, np.float32(0), w)
        assert np.array_equal(got[k][alive], w), k
    ls = want["salive"].astype(bool)
    for k in ("fx", "fy"):
        assert np.array_equal(got[k][ls], want[k][ls]), k


@pytest.mark.parametrize("rows,cols,T,seed,vp", [(2, 3, 5, 1, 0.5), (24, 40, 60, 1, 1.0), (40, 70, 40, 2, 1.0),
                                                  (33, 65, 30, 3, 0.5)])
def test_bit_exact_against_oracle(orc, rows, cols, T, seed, vp):
    g = inputs.structure_mesh(rows, cols, seed, v_pull=vp)
    sim = Structure(g)
    sim.step(T)
    got = sim.read()
    cnt = sim.counters()
    assert sim.heap.check() == 0
    sim.sync()
    sim.close()
    want, oc = orc.structure_run(g, T)
    compare(got, want, g)
    assert cnt["broken"] == oc[:, 0].sum()
    assert cnt["nodes_deleted"] == oc[:, 1].sum() + oc[:, 3].sum()
    assert cnt["springs_removed"] == oc[:, 2].sum()
    assert cnt["bfs_levels"] == oc[:, 4].sum()


def test_phases_one_by_one(orc):
    """pull only, compute only (a free mesh with velocities: every node
    moves), removal only (a random graph with many components)."""
    g = inputs.structure_mesh(20, 30, 4)
    for phases, T in ((1, 7), (2, 3), (3, 2)):
        sim = Structure(g, substeps=9)
        sim.step(T, phases)
        got = sim.read()
        sim.close()
        want, _ = orc.structure_run(g, T, substeps=9, phases=phases)
        compare(got, want, g, check_dist=False)
    free = dict(g, kind=np.full(len(g["kind"]), 2, np.int8),
                vx=np.random.default_rng(1).normal(0, 0.1, len(g["kind"])).astype(np.float32))
    sim = Structure(free, damping=0.0, substeps=25)
    sim.step(2, 2)
    got = sim.read()
    sim.close()
    want, _ = orc.structure_run(free, 2, damping=0.0, substeps=25, phases=2)
    compare(got, want, free, check_dist=False)


def random_graph(seed, n=3000):
    rng = np.random.default_rng(seed)
    deg = np.zeros(n, int)
    edges = set()
    for _ in range(20 * n):
        a, b = rng.integers(0, n, 2)
        if a == b or deg[a] >= 3 or deg[b] >= 3 or (min(a, b), max(a, b)) in edges:
            continue
        edges.add((min(a, b), max(a, b)))
        deg[a] += 1
        deg[b] += 1
        if len(edges) >= int(1.1 * n):
            break
    edges = sorted(edges)
    S = len(edges)
    slot = np.full((n, 3), -1, np.int32)
    nspr = np.zeros(n, np.int32)
    for s, (a, b) in enumerate(edges):
        for e in (a, b):
            slot[e, nspr[e]] = s
            nspr[e] += 1
    kind = rng.choice([0, 1, 2], size=n, p=[0.02, 0.03, 0.95]).astype(np.int8)
    xy = rng.uniform(0, 50, (n, 2)).astype(np.float32)
    return dict(kind=kind, x=xy[:, 0], y=xy[:, 1], vx=np.zeros(n, np.float32), vy=np.zeros(n, np.float32),
                m=np.ones(n, np.float32), slot=slot, nspr=nspr, p1=np.array([e[0] for e in edges], np.int32),
                p2=np.array([e[1] for e in edges], np.int32), k=np.ones(S, np.float32),
                L0=np.ones(S, np.float32), fmax=np.full(S, 1e30, np.float32))


@pytest.mark.parametrize("seed,every", [(1, 1), (2, 7), (3, 64)])
def test_removal_on_random_graphs(orc, seed, every):
    g = random_graph(seed)
    sim = Structure(g, bfs_check_every=every)
    sim.step(1, 4)
    got = sim.read()
    cnt = sim.counters()
    assert sim.heap.check() == 0
    sim.close()
    want, oc = orc.structure_run(g, 1, phases=4)
    compare(got, want, g)
    assert cnt["bfs_levels"] == oc[0, 4] and oc[0, 3] > 0


def test_rejects_inconsistent_slots():
    g = inputs.structure_mesh(4, 5, 1)
    bad = dict(g, slot=g["slot"].copy())
    v = int(np.nonzero(g["nspr"] >= 2)[0][0])
    bad["slot"][v, 0] = -1  # the node no longer lists a spring that names it
    with pytest.raises(RuntimeError):
        Structure(bad)


def test_full_size_mesh_two_iterations(orc):
    """The benchmark mesh (256 x 8192 nodes) for two iterations."""
    g = inputs.structure_mesh(256, 8192, 1)
    sim = Structure(g)
    sim.step(2)
    got = sim.read()
    cnt = sim.counters()
    sim.sync()
    sim.close()
    want, oc = orc.structure_run(g, 2)
    compare(got, want, g)
    assert cnt["broken"] == oc[:, 0].sum() and cnt["bfs_levels"] == oc[:, 4].sum()
