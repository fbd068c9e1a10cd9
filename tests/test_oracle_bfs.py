"""Pins of the BFS-distance oracle and the road-grid input (thesis Sec. 4.3
frontier BFS): Manhattan distances on a complete grid; scipy's unweighted
shortest paths on random graphs and on the road grid; the road grid is
symmetric with the thesis' road-network average degree."""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def test_complete_grid_is_manhattan(orc):
    side = 37
    rp, col = inputs.road_grid(side, 1, keep=(1, 1))
    for src in (0, 5 * side + 11, side * side - 1):
        d, lv = orc.bfs(rp, col, src)
        v = np.arange(side * side)
        want = np.abs(v % side - src % side) + np.abs(v // side - src // side)
        assert np.array_equal(d, want) and lv == want.max() + 1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_against_scipy(orc, seed):
    rng = np.random.default_rng(seed)
    n = 3000
    m = rng.integers(0, n, size=(9000, 2))
    a = scipy_sparse.csr_matrix((np.ones(len(m)), (m[:, 0], m[:, 1])), shape=(n, n))
    a = ((a + a.T) > 0).astype(np.int8).tocsr()
    a.sort_indices()
    d, _ = orc.bfs(a.indptr, a.indices, 7)
    ref = csgraph.shortest_path(a, unweighted=True, indices=7)
    reach = np.isfinite(ref)
    assert np.array_equal(d[reach], ref[reach].astype(np.int32)) and (d[~reach] == 2**31 - 1).all()


def test_road_grid(orc):
    side = 120
    rp, col = inputs.road_grid(side, 4)
    n = side * side
    a = scipy_sparse.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    assert (a != a.T).nnz == 0 and a.diagonal().sum() == 0
    deg = len(col) / n
    assert abs(deg - 2 * 0.71 * 2 * (1 - 1 / side)) < 0.05
    d, _ = orc.bfs(rp, col, 0)
    ref = csgraph.shortest_path(a, unweighted=True, indices=0)
    reach = np.isfinite(ref)
    assert reach.mean() > 0.8
    assert np.array_equal(d[reach], ref[reach].astype(np.int32))
