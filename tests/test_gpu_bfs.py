"""Frontier BFS with parallel_do_and_reduce (thesis Sec. 4.3, Sec. 3.2.2)
against the oracle: distances equal per vertex (unreachable vertices keep
2^31 - 1), level counts equal, for several sources, batch sizes and graph
shapes (road grids, a path, an isolated source)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.workloads import Bfs  # noqa: E402


@pytest.mark.parametrize("side,seed,check", [(50, 1, 1), (97, 2, 16), (200, 3, 7)])
def test_road_grid(orc, side, seed, check):
    rp, col = inputs.road_grid(side, seed)
    g = Bfs(rp, col)
    for src in (0, side * side // 2 + 3, side * side - 1):
        lv = g.run(src, check_every=check)
        d = g.distances()
        want, wl = orc.bfs(rp, col, src)
        assert np.array_equal(d, want) and lv == wl, (side, src)
    g.sync()
    g.close()


def test_path_and_isolated_vertex(orc):
    n = 1000  # a path 0-1-...-998 and an isolated vertex 999
    src = np.concatenate([np.arange(998), np.arange(1, 999)])
    dst = np.concatenate([np.arange(1, 999), np.arange(998)])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    g = Bfs(rp, dst.astype(np.int32))
    assert g.run(0, check_every=64) == 999
    d = g.distances()
    assert np.array_equal(d[:999], np.arange(999)) and d[999] == 2**31 - 1
    assert g.run(999) == 1 and (g.distances()[:999] == 2**31 - 1).all()
    g.close()
