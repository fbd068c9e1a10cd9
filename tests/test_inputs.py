"""The seeded input recipes (synthetic stand-ins for the thesis' inputs):
each generator produces the stated shapes, sizes and distributions, and
its random decisions re-derive from the oracle's separately written
Philox.  Statistical bounds are five standard deviations."""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs


def within(value, mean, sd):
    return abs(value - mean) < 5 * sd


def test_wator_recipe(orc):
    W = H = 2048
    N = W * H
    k, a, e = inputs.wator_initial(W, H, 1)
    x = orc.draw(1, inputs.TAG_INIT, 0, np.arange(N, dtype=np.uint32)).astype(np.uint64)
    fish = x < (30 << 32) // 100
    shark = ~fish & (x < (32 << 32) // 100)
    assert np.array_equal(k == 1, fish) and np.array_equal(k == 2, shark) and (k[~fish & ~shark] == 0).all()
    assert within(fish.sum(), 0.30 * N, np.sqrt(0.21 * N)) and within(shark.sum(), 0.02 * N, np.sqrt(0.0196 * N))
    assert (a == 0).all() and (e[shark] == 3).all() and (e[~shark] == 0).all()
    # another instance draws another stream
    k2, _, _ = inputs.wator_initial(64, 64, 1, inst=5)
    assert not np.array_equal(k2, k[:4096])


@pytest.mark.parametrize("side,p", [(256, (1, 10)), (1024, (3, 10))])
def test_life_recipe(orc, side, p):
    N = side * side
    kind, state = inputs.gol_initial(side, side, 1, p=p)
    alive = orc.draw(1, inputs.TAG_INIT, 0, np.arange(N, dtype=np.uint32)) < (p[0] << 32) // p[1]
    assert np.array_equal(kind == 1, alive) and (state == 0).all()
    q = p[0] / p[1]
    assert within(alive.sum(), q * N, np.sqrt(q * (1 - q) * N))
    a = alive.reshape(side, side)
    nb = sum(np.roll(np.roll(a, dy, 0), dx, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy)
    assert np.array_equal((kind == 2).reshape(side, side), ~a & (nb > 0))


def test_street_graph_and_cars(orc):
    g = inputs.nasch_graph(1)
    S = 2000
    L = g["street_len"]
    assert g["num_streets"] == S and L.min() >= 100 and L.max() <= 500
    assert within(g["num_cells"], S * 300, np.sqrt(S * (401 ** 2 - 1) / 12))
    assert np.array_equal(g["street_start"], np.concatenate([[0], np.cumsum(L)[:-1]]))
    s_ids = np.arange(S, dtype=np.uint32)
    assert np.array_equal(L, 100 + orc.draw(1, inputs.TAG_LEN, 0, s_ids) % 401)
    deg = g["out_deg"]
    want_deg = 1 + orc.draw(1, inputs.TAG_OUTDEG, 0, s_ids) % 3
    want_deg[64:128] = 0
    assert np.array_equal(deg, want_deg)
    assert (g["is_source"][:64] == 1).all() and (g["is_source"][64:] == 0).all()
    assert (deg[64:128] == 0).all() and set(np.unique(np.delete(deg, np.arange(64, 128)))) == {1, 2, 3}
    out = g["out_street"].reshape(S, 3)
    for s in range(S):
        t = out[s, :deg[s]]
        assert len(set(t.tolist())) == deg[s] and (t >= 64).all() and (t != s).all() and (out[s, deg[s]:] == -1).all()
    v = inputs.nasch_cars(g, 1)
    assert (v >= 0).sum() == 200_000 and set(np.unique(v)) == {-1, 0}
    d = orc.draw(1, inputs.TAG_PLACE, 0, np.arange(g["num_cells"], dtype=np.uint32))
    assert d[v >= 0].max() <= d[v < 0].min()  # the cells with the smallest placement draws


def test_controller_kinds(orc):
    g = inputs.nasch_graph(2)
    kind = inputs.nasch_controllers(g, 2)
    S = g["num_streets"]
    out = g["out_street"].reshape(S, 3)
    indeg = np.bincount(np.concatenate([out[s, :g["out_deg"][s]] for s in range(S)]), minlength=S)
    want = (orc.draw(2, inputs.TAG_CTRL, 0, np.arange(S, dtype=np.uint32)) % 3).astype(np.int8)
    assert np.array_equal(kind, np.where(indeg >= 2, want, -1))
    assert set(np.unique(kind[indeg >= 2])) == {0, 1, 2}


def test_nbody_recipe(orc):
    N = 65536
    st = inputs.nbody_initial(N, 1)
    i = np.arange(N, dtype=np.uint32)
    for k, c in enumerate(("x", "y", "z")):
        want = ((orc.draw(1, inputs.TAG_NBODY, k, i).astype(np.float64) + 0.5) / 2.0 ** 32).astype(np.float32)
        assert np.array_equal(st[c], want), c
    for c in ("x", "y", "z"):
        p = st[c].astype(np.float64)
        assert p.min() > 0 and p.max() < 1
        assert within(p.mean(), 0.5, np.sqrt(1 / 12 / N)) and within(p.var(), 1 / 12, np.sqrt(1 / 180 / N))
    lm = np.log(st["m"].astype(np.float64))
    assert within(lm.mean(), 0.0, 0.5 / np.sqrt(N)) and within(lm.std(), 0.5, 0.5 / np.sqrt(2 * N))
    for c in ("vx", "vy", "vz"):
        v = st[c].astype(np.float64)
        assert within(v.mean(), 0.0, 0.01 / np.sqrt(N)) and within(v.std(), 0.01, 0.01 / np.sqrt(2 * N))
    assert (st["live"] == 1).all()
    bh = inputs.bh_initial(N, 1)
    assert all(np.array_equal(bh[k], st[k]) for k in ("x", "y", "vx", "vy", "m"))


def test_batched_recipe(orc):
    kind, side = inputs.batched_instances(1)
    n = 256
    assert side.min() >= 64 and side.max() < 1024 and set(np.unique(kind)) == {0, 1}
    u = orc.draw(1, inputs.TAG_SIDE, 0, np.arange(n, dtype=np.uint32)).astype(np.float64) / 2.0 ** 32
    assert np.array_equal(side, np.floor(64 * 16.0 ** u).astype(np.int32))
    assert within(np.log(side / 64.0).mean() / np.log(16.0), 0.5, np.sqrt(1 / 12 / n))
    assert within((kind == 0).sum(), n / 2, np.sqrt(n / 4))
    assert 40e6 < (side.astype(np.int64) ** 2).sum() < 50e6  # about 44.5 M cells


def test_compaction_recipe():
    n = 100_000
    dead, a_ref, b_ref = inputs.compact_synthetic(n, 1)
    assert within(dead.sum(), 0.6 * n, np.sqrt(0.24 * n))
    assert a_ref.min() >= 0 and a_ref.max() < n and b_ref.min() >= 0 and b_ref.max() < n


def test_road_grid_recipe(orc):
    """Grid edge e (2 v to the right of v, 2 v + 1 below it) is kept iff its
    draw is below floor(0.71 2^32); the CSR lists both directions with
    neighbours in increasing id."""
    side = 64
    rp, col = inputs.road_grid(side, 3)
    n = side * side
    v = np.arange(n)
    thr = (71 << 32) // 100
    right = (v % side + 1 < side) & (orc.draw(3, inputs.TAG_EDGE, 0, (2 * v).astype(np.uint32)) < thr)
    down = (v // side + 1 < side) & (orc.draw(3, inputs.TAG_EDGE, 0, (2 * v + 1).astype(np.uint32)) < thr)
    want = [[] for _ in range(n)]
    for u in np.flatnonzero(right):
        want[u].append(u + 1)
        want[u + 1].append(u)
    for u in np.flatnonzero(down):
        want[u].append(u + side)
        want[u + side].append(u)
    assert rp[0] == 0 and rp[-1] == len(col)
    for u in range(n):
        assert col[rp[u]:rp[u + 1]].tolist() == sorted(want[u]), u


def test_mesh_draws(orc):
    """The spring mesh's random decisions, re-derived from the oracle's
    Philox: node jitter (+-0.15 on both axes), kept candidate links
    (probability 0.9, candidate e = 2 v right / 2 v + 1 up), stiffness
    0.5 + U and break limit 0.005 + 0.045 U, x10 at anchor and pull nodes."""
    rows, cols, seed = 12, 20, 4
    g = inputs.structure_mesh(rows, cols, seed)
    N = rows * cols
    v = np.arange(N)

    def u(step, idx):
        return orc.draw(seed, inputs.TAG_MESH, step, np.asarray(idx, np.uint32)).astype(np.float64) / 2.0 ** 32

    assert np.array_equal(g["x"], (v % cols + (u(0, v) - 0.5) * 0.3).astype(np.float32))
    assert np.array_equal(g["y"], (v // cols + (u(1, v) - 0.5) * 0.3).astype(np.float32))
    p1, p2 = g["p1"].astype(np.int64), g["p2"].astype(np.int64)
    e = 2 * p1 + (p2 == p1 + cols)
    keep = (9 << 32) // 10
    drawn = orc.draw(seed, inputs.TAG_MESH, 4, e.astype(np.uint32)) < keep
    # a link is kept by its draw, or as the only link of a node that kept none
    lonely = ~drawn
    assert all(g["nspr"][p1[j]] == 1 or g["nspr"][p2[j]] == 1 for j in np.flatnonzero(lonely))
    # every existing candidate whose draw keeps it is in the mesh
    kept = set(e.tolist())
    for a in range(N):
        r, c = divmod(a, cols)
        for ee, ok in ((2 * a, c + 1 < cols), (2 * a + 1, r + 1 < rows and (r + c) % 2 == 0)):
            if ok and orc.draw(seed, inputs.TAG_MESH, 4, np.array([ee], np.uint32))[0] < keep:
                assert ee in kept, ee
    assert np.array_equal(g["k"], (0.5 + u(2, e)).astype(np.float32))
    f = 0.005 + 0.045 * u(3, e)
    clamp = (g["kind"][p1] != 2) | (g["kind"][p2] != 2)
    assert np.array_equal(g["fmax"], np.where(clamp, f * 10.0, f).astype(np.float32))
