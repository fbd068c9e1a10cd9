"""Seeded synthetic inputs for the SMMO workloads.

This module builds the initial states that both the CUDA library and the
CPU oracle consume.  It holds no step of the method itself: it only turns a
seed into initial object populations, a street graph and n-body initial
conditions.  Its Philox4x32-10 (Salmon et al., SC'11, Sec. 3.2 and Table 2)
is a third, independent, vectorised numpy implementation.

Recipes (thesis workloads of Ch. 7 with the sizes of the benchmark
configurations; the thesis' own inputs -- a Turing-machine Life pattern and
OpenStreetMap street networks -- are not available, these stand in for them):

* Life: cell c alive iff draw(INIT, 0, c) < floor(0.1 * 2^32); a Candidate on
  every dead cell with at least one alive neighbour (torus).
* Wa-Tor: x = draw(INIT, 0, c); Fish if x < floor(0.30 * 2^32), else Shark if
  x < floor(0.32 * 2^32); ages 0, sharks start with energy `starve`.
* Streets: 2000 one-way streets of length 100 + draw(LEN, 0, s) % 401; streets
  0..63 are producers (no incoming), 64..127 sinks (no outgoing); every other
  street ends in an intersection with 1 + draw(OUTDEG, 0, s) % 3 distinct
  outgoing non-producer streets other than s, picked by successive draws
  draw(OUT, i, s); 200,000 cars (v = 0) on the cells with the smallest
  draw(PLACE, 0, c) (ties by c); a street with two or more incoming streets
  gets controller kind draw(CTRL, 0, s) % 3 (traffic light, smart traffic
  light, yield).
* N-body: per body i uniforms u_k = (draw(NBODY, k, i) + 0.5) / 2^32,
  positions u_0..u_2 in [0,1)^3, masses exp(0.5 z) and velocities N(0, 0.01)
  from Box-Muller on u_3..u_10 in float64, rounded to float32 once.
* Barnes-Hut (2-D): the x, y, vx, vy, m of the n-body recipe.
* BFS: a grid of side x side vertices whose edges are kept with
  probability 0.71 each (draw(EDGE, 0, e)), both directions.
* Structure (stand-in for the thesis' generated random mesh): a brick-wall
  (hexagonal) lattice of rows x cols nodes, node v = r cols + c at
  (c + jx, r + jy) with jitter (u - 0.5) 0.3 from draw(MESH, 0 / 1, v); a
  spring to the right neighbour (candidate 2 v) and, when r + c is even, to
  the node above (candidate 2 v + 1), each kept iff draw(MESH, 4, e) <
  floor(keep 2^32) (a node that would keep none keeps its first
  candidate); row 0 anchor nodes, the top row pull nodes moving up with
  v_pull, ordinary nodes elsewhere (mass 1); per spring stiffness
  0.5 + u and break limit f_lo + (f_hi - f_lo) u (draw(MESH, 2 / 3, e)),
  times `grip` for a spring at an anchor or pull node (the clamps of a
  tensile test), rest length the initial distance (float64, rounded once).
* Batched: instance i is Life if draw(KIND, 0, i) & 1 else Wa-Tor, side
  floor(64 * 16^u) with u = draw(SIDE, 0, i) / 2^32 (log-uniform 64..1024).
* Compaction (the thesis' synthetic defragmentation benchmark, Sec. 6.4):
  two classes of n objects each that point at each other at random; object
  i of the first class dies iff draw(KILL, 0, i) < floor(0.6 * 2^32), refers
  to object draw(AREF, 0, i) % n of the second class, and object j of the
  second class refers to object draw(BREF, 0, j) % n of the first class
  (null when that one dies).
"""
from __future__ import annotations

import numpy as np

TAG_INIT, TAG_FISH, TAG_SHARK, TAG_LEN, TAG_PLACE, TAG_ROUTE, TAG_BRAKE = 0, 1, 2, 3, 4, 5, 6
TAG_KIND, TAG_SIDE, TAG_OUTDEG, TAG_OUT, TAG_NBODY = 7, 8, 9, 10, 11
TAG_KILL, TAG_AREF, TAG_BREF, TAG_CTRL, TAG_EDGE, TAG_MESH = 12, 13, 14, 15, 16, 17

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; all arguments broadcast to uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint32) for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (c.astype(np.uint32).copy() for c in (c0, c1, c2, c3))
    k0 = np.uint32(int(k0) & 0xFFFFFFFF)
    k1 = np.uint32(int(k1) & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = np.uint32(k0 + _W0)
                k1 = np.uint32(k1 + _W1)
            p0 = c0.astype(np.uint64) * _M0
            p1 = c2.astype(np.uint64) * _M1
            hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & _MASK).astype(np.uint32)
            hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & _MASK).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def draw(seed: int, tag: int, step, cell, inst=0) -> np.ndarray:
    """Word 0 of Philox4x32-10, key (seed mod 2^32, seed >> 32), counter
    (step, cell, tag, inst)."""
    seed = int(seed)
    return philox4x32_10(step, cell, tag, inst, seed & 0xFFFFFFFF, seed >> 32)[0]


def threshold(p_num: int, p_den: int) -> int:
    """floor(p * 2^32) for a rational p = p_num / p_den, in integers."""
    return (p_num << 32) // p_den


# ---------------------------------------------------------------- Life
def gol_initial(W: int, H: int, seed: int, inst: int = 0, p=(1, 10)):
    c = np.arange(W * H, dtype=np.uint32)
    alive = draw(seed, TAG_INIT, 0, c, inst) < np.uint32(threshold(*p))
    a2 = alive.reshape(H, W)
    nb = sum(np.roll(np.roll(a2, dy, 0), dx, 1).astype(np.int32)
             for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy)
    kind = np.zeros((H, W), np.uint8)
    kind[a2] = 1
    kind[(~a2) & (nb >= 1)] = 2
    return kind.reshape(-1), np.zeros(W * H, np.uint8)


# -------------------------------------------------------------- Wa-Tor
def wator_initial(W: int, H: int, seed: int, inst: int = 0, starve: int = 3,
                  p_fish=(30, 100), p_shark=(32, 100)):
    c = np.arange(W * H, dtype=np.uint32)
    x = draw(seed, TAG_INIT, 0, c, inst).astype(np.uint64)
    kind = np.zeros(W * H, np.int8)
    fish = x < threshold(*p_fish)
    shark = (~fish) & (x < threshold(*p_shark))
    kind[fish] = 1
    kind[shark] = 2
    age = np.zeros(W * H, np.int16)
    energy = np.where(shark, starve, 0).astype(np.int16)
    return kind, age, energy


# -------------------------------------------------------------- streets
def nasch_graph(seed: int, num_streets: int = 2000, n_sources: int = 64, n_sinks: int = 64,
                len_min: int = 100, len_span: int = 401, p_brake=(1, 5)):
    s = np.arange(num_streets, dtype=np.uint32)
    length = (len_min + draw(seed, TAG_LEN, 0, s) % np.uint32(len_span)).astype(np.int32)
    start = np.zeros(num_streets, np.int32)
    start[1:] = np.cumsum(length[:-1])
    out_deg = (1 + draw(seed, TAG_OUTDEG, 0, s) % np.uint32(3)).astype(np.int32)
    is_source = np.zeros(num_streets, np.uint8)
    is_source[:n_sources] = 1
    out_deg[n_sources:n_sources + n_sinks] = 0
    out = np.full((num_streets, 3), -1, np.int32)
    n_targets = num_streets - n_sources
    for st in range(num_streets):
        k = int(out_deg[st])
        i = 0
        got = []
        while len(got) < k:
            r = int(draw(seed, TAG_OUT, i, st))
            i += 1
            o = n_sources + r % n_targets
            if o != st and o not in got:
                got.append(o)
        out[st, :k] = got
    return dict(num_streets=num_streets, street_start=start, street_len=length,
                out_deg=out_deg, out_street=out.reshape(-1), is_source=is_source,
                num_cells=int(length.sum()), v_max=5, brake_threshold=threshold(*p_brake),
                sources_enabled=1, sinks_enabled=1)


def nasch_controllers(graph: dict, seed: int):
    """Controller kind per street: -1 for streets with fewer than two
    incoming streets, else draw(CTRL, 0, street) % 3 (0 traffic light,
    1 smart traffic light, 2 yield controller)."""
    S = int(graph["num_streets"])
    indeg = np.zeros(S, np.int64)
    out = np.asarray(graph["out_street"]).reshape(S, 3)
    for s in range(S):
        for k in range(int(graph["out_deg"][s])):
            indeg[out[s, k]] += 1
    kind = (draw(seed, TAG_CTRL, 0, np.arange(S, dtype=np.uint32)) % np.uint32(3)).astype(np.int8)
    kind[indeg < 2] = -1
    return kind


def nasch_cars(graph: dict, seed: int, n_cars: int = 200_000):
    C = graph["num_cells"]
    c = np.arange(C, dtype=np.uint32)
    d = draw(seed, TAG_PLACE, 0, c)
    order = np.lexsort((c, d))[:n_cars]
    car_v = np.full(C, -1, np.int8)
    car_v[order] = 0
    return car_v


# -------------------------------------------------------------- n-body
def nbody_initial(N: int, seed: int, sigma_m: float = 0.5, sigma_v: float = 0.01):
    i = np.arange(N, dtype=np.uint32)
    u = [(draw(seed, TAG_NBODY, k, i).astype(np.float64) + 0.5) / 2.0 ** 32 for k in range(11)]

    def normal(a, b):
        return np.sqrt(-2.0 * np.log(a)) * np.cos(2.0 * np.pi * b)

    z = normal(u[3], u[4])
    st = dict(x=u[0].astype(np.float32), y=u[1].astype(np.float32), z=u[2].astype(np.float32),
              m=np.exp(sigma_m * z).astype(np.float32),
              vx=(sigma_v * normal(u[5], u[6])).astype(np.float32),
              vy=(sigma_v * normal(u[7], u[8])).astype(np.float32),
              vz=(sigma_v * normal(u[9], u[10])).astype(np.float32),
              live=np.ones(N, np.uint8))
    return st


def bh_initial(N: int, seed: int):
    """2-D Barnes-Hut bodies: the x, y, vx, vy and m of the n-body recipe."""
    st = nbody_initial(N, seed)
    return {k: st[k] for k in ("x", "y", "vx", "vy", "m")}


def road_grid(side: int, seed: int, keep=(71, 100)):
    """A road-network-like graph (stand-in for the thesis' Pennsylvania road
    network, avg. degree 2.83): side x side grid vertices, each grid edge
    kept iff draw(EDGE, 0, e) < floor(keep * 2^32) (edge e = 2 v for the
    edge to the right of v, 2 v + 1 for the one below), both directions.
    Returns CSR (row_ptr, col) with neighbours in increasing id."""
    n = side * side
    v = np.arange(n, dtype=np.int64)
    x, y = v % side, v // side
    thr = np.uint64(threshold(*keep))  # up to 2^32 (keep every edge)
    right = (x + 1 < side) & (draw(seed, TAG_EDGE, 0, (2 * v).astype(np.uint32)).astype(np.uint64) < thr)
    down = (y + 1 < side) & (draw(seed, TAG_EDGE, 0, (2 * v + 1).astype(np.uint32)).astype(np.uint64) < thr)
    src = np.concatenate([v[right], v[right] + 1, v[down], v[down] + side])
    dst = np.concatenate([v[right] + 1, v[right], v[down] + side, v[down]])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, src + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), dst.astype(np.int32)


# -------------------------------------------------------------- batched
LIFE, WATOR = 0, 1


def batched_instances(seed: int, n: int = 256, side_min: int = 64, ratio: float = 16.0):
    i = np.arange(n, dtype=np.uint32)
    kind = np.where(draw(seed, TAG_KIND, 0, i) & np.uint32(1), LIFE, WATOR).astype(np.int32)
    u = draw(seed, TAG_SIDE, 0, i).astype(np.float64) / 2.0 ** 32
    side = np.floor(side_min * ratio ** u).astype(np.int32)
    return kind, side


def batched_initial(seed: int, n: int = 256, **kw):
    """The batched heap's instances (kinds and sides from batched_instances)
    and their initial states, instance i drawn with instance id i, as
    concatenated per-cell arrays (kind i8, age i16, energy i16, state u8)."""
    kinds, sides = batched_instances(seed, n, **kw)
    ks, ags, ens, sts = [], [], [], []
    for i, (kd, sd) in enumerate(zip(kinds, sides)):
        sd = int(sd)
        if kd == LIFE:
            k, s = gol_initial(sd, sd, seed, inst=i)
            a = np.zeros(sd * sd, np.int16)
            e = np.zeros(sd * sd, np.int16)
        else:
            k, a, e = wator_initial(sd, sd, seed, inst=i)
            s = np.zeros(sd * sd, np.uint8)
        ks.append(k.astype(np.int8)); ags.append(a); ens.append(e); sts.append(s)
    return kinds, sides, (np.concatenate(ks), np.concatenate(ags), np.concatenate(ens), np.concatenate(sts))


# -------------------------------------------------------------- compaction
def compact_synthetic(n: int, seed: int, kill=(3, 5)):
    """(kill mask of the first class, its references into the second class,
    the second class's references into the first) as index arrays."""
    i = np.arange(n, dtype=np.uint32)
    dead = (draw(seed, TAG_KILL, 0, i) < np.uint32(threshold(*kill))).astype(np.int32)
    a_ref = (draw(seed, TAG_AREF, 0, i) % np.uint32(n)).astype(np.int64)
    b_ref = (draw(seed, TAG_BREF, 0, i) % np.uint32(n)).astype(np.int64)
    return dead, a_ref, b_ref


# -------------------------------------------------------------- structure
MESH_ANCHOR, MESH_PULL, MESH_NODE = 0, 1, 2


def structure_mesh(rows: int, cols: int, seed: int, keep=(9, 10), v_pull: float = 0.5,
                   f_lo: float = 0.005, f_hi: float = 0.05, grip: float = 10.0):
    """Node arrays (kind, x, y, vx, vy, m, slot[N, 3], nspr) and spring
    arrays (p1, p2, k, L0, fmax) of the brick-wall mesh; spring ids follow
    the candidate order, a node's slots hold its springs in increasing id."""
    N = rows * cols
    v = np.arange(N, dtype=np.int64)
    r, c = v // cols, v % cols
    u = lambda step, idx: draw(seed, TAG_MESH, step, idx.astype(np.uint32)).astype(np.float64) / 2.0 ** 32
    x = (c + (u(0, v) - 0.5) * 0.3).astype(np.float32)
    y = (r + (u(1, v) - 0.5) * 0.3).astype(np.float32)
    kind = np.full(N, MESH_NODE, np.int8)
    kind[r == 0] = MESH_ANCHOR
    kind[(r == rows - 1) & (rows > 1)] = MESH_PULL
    vx = np.zeros(N, np.float32)
    vy = np.where(kind == MESH_PULL, np.float32(v_pull), np.float32(0)).astype(np.float32)
    # candidates: e = 2 v (right), 2 v + 1 (up, when r + c is even)
    e = np.arange(2 * N, dtype=np.int64)
    a = e // 2
    ra, ca = a // cols, a % cols
    up = (e & 1) == 1
    exists = np.where(up, (ra + 1 < rows) & ((ra + ca) % 2 == 0), ca + 1 < cols)
    b = np.where(up, a + cols, a + 1)
    kept = exists & (draw(seed, TAG_MESH, 4, e.astype(np.uint32)).astype(np.uint64) < np.uint64(threshold(*keep)))
    # a node left without springs keeps its first existing candidate
    deg = np.zeros(N, np.int64)
    np.add.at(deg, a[kept], 1)
    np.add.at(deg, b[kept], 1)
    for node in np.nonzero(deg == 0)[0]:
        inc = np.nonzero(exists & ((a == node) | (b == node)))[0]
        if len(inc):
            kept[inc[0]] = True
    ids = np.nonzero(kept)[0]
    p1, p2 = a[ids].astype(np.int32), b[ids].astype(np.int32)
    S = len(ids)
    dx = x[p2].astype(np.float64) - x[p1].astype(np.float64)
    dy = y[p2].astype(np.float64) - y[p1].astype(np.float64)
    L0 = np.hypot(dx, dy).astype(np.float32)
    k = (0.5 + u(2, ids)).astype(np.float32)
    fmax = f_lo + (f_hi - f_lo) * u(3, ids)
    fmax = np.where((kind[p1] != MESH_NODE) | (kind[p2] != MESH_NODE), fmax * grip, fmax).astype(np.float32)
    # slots: springs of each node in increasing id
    ends = np.concatenate([p1, p2]).astype(np.int64)
    sid = np.concatenate([np.arange(S), np.arange(S)]).astype(np.int64)
    order = np.lexsort((sid, ends))
    ends, sid = ends[order], sid[order]
    nspr = np.bincount(ends, minlength=N).astype(np.int32)
    if nspr.max(initial=0) > 3:
        raise AssertionError("mesh degree above 3")
    start = np.concatenate([[0], np.cumsum(nspr)[:-1]])
    pos = np.arange(len(ends)) - start[ends]
    slot = np.full((N, 3), -1, np.int32)
    slot[ends, pos] = sid
    return dict(kind=kind, x=x, y=y, vx=vx, vy=vy, m=np.ones(N, np.float32), slot=slot, nspr=nspr,
                p1=p1, p2=p2, k=k, L0=L0, fmax=fmax, rows=rows, cols=cols)
