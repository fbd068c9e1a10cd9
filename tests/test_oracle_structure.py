"""Pins of the spring-mesh ("structure", thesis Sec. 7.4) oracle.

* One spring, one substep: the force, acceleration, damped velocity and new
  position against the closed form, with the free node as either endpoint;
  a compressed spring exerts nothing; the break limit is strict.
* A node between two anchors on pre-stretched springs is a harmonic
  oscillator with omega^2 = 2 k / m: position after a given time within
  O(dt) of the closed form, first-order convergence, damping envelope.
* A free mesh (no anchors) conserves momentum and (undamped) energy up to
  the integrator's bounded error; three symmetric springs hold a node still.
* The removal phase equals a connected-components computation (scipy):
  survivors are the components holding an anchor node, distances are the
  multi-source BFS distances, the level count is the largest distance + 2.
* Pull nodes move by exactly v dt per iteration; the phases run in the
  thesis' order (a crack made in the compute phase is removed in the same
  iteration); bookkeeping of springs and counts stays consistent.
"""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import connected_components, shortest_path  # noqa: E402

A, P, N_ = 0, 1, 2


def mesh_from(kind, xy, springs, k, L0, fmax, m=None, v=None):
    """Small mesh dict from explicit nodes and springs (slots in id order)."""
    n = len(kind)
    xy = np.asarray(xy, np.float64)
    S = len(springs)
    slot = np.full((n, 3), -1, np.int32)
    nspr = np.zeros(n, np.int32)
    for s, (a, b) in enumerate(springs):
        for e in (a, b):
            slot[e, nspr[e]] = s
            nspr[e] += 1
    v = np.zeros((n, 2)) if v is None else np.asarray(v, np.float64)
    return dict(kind=np.asarray(kind, np.int8), x=xy[:, 0].astype(np.float32), y=xy[:, 1].astype(np.float32),
                vx=v[:, 0].astype(np.float32), vy=v[:, 1].astype(np.float32),
                m=np.ones(n, np.float32) if m is None else np.asarray(m, np.float32), slot=slot, nspr=nspr,
                p1=np.array([s[0] for s in springs], np.int32).reshape(S),
                p2=np.array([s[1] for s in springs], np.int32).reshape(S),
                k=np.full(S, k, np.float32) if np.isscalar(k) else np.asarray(k, np.float32),
                L0=np.full(S, L0, np.float32) if np.isscalar(L0) else np.asarray(L0, np.float32),
                fmax=np.full(S, fmax, np.float32) if np.isscalar(fmax) else np.asarray(fmax, np.float32))


@pytest.mark.parametrize("node_is_p1", [True, False])
def test_single_spring_one_substep(orc, node_is_p1):
    k, L0, m, dt, damping = 0.8, 4.5, 2.0, 0.1, 0.1
    springs = [(1, 0)] if node_is_p1 else [(0, 1)]
    g = mesh_from([A, N_], [(0, 0), (3, 4)], springs, k, L0, 1e9, m=[1.0, m])
    st, cnt = orc.structure_run(g, 1, dt=dt, damping=damping, substeps=1, phases=orc.PHASE_COMPUTE)
    F = k * (5.0 - L0)  # pulls the node towards the anchor at the origin
    a = -F / m * np.array([0.6, 0.8])
    vel = a * dt * (1 - damping)
    pos = np.array([3.0, 4.0]) + vel * dt
    assert np.allclose([st["vx"][1], st["vy"][1]], vel, rtol=1e-5, atol=0)
    assert np.allclose([st["x"][1], st["y"][1]], pos, rtol=1e-6, atol=0)
    # the stored force acts on p1 and points to p2
    f_on_p1 = F * (np.array([-0.6, -0.8]) if node_is_p1 else np.array([0.6, 0.8]))
    assert np.allclose([st["fx"][0], st["fy"][0]], f_on_p1, rtol=1e-6)
    assert st["x"][0] == 0 and st["y"][0] == 0  # the anchor does not move
    assert cnt[0, 0] == 0


def test_compressed_spring_exerts_nothing(orc):
    g = mesh_from([A, N_], [(0, 0), (3, 4)], [(0, 1)], 0.8, 6.0, 1e9)
    st, _ = orc.structure_run(g, 1, dt=0.1, damping=0.0, substeps=5, phases=orc.PHASE_COMPUTE)
    assert st["x"][1] == np.float32(3) and st["y"][1] == np.float32(4)
    assert st["fx"][0] == 0 and st["fy"][0] == 0


def test_break_limit_is_strict_and_lonely_ends_die(orc):
    # len 5, L0 4.5, k 0.5: F = 0.25 exactly
    keep = mesh_from([A, N_], [(0, 0), (3, 4)], [(0, 1)], 0.5, 4.5, 0.25)
    st, cnt = orc.structure_run(keep, 1, dt=0.1, substeps=1, phases=orc.PHASE_COMPUTE)
    assert st["salive"][0] == 1 and cnt[0, 0] == 0
    brk = mesh_from([A, N_], [(0, 0), (3, 4)], [(0, 1)], 0.5, 4.5, np.nextafter(np.float32(0.25), np.float32(0)))
    st, cnt = orc.structure_run(brk, 1, dt=0.1, substeps=1, phases=orc.PHASE_COMPUTE)
    assert st["salive"][0] == 0 and cnt[0, 0] == 1
    assert cnt[0, 1] == 2 and st["nalive"].sum() == 0  # both ends lost their only spring
    assert (st["slot"] == -1).all() and (st["nspr"] == 0).all()


def oscillator(L, amp, k, m, dt, steps, damping=0.0):
    g = mesh_from([A, N_, A], [(0, 0), (L + amp, 0), (2 * L, 0)], [(0, 1), (1, 2)], k, L / 2, 1e9,
                  m=[1, m, 1])
    st, _ = _run(g, 1, dt=dt, damping=damping, substeps=steps)
    return float(st["x"][1])


def _run(g, T, **kw):
    import oracle
    return oracle.structure_run(g, T, phases=oracle.PHASE_COMPUTE, **kw)


def test_two_anchor_oscillator_closed_form(orc):
    L, amp, k, m = 8.0, 1.0, 0.7, 1.3
    w = np.sqrt(2 * k / m)
    t_end = 2.3
    errs = []
    for dt in (0.02, 0.01, 0.005):
        n = int(round(t_end / dt))
        x = oscillator(L, amp, k, m, dt, n)
        errs.append(abs(x - (L + amp * np.cos(w * n * dt))))
    assert errs[0] < 0.05 * amp
    assert 1.6 < errs[0] / errs[1] < 2.5 and 1.6 < errs[1] / errs[2] < 2.5  # first order


def test_oscillator_damping_envelope(orc):
    """Multiplying v by (1 - d) every step is, to first order in dt, a
    friction -gamma v with gamma = -ln(1 - d) / dt: the damped oscillator
    x = A e^(-gamma t / 2) (cos w_d t + gamma / (2 w_d) sin w_d t)."""
    L, amp, k, m, dt, damping = 8.0, 1.0, 0.7, 1.3, 0.005, 0.001
    w = np.sqrt(2 * k / m)
    n = 6000
    x = oscillator(L, amp, k, m, dt, n, damping=damping)
    g = -np.log1p(-damping) / dt
    wd = np.sqrt(w * w - g * g / 4)
    t = n * dt
    expect = amp * np.exp(-g * t / 2) * (np.cos(wd * t) + g / (2 * wd) * np.sin(wd * t))
    assert abs((x - L) - expect) < 0.02 * amp * np.exp(-g * t / 2)
    undamped = oscillator(L, amp, k, m, dt, n)
    assert abs(x - L) < 0.5 * abs(undamped - L) or abs(undamped - L) < 0.2


def free_mesh(seed, rows=8, cols=10):
    g = inputs.structure_mesh(rows, cols, seed)
    n, S = len(g["kind"]), len(g["p1"])
    rng = np.random.default_rng(seed)
    g["kind"] = np.full(n, N_, np.int8)
    g["m"] = rng.uniform(0.5, 2.0, n).astype(np.float32)
    g["vx"] = rng.normal(0, 0.05, n).astype(np.float32)
    g["vy"] = rng.normal(0, 0.05, n).astype(np.float32)
    g["L0"] = (g["L0"] * np.float32(0.9)).astype(np.float32)  # pre-stretched
    g["fmax"] = np.full(S, 1e30, np.float32)
    return g


def energy(g, st):
    m = g["m"].astype(np.float64)
    ke = 0.5 * (m * (st["vx"].astype(np.float64) ** 2 + st["vy"].astype(np.float64) ** 2)).sum()
    dx = st["x"][g["p2"]].astype(np.float64) - st["x"][g["p1"]]
    dy = st["y"][g["p2"]].astype(np.float64) - st["y"][g["p1"]]
    ext = np.maximum(np.hypot(dx, dy) - g["L0"], 0)
    return ke + 0.5 * (g["k"] * ext ** 2).sum()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_free_mesh_conserves_momentum(orc, seed):
    g = free_mesh(seed)
    st, _ = orc.structure_run(g, 1, dt=0.05, damping=0.0, substeps=400, phases=orc.PHASE_COMPUTE)
    m = g["m"].astype(np.float64)
    p0 = np.array([(m * g["vx"]).sum(), (m * g["vy"]).sum()])
    p1 = np.array([(m * st["vx"]).sum(), (m * st["vy"]).sum()])
    scale = (m * np.hypot(g["vx"], g["vy"])).sum()
    assert np.abs(p1 - p0).max() < 1e-4 * scale
    assert np.abs(st["vx"] - g["vx"]).max() > 1e-3  # the springs did act


def test_free_mesh_energy_bounded_and_first_order(orc):
    """Symplectic Euler keeps the energy error bounded and O(dt): the largest
    deviation over the run (sampled 20 times) halves with dt."""
    g = free_mesh(4)
    e0 = energy(g, g)
    worst = []
    for dt, n in ((0.04, 10), (0.02, 20), (0.01, 40)):
        st, dev = dict(g), 0.0
        for _ in range(20):
            out, _ = orc.structure_run(st, 1, dt=dt, damping=0.0, substeps=n, phases=orc.PHASE_COMPUTE)
            st = dict(st, **out)
            dev = max(dev, abs(energy(g, st) - e0) / e0)
        worst.append(dev)
    assert worst[0] < 0.05
    assert 1.6 < worst[0] / worst[1] < 2.6 and 1.6 < worst[1] / worst[2] < 2.6


def test_symmetric_star_holds_still(orc):
    ang = np.deg2rad([90, 210, 330])
    xy = [(0.0, 0.0)] + [(3 * np.cos(a), 3 * np.sin(a)) for a in ang]
    g = mesh_from([N_, A, A, A], xy, [(0, 1), (2, 0), (0, 3)], 0.9, 2.0, 1e9)
    st, _ = orc.structure_run(g, 1, dt=0.05, damping=0.0, substeps=500, phases=orc.PHASE_COMPUTE)
    assert abs(st["x"][0]) < 1e-4 and abs(st["y"][0]) < 1e-4
    # one sign flipped (the p2 spring seen as p1) would pull it away
    assert abs(st["fx"][1]) > 0.5  # the springs are loaded


def random_graph(seed, n=400, n_edges=420):
    rng = np.random.default_rng(seed)
    deg = np.zeros(n, int)
    edges = set()
    while len(edges) < n_edges:
        a, b = rng.integers(0, n, 2)
        if a == b or deg[a] >= 3 or deg[b] >= 3 or (min(a, b), max(a, b)) in edges:
            if len(edges) and rng.random() < 1e-3:
                break
            continue
        edges.add((min(a, b), max(a, b)))
        deg[a] += 1
        deg[b] += 1
    edges = sorted(edges)
    kind = rng.choice([A, P, N_], size=n, p=[0.05, 0.05, 0.9]).astype(np.int8)
    xy = rng.uniform(0, 20, (n, 2))
    return mesh_from(kind, xy, edges, 1.0, 1.0, 1e9), edges


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_removal_equals_components_with_an_anchor(orc, seed):
    g, edges = random_graph(seed)
    n = len(g["kind"])
    e = np.array(edges)
    adj = scipy_sparse.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    ncomp, lab = connected_components(adj, directed=False)
    anchored = np.zeros(ncomp, bool)
    anchored[lab[g["kind"] == A]] = True
    isolated = g["nspr"] == 0
    expect_alive = anchored[lab] | isolated
    st, cnt = orc.structure_run(g, 1, phases=orc.PHASE_REMOVE)
    assert np.array_equal(st["nalive"].astype(bool), expect_alive)
    assert np.array_equal(st["salive"].astype(bool), anchored[lab[e[:, 0]]])
    assert cnt[0, 2] == (~anchored[lab[e[:, 0]]]).sum()
    assert cnt[0, 3] == (~expect_alive).sum()
    # distances: multi-source BFS from the anchors (a virtual source joined to
    # every anchor, minus one)
    anchors = np.nonzero(g["kind"] == A)[0]
    src = np.concatenate([e[:, 0], np.full(len(anchors), n)])
    dst = np.concatenate([e[:, 1], anchors])
    big = scipy_sparse.coo_matrix((np.ones(len(src)), (src, dst)), shape=(n + 1, n + 1))
    d = shortest_path(big, directed=False, unweighted=True, indices=n)[:n] - 1
    reached = np.isfinite(d)
    assert np.array_equal(st["dist"][reached], d[reached].astype(np.int32))
    assert (st["dist"][~reached] == orc.INF_DIST).all()
    assert cnt[0, 4] == int(d[reached].max()) + 2
    assert (st["nspr"][st["nalive"] == 1] == (st["slot"][st["nalive"] == 1] >= 0).sum(1)).all()


def test_pull_nodes_move_by_v_dt(orc):
    g = inputs.structure_mesh(4, 6, 1, v_pull=0.37)
    T, dt = 37, 0.05
    st, _ = orc.structure_run(g, T, dt=dt, phases=orc.PHASE_PULL)
    pull = g["kind"] == P
    expect = g["y"][pull].astype(np.float64) + T * 0.37 * dt
    assert np.allclose(st["y"][pull], expect, rtol=0, atol=T * 4e-7 * 5)
    assert np.array_equal(st["y"][~pull], g["y"][~pull])


def test_phase_order_removes_a_fresh_crack(orc):
    """anchor 0 - 1 - 2 - 3 (pull): spring 1-2 breaks in the compute phase;
    the removal of the same iteration takes 2, 3 and spring 2-3."""
    xy = [(0, 0), (0, 1), (0, 2), (0, 3)]
    g = mesh_from([A, N_, N_, P], xy, [(0, 1), (1, 2), (2, 3)], 1.0, 1.0, [1e9, 0.01, 1e9],
                  v=[(0, 0), (0, 0), (0, 0), (0, 2.0)])
    st, cnt = orc.structure_run(g, 1, dt=0.05, damping=0.0, substeps=40)
    assert list(st["salive"]) == [1, 0, 0]
    assert list(st["nalive"]) == [1, 1, 0, 0]
    assert list(cnt[0, :4]) == [1, 0, 1, 2]


@pytest.mark.parametrize("seed", [1, 2])
def test_mesh_run_bookkeeping(orc, seed):
    g = inputs.structure_mesh(24, 40, seed, v_pull=1.0)
    n0, s0 = len(g["kind"]), len(g["p1"])
    st, cnt = orc.structure_run(g, 60)
    assert cnt[:, 0].sum() > 10  # cracks formed
    assert st["salive"].sum() == s0 - cnt[:, 0].sum() - cnt[:, 2].sum()
    assert st["nalive"].sum() == n0 - cnt[:, 1].sum() - cnt[:, 3].sum()
    live = st["nalive"] == 1
    assert (st["nspr"][live] == (st["slot"][live] >= 0).sum(1)).all()
    for v in np.nonzero(live)[0]:
        for s in st["slot"][v]:
            if s >= 0:
                assert st["salive"][s] and v in (g["p1"][s], g["p2"][s])
    ls = st["salive"] == 1
    assert st["nalive"][g["p1"][ls]].all() and st["nalive"][g["p2"][ls]].all()
    # anchors never move; every live node reaches an anchor after the removal
    anc = g["kind"] == A
    assert np.array_equal(st["x"][anc], g["x"][anc]) and np.array_equal(st["y"][anc], g["y"][anc])
    assert (st["dist"][live] != 0x7FFFFFFF).all()


@pytest.mark.parametrize("rows,cols,seed", [(8, 12, 1), (33, 65, 2)])
def test_mesh_recipe(rows, cols, seed):
    """The brick-wall input: degree at most 3 (exactly the lattice links
    that were kept), right links everywhere but the last column, up links
    where r + c is even, every node keeps a spring, kinds by row, slots in
    increasing spring id naming exactly the node's springs, rest lengths the
    float distance, about 90 % of the candidate links kept."""
    g = inputs.structure_mesh(rows, cols, seed)
    n, S = rows * cols, len(g["p1"])
    p1, p2 = g["p1"].astype(np.int64), g["p2"].astype(np.int64)
    r1, c1 = p1 // cols, p1 % cols
    right = (p2 == p1 + 1) & (c1 + 1 < cols)
    up = (p2 == p1 + cols) & ((r1 + c1) % 2 == 0)
    assert (right | up).all()
    assert np.array_equal(np.argsort(p1 * 2 + up, kind="stable"), np.arange(S))  # candidate order
    deg = np.bincount(np.concatenate([p1, p2]), minlength=n)
    assert deg.max() <= 3 and deg.min() >= 1 and np.array_equal(deg, g["nspr"])
    for v in range(n):
        mine = np.nonzero((p1 == v) | (p2 == v))[0]
        sl = g["slot"][v]
        assert np.array_equal(sl[:len(mine)], mine) and (sl[len(mine):] == -1).all()
    r = np.arange(n) // cols
    assert (g["kind"][r == 0] == A).all() and (g["kind"][r == rows - 1] == P).all()
    assert (g["kind"][(r > 0) & (r < rows - 1)] == N_).all()
    d = np.hypot(g["x"][p2].astype(np.float64) - g["x"][p1], g["y"][p2].astype(np.float64) - g["y"][p1])
    assert np.array_equal(g["L0"], d.astype(np.float32))
    cand = rows * (cols - 1) + sum(1 for rr in range(rows - 1) for cc in range(cols) if (rr + cc) % 2 == 0)
    assert 0.8 < S / cand < 0.97
    assert (g["vy"][g["kind"] == P] > 0).all() and (g["vy"][g["kind"] != P] == 0).all()
