"""Parity of the GPU Nagel-Schreckenberg traffic with the oracle: bit-exact
per-cell car velocities, car counts and consistency; closed-form pins on
the GPU (free flow, conservation)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs  # noqa: E402
from paper_1908_05845_gb300.workloads import Traffic  # noqa: E402


def ring(lengths, brake=(0, 1)):
    S = len(lengths)
    start = np.concatenate([[0], np.cumsum(lengths[:-1])]).astype(np.int32)
    out = np.full((S, 3), -1, np.int32)
    out[:, 0] = (np.arange(S) + 1) % S
    return dict(num_streets=S, street_start=start, street_len=np.array(lengths, np.int32),
                out_deg=np.ones(S, np.int32), out_street=out.reshape(-1),
                is_source=np.zeros(S, np.uint8), num_cells=int(sum(lengths)), v_max=5,
                brake_threshold=inputs.threshold(*brake), sources_enabled=0, sinks_enabled=0)


def test_small_graphs_many_seeds(orc):
    for seed in range(1, 31):
        g = inputs.nasch_graph(seed, num_streets=8, n_sources=2, n_sinks=2, len_min=6, len_span=10)
        v = inputs.nasch_cars(g, seed, n_cars=g["num_cells"] // 3)
        sim = Traffic(g, seed, v)
        sim.step(40)
        got = sim.read()
        want, _ = orc.nasch_run(g, seed, v, 40)
        assert np.array_equal(got, want), seed
        sim.sync()
        sim.close()


def test_full_graph_parity(orc):
    g = inputs.nasch_graph(1)
    v = inputs.nasch_cars(g, 1)
    sim = Traffic(g, 1, v)
    for chunk in (1, 29, 70):
        sim.step(chunk)
    got = sim.read()
    want, cnt = orc.nasch_run(g, 1, v, 100)
    assert np.array_equal(got, want)
    st = sim.heap.stats()
    car = sim.class_ids["Car"]
    assert st["live_objects"][car] == cnt[-1, 0]
    assert st["allocs"][car] == cnt[:, 1].sum() and st["frees"][car] == cnt[:, 2].sum()
    assert sim.heap.check() == 0
    sim.sync()


def test_free_flow_and_conservation_on_gpu():
    g = ring([1000])
    v = np.full(1000, -1, np.int8)
    v[10] = 0
    sim = Traffic(g, 1, v)
    sim.step(12)
    got = sim.read()
    assert np.flatnonzero(got >= 0).tolist() == [10 + 15 + 5 * 7] and got[60] == 5
    g = ring([100, 150, 120, 130], brake=(1, 5))
    rng = np.random.default_rng(0)
    v = np.full(g["num_cells"], -1, np.int8)
    v[rng.random(g["num_cells"]) < 0.4] = 0
    sim = Traffic(g, 3, v)
    sim.step(200)
    assert (sim.read() >= 0).sum() == (v >= 0).sum()


@pytest.mark.parametrize("seed", [1, 2])
def test_controllers_full_graph_parity(orc, seed):
    """Traffic with controllers (traffic lights, smart lights, yield) on the
    2000-street graph: car velocities per cell and every controller's green
    index and timer equal the oracle's after 200 steps."""
    g = inputs.nasch_graph(seed)
    v = inputs.nasch_cars(g, seed)
    kind = inputs.nasch_controllers(g, seed)
    sim = Traffic(g, seed, v)
    sim.set_controllers(kind, phase_len=8, lookahead=5)
    sim.step(200)
    got = sim.read()
    green, timer = sim.controller_state()
    sim.sync()
    sim.close()
    want, wg, wt, cnt = orc.nasch_ctrl_run(g, seed, v, 200, kind, phase_len=8, lookahead=5)
    assert (cnt[:, 4] == 0).all() and cnt[:, 5].sum() > 0
    assert np.array_equal(got, want)
    assert np.array_equal(green, wg) and np.array_equal(timer, wt)


def test_controllers_small_graphs_many_seeds(orc):
    for seed in range(1, 21):
        g = inputs.nasch_graph(seed, num_streets=10, n_sources=2, n_sinks=2, len_min=6, len_span=10)
        v = inputs.nasch_cars(g, seed, n_cars=g["num_cells"] // 3)
        kind = inputs.nasch_controllers(g, seed)
        sim = Traffic(g, seed, v)
        sim.set_controllers(kind, phase_len=3, lookahead=4)
        sim.step(50)
        got = sim.read()
        green, timer = sim.controller_state()
        sim.close()
        want, wg, wt, _ = orc.nasch_ctrl_run(g, seed, v, 50, kind, phase_len=3, lookahead=4)
        assert np.array_equal(got, want), seed
        assert np.array_equal(green, wg) and np.array_equal(timer, wt), seed


def junction():
    """Streets 0 (A) and 1 (B), 20 cells each, lead into street 2 (O, 60
    cells), a sink."""
    out = np.full(9, -1, np.int32)
    out[0] = out[3] = 2
    return dict(num_streets=3, street_start=np.array([0, 20, 40], np.int32),
                street_len=np.array([20, 20, 60], np.int32), out_deg=np.array([1, 1, 0], np.int32),
                out_street=out, is_source=np.zeros(3, np.uint8), num_cells=100, v_max=5,
                brake_threshold=0, sources_enabled=0, sinks_enabled=1)


def fork():
    """Street A turns into O or X (a random route per step), B only into O;
    O and X are sinks."""
    out = np.full(12, -1, np.int32)
    out[0:2] = [2, 3]
    out[3] = 2
    return dict(num_streets=4, street_start=np.array([0, 20, 40, 100], np.int32),
                street_len=np.array([20, 20, 60, 40], np.int32), out_deg=np.array([2, 1, 0, 0], np.int32),
                out_street=out, is_source=np.zeros(4, np.uint8), num_cells=140, v_max=5,
                brake_threshold=0, sources_enabled=0, sinks_enabled=1)


def single_entry():
    """Street A leads into street O and nothing else does."""
    return dict(num_streets=2, street_start=np.array([0, 20], np.int32), street_len=np.array([20, 60], np.int32),
                out_deg=np.array([1, 0], np.int32), out_street=np.array([1, -1, -1, -1, -1, -1], np.int32),
                is_source=np.zeros(2, np.uint8), num_cells=80, v_max=5, brake_threshold=0,
                sources_enabled=0, sinks_enabled=1)


def cars(n, cells, v=0):
    a = np.full(n, -1, np.int8)
    a[list(cells)] = v
    return a


def test_controller_worked_cases(orc):
    """The controllers' degenerate and boundary cases, each bit-exact
    against the oracle (velocities, green index and timer): a car just
    outside and just inside the lookahead window, both streets waiting at a
    smart light, a lost claim without controllers, a controller on a street
    with one entry (each kind), a red street's queue under a plain light, a
    yield controller, and route-dependent waiting on a fork for 16 seeds."""
    J, NONE = junction(), np.full(3, -1, np.int8)
    smart, light, yld = (np.array([-1, -1, k], np.int8) for k in (1, 0, 2))
    cases = [(J, 3, cars(100, [34]), smart, 50, 1), (J, 3, cars(100, [35]), smart, 50, 1),
             (J, 3, cars(100, [19, 39]), smart, 50, 1), (J, 3, cars(100, [19, 37], 4), NONE, 8, 1),
             (J, 3, cars(100, range(10, 20)), light, 4, 24),
             (J, 3, cars(100, list(range(0, 20)) + list(range(35, 40))), yld, 8, 10)]
    cases += [(single_entry(), 3, cars(80, range(15, 20), 3), np.array([-1, k], np.int8), 3, 7) for k in (0, 1, 2)]
    cases += [(fork(), seed, cars(140, [19, 39]), np.array([-1, -1, 1, -1], np.int8), 50, 1) for seed in range(1, 17)]
    for n, (g, seed, v, kind, P, T) in enumerate(cases):
        sim = Traffic(g, seed, v)
        sim.set_controllers(kind, phase_len=P, lookahead=5)
        sim.step(T)
        got = sim.read()
        green, timer = sim.controller_state()
        assert sim.heap.check() == 0
        sim.close()
        want, wg, wt, _ = orc.nasch_ctrl_run(g, seed, v, T, kind, phase_len=P, lookahead=5)
        assert np.array_equal(got, want), n
        guarded = kind >= 0
        assert np.array_equal(green[guarded], wg[guarded]) and np.array_equal(timer[guarded], wt[guarded]), n
