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
