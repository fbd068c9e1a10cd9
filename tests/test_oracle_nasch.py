"""Pins of the Nagel-Schreckenberg oracle (thesis Sec. 7.5).

Free-flow closed form x(t) = x0 + sum_{k<=t} min(k, v_max); car-count
conservation on a closed ring with and without braking; evenly spaced cars
reach flow N v_max / L within v_max steps; the street-entry claim goes to
the lowest cell index and the loser stops at the end of its street; a sink
removes a car that reaches its last cell; braking statistics (from rest
and the steady mean speed v_max - p); bookkeeping cars' = cars + spawned - sunk.
"""
import numpy as np

from paper_1908_05845_gb300 import inputs


def ring(lengths, brake=(0, 1)):
    S = len(lengths)
    start = np.concatenate([[0], np.cumsum(lengths[:-1])]).astype(np.int32)
    out = np.full((S, 3), -1, np.int32)
    out[:, 0] = (np.arange(S) + 1) % S
    return dict(num_streets=S, street_start=start, street_len=np.array(lengths, np.int32),
                out_deg=np.ones(S, np.int32), out_street=out.reshape(-1),
                is_source=np.zeros(S, np.uint8), num_cells=int(sum(lengths)), v_max=5,
                brake_threshold=inputs.threshold(*brake), sources_enabled=0, sinks_enabled=0)


def test_free_flow_closed_form(orc):
    g = ring([1000])
    v = np.full(1000, -1, np.int8)
    v[10] = 0
    for t in range(1, 30):
        v2, c = orc.nasch_run(g, 1, v, t)
        x = int(np.flatnonzero(v2 >= 0)[0])
        want = (10 + sum(min(k, 5) for k in range(1, t + 1))) % 1000
        assert x == want
        if t >= 5:
            assert x == (10 + 15 + 5 * (t - 5)) % 1000


def test_conservation_on_ring(orc):
    g = ring([100, 150, 120, 130], brake=(1, 5))
    rng = np.random.default_rng(0)
    for dens in (0.1, 0.4, 0.8):
        v = np.full(g["num_cells"], -1, np.int8)
        v[rng.random(g["num_cells"]) < dens] = 0
        n0 = int((v >= 0).sum())
        v2, c = orc.nasch_run(g, 3, v, 300)
        assert np.all(c[:, 0] == n0) and (v2 >= 0).sum() == n0
        assert np.all(c[:, 1] == 0) and np.all(c[:, 2] == 0)


def test_evenly_spaced_flow(orc):
    L, N = 120, 20
    g = ring([L])
    v = np.full(L, -1, np.int8)
    v[np.arange(N) * (L // N)] = 0
    v2, c = orc.nasch_run(g, 1, v, 5)
    assert np.all(v2[v2 >= 0] == 5)
    assert c[-1, 3] * 5 / L == N * 5 / L  # all N cars move v_max cells


def test_entry_claim_lowest_cell_wins(orc):
    lengths = [100, 100, 100]
    g = ring(lengths)
    g["out_street"] = np.array([2, -1, -1, 2, -1, -1, 2, -1, -1], np.int32)
    v = np.full(300, -1, np.int8)
    v[99] = 4
    v[199] = 4
    v2, c = orc.nasch_run(g, 1, v, 1)
    assert v2[204] == 5 and v2[199] == 0 and (v2 >= 0).sum() == 2


def test_bookkeeping_random_graph(orc):
    g = inputs.nasch_graph(2, num_streets=200, n_sources=16, n_sinks=16)
    v = inputs.nasch_cars(g, 2, n_cars=20000)
    n = int((v >= 0).sum())
    v2, c = orc.nasch_run(g, 2, v, 200)
    for row in c:
        assert row[0] == n + row[1] - row[2]
        n = row[0]
    assert (v2 >= 0).sum() == n
    assert np.all(v2[v2 >= 0] <= 5)


def test_braking_statistics(orc):
    """Step (d) with p = 1/5, on cars too far apart to meet.  From rest a car
    reaches speed 1 and brakes back to 0 with probability p; a free car that
    has reached v_max - 1 alternates between v_max and v_max - 1, so its mean
    speed is v_max - p.  Bounds: five standard deviations of the binomial
    estimate."""
    L, N = 20000, 2000
    g = ring([L], brake=(1, 5))
    v = np.full(L, -1, np.int8)
    v[np.arange(N) * (L // N)] = 0
    v1, _ = orc.nasch_run(g, 7, v, 1)
    assert abs((v1 == 0).sum() / N - 0.2) < 5 * np.sqrt(0.16 / N)
    N = 200
    v = np.full(L, -1, np.int8)
    v[np.arange(N) * (L // N)] = 0
    v, _ = orc.nasch_run(g, 8, v, 20)
    assert np.all(v[v >= 0] >= 4)
    speeds = []
    for t in range(20, 220):
        v, _ = orc.nasch_run(g, 8, v, 1, t0=t)
        speeds.append(v[v >= 0])
    speeds = np.concatenate(speeds)
    assert speeds.size == 200 * N and set(np.unique(speeds)) <= {4, 5}
    assert abs(speeds.mean() - 4.8) < 5 * np.sqrt(0.16 / speeds.size)


def test_claim_loser_stops_at_end_of_its_street(orc):
    """The car that loses the entry claim (the higher cell index) drives up to
    the last cell of its own street instead of standing still."""
    g = ring([100, 100, 100])
    g["out_street"] = np.array([2, -1, -1, 2, -1, -1, 2, -1, -1], np.int32)
    v = np.full(300, -1, np.int8)
    v[99] = 4
    v[197] = 4
    v2, _ = orc.nasch_run(g, 1, v, 1)
    assert v2[204] == 5 and v2[199] == 2 and (v2 >= 0).sum() == 2


def test_sink_removes_a_car_that_reaches_the_last_cell(orc):
    """On a sink street a car is removed when its move ends on or passes the
    last cell; one that stops short stays."""
    for start, sunk in ((94, 1), (93, 0), (99, 1)):
        g = ring([100])
        g.update(out_deg=np.zeros(1, np.int32), out_street=np.full(3, -1, np.int32), sinks_enabled=1)
        v = np.full(100, -1, np.int8)
        v[start] = 4
        v2, c = orc.nasch_run(g, 1, v, 1)
        assert c[0, 2] == sunk and (v2 >= 0).sum() == 1 - sunk
        if not sunk:
            assert v2[start + 5] == 5
