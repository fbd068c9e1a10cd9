"""Pins of the traffic oracle with traffic controllers (thesis Sec. 7.5).

* Without controllers it is the plain traffic oracle (whose own pins hold).
* With a controller on every street with two or more incoming streets, no
  crossing claim is ever lost (only one incoming street can enter at a time,
  and only its front car), and cars are conserved when sources and sinks
  are off.
* Worked cases on a two-into-one junction: a traffic light's green index and
  timer follow floor(t / P) mod n and t mod P; a red street's front car
  never enters; a yield controller lets the priority street through while it
  has waiting cars; a smart light turns green at once for the only street
  with a waiting car.
"""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs


def junction(LA=20, LB=20, LO=60, v_max=5):
    """Streets 0 (A) and 1 (B) both lead into street 2 (O), a sink."""
    lens = np.array([LA, LB, LO], np.int32)
    start = np.array([0, LA, LA + LB], np.int32)
    out = np.full(9, -1, np.int32)
    out[0] = 2
    out[3] = 2
    return dict(num_streets=3, street_start=start, street_len=lens,
                out_deg=np.array([1, 1, 0], np.int32), out_street=out,
                is_source=np.zeros(3, np.uint8), num_cells=int(lens.sum()), v_max=v_max,
                brake_threshold=0, sources_enabled=0, sinks_enabled=1)


def cars_on(g, v, street):
    a = int(g["street_start"][street])
    return int((v[a:a + int(g["street_len"][street])] >= 0).sum())


def test_without_controllers_equals_plain_traffic(orc):
    g = inputs.nasch_graph(2, num_streets=300, n_sources=16, n_sinks=16)
    v0 = inputs.nasch_cars(g, 2, n_cars=20000)
    none = np.full(300, -1, np.int8)
    for T in (1, 17, 60):
        a, _ = orc.nasch_run(g, 2, v0, T)
        b, _, _, cnt = orc.nasch_ctrl_run(g, 2, v0, T, none)
        assert np.array_equal(a, b)
        assert cnt[:, 5].sum() == 0


def test_controllers_never_lose_a_claim_and_conserve_cars(orc):
    g = inputs.nasch_graph(1, num_streets=400, n_sources=16, n_sinks=16)
    kind = inputs.nasch_controllers(g, 1)
    assert (kind >= 0).sum() > 100 and set(np.unique(kind)) == {-1, 0, 1, 2}
    v0 = inputs.nasch_cars(g, 1, n_cars=40000)
    _, _, _, cnt = orc.nasch_ctrl_run(g, 1, v0, 150, kind)
    assert (cnt[:, 4] == 0).all()
    assert cnt[:, 5].sum() > 0  # controllers did switch
    closed = dict(g, sources_enabled=0, sinks_enabled=0)
    v, _, _, cnt = orc.nasch_ctrl_run(closed, 1, v0, 120, kind)
    assert (cnt[:, 0] == (v0 >= 0).sum()).all() and (v >= 0).sum() == (v0 >= 0).sum()
    assert (cnt[:, 4] == 0).all()


@pytest.mark.parametrize("P", [1, 3, 4, 7])
def test_traffic_light_phases(orc, P):
    g = junction()
    v0 = np.full(g["num_cells"], -1, np.int8)
    kind = np.array([-1, -1, 0], np.int8)
    for T in range(0, 3 * P + 3):
        _, green, timer, _ = orc.nasch_ctrl_run(g, 3, v0, T, kind, phase_len=P)
        assert green[2] == (T // P) % 2 and timer[2] == T % P


def test_red_street_never_enters(orc):
    """Only A has cars; the light alternates A (steps 1..3), B (4..7), ...
    Cars enter O only in steps whose green is A."""
    g = junction()
    v = np.full(g["num_cells"], -1, np.int8)
    v[10:20] = 0  # a queue on A up to its last cell
    kind = np.array([-1, -1, 0], np.int8)
    green = timer = None
    on_o = 0
    for t in range(1, 25):
        v, green, timer, cnt = orc.nasch_ctrl_run(g, 3, v, 1, kind, phase_len=4, green=green,
                                                  timer=timer, t0=t - 1)
        now = cars_on(g, v, 2) + int(cnt[0, 2])
        if (t // 4) % 2 == 1:  # B green during this step
            assert now == on_o, t
        on_o = cars_on(g, v, 2)


def test_yield_gives_priority_street_the_way(orc):
    g = junction()
    v = np.full(g["num_cells"], -1, np.int8)
    v[0:20] = 0      # A full
    v[35:40] = 0     # five cars at the end of B
    kind = np.array([-1, -1, 2], np.int8)
    v1, _, _, _ = orc.nasch_ctrl_run(g, 3, v, 10, kind)
    assert cars_on(g, v1, 1) == 5 and (v1[35:40] >= 0).all()  # B waits
    assert cars_on(g, v1, 0) < 20 and cars_on(g, v1, 2) > 0  # A flows


def test_smart_light_turns_green_for_the_only_waiting_street(orc):
    g = junction()
    v = np.full(g["num_cells"], -1, np.int8)
    v[38:40] = 0  # cars only at the end of B; the light starts green on A
    kind = np.array([-1, -1, 1], np.int8)
    v1, green, timer, _ = orc.nasch_ctrl_run(g, 3, v, 1, kind, phase_len=50)
    assert green[2] == 1 and timer[2] == 0
    assert cars_on(g, v1, 2) == 1  # B's front car crossed at once
    plain = np.array([-1, -1, 0], np.int8)
    v2, green, _, _ = orc.nasch_ctrl_run(g, 3, v, 1, plain, phase_len=50)
    assert green[2] == 0 and cars_on(g, v2, 2) == 0  # a plain light keeps B red
