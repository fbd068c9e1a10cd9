"""Pins of the traffic oracle with traffic controllers (thesis Sec. 7.5).

* Without controllers it is the plain traffic oracle (whose own pins hold).
* With a controller on every street with two or more incoming streets, no
  crossing claim is ever lost (only one incoming street can enter at a time,
  and only its front car), and cars are conserved when sources and sinks
  are off.
* Worked cases on a two-into-one junction: a traffic light's green index and
  timer follow floor(t / P) mod n and t mod P; a red street's front car
  never enters; a yield controller lets the priority street through while it
  has waiting cars; a smart light turns green at once (timer restarted)
  for the only street with a waiting car and keeps its phase when both
  wait; "waiting" means within the lookahead window and routed into the
  guarded street in this step; the switch and lost-claim counters; a
  controller of a street with one entry does nothing.
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


def smart_light(orc, g, v, **kw):
    """One step of the junction with a smart light (phase 50) on O."""
    return orc.nasch_ctrl_run(g, 3, v, 1, np.array([-1, -1, 1], np.int8), phase_len=50, **kw)


def test_lookahead_window(orc):
    """A car waits when it is within `lookahead` (5) cells of the end of its
    street: the cell 5 before the last is outside the window."""
    g = junction()
    for p, waits in ((14, False), (15, True)):
        v = np.full(g["num_cells"], -1, np.int8)
        v[20 + p] = 0  # street B only; the smart light starts green on A
        _, green, timer, _ = smart_light(orc, g, v)
        assert (green[2], timer[2]) == ((1, 0) if waits else (0, 1)), p


def test_smart_light_keeps_its_phase_when_both_streets_wait(orc):
    g = junction()
    v = np.full(g["num_cells"], -1, np.int8)
    v[19] = v[39] = 0
    _, green, timer, cnt = smart_light(orc, g, v)
    assert (green[2], timer[2]) == (0, 1) and cnt[0, 5] == 0


def test_smart_light_restarts_its_timer_on_a_switch(orc):
    g = junction()
    v = np.full(g["num_cells"], -1, np.int8)
    v[39] = 0
    _, green, timer, cnt = smart_light(orc, g, v, timer=np.array([0, 0, 3], np.int16))
    assert (green[2], timer[2]) == (1, 0) and cnt[0, 5] == 1


@pytest.mark.parametrize("P", [2, 5])
def test_switch_counter_counts_phase_changes(orc, P):
    g = junction()
    v0 = np.full(g["num_cells"], -1, np.int8)
    _, _, _, cnt = orc.nasch_ctrl_run(g, 3, v0, 4 * P, np.array([-1, -1, 0], np.int8), phase_len=P)
    assert cnt[:, 5].tolist() == [int(t % P == 0) for t in range(1, 4 * P + 1)]


def test_lost_claim_is_counted_without_controllers(orc):
    """Two cars enter the same street in one step: the one on the lower cell
    index wins, the other stops at the end of its own street."""
    g = junction()
    v = np.full(g["num_cells"], -1, np.int8)
    v[19], v[37] = 4, 4
    v1, _, _, cnt = orc.nasch_ctrl_run(g, 3, v, 1, np.full(3, -1, np.int8))
    assert cnt[0, 4] == 1 and v1[39] == 2 and v1[44] == 5


def test_controller_on_a_street_with_one_entry_does_nothing(orc):
    """Street A leads into street O and nothing else does: whatever the
    controller on O, its state never changes and A's cars pass freely."""
    g = dict(num_streets=2, street_start=np.array([0, 20], np.int32), street_len=np.array([20, 60], np.int32),
             out_deg=np.array([1, 0], np.int32), out_street=np.array([1, -1, -1, -1, -1, -1], np.int32),
             is_source=np.zeros(2, np.uint8), num_cells=80, v_max=5, brake_threshold=0,
             sources_enabled=0, sinks_enabled=1)
    v = np.full(80, -1, np.int8)
    v[15:20] = 3
    free, _ = orc.nasch_run(g, 3, v, 7)
    for kind in (0, 1, 2):
        v1, green, timer, cnt = orc.nasch_ctrl_run(g, 3, v, 7, np.array([-1, kind], np.int8), phase_len=3)
        assert green[1] == 0 and timer[1] == 0 and cnt[:, 5].sum() == 0
        assert np.array_equal(v1, free)


def test_waiting_follows_this_steps_route(orc):
    """Street A turns into O or X (a random route per step), B only into O;
    a smart light guards O and starts green on A.  A car at the end of A
    waits for O only when this step's route of A leads there: when A's car
    turns into X, B is the only street waiting for O and gets green at once."""
    lens = np.array([20, 20, 60, 40], np.int32)
    start = np.array([0, 20, 40, 100], np.int32)
    out = np.full(12, -1, np.int32)
    out[0:2] = [2, 3]
    out[3] = 2
    g = dict(num_streets=4, street_start=start, street_len=lens, out_deg=np.array([2, 1, 0, 0], np.int32),
             out_street=out, is_source=np.zeros(4, np.uint8), num_cells=140, v_max=5,
             brake_threshold=0, sources_enabled=0, sinks_enabled=1)
    kind = np.array([-1, -1, 1, -1], np.int8)
    seen = set()
    for seed in range(1, 17):
        v = np.full(140, -1, np.int8)
        v[19] = v[39] = 0
        v1, green, timer, _ = orc.nasch_ctrl_run(g, seed, v, 1, kind, phase_len=50)
        to_x = bool(v1[100] >= 0)
        seen.add(to_x)
        if to_x:
            assert (green[2], timer[2]) == (1, 0) and v1[40] == 1 and v1[39] < 0
        else:
            assert (green[2], timer[2]) == (0, 1) and v1[40] == 1 and v1[39] == 0
    assert seen == {False, True}
