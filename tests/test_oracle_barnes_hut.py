"""Pins of the 2-D Barnes-Hut oracle (thesis Sec. 7.3).

* Never opening a tree node by the width criterion (theta = 0) gives the
  direct all-pairs sum, checked against an FP64 direct sum.
* The tree is the region quad tree of half-open squares: worked node
  counts and depths; the accelerations do not depend on the insertion
  order (bitwise); a body always opens the tree nodes that contain it.
* Visit and node counters: N (nodes - 1 + N) visits at theta = 0 and a
  worked three-body count.
* The error against the direct sum falls with theta; two bodies
  attract with equal and opposite accelerations times their masses.
* The body update is semi-implicit Euler (two-body step for G != 1); a body
  leaving the unit square at any wall is reflected with its velocity
  negated, and one landing on 1 is clamped below it.
"""
import numpy as np
import pytest

from paper_1908_05845_gb300 import inputs


def direct(x, y, m, eps):
    dx = x[None, :].astype(np.float64) - x[:, None]
    dy = y[None, :].astype(np.float64) - y[:, None]
    s2 = dx * dx + dy * dy + eps * eps
    f = m[None, :] / (s2 * np.sqrt(s2))
    np.fill_diagonal(f, 0.0)
    return (f * dx).sum(1), (f * dy).sum(1)


def test_theta_zero_is_the_direct_sum(orc):
    st = inputs.bh_initial(700, 3)
    ax, ay = orc.bh_accel(st["x"], st["y"], st["m"], eps=1e-2, theta=0.0)
    rx, ry = direct(st["x"], st["y"], st["m"], 1e-2)
    scale = np.sqrt(rx ** 2 + ry ** 2).max()
    assert np.abs(ax - rx).max() < 1e-5 * scale and np.abs(ay - ry).max() < 1e-5 * scale


def test_worked_trees(orc):
    x = np.array([0.1, 0.6, 0.1, 0.6], np.float32)
    y = np.array([0.1, 0.1, 0.6, 0.6], np.float32)
    assert orc.bh_build(x, y) == (1, 0)  # one body per quadrant: root only
    assert orc.bh_build(np.array([0.1, 0.2], np.float32), np.array([0.1, 0.2], np.float32)) == (3, 2)
    # x offsets 2^-11 and 3 2^-11 from 0.5 first differ in the 2^-10 digit:
    # the square of width 2^-9 at 0.5 (depth 9) is the first to separate them
    a, b = 0.5 + 2.0 ** -11, 0.5 + 3 * 2.0 ** -11
    assert orc.bh_build(np.array([a, b], np.float32), np.array([0.7, 0.7], np.float32)) == (10, 9)


def test_insertion_order_does_not_matter(orc):
    st = inputs.bh_initial(3000, 5)
    ax, ay = orc.bh_accel(st["x"], st["y"], st["m"])
    perm = np.random.default_rng(1).permutation(3000)
    px, py = orc.bh_accel(st["x"][perm], st["y"][perm], st["m"][perm])
    inv = np.argsort(perm)
    assert np.array_equal(px[inv], ax) and np.array_equal(py[inv], ay)


def test_approximation_error_shrinks_with_theta(orc):
    """Monopole Barnes-Hut: the error against the direct sum falls as theta
    falls (net forces in a uniform distribution are small residuals of
    large opposing terms, so relative errors of a few percent are usual)."""
    st = inputs.bh_initial(4000, 7)
    rx, ry = direct(st["x"], st["y"], st["m"], 1e-2)
    med = []
    for th in (0.7, 0.5, 0.3, 0.1):
        ax, ay = orc.bh_accel(st["x"], st["y"], st["m"], theta=th)
        err = np.hypot(ax - rx, ay - ry) / np.hypot(rx, ry)
        med.append(np.median(err))
        if th == 0.5:
            assert np.median(err) < 3e-2 and np.quantile(err, 0.9) < 6e-2
    assert med == sorted(med, reverse=True) and med[-1] < 1e-3


def test_two_bodies(orc):
    x = np.array([0.2, 0.7], np.float32)
    y = np.array([0.3, 0.4], np.float32)
    m = np.array([2.0, 3.0], np.float32)
    ax, ay = orc.bh_accel(x, y, m)
    assert abs(m[0] * ax[0] + m[1] * ax[1]) < 1e-6 * abs(m[0] * ax[0])
    assert abs(m[0] * ay[0] + m[1] * ay[1]) < 1e-6 * abs(m[0] * ay[0])
    rx, ry = direct(x, y, m, 1e-2)
    assert np.allclose(ax, rx, rtol=1e-6) and np.allclose(ay, ry, rtol=1e-6)


def test_wall_reflection(orc):
    st = dict(x=np.array([0.995], np.float32), y=np.array([0.5], np.float32),
              vx=np.array([1.0], np.float32), vy=np.array([-0.5], np.float32), m=np.array([1.0], np.float32))
    out, _ = orc.bh_run(st, 1, dt=0.01)
    assert out["vx"][0] == -1.0 and abs(out["x"][0] - (2.0 - 1.005)) < 1e-6
    assert out["vy"][0] == -0.5 and abs(out["y"][0] - 0.495) < 1e-6


def test_squares_are_half_open(orc):
    """A body on a midline belongs to the upper quadrant ([p, p + w) squares):
    bodies at x = 0.5 and x = 0.4 (or y) already sit in different quadrants
    of the root, and the same holds one level down."""
    f = lambda *v: np.array(v, np.float32)  # noqa: E731
    assert orc.bh_build(f(0.5, 0.4), f(0.1, 0.1)) == (1, 0)
    assert orc.bh_build(f(0.1, 0.1), f(0.5, 0.4)) == (1, 0)
    # (0.5, 0.5) and (0.75, 0.5) share the root's quadrant 3; in its tree
    # node [0.5, 1)^2 the one on the midline x = 0.75 goes to quadrant 1
    assert orc.bh_build(f(0.5, 0.75), f(0.5, 0.5)) == (2, 1)


def test_a_body_inside_a_tree_node_always_opens_it(orc):
    """With a huge theta only the body's own ancestors are opened: bodies 0
    and 1 share the tree node [0, 0.5)^2 and see each other and body 2
    exactly; body 2 sees that tree node as one body of mass 2 at its centre
    of gravity.  Visits: 4 + 4 + 2 (tree node, two bodies, body 2; tree
    node, body 2 itself)."""
    x = np.array([0.05, 0.45, 0.9], np.float32)
    y = np.array([0.05, 0.45, 0.9], np.float32)
    m = np.array([1.0, 1.0, 1.0], np.float32)
    eps = 1e-2
    ax, ay = orc.bh_accel(x, y, m, eps=eps, theta=10.0)
    rx, ry = direct(x, y, m, eps)
    assert np.allclose(ax[:2], rx[:2], rtol=1e-6) and np.allclose(ay[:2], ry[:2], rtol=1e-6)
    d = np.array([0.25 - 0.9, 0.25 - 0.9])
    s2 = d @ d + eps * eps
    want = 2.0 * d / (s2 * np.sqrt(s2))
    assert np.allclose([ax[2], ay[2]], want, rtol=1e-5)
    _, cnt = orc.bh_run(dict(x=x, y=y, vx=np.zeros(3, np.float32), vy=np.zeros(3, np.float32), m=m),
                        1, theta=10.0)
    assert cnt[0].tolist() == [2, 10]


def test_theta_zero_visits_every_child_of_every_tree_node(orc):
    """At theta = 0 every body opens every tree node, so one step visits
    N (nodes - 1 + N) non-empty child slots; the node count is the region
    quad tree's."""
    st = inputs.bh_initial(500, 2)
    nodes, _ = orc.bh_build(st["x"], st["y"])
    _, cnt = orc.bh_run(st, 1, theta=0.0)
    assert cnt[0].tolist() == [nodes, 500 * (nodes - 1 + 500)]


def test_body_update_is_semi_implicit_euler(orc):
    """v += G a dt, then x += v dt with the new velocity, for G != 1: two
    bodies at rest pulled towards each other by the softened pair force."""
    G, eps, dt = 0.5, 1e-2, 1e-3
    st = dict(x=np.array([0.3, 0.7], np.float32), y=np.array([0.5, 0.5], np.float32),
              vx=np.zeros(2, np.float32), vy=np.zeros(2, np.float32), m=np.array([1.0, 2.0], np.float32))
    out, _ = orc.bh_run(st, 1, G=G, eps=eps, dt=dt)
    d = 0.4
    for b, (other_m, sign) in enumerate(((2.0, 1), (1.0, -1))):
        v = sign * G * other_m * d / (d * d + eps * eps) ** 1.5 * dt
        assert abs(out["vx"][b] - v) < 1e-5 * abs(v)
        assert abs(out["x"][b] - (st["x"][b] + v * dt)) < 5e-8
        assert out["vy"][b] == 0 and out["y"][b] == 0.5


def test_low_walls_and_the_upper_clamp(orc):
    """A body crossing x = 0 (or y = 0) is reflected with its velocity
    negated; one that lands exactly on 1 is reflected onto 1 and clamped to
    the largest float below 1."""
    st = dict(x=np.array([0.004], np.float32), y=np.array([0.003], np.float32),
              vx=np.array([-1.0], np.float32), vy=np.array([-0.5], np.float32), m=np.array([1.0], np.float32))
    out, _ = orc.bh_run(st, 1, dt=0.01)
    assert out["vx"][0] == 1.0 and abs(out["x"][0] - 0.006) < 1e-7
    assert out["vy"][0] == 0.5 and abs(out["y"][0] - 0.002) < 1e-7
    st = dict(x=np.array([0.5], np.float32), y=np.array([0.25], np.float32),
              vx=np.array([0.5], np.float32), vy=np.array([0.0], np.float32), m=np.array([1.0], np.float32))
    out, _ = orc.bh_run(st, 1, dt=1.0)
    assert out["x"][0] == np.float32(1 - 2.0 ** -24) and out["vx"][0] == -0.5
