"""Pins of the 2-D Barnes-Hut oracle (thesis Sec. 7.3).

* Never opening a tree node by the width criterion (theta = 0) gives the
  direct all-pairs sum, checked against an FP64 direct sum.
* The tree is the region quad tree: worked node counts and depths; the
  accelerations do not depend on the insertion order (bitwise).
* The error against the direct sum falls with theta; two bodies
  attract with equal and opposite accelerations times their masses.
* A body leaving the unit square is reflected with its velocity negated.
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
