"""Pins of the oracle's Philox4x32-10 against the published known answers."""
import os

import numpy as np

from paper_1908_05845_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_oracle_philox_known_answers(orc):
    for ctr, key, out in _kat():
        assert orc.philox4x32_10(ctr, key) == out


def test_input_philox_known_answers():
    for ctr, key, out in _kat():
        got = inputs.philox4x32_10(*[np.uint32(c) for c in ctr], key[0], key[1])
        assert [int(g) for g in got] == out


def test_draw_streams_agree(orc):
    cells = np.arange(100_000, dtype=np.uint32)
    for seed, tag, step, inst in [(1, 0, 0, 0), (2**40 + 7, 6, 999, 3), (3, 2, 5, 255)]:
        assert np.array_equal(orc.draw(seed, tag, step, cells, inst),
                              inputs.draw(seed, tag, step, cells, inst))
