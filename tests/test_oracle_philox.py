"""Philox4x32-10 (Salmon et al., SC'11): the oracle's C implementation and
the input generator's numpy implementation, written separately from the
published definition, agree bit for bit on a million draws over several
keys, counters and tags (the CUDA library's own implementation is held to
the same streams by the bit-exact Wa-Tor and traffic parity tests).  The
published known-answer vectors are not available here, so agreement with
the reference generator itself is unpinned."""
import numpy as np

from paper_1908_05845_gb300 import inputs


def test_draw_streams_agree(orc):
    cells = np.arange(250_000, dtype=np.uint32)
    for seed, tag, step, inst in [(1, 0, 0, 0), (2**40 + 7, 6, 999, 3), (3, 2, 5, 255), (2**64 - 1, 17, 2**32 - 1, 7)]:
        assert np.array_equal(orc.draw(seed, tag, step, cells, inst),
                              inputs.draw(seed, tag, step, cells, inst))


def test_full_words_agree(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 2**32, 4)]
        key = [int(x) for x in rng.integers(0, 2**32, 2)]
        got = inputs.philox4x32_10(*[np.uint32(c) for c in ctr], key[0], key[1])
        assert [int(g) for g in got] == orc.philox4x32_10(ctr, key)


def test_draws_look_uniform():
    """Sanity of the stream (not a pin): bytes of a million draws are close
    to uniform and neighbouring counters are uncorrelated."""
    d = inputs.draw(1, 0, 0, np.arange(1_000_000, dtype=np.uint32))
    counts = np.bincount((d >> np.uint32(24)).astype(np.int64), minlength=256)
    chi2 = ((counts - 1e6 / 256) ** 2 / (1e6 / 256)).sum()
    assert chi2 < 400  # 255 degrees of freedom
    x = d.astype(np.float64) / 2**32
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 5e-3
