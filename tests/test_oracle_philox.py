"""Philox4x32-10 (Salmon et al., SC'11).

The oracle's C implementation is pinned to a third-party library
implementation of the same generator: Triton's `philox` (run on the CPU by
Triton's interpreter), whose key is (seed mod 2^32, seed >> 32) and whose
four counter words are free, agrees with it on every output word.  The
input generator's numpy implementation, written separately, agrees with
both on a million draws over several keys, counters and tags; the CUDA
library's own implementation is held to the same streams by the bit-exact
Wa-Tor and traffic parity tests."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

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


_TRITON_PHILOX = r"""
import json, sys
import numpy as np, torch, triton, triton.language as tl
from triton.language.random import philox

@triton.jit
def words(c0p, c1p, c2p, c3p, out, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out + 4 * i, a)
    tl.store(out + 4 * i + 1, b)
    tl.store(out + 4 * i + 2, c)
    tl.store(out + 4 * i + 3, d)

job = json.loads(sys.stdin.read())
ctr = np.array(job["ctr"], np.uint32)
res = {}
for seed in job["seeds"]:
    cs = [torch.from_numpy(ctr[:, j].copy().view(np.int32)) for j in range(4)]
    out = torch.zeros(4 * len(ctr), dtype=torch.int32)
    words[(1,)](*cs, out, seed, len(ctr))
    res[str(seed)] = out.numpy().view(np.uint32).reshape(-1, 4).tolist()
print(json.dumps(res))
"""


def test_agrees_with_tritons_philox(orc):
    """Every output word of 256 random counters (plus the all-zero and
    all-ones counters) under seven keys, against Triton's Philox4x32-10."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 2**32 - 1
    seeds = [0, 1, 2**31 + 5, 2**32 + 3, 2**40 + 7, 2**63 + 9, 2**64 - 1]
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(dict(ctr=ctr.tolist(), seeds=seeds)),
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    ref = json.loads(r.stdout.strip().splitlines()[-1])
    for seed in seeds:
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, want in zip(ctr, ref[str(seed)]):
            assert orc.philox4x32_10([int(v) for v in c], key) == want, (seed, c)
