"""Allocation-free export (smmo_world_export_noalloc).

Callers that cannot allocate device memory at the point where they read the
simulation state (their own memory pool owns the device, or a cudaMalloc's
device-wide synchronisation would stall a time-stepped loop) use this entry
point; its scratch is a fixed array inside the library.  The test calls it
through the C ABI and checks that it reports exactly what the allocating
export reports, on two calls in a row (the second call must clear what the
first left in the shared array), before and after more steps.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs, smmo  # noqa: E402
from paper_1908_05845_gb300.workloads import Life, WaTor  # noqa: E402

MAX_CELLS = 1 << 24


def export_noalloc(world):
    N = world.total
    k = torch.empty(N, dtype=torch.int8, device="cuda")
    a = torch.empty(N, dtype=torch.int16, device="cuda")
    e = torch.empty(N, dtype=torch.int16, device="cuda")
    s = torch.empty(N, dtype=torch.uint8, device="cuda")
    err = ctypes.c_int64(-1)
    st = smmo.lib().smmo_world_export_noalloc(
        world._w, ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(a.data_ptr()),
        ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(s.data_ptr()), ctypes.byref(err),
        smmo._stream(world.stream))
    return st, (k.cpu().numpy(), a.cpu().numpy(), e.cpu().numpy(), s.cpu().numpy()), err.value


def same_as_export(world):
    *ref, ref_err = world.export()
    for _ in range(2):
        st, got, err = export_noalloc(world)
        assert st == 0
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)
        assert err == ref_err == 0


def test_noalloc_export_matches_export_wator():
    k, a, e = inputs.wator_initial(96, 80, 7)
    sim = WaTor(96, 80, 7, k, a, e)
    sim.step(10)
    same_as_export(sim)
    sim.step(7)
    same_as_export(sim)
    sim.sync()


def test_noalloc_export_matches_export_life():
    k, s = inputs.gol_initial(128, 72, 3)
    sim = Life(128, 72, k, s)
    sim.step(9)
    same_as_export(sim)
    sim.step(4)
    same_as_export(sim)
    sim.sync()


def test_noalloc_export_rejects_worlds_above_the_limit():
    side = 4097  # 4097 * 4096 > 2^24 cells
    k = np.zeros(side * 4096, np.uint8)
    k[:3] = 1
    sim = Life(side, 4096, k, np.zeros_like(k))
    st, _, _ = export_noalloc(sim)
    assert st == -9  # SMMO_E_UNSUPPORTED: beyond the fixed scratch size
    sim.close()
