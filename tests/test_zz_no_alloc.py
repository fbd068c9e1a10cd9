"""Allocation-free export (smmo_world_export_noalloc).

Callers that cannot allocate device memory at the point where they read the
simulation state (their own memory pool owns the device, or a cudaMalloc's
device-wide synchronisation would stall a time-stepped loop) use this entry
point; its scratch is a fixed array inside the library.  The tests call it
through the C ABI and check that it reports exactly what the allocating
export reports, on two calls in a row (the second call must clear what the
first left in the shared array), before and after more steps; that it
counts a planted second agent on a cell exactly as the allocating export
does; that it works at exactly its size limit and refuses one row more; and
that it takes no memory from the device's stream-ordered pool (the one the
allocating export draws from), checked with the pool's high-water mark.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs, smmo  # noqa: E402
from paper_1908_05845_gb300.workloads import Life, WaTor  # noqa: E402

MAX_CELLS = 1 << 24


def outputs(world):
    N = world.total
    return [torch.empty(N, dtype=d, device="cuda") for d in (torch.int8, torch.int16, torch.int16, torch.uint8)]


def call_noalloc(world, outs):
    err = ctypes.c_int64(-1)
    st = smmo.lib().smmo_world_export_noalloc(world._w, *[ctypes.c_void_p(t.data_ptr()) for t in outs],
                                              ctypes.byref(err), smmo._stream(world.stream))
    return st, err.value


def export_noalloc(world):
    outs = outputs(world)
    st, err = call_noalloc(world, outs)
    return st, tuple(t.cpu().numpy() for t in outs), err


def same_as_export(world, want_errors=0):
    *ref, ref_err = world.export()
    for _ in range(2):
        st, got, err = export_noalloc(world)
        assert st == 0
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)
        assert err == ref_err == want_errors


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


def test_noalloc_export_counts_a_second_agent_on_a_cell():
    """Fish A's cell field is set to fish B's cell through the heap buffer:
    cell B then holds two agents and does not point back at A, and A's own
    cell points at an agent that lives elsewhere, three errors; both
    exports count them alike, twice in a row."""
    k, a, e = inputs.wator_initial(64, 48, 5)
    sim = WaTor(64, 48, 5, k, a, e)
    sim.step(6)
    F = sim.class_ids["Fish"]
    hd = sim.heap.enumerate_live(F, False)
    cells = torch.empty(hd.numel(), dtype=torch.int32, device="cuda")
    col = 0  # Fish's first column: the cell inherited from WAgent
    dst = (ctypes.c_void_p * 1)(cells.data_ptr())
    assert smmo.lib().smmo_gather_fields(sim.heap.handle, F, ctypes.c_void_p(hd.data_ptr()),
                                         ctypes.c_int64(hd.numel()), (ctypes.c_int * 1)(col), 1, dst,
                                         smmo._stream(sim.stream)) == 0
    cells = cells.cpu().numpy()
    handles = hd.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    ha, cell_b = int(handles[0]), int(cells[1])
    lay = sim.heap.layout(F)
    addr = lay["data_base"] + (ha >> 6) * lay["block_bytes"] + lay["col_off"][col] + (ha & 63) * 4
    off = addr - sim.heap.buf.data_ptr()
    sim.heap.buf[off:off + 4].view(torch.int32)[0] = cell_b
    torch.cuda.synchronize()
    same_as_export(sim, want_errors=3)
    sim.close()


def test_noalloc_export_at_exactly_the_limit():
    """4096 x 4096 = 2^24 cells, the largest world it accepts, with agents
    on the last cells, so the last word of the fixed bitmap is used."""
    side = 4096
    k = np.zeros(side * side, np.uint8)
    k[-3:] = 1
    k[-70] = 2
    sim = Life(side, side, k, np.zeros_like(k))
    assert sim.total == MAX_CELLS
    same_as_export(sim)
    sim.close()


def test_noalloc_export_rejects_worlds_above_the_limit():
    side = 4097  # 4097 * 4096 > 2^24 cells
    k = np.zeros(side * 4096, np.uint8)
    k[:3] = 1
    sim = Life(side, 4096, k, np.zeros_like(k))
    st, _, _ = export_noalloc(sim)
    assert st == -9  # SMMO_E_UNSUPPORTED: beyond the fixed scratch size
    sim.close()


def _cudart():
    """The CUDA runtime the library itself is linked against."""
    smmo.lib()
    for line in open("/proc/self/maps"):
        if "libcudart.so" in line:
            return ctypes.CDLL(line.split()[-1])
    return ctypes.CDLL("libcudart.so.13")


def pool_use_during(fn):
    """(bytes in use before, high-water mark during fn) of the current
    device's stream-ordered memory pool, and cudaMemGetInfo's free bytes
    before and after fn."""
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    torch.cuda.synchronize()
    used, high, zero = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, 0x7, ctypes.byref(used)) == 0  # used, current
    assert rt.cudaMemPoolSetAttribute(pool, 0x8, ctypes.byref(zero)) == 0  # high-water := current
    free0 = torch.cuda.mem_get_info()[0]
    fn()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert rt.cudaMemPoolGetAttribute(pool, 0x8, ctypes.byref(high)) == 0  # used, high-water
    return used.value, high.value, free0, free1


def test_noalloc_export_allocates_nothing():
    k, a, e = inputs.wator_initial(128, 96, 2)
    sim = WaTor(128, 96, 2, k, a, e)
    sim.step(5)
    outs = outputs(sim)
    assert call_noalloc(sim, outs) == (0, 0)  # first call: symbol lookup, warm-up
    used, high, free0, free1 = pool_use_during(lambda: call_noalloc(sim, outs))
    assert high == used and free1 == free0
    # the allocating export, measured the same way, does take pool memory
    used, high, _, _ = pool_use_during(lambda: sim.export())
    assert high >= used + sim.total * 4
    sim.close()
