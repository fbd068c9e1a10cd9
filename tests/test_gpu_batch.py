"""Batches (smmo_batch_define): independent instances whose objects share
one heap, stepped by one parallel_do per class over all of them (the
thesis' parallel_do, Sec. 5.2.7, over every object of a class); the
asynchronous bulk_new; cellular worlds built on the heap's instance
table."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs, smmo  # noqa: E402
from paper_1908_05845_gb300.workloads import WATOR, World  # noqa: E402

ROWS = [{"kind": 3, "id": 7, "param": (3, -5)}, {"kind": 1, "id": 11, "param": (-2, 100)}]


def batch_heap(rows=ROWS, **cfg):
    h = smmo.Heap(32 << 20, smmo.default_config(**cfg) if cfg else None)
    h.batch_define(rows)
    item = h.register("Item", [("inst", smmo.INSTANCE), ("v", smmo.I32), ("idsum", smmo.I32)])
    return h, item


def expect_affine(v, inst, rounds):
    v = v.astype(np.int64)
    p0 = np.array([r["param"][0] for r in ROWS], np.int64)[inst]
    p1 = np.array([r["param"][1] for r in ROWS], np.int64)[inst]
    kd = np.array([r["kind"] for r in ROWS], np.int64)[inst]
    for _ in range(rounds):
        v = (v * p0 + p1 + kd) & 0xFFFFFFFF
        v = np.where(v >= 1 << 31, v - (1 << 32), v)
    return v.astype(np.int32)


@pytest.mark.parametrize("fanout", [64, 32])
def test_two_instances_of_a_test_class_in_one_parallel_do(fanout):
    h, item = batch_heap(bitmap_fanout=fanout)
    n = 5000
    rng = np.random.default_rng(1)
    inst = rng.integers(0, 2, n).astype(np.int32)
    v = rng.integers(-1000, 1000, n).astype(np.int32)
    cols = [torch.as_tensor(x).cuda() for x in (inst, v, np.zeros(n, np.int32))]
    h.bulk_new(item, n, cols, asynchronous=True)
    for _ in range(2):
        h.parallel_do(item, "test.batch_affine", smmo.BatchAffineArgs(1, 2))
    h.sync()
    hd = h.enumerate_live(item)
    gi, gv, gs = (t.cpu().numpy() for t in h.gather(item, hd, ["inst", "v", "idsum"]))
    assert gi.size == n
    ids = np.array([r["id"] for r in ROWS], np.int32)
    # objects are unordered after enumeration: match them through (inst, v0)
    want = expect_affine(v, inst, 2)
    key_g = np.lexsort((gv, gi))
    key_w = np.lexsort((want, inst))
    assert np.array_equal(gi[key_g], inst[key_w])
    assert np.array_equal(gv[key_g], want[key_w])
    assert np.array_equal(gs[key_g], 2 * ids[inst[key_w]])
    n_inst = ctypes.c_int()
    assert smmo.lib().smmo_batch_count(h.handle, ctypes.byref(n_inst)) == 0 and n_inst.value == 2
    assert h.check() == 0


def test_bulk_new_records_an_instance_outside_the_table():
    h, item = batch_heap()
    cols = [torch.tensor([0, 2, 1], dtype=torch.int32).cuda(), torch.zeros(3, dtype=torch.int32).cuda(),
            torch.zeros(3, dtype=torch.int32).cuda()]
    h.bulk_new(item, 3, cols)
    assert h.sync(raise_on_error=False)[0] == -8  # SMMO_E_BOUNDS


def test_batch_method_needs_an_instance_table():
    h = smmo.Heap(8 << 20)
    a = h.register("A", [("v", smmo.I32), ("w", smmo.I32)])
    h.bulk_new(a, 10, [torch.zeros(10, dtype=torch.int32).cuda(), None])
    mid = ctypes.c_int()
    assert smmo.lib().smmo_method_lookup(h.handle, b"test.batch_affine", ctypes.byref(mid)) == -9
    assert smmo.lib().smmo_method_lookup(h.handle, b"test.add_i32", ctypes.byref(mid)) == 0
    rows = (smmo.InstanceDesc * 1)()
    assert smmo.lib().smmo_batch_define(h.handle, rows, 1) == -10  # geometry fixed: SMMO_E_FROZEN


def test_asynchronous_bulk_new_reports_a_short_heap_at_sync():
    h = smmo.Heap(4 << 20)
    a = h.register("A", [("v", smmo.I32), ("w", smmo.I32)])
    h.freeze()
    st = h.stats()
    cap = h.class_info(a)["capacity"]
    n = cap * (st["num_blocks"] - 2)  # fits the heap, needs almost every block
    h.bulk_new(a, n, [torch.zeros(n, dtype=torch.int32).cuda(), None], asynchronous=True)
    h.bulk_new(a, 4 * cap, [torch.zeros(4 * cap, dtype=torch.int32).cuda(), None], asynchronous=True)
    assert h.sync(raise_on_error=False)[0] == -2  # SMMO_E_OOM: the second creation found too few free blocks
    st = h.stats()
    assert st["live_objects"][a] == n  # the second created nothing
    assert h.check() == 0


def test_plain_world_create_equals_the_batch_form(orc):
    """smmo_world_create (instance i draws with number i) and
    smmo_world_create_batch with explicit rows give the same world; an
    instance of a batch run alone with its own number equals the oracle's
    run of that instance."""
    kinds, sides, init = inputs.batched_initial(3, 6, side_min=8, ratio=4.0)
    n = len(kinds)
    heap = smmo.Heap(64 << 20)
    w = ctypes.c_void_p()
    dev = [torch.as_tensor(x).cuda() for x in init]
    smmo.check(smmo.lib().smmo_world_create(
        heap.handle, n, (ctypes.c_int * n)(*kinds), (ctypes.c_uint32 * n)(*sides), (ctypes.c_uint32 * n)(*sides),
        ctypes.c_uint64(3), None, *[ctypes.c_void_p(t.data_ptr()) for t in dev], None, ctypes.byref(w)),
        "world_create")
    smmo.check(smmo.lib().smmo_world_step(w, 12, None), "world_step")
    N = int(init[0].size)
    out = [torch.empty(N, dtype=d, device="cuda") for d in (torch.int8, torch.int16, torch.int16, torch.uint8)]
    err = ctypes.c_int64()
    smmo.check(smmo.lib().smmo_world_export(w, *[ctypes.c_void_p(t.data_ptr()) for t in out], ctypes.byref(err),
                                            None), "world_export")
    smmo.lib().smmo_world_destroy(w)
    plain = [t.cpu().numpy() for t in out]
    b = World(kinds, sides, sides, 3, *init)
    b.step(12)
    got = b.export()
    assert got[4] == 0 and err.value == 0
    for x, y in zip(plain, got[:4]):
        assert np.array_equal(x, y)
    offs = np.concatenate([[0], np.cumsum(sides.astype(np.int64) ** 2)])
    i = int(np.flatnonzero(kinds == WATOR)[-1])
    sl = slice(offs[i], offs[i + 1])
    sd = int(sides[i])
    alone = World([WATOR], [sd], [sd], 3, *(x[sl] for x in init), inst_ids=[i])
    alone.step(12)
    k, a, e, _, er = alone.export()
    wk, wa, we, _ = orc.wator_run(sd, sd, 3, init[0][sl], init[1][sl], init[2][sl], 12, inst=i)
    assert er == 0 and np.array_equal(k, wk) and np.array_equal(a, wa) and np.array_equal(e, we)
    assert np.array_equal(k, got[0][sl])
