"""GPU tests of the heap core: bulk creation, parallel_do, device new /
delete (warp-aggregated allocation, block invalidation), enumeration,
inheritance, statistics and the post-kernel invariants (Sec. 5.4)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import smmo  # noqa: E402


def make(nbytes=64 << 20, **cfg):
    h = smmo.Heap(nbytes, smmo.default_config(**cfg) if cfg else None)
    A = h.register("A", [("v", smmo.I32), ("w", smmo.I32)])
    B = h.register("B", [("marker", smmo.I32), ("parent", smmo.I32)])
    C = h.register("C", [("x", smmo.I32), ("pad", smmo.I16, 3)])
    return h, A, B, C


def values(h, cls, names, sub=True):
    hd = h.enumerate_live(cls, sub)
    return hd, [t.cpu().numpy() for t in h.gather(cls, hd, names)]


def test_bulk_new_enumerate_gather():
    h, A, B, C = make()
    n = 10_000
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    w = v * 7
    hd, first = h.bulk_new(A, n, [v, w], want_handles=True)
    assert first == 0
    cap = h.class_info(A)["capacity"]
    want = (np.arange(n) // cap) * 64 + np.arange(n) % cap
    assert np.array_equal(hd.cpu().numpy().astype(np.int64) & 0xFFFFFFFF, want)
    hd2, (vv, ww) = values(h, A, ["v", "w"])
    assert hd2.numel() == n
    o = np.argsort(vv)
    assert np.array_equal(vv[o], np.arange(n)) and np.array_equal(ww[o], 7 * np.arange(n))
    assert h.check() == 0
    st = h.stats()
    assert st["live_objects"][A] == n and st["blocks"][A] == -(-n // cap)
    h.sync()


def test_parallel_do_add_and_free_self():
    h, A, B, C = make()
    n = 50_001
    h.bulk_new(A, n, [torch.arange(n, dtype=torch.int32, device="cuda"), None])
    h.parallel_do(A, "test.add_i32", smmo.AddI32Args(0, 5))
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 3, 0))
    h.sync()
    _, (vv,) = values(h, A, ["v"])
    want = np.arange(n) + 5
    want = want[want % 3 != 0]
    assert np.array_equal(np.sort(vv), want)
    assert h.check() == 0
    st = h.stats()
    assert st["frees"][A] == n - want.size
    assert 0.3 < st["fragmentation"][A] < 0.36  # one third of every block freed


def test_device_new_coalesced_and_counts():
    h, A, B, C = make()
    n = 20_000
    h.bulk_new(A, n, [torch.arange(n, dtype=torch.int32, device="cuda"), None])
    for k in (1, 3):
        h.parallel_do(A, "test.alloc_k", smmo.AllocKArgs(B, k, 0, 1, 0, 77))
    h.sync()
    _, (mk, par) = values(h, B, ["marker", "parent"])
    assert mk.size == 4 * n and np.all(mk == 77)
    assert np.array_equal(np.bincount(par, minlength=n), np.full(n, 4))
    st = h.stats()
    assert st["allocs"][B] == 4 * n and st["live_objects"][B] == 4 * n
    assert st["fragmentation"][B] < 0.1  # new objects fill active blocks first
    assert h.check() == 0


@pytest.mark.parametrize("fanout", [64, 32])
def test_replace_alloc_and_free_in_one_kernel(fanout):
    h, A, B, C = make(bitmap_fanout=fanout)
    n = 30_000
    h.bulk_new(A, n, [torch.arange(n, dtype=torch.int32, device="cuda"), None])
    for _ in range(3):
        h.parallel_do(A, "test.replace", smmo.ReplaceArgs(C, 0, 0))
        h.sync()
        assert h.check() == 0
        h.parallel_do(C, "test.replace", smmo.ReplaceArgs(A, 0, 0))
        h.sync()
        assert h.check() == 0
    _, (vv,) = values(h, A, ["v"])
    assert np.array_equal(np.sort(vv), np.arange(n))
    st = h.stats()
    assert st["live_objects"][C] == 0 and st["blocks"][C] == 0
    # every A block of the first generation was emptied and invalidated
    assert st["free_blocks"] + st["blocks"][A] == st["num_blocks"]


@pytest.mark.parametrize("fanout", [64, 32])
def test_churn_against_host_model(fanout):
    h, A, B, C = make(bitmap_fanout=fanout)
    rng = np.random.default_rng(0)
    n = 8192
    h.bulk_new(A, n, [torch.arange(n, dtype=torch.int32, device="cuda"), None])
    live = np.arange(n)
    for r in range(12):
        mod, rem = int(rng.integers(2, 6)), int(rng.integers(0, 2))
        h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, mod, rem))
        live = live[live % mod != rem]
        h.parallel_do(A, "test.alloc_k", smmo.AllocKArgs(A, 1, 0, 1, 0, 0))
        # every survivor allocated one A with v = 0 (marker), which then
        # gets renumbered by the add below so values stay distinct
        h.sync()
        assert h.check() == 0
        _, (vv,) = values(h, A, ["v"])
        assert np.count_nonzero(vv == 0) >= live.size
        h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 1 << 30, 0))  # frees v == 0
        live = live[live != 0]
        h.sync()
        _, (vv,) = values(h, A, ["v"])
        assert np.array_equal(np.sort(vv), live)
        assert h.check() == 0


def test_inheritance_parallel_do_visits_subclasses():
    h = smmo.Heap(32 << 20)
    Ag = h.register("Agent", [("v", smmo.I32)], abstract=True)
    F = h.register("Fish", [("age", smmo.I16)], parent=Ag)
    S = h.register("Shark", [("age", smmo.I16), ("energy", smmo.I16)], parent=Ag)
    h.bulk_new(F, 1000, [torch.zeros(1000, dtype=torch.int32, device="cuda"), None])
    h.bulk_new(S, 300, [torch.ones(300, dtype=torch.int32, device="cuda"), None, None])
    h.parallel_do(Ag, "test.add_i32", smmo.AddI32Args(0, 10))
    h.sync()
    hd = h.enumerate_live(Ag, True)
    (v,) = h.gather(Ag, hd, ["v"])
    assert sorted(v.cpu().tolist()) == [10] * 1000 + [11] * 300
    assert h.enumerate_live(F, False).numel() == 1000


def test_device_oom_is_reported_not_hung():
    h, A, B, C = make(nbytes=1 << 20)
    h.freeze()
    M = h.stats()["num_blocks"]
    n = 64 * (M // 32)  # each A allocates 64 B objects: 2x more blocks than exist
    h.bulk_new(A, n, [torch.arange(n, dtype=torch.int32, device="cuda"), None])
    h.parallel_do(A, "test.alloc_k", smmo.AllocKArgs(B, 64, 0, 1, 0, 1))
    st, _ = h.sync(raise_on_error=False)
    assert st == -3
    assert h.check() == 0
    assert h.stats()["free_blocks"] == 0 and M > 4


def test_double_free_detected():
    h = smmo.Heap(16 << 20)
    B = h.register("B", [("x", smmo.I32)])
    Rf = h.register("R", [("ref", smmo.HANDLE, 1, B)])
    hb, _ = h.bulk_new(B, 10, [torch.zeros(10, dtype=torch.int32, device="cuda")], want_handles=True)
    ref = torch.cat([hb, hb[:1]])  # object 0 referenced twice
    h.bulk_new(Rf, 11, [ref])
    h.parallel_do(Rf, "test.free_ref", smmo.FreeRefArgs(0))
    st, detail = h.sync(raise_on_error=False)
    assert st == -7 and detail == int(hb[0].item()) & 0xFFFFFFFF
    assert h.check() == 0


def test_parallel_do_and_reduce_all_reducers():
    """parallel_do_and_reduce over a class with holes and a subclass: sum,
    min, max, or, and and a count equal numpy over the live objects; an
    empty class gives the reducers' identities; a plain method is refused."""
    h = smmo.Heap(64 << 20)
    A = h.register("A", [("v", smmo.I32)])
    B = h.register("B", [("w", smmo.I32)], parent=A)
    rng = np.random.default_rng(3)
    va = rng.integers(-10**6, 10**6, 5000).astype(np.int32)
    vb = rng.integers(0, 1 << 20, 3000).astype(np.int32)
    h.bulk_new(A, len(va), [torch.as_tensor(va).cuda()])
    h.bulk_new(B, len(vb), [torch.as_tensor(vb).cuda(), torch.zeros(len(vb), dtype=torch.int32).cuda()])
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 7, 3))  # holes in A and B
    keep = np.concatenate([va, vb])
    keep = keep[((keep % 7) + 7) % 7 != 3].astype(np.int64)
    arg = smmo.ValueI32Args(0, 0)
    assert h.parallel_do_and_reduce(A, "test.value_i32", arg, smmo.REDUCE_SUM) == keep.sum()
    assert h.parallel_do_and_reduce(A, "test.value_i32", arg, smmo.REDUCE_MIN) == keep.min()
    assert h.parallel_do_and_reduce(A, "test.value_i32", arg, smmo.REDUCE_MAX) == keep.max()
    orv = 0
    andv = -1
    for x in keep.tolist():
        orv |= x
        andv &= x
    assert h.parallel_do_and_reduce(A, "test.value_i32", arg, smmo.REDUCE_OR) == orv
    assert h.parallel_do_and_reduce(A, "test.value_i32", arg, smmo.REDUCE_AND) == andv
    assert h.parallel_do_and_reduce(A, "test.value_i32", smmo.ValueI32Args(0, 1), smmo.REDUCE_SUM) == len(keep)
    C = smmo.Heap(8 << 20)
    E = C.register("E", [("v", smmo.I32)])
    C.bulk_new(E, 1, [torch.zeros(1, dtype=torch.int32).cuda()])
    C.parallel_do(E, "test.free_self_if", smmo.FreeSelfIfArgs(0, 0, 0))
    assert C.parallel_do_and_reduce(E, "test.value_i32", arg, smmo.REDUCE_MIN) == 2**63 - 1
    assert C.parallel_do_and_reduce(E, "test.value_i32", arg, smmo.REDUCE_SUM) == 0
    with pytest.raises(smmo.SmmoError):
        h.parallel_do_and_reduce(A, "test.add_i32", smmo.AddI32Args(0, 1), smmo.REDUCE_SUM)
    with pytest.raises(smmo.SmmoError):
        h.parallel_do(A, "test.value_i32", arg)
    h.sync()


def test_bounded_wait_runs_out_and_context_stays_usable():
    """A grid-barrier wait that nothing releases gives up after its poll
    limit with SMMO_E_TIMEOUT (read on the host); the next kernels run."""
    h = smmo.Heap(8 << 20)
    A = h.register("A", [("v", smmo.I32)])
    h.freeze()
    t0 = time.perf_counter()
    smmo.check(smmo.lib().smmo_selftest_barrier_timeout(h.handle, 4096, smmo._stream(None)), "selftest")
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(smmo.SmmoError) as ei:
        h.sync()
    assert ei.value.status == -6  # SMMO_E_TIMEOUT
    h.sync()  # the error was cleared
    v = torch.arange(640, dtype=torch.int32, device="cuda")
    h.bulk_new(A, 640, [v])
    h.parallel_do(A, "test.add_i32", smmo.AddI32Args(0, 5))
    (got,) = h.gather(A, h.enumerate_live(A), ["v"])
    assert np.array_equal(np.sort(got.cpu().numpy()), np.arange(640) + 5)


def test_calls_on_a_class_without_objects():
    """Degenerate calls on a class with no objects are no-ops: creating
    zero objects, a do-all, an enumeration and a gather, a compaction (no
    candidates: no pass); the class works normally afterwards."""
    h, A, B, C = make()
    h.bulk_new(B, 100, [torch.arange(100, dtype=torch.int32, device="cuda"), None])
    hd, first = h.bulk_new(A, 0, None, want_handles=True)
    assert hd.numel() == 0 and first == -1
    h.parallel_do(A, "test.add_i32", smmo.AddI32Args(0, 5))
    hd = h.enumerate_live(A)
    assert hd.numel() == 0
    (v,) = h.gather(A, hd, ["v"])
    assert v.numel() == 0
    cs = h.compact(A, 1, 0)
    assert cs["passes"] == 0 and cs["objects_moved"] == 0 and cs["blocks_freed"] == 0
    h.sync()
    assert h.check() == 0
    st = h.stats()
    assert st["live_objects"][A] == 0 and st["live_objects"][B] == 100
    h.bulk_new(A, 70, [torch.arange(70, dtype=torch.int32, device="cuda"), None])
    h.parallel_do(A, "test.add_i32", smmo.AddI32Args(0, 5))
    h.sync()
    _, (vv,) = values(h, A, ["v"])
    assert np.array_equal(np.sort(vv), np.arange(5, 75))
    assert h.check() == 0
