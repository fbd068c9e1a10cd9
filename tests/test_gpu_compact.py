"""GPU tests of compact (CompactGpu, Ch. 6): the relocated multiset is
unchanged, every HANDLE column referring to the class is rewritten, the
fragmentation bound F < 1/(n+1) holds when all candidates are eliminated,
the pass count respects the worst-case bound, and the thesis' worked
examples of source/target assignment and relocation come out as printed."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_05845_gb300 import inputs, smmo  # noqa: E402
from paper_1908_05845_gb300.workloads import WaTor  # noqa: E402


def cuda_i32(a):
    return torch.as_tensor(np.asarray(a, dtype=np.int32)).cuda()


def test_compact_preserves_objects_and_rewrites_handles():
    h = smmo.Heap(64 << 20)
    A = h.register("A", [("v", smmo.I32), ("w", smmo.I32)])
    Rf = h.register("Ref", [("ref", smmo.HANDLE, 1, A), ("val", smmo.I32)])
    n = 64 * 50
    v = np.arange(n)
    hd, first = h.bulk_new(A, n, [cuda_i32(v), cuda_i32(7 * v)], want_handles=True)
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 3, 1))
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 3, 2))
    keep = v % 3 == 0
    h.bulk_new(Rf, int(keep.sum()), [hd[torch.as_tensor(keep).cuda()], cuda_i32(v[keep])])
    h.sync()
    d0 = 50  # every A block is ~1/3 full: all are candidates for n = 2
    st = h.compact(A, n=2, k1=0)
    h.sync()
    assert h.check() == 0
    assert st["blocks_freed"] > 0 and st["objects_moved"] > 0
    assert st["pointers_rewritten"] > 0
    assert st["passes"] <= math.ceil(math.log(d0) / math.log(1.5)) + 1
    hd2 = h.enumerate_live(A)
    vv, ww = (t.cpu().numpy() for t in h.gather(A, hd2, ["v", "w"]))
    assert np.array_equal(np.sort(vv), v[keep]) and np.array_equal(ww[np.argsort(vv)], 7 * v[keep])
    rh = h.enumerate_live(Rf)
    ref, val = h.gather(Rf, rh, ["ref", "val"])
    (tv,) = h.gather(A, ref, ["v"])
    assert np.array_equal(tv.cpu().numpy(), val.cpu().numpy())
    stt = h.stats()
    assert stt["fragmentation"][A] < 1 / 3
    assert stt["live_objects"][A] == keep.sum()


def _kill_all_but(h, A, fill_per_block, nblocks, cap):
    n = nblocks * cap
    v = np.arange(n)
    kill = np.zeros(n, np.int32)
    for b, f in fill_per_block.items():
        kill[b * cap + f:(b + 1) * cap] = 1
    _, first = h.bulk_new(A, n, [cuda_i32(v), cuda_i32(kill)])
    assert first == 0
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(1, 2, 1))
    h.sync()
    return v, kill


def where_now(h, A):
    hd = h.enumerate_live(A)
    (vv,) = h.gather(A, hd, ["v"])
    blk = (hd.cpu().numpy().astype(np.int64) & 0xFFFFFFFF) >> 6
    return dict(zip(vv.cpu().numpy().tolist(), blk.tolist()))


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "compactgpu_worked_examples.txt")


def worked_examples():
    """Cases of tests/golden/compactgpu_worked_examples.txt (Sec. 6.3.3)."""
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, fills, moves, left = (p.strip() for p in line.split("|"))
        name, n, k1, cap = head.split()
        fills = {int(b): int(f) for b, f in (x.split(":") for x in fills.split())}
        mv = []
        for x in moves.split():
            src, rest = x.split(">")
            tgt, cnt = rest.split(":")
            mv.append((int(src), int(tgt), int(cnt)))
        cases.append((name, int(n), int(k1), int(cap), fills, mv, [int(x) for x in left.split()]))
    return cases


@pytest.mark.parametrize("case", worked_examples(), ids=lambda c: c[0])
def test_worked_examples(case):
    """The thesis' worked examples of source/target assignment (n = 2) and
    relocation (n = 3, capacity 32): one pass moves each source's objects
    into its targets in order, as many into a target as it has free slots;
    the left-over candidate and every other block keep their objects."""
    name, n, k1, cap, fills, moves, left = case
    cfg = smmo.default_config(block_data_bytes=256) if cap == 32 else None
    h = smmo.Heap(32 << 20, cfg)
    A = h.register("A", [("v", smmo.I32), ("kill", smmo.I32)])
    h.freeze()
    assert h.class_info(A)["capacity"] == cap
    _kill_all_but(h, A, fills, max(fills) + 1, cap)
    st = h.compact(A, n=n, k1=k1)
    h.sync()
    sources = sorted({s for s, _, _ in moves})
    assert st["passes"] == 1 and st["blocks_freed"] == len(sources)
    assert st["objects_moved"] == sum(c for _, _, c in moves)
    loc = where_now(h, A)
    for s in sources:
        objs = range(s * cap, s * cap + fills[s])
        want = sorted(t for src, t, c in moves if src == s for _ in range(c))
        assert sorted(loc[x] for x in objs) == want, s
    assert all(loc[x] == x // cap for x in loc if x // cap not in sources)
    assert all(any(loc[x] == b for x in loc) for b in left)
    assert h.check() == 0


def test_wator_with_periodic_compaction_matches_oracle(orc):
    W = H = 256
    k, a, e = inputs.wator_initial(W, H, 2)
    sim = WaTor(W, H, 2, k, a, e)
    F, S = sim.class_ids["Fish"], sim.class_ids["Shark"]
    for _ in range(6):
        sim.step(10)
        for c in (F, S):
            sim.heap.compact(c, n=2, k1=0)
            assert sim.heap.stats()["fragmentation"][c] < 1 / 3
    got = sim.read()
    want = orc.wator_run(W, H, 2, k, a, e, 60)
    for g, w in zip(got, want[:3]):
        assert np.array_equal(g, w)
    assert sim.heap.check() == 0
    sim.sync()


def test_synthetic_two_class_benchmark_small():
    """The synthetic defragmentation benchmark (Sec. 6.4) at 64 x 1000
    objects per class: after compact(A, n=3) every A object survives with
    its fields, every B reference leads to the same A object as before, no
    A candidate (fill <= 48 of 64) is left, and the phases were timed."""
    from paper_1908_05845_gb300.workloads import CompactSynthetic
    w = CompactSynthetic(64 * 1000, seed=2)
    h = w.heap
    st0 = h.stats()
    assert st0["live_objects"][w.A] == w.survivors
    assert 0.55 < 1 - w.survivors / w.n < 0.65
    st = h.compact(w.A, n=3, k1=0)
    v = w.verify()
    assert v == {"a_objects_ok": True, "b_references_ok": True, "heap_violations": 0}
    assert st["candidates_left"] < 4 and st["passes"] >= 2
    assert st["objects_moved"] > 0 and st["pointers_rewritten"] > 0
    assert min(st["scan_ms"], st["copy_ms"], st["state_ms"], st["rewrite_ms"]) > 0
    st1 = h.stats()
    assert st1["blocks"][w.A] < st0["blocks"][w.A] * 0.6
    assert st1["fragmentation"][w.A] < 0.25 + 1.0 / 64
    w.close()


def test_self_referencing_ring_survives_multi_pass_compaction():
    """A class referring to itself (a ring through the survivors) keeps
    every link through several passes, so objects that move twice are
    reached by following forwarding pointers across passes."""
    h = smmo.Heap(64 << 20)
    N = h.register("Node", [("next", smmo.HANDLE), ("v", smmo.I32), ("kill", smmo.I32)])
    n = 64 * 300
    rng = np.random.default_rng(5)
    kill = (rng.random(n) < 0.7).astype(np.int32)
    v = np.arange(n)
    nul = np.full(n, -1, np.int32)
    hd, _ = h.bulk_new(N, n, [cuda_i32(nul), cuda_i32(v), cuda_i32(kill)], want_handles=True)
    alive = np.flatnonzero(kill == 0)
    nxt = np.full(n, -1, np.int64)
    nxt[alive] = np.roll(alive, -1)
    hd_np = hd.cpu().numpy()
    table = np.where(nxt >= 0, hd_np[np.maximum(nxt, 0)], -1).astype(np.int32)
    tt = cuda_i32(table)
    h.parallel_do(N, "test.set_ref_from", smmo.SetRefFromArgs(0, 1, tt.data_ptr()))
    h.parallel_do(N, "test.free_self_if", smmo.FreeSelfIfArgs(2, 2, 1))
    h.sync()
    st = h.compact(N, n=3, k1=0)
    assert st["passes"] >= 3 and st["objects_moved"] > len(alive) // 2
    assert h.check() == 0
    hh = h.enumerate_live(N)
    nv, vv = h.gather(N, hh, ["next", "v"])
    (tv,) = h.gather(N, nv, ["v"])
    got = dict(zip(vv.cpu().numpy().tolist(), tv.cpu().numpy().tolist()))
    assert sorted(got) == alive.tolist()
    assert all(got[a] == b for a, b in zip(alive.tolist(), np.roll(alive, -1).tolist()))


def test_candidate_count_and_massive_deallocation_policy():
    """Sec. 6.3.8: candidates counted for several n against the fills set
    by hand; the policy compacts only once the count reaches k2 n / (n + 1)
    (k2 absolute or as a fraction of the heap's blocks)."""
    h = smmo.Heap(32 << 20)
    A = h.register("A", [("v", smmo.I32), ("kill", smmo.I32)])
    h.freeze()
    cap = h.stats()["capacity"][A]
    fills = {b: f for b, f in enumerate([1, 5, cap // 2, cap // 2 + 1, cap - 1, cap, 3, cap // 3] * 5)}
    _kill_all_but(h, A, fills, len(fills), cap)
    h.sync()
    for n in (1, 2, 5, 63):
        limit = cap * n // (n + 1)
        assert h.defrag_candidates(A, n) == sum(1 for f in fills.values() if f <= limit), n
    n = 2
    cand = h.defrag_candidates(A, n)
    M = h.stats()["num_blocks"]
    thr_blocks = (cand * (n + 1)) // n  # the largest k2 with k2 n / (n + 1) <= cand
    ran, st = h.compact_if(A, n, k2_blocks=thr_blocks + 1)
    assert not ran and st["candidates_left"] == cand and st["passes"] == 0
    ran, st = h.compact_if(A, n, k2_fraction=min(1.0, (thr_blocks + 1.5) / M))
    assert not ran
    live = h.stats()["live_objects"][A]
    ran, st = h.compact_if(A, n, k2_blocks=thr_blocks)
    assert ran and st["passes"] >= 1 and st["blocks_freed"] > 0
    h.sync()
    assert h.check() == 0 and h.stats()["live_objects"][A] == live
    assert h.defrag_candidates(A, n) < cand


def test_remap_caller_handles_after_compaction():
    """Handles held outside the heap follow the objects through a
    multi-pass compaction (smmo_remap_handles); once an object is allocated
    afterwards the forwarding slots may be gone and remap refuses."""
    h = smmo.Heap(64 << 20)
    A = h.register("A", [("v", smmo.I32), ("w", smmo.I32)])
    n = 64 * 80
    v = np.arange(n)
    hd, _ = h.bulk_new(A, n, [cuda_i32(v), cuda_i32(np.zeros(n))], want_handles=True)
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 4, 1))
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 4, 2))
    h.parallel_do(A, "test.free_self_if", smmo.FreeSelfIfArgs(0, 4, 3))
    keep = v % 4 == 0
    held = hd[torch.as_tensor(keep).cuda()].clone()
    st = h.compact(A, n=3, k1=0)
    h.sync()
    assert st["passes"] >= 2 and st["objects_moved"] > 0
    (before,) = h.gather(A, held, ["v"])  # stale handles: not all still name their object
    assert not np.array_equal(before.cpu().numpy(), v[keep])
    h.remap_handles(held)
    (after,) = h.gather(A, held, ["v"])
    assert np.array_equal(after.cpu().numpy(), v[keep])
    code, _ = h.last_device_error()
    assert code == 0
    h.bulk_new(A, 64, [cuda_i32(np.arange(64)), cuda_i32(np.zeros(64))])
    with pytest.raises(smmo.SmmoError):
        h.remap_handles(held)
