"""Python side of the cellular workloads (smmo_world_* in include/smmo.h).

Argument marshalling only; the simulation runs in libsmmo.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import smmo

LIFE, WATOR = 0, 1
# how a Wa-Tor iteration is launched (smmo_world_set_step_kernels)
FOUR_DO_ALLS, PHASED1, PHASED2 = 0, 1, 2
QUEUED = 4  # or-ed with one of the above: creations queued and made by a launch of their own
MARKED = 8  # or-ed with FOUR_DO_ALLS: the update runs only on the agents its prepare marked


class WatorParams(ctypes.Structure):
    _fields_ = [("fish_breed", ctypes.c_int), ("shark_breed", ctypes.c_int),
                ("starve", ctypes.c_int), ("breed_strict", ctypes.c_int)]


def heap_bytes_for(total_cells: int, agent_fill: float = 1.0) -> int:
    """Heap buffer size: the dense Cell blocks plus room for agents on up to
    `agent_fill` of the cells at 50% block fill, plus metadata slack."""
    blocks = total_cells / 64.0
    return int((blocks * (1.0 + 2.0 * agent_fill) + 4096) * 800) + (32 << 20)


class World:
    """Independent Life / Wa-Tor instances sharing one SMMO heap."""

    def __init__(self, kinds, widths, heights, seed: int, init_kind, init_age=None,
                 init_energy=None, init_state=None, params: WatorParams | None = None,
                 heap_bytes: int | None = None, config: smmo.HeapConfig | None = None,
                 stream=None, inst_ids=None, step_kernels: int | None = None):
        """inst_ids: the instance numbers of the draws (default 0..n-1), so
        that one instance of a larger batch can be run alone.  step_kernels:
        FOUR_DO_ALLS, PHASED1 or PHASED2 (the library's default when None)."""
        n = len(kinds)
        self.kinds = [int(k) for k in kinds]
        self.W = [int(w) for w in widths]
        self.H = [int(h) for h in heights]
        self.sizes = [w * h for w, h in zip(self.W, self.H)]
        self.total = int(sum(self.sizes))
        self.stream = stream
        dev = torch.device("cuda")

        def dt(a, dtype):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return a.to(dev, dtype).contiguous()
            return torch.as_tensor(np.ascontiguousarray(a)).to(dev, dtype).contiguous()

        k = dt(init_kind, torch.int8)
        a = dt(init_age, torch.int16)
        e = dt(init_energy, torch.int16)
        s = dt(init_state, torch.uint8)
        self.heap = smmo.Heap(heap_bytes or heap_bytes_for(self.total), config, stream=stream)
        self._w = ctypes.c_void_p()
        ids = list(range(n)) if inst_ids is None else [int(i) for i in inst_ids]
        rows = (smmo.InstanceDesc * n)()
        base = 0
        for i in range(n):
            rows[i] = smmo.InstanceDesc(self.kinds[i], ids[i], self.W[i], self.H[i], base, self.sizes[i],
                                        (ctypes.c_int64 * 2)(0, 0))
            base += self.sizes[i]
        p = ctypes.byref(params) if params is not None else None

        def ptr(t):
            return ctypes.c_void_p(t.data_ptr()) if t is not None else None

        smmo.check(smmo.lib().smmo_world_create_batch(
            self.heap.handle, rows, n, ctypes.c_uint64(seed), p, ptr(k), ptr(a), ptr(e),
            ptr(s), smmo._stream(stream), ctypes.byref(self._w)), "world_create")
        ids = (ctypes.c_int * 7)()
        smmo.check(smmo.lib().smmo_world_info(self._w, None, ids, None), "world_info")
        names = ["Cell", "WAgent", "Fish", "Shark", "LAgent", "Alive", "Candidate"]
        self.class_ids = dict(zip(names, list(ids)))
        if step_kernels is not None:
            self.set_step_kernels(step_kernels)

    def set_step_kernels(self, mode: int):
        """FOUR_DO_ALLS, PHASED1 or PHASED2, optionally | QUEUED, and
        FOUR_DO_ALLS optionally | MARKED (see smmo_world_set_step_kernels)."""
        smmo.check(smmo.lib().smmo_world_set_step_kernels(self._w, int(mode)), "world_set_step_kernels")

    def step(self, n: int = 1):
        smmo.check(smmo.lib().smmo_world_step(self._w, n, smmo._stream(self.stream)), "world_step")

    def set_life_rule(self, survive: int, born: int, block: int):
        """Rule of the Life-kind instances (see smmo_world_set_life_rule)."""
        smmo.check(smmo.lib().smmo_world_set_life_rule(self._w, ctypes.c_uint32(survive), ctypes.c_uint32(born),
                                                       ctypes.c_uint32(block)), "world_set_life_rule")

    def capture(self, n: int):
        """Captures n steps into a CUDA graph (needs a non-default stream)."""
        smmo.check(smmo.lib().smmo_world_capture(self._w, n, smmo._stream(self.stream)), "world_capture")

    def replay(self):
        smmo.check(smmo.lib().smmo_world_replay(self._w, smmo._stream(self.stream)), "world_replay")

    def step_profiled(self, n: int = 1):
        """Steps n times and returns (phase_ms[16], step_ms, launches): device
        times from CUDA events on the launching stream (see the C header)."""
        ph = (ctypes.c_double * 16)()
        sm = ctypes.c_double()
        la = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_world_step_profiled(self._w, n, ph, ctypes.byref(sm),
                                                       ctypes.byref(la), smmo._stream(self.stream)),
                   "world_step_profiled")
        return list(ph), sm.value, la.value

    def export(self):
        """Per-cell numpy arrays (kind, age, energy, state) and error count."""
        N = self.total
        dev = torch.device("cuda")
        k = torch.empty(N, dtype=torch.int8, device=dev)
        a = torch.empty(N, dtype=torch.int16, device=dev)
        e = torch.empty(N, dtype=torch.int16, device=dev)
        s = torch.empty(N, dtype=torch.uint8, device=dev)
        err = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_world_export(
            self._w, ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(a.data_ptr()),
            ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(s.data_ptr()), ctypes.byref(err),
            smmo._stream(self.stream)), "world_export")
        return k.cpu().numpy(), a.cpu().numpy(), e.cpu().numpy(), s.cpu().numpy(), err.value

    def split(self, arr):
        out, o = [], 0
        for n in self.sizes:
            out.append(arr[o:o + n])
            o += n
        return out

    def sync(self):
        return self.heap.sync()

    def close(self):
        if self._w:
            smmo.lib().smmo_world_destroy(self._w)
            self._w = ctypes.c_void_p()
        self.heap.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WaTor(World):
    """A single Wa-Tor instance (thesis Sec. 7.6)."""

    def __init__(self, W, H, seed, kind, age, energy, **kw):
        super().__init__([WATOR], [W], [H], seed, kind, age, energy, None, **kw)

    def read(self):
        k, a, e, _, err = self.export()
        if err:
            raise AssertionError("Wa-Tor heap inconsistent: %d errors" % err)
        return k, a, e


class Life(World):
    """A single object-based Game of Life instance (thesis Sec. 7.8)."""

    def __init__(self, W, H, kind, state, seed: int = 0, **kw):
        super().__init__([LIFE], [W], [H], seed, kind, None, None, state, **kw)

    def read(self):
        k, _, _, s, err = self.export()
        if err:
            raise AssertionError("Life heap inconsistent: %d errors" % err)
        return k.astype(np.uint8), s


# Burst (0235678/3468) with a dead cell blocked for 255 generations: the
# generation application's rule as masks over the alive-neighbour count
BURST = (0b111101101, 0b101011000, 255)


class Generation(World):
    """A single instance of the generational automaton (thesis Sec. 7.8,
    "generation"): the object-based Life in which a dead Alive blocks its
    cell for `block` generations; rule = (survive mask, born mask, block)."""

    def __init__(self, W, H, kind, state, blocked=None, rule=BURST, seed: int = 0, **kw):
        b = None if blocked is None else np.asarray(blocked).astype(np.int16)
        super().__init__([LIFE], [W], [H], seed, kind, b, None, state, **kw)
        self.set_life_rule(*rule)

    def read(self):
        """(kind, is_new, blocked) per cell."""
        k, a, _, s, err = self.export()
        if err:
            raise AssertionError("generation heap inconsistent: %d errors" % err)
        return k.astype(np.uint8), s, a.astype(np.uint16)


class Traffic:
    """Nagel-Schreckenberg traffic on a street graph (thesis Sec. 7.5)."""

    def __init__(self, graph: dict, seed: int, car_v, heap_bytes: int | None = None,
                 config: smmo.HeapConfig | None = None, stream=None):
        self.stream = stream
        self.num_cells = int(graph["num_cells"])
        S = int(graph["num_streets"])
        nbytes = heap_bytes or int((self.num_cells / 64.0 * 3 + 4096) * 1000) + (32 << 20)
        self.heap = smmo.Heap(nbytes, config, stream=stream)
        self._w = ctypes.c_void_p()

        def arr(name, ct, n):
            a = np.ascontiguousarray(graph[name], dtype=np.int32 if ct is ctypes.c_int32 else np.uint8)
            return (ct * n)(*a.tolist())

        cv = torch.as_tensor(np.ascontiguousarray(car_v, dtype=np.int8)).cuda() \
            if not isinstance(car_v, torch.Tensor) else car_v.to("cuda", torch.int8).contiguous()
        smmo.check(smmo.lib().smmo_traffic_create(
            self.heap.handle, S, arr("street_start", ctypes.c_int32, S),
            arr("street_len", ctypes.c_int32, S), arr("out_deg", ctypes.c_int32, S),
            arr("out_street", ctypes.c_int32, 3 * S), arr("is_source", ctypes.c_uint8, S),
            int(graph.get("v_max", 5)), ctypes.c_uint32(int(graph["brake_threshold"])),
            int(graph.get("sources_enabled", 1)), int(graph.get("sinks_enabled", 1)),
            ctypes.c_uint64(seed), ctypes.c_void_p(cv.data_ptr()), smmo._stream(stream),
            ctypes.byref(self._w)), "traffic_create")
        ids = (ctypes.c_int * 4)()
        smmo.check(smmo.lib().smmo_traffic_info(self._w, None, ids, None), "traffic_info")
        self.class_ids = dict(zip(["Cell", "Car", "Source", "Controller"], list(ids)))
        self.num_streets = S

    def step(self, n: int = 1):
        smmo.check(smmo.lib().smmo_traffic_step(self._w, n, smmo._stream(self.stream)), "traffic_step")

    def set_controllers(self, ctrl_kind, phase_len: int = 8, lookahead: int = 5):
        """Traffic controllers (smmo_traffic_set_controllers); ctrl_kind per
        street: -1 none, 0 traffic light, 1 smart traffic light, 2 yield."""
        k = np.ascontiguousarray(ctrl_kind, dtype=np.int8)
        arr = (ctypes.c_int8 * len(k))(*k.tolist())
        smmo.check(smmo.lib().smmo_traffic_set_controllers(self._w, arr, int(phase_len), int(lookahead),
                                                           smmo._stream(self.stream)), "traffic_set_controllers")

    def controller_state(self):
        """(green index, timer) per street."""
        S = self.num_streets
        g, t = (ctypes.c_int16 * S)(), (ctypes.c_int16 * S)()
        smmo.check(smmo.lib().smmo_traffic_controller_state(self._w, g, t, smmo._stream(self.stream)),
                   "traffic_controller_state")
        return np.array(g, np.int16), np.array(t, np.int16)

    def read(self):
        v = torch.empty(self.num_cells, dtype=torch.int8, device="cuda")
        err = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_traffic_export(self._w, ctypes.c_void_p(v.data_ptr()),
                                                  ctypes.byref(err), smmo._stream(self.stream)),
                   "traffic_export")
        if err.value:
            raise AssertionError("traffic heap inconsistent: %d errors" % err.value)
        return v.cpu().numpy()

    def sync(self):
        return self.heap.sync()

    def close(self):
        if self._w:
            smmo.lib().smmo_traffic_destroy(self._w)
            self._w = ctypes.c_void_p()
        self.heap.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CompactSynthetic:
    """The thesis' synthetic defragmentation benchmark (Sec. 6.4): classes A
    and B of n objects each (32 bytes: a reference to the other class, an
    index and padding), A objects referring to random B objects and B
    objects to random A objects; 60 % of the A objects are deleted (B
    references to them are null), leaving every A block about 40 % full.
    ``verify()`` checks, after a compaction of A, that every object and
    every reference survived the relocation."""

    def __init__(self, n: int, seed: int = 1, block_data_bytes: int = 64 * 32, stream=None):
        from . import inputs
        dev = "cuda"
        dead, a_ref, b_ref = inputs.compact_synthetic(n, seed)
        self.n = n
        self.dead = torch.as_tensor(dead, device=dev)
        self.a_ref = torch.as_tensor(a_ref, device=dev)
        self.b_ref = torch.as_tensor(b_ref, device=dev)
        nbytes = int(2 * n * 32 * 1.12) + (64 << 20)
        h = self.heap = smmo.Heap(nbytes, smmo.default_config(block_data_bytes=block_data_bytes), stream=stream)
        # B first, so that A's reference column can name B as its target
        # class (compacting A then scans B's references only)
        self.B = h.register("B", [("ref", smmo.HANDLE), ("idx", smmo.I32), ("pad", smmo.I32, 6)])
        self.A = h.register("A", [("ref", smmo.HANDLE, 1, self.B), ("idx", smmo.I32), ("dead", smmo.I32),
                                  ("pad", smmo.I32, 5)])
        idx = torch.arange(n, dtype=torch.int32, device=dev)
        nul = torch.full((n,), -1, dtype=torch.int32, device=dev)
        pad = torch.zeros(n, dtype=torch.int32, device=dev)
        hb, _ = h.bulk_new(self.B, n, [nul, idx] + [pad] * 6, want_handles=True)
        self.hb = hb
        ha, _ = h.bulk_new(self.A, n, [hb[self.a_ref], idx, self.dead] + [pad] * 5, want_handles=True)
        table = torch.where(self.dead[self.b_ref] == 1, nul, ha[self.b_ref]).contiguous()
        h.parallel_do(self.B, "test.set_ref_from", smmo.SetRefFromArgs(0, 1, table.data_ptr()))
        h.parallel_do(self.A, "test.free_self_if", smmo.FreeSelfIfArgs(2, 2, 1))
        h.sync()
        del table, ha, nul, pad, idx
        self.survivors = int(n - int(self.dead.sum()))

    def verify(self) -> dict:
        """Relocation checks after compact(A): A keeps exactly the survivors
        with their fields; every B reference leads to the A object it led to
        before (same index), or stays null."""
        h = self.heap
        ha = h.enumerate_live(self.A)
        ai, aref, adead = h.gather(self.A, ha, ["idx", "ref", "dead"])
        ok_a = (ha.numel() == self.survivors and bool((adead == 0).all())
                and bool((aref == self.hb[self.a_ref[ai.long()]]).all())
                and int(torch.unique(ai).numel()) == self.survivors)
        hbl = h.enumerate_live(self.B)
        bi, bref = h.gather(self.B, hbl, ["idx", "ref"])
        want_null = self.dead[self.b_ref[bi.long()]] == 1
        null_ok = bool((bref[want_null] == -1).all())
        live_refs = bref[~want_null]
        (ti,) = h.gather(self.A, live_refs, ["idx"])
        ok_b = null_ok and bool((ti.long() == self.b_ref[bi.long()][~want_null]).all())
        return {"a_objects_ok": ok_a, "b_references_ok": ok_b, "heap_violations": h.check()}

    def close(self):
        self.heap.close()


class BHParams(ctypes.Structure):
    _fields_ = [("G", ctypes.c_float), ("eps", ctypes.c_float), ("dt", ctypes.c_float),
                ("theta", ctypes.c_float)]


class BarnesHut:
    """2-D Barnes-Hut with a dynamic quad tree (thesis Sec. 7.3) on one heap.
    state: float32 arrays x, y (in [0,1), pairwise distinct), vx, vy, m."""

    def __init__(self, state: dict, G: float = 1e-5, eps: float = 1e-2, dt: float = 1e-3,
                 theta: float = 0.5, heap_bytes: int | None = None, config: smmo.HeapConfig | None = None,
                 stream=None):
        self.stream = stream
        n = len(state["x"])
        self.n = n
        cols = [torch.as_tensor(np.ascontiguousarray(state[k], dtype=np.float32)).cuda()
                for k in ("x", "y", "vx", "vy", "m")]
        self.heap = smmo.Heap(heap_bytes or int(n * 3.2 * 3200 / 64 * 1.25) + (64 << 20), config, stream=stream)
        arr = (ctypes.c_void_p * 5)(*[c.data_ptr() for c in cols])
        self._w = ctypes.c_void_p()
        smmo.check(smmo.lib().smmo_bh_create(self.heap.handle, ctypes.c_int64(n), arr,
                                             ctypes.byref(BHParams(G, eps, dt, theta)), smmo._stream(stream),
                                             ctypes.byref(self._w)), "bh_create")
        ids = (ctypes.c_int * 3)()
        smmo.check(smmo.lib().smmo_bh_info(self._w, ids, None), "bh_info")
        self.class_ids = dict(zip(["NodeBase", "BodyNode", "TreeNode"], list(ids)))

    def step(self, n: int = 1):
        smmo.check(smmo.lib().smmo_bh_step(self._w, n, smmo._stream(self.stream)), "bh_step")

    def read(self):
        """(state dict by id, live TreeNodes)."""
        out = torch.empty(5 * self.n, dtype=torch.float32, device="cuda")
        tn = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_bh_export(self._w, ctypes.c_void_p(out.data_ptr()), ctypes.byref(tn),
                                             smmo._stream(self.stream)), "bh_export")
        o = out.cpu().numpy().reshape(5, self.n)
        return dict(zip(("x", "y", "vx", "vy", "m"), o)), tn.value

    def levels(self) -> int:
        """Bottom-up tree traversals run so far (two per step)."""
        lv = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_bh_info(self._w, None, ctypes.byref(lv)), "bh_info")
        return lv.value

    def sync(self):
        return self.heap.sync()

    def close(self):
        if self._w:
            smmo.lib().smmo_bh_destroy(self._w)
            self._w = ctypes.c_void_p()
        self.heap.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Bfs:
    """Frontier-based BFS over Vertex objects (thesis Sec. 4.3), terminated
    with parallel_do_and_reduce.  row_ptr/col: CSR graph (host arrays)."""

    def __init__(self, row_ptr, col, heap_bytes: int | None = None, config: smmo.HeapConfig | None = None,
                 stream=None):
        self.stream = stream
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        self.n = len(rp) - 1
        self.heap = smmo.Heap(heap_bytes or int(self.n * 44 * 1.3) + (64 << 20), config, stream=stream)
        self._w = ctypes.c_void_p()
        smmo.check(smmo.lib().smmo_bfs_create(self.heap.handle, ctypes.c_int64(self.n),
                                              rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                                              smmo._stream(stream), ctypes.byref(self._w)), "bfs_create")

    def run(self, source: int, check_every: int = 16) -> int:
        lv = ctypes.c_int32()
        smmo.check(smmo.lib().smmo_bfs_run(self._w, int(source), int(check_every), ctypes.byref(lv),
                                           smmo._stream(self.stream)), "bfs_run")
        return lv.value

    def distances(self):
        d = torch.empty(self.n, dtype=torch.int32, device="cuda")
        smmo.check(smmo.lib().smmo_bfs_export(self._w, ctypes.c_void_p(d.data_ptr()), smmo._stream(self.stream)),
                   "bfs_export")
        return d.cpu().numpy()

    def sync(self):
        return self.heap.sync()

    def close(self):
        if self._w:
            smmo.lib().smmo_bfs_destroy(self._w)
            self._w = ctypes.c_void_p()
        self.heap.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StructureParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("damping", ctypes.c_float), ("substeps", ctypes.c_int32),
                ("bfs_check_every", ctypes.c_int32)]


class _StructureOut(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("node_alive", "x", "y", "vx", "vy", "num_springs", "distance",
                                               "slot", "spring_alive", "fx", "fy")]


STRUCT_PHASE_PULL, STRUCT_PHASE_COMPUTE, STRUCT_PHASE_REMOVE = 1, 2, 4


class Structure:
    """The spring mesh that cracks under load (thesis Sec. 7.4) on one heap.
    mesh: the dict of ``inputs.structure_mesh`` (host arrays kind, x, y, vx,
    vy, m, slot[N, 3], p1, p2, k, L0, fmax)."""

    NAMES = ["NodeBase", "AnchorNode", "AnchorPullNode", "Node", "Spring"]

    def __init__(self, mesh: dict, dt: float = 0.05, damping: float = 0.01, substeps: int = 40,
                 bfs_check_every: int = 1024, heap_bytes: int | None = None,
                 config: smmo.HeapConfig | None = None, stream=None):
        self.stream = stream
        self.n, self.ns = len(mesh["kind"]), len(mesh["p1"])
        host = lambda k, t: np.ascontiguousarray(mesh[k], dtype=t)
        self._keep = [host("kind", np.int8), host("slot", np.int32).reshape(-1), host("p1", np.int32),
                      host("p2", np.int32)]
        ncols = [host(k, np.float32) for k in ("x", "y", "vx", "vy", "m")]
        scols = [host(k, np.float32) for k in ("k", "L0", "fmax")]
        nptr = (ctypes.c_void_p * 5)(*[c.ctypes.data for c in ncols])
        sptr = (ctypes.c_void_p * 3)(*[c.ctypes.data for c in scols])
        # 64-slot blocks of 2,816 data bytes, for nodes and springs
        self.heap = smmo.Heap(heap_bytes or int((self.n + self.ns) * 48 * 1.25) + (64 << 20), config,
                              stream=stream)
        self._w = ctypes.c_void_p()
        p = StructureParams(dt, damping, substeps, bfs_check_every)
        kind, slot, p1, p2 = self._keep
        smmo.check(smmo.lib().smmo_structure_create(
            self.heap.handle, ctypes.c_int64(self.n), ctypes.c_void_p(kind.ctypes.data), nptr,
            ctypes.c_void_p(slot.ctypes.data), ctypes.c_int64(self.ns), ctypes.c_void_p(p1.ctypes.data),
            ctypes.c_void_p(p2.ctypes.data), sptr, ctypes.byref(p), smmo._stream(stream),
            ctypes.byref(self._w)), "structure_create")
        ids = (ctypes.c_int * 5)()
        smmo.check(smmo.lib().smmo_structure_info(self._w, ids, None, None), "structure_info")
        self.class_ids = dict(zip(self.NAMES, list(ids)))

    def step(self, iterations: int = 1, phases: int = 7):
        smmo.check(smmo.lib().smmo_structure_step(self._w, int(iterations), int(phases),
                                                  smmo._stream(self.stream)), "structure_step")

    def read(self) -> dict:
        """Node and spring arrays by id (host): nalive, x, y, vx, vy, nspr,
        dist, slot[N, 3]; salive, fx, fy.  Deleted objects read 0."""
        dev = dict(nalive=torch.zeros(self.n, dtype=torch.uint8, device="cuda"),
                   **{k: torch.zeros(self.n, dtype=torch.float32, device="cuda") for k in ("x", "y", "vx", "vy")},
                   nspr=torch.zeros(self.n, dtype=torch.int32, device="cuda"),
                   dist=torch.zeros(self.n, dtype=torch.int32, device="cuda"),
                   slot=torch.full((self.n, 3), -1, dtype=torch.int32, device="cuda"),
                   salive=torch.zeros(max(self.ns, 1), dtype=torch.uint8, device="cuda"),
                   fx=torch.zeros(max(self.ns, 1), dtype=torch.float32, device="cuda"),
                   fy=torch.zeros(max(self.ns, 1), dtype=torch.float32, device="cuda"))
        ptr = lambda k: dev[k].data_ptr()
        o = _StructureOut(ptr("nalive"), ptr("x"), ptr("y"), ptr("vx"), ptr("vy"), ptr("nspr"), ptr("dist"),
                          ptr("slot"), ptr("salive"), ptr("fx"), ptr("fy"))
        smmo.check(smmo.lib().smmo_structure_export(self._w, ctypes.byref(o), smmo._stream(self.stream)),
                   "structure_export")
        out = {k: v.cpu().numpy() for k, v in dev.items()}
        for k in ("salive", "fx", "fy"):
            out[k] = out[k][:self.ns]
        return out

    def counters(self) -> dict:
        """springs broken, nodes deleted, springs removed by the removal
        phase, BFS levels run, BFS launches (cumulative)."""
        c = (ctypes.c_int64 * 5)()
        smmo.check(smmo.lib().smmo_structure_info(self._w, None, c, smmo._stream(self.stream)), "structure_info")
        return dict(zip(("broken", "nodes_deleted", "springs_removed", "bfs_levels", "bfs_launches"), list(c)))

    def sync(self):
        return self.heap.sync()

    def close(self):
        if self._w:
            smmo.lib().smmo_structure_destroy(self._w)
            self._w = ctypes.c_void_p()
        self.heap.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
