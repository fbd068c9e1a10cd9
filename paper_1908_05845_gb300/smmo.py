"""ctypes binding of libsmmo.so (include/smmo.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  PyTorch supplies device memory (the heap buffer and the caller's
arrays) and streams.  If the library has not been built the import of
this module succeeds but every call raises ``SmmoError`` -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsmmo.so")
_lock = threading.Lock()
_lib = None

NULL = 0xFFFFFFFF
I8, U8, I16, U16, I32, U32, F32, I64, U64, F64, HANDLE, INSTANCE = range(1, 13)
_TORCH = {I8: torch.int8, U8: torch.uint8, I16: torch.int16, U16: torch.int16, I32: torch.int32,
          U32: torch.int32, F32: torch.float32, I64: torch.int64, U64: torch.int64,
          F64: torch.float64, HANDLE: torch.int32, INSTANCE: torch.int32}
MAX_CLASSES = 16

STATUS = {0: "ok", -1: "invalid argument", -2: "heap has too few free blocks",
          -3: "device new found no free block", -4: "device retry budget exhausted",
          -5: "CUDA error", -6: "timeout", -7: "bad handle", -8: "bounds check failed",
          -9: "unsupported", -10: "heap geometry already fixed"}


class SmmoError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = "%s: %s (%d)" % (what, STATUS.get(status, "?"), status)
        if status == -5 and _lib is not None:
            msg += " cuda error %d" % _lib.smmo_last_cuda_error()
        super().__init__(msg)


def lib():
    """Loads libsmmo.so; raises if it is missing (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise SmmoError(-9, "libsmmo.so not built (run __graft_entry__.build())")
            _lib = ctypes.CDLL(LIB_PATH)
            _lib.smmo_status_string.restype = ctypes.c_char_p
    return _lib


def check(st: int, what: str):
    if st != 0:
        raise SmmoError(st, what)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class FieldDesc(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("elem_type", ctypes.c_int), ("count", ctypes.c_int),
                ("ref_class", ctypes.c_int)]


class HeapConfig(ctypes.Structure):
    _fields_ = [("block_data_bytes", ctypes.c_uint32), ("lookup_retries", ctypes.c_int32),
                ("alloc_retries", ctypes.c_int32), ("bitmap_spins", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("debug_checks", ctypes.c_int32), ("defrag_factor", ctypes.c_int32),
                ("bitmap_fanout", ctypes.c_int32)]


class InstanceDesc(ctypes.Structure):
    """One row of a heap's instance table (smmo_instance_desc)."""
    _fields_ = [("kind", ctypes.c_int32), ("id", ctypes.c_uint32), ("W", ctypes.c_uint32),
                ("H", ctypes.c_uint32), ("base", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("param", ctypes.c_int64 * 2)]


class HeapStats(ctypes.Structure):
    _fields_ = [("live_objects", ctypes.c_int64 * MAX_CLASSES),
                ("blocks", ctypes.c_int64 * MAX_CLASSES), ("free_blocks", ctypes.c_int64),
                ("num_blocks", ctypes.c_int64), ("fragmentation", ctypes.c_double * MAX_CLASSES),
                ("fragmentation_all", ctypes.c_double),
                ("allocs", ctypes.c_int64 * MAX_CLASSES), ("frees", ctypes.c_int64 * MAX_CLASSES),
                ("slow_paths", ctypes.c_int64), ("enumerated_objects", ctypes.c_int64),
                ("enumerated_blocks", ctypes.c_int64), ("capacity", ctypes.c_int32 * MAX_CLASSES),
                ("object_bytes", ctypes.c_int32 * MAX_CLASSES), ("block_bytes", ctypes.c_int32),
                ("num_classes", ctypes.c_int32)]


class CompactStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("blocks_freed", ctypes.c_int64),
                ("objects_moved", ctypes.c_int64), ("pointers_rewritten", ctypes.c_int64),
                ("candidates_left", ctypes.c_int64), ("scan_ms", ctypes.c_double),
                ("copy_ms", ctypes.c_double), ("state_ms", ctypes.c_double), ("rewrite_ms", ctypes.c_double)]


def default_config(**kw) -> HeapConfig:
    c = HeapConfig()
    lib().smmo_heap_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


_method_ids = {}


def method_id(name: str, heap=None) -> int:
    """Id of a compiled-in method; with a heap, the library also checks
    that the heap can run it (a batch method needs an instance table)."""
    if heap is not None:
        mid = ctypes.c_int()
        check(lib().smmo_method_lookup(heap.handle, name.encode(), ctypes.byref(mid)), "method_lookup " + name)
        return mid.value
    if name not in _method_ids:
        mid = ctypes.c_int()
        check(lib().smmo_method_lookup(None, name.encode(), ctypes.byref(mid)), "method_lookup " + name)
        _method_ids[name] = mid.value
    return _method_ids[name]


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class Heap:
    """A heap inside a torch-owned uint8 CUDA buffer (the buffer is the
    caller-owned memory of smmo_heap_create)."""

    def __init__(self, nbytes: int, config: HeapConfig | None = None, device="cuda", stream=None):
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        self.stream = stream
        self._h = ctypes.c_void_p()
        cfg = ctypes.byref(config) if config is not None else None
        check(lib().smmo_heap_create(cfg, _ptr(self.buf), ctypes.c_size_t(self.buf.numel()),
                                     _stream(stream), ctypes.byref(self._h)), "heap_create")
        self.classes = {}
        self.fields = {}

    def close(self):
        if self._h:
            lib().smmo_heap_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---------------------------------------------------------- classes
    def register(self, name: str, fields, parent: int = -1, abstract: bool = False) -> int:
        """fields: list of (name, elem_type[, count[, ref_class]])."""
        arr = (FieldDesc * max(1, len(fields)))()
        keep = []
        for i, f in enumerate(fields):
            nm = f[0].encode()
            keep.append(nm)
            arr[i] = FieldDesc(nm, f[1], f[2] if len(f) > 2 else 1, f[3] if len(f) > 3 else -1)
        cid = ctypes.c_int()
        check(lib().smmo_class_register(self._h, name.encode(), arr, len(fields), parent,
                                        1 if abstract else 0, ctypes.byref(cid)), "class_register")
        self.classes[name] = cid.value
        base = list(self.fields[parent]) if parent >= 0 else []
        self.fields[cid.value] = base + [(f[0], f[1], f[2] if len(f) > 2 else 1) for f in fields]
        return cid.value

    def columns(self, cls: int):
        """[(column name, elem_type)] with inner arrays expanded."""
        out = []
        for nm, t, cnt in self.fields[cls]:
            if cnt == 1:
                out.append((nm, t))
            else:
                out += [("%s[%d]" % (nm, k), t) for k in range(cnt)]
        return out

    def column_index(self, cls: int, name: str) -> int:
        return [c[0] for c in self.columns(cls)].index(name)

    def class_id(self, name: str) -> int:
        c = ctypes.c_int()
        check(lib().smmo_class_lookup(self._h, name.encode(), ctypes.byref(c)), "class_lookup")
        return c.value

    def freeze(self):
        check(lib().smmo_heap_freeze(self._h), "heap_freeze")

    def class_info(self, cls: int):
        nf, cap, ob = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().smmo_class_info(self._h, cls, ctypes.byref(nf), ctypes.byref(cap),
                                    ctypes.byref(ob)), "class_info")
        return dict(nfields=nf.value, capacity=cap.value, object_bytes=ob.value)

    def layout(self, cls: int):
        off = (ctypes.c_uint32 * 32)()
        n, bb, base = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_void_p()
        check(lib().smmo_class_layout(self._h, cls, off, ctypes.byref(n), ctypes.byref(bb),
                                      ctypes.byref(base)), "class_layout")
        return dict(col_off=list(off[:n.value]), block_bytes=bb.value, data_base=base.value)

    # ---------------------------------------------------------- objects
    def bulk_new(self, cls: int, n: int, columns=None, want_handles: bool = False, asynchronous: bool = False):
        """columns: list (one per SOA column) of device tensors or None.
        Returns (handles or None, first block or -1).  asynchronous=True
        only enqueues the kernels (the first block is then not read back,
        -1; a shortage of free blocks shows up in sync()); the column
        tensors are kept alive for the heap's stream with record_stream."""
        cols = self.columns(cls)
        src = (ctypes.c_void_p * max(1, len(cols)))()
        keep = []
        if columns is not None:
            assert len(columns) == len(cols)
            for k, t in enumerate(columns):
                if t is not None:
                    t = t.contiguous()
                    assert t.is_cuda and t.numel() == n
                    keep.append(t)
                    src[k] = t.data_ptr()
        out = torch.empty(max(1, n), dtype=torch.int32, device=self.buf.device) if want_handles else None
        first = ctypes.c_int64(-1)
        check(lib().smmo_bulk_new(self._h, cls, ctypes.c_int64(n), src,
                                  _ptr(out) if out is not None else None,
                                  None if asynchronous else ctypes.byref(first),
                                  _stream(self.stream)), "bulk_new")
        if asynchronous:
            st = self.stream if self.stream is not None else torch.cuda.current_stream()
            for t in keep:
                t.record_stream(st)
        return (out[:n] if out is not None else None), first.value

    def batch_define(self, rows) -> None:
        """Instance table (smmo_batch_define): rows of dicts with keys kind,
        id, W, H, base, count, param (all optional, default 0)."""
        arr = (InstanceDesc * len(rows))()
        for i, r in enumerate(rows):
            p = list(r.get("param", (0, 0))) + [0, 0]
            arr[i] = InstanceDesc(int(r.get("kind", 0)), int(r.get("id", i)), int(r.get("W", 0)),
                                  int(r.get("H", 0)), int(r.get("base", 0)), int(r.get("count", 0)),
                                  (ctypes.c_int64 * 2)(int(p[0]), int(p[1])))
        check(lib().smmo_batch_define(self._h, arr, len(rows)), "batch_define")

    def _mid(self, method) -> int:
        if not isinstance(method, str):
            return int(method)
        mids = self.__dict__.setdefault("_mids", {})
        if method not in mids:
            mids[method] = method_id(method, self)
        return mids[method]

    def parallel_do(self, cls: int, method, args=None):
        mid = self._mid(method)
        if args is None:
            ap, n = None, 0
        else:
            ap, n = ctypes.byref(args), ctypes.sizeof(args)
        check(lib().smmo_parallel_do(self._h, cls, mid, ap, ctypes.c_size_t(n),
                                     _stream(self.stream)), "parallel_do")

    def parallel_do_and_reduce(self, cls: int, method, args=None, op: int = 0, out: torch.Tensor | None = None):
        """Runs a reducing method and returns the combined int64 (reads it
        back) or, with `out` (a one-element int64 CUDA tensor), leaves it
        there without synchronising."""
        mid = method_id(method) if isinstance(method, str) else int(method)
        ap, n = (None, 0) if args is None else (ctypes.byref(args), ctypes.sizeof(args))
        dst = out if out is not None else torch.empty(1, dtype=torch.int64, device=self.buf.device)
        check(lib().smmo_parallel_do_and_reduce(self._h, cls, mid, ap, ctypes.c_size_t(n), int(op), _ptr(dst),
                                                _stream(self.stream)), "parallel_do_and_reduce")
        return None if out is not None else int(dst.item())

    def enumerate_live(self, cls: int, include_subclasses: bool = True, cap: int | None = None):
        if cap is None:
            st = self.stats()
            cap = max(1, int(sum(st["live_objects"])))
        out = torch.empty(max(1, cap), dtype=torch.int32, device=self.buf.device)
        cnt = ctypes.c_int64()
        check(lib().smmo_enumerate_live(self._h, cls, 1 if include_subclasses else 0, _ptr(out),
                                        ctypes.c_int64(cap), ctypes.byref(cnt),
                                        _stream(self.stream)), "enumerate_live")
        if cnt.value > cap:
            return self.enumerate_live(cls, include_subclasses, cnt.value)
        return out[:cnt.value]

    def gather(self, cls: int, handles: torch.Tensor, names):
        cols = self.columns(cls)
        idx = [self.column_index(cls, n) for n in names]
        outs = [torch.empty(handles.numel(), dtype=_TORCH[cols[i][1]], device=self.buf.device)
                for i in idx]
        if handles.numel():
            ci = (ctypes.c_int * len(idx))(*idx)
            dp = (ctypes.c_void_p * len(idx))(*[o.data_ptr() for o in outs])
            check(lib().smmo_gather_fields(self._h, cls, _ptr(handles.contiguous()),
                                           ctypes.c_int64(handles.numel()), ci, len(idx), dp,
                                           _stream(self.stream)), "gather_fields")
        return outs

    def compact(self, cls: int, n: int = 1, k1: int = 0):
        cs = CompactStats()
        check(lib().smmo_compact(self._h, cls, n, ctypes.c_int64(k1), ctypes.byref(cs),
                                 _stream(self.stream)), "compact")
        return {k: getattr(cs, k) for k, _ in CompactStats._fields_}

    def remap_handles(self, handles):
        """Caller-held handles (int32/uint32 CUDA tensor, rewritten in place)
        to where the last compact moved their objects."""
        check(lib().smmo_remap_handles(self._h, ctypes.c_void_p(handles.data_ptr()), ctypes.c_int64(handles.numel()),
                                       _stream(self.stream)), "remap_handles")
        return handles

    def last_device_error(self):
        """(status, detail) of the first device error since the last sync,
        without clearing it."""
        code, detail = ctypes.c_int(), ctypes.c_uint64()
        check(lib().smmo_heap_last_device_error(self._h, ctypes.byref(code), ctypes.byref(detail),
                                                _stream(self.stream)), "last_device_error")
        return code.value, detail.value

    def defrag_candidates(self, cls: int, n: int = 1) -> int:
        """Blocks of class cls at most n/(n+1) full."""
        v = ctypes.c_int64()
        check(lib().smmo_defrag_candidates(self._h, cls, n, ctypes.byref(v), _stream(self.stream)),
              "defrag_candidates")
        return v.value

    def compact_if(self, cls: int, n: int = 1, k1: int = 0, k2_blocks: int = 0, k2_fraction: float = 0.0):
        """The 'after massive deallocations' policy: (ran, stats)."""
        cs = CompactStats()
        ran = ctypes.c_int()
        check(lib().smmo_compact_if(self._h, cls, n, ctypes.c_int64(k1), ctypes.c_int64(k2_blocks),
                                    ctypes.c_double(k2_fraction), ctypes.byref(cs), ctypes.byref(ran),
                                    _stream(self.stream)), "compact_if")
        return bool(ran.value), {k: getattr(cs, k) for k, _ in CompactStats._fields_}

    # ---------------------------------------------------------- status
    def stats(self):
        s = HeapStats()
        check(lib().smmo_heap_get_stats(self._h, ctypes.byref(s), _stream(self.stream)), "heap_stats")
        nc = s.num_classes
        out = {}
        for k, _ in HeapStats._fields_:
            v = getattr(s, k)
            out[k] = list(v)[:nc] if hasattr(v, "__len__") else v
        return out

    def counters(self):
        """(objects visited by do-all kernels, device news, device deletes),
        cumulative."""
        e, a, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().smmo_heap_counters(self._h, ctypes.byref(e), ctypes.byref(a), ctypes.byref(f),
                                       _stream(self.stream)), "heap_counters")
        return e.value, a.value, f.value

    def alloc_counters(self):
        v = (ctypes.c_int64 * 6)()
        check(lib().smmo_heap_alloc_counters(self._h, v, _stream(self.stream)), "alloc_counters")
        return dict(zip(["slow_paths", "retries", "refills", "lookup_misses", "reserve_fails",
                         "enumerated_blocks"], list(v)))

    def check(self) -> int:
        v = ctypes.c_int64()
        check(lib().smmo_heap_check(self._h, ctypes.byref(v), _stream(self.stream)), "heap_check")
        return v.value

    def sync(self, raise_on_error: bool = True):
        detail = ctypes.c_uint64()
        st = lib().smmo_heap_sync(self._h, _stream(self.stream), ctypes.byref(detail))
        if st and raise_on_error:
            raise SmmoError(st, "device error (detail 0x%x)" % detail.value)
        return st, detail.value


# ------------------------------------------------------ method argument blocks
class BatchAffineArgs(ctypes.Structure):
    _fields_ = [("col", ctypes.c_uint32), ("col_id", ctypes.c_uint32)]


class AddI32Args(ctypes.Structure):
    _fields_ = [("col", ctypes.c_uint32), ("value", ctypes.c_int32)]


class AllocKArgs(ctypes.Structure):
    _fields_ = [("target", ctypes.c_uint32), ("k", ctypes.c_uint32), ("col", ctypes.c_uint32),
                ("col2", ctypes.c_uint32), ("src_col", ctypes.c_uint32), ("marker", ctypes.c_int32)]


class FreeSelfIfArgs(ctypes.Structure):
    _fields_ = [("col", ctypes.c_uint32), ("mod", ctypes.c_int32), ("rem", ctypes.c_int32)]


class FreeRefArgs(ctypes.Structure):
    _fields_ = [("col", ctypes.c_uint32)]


class ReplaceArgs(ctypes.Structure):
    _fields_ = [("target", ctypes.c_uint32), ("col", ctypes.c_uint32), ("tcol", ctypes.c_uint32)]


REDUCE_SUM, REDUCE_MIN, REDUCE_MAX, REDUCE_OR, REDUCE_AND = range(5)


class ValueI32Args(ctypes.Structure):
    _fields_ = [("col", ctypes.c_uint32), ("count", ctypes.c_uint32)]


class SetRefFromArgs(ctypes.Structure):
    _fields_ = [("col_ref", ctypes.c_uint32), ("col_idx", ctypes.c_uint32), ("table", ctypes.c_void_p)]
