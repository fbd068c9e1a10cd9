"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: symbols only, no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:int|void|const char\*)\s+(smmo_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libsmmo():
    from paper_1908_05845_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_calls():
    names = declared()
    for n in ("smmo_heap_create", "smmo_class_register", "smmo_bulk_new", "smmo_parallel_do",
              "smmo_enumerate_live", "smmo_compact", "smmo_method_lookup", "smmo_batch_define",
              "smmo_batch_count", "smmo_world_create_batch"):
        assert n in names


def test_every_declared_symbol_exported(libsmmo):
    missing = [n for n in declared() if not hasattr(libsmmo, n)]
    assert not missing, missing


def test_status_strings(libsmmo):
    libsmmo.smmo_status_string.restype = ctypes.c_char_p
    assert libsmmo.smmo_status_string(0) == b"ok"
    assert b"double free" in libsmmo.smmo_status_string(-7)


def test_method_table(libsmmo):
    mid = ctypes.c_int()
    assert libsmmo.smmo_method_lookup(None, b"test.add_i32", ctypes.byref(mid)) == 0
    assert libsmmo.smmo_method_lookup(None, b"no.such.method", ctypes.byref(mid)) == -1
    assert libsmmo.smmo_method_lookup(None, b"test.batch_affine", ctypes.byref(mid)) == 0


def test_create_rejects_bad_args(libsmmo):
    h = ctypes.c_void_p()
    assert libsmmo.smmo_heap_create(None, None, ctypes.c_size_t(1 << 20), None, ctypes.byref(h)) == -1
    # misaligned buffer pointer is rejected before any CUDA call
    assert libsmmo.smmo_heap_create(None, ctypes.c_void_p(0x1001), ctypes.c_size_t(1 << 20), None,
                                    ctypes.byref(h)) == -1


def test_every_workload_method_is_registered(libsmmo):
    """Each workload's compiled-in methods are found by name (the method
    table is host data: no GPU needed)."""
    mid = ctypes.c_int()
    for name in (b"wator.fish_update", b"gol.candidate_prepare", b"bh.body_insert",
                 b"bfs.vertex_visit", b"structure.spring_compute_force", b"structure.node_visit",
                 b"structure.spring_delete", b"test.value_i32"):
        assert libsmmo.smmo_method_lookup(None, name, ctypes.byref(mid)) == 0, name


def test_entry_points_reject_null_objects(libsmmo):
    """Argument checks that run on the host before any CUDA call."""
    c = ctypes.c_int64()
    d = ctypes.c_double()
    ran = ctypes.c_int()
    assert libsmmo.smmo_compact(None, 0, 1, ctypes.c_int64(0), None, None) == -1
    assert libsmmo.smmo_compact_if(None, 0, 1, ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0), None,
                                   ctypes.byref(ran), None) == -1
    assert ran.value == 0
    assert libsmmo.smmo_defrag_candidates(None, 0, 1, ctypes.byref(c), None) == -1
    assert libsmmo.smmo_remap_handles(None, None, ctypes.c_int64(0), None) == -1
    assert libsmmo.smmo_heap_last_device_error(None, None, None, None) == -1
    assert libsmmo.smmo_parallel_do_and_reduce(None, 0, 0, None, ctypes.c_size_t(0), 0, None, None) == -1
    assert libsmmo.smmo_bfs_run(None, 0, 16, None, None) == -1
    assert libsmmo.smmo_structure_step(None, 1, 7, None) == -1
    assert libsmmo.smmo_structure_create(None, ctypes.c_int64(1), None, None, None, ctypes.c_int64(0), None, None,
                                         None, None, None, None) == -1
    assert libsmmo.smmo_bh_step(None, 1, None) == -1
    assert libsmmo.smmo_measure_fp32_peak(0, ctypes.byref(d), None) == -1
    assert libsmmo.smmo_measure_mufu_peak(1, None, None) == -1
    assert libsmmo.smmo_selftest_barrier_timeout(None, 16, None) == -1


def test_missing_library_fails_loudly(monkeypatch):
    """Without libsmmo.so the binding raises; there is no CPU fallback."""
    from paper_1908_05845_gb300 import smmo
    monkeypatch.setattr(smmo, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libsmmo.so"))
    monkeypatch.setattr(smmo, "_lib", None)
    with pytest.raises(smmo.SmmoError):
        smmo.lib()


def test_the_package_never_uses_the_oracle():
    """Nothing in the product package imports, loads or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_1908_05845_gb300")
    bad = []
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                if re.search(r"^\s*(import oracle|from oracle)|liboracle|oracle\.h|orc_", src, flags=re.M):
                    bad.append(f)
    assert not bad, bad


def test_the_oracle_shares_no_code_with_the_package():
    """The oracle includes only its own header and the C library, and its
    wrapper imports nothing from the product package."""
    od = os.path.join(ROOT, "oracle")
    for f in os.listdir(od):
        p = os.path.join(od, f)
        if f.endswith((".c", ".h")):
            incs = re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(p).read(), flags=re.M)
            assert all(i == "oracle.h" or "/" not in i and i.endswith(".h") and not i.startswith("smmo") for i in incs), (f, incs)
            assert "oracle.h" in incs or f == "oracle.h", f
        elif f.endswith(".py"):
            assert not re.search(r"^\s*(import|from)\s+paper_1908_05845_gb300|libsmmo", open(p).read(),
                                 flags=re.M), f


def test_header_method_lookup_takes_a_heap():
    """The method table lookup names the heap it will run on (the scope
    table's signature), and bulk_new's contract is asynchronous."""
    src = open(os.path.join(ROOT, "include", "smmo.h")).read()
    assert re.search(r"int smmo_method_lookup\(smmo_heap\* heap, const char\* name, int\* method_id\);", src)
    i = src.index("int smmo_bulk_new(")
    assert "Asynchronous on `stream`" in src[src.rindex("/*", 0, i):i]


def test_batch_define_checks_its_arguments(libsmmo):
    """Host-side checks of smmo_batch_define (before any CUDA call)."""
    class Desc(ctypes.Structure):
        _fields_ = [("kind", ctypes.c_int32), ("id", ctypes.c_uint32), ("W", ctypes.c_uint32),
                    ("H", ctypes.c_uint32), ("base", ctypes.c_uint64), ("count", ctypes.c_uint64),
                    ("param", ctypes.c_int64 * 2)]
    rows = (Desc * 2)()
    assert libsmmo.smmo_batch_define(None, rows, 2) == -1
    n = ctypes.c_int()
    assert libsmmo.smmo_batch_count(None, ctypes.byref(n)) == -1


def test_step_kernel_modes_agree_with_the_header(libsmmo):
    """The Wa-Tor step-kernel mode values of include/smmo.h, the Python
    binding and bench.py's names are the same numbers, and the host rejects
    a null world before any CUDA call."""
    src = open(os.path.join(ROOT, "include", "smmo.h")).read()
    hdr = {k: int(v) for k, v in re.findall(r"(SMMO_WATOR_\w+)\s*=\s*(\d+)", src)}
    from paper_1908_05845_gb300 import workloads as wl
    assert hdr == {"SMMO_WATOR_FOUR_DO_ALLS": wl.FOUR_DO_ALLS, "SMMO_WATOR_PHASED1": wl.PHASED1,
                   "SMMO_WATOR_PHASED2": wl.PHASED2, "SMMO_WATOR_QUEUED_CREATION": wl.QUEUED,
                   "SMMO_WATOR_MARKED_UPDATE": wl.MARKED}
    import bench
    assert bench.STEP_KERNELS["four_do_alls"] == wl.FOUR_DO_ALLS
    assert bench.STEP_KERNELS["phased2_queued"] == wl.PHASED2 | wl.QUEUED
    assert bench.STEP_KERNELS["four_do_alls_marked_queued"] == wl.FOUR_DO_ALLS | wl.MARKED | wl.QUEUED
    # every mode the bench compares is one the library accepts (checked on a GPU);
    # here: no fused mode is combined with the marked update
    for mode in bench.STEP_KERNELS.values():
        assert not (mode & wl.MARKED and mode & 3)
    assert libsmmo.smmo_world_set_step_kernels(None, 0) == -1


def test_fused_phase_bytes_are_the_sum_of_the_pair():
    """A fused species launch is charged the bytes of its prepare and its
    update, and the whole-step byte count is the same in either form."""
    import bench
    b = bench.BYTES_PER_OBJECT
    assert b["fish_step"] == b["fish_prepare"] + b["fish_update"]
    assert b["shark_step"] == b["shark_prepare"] + b["shark_update"]
    objs = [0, 0, 0, 0, 7.0, 7.0, 3.0, 3.0]
    four = sum(b.get(bench.PHASES[p], 0) * objs[p] for p in range(8))
    fused = sum(b.get(bench.PHASES_FUSED[p], 0) * objs[p] for p in range(8) if bench.PHASES_FUSED[p])
    assert four == fused
