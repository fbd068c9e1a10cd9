"""CPU oracle for the SMMO hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, array-of-structs restatement (in C, see the
``*.c`` files beside this one) of the thesis' SMMO workloads: object-based
Game of Life and the generational automaton (Sec. 7.8), Wa-Tor (Sec. 7.6),
Nagel-Schreckenberg traffic with and without traffic controllers
(Sec. 7.5), n-body with collision merge (Sec. 7.1/7.2) and the n-body
adjoint, Barnes-Hut (Sec. 7.3), the spring mesh "structure" (Sec. 7.4) and
frontier BFS (Sec. 4.3).  It has its own Philox4x32-10 (Salmon et al.,
SC'11).  Everything runs on one thread except the n-body receiver loops,
which OpenMP may spread over cores (each receiver keeps its partner order,
so results do not depend on the thread count; ``set_threads``).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It never imports the CUDA library and the CUDA
library never imports it; both consume the same seeded inputs from
``paper_1908_05845_gb300.inputs``.

Pins (tests/test_oracle_*.py): Philox against Triton's implementation of
the same generator (every output word) and the input generator's separately
written numpy one (a million draws); Life blinker / glider / block, all 512
3x3 neighbourhoods and dense B3/S23 on random tori, the candidate set and
every counter from the dense boards; Wa-Tor bookkeeping, lone fish / lone
shark / breeding shark histories, the fish phase before the shark phase, a
full grid without sharks, the lowest-index grant; NaSch free-flow closed
form, car conservation on a ring, evenly spaced flow, braking statistics,
the entry claim and its loser, the sink rule; n-body momentum conservation
(also through merges), two-body circular orbit and acceleration closed
forms, energy drift O(dt^2), merge rules in every component; adjoint
against central finite differences and the pair kernel against finite
differences of the acceleration; generation rules and counters against a
textbook Generations automaton; traffic-light phases, smart lights, yield
priorities, the lookahead window, route-dependent waiting and the
controller counters; Barnes-Hut against direct summation at theta 0, the
region tree's node counts, half-open squares, the visit count, the body
update and the walls; spring mesh against one-spring and oscillator closed
forms, momentum and energy conservation and connected components; BFS
against Manhattan distances and scipy shortest paths.  Parity of every
function here is pinned by at least one of those, and each pin set was
checked by planting mistakes in a copy of this oracle: every planted
mistake that changes an output fails a pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["philox.c", "gol.c", "generation.c", "wator.c", "nasch.c", "nasch_ctrl.c", "barnes_hut.c", "bfs.c", "structure.c", "nbody.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, strict IEEE; OpenMP
    for the n-body receiver loops only)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> int:
    """Threads for the n-body receiver loops (n <= 0: OpenMP's default, all
    cores); returns the count now in use.  Results do not depend on it."""
    return int(_load().orc_set_threads(int(n)))


# ------------------------------------------------------------------ Philox
def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def draw(seed: int, tag: int, step: int, cells, inst: int = 0) -> np.ndarray:
    lib = _load()
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    out = np.empty_like(cells)
    lib.orc_draw_many(ctypes.c_uint64(seed), ctypes.c_uint32(tag), ctypes.c_uint32(step),
                      _p(cells), ctypes.c_int64(cells.size), ctypes.c_uint32(inst), _p(out))
    return out


# -------------------------------------------------------------- Game of Life
EMPTY, ALIVE, CANDIDATE = 0, 1, 2


def gol_run(W: int, H: int, kind, state, T: int):
    """Returns (kind, state, counters[T, 7]) after T generations."""
    lib = _load()
    kind = np.ascontiguousarray(kind, dtype=np.uint8).copy()
    state = np.ascontiguousarray(state, dtype=np.uint8).copy()
    cnt = np.zeros((max(T, 1), 7), dtype=np.int64)
    rc = lib.orc_gol_run(int(W), int(H), _p(kind), _p(state), int(T), _p(cnt))
    if rc != 0:
        raise ValueError("orc_gol_run: bad arguments")
    return kind, state, cnt[:T]


# ----------------------------------------------------- generational automaton
BURST = (0b111101101, 0b101011000, 255)  # survive {0,2,3,5,6,7,8}, born {3,4,6,8}, block 255
LIFE_RULE = (0b1100, 0b1000, 0)


def gen_run(W: int, H: int, kind, state, blocked, T: int, rule=BURST):
    """Returns (kind, state, blocked, counters[T, 8]) after T generations of
    the generational automaton with rule (survive mask, born mask, block)."""
    lib = _load()
    kind = np.ascontiguousarray(kind, dtype=np.uint8).copy()
    state = np.ascontiguousarray(state, dtype=np.uint8).copy()
    blocked = np.ascontiguousarray(blocked, dtype=np.uint16).copy()
    cnt = np.zeros((max(T, 1), 8), dtype=np.int64)
    s, b, blk = rule
    rc = lib.orc_gen_run(int(W), int(H), ctypes.c_uint32(s), ctypes.c_uint32(b), int(blk), _p(kind),
                         _p(state), _p(blocked), int(T), _p(cnt))
    if rc != 0:
        raise ValueError("orc_gen_run: bad arguments")
    return kind, state, blocked, cnt[:T]


# ------------------------------------------------------------------- Wa-Tor
FISH, SHARK = 1, 2


class _WatorParams(ctypes.Structure):
    _fields_ = [("fish_breed", ctypes.c_int), ("shark_breed", ctypes.c_int),
                ("starve", ctypes.c_int), ("breed_strict", ctypes.c_int)]


def wator_run(W, H, seed, kind, age, energy, T, t0=0, inst=0, fish_breed=4,
              shark_breed=12, starve=3, breed_strict=0):
    """Returns (kind, age, energy, counters[T, 8])."""
    lib = _load()
    kind = np.ascontiguousarray(kind, dtype=np.int8).copy()
    age = np.ascontiguousarray(age, dtype=np.int16).copy()
    energy = np.ascontiguousarray(energy, dtype=np.int16).copy()
    cnt = np.zeros((max(T, 1), 8), dtype=np.int64)
    p = _WatorParams(fish_breed, shark_breed, starve, breed_strict)
    rc = lib.orc_wator_run(int(W), int(H), ctypes.c_uint64(int(seed)), ctypes.c_uint32(int(inst)),
                           ctypes.byref(p), _p(kind), _p(age), _p(energy), int(t0), int(T), _p(cnt))
    if rc != 0:
        raise ValueError("orc_wator_run: bad arguments")
    return kind, age, energy, cnt[:T]


def batched_instance_run(job):
    """One instance of a batched heap run alone, for a process pool (a
    top-level function, so a spawned worker can unpickle it).  job = (index,
    kind 0 Life / 1 Wa-Tor, side, seed, k, a, e, s, T); returns (index,
    kind, age, energy, state) per cell after T steps, with the arrays of the
    kind that does not have them zero."""
    i, kind, side, seed, k, a, e, s, T = job
    if kind == 0:
        wk, ws, _ = gol_run(side, side, np.asarray(k).astype(np.uint8), s, T)
        return i, wk.astype(np.int8), np.zeros_like(a), np.zeros_like(e), ws
    wk, wa, we, _ = wator_run(side, side, seed, k, a, e, T, inst=i)
    return i, wk, wa, we, np.zeros_like(s)


# ------------------------------------------------------ Nagel-Schreckenberg
class _NaschGraph(ctypes.Structure):
    _fields_ = [("num_streets", ctypes.c_int), ("street_start", ctypes.c_void_p),
                ("street_len", ctypes.c_void_p), ("out_deg", ctypes.c_void_p),
                ("out_street", ctypes.c_void_p), ("is_source", ctypes.c_void_p),
                ("num_cells", ctypes.c_int), ("v_max", ctypes.c_int),
                ("brake_threshold", ctypes.c_uint32), ("sources_enabled", ctypes.c_int),
                ("sinks_enabled", ctypes.c_int)]


def nasch_run(graph: dict, seed: int, car_v, T: int, t0: int = 0):
    """graph: dict from inputs.nasch_graph (or a hand-built one).
    Returns (car_v, counters[T, 4])."""
    lib = _load()
    keep = {k: np.ascontiguousarray(graph[k], dtype=dt) for k, dt in
            [("street_start", np.int32), ("street_len", np.int32), ("out_deg", np.int32),
             ("out_street", np.int32), ("is_source", np.uint8)]}
    g = _NaschGraph(int(graph["num_streets"]), _p(keep["street_start"]).value,
                    _p(keep["street_len"]).value, _p(keep["out_deg"]).value,
                    _p(keep["out_street"]).value, _p(keep["is_source"]).value,
                    int(graph["num_cells"]), int(graph.get("v_max", 5)),
                    int(graph["brake_threshold"]), int(graph.get("sources_enabled", 1)),
                    int(graph.get("sinks_enabled", 1)))
    car_v = np.ascontiguousarray(car_v, dtype=np.int8).copy()
    cnt = np.zeros((max(T, 1), 4), dtype=np.int64)
    rc = lib.orc_nasch_run(ctypes.byref(g), ctypes.c_uint64(int(seed)), _p(car_v), int(t0), int(T), _p(cnt))
    if rc != 0:
        raise ValueError("orc_nasch_run: bad arguments")
    return car_v, cnt[:T]


class _NaschCtrl(ctypes.Structure):
    _fields_ = [("ctrl_kind", ctypes.c_void_p), ("phase_len", ctypes.c_int), ("lookahead", ctypes.c_int)]


def nasch_ctrl_run(graph: dict, seed: int, car_v, T: int, ctrl_kind, phase_len: int = 8,
                   lookahead: int = 5, green=None, timer=None, t0: int = 0):
    """Traffic with controllers (ctrl_kind per street: -1 none, 0 light,
    1 smart light, 2 yield).  Returns (car_v, green, timer, counters[T, 6])."""
    lib = _load()
    keep = {k: np.ascontiguousarray(graph[k], dtype=dt) for k, dt in
            [("street_start", np.int32), ("street_len", np.int32), ("out_deg", np.int32),
             ("out_street", np.int32), ("is_source", np.uint8)]}
    g = _NaschGraph(int(graph["num_streets"]), _p(keep["street_start"]).value,
                    _p(keep["street_len"]).value, _p(keep["out_deg"]).value,
                    _p(keep["out_street"]).value, _p(keep["is_source"]).value,
                    int(graph["num_cells"]), int(graph.get("v_max", 5)),
                    int(graph["brake_threshold"]), int(graph.get("sources_enabled", 1)),
                    int(graph.get("sinks_enabled", 1)))
    S = int(graph["num_streets"])
    kind = np.ascontiguousarray(ctrl_kind, dtype=np.int8)
    c = _NaschCtrl(_p(kind).value, int(phase_len), int(lookahead))
    car_v = np.ascontiguousarray(car_v, dtype=np.int8).copy()
    green = np.zeros(S, np.int16) if green is None else np.ascontiguousarray(green, np.int16).copy()
    timer = np.zeros(S, np.int16) if timer is None else np.ascontiguousarray(timer, np.int16).copy()
    cnt = np.zeros((max(T, 1), 6), dtype=np.int64)
    rc = lib.orc_nasch_ctrl_run(ctypes.byref(g), ctypes.byref(c), ctypes.c_uint64(int(seed)), _p(car_v),
                                _p(green), _p(timer), int(t0), int(T), _p(cnt))
    if rc != 0:
        raise ValueError("orc_nasch_ctrl_run: bad arguments")
    return car_v, green, timer, cnt[:T]


# ---------------------------------------------------------------------- BFS
def bfs(row_ptr, col, source: int):
    """(distances int32 with 2^31-1 for unreachable, levels)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    d = np.empty(len(rp) - 1, np.int32)
    lv = ctypes.c_int()
    rc = lib.orc_bfs(len(rp) - 1, _p(rp), _p(cl), int(source), _p(d), ctypes.byref(lv))
    if rc != 0:
        raise ValueError("orc_bfs: bad arguments")
    return d, lv.value


# --------------------------------------------------------------- Barnes-Hut
class _BHParams(ctypes.Structure):
    _fields_ = [("G", ctypes.c_float), ("eps", ctypes.c_float), ("dt", ctypes.c_float),
                ("theta", ctypes.c_float)]


def bh_run(state: dict, T: int, G=1.0, eps=1e-2, dt=1e-4, theta=0.5):
    """state: float32 arrays x, y, vx, vy, m.  Returns (new_state, counters[T, 2])."""
    lib = _load()
    st = {k: np.ascontiguousarray(state[k], dtype=np.float32).copy() for k in ("x", "y", "vx", "vy", "m")}
    p = _BHParams(G, eps, dt, theta)
    cnt = np.zeros((max(T, 1), 2), np.int64)
    rc = lib.orc_bh_run(len(st["x"]), ctypes.byref(p), _p(st["x"]), _p(st["y"]), _p(st["vx"]), _p(st["vy"]),
                        _p(st["m"]), int(T), _p(cnt))
    if rc != 0:
        raise ValueError("orc_bh_run: bad arguments or coincident bodies")
    return st, cnt[:T]


def bh_accel(x, y, m, eps=1e-2, theta=0.5):
    lib = _load()
    x, y, m = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, m))
    ax, ay = np.zeros_like(x), np.zeros_like(x)
    rc = lib.orc_bh_accel(len(x), ctypes.c_float(eps), ctypes.c_float(theta), _p(x), _p(y), _p(m), _p(ax), _p(ay))
    if rc != 0:
        raise ValueError("orc_bh_accel: bad arguments")
    return ax, ay


def bh_build(x, y):
    lib = _load()
    x, y = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y))
    n, d = ctypes.c_int(), ctypes.c_int()
    rc = lib.orc_bh_build(len(x), _p(x), _p(y), ctypes.byref(n), ctypes.byref(d))
    if rc != 0:
        raise ValueError("orc_bh_build: coincident bodies")
    return n.value, d.value


# ------------------------------------------------------------------- N-body
class _NBodyParams(ctypes.Structure):
    _fields_ = [("G", ctypes.c_float), ("eps", ctypes.c_float), ("dt", ctypes.c_float),
                ("merge_r", ctypes.c_float), ("merge", ctypes.c_int)]


def nbody_run_f32(state: dict, T: int, G=1.0, eps=1e-2, dt=1e-3, merge_r=5e-3, merge=True):
    """state: dict of float32 arrays x, y, z, vx, vy, vz, m and uint8 live
    (indexed by body id).  Returns (new_state, merges_per_step[T])."""
    lib = _load()
    st = {k: np.ascontiguousarray(state[k], dtype=np.float32).copy()
          for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    st["live"] = np.ascontiguousarray(state["live"], dtype=np.uint8).copy()
    N = st["x"].size
    cnt = np.zeros(max(T, 1), dtype=np.int64)
    p = _NBodyParams(G, eps, dt, merge_r, 1 if merge else 0)
    rc = lib.orc_nbody_run_f32(N, ctypes.byref(p), *[_p(st[k]) for k in
                               ("x", "y", "z", "vx", "vy", "vz", "m", "live")], T, _p(cnt))
    if rc != 0:
        raise ValueError("orc_nbody_run_f32: bad arguments")
    return st, cnt[:T]


def nbody_accel_f32(state: dict, G=1.0, eps=1e-2):
    lib = _load()
    x, y, z, m = (np.ascontiguousarray(state[k], dtype=np.float32) for k in ("x", "y", "z", "m"))
    live = np.ascontiguousarray(state["live"], dtype=np.uint8)
    N = x.size
    ax, ay, az = (np.zeros(N, np.float32) for _ in range(3))
    lib.orc_nbody_accel_f32(N, ctypes.c_float(G), ctypes.c_float(eps), _p(x), _p(y), _p(z),
                            _p(m), _p(live), _p(ax), _p(ay), _p(az))
    return ax, ay, az


def nbody_step_sample_f32(state: dict, idx, G=1.0, eps=1e-2, dt=1e-3):
    """One no-merge FP32 step for the receivers in idx: [len(idx), 6]
    (x, y, z, vx, vy, vz)."""
    lib = _load()
    cols = [np.ascontiguousarray(state[k], dtype=np.float32) for k in ("x", "y", "z", "vx", "vy", "vz", "m")]
    live = np.ascontiguousarray(state["live"], dtype=np.uint8)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros((idx.size, 6), np.float32)
    lib.orc_nbody_step_sample_f32(cols[0].size, ctypes.c_float(G), ctypes.c_float(eps),
                                  ctypes.c_float(dt), *[_p(c) for c in cols], _p(live), _p(idx),
                                  int(idx.size), _p(out))
    return out


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nbody_run_f64(pos, vel, m, T, G=1.0, eps=1e-2, dt=1e-3):
    lib = _load()
    pos, vel, m = _d(pos).copy(), _d(vel).copy(), _d(m)
    lib.orc_nbody_run_f64(m.size, ctypes.c_double(G), ctypes.c_double(eps), ctypes.c_double(dt),
                          _p(pos), _p(vel), _p(m), T)
    return pos, vel


def nbody_accel_f64(pos, m, G=1.0, eps=1e-2):
    lib = _load()
    pos, m = _d(pos), _d(m)
    acc = np.zeros_like(pos)
    lib.orc_nbody_accel_f64(m.size, ctypes.c_double(G), ctypes.c_double(eps), _p(pos), _p(m), _p(acc))
    return acc


def nbody_energy_f64(pos, vel, m, G=1.0, eps=1e-2):
    lib = _load()
    pos, vel, m = _d(pos), _d(vel), _d(m)
    E = ctypes.c_double()
    P = (ctypes.c_double * 3)()
    lib.orc_nbody_energy_f64(m.size, ctypes.c_double(G), ctypes.c_double(eps), _p(pos), _p(vel),
                             _p(m), ctypes.byref(E), P)
    return E.value, np.array(list(P))


def nbody_pair_adjoint_f64(pos, m, mu, G=1.0, eps=1e-2):
    lib = _load()
    pos, m, mu = _d(pos), _d(m), _d(mu)
    g = np.zeros_like(pos)
    lib.orc_nbody_pair_adjoint_f64(m.size, ctypes.c_double(G), ctypes.c_double(eps), _p(pos),
                                   _p(m), _p(mu), _p(g))
    return g


def nbody_adjoint_f64(pos0, vel0, m, T, ckpt=10, G=1.0, eps=1e-2, dt=1e-3):
    """Returns (grad wrt v0 [N,3], loss)."""
    lib = _load()
    pos0, vel0, m = _d(pos0), _d(vel0), _d(m)
    grad = np.zeros_like(pos0)
    loss = ctypes.c_double()
    rc = lib.orc_nbody_adjoint_f64(m.size, ctypes.c_double(G), ctypes.c_double(eps),
                                   ctypes.c_double(dt), _p(pos0), _p(vel0), _p(m), T, ckpt,
                                   _p(grad), ctypes.byref(loss))
    if rc != 0:
        raise ValueError("orc_nbody_adjoint_f64: bad arguments")
    return grad, loss.value


def nbody_adjoint_f32traj(state: dict, T, G=1.0, eps=1e-2, dt=1e-3):
    """FP64 reverse sweep along the FP32 trajectory: (grad [N,3], loss)."""
    lib = _load()
    cols = [np.ascontiguousarray(state[k], dtype=np.float32) for k in ("x", "y", "z", "vx", "vy", "vz", "m")]
    N = cols[0].size
    grad = np.zeros((N, 3), np.float64)
    loss = ctypes.c_double()
    rc = lib.orc_nbody_adjoint_f32traj(N, ctypes.c_float(G), ctypes.c_float(eps), ctypes.c_float(dt),
                                       *[_p(c) for c in cols], int(T), _p(grad), ctypes.byref(loss))
    if rc != 0:
        raise ValueError("orc_nbody_adjoint_f32traj: bad arguments")
    return grad, loss.value


def nbody_loss_f64(pos0, vel0, m, T, G=1.0, eps=1e-2, dt=1e-3):
    _, v = nbody_run_f64(pos0, vel0, m, T, G, eps, dt)
    m = _d(m)
    return 0.5 * float(np.sum(m[:, None] * v * v))


# ---------------------------------------------------------------- structure
STRUCT_ANCHOR, STRUCT_PULL, STRUCT_NODE = 0, 1, 2
PHASE_PULL, PHASE_COMPUTE, PHASE_REMOVE = 1, 2, 4
INF_DIST = 0x7FFFFFFF


class _StructParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("damping", ctypes.c_float), ("substeps", ctypes.c_int32)]


def structure_run(mesh: dict, T: int, dt=0.05, damping=0.01, substeps=40, phases=7):
    """mesh: the dict of ``inputs.structure_mesh`` (or any dict with its
    keys).  Returns (state, counters[T, 5]); state holds the updated node
    arrays x, y, vx, vy, slot, nspr, nalive, dist and spring arrays fx, fy,
    salive (the constant arrays are not copied)."""
    lib = _load()
    N, S = len(mesh["kind"]), len(mesh["p1"])
    f32 = lambda k: np.ascontiguousarray(mesh[k], dtype=np.float32).copy()
    st = {k: f32(k) for k in ("x", "y", "vx", "vy")}
    st["slot"] = np.ascontiguousarray(mesh["slot"], dtype=np.int32).reshape(N, 3).copy()
    st["nspr"] = np.ascontiguousarray(mesh["nspr"], dtype=np.int32).copy()
    st["nalive"] = np.ascontiguousarray(mesh.get("nalive", np.ones(N, np.uint8)), dtype=np.uint8).copy()
    st["fx"] = np.ascontiguousarray(mesh.get("fx", np.zeros(S, np.float32)), dtype=np.float32).copy()
    st["fy"] = np.ascontiguousarray(mesh.get("fy", np.zeros(S, np.float32)), dtype=np.float32).copy()
    st["salive"] = np.ascontiguousarray(mesh.get("salive", np.ones(S, np.uint8)), dtype=np.uint8).copy()
    st["dist"] = np.zeros(N, np.int32)
    const = {k: np.ascontiguousarray(mesh[k], dtype=t) for k, t in
             (("kind", np.int8), ("m", np.float32), ("p1", np.int32), ("p2", np.int32), ("k", np.float32),
              ("L0", np.float32), ("fmax", np.float32))}
    cnt = np.zeros((max(T, 1), 5), np.int64)
    p = _StructParams(dt, damping, substeps)
    rc = lib.orc_structure_run(N, S, ctypes.byref(p), _p(const["kind"]), _p(st["x"]), _p(st["y"]), _p(st["vx"]),
                               _p(st["vy"]), _p(const["m"]), _p(st["slot"]), _p(st["nspr"]), _p(st["nalive"]),
                               _p(const["p1"]), _p(const["p2"]), _p(const["k"]), _p(const["L0"]),
                               _p(const["fmax"]), _p(st["fx"]), _p(st["fy"]), _p(st["salive"]), _p(st["dist"]),
                               int(T), int(phases), _p(cnt))
    if rc != 0:
        raise ValueError("orc_structure_run: bad arguments")
    return st, cnt[:T]
