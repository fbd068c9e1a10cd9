// wl_nasch.cu -- Nagel-Schreckenberg traffic on a street graph as an SMMO
// application (thesis Sec. 7.5).  Classes: Cell {car: handle}, Car {cell,
// street, v, route, cross}, Source {street}.  One step is three do-alls:
//   Car::prepare  accelerate, compute the path of the next v cells
//                 (choosing the outgoing street at the end of the street),
//                 cut v to the free cells on the path (occupancy at step
//                 start), brake with probability p, and post a claim on the
//                 first cell of the street the car would enter;
//   Car::move     a car that lost its claim stops at the end of its street;
//                 a car on a sink street that ends on or passes the last
//                 cell deletes itself; the others move;
//   Source::spawn a producer street whose first cell is empty creates a Car.
// Claims are u64 words per street: ((2^32-1-t) << 32) | cell, atomicMin, so
// the lowest cell wins and words of older steps never match (no reset).
//
// Traffic controllers (Sec. 7.5, optional): a Controller object guards the
// entry of a street o with two or more incoming streets (listed in an
// inlined inner array, increasing street id) and runs first in every step,
// Controller::step, reading the occupancy at step start: a traffic light
// moves its green on after `phase_len` steps (round robin), a smart traffic
// light turns green at once for the only incoming street with a waiting
// car, a yield controller gives green to the first incoming street with a
// waiting car (a car within `lookahead` cells of the end of a street whose
// route in this step leads to o).  It publishes the green street per street
// o; Car::prepare then follows the thesis' adjust-velocity rule with speed
// limits: the first cell of o has limit 0 for cars from a red street, every
// other cell v_max (with no controller this is the plain free-cell count).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "grid_common.cuh"
#include "heap_internal.h"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

struct TrafficArgs {
  const int32_t* start;   // per street
  const int32_t* len;
  const int32_t* deg;
  const int32_t* out;     // 3 per street
  unsigned long long* claim;  // per street
  CellRef cells;
  uint32_t occ_off;
  uint32_t car_cls;
  uint32_t c_cell, c_street, c_v, c_route, c_cross;
  uint32_t s_street;      // Source.street column offset
  int32_t* green_street;  // per street: green incoming street, -1 = no controller
  // Controller column offsets; k_in is the column index of the first of the
  // SMMO_TRAFFIC_MAX_IN inlined incoming-street columns
  uint32_t k_street, k_kind, k_nin, k_green, k_timer, k_in;
  int32_t phase_len, lookahead;
  uint64_t seed;
  const uint32_t* tp;  // device step counter
  int32_t v_max;
  uint32_t brake_threshold;
  int32_t sinks_enabled;
  // export
  int8_t* out_v;
  uint32_t* out_count;
  unsigned long long* errors;
};

template <class T>
__device__ __forceinline__ T* fld(const HeapView& h, uint32_t self, uint32_t off) {
  return field_ptr<T>(h, off, self);
}

struct CarPrepare {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const int32_t c = *fld<int32_t>(h, self, a.c_cell);
    const int32_t s = *fld<int32_t>(h, self, a.c_street);
    int8_t* vp = fld<int8_t>(h, self, a.c_v);
    const int32_t st = __ldg(a.start + s), L = __ldg(a.len + s), dg = __ldg(a.deg + s);
    const int32_t p = c - st;
    int v = *vp + 1 < a.v_max ? *vp + 1 : a.v_max;
    int32_t o = -1;
    const uint32_t t = *a.tp;
    if (dg > 0) {
      const uint32_t r = philox_draw(a.seed, TAG_ROUTE, t, (uint32_t)(st + L - 1), 0);
      o = __ldg(a.out + 3 * s + (int)(r % (uint32_t)dg));
    }
    // adjust velocity along the path: an occupied cell stops the car before
    // it; a cell whose limit is below v lowers v to the limit if that still
    // reaches the cell, else the car stops before it
    const int32_t gs = o >= 0 ? a.green_street[o] : -1;
    for (int d = 1; d <= v; ++d) {
      const int32_t q = p + d;
      int32_t cell, limit = a.v_max;
      if (q < L) {
        cell = st + q;
      } else if (o >= 0) {
        cell = __ldg(a.start + o) + (q - L);
        if (q == L && gs >= 0 && gs != s) limit = 0;  // red at the crossing
      } else if (a.sinks_enabled) {
        continue;  // leaving the network: free, no limit
      } else {
        v = d - 1;  // dead end
        break;
      }
      if (*a.cells.col<uint32_t>((uint32_t)cell, a.occ_off) != kNull) { v = d - 1; break; }
      if (v > limit) {
        if (limit > d - 1) v = limit;
        else { v = d - 1; break; }
      }
    }
    if (v > 0 && philox_draw(a.seed, TAG_BRAKE, t, (uint32_t)c, 0) < a.brake_threshold) --v;
    const bool cross = o >= 0 && p + v >= L;
    if (cross)
      atomicMin(a.claim + o, ((unsigned long long)(0xFFFFFFFFu - t) << 32) | (uint32_t)c);
    *vp = (int8_t)v;
    *fld<int32_t>(h, self, a.c_route) = o;
    *fld<uint8_t>(h, self, a.c_cross) = cross ? 1 : 0;
  }
};

struct CarMove {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    int32_t* cp = fld<int32_t>(h, self, a.c_cell);
    int32_t* sp = fld<int32_t>(h, self, a.c_street);
    int8_t* vp = fld<int8_t>(h, self, a.c_v);
    const int32_t c = *cp, s = *sp;
    const int32_t st = __ldg(a.start + s), L = __ldg(a.len + s);
    const int32_t p = c - st;
    int v = *vp;
    const int32_t o = *fld<int32_t>(h, self, a.c_route);
    bool cross = *fld<uint8_t>(h, self, a.c_cross);
    if (cross && a.claim[o] != (((unsigned long long)(0xFFFFFFFFu - *a.tp) << 32) | (uint32_t)c)) {
      v = L - 1 - p;  // lost the claim: stop on the last cell of the street
      cross = false;
      *vp = (int8_t)v;
    }
    if (__ldg(a.deg + s) == 0 && a.sinks_enabled && p + v >= L - 1) {
      *a.cells.col<uint32_t>((uint32_t)c, a.occ_off) = kNull;
      smmo_delete(h, self);
      return;
    }
    if (v == 0) return;
    const int32_t q = p + v;
    const int32_t dst = q < L ? st + q : __ldg(a.start + o) + (q - L);
    *a.cells.col<uint32_t>((uint32_t)c, a.occ_off) = kNull;
    *a.cells.col<uint32_t>((uint32_t)dst, a.occ_off) = self;
    *cp = dst;
    if (q >= L) *sp = o;
  }
};

struct SourceSpawn {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const int32_t s = *fld<int32_t>(h, self, a.s_street);
    const uint32_t c = (uint32_t)__ldg(a.start + s);
    uint32_t* occ = a.cells.col<uint32_t>(c, a.occ_off);
    if (*occ != kNull) return;
    const uint32_t car = smmo_new(h, a.car_cls);
    if (car == kNull) return;
    *fld<int32_t>(h, car, a.c_cell) = (int32_t)c;
    *fld<int32_t>(h, car, a.c_street) = s;
    *fld<int8_t>(h, car, a.c_v) = 0;
    *fld<int32_t>(h, car, a.c_route) = -1;
    *fld<uint8_t>(h, car, a.c_cross) = 0;
    *occ = car;
  }
};

enum { CTRL_LIGHT = 0, CTRL_SMART = 1, CTRL_YIELD = 2 };

struct CtrlStep {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t o = *fld<int32_t>(h, self, a.k_street);
    const int kind = *fld<int8_t>(h, self, a.k_kind);
    const int n = *fld<int8_t>(h, self, a.k_nin);
    int16_t* gp = fld<int16_t>(h, self, a.k_green);
    int16_t* tp = fld<int16_t>(h, self, a.k_timer);
    const uint32_t t = *a.tp;
    uint32_t wait = 0;  // bit i: incoming street i has a car waiting for o
    for (int i = 0; i < n; ++i) {
      const int32_t s = *fld<int32_t>(h, self, __ldg(&h.cls[c].col_off[a.k_in + i]));
      const int32_t st = __ldg(a.start + s), L = __ldg(a.len + s), dg = __ldg(a.deg + s);
      if (dg <= 0) continue;
      const uint32_t r = philox_draw(a.seed, TAG_ROUTE, t, (uint32_t)(st + L - 1), 0);
      if (__ldg(a.out + 3 * s + (int)(r % (uint32_t)dg)) != o) continue;
      for (int k = 0; k < a.lookahead && k < L; ++k)
        if (*a.cells.col<uint32_t>((uint32_t)(st + L - 1 - k), a.occ_off) != kNull) { wait |= 1u << i; break; }
    }
    int gi = *gp, tm = *tp;
    if (kind == CTRL_YIELD) {
      if (wait) gi = __ffs(wait) - 1;
    } else if (kind == CTRL_SMART && __popc(wait) == 1 && !((wait >> gi) & 1)) {
      gi = __ffs(wait) - 1;
      tm = 0;
    } else if (++tm >= a.phase_len) {
      gi = gi + 1 == n ? 0 : gi + 1;
      tm = 0;
    }
    *gp = (int16_t)gi;
    *tp = (int16_t)tm;
    a.green_street[o] = *fld<int32_t>(h, self, __ldg(&h.cls[c].col_off[a.k_in + gi]));
  }
};

struct CtrlExport {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const int32_t o = *fld<int32_t>(h, self, a.k_street);
    // green and timer of street o, packed into the export's 32-bit array
    reinterpret_cast<int32_t*>(a.out_count)[o] =
        ((int32_t)*fld<int16_t>(h, self, a.k_green) << 16) | (uint16_t)*fld<int16_t>(h, self, a.k_timer);
  }
};

struct CarLink {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    *a.cells.col<uint32_t>((uint32_t)*fld<int32_t>(h, self, a.c_cell), a.occ_off) = self;
  }
};

struct CarExport {
  using Args = TrafficArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t c = (uint32_t)*fld<int32_t>(h, self, a.c_cell);
    if (atomicAdd(a.out_count + c, 1u)) atomicAdd(a.errors, 1ull);
    if (*a.cells.col<uint32_t>(c, a.occ_off) != self) atomicAdd(a.errors, 1ull);
    a.out_v[c] = *fld<int8_t>(h, self, a.c_v);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_nasch[] = {
    SMMO_METHOD("nasch.car_prepare", CarPrepare), SMMO_METHOD("nasch.car_move", CarMove),
    SMMO_METHOD("nasch.source_spawn", SourceSpawn), SMMO_METHOD("nasch.car_link", CarLink),
    SMMO_METHOD("nasch.car_export", CarExport), SMMO_METHOD("nasch.controller_step", CtrlStep),
    SMMO_METHOD("nasch.controller_export", CtrlExport)};
const int g_methods_nasch_n = sizeof(g_methods_nasch) / sizeof(g_methods_nasch[0]);

struct smmo_traffic {
  smmo_heap* heap = nullptr;
  int cls_cell = -1, cls_car = -1, cls_src = -1, cls_ctrl = -1;
  int num_streets = 0, num_cells = 0;
  bool controllers = false;
  int32_t* d_tab = nullptr;  // start | len | deg | out[3]
  int32_t* d_green = nullptr;  // per street green incoming street (-1: none)
  unsigned long long* d_claim = nullptr;
  uint32_t t = 0;
  uint32_t* d_t = nullptr;
  TrafficArgs args{};
};

namespace {
int pdo(smmo_traffic* w, int cls, method_launch_fn fn, const TrafficArgs& a, cudaStream_t s,
        bool reuse = false) {
  int st = reuse ? SMMO_OK : enumerate(w->heap, cls, s);
  if (!st) st = fn(w->heap, cls, &a, s);
  return st;
}
}  // namespace

extern "C" {

int smmo_traffic_create(smmo_heap* heap, int num_streets, const int32_t* street_start,
                        const int32_t* street_len, const int32_t* out_deg, const int32_t* out_street,
                        const uint8_t* is_source, int v_max, uint32_t brake_threshold,
                        int sources_enabled, int sinks_enabled, uint64_t seed, const int8_t* car_v,
                        void* stream, smmo_traffic** out) {
  if (!heap || num_streets < 1 || !street_start || !street_len || !out_deg || !out_street ||
      !is_source || !car_v || !out || v_max < 1 || v_max > 100)
    return SMMO_E_INVALID_ARG;
  if (!heap->classes.empty() || heap->frozen) return SMMO_E_FROZEN;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t cells = 0;
  for (int i = 0; i < num_streets; ++i) {
    if (street_len[i] < 2 || street_start[i] != cells || out_deg[i] < 0 || out_deg[i] > 3)
      return SMMO_E_INVALID_ARG;
    for (int k = 0; k < out_deg[i]; ++k)
      if (out_street[3 * i + k] < 0 || out_street[3 * i + k] >= num_streets) return SMMO_E_INVALID_ARG;
    cells += street_len[i];
  }
  if (cells >= (1ll << 31)) return SMMO_E_INVALID_ARG;
  smmo_traffic* w = new smmo_traffic();
  w->heap = heap;
  w->num_streets = num_streets;
  w->num_cells = (int)cells;
  smmo_field_desc cf[1] = {{"car", SMMO_HANDLE, 1, -1}};
  smmo_field_desc kf[5] = {{"cell", SMMO_I32, 1, -1}, {"street", SMMO_I32, 1, -1}, {"v", SMMO_I8, 1, -1},
                           {"route", SMMO_I32, 1, -1}, {"cross", SMMO_U8, 1, -1}};
  smmo_field_desc sf[1] = {{"street", SMMO_I32, 1, -1}};
  smmo_field_desc tf[6] = {{"street", SMMO_I32, 1, -1}, {"kind", SMMO_I8, 1, -1}, {"n_in", SMMO_I8, 1, -1},
                           {"green", SMMO_I16, 1, -1}, {"timer", SMMO_I16, 1, -1},
                           {"in", SMMO_I32, SMMO_TRAFFIC_MAX_IN, -1}};
  int st = smmo_class_register(heap, "Car", kf, 5, -1, 0, &w->cls_car);
  if (!st) st = smmo_class_register(heap, "Cell", cf, 1, -1, 0, &w->cls_cell);
  if (!st) st = smmo_class_register(heap, "Source", sf, 1, -1, 0, &w->cls_src);
  if (!st) st = smmo_class_register(heap, "Controller", tf, 6, -1, 0, &w->cls_ctrl);
  if (heap->cfg.block_data_bytes == 0) heap->cfg.block_data_bytes = 256 + 256 + 64 + 256 + 64;
  if (!st) st = freeze(heap, s);
  if (!st && heap->classes[w->cls_cell].layout.cap != 64) st = SMMO_E_UNSUPPORTED;
  if (st) { delete w; return st; }
  std::vector<int32_t> tab(6 * (size_t)num_streets, -1);
  for (int i = 0; i < num_streets; ++i) {
    tab[i] = street_start[i];
    tab[num_streets + i] = street_len[i];
    tab[2 * num_streets + i] = out_deg[i];
    for (int k = 0; k < 3; ++k) tab[3 * num_streets + 3 * i + k] = k < out_deg[i] ? out_street[3 * i + k] : -1;
  }
  cudaError_t e = cudaMalloc(&w->d_tab, sizeof(int32_t) * tab.size());
  if (e == cudaSuccess) e = cudaMalloc(&w->d_claim, sizeof(unsigned long long) * num_streets);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_t, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&w->d_green, sizeof(int32_t) * num_streets);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_green, 0xFF, sizeof(int32_t) * num_streets, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_t, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->d_tab, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_claim, 0xFF, sizeof(unsigned long long) * num_streets, s);
  if (e != cudaSuccess) { smmo_traffic_destroy(w); return cuda_status(e); }
  // cells (dense, in cell order), empty
  uint32_t* occ0 = nullptr;
  e = cudaMallocAsync(&occ0, (size_t)cells * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(occ0, 0xFF, (size_t)cells * 4, s);
  if (e != cudaSuccess) { smmo_traffic_destroy(w); return cuda_status(e); }
  const void* csrc[1] = {occ0};
  int64_t first = -1;
  st = smmo_bulk_new(heap, w->cls_cell, cells, csrc, nullptr, &first, stream);
  cudaFreeAsync(occ0, s);
  if (!st && first < 0) st = SMMO_E_OOM;
  if (st) { smmo_traffic_destroy(w); return st; }
  TrafficArgs& a = w->args;
  memset(&a, 0, sizeof(a));
  a.start = w->d_tab;
  a.len = w->d_tab + num_streets;
  a.deg = w->d_tab + 2 * num_streets;
  a.out = w->d_tab + 3 * num_streets;
  a.claim = w->d_claim;
  a.cells.data = heap->view.data;
  a.cells.block_bytes = heap->view.block_bytes;
  a.cells.b0 = (uint32_t)first;
  a.cells.shift = 6;
  a.tp = w->d_t;
  a.occ_off = heap->classes[w->cls_cell].layout.col_off[0];
  const ClassLayout& K = heap->classes[w->cls_car].layout;
  a.car_cls = w->cls_car;
  a.c_cell = K.col_off[0]; a.c_street = K.col_off[1]; a.c_v = K.col_off[2];
  a.c_route = K.col_off[3]; a.c_cross = K.col_off[4];
  a.s_street = heap->classes[w->cls_src].layout.col_off[0];
  a.green_street = w->d_green;
  {
    const ClassLayout& T = heap->classes[w->cls_ctrl].layout;
    a.k_street = T.col_off[0]; a.k_kind = T.col_off[1]; a.k_nin = T.col_off[2];
    a.k_green = T.col_off[3]; a.k_timer = T.col_off[4];
    a.k_in = 5;  // first column index of the inlined incoming-street array
  }
  a.phase_len = 8;
  a.lookahead = v_max;
  a.seed = seed;
  a.v_max = v_max;
  a.brake_threshold = brake_threshold;
  a.sinks_enabled = sinks_enabled;
  // cars and sources from the host copies (setup only)
  std::vector<int8_t> hv((size_t)cells);
  e = cudaMemcpyAsync(hv.data(), car_v, (size_t)cells, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { smmo_traffic_destroy(w); return cuda_status(e); }
  std::vector<int32_t> kc, ks, kr;
  std::vector<int8_t> kv;
  std::vector<uint8_t> kx;
  int sidx = 0;
  for (int64_t c = 0; c < cells; ++c) {
    while (sidx + 1 < num_streets && street_start[sidx + 1] <= c) ++sidx;
    if (hv[c] < 0) continue;
    kc.push_back((int32_t)c); ks.push_back(sidx); kv.push_back(hv[c]); kr.push_back(-1); kx.push_back(0);
  }
  std::vector<int32_t> src;
  if (sources_enabled)
    for (int i = 0; i < num_streets; ++i) if (is_source[i]) src.push_back(i);
  auto upload = [&](int cls, std::vector<const void*> cols, std::vector<size_t> esz, size_t n) -> int {
    if (n == 0) return SMMO_OK;
    std::vector<void*> d(cols.size(), nullptr);
    cudaError_t ee = cudaSuccess;
    for (size_t k = 0; k < cols.size() && ee == cudaSuccess; ++k) {
      ee = cudaMallocAsync(&d[k], n * esz[k], s);
      if (ee == cudaSuccess) ee = cudaMemcpyAsync(d[k], cols[k], n * esz[k], cudaMemcpyHostToDevice, s);
    }
    int r = ee == cudaSuccess ? smmo_bulk_new(heap, cls, (int64_t)n, (const void* const*)d.data(), nullptr, nullptr, stream)
                              : cuda_status(ee);
    for (void* p : d) if (p) cudaFreeAsync(p, s);
    return r;
  };
  st = upload(w->cls_car, {kc.data(), ks.data(), kv.data(), kr.data(), kx.data()}, {4, 4, 1, 4, 1}, kc.size());
  if (!st) st = upload(w->cls_src, {src.data()}, {4}, src.size());
  if (!st) st = pdo(w, w->cls_car, &launch_do_all<CarLink>, a, s);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  if (st) { smmo_traffic_destroy(w); return st; }
  *out = w;
  return SMMO_OK;
}

int smmo_traffic_step(smmo_traffic* w, int nsteps, void* stream) {
  if (!w || nsteps < 0) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  TrafficArgs a = w->args;
  for (int k = 0; k < nsteps; ++k) {
    ++w->t;
    k_step_begin<<<1, 1, 0, s>>>(w->d_t);
    int st = cuda_status(cudaGetLastError());
    if (!st && w->controllers) st = pdo(w, w->cls_ctrl, &launch_do_all<CtrlStep>, a, s);
    if (!st) st = pdo(w, w->cls_car, &launch_do_all<CarPrepare>, a, s);
    if (!st) st = pdo(w, w->cls_car, &launch_do_all<CarMove>, a, s, true);  // prepare keeps the cars
    if (!st) st = pdo(w, w->cls_src, &launch_do_all<SourceSpawn>, a, s);
    if (st) return st;
  }
  return SMMO_OK;
}

int smmo_traffic_export(smmo_traffic* w, int8_t* car_v, int64_t* errors, void* stream) {
  if (!w || !car_v) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  TrafficArgs a = w->args;
  uint32_t* cnt = nullptr;
  unsigned long long* err = nullptr;
  cudaError_t e = cudaMallocAsync(&cnt, (size_t)w->num_cells * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&err, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)w->num_cells * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(car_v, 0xFF, (size_t)w->num_cells, s);
  if (e != cudaSuccess) return cuda_status(e);
  a.out_v = car_v;
  a.out_count = cnt;
  a.errors = err;
  int st = pdo(w, w->cls_car, &launch_do_all<CarExport>, a, s);
  unsigned long long herr = 0;
  if (!st) {
    e = cudaMemcpyAsync(&herr, err, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(err, s);
  if (errors) *errors = (int64_t)herr;
  return st;
}

int smmo_traffic_set_controllers(smmo_traffic* w, const int8_t* ctrl_kind, int phase_len, int lookahead,
                                 void* stream) {
  if (!w || !ctrl_kind || phase_len < 1 || phase_len > 32767 || lookahead < 0) return SMMO_E_INVALID_ARG;
  if (w->controllers) return SMMO_E_INVALID_ARG;  // once per traffic object
  cudaStream_t s = (cudaStream_t)stream;
  const int S = w->num_streets;
  // incoming lists in increasing street id, from the host copy of the table
  std::vector<int32_t> tab(6 * (size_t)S);
  cudaError_t e = cudaMemcpyAsync(tab.data(), w->d_tab, sizeof(int32_t) * tab.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<std::vector<int32_t>> in((size_t)S);
  for (int i = 0; i < S; ++i)
    for (int k = 0; k < tab[2 * S + i]; ++k) in[(size_t)tab[3 * S + 3 * i + k]].push_back(i);
  std::vector<int32_t> street, ins;
  std::vector<int8_t> kind, nin;
  std::vector<int16_t> zero;
  for (int o = 0; o < S; ++o) {
    if (ctrl_kind[o] < 0 || in[o].size() < 2) continue;
    if (ctrl_kind[o] > 2 || in[o].size() > SMMO_TRAFFIC_MAX_IN) return SMMO_E_UNSUPPORTED;
    street.push_back(o);
    kind.push_back(ctrl_kind[o]);
    nin.push_back((int8_t)in[o].size());
    zero.push_back(0);
  }
  const size_t n = street.size();
  w->args.phase_len = phase_len;
  w->args.lookahead = lookahead;
  w->controllers = true;
  if (n == 0) return SMMO_OK;
  // the inlined array: column k holds the k-th incoming street (-1 past n_in)
  ins.assign(n * SMMO_TRAFFIC_MAX_IN, -1);
  for (size_t j = 0; j < n; ++j)
    for (size_t k = 0; k < in[(size_t)street[j]].size(); ++k) ins[k * n + j] = in[(size_t)street[j]][k];
  std::vector<const void*> cols = {street.data(), kind.data(), nin.data(), zero.data(), zero.data()};
  std::vector<size_t> esz = {4, 1, 1, 2, 2};
  for (int k = 0; k < SMMO_TRAFFIC_MAX_IN; ++k) { cols.push_back(ins.data() + (size_t)k * n); esz.push_back(4); }
  std::vector<void*> d(cols.size(), nullptr);
  for (size_t k = 0; k < cols.size() && e == cudaSuccess; ++k) {
    e = cudaMallocAsync(&d[k], n * esz[k], s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d[k], cols[k], n * esz[k], cudaMemcpyHostToDevice, s);
  }
  int st = e == cudaSuccess ? smmo_bulk_new(w->heap, w->cls_ctrl, (int64_t)n, (const void* const*)d.data(), nullptr,
                                            nullptr, stream)
                            : cuda_status(e);
  for (void* p : d) if (p) cudaFreeAsync(p, s);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  return st;
}

int smmo_traffic_controller_state(smmo_traffic* w, int16_t* green, int16_t* timer, void* stream) {
  if (!w || !green || !timer) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int S = w->num_streets;
  for (int i = 0; i < S; ++i) { green[i] = 0; timer[i] = 0; }
  if (!w->controllers) return SMMO_OK;
  int32_t* packed = nullptr;
  cudaError_t e = cudaMallocAsync(&packed, sizeof(int32_t) * S, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(packed, 0, sizeof(int32_t) * S, s);
  if (e != cudaSuccess) return cuda_status(e);
  TrafficArgs a = w->args;
  a.out_count = reinterpret_cast<uint32_t*>(packed);
  int st = pdo(w, w->cls_ctrl, &launch_do_all<CtrlExport>, a, s);
  std::vector<int32_t> h((size_t)S);
  if (!st) {
    e = cudaMemcpyAsync(h.data(), packed, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  cudaFreeAsync(packed, s);
  if (st) return st;
  for (int i = 0; i < S; ++i) { green[i] = (int16_t)(h[(size_t)i] >> 16); timer[i] = (int16_t)(h[(size_t)i] & 0xFFFF); }
  return SMMO_OK;
}

int smmo_traffic_info(smmo_traffic* w, int64_t* num_cells, int* class_ids, uint32_t* steps_done) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (num_cells) *num_cells = w->num_cells;
  if (class_ids) {
    class_ids[0] = w->cls_cell; class_ids[1] = w->cls_car; class_ids[2] = w->cls_src; class_ids[3] = w->cls_ctrl;
  }
  if (steps_done) *steps_done = w->t;
  return SMMO_OK;
}

int smmo_traffic_destroy(smmo_traffic* w) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (w->d_tab) cudaFree(w->d_tab);
  if (w->d_claim) cudaFree(w->d_claim);
  if (w->d_t) cudaFree(w->d_t);
  if (w->d_green) cudaFree(w->d_green);
  delete w;
  return SMMO_OK;
}

}  // extern "C"
