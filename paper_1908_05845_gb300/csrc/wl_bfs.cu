// wl_bfs.cu -- frontier-based breadth-first search as an SMMO application
// (the thesis' BFS of Sec. 4.3, run with parallel_do_and_reduce of Sec.
// 3.2.2 for termination).
//
// Class Vertex {distance, degree, id, nbr[SMMO_BFS_MAX_DEGREE]}: the
// neighbours are an inner array inlined into the SOA block (one column per
// entry).  Level f is one parallel_do_and_reduce of Vertex::visit(f): a
// vertex at distance f lowers every neighbour whose distance exceeds f + 1
// to f + 1 and returns whether it changed one; the OR of the results tells
// whether level f + 1 is non-empty.  Racing writers of a neighbour write
// the same value, so distances do not depend on timing.  The vertex set is
// fixed during a search: one snapshot serves every level, and the levels
// run check_every at a time in one cooperative launch (levels.cuh).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "heap_internal.h"
#include "levels.cuh"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

enum { V_DIST = 0, V_DEG = 1, V_ID = 2, V_NBR = 3 };
constexpr int32_t kInf = 0x7FFFFFFF;

struct BfsArgs {
  int32_t frontier;
  int32_t source;
  const uint32_t* handles;  // vertex id -> handle (linking)
  int32_t* out;             // export: distance by id
  uint32_t n0;
};

template <class T>
__device__ __forceinline__ T* V(const HeapView& h, uint32_t c, uint32_t self, int col) {
  return field_ptr<T>(h, __ldg(&h.cls[c].col_off[col]), self);
}

// neighbour columns hold vertex ids after creation: replace them by handles
struct VertexLink {
  using Args = BfsArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int deg = *V<int32_t>(h, c, self, V_DEG);
    for (int k = 0; k < deg; ++k) {
      uint32_t* p = V<uint32_t>(h, c, self, V_NBR + k);
      const uint32_t id = *p;
      *p = id < a.n0 ? a.handles[id] : kNull;
      if (id >= a.n0) set_error(h, SMMO_E_BOUNDS, id);
    }
  }
};

struct VertexReset {
  using Args = BfsArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    *V<int32_t>(h, c, self, V_DIST) = *V<int32_t>(h, c, self, V_ID) == a.source ? 0 : kInf;
  }
};

// Vertex::visit(frontier), reducing with OR: 1 if a neighbour was lowered.
// The frontier vertices are a level's critical path: the neighbour handles,
// then all neighbour distances, are loaded before any store.  Distances,
// which other CTAs write between levels of one launch, are read through L2.
struct VertexVisit {
  using Args = BfsArgs;
  __device__ static bool active(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    return __ldcg(V<int32_t>(h, c, self, V_DIST)) == a.frontier;
  }
  __device__ static long long run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (!active(h, a, c, self)) return 0;
    const int deg = *V<int32_t>(h, c, self, V_DEG);
    uint32_t nb[SMMO_BFS_MAX_DEGREE];
    int32_t dv[SMMO_BFS_MAX_DEGREE];
#pragma unroll
    for (int k = 0; k < SMMO_BFS_MAX_DEGREE; ++k) nb[k] = k < deg ? *V<uint32_t>(h, c, self, V_NBR + k) : kNull;
#pragma unroll
    for (int k = 0; k < SMMO_BFS_MAX_DEGREE; ++k) dv[k] = nb[k] != kNull ? __ldcg(V<int32_t>(h, c, nb[k], V_DIST)) : 0;
    long long changed = 0;
#pragma unroll
    for (int k = 0; k < SMMO_BFS_MAX_DEGREE; ++k)
      if (nb[k] != kNull && dv[k] > a.frontier + 1) {
        *V<int32_t>(h, c, nb[k], V_DIST) = a.frontier + 1;
        changed = 1;
      }
    return changed;
  }
};

struct VertexExport {
  using Args = BfsArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t id = *V<int32_t>(h, c, self, V_ID);
    if (id >= 0 && (uint32_t)id < a.n0) a.out[id] = *V<int32_t>(h, c, self, V_DIST);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_bfs[] = {
    SMMO_METHOD("bfs.vertex_link", VertexLink), SMMO_METHOD("bfs.vertex_reset", VertexReset),
    SMMO_METHOD_REDUCE("bfs.vertex_visit", VertexVisit), SMMO_METHOD("bfs.vertex_export", VertexExport)};
const int g_methods_bfs_n = sizeof(g_methods_bfs) / sizeof(g_methods_bfs[0]);

struct smmo_bfs {
  smmo_heap* heap = nullptr;
  int cls = -1;
  uint32_t n0 = 0;
  unsigned long long* d_flags = nullptr;  // one OR result per level of a launch
  unsigned long long* d_arrive = nullptr;  // level barrier words
  int flags_cap = 0;
  BfsArgs args{};
  smmo::Snapshot snap;                    // the vertices (fixed during a search)
};

extern "C" {

int smmo_bfs_create(smmo_heap* heap, int64_t n, const int32_t* row_ptr, const int32_t* col, void* stream,
                    smmo_bfs** out) {
  if (!heap || n < 1 || n >= (1ll << 31) || !row_ptr || !col || !out) return SMMO_E_INVALID_ARG;
  if (!heap->classes.empty() || heap->frozen) return SMMO_E_FROZEN;
  if (row_ptr[0] != 0) return SMMO_E_INVALID_ARG;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t d = (int64_t)row_ptr[v + 1] - row_ptr[v];
    if (d < 0) return SMMO_E_INVALID_ARG;
    if (d > SMMO_BFS_MAX_DEGREE) return SMMO_E_UNSUPPORTED;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
      if (col[e] < 0 || col[e] >= n) return SMMO_E_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  smmo_bfs* w = new smmo_bfs();
  w->heap = heap;
  w->n0 = (uint32_t)n;
  smmo_field_desc f[4] = {{"distance", SMMO_I32, 1, -1}, {"degree", SMMO_I32, 1, -1}, {"id", SMMO_I32, 1, -1},
                          {"nbr", SMMO_HANDLE, SMMO_BFS_MAX_DEGREE, -1}};
  int st = smmo_class_register(heap, "Vertex", f, 4, -1, 0, &w->cls);
  if (!st) st = freeze(heap, s);
  if (st) { delete w; return st; }
  // columns: distance, degree, id, then neighbour ids (-1 past the degree)
  const size_t N = (size_t)n;
  std::vector<int32_t> dist(N, kInf), deg(N), ids(N), nbr(N * SMMO_BFS_MAX_DEGREE, -1);
  for (size_t v = 0; v < N; ++v) {
    deg[v] = row_ptr[v + 1] - row_ptr[v];
    ids[v] = (int32_t)v;
    for (int k = 0; k < deg[v]; ++k) nbr[(size_t)k * N + v] = col[row_ptr[v] + k];
  }
  std::vector<const void*> cols = {dist.data(), deg.data(), ids.data()};
  for (int k = 0; k < SMMO_BFS_MAX_DEGREE; ++k) cols.push_back(nbr.data() + (size_t)k * N);
  std::vector<void*> d(cols.size(), nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < cols.size() && e == cudaSuccess; ++k) {
    e = cudaMallocAsync(&d[k], N * 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d[k], cols[k], N * 4, cudaMemcpyHostToDevice, s);
  }
  uint32_t* handles = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&handles, N * 4, s);
  if (e == cudaSuccess) st = smmo_bulk_new(heap, w->cls, n, (const void* const*)d.data(), handles, nullptr, stream);
  for (void* p : d) if (p) cudaFreeAsync(p, s);
  if (e != cudaSuccess) st = cuda_status(e);
  BfsArgs& a = w->args;
  memset(&a, 0, sizeof(a));
  a.n0 = (uint32_t)n;
  if (!st) {
    a.handles = handles;
    st = enumerate(heap, w->cls, s);
    if (!st) st = launch_do_all<VertexLink>(heap, w->cls, &a, s);
    a.handles = nullptr;
  }
  if (handles) cudaFreeAsync(handles, s);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  if (st) { delete w; return st; }
  *out = w;
  return SMMO_OK;
}

int smmo_bfs_run(smmo_bfs* w, int32_t source, int check_every, int32_t* levels, void* stream) {
  if (!w || source < 0 || (uint32_t)source >= w->n0 || check_every < 1 || check_every > 4096)
    return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!w->d_arrive) {
    cudaError_t e = cudaMalloc(&w->d_arrive, sizeof(unsigned long long) * kBarrierWords);
    if (e != cudaSuccess) { w->d_arrive = nullptr; return cuda_status(e); }
  }
  if (w->flags_cap < check_every) {
    if (w->d_flags) cudaFree(w->d_flags);
    w->d_flags = nullptr;
    cudaError_t e = cudaMalloc(&w->d_flags, sizeof(unsigned long long) * check_every);
    if (e != cudaSuccess) { w->flags_cap = 0; return cuda_status(e); }
    w->flags_cap = check_every;
  }
  BfsArgs a = w->args;
  a.source = source;
  // the vertex set does not change during the search, so one enumeration
  // serves every level; check_every levels run per cooperative launch
  // (parallel_do_and_reduce with OR per level, a grid barrier between)
  int st = w->snap.take(w->heap, w->cls, s);
  if (!st) st = launch_do_all_view<VertexReset>(w->heap, w->cls, &a, s, &w->snap.view);
  std::vector<unsigned long long> hf((size_t)check_every);
  for (int32_t base = 0; !st; base += check_every) {
    if (base > (int32_t)w->n0) return SMMO_E_TIMEOUT;  // more levels than vertices: impossible
    st = launch_levels<VertexVisit, false>(w->heap, w->snap.view, w->cls, a, base, check_every, w->d_flags,
                                           w->d_arrive, s);
    if (st) break;
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(hf.data(), w->d_flags, sizeof(unsigned long long) * check_every,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &w->heap->view.st->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (err) return err;  // a barrier gave up
    for (int k = 0; k < check_every; ++k)
      if (hf[(size_t)k] == 0) {  // level base + k found nothing new
        if (levels) *levels = base + k + 1;
        return SMMO_OK;
      }
  }
  return st;
}

int smmo_bfs_export(smmo_bfs* w, int32_t* dist, void* stream) {
  if (!w || !dist) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  BfsArgs a = w->args;
  a.out = dist;
  int st = enumerate(w->heap, w->cls, s);
  if (!st) st = launch_do_all<VertexExport>(w->heap, w->cls, &a, s);
  if (!st) { cudaError_t e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  return st;
}

int smmo_bfs_destroy(smmo_bfs* w) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (w->d_flags) cudaFree(w->d_flags);
  if (w->d_arrive) cudaFree(w->d_arrive);
  w->snap.release();
  delete w;
  return SMMO_OK;
}

}  // extern "C"
