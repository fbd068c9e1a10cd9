// wl_structure.cu -- a spring mesh that cracks under load (the thesis'
// finite-element application "structure", Sec. 7.4) as an SMMO application.
//
// Classes: NodeBase (abstract) {x, y, springs[3], num_springs, distance,
// id}; AnchorNode (fixed); AnchorPullNode {vx, vy} (moves with a constant
// velocity); Node {vx, vy, m}; Spring {p1, p2, k, L0, fmax, fx, fy, flag,
// id}.  The spring array is an inner array inlined into the SOA block (one
// column per entry).  One iteration:
//   pull      AnchorPullNode::pull: x += v dt;
//   compute   `substeps` times
//               Spring::compute_force: d = p2 - p1, len = |d|,
//                 F = k (len - L0) when len > L0 else 0; F > fmax breaks the
//                 spring: it leaves both endpoints' arrays (a node whose
//                 count drops to zero is deleted: the thread whose atomic
//                 decrement took the last spring deletes it) and deletes
//                 itself; otherwise it keeps the force on p1, F (d / len);
//               Node::update: the sum of its springs' forces in slot order
//                 (+f as p1, -f as p2), v = (v + F/m dt) (1 - damping),
//                 x += v dt;
//   remove    distance 0 at AnchorNodes, infinity elsewhere; BFS level l
//             is parallel_do_and_reduce of NodeBase::visit(l) (OR of "was
//             in the frontier") over all node classes, the levels of a
//             search run in one cooperative launch (levels.cuh) over one
//             snapshot of the node classes; NodeBase::delete_node flags the
//             springs of unreached nodes; Spring::delete_spring removes the
//             flagged springs from their endpoints and deletes them.
// The compute phase, which deletes but never creates, runs over one
// snapshot per class per iteration; its methods skip objects deleted since.
// FP32 with round-to-nearest intrinsics in the order above: results equal
// the CPU oracle bit for bit.  A node is deleted only after every spring
// that names it is gone, so no thread reads a deleted node.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "heap_internal.h"
#include "levels.cuh"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

enum { N_X = 0, N_Y = 1, N_SPR = 2, N_NSPR = 5, N_DIST = 6, N_ID = 7, N_VX = 8, N_VY = 9, N_M = 10 };
enum { S_P1 = 0, S_P2 = 1, S_K = 2, S_L0 = 3, S_FMAX = 4, S_FX = 5, S_FY = 6, S_FLAG = 7, S_ID = 8 };
constexpr int32_t kInf = 0x7FFFFFFF;
// device counters of the workload
enum { CTR_BROKEN = 0, CTR_NODES_DELETED = 1, CTR_SPRINGS_REMOVED = 2, CTR_N = 4 };

struct StructArgs {
  uint32_t anchor_cls, pull_cls, node_cls, spring_cls;
  float dt, keep;          // keep = 1 - damping
  int32_t frontier;        // BFS level
  unsigned long long* ctr; // CTR_N counters
  // export (by id; nullable)
  uint8_t* o_nalive;
  float *o_x, *o_y, *o_vx, *o_vy;
  int32_t *o_nspr, *o_dist, *o_slot;
  uint8_t* o_salive;
  float *o_fx, *o_fy;
  uint32_t n0, s0;
  const uint32_t* handles;  // creation: node id -> handle
  // byte offsets of the NodeBase columns when every node class has them at
  // the same place (equal capacities), else base_uniform = 0
  int32_t base_uniform;
  uint32_t base_off[N_ID + 1];
};

__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }

template <class T>
__device__ __forceinline__ T* F(const HeapView& h, uint32_t cls, uint32_t self, int col) {
  return field_ptr<T>(h, __ldg(&h.cls[cls].col_off[col]), self);
}

// A NodeBase column of a node whose class is not known: without the type
// id when every node class keeps the column at the same offset.
template <class T>
__device__ __forceinline__ T* NB(const HeapView& h, const StructArgs& a, uint32_t v, int col) {
  return a.base_uniform ? field_ptr<T>(h, a.base_off[col], v) : F<T>(h, type_of(h, v), v, col);
}

// Spring s leaves node v's array; the node is deleted when it held only s.
__device__ __forceinline__ void unlink_end(const HeapView& h, const StructArgs& a, uint32_t v, uint32_t s) {
  for (int i = 0; i < 3; ++i) {
    uint32_t* sl = NB<uint32_t>(h, a, v, N_SPR + i);
    if (*sl == s) {
      *sl = kNull;
      if (atomicSub(NB<int32_t>(h, a, v, N_NSPR), 1) == 1) {
        smmo_delete(h, v);
        atomicAdd(&a.ctr[CTR_NODES_DELETED], 1ull);
      }
      return;
    }
  }
  set_error(h, SMMO_E_BAD_HANDLE, s);  // the node does not hold the spring
}

__device__ __forceinline__ void remove_spring(const HeapView& h, const StructArgs& a, uint32_t c, uint32_t self) {
  unlink_end(h, a, *F<uint32_t>(h, c, self, S_P1), self);
  unlink_end(h, a, *F<uint32_t>(h, c, self, S_P2), self);
  smmo_delete(h, self);
}

struct PullMove {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    float* x = F<float>(h, c, self, N_X);
    float* y = F<float>(h, c, self, N_Y);
    *x = fa(*x, fm(*F<float>(h, c, self, N_VX), a.dt));
    *y = fa(*y, fm(*F<float>(h, c, self, N_VY), a.dt));
  }
};

// The compute phase runs over one snapshot per class per iteration (no
// object is created during it): an object deleted since the snapshot (a
// broken spring, a node left without springs) is skipped by this test.  A
// block whose last object was freed keeps an all-ones slot bitmap (it is
// invalidated) but has left the class's allocated bitmap, hence both tests;
// every deletion it could see finished in an earlier do-all (a spring
// deletes only itself, nodes are deleted in the spring pass).
__device__ __forceinline__ bool still_allocated(const HeapView& h, uint32_t c, uint32_t self) {
  return bm_get(h, bm_alloc(h, c), self >> 6) && ((ld_cg(h.alloc_bm + (self >> 6)) >> (self & 63)) & 1);
}

struct SpringForce {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (!still_allocated(h, c, self)) return;
    const uint32_t p1 = *F<uint32_t>(h, c, self, S_P1), p2 = *F<uint32_t>(h, c, self, S_P2);
    const float dx = fs(*NB<float>(h, a, p2, N_X), *NB<float>(h, a, p1, N_X));
    const float dy = fs(*NB<float>(h, a, p2, N_Y), *NB<float>(h, a, p1, N_Y));
    const float len = __fsqrt_rn(fa(fm(dx, dx), fm(dy, dy)));
    const float stretch = fs(len, *F<float>(h, c, self, S_L0));
    const float f = stretch > 0.0f ? fm(*F<float>(h, c, self, S_K), stretch) : 0.0f;
    if (f > *F<float>(h, c, self, S_FMAX)) {
      atomicAdd(&a.ctr[CTR_BROKEN], 1ull);
      remove_spring(h, a, c, self);
      return;
    }
    float fx = 0.0f, fy = 0.0f;
    if (f > 0.0f) {
      fx = fm(f, __fdiv_rn(dx, len));
      fy = fm(f, __fdiv_rn(dy, len));
    }
    *F<float>(h, c, self, S_FX) = fx;
    *F<float>(h, c, self, S_FY) = fy;
  }
};

struct NodeMove {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (!still_allocated(h, c, self)) return;
    float sx = 0.0f, sy = 0.0f;
    for (int i = 0; i < 3; ++i) {
      const uint32_t s = *F<uint32_t>(h, c, self, N_SPR + i);
      if (s == kNull) continue;
      const float fx = *F<float>(h, a.spring_cls, s, S_FX), fy = *F<float>(h, a.spring_cls, s, S_FY);
      if (*F<uint32_t>(h, a.spring_cls, s, S_P1) == self) {
        sx = fa(sx, fx);
        sy = fa(sy, fy);
      } else {
        sx = fs(sx, fx);
        sy = fs(sy, fy);
      }
    }
    const float m = *F<float>(h, c, self, N_M);
    float* vx = F<float>(h, c, self, N_VX);
    float* vy = F<float>(h, c, self, N_VY);
    const float nvx = fm(fa(*vx, fm(__fdiv_rn(sx, m), a.dt)), a.keep);
    const float nvy = fm(fa(*vy, fm(__fdiv_rn(sy, m), a.dt)), a.keep);
    *vx = nvx;
    *vy = nvy;
    float* x = F<float>(h, c, self, N_X);
    float* y = F<float>(h, c, self, N_Y);
    *x = fa(*x, fm(nvx, a.dt));
    *y = fa(*y, fm(nvy, a.dt));
  }
};

// ------------------------------------------------------------- BFS removal
struct NodeInitFrontier {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    *F<int32_t>(h, c, self, N_DIST) = c == a.anchor_cls ? 0 : kInf;
  }
};

// NodeBase::visit(frontier), reducing with OR: 1 iff the node is in the
// frontier (the thesis' continue flag).  The few frontier nodes of a level
// are its critical path, so each stage's loads are issued for all three
// springs before the next stage (slots, endpoints, neighbour classes,
// distances), and the stores come last.  Distances, which other CTAs write
// between levels of one launch, are read through L2.
struct NodeVisit {
  using Args = StructArgs;
  __device__ static bool active(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    return __ldcg(F<int32_t>(h, c, self, N_DIST)) == a.frontier;
  }
  __device__ static long long run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (!active(h, a, c, self)) return 0;
    uint32_t s[3], u[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = *F<uint32_t>(h, c, self, N_SPR + i);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      u[i] = kNull;
      if (s[i] == kNull) continue;
      const uint32_t p1 = *F<uint32_t>(h, a.spring_cls, s[i], S_P1), p2 = *F<uint32_t>(h, a.spring_cls, s[i], S_P2);
      u[i] = p1 == self ? p2 : p1;
    }
    int32_t* d[3];
    int32_t dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = u[i] == kNull ? nullptr : NB<int32_t>(h, a, u[i], N_DIST);
#pragma unroll
    for (int i = 0; i < 3; ++i) dv[i] = d[i] ? __ldcg(d[i]) : 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (d[i] && dv[i] == kInf) *d[i] = a.frontier + 1;
    return 1;
  }
};

struct NodeFlagSprings {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (*F<int32_t>(h, c, self, N_DIST) != kInf) return;
    for (int i = 0; i < 3; ++i) {
      const uint32_t s = *F<uint32_t>(h, c, self, N_SPR + i);
      if (s != kNull) *F<uint8_t>(h, a.spring_cls, s, S_FLAG) = 1;
    }
  }
};

struct SpringDelete {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (!*F<uint8_t>(h, c, self, S_FLAG)) return;
    atomicAdd(&a.ctr[CTR_SPRINGS_REMOVED], 1ull);
    remove_spring(h, a, c, self);
  }
};

// ------------------------------------------------------- creation, export
// spring endpoints and node arrays hold ids after creation: replace them by
// handles (node ids through the handle table; spring ids through the
// springs' own table, passed in `handles` + n0)
struct SpringLink {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    for (int e = S_P1; e <= S_P2; ++e) {
      uint32_t* p = F<uint32_t>(h, c, self, e);
      const uint32_t id = *p;
      if (id >= a.n0) { set_error(h, SMMO_E_BOUNDS, self); *p = kNull; continue; }
      *p = a.handles[id];
    }
  }
};

struct NodeLink {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    for (int i = 0; i < 3; ++i) {
      uint32_t* p = F<uint32_t>(h, c, self, N_SPR + i);
      const uint32_t id = *p;
      if (id == kNull) continue;
      if (id >= a.s0) { set_error(h, SMMO_E_BOUNDS, self); *p = kNull; continue; }
      *p = a.handles[a.n0 + id];
    }
  }
};

struct NodeExport {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t id = *F<int32_t>(h, c, self, N_ID);
    if (id < 0 || (uint32_t)id >= a.n0) { set_error(h, SMMO_E_BOUNDS, self); return; }
    if (a.o_nalive) a.o_nalive[id] = 1;
    if (a.o_x) a.o_x[id] = *F<float>(h, c, self, N_X);
    if (a.o_y) a.o_y[id] = *F<float>(h, c, self, N_Y);
    const bool moving = c != a.anchor_cls;
    if (a.o_vx) a.o_vx[id] = moving ? *F<float>(h, c, self, N_VX) : 0.0f;
    if (a.o_vy) a.o_vy[id] = moving ? *F<float>(h, c, self, N_VY) : 0.0f;
    if (a.o_nspr) a.o_nspr[id] = *F<int32_t>(h, c, self, N_NSPR);
    if (a.o_dist) a.o_dist[id] = *F<int32_t>(h, c, self, N_DIST);
    if (a.o_slot)
      for (int i = 0; i < 3; ++i) {
        const uint32_t s = *F<uint32_t>(h, c, self, N_SPR + i);
        a.o_slot[3 * (size_t)id + i] = s == kNull ? -1 : *F<int32_t>(h, a.spring_cls, s, S_ID);
      }
  }
};

struct SpringExport {
  using Args = StructArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t id = *F<int32_t>(h, c, self, S_ID);
    if (id < 0 || (uint32_t)id >= a.s0) { set_error(h, SMMO_E_BOUNDS, self); return; }
    if (a.o_salive) a.o_salive[id] = 1;
    if (a.o_fx) a.o_fx[id] = *F<float>(h, c, self, S_FX);
    if (a.o_fy) a.o_fy[id] = *F<float>(h, c, self, S_FY);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_structure[] = {
    SMMO_METHOD("structure.pull", PullMove),
    SMMO_METHOD("structure.spring_compute_force", SpringForce),
    SMMO_METHOD("structure.node_update", NodeMove),
    SMMO_METHOD("structure.node_init_frontier", NodeInitFrontier),
    SMMO_METHOD_REDUCE("structure.node_visit", NodeVisit),
    SMMO_METHOD("structure.node_delete", NodeFlagSprings),
    SMMO_METHOD("structure.spring_delete", SpringDelete),
    SMMO_METHOD("structure.node_export", NodeExport),
    SMMO_METHOD("structure.spring_export", SpringExport)};
const int g_methods_structure_n = sizeof(g_methods_structure) / sizeof(g_methods_structure[0]);

struct smmo_structure {
  smmo_heap* heap = nullptr;
  int cls_base = -1, cls_anchor = -1, cls_pull = -1, cls_node = -1, cls_spring = -1;
  uint32_t n0 = 0, s0 = 0;
  int32_t substeps = 0, check_every = 16;
  StructArgs args{};
  unsigned long long* d_ctr = nullptr;  // CTR_N counters
  unsigned long long* d_flags = nullptr;  // one OR result per level of a launch
  unsigned long long* d_arrive = nullptr;  // level barrier words
  int flags_cap = 0;
  smmo::Snapshot nodes;                 // all node classes (one POLY snapshot)
  smmo::Snapshot springs, free_nodes;   // the compute phase's snapshots
  int64_t bfs_levels = 0;               // levels run (statistics)
  int64_t bfs_launches = 0;
};

namespace {
int sync_status(cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SMMO_OK : cuda_status(e);
}

int pdo(smmo_structure* w, int cls, method_launch_fn fn, const StructArgs& a, cudaStream_t s) {
  int st = enumerate(w->heap, cls, s);
  if (!st) st = fn(w->heap, cls, &a, s);
  return st;
}

// the removal phase: BFS levels, check_every per cooperative launch, over
// one snapshot of all node classes (no node is created or deleted during
// the search), then flags and deletions
int remove_disconnected(smmo_structure* w, cudaStream_t s) {
  StructArgs a = w->args;
  smmo_heap* h = w->heap;
  int st = w->nodes.take_subtree(h, w->cls_base, s);
  if (!st) st = launch_do_all_view<NodeInitFrontier, true>(h, w->cls_base, &a, s, &w->nodes.view);
  if (st) return st;
  const int ce = w->check_every;
  if (w->flags_cap < ce) {
    if (w->d_flags) cudaFree(w->d_flags);
    w->d_flags = nullptr;
    cudaError_t e = cudaMalloc(&w->d_flags, sizeof(unsigned long long) * ce);
    if (e != cudaSuccess) { w->flags_cap = 0; return cuda_status(e); }
    w->flags_cap = ce;
  }
  std::vector<unsigned long long> hf((size_t)ce);
  bool done = false;
  for (int32_t base = 0; !done; base += ce) {
    if (base > (int32_t)w->n0 + 1) return SMMO_E_TIMEOUT;  // more levels than nodes: impossible
    st = launch_levels<NodeVisit, true>(h, w->nodes.view, w->cls_base, a, base, ce, w->d_flags, w->d_arrive, s);
    ++w->bfs_launches;
    if (st) return st;
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(hf.data(), w->d_flags, sizeof(unsigned long long) * ce, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &h->view.st->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (err) return err;  // a barrier gave up (left for smmo_heap_sync to report too)
    for (int k = 0; k < ce; ++k)
      if (hf[(size_t)k] == 0) {  // level base + k had no frontier: the search is over
        w->bfs_levels += base + k + 1;
        done = true;
        break;
      }
  }
  st = launch_do_all_view<NodeFlagSprings, true>(h, w->cls_base, &a, s, &w->nodes.view);
  if (!st) st = pdo(w, w->cls_spring, &launch_do_all<SpringDelete>, a, s);
  return st;
}
}  // namespace

extern "C" {

int smmo_structure_create(smmo_heap* heap, int64_t n, const int8_t* kind, const float* const* node_cols,
                          const int32_t* slot, int64_t ns, const int32_t* p1, const int32_t* p2,
                          const float* const* spring_cols, const smmo_structure_params* p, void* stream,
                          smmo_structure** out) {
  if (!heap || n < 1 || n >= (1ll << 31) || ns < 0 || ns >= (1ll << 31) || !kind || !node_cols || !slot || !p ||
      !out || (ns > 0 && (!p1 || !p2 || !spring_cols)) || p->substeps < 0 || p->bfs_check_every < 1 ||
      p->bfs_check_every > 4096)
    return SMMO_E_INVALID_ARG;
  for (int k = 0; k < 5; ++k)
    if (!node_cols[k]) return SMMO_E_INVALID_ARG;
  for (int k = 0; ns > 0 && k < 3; ++k)
    if (!spring_cols[k]) return SMMO_E_INVALID_ARG;
  if (!heap->classes.empty() || heap->frozen) return SMMO_E_FROZEN;
  // host checks: kinds, endpoints, and slots that list exactly the springs
  // naming the node
  std::vector<int32_t> held((size_t)n, 0);
  for (int64_t v = 0; v < n; ++v)
    if (kind[v] < SMMO_STRUCT_ANCHOR || kind[v] > SMMO_STRUCT_NODE) return SMMO_E_INVALID_ARG;
  for (int64_t s = 0; s < ns; ++s) {
    if (p1[s] < 0 || p1[s] >= n || p2[s] < 0 || p2[s] >= n || p1[s] == p2[s]) return SMMO_E_INVALID_ARG;
    ++held[(size_t)p1[s]];
    ++held[(size_t)p2[s]];
  }
  std::vector<int32_t> nspr((size_t)n, 0);
  for (int64_t v = 0; v < n; ++v) {
    for (int i = 0; i < 3; ++i) {
      const int32_t s = slot[3 * v + i];
      if (s == -1) continue;
      if (s < 0 || s >= ns || (p1[s] != v && p2[s] != v)) return SMMO_E_INVALID_ARG;
      for (int j = 0; j < i; ++j)
        if (slot[3 * v + j] == s) return SMMO_E_INVALID_ARG;
      ++nspr[(size_t)v];
    }
    if (nspr[(size_t)v] != held[(size_t)v]) return SMMO_E_INVALID_ARG;
  }
  cudaStream_t st_ = (cudaStream_t)stream;
  smmo_structure* w = new smmo_structure();
  w->heap = heap;
  w->n0 = (uint32_t)n;
  w->s0 = (uint32_t)ns;
  w->substeps = p->substeps;
  w->check_every = p->bfs_check_every;
  // classes: NodeBase's springs refer to Spring (registered last, id base + 4)
  smmo_field_desc nb[6] = {{"x", SMMO_F32, 1, -1},           {"y", SMMO_F32, 1, -1},
                           {"springs", SMMO_HANDLE, 3, -1},  {"num_springs", SMMO_I32, 1, -1},
                           {"distance", SMMO_I32, 1, -1},    {"id", SMMO_I32, 1, -1}};
  const int base_id = (int)heap->classes.size();
  nb[2].ref_class = base_id + 4;
  smmo_field_desc pf[2] = {{"vx", SMMO_F32, 1, -1}, {"vy", SMMO_F32, 1, -1}};
  smmo_field_desc nf[3] = {{"vx", SMMO_F32, 1, -1}, {"vy", SMMO_F32, 1, -1}, {"m", SMMO_F32, 1, -1}};
  smmo_field_desc sf[9] = {{"p1", SMMO_HANDLE, 1, base_id}, {"p2", SMMO_HANDLE, 1, base_id},
                           {"k", SMMO_F32, 1, -1},          {"L0", SMMO_F32, 1, -1},
                           {"fmax", SMMO_F32, 1, -1},       {"fx", SMMO_F32, 1, -1},
                           {"fy", SMMO_F32, 1, -1},         {"flag", SMMO_U8, 1, -1},
                           {"id", SMMO_I32, 1, -1}};
  int st = smmo_class_register(heap, "NodeBase", nb, 6, -1, 1, &w->cls_base);
  if (!st) st = smmo_class_register(heap, "AnchorNode", nullptr, 0, w->cls_base, 0, &w->cls_anchor);
  if (!st) st = smmo_class_register(heap, "AnchorPullNode", pf, 2, w->cls_base, 0, &w->cls_pull);
  if (!st) st = smmo_class_register(heap, "Node", nf, 3, w->cls_base, 0, &w->cls_node);
  if (!st) st = smmo_class_register(heap, "Spring", sf, 9, -1, 0, &w->cls_spring);
  if (!st && w->cls_spring != base_id + 4) st = SMMO_E_INVALID_ARG;
  // 64 slots of the largest class (Node: eleven 4-byte columns)
  if (heap->cfg.block_data_bytes == 0) heap->cfg.block_data_bytes = 64 * 44;
  if (!st) st = freeze(heap, st_);
  if (st) { delete w; return st; }
  StructArgs& a = w->args;
  memset(&a, 0, sizeof(a));
  a.anchor_cls = (uint32_t)w->cls_anchor;
  a.pull_cls = (uint32_t)w->cls_pull;
  a.node_cls = (uint32_t)w->cls_node;
  a.spring_cls = (uint32_t)w->cls_spring;
  a.dt = p->dt;
  a.keep = 1.0f - p->damping;
  a.n0 = (uint32_t)n;
  a.s0 = (uint32_t)ns;
  {
    const ClassLayout& L0 = heap->classes[w->cls_anchor].layout;
    a.base_uniform = 1;
    for (int cls : {w->cls_pull, w->cls_node})
      for (int k = 0; k <= N_ID; ++k)
        if (heap->classes[cls].layout.col_off[k] != L0.col_off[k]) a.base_uniform = 0;
    for (int k = 0; k <= N_ID; ++k) a.base_off[k] = L0.col_off[k];
  }
  cudaError_t e = cudaMalloc(&w->d_ctr, sizeof(unsigned long long) * CTR_N);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_ctr, 0, sizeof(unsigned long long) * CTR_N, st_);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_arrive, sizeof(unsigned long long) * kBarrierWords);
  if (e != cudaSuccess) { smmo_structure_destroy(w); return cuda_status(e); }
  a.ctr = w->d_ctr;
  // handle table: nodes by id, then springs by id
  uint32_t* handles = nullptr;
  e = cudaMallocAsync(&handles, sizeof(uint32_t) * (size_t)(n + ns + 1), st_);
  if (e != cudaSuccess) { smmo_structure_destroy(w); return cuda_status(e); }
  std::vector<void*> dev;
  auto upload = [&](const void* src, size_t bytes) -> void* {
    void* d = nullptr;
    if (e != cudaSuccess) return nullptr;
    e = cudaMallocAsync(&d, bytes ? bytes : 4, st_);
    if (e == cudaSuccess) { dev.push_back(d); if (bytes) e = cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st_); }
    return d;
  };
  // nodes: one bulk_new per kind, columns gathered on the host
  std::vector<uint32_t> table((size_t)n, kNull);
  for (int kk = SMMO_STRUCT_ANCHOR; kk <= SMMO_STRUCT_NODE && !st && e == cudaSuccess; ++kk) {
    std::vector<int64_t> ids;
    for (int64_t v = 0; v < n; ++v)
      if (kind[v] == kk) ids.push_back(v);
    if (ids.empty()) continue;
    const size_t m = ids.size();
    std::vector<float> col[5];
    std::vector<uint32_t> sl[3];
    std::vector<int32_t> cnt(m), dist(m, kInf), id32(m);
    for (int k = 0; k < 5; ++k) col[k].resize(m);
    for (int i = 0; i < 3; ++i) sl[i].resize(m);
    for (size_t j = 0; j < m; ++j) {
      const int64_t v = ids[j];
      for (int k = 0; k < 5; ++k) col[k][j] = node_cols[k][v];
      for (int i = 0; i < 3; ++i) sl[i][j] = slot[3 * v + i] < 0 ? kNull : (uint32_t)slot[3 * v + i];
      cnt[j] = nspr[(size_t)v];
      id32[j] = (int32_t)v;
    }
    std::vector<const void*> src = {upload(col[0].data(), m * 4), upload(col[1].data(), m * 4),
                                    upload(sl[0].data(), m * 4),  upload(sl[1].data(), m * 4),
                                    upload(sl[2].data(), m * 4),  upload(cnt.data(), m * 4),
                                    upload(dist.data(), m * 4),   upload(id32.data(), m * 4)};
    int cls = w->cls_anchor;
    if (kk == SMMO_STRUCT_PULL) {
      cls = w->cls_pull;
      src.push_back(upload(col[2].data(), m * 4));
      src.push_back(upload(col[3].data(), m * 4));
    } else if (kk == SMMO_STRUCT_NODE) {
      cls = w->cls_node;
      src.push_back(upload(col[2].data(), m * 4));
      src.push_back(upload(col[3].data(), m * 4));
      src.push_back(upload(col[4].data(), m * 4));
    }
    uint32_t* h_out = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&h_out, m * 4, st_);
    if (e == cudaSuccess) dev.push_back(h_out);
    if (e == cudaSuccess) st = smmo_bulk_new(heap, cls, (int64_t)m, src.data(), h_out, nullptr, stream);
    // the new handles, by node id, into the host copy of the table
    std::vector<uint32_t> hh(m);
    if (!st && e == cudaSuccess) e = cudaMemcpyAsync(hh.data(), h_out, m * 4, cudaMemcpyDeviceToHost, st_);
    if (!st && e == cudaSuccess) e = cudaStreamSynchronize(st_);
    for (size_t j = 0; !st && e == cudaSuccess && j < m; ++j) table[(size_t)ids[j]] = hh[j];
  }
  // springs
  if (!st && e == cudaSuccess && ns > 0) {
    const size_t m = (size_t)ns;
    std::vector<int32_t> id32(m);
    std::vector<float> zf(m, 0.0f);
    std::vector<uint8_t> zb(m, 0);
    for (size_t j = 0; j < m; ++j) id32[j] = (int32_t)j;
    const void* src[9] = {upload(p1, m * 4),           upload(p2, m * 4),           upload(spring_cols[0], m * 4),
                          upload(spring_cols[1], m * 4), upload(spring_cols[2], m * 4), upload(zf.data(), m * 4),
                          upload(zf.data(), m * 4),     upload(zb.data(), m),        upload(id32.data(), m * 4)};
    if (e == cudaSuccess) st = smmo_bulk_new(heap, w->cls_spring, ns, src, handles + n, nullptr, stream);
  }
  // node handles by id into the device table
  if (!st && e == cudaSuccess) e = cudaMemcpyAsync(handles, table.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st_);
  if (!st && e == cudaSuccess) {
    a.handles = handles;
    if (ns > 0) st = pdo(w, w->cls_spring, &launch_do_all<SpringLink>, a, st_);
    for (int cls : {w->cls_anchor, w->cls_pull, w->cls_node})
      if (!st) st = pdo(w, cls, &launch_do_all<NodeLink>, a, st_);
    a.handles = nullptr;
  }
  if (!st && e == cudaSuccess) st = sync_status(st_);
  for (void* d : dev) cudaFreeAsync(d, st_);
  cudaFreeAsync(handles, st_);
  if (e != cudaSuccess && !st) st = cuda_status(e);
  if (!st) st = sync_status(st_);
  if (st) { smmo_structure_destroy(w); return st; }
  *out = w;
  return SMMO_OK;
}

int smmo_structure_step(smmo_structure* w, int iterations, int phases, void* stream) {
  if (!w || iterations < 0 || phases < 0 || phases > 7) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const StructArgs& a = w->args;
  for (int it = 0; it < iterations; ++it) {
    int st = SMMO_OK;
    if (phases & SMMO_STRUCT_PHASE_PULL) st = pdo(w, w->cls_pull, &launch_do_all<PullMove>, a, s);
    if ((phases & SMMO_STRUCT_PHASE_COMPUTE) && w->substeps > 0 && !st) {
      // one snapshot of each class for all compute steps: breaks only
      // delete, and the methods skip what was deleted since
      st = w->springs.take(w->heap, w->cls_spring, s);
      if (!st) st = w->free_nodes.take(w->heap, w->cls_node, s);
      for (int k = 0; k < w->substeps && !st; ++k) {
        st = launch_do_all_view<SpringForce>(w->heap, w->cls_spring, &a, s, &w->springs.view);
        if (!st) st = launch_do_all_view<NodeMove>(w->heap, w->cls_node, &a, s, &w->free_nodes.view);
      }
    }
    if (!st && (phases & SMMO_STRUCT_PHASE_REMOVE)) st = remove_disconnected(w, s);
    if (st) return st;
  }
  return SMMO_OK;
}

int smmo_structure_export(smmo_structure* w, const smmo_structure_out* o, void* stream) {
  if (!w || !o) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (o->node_alive) e = cudaMemsetAsync(o->node_alive, 0, w->n0, s);
  if (e == cudaSuccess && o->spring_alive && w->s0) e = cudaMemsetAsync(o->spring_alive, 0, w->s0, s);
  if (e != cudaSuccess) return cuda_status(e);
  StructArgs a = w->args;
  a.o_nalive = o->node_alive;
  a.o_x = o->x;
  a.o_y = o->y;
  a.o_vx = o->vx;
  a.o_vy = o->vy;
  a.o_nspr = o->num_springs;
  a.o_dist = o->distance;
  a.o_slot = o->slot;
  a.o_salive = o->spring_alive;
  a.o_fx = o->fx;
  a.o_fy = o->fy;
  int st = SMMO_OK;
  for (int cls : {w->cls_anchor, w->cls_pull, w->cls_node})
    if (!st) st = pdo(w, cls, &launch_do_all<NodeExport>, a, s);
  if (!st) st = pdo(w, w->cls_spring, &launch_do_all<SpringExport>, a, s);
  if (!st) st = sync_status(s);
  return st;
}

int smmo_structure_info(smmo_structure* w, int* class_ids, int64_t* counters, void* stream) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (class_ids) {
    class_ids[0] = w->cls_base;
    class_ids[1] = w->cls_anchor;
    class_ids[2] = w->cls_pull;
    class_ids[3] = w->cls_node;
    class_ids[4] = w->cls_spring;
  }
  if (counters) {
    unsigned long long c[CTR_N];
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(c, w->d_ctr, sizeof(c), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    counters[0] = (int64_t)c[CTR_BROKEN];
    counters[1] = (int64_t)c[CTR_NODES_DELETED];
    counters[2] = (int64_t)c[CTR_SPRINGS_REMOVED];
    counters[3] = w->bfs_levels;
    counters[4] = w->bfs_launches;
  }
  return SMMO_OK;
}

int smmo_structure_destroy(smmo_structure* w) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (w->d_ctr) cudaFree(w->d_ctr);
  if (w->d_flags) cudaFree(w->d_flags);
  if (w->d_arrive) cudaFree(w->d_arrive);
  w->nodes.release();
  w->springs.release();
  w->free_nodes.release();
  delete w;
  return SMMO_OK;
}

}  // extern "C"
