// wl_bh.cu -- 2-D Barnes-Hut with a dynamic quad tree as an SMMO application
// (thesis Sec. 7.3).
//
// Classes: NodeBase (abstract) {parent, child_idx, px, py, m}; BodyNode
// {vx, vy, ax, ay, id}; TreeNode {children[4], p1x, p1y, w, frontier, done}.
// A tree node covers the square [p1x, p1x + w) x [p1y, p1y + w) of the unit
// square and splits it into quadrants (x >= mid_x) + 2 (y >= mid_y); a
// child slot holds null, a BodyNode or a TreeNode.  One step:
//   summaries   bottom-up traversal over TreeNodes (a node is processed
//               once all its TreeNode children are done; walks up the tree,
//               see TreePending): mass and centre of gravity from the
//               children in child order;
//   force       per body, preorder depth-first traversal from the root with
//               an explicit stack: a tree node is opened if the body lies in
//               its square or w^2 >= theta^2 d^2, else its summary acts;
//   update      v += G a dt, x += v dt, reflection at the walls;
//   remove      a body that left its parent's quadrant clears its slot;
//   insert      bodies without parent descend from the root and claim an
//               empty slot with compare-and-swap; a slot holding a body is
//               replaced by a new TreeNode (device new) holding that body,
//               installed with compare-and-swap (losers delete theirs);
//   collapse    bottom-up traversal: a tree node with no child is deleted,
//               one with a single body child is replaced by that body.
// After the collapse the tree is the region quad tree of the positions, so
// results are independent of thread timing.  FP32 arithmetic follows a
// fixed order (see the oracle's description) with round-to-nearest
// intrinsics; every retry and wait loop is bounded and records an error.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "fp32_rn.cuh"
#include "heap_internal.h"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

// column indices (NodeBase columns first in both subclasses)
enum { C_PARENT = 0, C_CIDX = 1, C_PX = 2, C_PY = 3, C_M = 4 };
enum { B_VX = 5, B_VY = 6, B_AX = 7, B_AY = 8, B_ID = 9 };
enum { T_CH = 5, T_P1X = 9, T_P1Y = 10, T_W = 11, T_FRONT = 12, T_DONE = 13 };

constexpr int kMaxDepth = 60;      // squares down to 2^-60
// error details: the handle, tagged with the place that gave up
constexpr unsigned long long kTagWaitParent = 1ull << 40, kTagBudget = 2ull << 40, kTagDepth = 3ull << 40,
                             kTagStack = 4ull << 40;
constexpr int kStack = 3 * kMaxDepth + 4;
constexpr int kInsertBudget = 1 << 14;

struct BHArgs {
  uint32_t body_cls, tree_cls;
  uint32_t root;
  float G, eps2, dt, theta2;
  int32_t fast;   // branch-free sqrt / reciprocal valid for this eps
  float* out;     // export: 5 x n0 floats by id
  uint32_t n0;
};

__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }

template <class T>
__device__ __forceinline__ T* F(const HeapView& h, uint32_t cls, uint32_t self, int col) {
  return field_ptr<T>(h, __ldg(&h.cls[cls].col_off[col]), self);
}

// field read through L2: nodes created or relinked in the current kernel
template <class T>
__device__ __forceinline__ T Lcg(const HeapView& h, uint32_t cls, uint32_t self, int col) {
  return __ldcg(F<T>(h, cls, self, col));
}

__device__ __forceinline__ int quadrant(float p1x, float p1y, float w, float x, float y) {
  const float hw = fm(w, 0.5f);
  return (x >= fa(p1x, hw) ? 1 : 0) + (y >= fa(p1y, hw) ? 2 : 0);
}

template <bool FAST>
__device__ __forceinline__ void pair_acc(float xi, float yi, float xj, float yj, float mj, float eps2, float& ax,
                                         float& ay) {
  const float dx = fs(xj, xi), dy = fs(yj, yi);
  const float s2 = fa(fa(fm(dx, dx), fm(dy, dy)), eps2);
  const float inv = FAST ? rcp_rn_fast(fm(s2, sqrt_rn_fast(s2))) : __fdiv_rn(1.0f, fm(s2, __fsqrt_rn(s2)));
  const float f = fm(mj, inv);
  ax = fa(ax, fm(f, dx));
  ay = fa(ay, fm(f, dy));
}

// ---------------------------------------------------------------- traversal
// Bottom-up traversals (summaries, collapse) as walks up the tree instead of
// one launch per level: TreePending stores per tree node the number of its
// children that are tree nodes (in the frontier byte) and marks the nodes
// without any (done = 2) as the starts; the walk do-all processes each start
// node, then counts down its parent's pending children, and the thread that
// brings a parent to zero processes the parent and goes on up.  A node is
// therefore processed once, after all its tree-node children, exactly as in
// a level-by-level frontier traversal (Sec. 7.3), and computes the same
// values from its children in child order.  Values written by other threads
// in the same launch are read through L2, after the fence that follows the
// count-down.  The walks wait for nobody.
struct TreePending {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint8_t pending = 0;
    for (int i = 0; i < 4; ++i) {
      const uint32_t ch = *F<uint32_t>(h, c, self, T_CH + i);
      if (ch != kNull && type_of(h, ch) == a.tree_cls) ++pending;
    }
    *F<uint8_t>(h, c, self, T_FRONT) = pending;
    *F<uint8_t>(h, c, self, T_DONE) = pending == 0 ? 2 : 0;
  }
};

// Counts down the pending tree-node children of p (its frontier byte, with
// an atomic on the byte's 32-bit word: the column starts on a 64-byte
// boundary, and a count never goes below 0, so no borrow reaches the
// neighbouring bytes); true for the thread that brings it to 0.
__device__ __forceinline__ bool last_child_done(const HeapView& h, uint32_t T, uint32_t p) {
  uint8_t* b = F<uint8_t>(h, T, p, T_FRONT);
  unsigned int* word = reinterpret_cast<unsigned int*>(reinterpret_cast<uintptr_t>(b) & ~uintptr_t(3));
  const uint32_t shift = (uint32_t)(reinterpret_cast<uintptr_t>(b) & 3) * 8u;
  __threadfence();  // this node's results before the count-down
  const uint32_t old = atomicSub(word, 1u << shift);
  if (((old >> shift) & 0xFFu) != 1u) return false;
  __threadfence();  // the other children's results before the parent's reads
  return true;
}

// Mass and centre of gravity of tree node `self` from its children.
__device__ __forceinline__ void summarize(const HeapView& h, uint32_t T, uint32_t self) {
  float ms = 0.0f, sx = 0.0f, sy = 0.0f;
  for (int i = 0; i < 4; ++i) {
    const uint32_t ch = Lcg<uint32_t>(h, T, self, T_CH + i);
    if (ch == kNull) continue;
    const uint32_t t = type_of(h, ch);
    const float cm = Lcg<float>(h, t, ch, C_M), cx = Lcg<float>(h, t, ch, C_PX), cy = Lcg<float>(h, t, ch, C_PY);
    ms = fa(ms, cm);
    sx = fa(sx, fm(cm, cx));
    sy = fa(sy, fm(cm, cy));
  }
  *F<float>(h, T, self, C_M) = ms;
  *F<float>(h, T, self, C_PX) = ms > 0.0f ? __fdiv_rn(sx, ms) : 0.0f;
  *F<float>(h, T, self, C_PY) = ms > 0.0f ? __fdiv_rn(sy, ms) : 0.0f;
  *F<uint8_t>(h, T, self, T_DONE) = 1;
}

struct TreeSummaryWalk {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (*F<uint8_t>(h, c, self, T_DONE) != 2) return;  // not a start of a walk
    uint32_t node = self;
    for (int depth = 0; depth <= kMaxDepth + 1; ++depth) {
      summarize(h, c, node);
      const uint32_t p = Lcg<uint32_t>(h, c, node, C_PARENT);
      if (p == kNull || !last_child_done(h, c, p)) return;
      node = p;
    }
    set_error(h, SMMO_E_BOUNDS, kTagDepth | self);  // deeper than any tree the insertion builds
  }
};

// Collapse of tree node `self` (all its tree-node children collapsed): a
// node without children is unlinked and deleted, one whose only child is a
// body is replaced by that body; returns its parent (kNull for the root).
__device__ __forceinline__ uint32_t collapse_node(const HeapView& h, const BHArgs& a, uint32_t T, uint32_t self) {
  int n = 0;
  uint32_t single = kNull;
  for (int i = 0; i < 4; ++i) {
    const uint32_t ch = Lcg<uint32_t>(h, T, self, T_CH + i);
    if (ch != kNull) { ++n; single = ch; }
  }
  const uint32_t parent = Lcg<uint32_t>(h, T, self, C_PARENT);
  if (parent != kNull) {
    const int idx = Lcg<int8_t>(h, T, self, C_CIDX);
    uint32_t* slot = F<uint32_t>(h, T, parent, T_CH + idx);
    if (n == 0) {  // empty: unlink and delete
      *slot = kNull;
      smmo_delete(h, self);
      return parent;
    }
    if (n == 1 && type_of(h, single) == a.body_cls) {  // single body: it takes our slot
      *F<uint32_t>(h, a.body_cls, single, C_PARENT) = parent;
      *F<int8_t>(h, a.body_cls, single, C_CIDX) = (int8_t)idx;
      *slot = single;
      smmo_delete(h, self);
      return parent;
    }
  }
  *F<uint8_t>(h, T, self, T_DONE) = 1;
  return parent;
}

struct TreeCollapseWalk {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (*F<uint8_t>(h, c, self, T_DONE) != 2) return;  // not a start of a walk
    uint32_t node = self;
    for (int depth = 0; depth <= kMaxDepth + 1; ++depth) {
      const uint32_t p = collapse_node(h, a, c, node);
      if (p == kNull || !last_child_done(h, c, p)) return;
      node = p;
    }
    set_error(h, SMMO_E_BOUNDS, kTagDepth | self);
  }
};

// ------------------------------------------------------------------ bodies
template <bool FAST>
__device__ void body_force(const HeapView& h, const BHArgs& a, uint32_t self) {
  const uint32_t B = a.body_cls, T = a.tree_cls;
  const float xs = *F<float>(h, B, self, C_PX), ys = *F<float>(h, B, self, C_PY);
  float ax = 0.0f, ay = 0.0f;
  uint32_t stack[kStack];
  int sp = 0;
  // the root's children, child 0 on top
  for (int i = 3; i >= 0; --i) {
    const uint32_t ch = *F<uint32_t>(h, T, a.root, T_CH + i);
    if (ch != kNull) stack[sp++] = ch;
  }
  // a region quad tree of n0 bodies has fewer than n0 * kMaxDepth nodes;
  // the budget only guards against a damaged tree
  uint64_t budget = (uint64_t)a.n0 * kMaxDepth + 64;
  while (sp > 0) {
    if (budget-- == 0) { set_error(h, SMMO_E_BOUNDS, kTagStack | self); break; }
    const uint32_t nd = stack[--sp];
    if (type_of(h, nd) == B) {
      if (nd != self) pair_acc<FAST>(xs, ys, *F<float>(h, B, nd, C_PX), *F<float>(h, B, nd, C_PY),
                                     *F<float>(h, B, nd, C_M), a.eps2, ax, ay);
      continue;
    }
    const float p1x = *F<float>(h, T, nd, T_P1X), p1y = *F<float>(h, T, nd, T_P1Y), w = *F<float>(h, T, nd, T_W);
    const float cx = *F<float>(h, T, nd, C_PX), cy = *F<float>(h, T, nd, C_PY);
    const bool inside = xs >= p1x && xs < fa(p1x, w) && ys >= p1y && ys < fa(p1y, w);
    const float dx = fs(cx, xs), dy = fs(cy, ys);
    const float d2 = fa(fm(dx, dx), fm(dy, dy));
    if (inside || fm(w, w) >= fm(a.theta2, d2)) {
      if (sp + 4 > kStack) { set_error(h, SMMO_E_BOUNDS, kTagStack | nd); break; }
      for (int i = 3; i >= 0; --i) {
        const uint32_t ch = *F<uint32_t>(h, T, nd, T_CH + i);
        if (ch != kNull) stack[sp++] = ch;
      }
    } else {
      pair_acc<FAST>(xs, ys, cx, cy, *F<float>(h, T, nd, C_M), a.eps2, ax, ay);
    }
  }
  *F<float>(h, B, self, B_AX) = ax;
  *F<float>(h, B, self, B_AY) = ay;
}

struct BodyForce {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    if (a.fast) body_force<true>(h, a, self);
    else body_force<false>(h, a, self);
  }
};

__device__ __forceinline__ void bounce(float& p, float& v) {
  if (p < 0.0f) { p = -p; v = -v; }
  else if (p >= 1.0f) { p = fs(2.0f, p); v = -v; }
  if (p < 0.0f) p = 0.0f;
  if (p > 0x1.fffffep-1f) p = 0x1.fffffep-1f;
}

struct BodyUpdate {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    float& x = *F<float>(h, c, self, C_PX);
    float& y = *F<float>(h, c, self, C_PY);
    float& vx = *F<float>(h, c, self, B_VX);
    float& vy = *F<float>(h, c, self, B_VY);
    vx = fa(vx, fm(fm(a.G, *F<float>(h, c, self, B_AX)), a.dt));
    vy = fa(vy, fm(fm(a.G, *F<float>(h, c, self, B_AY)), a.dt));
    x = fa(x, fm(vx, a.dt));
    y = fa(y, fm(vy, a.dt));
    bounce(x, vx);
    bounce(y, vy);
  }
};

struct BodyRemove {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint32_t* pp = F<uint32_t>(h, c, self, C_PARENT);
    const uint32_t p = *pp;
    if (p == kNull) return;
    const uint32_t T = a.tree_cls;
    const int i = *F<int8_t>(h, c, self, C_CIDX);
    const float w = *F<float>(h, T, p, T_W), hw = fm(w, 0.5f);
    const float qx = fa(*F<float>(h, T, p, T_P1X), (i & 1) ? hw : 0.0f);
    const float qy = fa(*F<float>(h, T, p, T_P1Y), (i & 2) ? hw : 0.0f);
    const float x = *F<float>(h, c, self, C_PX), y = *F<float>(h, c, self, C_PY);
    if (x >= qx && x < fa(qx, hw) && y >= qy && y < fa(qy, hw)) return;
    *F<uint32_t>(h, T, p, T_CH + i) = kNull;
    *pp = kNull;
  }
};

// Insertion of a body without parent (the thesis' add_to_tree).
struct BodyInsert {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (*F<uint32_t>(h, c, self, C_PARENT) != kNull) return;
    const uint32_t B = a.body_cls, T = a.tree_cls;
    const float x = *F<float>(h, B, self, C_PX), y = *F<float>(h, B, self, C_PY);
    uint32_t cur = a.root;
    int depth = 0;
    for (int it = 0; it < kInsertBudget; ++it) {
      const float p1x = Lcg<float>(h, T, cur, T_P1X), p1y = Lcg<float>(h, T, cur, T_P1Y),
                  w = Lcg<float>(h, T, cur, T_W);
      const int idx = quadrant(p1x, p1y, w, x, y);
      uint32_t* slot = F<uint32_t>(h, T, cur, T_CH + idx);
      const uint32_t child = __ldcg(slot);
      if (child == kNull) {
        // the child index goes in before the parent, which others wait for
        *F<int8_t>(h, B, self, C_CIDX) = (int8_t)idx;
        __threadfence();
        if (atomicCAS(slot, kNull, self) == kNull) {
          atomicExch(F<uint32_t>(h, B, self, C_PARENT), cur);
          return;
        }
        continue;  // lost the slot: look again
      }
      if (type_of(h, child) == T) {
        cur = child;
        if (++depth > kMaxDepth) { set_error(h, SMMO_E_BOUNDS, kTagDepth | self); return; }
        continue;
      }
      // the slot holds a body: put both under a new tree node
      if (depth + 1 > kMaxDepth) { set_error(h, SMMO_E_BOUNDS, kTagDepth | self); return; }  // coincident bodies
      const uint32_t nn = smmo_new(h, T);
      if (nn == kNull) return;  // out of memory, recorded by new
      const float hw = fm(w, 0.5f);
      const float np1x = fa(p1x, (idx & 1) ? hw : 0.0f), np1y = fa(p1y, (idx & 2) ? hw : 0.0f);
      const float ox = __ldcg(F<float>(h, B, child, C_PX)), oy = __ldcg(F<float>(h, B, child, C_PY));
      const int oidx = quadrant(np1x, np1y, hw, ox, oy);
      *F<uint32_t>(h, T, nn, C_PARENT) = cur;
      *F<int8_t>(h, T, nn, C_CIDX) = (int8_t)idx;
      *F<float>(h, T, nn, C_PX) = 0.0f;
      *F<float>(h, T, nn, C_PY) = 0.0f;
      *F<float>(h, T, nn, C_M) = 0.0f;
      for (int i = 0; i < 4; ++i) *F<uint32_t>(h, T, nn, T_CH + i) = i == oidx ? child : kNull;
      *F<float>(h, T, nn, T_P1X) = np1x;
      *F<float>(h, T, nn, T_P1Y) = np1y;
      *F<float>(h, T, nn, T_W) = hw;
      *F<uint8_t>(h, T, nn, T_FRONT) = 0;
      *F<uint8_t>(h, T, nn, T_DONE) = 0;
      __threadfence();  // the new node is complete before it becomes visible
      if (atomicCAS(slot, child, nn) == child) {
        // the moved body may still be finishing its own insertion: wait
        // until its parent is cur (only this thread may change it from cur
        // now), then write its child index and only then its new parent,
        // which the next thread to move it waits for (a later child-index
        // write can then not be overtaken by this one)
        uint32_t* op = F<uint32_t>(h, B, child, C_PARENT);
        int spins = 0;
        while (__ldcg(op) != cur) {
          if (++spins > h.bitmap_spins) { set_error(h, SMMO_E_CONTENTION, kTagWaitParent | child); return; }
          __nanosleep(32);
        }
        *F<int8_t>(h, B, child, C_CIDX) = (int8_t)oidx;
        __threadfence();
        atomicExch(op, nn);
        cur = nn;
        ++depth;
      } else {
        smmo_delete(h, nn);  // another thread changed the slot first
      }
    }
    set_error(h, SMMO_E_CONTENTION, kTagBudget | self);
  }
};

struct BodyExport {
  using Args = BHArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t id = *F<int32_t>(h, c, self, B_ID);
    if (id < 0 || (uint32_t)id >= a.n0) { set_error(h, SMMO_E_BOUNDS, self); return; }
    a.out[id] = *F<float>(h, c, self, C_PX);
    a.out[a.n0 + id] = *F<float>(h, c, self, C_PY);
    a.out[2 * a.n0 + id] = *F<float>(h, c, self, B_VX);
    a.out[3 * a.n0 + id] = *F<float>(h, c, self, B_VY);
    a.out[4 * a.n0 + id] = *F<float>(h, c, self, C_M);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_bh[] = {
    SMMO_METHOD("bh.tree_pending", TreePending), SMMO_METHOD("bh.tree_summary", TreeSummaryWalk),
    SMMO_METHOD("bh.tree_collapse", TreeCollapseWalk),
    SMMO_METHOD("bh.body_force", BodyForce), SMMO_METHOD("bh.body_update", BodyUpdate),
    SMMO_METHOD("bh.body_remove", BodyRemove), SMMO_METHOD("bh.body_insert", BodyInsert),
    SMMO_METHOD("bh.body_export", BodyExport)};
const int g_methods_bh_n = sizeof(g_methods_bh) / sizeof(g_methods_bh[0]);

struct smmo_bh {
  smmo_heap* heap = nullptr;
  int cls_base = -1, cls_body = -1, cls_tree = -1;
  uint32_t n0 = 0;
  BHArgs args{};
  int64_t levels = 0;  // bottom-up traversals run (statistics)
};

namespace {
int pdo(smmo_bh* w, int cls, method_launch_fn fn, const BHArgs& a, cudaStream_t s, bool reuse = false) {
  int st = reuse ? SMMO_OK : enumerate(w->heap, cls, s);
  if (!st) st = fn(w->heap, cls, &a, s);
  return st;
}

// Bottom-up traversal: the pending counts, then one walk do-all over the
// same snapshot (the count creates and deletes nothing; the walk of the
// collapse deletes tree nodes, which it never visits again).  Two launches
// and one enumeration, no host round trip.
int bottom_up(smmo_bh* w, method_launch_fn walk, cudaStream_t s) {
  const BHArgs& a = w->args;
  int st = pdo(w, w->cls_tree, &launch_do_all<TreePending>, a, s);
  if (!st) st = pdo(w, w->cls_tree, walk, a, s, true);
  if (!st) ++w->levels;
  return st;
}
}  // namespace

extern "C" {

int smmo_bh_create(smmo_heap* heap, int64_t n, const float* const* cols, const smmo_bh_params* p, void* stream,
                   smmo_bh** out) {
  if (!heap || n < 1 || n >= (1ll << 31) || !cols || !p || !out || !(p->theta >= 0.0f) || !(p->eps > 0.0f))
    return SMMO_E_INVALID_ARG;
  for (int k = 0; k < 5; ++k)
    if (!cols[k]) return SMMO_E_INVALID_ARG;
  if (!heap->classes.empty() || heap->frozen) return SMMO_E_FROZEN;
  cudaStream_t s = (cudaStream_t)stream;
  smmo_bh* w = new smmo_bh();
  w->heap = heap;
  w->n0 = (uint32_t)n;
  smmo_field_desc nb[5] = {{"parent", SMMO_HANDLE, 1, -1}, {"child_idx", SMMO_I8, 1, -1},
                           {"px", SMMO_F32, 1, -1}, {"py", SMMO_F32, 1, -1}, {"m", SMMO_F32, 1, -1}};
  smmo_field_desc bf[5] = {{"vx", SMMO_F32, 1, -1}, {"vy", SMMO_F32, 1, -1}, {"ax", SMMO_F32, 1, -1},
                           {"ay", SMMO_F32, 1, -1}, {"id", SMMO_I32, 1, -1}};
  int st = smmo_class_register(heap, "NodeBase", nb, 5, -1, 1, &w->cls_base);
  smmo_field_desc tf[6] = {{"children", SMMO_HANDLE, 4, w->cls_base}, {"p1x", SMMO_F32, 1, -1},
                           {"p1y", SMMO_F32, 1, -1}, {"w", SMMO_F32, 1, -1},
                           {"frontier", SMMO_U8, 1, -1}, {"done", SMMO_U8, 1, -1}};
  if (!st) st = smmo_class_register(heap, "BodyNode", bf, 5, w->cls_base, 0, &w->cls_body);
  if (!st) st = smmo_class_register(heap, "TreeNode", tf, 6, w->cls_base, 0, &w->cls_tree);
  if (heap->cfg.block_data_bytes == 0) heap->cfg.block_data_bytes = 3072;  // 64 slots for both classes
  if (!st) st = freeze(heap, s);
  if (st) { delete w; return st; }
  BHArgs& a = w->args;
  memset(&a, 0, sizeof(a));
  a.body_cls = (uint32_t)w->cls_body;
  a.tree_cls = (uint32_t)w->cls_tree;
  a.G = p->G;
  a.eps2 = p->eps * p->eps;
  a.dt = p->dt;
  a.theta2 = p->theta * p->theta;
  // positions stay in [0,1)^2, so s2 <= 2 + eps^2: the branch-free square
  // root and reciprocal are exact whenever eps^2 is in [2^-40, 2^38]
  a.fast = (a.eps2 >= 0x1p-40f && a.eps2 <= 0x1p38f) ? 1 : 0;
  a.n0 = (uint32_t)n;
  // root tree node: the unit square, no children
  std::vector<void*> d(14, nullptr);
  const uint32_t nul = kNull;
  const int8_t zi = 0;
  const float zf = 0.0f, one = 1.0f;
  const uint8_t zb = 0;
  const void* rv[14] = {&nul, &zi, &zf, &zf, &zf, &nul, &nul, &nul, &nul, &zf, &zf, &one, &zb, &zb};
  const size_t rs[14] = {4, 1, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 1, 1};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 14 && e == cudaSuccess; ++k) {
    e = cudaMallocAsync(&d[k], 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d[k], rv[k], rs[k], cudaMemcpyHostToDevice, s);
  }
  uint32_t* d_root = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&d_root, 4, s);
  if (e == cudaSuccess) st = smmo_bulk_new(heap, w->cls_tree, 1, (const void* const*)d.data(), d_root, nullptr, stream);
  uint32_t root = kNull;
  if (e == cudaSuccess && !st) e = cudaMemcpyAsync(&root, d_root, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* q : d) if (q) cudaFreeAsync(q, s);
  if (d_root) cudaFreeAsync(d_root, s);
  if (e != cudaSuccess) st = cuda_status(e);
  if (st) { smmo_bh_destroy(w); return st; }
  a.root = root;
  // bodies: parent null, fields from the caller's columns, id = index
  std::vector<void*> bd(10, nullptr);
  e = cudaSuccess;
  for (int k : {0, 1, 7, 8, 9}) {  // parent, child_idx, ax, ay, id
    const size_t sz = k == 1 ? 1 : 4;
    e = e == cudaSuccess ? cudaMallocAsync(&bd[k], (size_t)n * sz, s) : e;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(bd[0], 0xFF, (size_t)n * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bd[1], 0, (size_t)n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bd[7], 0, (size_t)n * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bd[8], 0, (size_t)n * 4, s);
  std::vector<int32_t> ids((size_t)n);
  for (int64_t i = 0; i < n; ++i) ids[(size_t)i] = (int32_t)i;
  if (e == cudaSuccess) e = cudaMemcpyAsync(bd[9], ids.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
  const void* src[10] = {bd[0], bd[1], cols[0], cols[1], cols[4], cols[2], cols[3], bd[7], bd[8], bd[9]};
  st = e == cudaSuccess ? smmo_bulk_new(heap, w->cls_body, n, src, nullptr, nullptr, stream) : cuda_status(e);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  for (void* q : bd) if (q) cudaFreeAsync(q, s);
  if (st) { smmo_bh_destroy(w); return st; }
  // initial tree: insert every body (an insert-only build is already the
  // region quad tree)
  st = pdo(w, w->cls_body, &launch_do_all<BodyInsert>, a, s);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  if (st) { smmo_bh_destroy(w); return st; }
  *out = w;
  return SMMO_OK;
}

int smmo_bh_step(smmo_bh* w, int nsteps, void* stream) {
  if (!w || nsteps < 0) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const BHArgs& a = w->args;
  for (int k = 0; k < nsteps; ++k) {
    int st = bottom_up(w, &launch_do_all<TreeSummaryWalk>, s);
    // no body is created or deleted in a step: one enumeration of the
    // bodies serves the four body do-alls
    if (!st) st = pdo(w, w->cls_body, &launch_do_all<BodyForce>, a, s);
    if (!st) st = pdo(w, w->cls_body, &launch_do_all<BodyUpdate>, a, s, true);
    if (!st) st = pdo(w, w->cls_body, &launch_do_all<BodyRemove>, a, s, true);
    if (!st) st = pdo(w, w->cls_body, &launch_do_all<BodyInsert>, a, s, true);
    if (!st) st = bottom_up(w, &launch_do_all<TreeCollapseWalk>, s);
    if (st) return st;
  }
  return SMMO_OK;
}

int smmo_bh_export(smmo_bh* w, float* out5, int64_t* tree_nodes, void* stream) {
  if (!w || !out5) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(out5, 0, sizeof(float) * 5 * (size_t)w->n0, s);
  if (e != cudaSuccess) return cuda_status(e);
  BHArgs a = w->args;
  a.out = out5;
  int st = pdo(w, w->cls_body, &launch_do_all<BodyExport>, a, s);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  if (!st && tree_nodes) {
    smmo_heap_stats hs;
    st = smmo_heap_get_stats(w->heap, &hs, stream);
    if (!st) *tree_nodes = hs.live_objects[w->cls_tree];
  }
  return st;
}

int smmo_bh_info(smmo_bh* w, int* class_ids, int64_t* levels) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (class_ids) { class_ids[0] = w->cls_base; class_ids[1] = w->cls_body; class_ids[2] = w->cls_tree; }
  if (levels) *levels = w->levels;
  return SMMO_OK;
}

int smmo_bh_destroy(smmo_bh* w) {
  if (!w) return SMMO_E_INVALID_ARG;
  delete w;
  return SMMO_OK;
}

}  // extern "C"
