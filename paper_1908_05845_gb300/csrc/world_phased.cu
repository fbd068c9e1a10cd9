// world_phased.cu -- Wa-Tor with each species' prepare and update fused
// into one cooperative launch (phased.cuh), with or without queued
// creation (smmo_world_set_step_kernels modes SMMO_WATOR_PHASED1/2).  A
// translation unit of its own, so that these kernel instantiations compile
// in parallel with the others.
#include "world_wator.cuh"

namespace {

// ------------------------------------------------- Wa-Tor in two phases
// The same fish and shark rules as the four do-alls above, for the fused
// launch of phased.cuh: the prepare phase returns the request word
// (target | rank << 30) as the carry instead of storing it in the agent's
// target field, kIdle for an agent that posts no request, and for a shark
// kStarve when it starves; the update phase runs only for those.  The
// carries are distinct from every request word because cells stay below
// 2^30 - 2 (smmo_world_create_batch).
constexpr uint32_t kIdleWord = 0xFFFFFFFFu, kStarveWord = 0xFFFFFFFEu;

struct FishPhased {
  using Args = WorldArgs;
  static constexpr uint32_t kIdle = kIdleWord;
  static constexpr uint32_t kDeferMax = 1;
  struct P {
    uint32_t g, x, y, occ[4];
    int32_t age;
    const Inst* in;
  };
  struct U {
    uint32_t g, req;
    int32_t age;
  };
  __device__ static uint32_t child_class(const Args& a) { return a.fish; }
  __device__ static void create(const HeapView& h, const Args& a, uint32_t child, uint32_t g) {
    FishUpdate::create(h, a, child, g);
  }
  __device__ static void load1(const HeapView& h, const Args& a, uint32_t, uint32_t self, P& p) {
    p.g = *fld<int32_t>(h, self, a.f_cell);
    p.age = *fld<int16_t>(h, self, a.f_age);
  }
  __device__ static void load2(const HeapView& h, const Args& a, uint32_t, uint32_t, P& p) {
    p.in = find_inst(h, p.g);
    cell_xy(p.in, p.g - p.in->cell_base, &p.x, &p.y);
#pragma unroll
    for (int d = 0; d < 4; ++d)
      p.occ[d] = *a.cells.col<uint32_t>(p.in->cell_base + torus_nb4(p.x, p.y, p.in->W, p.in->H, d), a.occ_off);
  }
  __device__ static uint32_t prepare(const HeapView& h, const Args& a, uint32_t, uint32_t self, P& p) {
    *fld<int16_t>(h, self, a.f_age) = (int16_t)(p.age + 1);
    uint32_t empty = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (p.occ[d] == kNull) empty |= 1u << d;
    if (!empty) return kIdle;
    const uint32_t t = *a.tp;
    return post_request(a, p.in, p.x, p.y, choose_dir(a, p.in, TAG_FISH, t, p.g - p.in->cell_base, empty), t);
  }
  __device__ static void spill(const HeapView& h, const Args& a, uint32_t, uint32_t self, uint32_t w) {
    *fld<int32_t>(h, self, a.f_target) = (int32_t)w;
  }
  __device__ static uint32_t unspill(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    return (uint32_t)*fld<int32_t>(h, self, a.f_target);
  }
  __device__ static void uload(const HeapView& h, const Args& a, uint32_t, uint32_t self, uint32_t w, U& q) {
    q.req = __ldcg(a.cells.col<uint32_t>(w & kCellMask, a.req_off));
    q.g = *fld<int32_t>(h, self, a.f_cell);
    q.age = *fld<int16_t>(h, self, a.f_age);
  }
  __device__ static void update(const HeapView& h, const Args& a, uint32_t, uint32_t self, uint32_t w, U& q) {
    if (q.req != req_key(*a.tp, a.phase, w >> 30)) return;  // another fish won the target
    const uint32_t tgt = w & kCellMask;
    set_occ(a, tgt, self);
    *fld<int32_t>(h, self, a.f_cell) = (int32_t)tgt;
    const bool ripe = a.breed_strict ? q.age > a.fish_breed : q.age >= a.fish_breed;
    if (ripe) {
      *fld<int16_t>(h, self, a.f_age) = 0;
      defer_new(q.g);
    } else {
      set_occ(a, q.g, kNull);
    }
  }
};

struct SharkPhased {
  using Args = WorldArgs;
  static constexpr uint32_t kIdle = kIdleWord;
  static constexpr uint32_t kDeferMax = 1;
  struct P {
    uint32_t g, x, y, occ[4];
    int32_t age, energy;
    const Inst* in;
  };
  struct U {
    uint32_t g, req, prey;
    int32_t age;
  };
  __device__ static uint32_t child_class(const Args& a) { return a.shark; }
  __device__ static void create(const HeapView& h, const Args& a, uint32_t child, uint32_t g) {
    SharkUpdate::create(h, a, child, g);
  }
  __device__ static void load1(const HeapView& h, const Args& a, uint32_t, uint32_t self, P& p) {
    p.g = *fld<int32_t>(h, self, a.s_cell);
    p.age = *fld<int16_t>(h, self, a.s_age);
    p.energy = *fld<int16_t>(h, self, a.s_energy);
  }
  __device__ static void load2(const HeapView& h, const Args& a, uint32_t, uint32_t, P& p) {
    p.in = find_inst(h, p.g);
    cell_xy(p.in, p.g - p.in->cell_base, &p.x, &p.y);
    if (p.energy == 1) return;  // starves in this step: no neighbour is looked at
#pragma unroll
    for (int d = 0; d < 4; ++d)
      p.occ[d] = *a.cells.col<uint32_t>(p.in->cell_base + torus_nb4(p.x, p.y, p.in->W, p.in->H, d), a.occ_off);
  }
  __device__ static uint32_t prepare(const HeapView& h, const Args& a, uint32_t, uint32_t self, P& p) {
    *fld<int16_t>(h, self, a.s_age) = (int16_t)(p.age + 1);
    const int16_t en = (int16_t)(p.energy - 1);
    *fld<int16_t>(h, self, a.s_energy) = en;
    if (en == 0) return kStarveWord;
    uint32_t fish = 0, empty = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (p.occ[d] == kNull) empty |= 1u << d;
      else if (type_of(h, p.occ[d]) == a.fish) fish |= 1u << d;
    }
    if (!(fish | empty)) return kIdle;
    const uint32_t t = *a.tp;
    return post_request(a, p.in, p.x, p.y,
                        choose_dir(a, p.in, TAG_SHARK, t, p.g - p.in->cell_base, fish ? fish : empty), t);
  }
  __device__ static void spill(const HeapView& h, const Args& a, uint32_t, uint32_t self, uint32_t w) {
    *fld<int32_t>(h, self, a.s_target) = (int32_t)w;
  }
  __device__ static uint32_t unspill(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    return (uint32_t)*fld<int32_t>(h, self, a.s_target);
  }
  __device__ static void uload(const HeapView& h, const Args& a, uint32_t, uint32_t self, uint32_t w, U& q) {
    q.g = *fld<int32_t>(h, self, a.s_cell);
    if (w == kStarveWord) return;
    const uint32_t tgt = w & kCellMask;
    q.req = __ldcg(a.cells.col<uint32_t>(tgt, a.req_off));
    // only the winner of the target writes its occupant in this phase
    q.prey = __ldcg(a.cells.col<uint32_t>(tgt, a.occ_off));
    q.age = *fld<int16_t>(h, self, a.s_age);
  }
  __device__ static void update(const HeapView& h, const Args& a, uint32_t, uint32_t self, uint32_t w, U& q) {
    if (w == kStarveWord) {  // starved: leave the cell and delete itself
      set_occ(a, q.g, kNull);
      smmo_delete(h, self);
      return;
    }
    if (q.req != req_key(*a.tp, a.phase, w >> 30)) return;  // another shark won the target
    const uint32_t tgt = w & kCellMask;
    if (q.prey != kNull) {  // eat the fish (deleting an object of another class)
      smmo_delete(h, q.prey);
      *fld<int16_t>(h, self, a.s_energy) = (int16_t)a.starve;
    }
    set_occ(a, tgt, self);
    *fld<int32_t>(h, self, a.s_cell) = (int32_t)tgt;
    const bool ripe = a.breed_strict ? q.age > a.shark_breed : q.age >= a.shark_breed;
    if (ripe) {
      *fld<int16_t>(h, self, a.s_age) = 0;
      defer_new(q.g);
    } else {
      set_occ(a, q.g, kNull);
    }
  }
};

// The same with their creations queued.
struct FishPhasedQ : FishPhased {
  static constexpr bool kQueued = true;
  __device__ static DeferQueue queue(const Args& a) { return a.fq; }
};
struct SharkPhasedQ : SharkPhased {
  static constexpr bool kQueued = true;
  __device__ static DeferQueue queue(const Args& a) { return a.sq; }
};

// The fused fish or shark phase (phased.cuh) with K units per round; the
// barrier words come with the arguments.  The register budget: 48 warps
// per SM (40 registers) for one unit per round, 40 warps (48 registers)
// for two.
#ifndef SMMO_PHASED_WARPS1
#define SMMO_PHASED_WARPS1 48
#endif
#ifndef SMMO_PHASED_WARPS2
#define SMMO_PHASED_WARPS2 40
#endif
template <class M, int K>
int launch_wator_phased(smmo_heap* h, int cls, const void* args, cudaStream_t s) {
  constexpr int kMinb = (K == 1 ? SMMO_PHASED_WARPS1 : SMMO_PHASED_WARPS2) / (kPhasedThreads / 32);
  const WorldArgs* a = static_cast<const WorldArgs*>(args);
  return launch_phased<M, K, (kMinb > 0 ? kMinb : 1)>(h, cls, *a, a->ctl, s);
}
}  // namespace

smmo::method_launch_fn wator_phased_launcher(int which, int mode) {
  const bool q = (mode & SMMO_WATOR_QUEUED_CREATION) != 0, k2 = (mode & 3) == SMMO_WATOR_PHASED2;
  switch (which) {
    case kWFishPrepare:
      return q ? (k2 ? &launch_wator_phased<FishPhasedQ, 2> : &launch_wator_phased<FishPhasedQ, 1>)
               : (k2 ? &launch_wator_phased<FishPhased, 2> : &launch_wator_phased<FishPhased, 1>);
    case kWSharkPrepare:
      return q ? (k2 ? &launch_wator_phased<SharkPhasedQ, 2> : &launch_wator_phased<SharkPhasedQ, 1>)
               : (k2 ? &launch_wator_phased<SharkPhased, 2> : &launch_wator_phased<SharkPhased, 1>);
    case kWFishCreate: return q ? &launch_create_queued<FishPhasedQ> : nullptr;
    case kWSharkCreate: return q ? &launch_create_queued<SharkPhasedQ> : nullptr;
    default: return nullptr;
  }
}
