// world_wator.cuh -- what the cellular workloads' translation units share:
// the argument block of the world methods and the Wa-Tor methods of the
// four plain do-alls (world.cu), on which the other Wa-Tor step kernels
// (world_modes.cu: queued creation, marked updates; world_phased.cu: fused
// phases) build.
// Everything here has internal linkage (an anonymous namespace), so each
// translation unit instantiates its own kernels.
#pragma once
#include <cuda_runtime.h>

#include "grid_common.cuh"
#include "heap_internal.h"
#include "phased.cuh"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

// Launchers of the Wa-Tor step kernels other than the four plain do-alls
// (world_modes.cu; the fused phases in world_phased.cu): `which` names the
// launch, `mode` is a value of smmo_world_set_step_kernels; null where the
// mode has no such launch (the plain do-all of world.cu serves).
enum WatorLaunch { kWFishPrepare = 0, kWFishUpdate, kWFishCreate, kWSharkPrepare, kWSharkUpdate, kWSharkCreate };
smmo::method_launch_fn wator_mode_launcher(int which, int mode);
smmo::method_launch_fn wator_phased_launcher(int which, int mode);

namespace {

struct WorldArgs {
  CellRef cells;
  uint32_t occ_off, req_off, kind_off;
  uint32_t fish, shark, alive, cand;
  uint32_t f_cell, f_target, f_age;
  uint32_t s_cell, s_target, s_age, s_energy;
  uint32_t a_cell, a_action, a_isnew, a_blocked;
  uint32_t c_cell, c_action;
  uint32_t survive, born, block;  // rule of the Life-kind instances
  uint64_t seed;
  const uint32_t* tp;  // device step counter (1-based during a step)
  uint32_t phase;      // 0 fish, 1 shark
  int32_t fish_breed, shark_breed, starve, breed_strict;
  int8_t* out_kind;
  int16_t* out_age;
  int16_t* out_energy;
  uint8_t* out_state;
  uint32_t* out_count;
  unsigned long long* errors;
  uint32_t* seen;  // one bit per cell (allocation-free export only)
  unsigned long long* ctl;  // grid-barrier words of a two-phase launch (zeroed per step)
  DeferQueue fq, sq;        // queued creations of fish and sharks (one buffer, two counters)
};

template <class T>
__device__ __forceinline__ T* fld(const HeapView& h, uint32_t self, uint32_t off) {
  return field_ptr<T>(h, off, self);
}

// ================================================================ Wa-Tor
// A cell holds its occupant's handle, a 32-bit request word and a one-byte
// kind that only the Life instances use (see the Life section).  One phase
// = prepare (choose a neighbour, post a request) + update (move if
// granted).  The thesis' Cell::prepare / Cell::decide passes are folded into
// the request word of the target cell: the movers into a cell are among its
// four neighbours, so the lowest source cell is the requester of lowest rank
// among them (rank = how many of the target's neighbours have a smaller cell
// index); a requester posts key = ((2^30 - 1 - epoch) << 2) | rank with
// atomicMin, epoch = 2 t + phase.  The smallest key of the current phase
// wins, keys of older phases are larger and never win, so no pass over all
// cells resets them (2^29 steps).  The prepare keeps target | rank << 30 in
// the agent's target field (cells are below 2^30), so the update finds
// both without recomputing.  (A kind byte per cell for the Wa-Tor
// neighbour tests, replacing the handle and type-id loads, was measured:
// the prepares gained less than the two extra byte stores per mover cost
// the updates.)
enum : uint8_t { K_EMPTY = 0, K_ALIVE = 1, K_CAND = 2, K_BLOCK = 3 };
constexpr uint32_t kCellMask = 0x3FFFFFFFu;

__device__ __forceinline__ uint32_t req_key(uint32_t t, uint32_t phase, uint32_t rank) {
  return ((0x3FFFFFFFu - (2u * t + phase)) << 2) | rank;
}

// Rank (0..3) of the neighbour in direction e of cell (tx, ty) among its
// four neighbours by cell index, on a W x H torus (W, H >= 3).  Cell index
// = row W + column, so neighbours order by row first: the row above
// (ty - 1), the cell's own row (the horizontal pair) and the row below
// (ty + 1), taken mod H.  Inside the torus that is up, pair, down; on the
// first row (up wraps to the last row) pair, down, up; on the last row
// (down wraps to row 0) down, up, pair.  Within the pair left comes before
// right except on the first and last columns, where one of them wraps.
__device__ __forceinline__ uint32_t nb_rank(uint32_t tx, uint32_t ty, uint32_t W, uint32_t H, int e) {
  const bool top = ty == 0, bottom = ty + 1 == H;
  if (e == 0) return top ? 3u : bottom ? 1u : 0u;  // up
  if (e == 2) return top ? 2u : bottom ? 0u : 3u;  // down
  const uint32_t pair = top ? 0u : bottom ? 2u : 1u;
  const bool hwrap = tx == 0 || tx + 1 == W;
  return pair + ((e == 3) == hwrap ? 1u : 0u);     // left (3) or right (1)
}

// (x, y) of the neighbour in direction d of local cell (x, y).
__device__ __forceinline__ void nb_xy(uint32_t x, uint32_t y, uint32_t W, uint32_t H, int d, uint32_t* nx,
                                      uint32_t* ny) {
  *nx = x; *ny = y;
  if (d == 0) *ny = y == 0 ? H - 1 : y - 1;
  else if (d == 1) *nx = x + 1 == W ? 0 : x + 1;
  else if (d == 2) *ny = y + 1 == H ? 0 : y + 1;
  else *nx = x == 0 ? W - 1 : x - 1;
}

// The (r mod k)-th of the k directions set in mask (in direction order 0..3).
__device__ __forceinline__ int pick_dir(uint32_t mask, uint32_t r) {
  const uint32_t n = (uint32_t)__popc(mask);
  uint32_t k = n == 3 ? r % 3u : r & (n - 1);  // n is 1, 2, 3 or 4
  while (k--) mask &= mask - 1;
  return __ffs(mask) - 1;
}

// The direction an agent on local cell lc of `in` takes among the set bits
// of mask (non-empty): the (draw mod k)-th of the k choices.  With a single
// choice the draw cannot change the result and is not computed (the draws
// are counter-based, so skipping one affects no other).
__device__ __forceinline__ int choose_dir(const WorldArgs& a, const Inst* in, uint32_t tag, uint32_t t,
                                          uint32_t lc, uint32_t mask) {
  if ((mask & (mask - 1)) == 0) return __ffs(mask) - 1;
  return pick_dir(mask, philox_draw(a.seed, tag, t, lc, in->id));
}

// Posts the request of the agent on local cell (x, y) of `in` to move in
// direction d; returns target | rank << 30 for the agent's target field.
__device__ __forceinline__ uint32_t post_request(const WorldArgs& a, const Inst* in, uint32_t x, uint32_t y,
                                                 int d, uint32_t t) {
  uint32_t tx, ty;
  nb_xy(x, y, in->W, in->H, d, &tx, &ty);
  const uint32_t rank = nb_rank(tx, ty, in->W, in->H, (d + 2) & 3);  // we are its neighbour d + 2
  const uint32_t tgt = in->cell_base + ty * in->W + tx;
  atomicMin(a.cells.col<uint32_t>(tgt, a.req_off), req_key(t, a.phase, rank));
  return tgt | (rank << 30);
}

// Whether the request recorded in target field value tv (see post_request)
// won.
__device__ __forceinline__ bool won_request(const WorldArgs& a, uint32_t tv) {
  return *a.cells.col<uint32_t>(tv & kCellMask, a.req_off) == req_key(*a.tp, a.phase, tv >> 30);
}

// Occupant of a Wa-Tor cell (the Wa-Tor methods test neighbours through
// the handle; their cells' kind bytes stay K_EMPTY).
__device__ __forceinline__ void set_occ(const WorldArgs& a, uint32_t g, uint32_t handle) {
  *a.cells.col<uint32_t>(g, a.occ_off) = handle;
}

// Occupant of a Life cell and its kind byte.
__device__ __forceinline__ void set_cell(const WorldArgs& a, uint32_t g, uint32_t handle, uint8_t kind) {
  *a.cells.col<uint32_t>(g, a.occ_off) = handle;
  *a.cells.col<uint8_t>(g, a.kind_off) = kind;
}

// The prepares return whether the agent has anything to do in the update
// (a posted request, or a starving shark), for the marking do-all below.
struct FishPrepare {
  using Args = WorldArgs;
  __device__ static bool run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t g = *fld<int32_t>(h, self, a.f_cell);
    int16_t* agep = fld<int16_t>(h, self, a.f_age);
    *agep = (int16_t)(*agep + 1);
    const Inst* in = find_inst(h, g);
    const uint32_t lc = g - in->cell_base, W = in->W, H = in->H;
    uint32_t x, y;
    cell_xy(in, lc, &x, &y);
    uint32_t empty = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (*a.cells.col<uint32_t>(in->cell_base + torus_nb4(x, y, W, H, d), a.occ_off) == kNull) empty |= 1u << d;
    uint32_t tgt = g;
    if (empty) {
      const uint32_t t = *a.tp;
      tgt = post_request(a, in, x, y, choose_dir(a, in, TAG_FISH, t, lc, empty), t);
    }
    *fld<int32_t>(h, self, a.f_target) = (int32_t)tgt;
    return tgt != g;
  }
};

// Moves a fish whose request won; a ripe mover leaves a newborn fish on its
// old cell (created after the round, see defer_new), every other mover
// leaves it empty.
struct FishUpdate {
  using Args = WorldArgs;
  static constexpr uint32_t kDeferMax = 1;
  __device__ static uint32_t child_class(const Args& a) { return a.fish; }
  __device__ static void create(const HeapView& h, const Args& a, uint32_t child, uint32_t g) {
    if (child != kNull) {
      *fld<int32_t>(h, child, a.f_cell) = (int32_t)g;
      *fld<int32_t>(h, child, a.f_target) = (int32_t)g;
      *fld<int16_t>(h, child, a.f_age) = 0;
    }
    set_occ(a, g, child);
  }
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    int32_t* cellp = fld<int32_t>(h, self, a.f_cell);
    const uint32_t g = *cellp;
    const uint32_t tv = *fld<int32_t>(h, self, a.f_target);
    const uint32_t tgt = tv & kCellMask;
    if (tgt == g || !won_request(a, tv)) return;
    set_occ(a, tgt, self);
    *cellp = (int32_t)tgt;
    int16_t* agep = fld<int16_t>(h, self, a.f_age);
    const int age = *agep;
    const bool ripe = a.breed_strict ? age > a.fish_breed : age >= a.fish_breed;
    if (ripe) {
      *agep = 0;
      defer_new(g);
    } else {
      set_occ(a, g, kNull);
    }
  }
};

struct SharkPrepare {
  using Args = WorldArgs;
  __device__ static bool run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t g = *fld<int32_t>(h, self, a.s_cell);
    int16_t* agep = fld<int16_t>(h, self, a.s_age);
    int16_t* enp = fld<int16_t>(h, self, a.s_energy);
    *agep = (int16_t)(*agep + 1);
    const int16_t en = (int16_t)(*enp - 1);
    *enp = en;
    uint32_t tgt = g;
    if (en != 0) {
      const Inst* in = find_inst(h, g);
      const uint32_t lc = g - in->cell_base, W = in->W, H = in->H;
      uint32_t x, y;
      cell_xy(in, lc, &x, &y);
      uint32_t fish = 0, empty = 0;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const uint32_t o = *a.cells.col<uint32_t>(in->cell_base + torus_nb4(x, y, W, H, d), a.occ_off);
        if (o == kNull) empty |= 1u << d;
        else if (type_of(h, o) == a.fish) fish |= 1u << d;
      }
      if (fish | empty) {
        const uint32_t t = *a.tp;
        tgt = post_request(a, in, x, y, choose_dir(a, in, TAG_SHARK, t, lc, fish ? fish : empty), t);
      }
    }
    *fld<int32_t>(h, self, a.s_target) = (int32_t)tgt;
    return en == 0 || tgt != g;
  }
};

// A starved shark leaves its cell and deletes itself; a mover eats the fish
// on its target (deleting an object of another class) and, when ripe,
// leaves a newborn shark on its old cell (deferred, as for fish).
struct SharkUpdate {
  using Args = WorldArgs;
  static constexpr uint32_t kDeferMax = 1;
  __device__ static uint32_t child_class(const Args& a) { return a.shark; }
  __device__ static void create(const HeapView& h, const Args& a, uint32_t child, uint32_t g) {
    if (child != kNull) {
      *fld<int32_t>(h, child, a.s_cell) = (int32_t)g;
      *fld<int32_t>(h, child, a.s_target) = (int32_t)g;
      *fld<int16_t>(h, child, a.s_age) = 0;
      *fld<int16_t>(h, child, a.s_energy) = (int16_t)a.starve;
    }
    set_occ(a, g, child);
  }
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    int32_t* cellp = fld<int32_t>(h, self, a.s_cell);
    const uint32_t g = *cellp;
    int16_t* enp = fld<int16_t>(h, self, a.s_energy);
    const uint32_t tv = *fld<int32_t>(h, self, a.s_target);
    int16_t* agep = fld<int16_t>(h, self, a.s_age);
    const int age = *agep;
    if (*enp == 0) {  // starved: leave the cell and delete itself (last statement)
      set_occ(a, g, kNull);
      smmo_delete(h, self);
      return;
    }
    const uint32_t tgt = tv & kCellMask;
    if (tgt == g || !won_request(a, tv)) return;
    const uint32_t prey = *a.cells.col<uint32_t>(tgt, a.occ_off);
    if (prey != kNull) {  // eat the fish (deleting an object of another class)
      smmo_delete(h, prey);
      *enp = (int16_t)a.starve;
    }
    set_occ(a, tgt, self);
    *cellp = (int32_t)tgt;
    const bool ripe = a.breed_strict ? age > a.shark_breed : age >= a.shark_breed;
    if (ripe) {
      *agep = 0;
      defer_new(g);
    } else {
      set_occ(a, g, kNull);
    }
  }
};

}  // namespace
