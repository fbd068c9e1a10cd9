// world.cu -- the cellular SMMO workloads of the thesis' Ch. 7 on one heap:
// object-based Game of Life and its generational extension (Sec. 7.8,
// "gol" and "generation") and Wa-Tor (Sec. 7.6), for one or many
// independent instances ("batched heap": all instances' objects share the
// heap and every step runs one parallel_do per class over all of them).
//
// Classes: Cell {occ: handle of the agent on the cell, req: u32 request
// word, kind: u8}; WAgent (abstract) {cell, target} with Fish {age} and
// Shark {age, energy}; LAgent (abstract) {cell, action} with Alive {is_new,
// blocked} and Candidate {}.  Cells are created once by bulk_new in global
// cell order and addressed densely; agents hold their global cell index.
// The Wa-Tor methods are in world_wator.cuh (the four plain do-alls, here)
// and world_modes.cu / world_phased.cu (the other step kernels); this file
// holds the Life methods, the exports and the world API.
//
// The Life-kind instances follow one rule: an alive object survives iff bit
// n of `survive` is set (n = alive, i.e. not blocking, Alive objects among
// the 8 neighbours), a Candidate becomes alive iff bit n of `born` is set,
// and a dead Alive blocks its cell for `block` generations (field blocked
// counts them) before a Candidate replaces it.  Life is survive {2,3},
// born {3}, block 0 (a dead Alive is replaced at once); the generation
// application's Burst rule is survive {0,2,3,5,6,7,8}, born {3,4,6,8},
// block 255.
//
// Conflict resolution and randomness are keyed by (seed, step, local cell,
// tag, instance) and by lowest cell index, so a run is deterministic
// whatever the enumeration order or slot placement.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "world_wator.cuh"

namespace {

// ================================================================ Life
enum : uint8_t { ACT_KEEP = 0, ACT_BORN = 1, ACT_DELETE = 2, ACT_DIE = 3, ACT_AGE = 4, ACT_EXPIRE = 5 };

__device__ __forceinline__ uint32_t torus8(uint32_t x, uint32_t y, int dx, int dy, uint32_t W,
                                           uint32_t H) {
  const uint32_t nx = dx < 0 ? (x == 0 ? W - 1 : x - 1) : (dx > 0 ? (x + 1 == W ? 0 : x + 1) : x);
  const uint32_t ny = dy < 0 ? (y == 0 ? H - 1 : y - 1) : (dy > 0 ? (y + 1 == H ? 0 : y + 1) : y);
  return ny * W + nx;
}

// Kind byte of a Life cell (see the Wa-Tor section): an Alive born in this
// generation's candidate update is K_NEW until the alive prepare of the
// next generation clears its is_new; a dead Alive that blocks its cell is
// K_BLOCK.  Alive neighbours are those of kind K_ALIVE or K_NEW.
enum : uint8_t { K_NEW = 4 };

__device__ __forceinline__ int alive_neighbours(const WorldArgs& a, const Inst* in, uint32_t x, uint32_t y) {
  int n = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (!dx && !dy) continue;
      const uint8_t k = *a.cells.col<uint8_t>(in->cell_base + torus8(x, y, dx, dy, in->W, in->H), a.kind_off);
      n += (k == K_ALIVE) | (k == K_NEW);
    }
  return n;
}

struct CandPrepare {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t g = *fld<int32_t>(h, self, a.c_cell);
    const Inst* in = find_inst(h, g);
    const uint32_t lc = g - in->cell_base;
    uint32_t x, y;
    cell_xy(in, lc, &x, &y);
    const int n = alive_neighbours(a, in, x, y);
    *fld<uint8_t>(h, self, a.c_action) = ((a.born >> n) & 1) ? ACT_BORN : (n == 0 ? ACT_DELETE : ACT_KEEP);
  }
};

struct AlivePrepare {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t g = *fld<int32_t>(h, self, a.a_cell);
    uint8_t* isnew = fld<uint8_t>(h, self, a.a_isnew);
    if (*isnew) {  // K_NEW -> K_ALIVE; concurrent neighbour counts see either
      *isnew = 0;
      *a.cells.col<uint8_t>(g, a.kind_off) = K_ALIVE;
    }
    const uint32_t blocked = a.block ? *fld<uint16_t>(h, self, a.a_blocked) : 0u;
    if (blocked) {  // dead and blocking its cell
      *fld<uint8_t>(h, self, a.a_action) = blocked >= a.block ? ACT_EXPIRE : ACT_AGE;
      return;
    }
    const Inst* in = find_inst(h, g);
    const uint32_t lc = g - in->cell_base;
    uint32_t x, y;
    cell_xy(in, lc, &x, &y);
    const int n = alive_neighbours(a, in, x, y);
    *fld<uint8_t>(h, self, a.a_action) = ((a.survive >> n) & 1) ? ACT_KEEP : ACT_DIE;
  }
};

// A candidate that is born is replaced by a new Alive (created after the
// round, see defer_new: nothing else in this do-all reads its cell); one
// without alive neighbours leaves its cell empty.
struct CandUpdate {
  using Args = WorldArgs;
  static constexpr uint32_t kDeferMax = 1;
  __device__ static uint32_t child_class(const Args& a) { return a.alive; }
  __device__ static void create(const HeapView& h, const Args& a, uint32_t child, uint32_t g) {
    if (child != kNull) {
      *fld<int32_t>(h, child, a.a_cell) = (int32_t)g;
      *fld<uint8_t>(h, child, a.a_action) = ACT_KEEP;
      *fld<uint8_t>(h, child, a.a_isnew) = 1;
      *fld<uint16_t>(h, child, a.a_blocked) = 0;
    }
    set_cell(a, g, child, child != kNull ? K_NEW : K_EMPTY);
  }
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint8_t act = *fld<uint8_t>(h, self, a.c_action);
    if (act == ACT_KEEP) return;
    const uint32_t g = *fld<int32_t>(h, self, a.c_cell);
    if (act == ACT_BORN) defer_new(g);
    else set_cell(a, g, kNull, K_EMPTY);
    smmo_delete(h, self);
  }
};

struct AliveUpdate {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t g = *fld<int32_t>(h, self, a.a_cell);
    if (*fld<uint8_t>(h, self, a.a_isnew)) {
      // create Candidates on empty surrounding cells; the creator of an empty
      // cell e is the first new Alive of e's neighbourhood in scan order.
      // The kinds of the 5 x 5 window around g are read once (bit 5 a + b
      // for offset (a - 2, b - 2), so increasing bit numbers are the scan
      // order, dx outer, dy inner) and every decision is taken from them:
      // K_NEW never changes during this do-all, a cell turns neither empty
      // nor new in it, and only the creator of e writes e, so a kind read
      // earlier gives the same decisions as one read at the time.  The first
      // new Alive around e is the lowest set bit of the new-Alive bits under
      // e's 3 x 3 mask; W, H >= 3, so of the offsets -2..2 only (0, 0) (bit
      // 12) is g itself.
      const Inst* in = find_inst(h, g);
      const uint32_t lc = g - in->cell_base, W = in->W, H = in->H;
      uint32_t x, y;
      cell_xy(in, lc, &x, &y);
      uint32_t isnew = 0, isempty = 0;
#pragma unroll
      for (int ia = 0; ia < 5; ++ia) {
        const int xv = (int)x + ia - 2;
        const uint32_t col = (uint32_t)(xv < 0 ? xv + (int)W : (xv >= (int)W ? xv - (int)W : xv));
#pragma unroll
        for (int ib = 0; ib < 5; ++ib) {
          const int yv = (int)y + ib - 2;
          const uint32_t row = (uint32_t)(yv < 0 ? yv + (int)H : (yv >= (int)H ? yv - (int)H : yv));
          const uint8_t k = *a.cells.col<uint8_t>(in->cell_base + row * W + col, a.kind_off);
          isnew |= (uint32_t)(k == K_NEW) << (5 * ia + ib);
          isempty |= (uint32_t)(k == K_EMPTY) << (5 * ia + ib);
        }
      }
      constexpr uint32_t kBlock3 = 0x7u | (0x7u << 5) | (0x7u << 10);  // 3 x 3 at offset (-2, -2)
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
          const uint32_t eb = 5 * (dx + 2) + dy + 2;
          if (!((isempty >> eb) & 1u)) continue;
          const uint32_t around = isnew & (kBlock3 << (eb - 6));
          if ((uint32_t)(__ffs(around) - 1) != 12u) continue;  // another new Alive comes first
          const uint32_t e = in->cell_base + torus8(x, y, dx, dy, W, H);
          const uint32_t cnd = smmo_new(h, a.cand);
          if (cnd != kNull) {
            *fld<int32_t>(h, cnd, a.c_cell) = (int32_t)e;
            *fld<uint8_t>(h, cnd, a.c_action) = ACT_KEEP;
          }
          set_cell(a, e, cnd, cnd != kNull ? K_CAND : K_EMPTY);
        }
    } else {
      const uint8_t act = *fld<uint8_t>(h, self, a.a_action);
      if (act == ACT_DIE && a.block) {
        *fld<uint16_t>(h, self, a.a_blocked) = 1;  // dead: blocks its cell
        *a.cells.col<uint8_t>(g, a.kind_off) = K_BLOCK;
      } else if (act == ACT_AGE) {
        uint16_t* b = fld<uint16_t>(h, self, a.a_blocked);
        *b = (uint16_t)(*b + 1);
      } else if (act == ACT_DIE || act == ACT_EXPIRE) {  // replaced by a Candidate
        const uint32_t cnd = smmo_new(h, a.cand);
        if (cnd != kNull) {
          *fld<int32_t>(h, cnd, a.c_cell) = (int32_t)g;
          *fld<uint8_t>(h, cnd, a.c_action) = ACT_KEEP;
        }
        set_cell(a, g, cnd, cnd != kNull ? K_CAND : K_EMPTY);
        smmo_delete(h, self);
      }
    }
  }
};

// ================================================================ export
// Writes every agent into dense per-cell arrays (kind/age/energy/state) and
// counts agents per cell; an agent whose cell does not point back at it is
// counted as an error.
struct Export {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint32_t off = c == a.fish ? a.f_cell : c == a.shark ? a.s_cell : c == a.alive ? a.a_cell : a.c_cell;
    const uint32_t g = *fld<int32_t>(h, self, off);
    atomicAdd(a.out_count + g, 1u);
    if (*a.cells.col<uint32_t>(g, a.occ_off) != self) atomicAdd(a.errors, 1ull);
    if (c == a.fish) {
      a.out_kind[g] = 1;
      a.out_age[g] = *fld<int16_t>(h, self, a.f_age);
      a.out_energy[g] = 0;
    } else if (c == a.shark) {
      a.out_kind[g] = 2;
      a.out_age[g] = *fld<int16_t>(h, self, a.s_age);
      a.out_energy[g] = *fld<int16_t>(h, self, a.s_energy);
    } else if (c == a.alive) {
      a.out_kind[g] = 1;
      a.out_age[g] = (int16_t)*fld<uint16_t>(h, self, a.a_blocked);
      a.out_state[g] = *fld<uint8_t>(h, self, a.a_isnew);
    } else {
      a.out_kind[g] = 2;
      a.out_state[g] = 0;
    }
  }
};

// Export variant for smmo_world_export_noalloc: instead of a per-cell agent
// count it sets one bit per cell in a fixed scratch bitmap; finding the bit
// already set means a second agent on the cell (one error per extra agent,
// the same total as the counting export).
struct ExportBits {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint32_t off = c == a.fish ? a.f_cell : c == a.shark ? a.s_cell : c == a.alive ? a.a_cell : a.c_cell;
    const uint32_t g = *fld<int32_t>(h, self, off);
    const uint32_t bit = 1u << (g & 31);
    if (atomicOr(a.seen + (g >> 5), bit) & bit) atomicAdd(a.errors, 1ull);
    if (*a.cells.col<uint32_t>(g, a.occ_off) != self) atomicAdd(a.errors, 1ull);
    if (c == a.fish) {
      a.out_kind[g] = 1;
      a.out_age[g] = *fld<int16_t>(h, self, a.f_age);
      a.out_energy[g] = 0;
    } else if (c == a.shark) {
      a.out_kind[g] = 2;
      a.out_age[g] = *fld<int16_t>(h, self, a.s_age);
      a.out_energy[g] = *fld<int16_t>(h, self, a.s_energy);
    } else if (c == a.alive) {
      a.out_kind[g] = 1;
      a.out_age[g] = (int16_t)*fld<uint16_t>(h, self, a.a_blocked);
      a.out_state[g] = *fld<uint8_t>(h, self, a.a_isnew);
    } else {
      a.out_kind[g] = 2;
      a.out_state[g] = 0;
    }
  }
};

// Kind byte of the cell of agent `self` of class c.
__device__ __forceinline__ uint8_t kind_code(const HeapView& h, const WorldArgs& a, uint32_t c, uint32_t self) {
  if (c == a.fish || c == a.shark) return K_EMPTY;  // Wa-Tor keeps no kind bytes
  if (c == a.cand) return K_CAND;
  if (*fld<uint16_t>(h, self, a.a_blocked)) return K_BLOCK;
  return *fld<uint8_t>(h, self, a.a_isnew) ? K_NEW : K_ALIVE;
}

// Initial back-references: every agent writes its handle and kind into its
// cell.
struct Link {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint32_t off = c == a.fish ? a.f_cell : c == a.shark ? a.s_cell : c == a.alive ? a.a_cell : a.c_cell;
    set_cell(a, *fld<int32_t>(h, self, off), self, kind_code(h, a, c, self));
  }
};

// Occupied cells whose agent does not live on them, and cells whose kind
// byte disagrees with their occupant, count as errors.
struct CheckCells {
  using Args = WorldArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t, uint32_t self) {
    const uint32_t g = a.cells.cell_of(self);
    const uint32_t o = *a.cells.col<uint32_t>(g, a.occ_off);
    const uint8_t k = *a.cells.col<uint8_t>(g, a.kind_off);
    if (o == kNull) {
      if (k != K_EMPTY) atomicAdd(a.errors, 1ull);
      return;
    }
    const uint32_t t = type_of(h, o);
    if (t >= (uint32_t)h.num_classes) { atomicAdd(a.errors, 1ull); return; }
    uint32_t off = t == a.fish ? a.f_cell : t == a.shark ? a.s_cell : t == a.alive ? a.a_cell : a.c_cell;
    if ((uint32_t)*fld<int32_t>(h, o, off) != g || k != kind_code(h, a, t, o)) atomicAdd(a.errors, 1ull);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_wator[] = {
    SMMO_METHOD("wator.fish_prepare", FishPrepare), SMMO_METHOD("wator.fish_update", FishUpdate),
    SMMO_METHOD("wator.shark_prepare", SharkPrepare), SMMO_METHOD("wator.shark_update", SharkUpdate),
    SMMO_METHOD("world.export", Export), SMMO_METHOD("world.link", Link),
    SMMO_METHOD("world.check_cells", CheckCells)};
const int g_methods_wator_n = sizeof(g_methods_wator) / sizeof(g_methods_wator[0]);

const smmo::MethodEntry g_methods_gol[] = {
    SMMO_METHOD("gol.candidate_prepare", CandPrepare), SMMO_METHOD("gol.alive_prepare", AlivePrepare),
    SMMO_METHOD("gol.candidate_update", CandUpdate), SMMO_METHOD("gol.alive_update", AliveUpdate)};
const int g_methods_gol_n = sizeof(g_methods_gol) / sizeof(g_methods_gol[0]);

// ================================================================ world API
struct smmo_world {
  smmo_heap* heap = nullptr;
  int n_inst = 0;
  std::vector<int> kind;
  std::vector<uint32_t> W, H, base;
  uint64_t total_cells = 0;
  int cls_cell = -1, cls_wagent = -1, cls_fish = -1, cls_shark = -1;
  int cls_lagent = -1, cls_alive = -1, cls_cand = -1;
  uint32_t nw = 0, nl = 0;  // Wa-Tor and Life instances
  uint32_t t = 0;  // steps done
  uint32_t* d_t = nullptr;  // device step counter, followed by the barrier words of the fused phases
  int step_kernels = SMMO_WATOR_FOUR_DO_ALLS;  // how a Wa-Tor iteration is launched
  uint32_t* d_queue = nullptr;  // queued creations: items, then one hint per 32 items
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  WorldArgs args{};
  smmo_wator_params p{};
};

namespace {
// Optional per-phase timing: events recorded on the launching stream.
struct PhaseTimer {
  std::vector<cudaEvent_t> ev;  // 3 per pdo: before enum, between, after
  std::vector<int> phase;
  int64_t launches = 0;
};

// Opens a step: t <- t + 1, and clears the grid-barrier words of the
// step's two fused Wa-Tor launches (2 x kBarrierWords, behind t) and the
// two creation-queue counters (one more word behind them).
__global__ void k_world_step_begin(uint32_t* t, unsigned long long* ctl) {
  if (threadIdx.x == 0) *t += 1;
  for (int i = threadIdx.x; i < 2 * kBarrierWords + 1; i += blockDim.x) ctl[i] = 0ull;
}

unsigned long long* world_ctl(const smmo_world* w) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<uint8_t*>(w->d_t) + 256);
}

// reuse = the previous do-all enumerated the same concrete class and did
// not create or delete objects of it, so its snapshot is still exact
int pdo(smmo_world* w, int cls, method_launch_fn fn, const WorldArgs& a, cudaStream_t s,
        PhaseTimer* pt = nullptr, int phase = 0, bool reuse = false) {
  std::vector<int> cl;
  concrete_subtree(w->heap, cls, &cl);
  for (int k : cl) {
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (pt) {
      cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
      cudaEventRecord(e0, s);
    }
    int st = (reuse && cl.size() == 1) ? SMMO_OK : enumerate(w->heap, k, s);
    if (pt) cudaEventRecord(e1, s);
    if (!st) st = fn(w->heap, k, &a, s);
    if (pt) {
      cudaEventRecord(e2, s);
      pt->ev.push_back(e0); pt->ev.push_back(e1); pt->ev.push_back(e2);
      pt->phase.push_back(phase);
      pt->launches += (reuse && cl.size() == 1) ? 1 : 2;
    }
    if (st) return st;
  }
  return SMMO_OK;
}

int world_steps(smmo_world* w, int nsteps, cudaStream_t s, PhaseTimer* pt) {
  WorldArgs a = w->args;
  for (int k = 0; k < nsteps; ++k) {
    ++w->t;
    k_world_step_begin<<<1, 128, 0, s>>>(w->d_t, world_ctl(w));
    if (pt) pt->launches += 1;
    int st = cuda_status(cudaGetLastError());
    if (w->nl) {  // one Life generation (Sec. 7.8, four do-alls)
      st = pdo(w, w->cls_cand, &launch_do_all<CandPrepare>, a, s, pt, 0);
      if (!st) st = pdo(w, w->cls_alive, &launch_do_all<AlivePrepare>, a, s, pt, 1);
      if (!st) st = pdo(w, w->cls_cand, &launch_do_all<CandUpdate>, a, s, pt, 2);
      if (!st) st = pdo(w, w->cls_alive, &launch_do_all<AliveUpdate>, a, s, pt, 3);
    }
    const int mode = w->step_kernels;
    if (!st && w->nw && (mode & 3) != SMMO_WATOR_FOUR_DO_ALLS) {
      // one Wa-Tor iteration, each phase (prepare + update) in one launch
      // (world_modes.cu), the creations after it when they are queued
      method_launch_fn fc = wator_mode_launcher(kWFishCreate, mode), sc = wator_mode_launcher(kWSharkCreate, mode);
      a.phase = 0;
      a.ctl = world_ctl(w);
      st = pdo(w, w->cls_fish, wator_mode_launcher(kWFishPrepare, mode), a, s, pt, 4);
      if (!st && fc) st = pdo(w, w->cls_fish, fc, a, s, pt, 4, true);
      a.phase = 1;
      a.ctl = world_ctl(w) + kBarrierWords;
      if (!st) st = pdo(w, w->cls_shark, wator_mode_launcher(kWSharkPrepare, mode), a, s, pt, 6);
      if (!st && sc) st = pdo(w, w->cls_shark, sc, a, s, pt, 6, true);
    } else if (!st && w->nw) {  // one Wa-Tor iteration (Sec. 7.6): fish phase, shark phase
      // the four plain do-alls here; marked, filtered and queued variants
      // from world_modes.cu
      method_launch_fn fp = wator_mode_launcher(kWFishPrepare, mode), sp = wator_mode_launcher(kWSharkPrepare, mode);
      method_launch_fn fu = wator_mode_launcher(kWFishUpdate, mode), su = wator_mode_launcher(kWSharkUpdate, mode);
      method_launch_fn fc = wator_mode_launcher(kWFishCreate, mode), sc = wator_mode_launcher(kWSharkCreate, mode);
      if (!fp) fp = &launch_do_all<FishPrepare>;
      if (!sp) sp = &launch_do_all<SharkPrepare>;
      if (!fu) fu = &launch_do_all<FishUpdate>;
      if (!su) su = &launch_do_all<SharkUpdate>;
      a.phase = 0;
      st = pdo(w, w->cls_fish, fp, a, s, pt, 4);
      if (!st) st = pdo(w, w->cls_fish, fu, a, s, pt, 5, true);
      if (!st && fc) st = pdo(w, w->cls_fish, fc, a, s, pt, 5, true);
      a.phase = 1;
      if (!st) st = pdo(w, w->cls_shark, sp, a, s, pt, 6);
      if (!st) st = pdo(w, w->cls_shark, su, a, s, pt, 7, true);
      if (!st && sc) st = pdo(w, w->cls_shark, sc, a, s, pt, 7, true);
    }
    if (st) return st;
  }
  return SMMO_OK;
}
// ----------------------------------------------------------- world creation
// The agents of the initial state, gathered on the device: a class code per
// cell (0 none, 1 Fish, 2 Shark, 3 Alive, 4 Candidate, from the kind of the
// cell's instance and init_kind), counted per chunk of kGatherChunk cells,
// scanned, and scattered in ascending cell order into the SOA columns of
// each class, so that bulk creation places the objects exactly as a host
// loop over the cells would.
constexpr uint32_t kGatherChunk = 1024;  // 256 threads x 4 cells

__device__ __forceinline__ int agent_code(const Inst* tab, uint32_t n_inst, const int8_t* kind, uint64_t g) {
  const int k = kind[g];
  if (k != 1 && k != 2) return 0;
  return instance_at(tab, n_inst, (uint32_t)g)->kind == SMMO_WORLD_WATOR ? k : 2 + k;
}

__global__ void __launch_bounds__(256) k_agent_count(const Inst* tab, uint32_t n_inst, const int8_t* kind, uint64_t N,
                                                     uint32_t* counts, uint32_t nchunks) {
  __shared__ uint32_t c[4];
  if (threadIdx.x < 4) c[threadIdx.x] = 0u;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kGatherChunk;
  for (int r = 0; r < 4; ++r) {
    const uint64_t g = base + (uint64_t)r * 256u + threadIdx.x;
    if (g < N) {
      const int code = agent_code(tab, n_inst, kind, g);
      if (code) atomicAdd(&c[code - 1], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) counts[(size_t)threadIdx.x * nchunks + blockIdx.x] = c[threadIdx.x];
}

// Exclusive scan of each code's chunk counts in place (one CTA); totals in tot.
__global__ void __launch_bounds__(1024) k_agent_scan(uint32_t* counts, uint32_t nchunks, uint32_t* tot) {
  __shared__ uint32_t sc[1024];
  for (int code = 0; code < 4; ++code) {
    uint32_t* cc = counts + (size_t)code * nchunks;
    uint32_t run = 0;
    for (uint32_t b0 = 0; b0 < nchunks; b0 += 1024) {
      const uint32_t i = b0 + threadIdx.x;
      const uint32_t v = i < nchunks ? cc[i] : 0u;
      sc[threadIdx.x] = v;
      __syncthreads();
      for (uint32_t o = 1; o < 1024; o <<= 1) {
        const uint32_t x = threadIdx.x >= o ? sc[threadIdx.x - o] : 0u;
        __syncthreads();
        sc[threadIdx.x] += x;
        __syncthreads();
      }
      if (i < nchunks) cc[i] = run + sc[threadIdx.x] - v;
      run += sc[1023];
      __syncthreads();
    }
    if (threadIdx.x == 0) tot[code] = run;
    __syncthreads();
  }
}

struct AgentCols {
  int32_t* cell[4];    // Fish, Shark, Alive, Candidate
  int32_t* target[2];  // Fish, Shark
  int16_t* age[2];     // Fish, Shark
  int16_t* energy;     // Shark
  uint8_t* act[2];     // Alive, Candidate
  uint8_t* isnew;      // Alive
  uint16_t* blocked;   // Alive
};

__global__ void __launch_bounds__(256) k_agent_scatter(const Inst* tab, uint32_t n_inst, const int8_t* kind,
                                                       const int16_t* age, const int16_t* energy,
                                                       const uint8_t* state, uint64_t N, const uint32_t* offs,
                                                       uint32_t nchunks, AgentCols c) {
  __shared__ uint32_t wsum[4][8], run[4];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 4) run[threadIdx.x] = offs[(size_t)threadIdx.x * nchunks + blockIdx.x];
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kGatherChunk;
  for (int r = 0; r < 4; ++r) {
    const uint64_t g = base + (uint64_t)r * 256u + threadIdx.x;
    const int code = g < N ? agent_code(tab, n_inst, kind, g) : 0;
    uint32_t rank = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, code == k + 1);
      if (code == k + 1) rank = __popc(m & ((1u << lane) - 1));
      if (lane == 0) wsum[k][w] = __popc(m);
    }
    __syncthreads();
    if (code) {
      const int k = code - 1;
      uint32_t pos = run[k] + rank;
      for (uint32_t v = 0; v < w; ++v) pos += wsum[k][v];
      const int16_t a0 = age ? age[g] : (int16_t)0;
      c.cell[k][pos] = (int32_t)g;
      if (k < 2) {
        c.target[k][pos] = (int32_t)g;
        c.age[k][pos] = a0;
        if (k == 1) c.energy[pos] = energy ? energy[g] : (int16_t)0;
      } else {
        c.act[k - 2][pos] = 0;
        if (k == 2) {
          c.isnew[pos] = state ? state[g] : (uint8_t)0;
          c.blocked[pos] = (uint16_t)a0;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      uint32_t t = 0;
      for (int v = 0; v < 8; ++v) t += wsum[threadIdx.x][v];
      run[threadIdx.x] += t;
    }
    __syncthreads();
  }
}

// Agents with more than one agent on their cell: sum of (count - 1) over the
// cells (the allocating export's duplicate count), warp-aggregated.
__global__ void k_count_extra(const uint32_t* cnt, uint64_t N, unsigned long long* err) {
  unsigned long long extra = 0;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (uint64_t)gridDim.x * blockDim.x)
    if (cnt[g] > 1u) extra += cnt[g] - 1u;
#pragma unroll
  for (int o = 16; o; o >>= 1) extra += __shfl_xor_sync(0xFFFFFFFFu, extra, o);
  if ((threadIdx.x & 31) == 0 && extra) atomicAdd(err, extra);
}
}  // namespace

extern "C" {

int smmo_world_create_batch(smmo_heap* heap, const smmo_instance_desc* inst, int n_inst, uint64_t seed,
                            const smmo_wator_params* params, const int8_t* init_kind, const int16_t* init_age,
                            const int16_t* init_energy, const uint8_t* init_state, void* stream,
                            smmo_world** out) {
  if (!heap || n_inst < 1 || !inst || !init_kind || !out) return SMMO_E_INVALID_ARG;
  if (!heap->classes.empty() || heap->frozen) return SMMO_E_FROZEN;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t total = 0;
  for (int i = 0; i < n_inst; ++i) {
    const smmo_instance_desc& d = inst[i];
    if ((d.kind != SMMO_WORLD_LIFE && d.kind != SMMO_WORLD_WATOR) || d.W < 3 || d.H < 3) return SMMO_E_INVALID_ARG;
    if (d.base != total || d.count != (uint64_t)d.W * d.H) return SMMO_E_INVALID_ARG;
    total += d.count;
    if (total > kCellMask - 1ull) return SMMO_E_INVALID_ARG;  // cells below 2^30 - 2
  }
  int st = smmo_batch_define(heap, inst, n_inst);  // the heap owns the instance table
  if (st) return st;
  smmo_world* w = new smmo_world();
  w->heap = heap;
  w->n_inst = n_inst;
  w->p.fish_breed = 4; w->p.shark_breed = 12; w->p.starve = 3; w->p.breed_strict = 0;
  if (params) w->p = *params;
  for (int i = 0; i < n_inst; ++i) {
    w->kind.push_back(inst[i].kind);
    w->W.push_back(inst[i].W);
    w->H.push_back(inst[i].H);
    w->base.push_back((uint32_t)inst[i].base);
    (inst[i].kind == SMMO_WORLD_WATOR ? w->nw : w->nl) += 1;
  }
  w->total_cells = total;
  // classes
  smmo_field_desc cell_f[3] = {{"occ", SMMO_HANDLE, 1, -1}, {"req", SMMO_U32, 1, -1}, {"kind", SMMO_U8, 1, -1}};
  st = smmo_class_register(heap, "Cell", cell_f, 3, -1, 0, &w->cls_cell);
  if (!st && w->nw) {
    smmo_field_desc ag[2] = {{"cell", SMMO_I32, 1, -1}, {"target", SMMO_I32, 1, -1}};
    smmo_field_desc fi[1] = {{"age", SMMO_I16, 1, -1}};
    smmo_field_desc sh[2] = {{"age", SMMO_I16, 1, -1}, {"energy", SMMO_I16, 1, -1}};
    st = smmo_class_register(heap, "WAgent", ag, 2, -1, 1, &w->cls_wagent);
    if (!st) st = smmo_class_register(heap, "Fish", fi, 1, w->cls_wagent, 0, &w->cls_fish);
    if (!st) st = smmo_class_register(heap, "Shark", sh, 2, w->cls_wagent, 0, &w->cls_shark);
  }
  if (!st && w->nl) {
    smmo_field_desc ag[2] = {{"cell", SMMO_I32, 1, -1}, {"action", SMMO_U8, 1, -1}};
    smmo_field_desc al[2] = {{"is_new", SMMO_U8, 1, -1}, {"blocked", SMMO_U16, 1, -1}};
    st = smmo_class_register(heap, "LAgent", ag, 2, -1, 1, &w->cls_lagent);
    if (!st) st = smmo_class_register(heap, "Alive", al, 2, w->cls_lagent, 0, &w->cls_alive);
    if (!st) st = smmo_class_register(heap, "Candidate", nullptr, 0, w->cls_lagent, 0, &w->cls_cand);
  }
  // 768 bytes: Cell (9 bytes), Fish, Shark and the Life agents get N_T = 64
  if (heap->cfg.block_data_bytes == 0) heap->cfg.block_data_bytes = 768;
  if (!st) st = freeze(heap, s);
  if (!st && heap->classes[w->cls_cell].layout.cap != 64 && heap->classes[w->cls_cell].layout.cap != 32)
    st = SMMO_E_UNSUPPORTED;  // dense cell addressing needs N = 32 or 64
  if (st) { delete w; return st; }
  // the step counter (the instance table is the heap's)
  const size_t tbytes = 256 + (2 * kBarrierWords + 1) * sizeof(unsigned long long);
  cudaError_t e = cudaMalloc(&w->d_t, tbytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_t, 0, tbytes, s);
  // creation queue of the Wa-Tor updates: at most one creation per agent
  // (agents <= cells), plus a partly filled chunk per warp of the grid
  uint32_t qcap = 0;
  if (e == cudaSuccess && w->nw) {
    qcap = (uint32_t)(((total + 32ull * (uint64_t)heap->num_sms * 64ull) + 31ull) & ~31ull);
    e = cudaMalloc(&w->d_queue, (size_t)qcap * 4 + (size_t)(qcap / 32) * 4);
  }
  if (e != cudaSuccess) { smmo_world_destroy(w); return cuda_status(e); }
  // cells: occ = null, req = all ones (above every key), kind = empty
  const uint64_t N = w->total_cells;
  uint32_t* ones = nullptr;
  uint8_t* zeros = nullptr;
  e = cudaMallocAsync(&ones, N * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&zeros, N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ones, 0xFF, N * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(zeros, 0, N, s);
  if (e != cudaSuccess) { smmo_world_destroy(w); return cuda_status(e); }
  const void* csrc[3] = {ones, ones, zeros};
  int64_t first = -1;
  st = smmo_bulk_new(heap, w->cls_cell, (int64_t)N, csrc, nullptr, &first, stream);
  cudaFreeAsync(ones, s);
  cudaFreeAsync(zeros, s);
  if (!st && first < 0) st = SMMO_E_OOM;  // cells must be contiguous
  if (st) { smmo_world_destroy(w); return st; }
  // argument block
  WorldArgs& a = w->args;
  memset(&a, 0, sizeof(a));
  a.cells.data = heap->view.data;
  a.cells.block_bytes = heap->view.block_bytes;
  a.cells.b0 = (uint32_t)first;
  a.cells.shift = heap->classes[w->cls_cell].layout.cap == 64 ? 6 : 5;
  a.tp = w->d_t;
  const ClassLayout& CL = heap->classes[w->cls_cell].layout;
  a.occ_off = CL.col_off[0];
  a.req_off = CL.col_off[1];
  a.kind_off = CL.col_off[2];
  a.fish = a.shark = a.alive = a.cand = kNull;
  if (w->nw) {
    const ClassLayout& F = heap->classes[w->cls_fish].layout;
    const ClassLayout& S = heap->classes[w->cls_shark].layout;
    a.fish = w->cls_fish; a.shark = w->cls_shark;
    a.f_cell = F.col_off[0]; a.f_target = F.col_off[1]; a.f_age = F.col_off[2];
    a.s_cell = S.col_off[0]; a.s_target = S.col_off[1]; a.s_age = S.col_off[2]; a.s_energy = S.col_off[3];
  }
  if (w->nl) {
    const ClassLayout& A = heap->classes[w->cls_alive].layout;
    const ClassLayout& C = heap->classes[w->cls_cand].layout;
    a.alive = w->cls_alive; a.cand = w->cls_cand;
    a.a_cell = A.col_off[0]; a.a_action = A.col_off[1]; a.a_isnew = A.col_off[2];
    a.a_blocked = A.col_off[3];
    a.c_cell = C.col_off[0]; a.c_action = C.col_off[1];
  }
  if (w->d_queue) {
    uint32_t* qcnt = reinterpret_cast<uint32_t*>(world_ctl(w) + 2 * kBarrierWords);
    a.fq.item = w->d_queue;
    a.fq.hint = w->d_queue + qcap;
    a.fq.cap = qcap;
    a.fq.count = qcnt;
    a.sq = a.fq;
    a.sq.count = qcnt + 1;
  }
  a.seed = seed;
  a.survive = (1u << 2) | (1u << 3);  // Life until smmo_world_set_life_rule
  a.born = 1u << 3;
  a.block = 0;
  a.fish_breed = w->p.fish_breed; a.shark_breed = w->p.shark_breed; a.starve = w->p.starve;
  a.breed_strict = w->p.breed_strict;
  // agents: gathered per class on the device in ascending cell order (see
  // k_agent_scatter), then created by one bulk creation per class
  const uint32_t nchunks = (uint32_t)((N + kGatherChunk - 1) / kGatherChunk);
  uint32_t* counts = nullptr;
  uint32_t tot[4] = {0, 0, 0, 0};
  e = cudaMallocAsync(&counts, ((size_t)4 * nchunks + 4) * sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    k_agent_count<<<nchunks, 256, 0, s>>>(heap->d_inst, (uint32_t)n_inst, init_kind, N, counts, nchunks);
    k_agent_scan<<<1, 1024, 0, s>>>(counts, nchunks, counts + (size_t)4 * nchunks);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tot, counts + (size_t)4 * nchunks, sizeof(tot), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  AgentCols cols;
  memset(&cols, 0, sizeof(cols));
  std::vector<void*> tmp;
  auto col = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (e == cudaSuccess && bytes) e = cudaMallocAsync(&q, bytes, s);
    if (q) tmp.push_back(q);
    return q;
  };
  for (int k = 0; k < 4; ++k) cols.cell[k] = (int32_t*)col((size_t)tot[k] * 4);
  for (int k = 0; k < 2; ++k) {
    cols.target[k] = (int32_t*)col((size_t)tot[k] * 4);
    cols.age[k] = (int16_t*)col((size_t)tot[k] * 2);
    cols.act[k] = (uint8_t*)col((size_t)tot[2 + k]);
  }
  cols.energy = (int16_t*)col((size_t)tot[1] * 2);
  cols.isnew = (uint8_t*)col((size_t)tot[2]);
  cols.blocked = (uint16_t*)col((size_t)tot[2] * 2);
  if (e == cudaSuccess) {
    k_agent_scatter<<<nchunks, 256, 0, s>>>(heap->d_inst, (uint32_t)n_inst, init_kind, init_age, init_energy,
                                            init_state, N, counts, nchunks, cols);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) st = cuda_status(e);
  auto create = [&](int cls, std::vector<const void*> src, uint32_t n) -> int {
    if (n == 0) return SMMO_OK;
    return smmo_bulk_new(heap, cls, (int64_t)n, src.data(), nullptr, nullptr, stream);
  };
  if (!st && w->nw) {
    st = create(w->cls_fish, {cols.cell[0], cols.target[0], cols.age[0]}, tot[0]);
    if (!st) st = create(w->cls_shark, {cols.cell[1], cols.target[1], cols.age[1], cols.energy}, tot[1]);
  }
  if (!st && w->nl) {
    st = create(w->cls_alive, {cols.cell[2], cols.act[0], cols.isnew, cols.blocked}, tot[2]);
    if (!st) st = create(w->cls_cand, {cols.cell[3], cols.act[1]}, tot[3]);
  }
  for (void* q : tmp) cudaFreeAsync(q, s);
  if (counts) cudaFreeAsync(counts, s);
  if (!st && w->nw) st = pdo(w, w->cls_wagent, &launch_do_all<Link>, a, s);
  if (!st && w->nl) st = pdo(w, w->cls_lagent, &launch_do_all<Link>, a, s);
  if (!st) { e = cudaStreamSynchronize(s); if (e != cudaSuccess) st = cuda_status(e); }
  if (st) { smmo_world_destroy(w); return st; }
  *out = w;
  return SMMO_OK;
}

int smmo_world_create(smmo_heap* heap, int n_inst, const int* kind, const uint32_t* W,
                      const uint32_t* H, uint64_t seed, const smmo_wator_params* params,
                      const int8_t* init_kind, const int16_t* init_age, const int16_t* init_energy,
                      const uint8_t* init_state, void* stream, smmo_world** out) {
  if (!heap || n_inst < 1 || !kind || !W || !H) return SMMO_E_INVALID_ARG;
  std::vector<smmo_instance_desc> d(n_inst);
  uint64_t base = 0;
  for (int i = 0; i < n_inst; ++i) {
    memset(&d[i], 0, sizeof(d[i]));
    d[i].kind = kind[i];
    d[i].id = (uint32_t)i;
    d[i].W = W[i];
    d[i].H = H[i];
    d[i].base = base;
    d[i].count = (uint64_t)W[i] * H[i];
    base += d[i].count;
  }
  return smmo_world_create_batch(heap, d.data(), n_inst, seed, params, init_kind, init_age, init_energy,
                                 init_state, stream, out);
}

int smmo_world_step(smmo_world* w, int nsteps, void* stream) {
  if (!w || nsteps < 0) return SMMO_E_INVALID_ARG;
  return world_steps(w, nsteps, (cudaStream_t)stream, nullptr);
}

int smmo_world_set_life_rule(smmo_world* w, uint32_t survive, uint32_t born, uint32_t block) {
  if (!w || survive >= (1u << 9) || born >= (1u << 9) || block > 65535u) return SMMO_E_INVALID_ARG;
  if ((born & 1u) != 0) return SMMO_E_INVALID_ARG;  // birth with no alive neighbour: candidates would be deleted
  w->args.survive = survive;
  w->args.born = born;
  w->args.block = block;
  if (w->graph) { cudaGraphExecDestroy(w->graph); w->graph = nullptr; }  // captured with the old rule
  return SMMO_OK;
}

int smmo_world_set_step_kernels(smmo_world* w, int mode) {
  if (!w || mode < 0 || (mode & ~(3 | SMMO_WATOR_QUEUED_CREATION | SMMO_WATOR_MARKED_UPDATE)) || (mode & 3) == 3 ||
      ((mode & SMMO_WATOR_MARKED_UPDATE) && (mode & 3)))
    return SMMO_E_INVALID_ARG;
  w->step_kernels = mode;
  if (w->graph) { cudaGraphExecDestroy(w->graph); w->graph = nullptr; }  // captured with the old kernels
  return SMMO_OK;
}

int smmo_world_capture(smmo_world* w, int nsteps, void* stream) {
  if (!w || nsteps < 1 || !stream) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (w->graph) { cudaGraphExecDestroy(w->graph); w->graph = nullptr; }
  const uint32_t t_save = w->t;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  int st = world_steps(w, nsteps, s, nullptr);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  w->t = t_save;  // capturing does not run the steps
  if (st) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&w->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { w->graph = nullptr; return cuda_status(e); }
  w->graph_steps = nsteps;
  return SMMO_OK;
}

int smmo_world_replay(smmo_world* w, void* stream) {
  if (!w || !w->graph) return SMMO_E_INVALID_ARG;
  cudaError_t e = cudaGraphLaunch(w->graph, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e);
  w->t += (uint32_t)w->graph_steps;
  return SMMO_OK;
}

int smmo_world_step_profiled(smmo_world* w, int nsteps, double* phase_ms, double* step_ms,
                             int64_t* launches, void* stream) {
  if (!w || nsteps < 0 || !phase_ms) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PhaseTimer pt;
  std::vector<cudaEvent_t> se;  // begin/end event of every step
  int st = SMMO_OK;
  for (int k = 0; k < nsteps && !st; ++k) {
    cudaEvent_t b, e;
    cudaEventCreate(&b);
    cudaEventCreate(&e);
    cudaEventRecord(b, s);
    st = world_steps(w, 1, s, &pt);
    cudaEventRecord(e, s);
    se.push_back(b);
    se.push_back(e);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  for (size_t i = 0; i < pt.phase.size(); ++i) {
    float m1 = 0, m2 = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m1, pt.ev[3 * i], pt.ev[3 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m2, pt.ev[3 * i + 1], pt.ev[3 * i + 2]);
    phase_ms[2 * pt.phase[i]] += m1;
    phase_ms[2 * pt.phase[i] + 1] += m2;
  }
  for (size_t i = 0; i + 1 < se.size(); i += 2) {
    float m = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m, se[i], se[i + 1]);
    if (step_ms) *step_ms += m;
  }
  for (cudaEvent_t ev : pt.ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : se) cudaEventDestroy(ev);
  if (launches) *launches += pt.launches;
  if (st) return st;
  return cuda_status(e);
}

int smmo_world_export(smmo_world* w, int8_t* kind, int16_t* age, int16_t* energy, uint8_t* state,
                      int64_t* errors, void* stream) {
  if (!w || !kind || !age || !energy || !state) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t N = w->total_cells;
  WorldArgs a = w->args;
  uint32_t* cnt = nullptr;
  unsigned long long* err = nullptr;
  cudaError_t e = cudaMallocAsync(&cnt, N * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&err, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, N * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(kind, 0, N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(age, 0, N * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(energy, 0, N * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, N, s);
  if (e != cudaSuccess) return cuda_status(e);
  a.out_kind = kind; a.out_age = age; a.out_energy = energy; a.out_state = state;
  a.out_count = cnt; a.errors = err;
  int st = SMMO_OK;
  if (w->nw) st = pdo(w, w->cls_wagent, &launch_do_all<Export>, a, s);
  if (!st && w->nl) st = pdo(w, w->cls_lagent, &launch_do_all<Export>, a, s);
  if (!st) st = pdo(w, w->cls_cell, &launch_do_all<CheckCells>, a, s);
  // agents beyond the first on a cell, counted on the device
  unsigned long long herr = 0;
  if (!st) {
    k_count_extra<<<w->heap->num_sms * 8, 256, 0, s>>>(cnt, N, err);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(err, s);
  if (st) return st;
  if (errors) *errors = (int64_t)herr;
  return SMMO_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free export.  Its scratch is this fixed array, part of the
// library image, so every GPU that loads the library holds it until exit:
// 8 bytes of error counter (padded to 256) and one bit per cell for
// SMMO_EXPORT_NOALLOC_MAX_CELLS cells (2 MiB).  Host code cannot use the
// array's name as a device address; the address is looked up once per
// device with cudaGetSymbolAddress (first call on that device).
}  // extern "C"

namespace {
struct NoAllocScratch {
  unsigned long long errors;
  unsigned long long pad[31];
  uint32_t seen[SMMO_EXPORT_NOALLOC_MAX_CELLS / 32];
};
static __device__ __align__(256) NoAllocScratch g_export_scratch;

std::mutex g_scratch_mu;
NoAllocScratch* g_scratch_addr[256];  // per device ordinal, set on first use

int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 256) return SMMO_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_export_scratch);
    if (e != cudaSuccess) return cuda_status(e);
    g_scratch_addr[dev] = (NoAllocScratch*)p;
  }
  *out = g_scratch_addr[dev];
  return SMMO_OK;
}
}  // namespace

extern "C" {

int smmo_world_export_noalloc(smmo_world* w, int8_t* kind, int16_t* age, int16_t* energy,
                              uint8_t* state, int64_t* errors, void* stream) {
  if (!w || !kind || !age || !energy || !state || !errors) return SMMO_E_INVALID_ARG;
  const uint64_t N = w->total_cells;
  if (N > SMMO_EXPORT_NOALLOC_MAX_CELLS) return SMMO_E_UNSUPPORTED;
  NoAllocScratch* scr = nullptr;
  int st = scratch_for_current_device(&scr);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear what must start at 0
  cudaError_t e = cudaMemsetAsync(&scr->errors, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scr->seen, 0, (N + 31) / 32 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(kind, 0, N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(age, 0, N * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(energy, 0, N * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, N, s);
  if (e != cudaSuccess) return cuda_status(e);
  WorldArgs a = w->args;
  a.out_kind = kind; a.out_age = age; a.out_energy = energy; a.out_state = state;
  a.out_count = nullptr;
  a.errors = &scr->errors;
  a.seen = scr->seen;
  if (w->nw) st = pdo(w, w->cls_wagent, &launch_do_all<ExportBits>, a, s);
  if (!st && w->nl) st = pdo(w, w->cls_lagent, &launch_do_all<ExportBits>, a, s);
  if (!st) st = pdo(w, w->cls_cell, &launch_do_all<CheckCells>, a, s);
  if (st) return st;
  unsigned long long herr = 0;
  e = cudaMemcpyAsync(&herr, &scr->errors, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *errors = (int64_t)herr;
  return SMMO_OK;
}

int smmo_world_info(smmo_world* w, int64_t* total_cells, int* class_ids, uint32_t* steps_done) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (total_cells) *total_cells = (int64_t)w->total_cells;
  if (class_ids) {
    const int ids[7] = {w->cls_cell, w->cls_wagent, w->cls_fish, w->cls_shark, w->cls_lagent, w->cls_alive, w->cls_cand};
    memcpy(class_ids, ids, sizeof(ids));
  }
  if (steps_done) *steps_done = w->t;
  return SMMO_OK;
}

int smmo_world_destroy(smmo_world* w) {
  if (!w) return SMMO_E_INVALID_ARG;
  if (w->graph) cudaGraphExecDestroy(w->graph);
  if (w->d_t) cudaFree(w->d_t);
  if (w->d_queue) cudaFree(w->d_queue);
  delete w;
  return SMMO_OK;
}

}  // extern "C"
