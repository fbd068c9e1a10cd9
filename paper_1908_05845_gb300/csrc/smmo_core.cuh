// smmo_core.cuh -- device-side core of the SMMO heap (sm_103a).
//
// Heap layout (all inside the caller's buffer):
//   * per block: a 64-bit object allocation bitmap (alloc_bm) and a type id
//     (block_type); Sec. 5.2.1 "block structure".  The data segments of all
//     blocks form one array of M equal-size blocks, each holding the SOA
//     columns of up to N_T <= 64 objects of one class (Sec. 5.2).
//     Bitmaps and type ids live in their own arrays instead of a block
//     header, so enumeration and statistics read 8 bytes per block.
//   * hierarchical bitmaps (Sec. 5.3.1) of M bits: free, and per class
//     allocated[T], active[T], defrag[T].  All of them share one geometry
//     (levels of 64-bit containers until one container remains).
//   * a device state word block: error word, enumeration counter and
//     sharded event counters.
//
// Every loop that waits for another thread has a budget; on exhaustion it
// records SMMO_E_CONTENTION / SMMO_E_DEVICE_OOM in the state and gives up
// (the thesis' allocator loops forever on OOM, Alg. 5.1; that is not
// acceptable on a shared GPU).
#pragma once
#include <cstdint>

#include "smmo.h"

#define SMMO_MAX_COLS 32
// CTAs of 512 threads per SM that the do-all kernels are compiled for (the
// register cap: 65536 / (512 x this)); 3 gives 40 registers.
#ifndef SMMO_DOALL_MIN_CTAS
#define SMMO_DOALL_MIN_CTAS 3
#endif
// warp_new: the first nearby round that may end the search when its 32
// blocks have no free slot, and the number of missing slots from which the
// warp takes a fresh block instead of refilling one leader at a time
#ifndef SMMO_NEAR_STOP_FROM
#define SMMO_NEAR_STOP_FROM 2
#endif
#ifndef SMMO_FRESH_MIN
#define SMMO_FRESH_MIN 16
#endif
#define SMMO_MAX_LEVELS 6
#define SMMO_NSHARD 32
#define SMMO_CTR_SLOW 0
#define SMMO_CTR_RETRY 1
#define SMMO_CTR_ENUM_OBJ 34
#define SMMO_CTR_ENUM_BLK 35
#define SMMO_CTR_REFILL 36
#define SMMO_CTR_LOOKUP_MISS 37
#define SMMO_CTR_RESERVE_FAIL 38
#define SMMO_CTR_VISIT 39
#define SMMO_CTR_ALLOC(c) (2 + (c))
#define SMMO_CTR_FREE(c) (2 + SMMO_MAX_CLASSES + (c))
#define SMMO_NCTR (8 + 2 * SMMO_MAX_CLASSES)

namespace smmo {

constexpr uint32_t kNull = 0xFFFFFFFFu;
constexpr unsigned long long kAll = ~0ull;

struct ClassLayout {
  uint32_t cap;                       // N_T
  uint32_t ncols;
  unsigned long long capmask;         // low N_T bits set
  uint32_t dlimit;                    // defrag candidate iff fill <= dlimit
  int32_t inst_col;                   // column of the SMMO_INSTANCE field (-1: none)
  uint32_t col_off[SMMO_MAX_COLS];    // byte offset of each SOA column
  uint32_t col_size[SMMO_MAX_COLS];   // element size of each column
};

struct DeviceState {
  int err;
  int pad0;
  unsigned long long err_detail;
  uint32_t rcount;                    // enumeration result count
  uint32_t pad1;
  unsigned long long aux[6];          // per-call scratch counters
  unsigned long long stat_live[SMMO_MAX_CLASSES];
  unsigned long long stat_blocks[SMMO_MAX_CLASSES];
  unsigned long long stat_free_slots[SMMO_MAX_CLASSES];
  unsigned long long stat_free_blocks;
  unsigned long long pad2;
  unsigned long long ctr[SMMO_NSHARD][SMMO_NCTR];
};

// One row of a heap's instance table (smmo_batch_define): a problem
// instance whose objects share the heap with the other instances'.  The
// instances that own a range of a global numbering (the cells of the
// cellular worlds) are sorted by it, so an index finds its instance.
struct Inst {
  uint32_t cell_base;  // first index of the instance's range
  uint32_t W;
  uint32_t H;
  uint32_t id;         // instance number in the random counters
  uint64_t wdiv;       // floor((2^64 - 1) / W) + 1 (division by W), 0 if W = 0
  uint32_t count;      // length of the range
  int32_t kind;
  long long param[2];
};

// An enumerated block: its index, its class and the snapshot of its
// allocation bitmap (the thesis' "iteration bitmap", Sec. 5.2.1, carried
// with the index).
struct __align__(16) REntry {
  uint32_t block;
  uint32_t cls;
  unsigned long long bits;
};

struct HeapView {
  uint8_t* data;                      // block data segments
  unsigned long long* alloc_bm;       // per-block allocation bitmaps
  uint32_t* block_type;               // per-block class id
  unsigned long long* bitmaps;        // all hierarchical bitmaps
  DeviceState* st;
  const ClassLayout* cls;             // per-class layouts (device)
  REntry* R;                          // enumeration scratch
  uint32_t* rcnt;                     // its entry count (the heap's, or a saved snapshot's)
  uint32_t* umark;                    // per unit of R: slots marked by a marking do-all
  const Inst* inst;                   // instance table (null: no batch)
  uint32_t n_inst;
  uint32_t block_bytes;
  uint32_t num_blocks;
  uint32_t bm_words;                  // words of one hierarchical bitmap
  uint32_t nlevels;
  uint32_t bm_shift;                  // log2 of the bitmap fan-out (5 or 6)
  uint32_t level_off[SMMO_MAX_LEVELS];
  uint32_t level_words[SMMO_MAX_LEVELS];
  uint32_t level_bits[SMMO_MAX_LEVELS];
  int32_t num_classes;
  int32_t lookup_retries;
  int32_t alloc_retries;
  int32_t bitmap_spins;
  int32_t debug;
};

// bitmap ids
__host__ __device__ __forceinline__ int bm_free() { return 0; }
__host__ __device__ __forceinline__ int bm_alloc(const HeapView& h, int c) { return 1 + c; }
__host__ __device__ __forceinline__ int bm_active(const HeapView& h, int c) {
  return 1 + h.num_classes + c;
}
__host__ __device__ __forceinline__ int bm_defrag(const HeapView& h, int c) {
  return 1 + 2 * h.num_classes + c;
}

#ifdef __CUDACC__

__device__ __forceinline__ unsigned long long* bm_level(const HeapView& h, int k, int l) {
  return h.bitmaps + (size_t)k * h.bm_words + h.level_off[l];
}

__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long* p) {
  return __ldcg(p);
}

// Site of a SMMO_E_CONTENTION, in bits 48..55 of its detail word.
constexpr unsigned long long kSitePropagate = 1ull << 48, kSiteSet = 2ull << 48, kSiteClear = 3ull << 48,
                             kSiteDealloc = 4ull << 48, kSiteCacheLock = 5ull << 48, kSiteRounds = 6ull << 48;

__device__ __forceinline__ void set_error(const HeapView& h, int code,
                                          unsigned long long detail) {
  if (atomicCAS(&h.st->err, 0, code) == 0) h.st->err_detail = detail;
}

__device__ __forceinline__ void count(const HeapView& h, int ctr, unsigned long long v) {
  atomicAdd(&h.st->ctr[blockIdx.x % SMMO_NSHARD][ctr], v);
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  // integer finaliser (murmur3 fmix32) for rotation seeds
  x ^= x >> 16; x *= 0x85ebca6bu; x ^= x >> 13; x *= 0xc2b2ae35u; x ^= x >> 16;
  return x;
}

// Position of set bit number n (0-based, n < popcount(b)) of b (the
// nth_set_bit of Alg. 5.9, which clears the n lowest set bits one at a
// time; here a binary search on population counts of halves).
__device__ __forceinline__ int nth_set_bit64(unsigned long long b, uint32_t n) {
  int pos = 0;
#pragma unroll
  for (int w = 32; w >= 1; w >>= 1) {
    const uint32_t c = __popcll(b & ((1ull << w) - 1));
    if (n >= c) { n -= c; b >>= w; pos += w; }
  }
  return pos;
}

// The k lowest set bits of b (all of them if b has at most k): a mask up
// to the position of set bit number k, found by the binary search above,
// instead of clearing the lowest set bit k times.
__device__ __forceinline__ unsigned long long lowest_set_bits(unsigned long long b, uint32_t k) {
  if ((uint32_t)__popcll(b) <= k) return b;
  return b & ((1ull << nth_set_bit64(b, k)) - 1);
}

// ---------------------------------------------------- hierarchical bitmaps
// Every level is a dense bit array in 64-bit words; a container is F =
// 2^bm_shift consecutive bits (F = 64: one word; F = 32: half a word), and
// bit i of level l + 1 says whether container i of level l has a set bit
// (Sec. 5.3.1).  So level 0 holds one bit per block whatever F is.
// Container mask of bit `pos` inside its storage word.
__device__ __forceinline__ unsigned long long bm_cmask(const HeapView& h, uint32_t pos) {
  return h.bm_shift == 6 ? kAll : (0xFFFFFFFFull << (pos & 32));
}

// Blocking set/clear of bit `pos` at level l >= 1 (higher levels are always
// changed with the blocking form, Sec. 5.3.1 "set and clear with atomic
// operations"), then propagation upwards while a container changes between
// empty and non-empty.
static __device__ __forceinline__ void bm_propagate(const HeapView& h, int k, int l, uint32_t pos,
                                          bool set) {
  for (; l < (int)h.nlevels; ++l) {
    unsigned long long* w = bm_level(h, k, l) + (pos >> 6);
    const unsigned long long m = 1ull << (pos & 63);
    unsigned long long prev = 0;
    bool done = false;
    for (int s = 0; s < h.bitmap_spins; ++s) {
      prev = set ? atomicOr(w, m) : atomicAnd(w, ~m);
      if (set ? !(prev & m) : (prev & m)) { done = true; break; }
      __nanosleep(32);
    }
    if (!done) { set_error(h, SMMO_E_CONTENTION, kSitePropagate | ((unsigned long long)k << 32) | pos); return; }
    // continue only on set-first / clear-last of this container
    const unsigned long long cm = bm_cmask(h, pos);
    if (set ? ((prev & cm) != 0) : ((prev & cm) != m)) return;
    pos >>= h.bm_shift;
  }
}

// try_set / try_clear of a level-0 bit (Alg. 5.3 try_clear; try_set is its
// mirror).  Returns true iff this thread flipped the bit.
__device__ __forceinline__ bool bm_try_set(const HeapView& h, int k, uint32_t pos) {
  unsigned long long* w = bm_level(h, k, 0) + (pos >> 6);
  const unsigned long long m = 1ull << (pos & 63);
  const unsigned long long prev = atomicOr(w, m);
  if (prev & m) return false;
  if ((prev & bm_cmask(h, pos)) == 0 && h.nlevels > 1) bm_propagate(h, k, 1, pos >> h.bm_shift, true);
  return true;
}

__device__ __forceinline__ bool bm_try_clear(const HeapView& h, int k, uint32_t pos) {
  unsigned long long* w = bm_level(h, k, 0) + (pos >> 6);
  const unsigned long long m = 1ull << (pos & 63);
  const unsigned long long prev = atomicAnd(w, ~m);
  if (!(prev & m)) return false;
  if ((prev & bm_cmask(h, pos)) == m && h.nlevels > 1) bm_propagate(h, k, 1, pos >> h.bm_shift, false);
  return true;
}

// Blocking forms (retry until this thread flipped the bit), bounded.
__device__ __forceinline__ void bm_set(const HeapView& h, int k, uint32_t pos) {
  for (int s = 0; s < h.bitmap_spins; ++s) {
    if (bm_try_set(h, k, pos)) return;
    __nanosleep(32);
  }
  set_error(h, SMMO_E_CONTENTION, kSiteSet | ((unsigned long long)k << 32) | pos);
}

__device__ __forceinline__ void bm_clear(const HeapView& h, int k, uint32_t pos) {
  for (int s = 0; s < h.bitmap_spins; ++s) {
    if (bm_try_clear(h, k, pos)) return;
    __nanosleep(32);
  }
  set_error(h, SMMO_E_CONTENTION, kSiteClear | ((unsigned long long)k << 32) | pos);
}

__device__ __forceinline__ bool bm_get(const HeapView& h, int k, uint32_t pos) {
  return (ld_cg(bm_level(h, k, 0) + (pos >> 6)) >> (pos & 63)) & 1;
}

// The bits of container `idx` of level l (right-aligned).
__device__ __forceinline__ unsigned long long bm_container(const HeapView& h, int k, int l, uint32_t idx) {
  const uint32_t first = idx << h.bm_shift;
  const unsigned long long w = ld_cg(bm_level(h, k, l) + (first >> 6));
  return h.bm_shift == 6 ? w : (w >> (first & 32)) & 0xFFFFFFFFull;
}

// Top-down search for any set bit (Alg. 5.4 try_find_set).  Against
// contention (the purpose of the bitmap rotation of Sec. 5.3.2) each level
// picks a seed-dependent set bit uniformly among the set bits of the
// container: rotation followed by find-first-set favours the first set bit
// after a gap, so when the set bits are clustered most threads would land on
// the same container.  Returns -1 (FAIL) on an empty or inconsistent path.
__device__ __forceinline__ int bm_try_find_set(const HeapView& h, int k, uint32_t seed) {
  uint32_t idx = 0;  // container index at the current level (one at the top)
  for (int l = (int)h.nlevels - 1; l >= 0; --l) {
    const unsigned long long w = bm_container(h, k, l, idx);
    if (w == 0) return -1;
    const uint32_t pick = mix32(seed + 0x9E3779B9u * (uint32_t)(l + 1)) % (uint32_t)__popcll(w);
    idx = (idx << h.bm_shift) + (uint32_t)nth_set_bit64(w, pick);
  }
  return idx < h.num_blocks ? (int)idx : -1;
}

// clear(): find a set bit and clear it atomically (Sec. 5.3.1), bounded.
__device__ __forceinline__ int bm_clear_any(const HeapView& h, int k, uint32_t seed) {
  for (int s = 0; s < h.bitmap_spins; ++s) {
    const int i = bm_try_find_set(h, k, seed + 7919u * (uint32_t)s);
    if (i < 0) {
      // an empty top-level word means the bitmap is (momentarily) empty
      if (ld_cg(bm_level(h, k, h.nlevels - 1)) == 0) return -1;
      __nanosleep(64);
      continue;
    }
    if (bm_try_clear(h, k, (uint32_t)i)) return i;
  }
  return -2;
}

// ----------------------------------------------------------- field access
__device__ __forceinline__ uint8_t* block_data(const HeapView& h, uint32_t bid) {
  return h.data + (size_t)bid * h.block_bytes;
}

template <class T>
__device__ __forceinline__ T* field_ptr(const HeapView& h, uint32_t col_off, uint32_t handle) {
  return reinterpret_cast<T*>(block_data(h, handle >> 6) + col_off) + (handle & 63);
}

__device__ __forceinline__ uint32_t type_of(const HeapView& h, uint32_t handle) {
  return __ldcg(h.block_type + (handle >> 6));
}

// ----------------------------------------------------------- instances
// The instance-table row of object `self` of class c, named by the class's
// SMMO_INSTANCE field (null if the class has none or the index is out of
// the table).
__device__ __forceinline__ const Inst* instance_of(const HeapView& h, uint32_t c, uint32_t self) {
  const int col = __ldg(&h.cls[c].inst_col);
  if (col < 0) return nullptr;
  const uint32_t i = *field_ptr<uint32_t>(h, __ldg(&h.cls[c].col_off[col]), self);
  return i < h.n_inst ? h.inst + i : nullptr;
}

// The row whose range [cell_base, cell_base + count) holds global index g
// (rows sorted by cell_base; g must lie in some range).
__device__ __forceinline__ const Inst* instance_at(const Inst* tab, uint32_t n, uint32_t g) {
  uint32_t lo = 0, hi = n;  // invariant: tab[lo].cell_base <= g
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&tab[mid].cell_base) <= g) lo = mid; else hi = mid;
  }
  return tab + lo;
}

// ------------------------------------------------------------- deallocation
// Frees the slots `bits` of block `bid` of class t: the divergence-safe
// deallocation of Alg. 5.12 with block invalidation (Alg. 5.11) folded in,
// extended with the defragmentation-candidate state of Alg. 6.3 (a block is
// a candidate iff it is allocated and holds at most dlimit objects).  All
// block-state bitmap changes are collected as pending +1/-1 operations first
// and then retried with try_ operations in one converged loop, so no lane
// waits on a bit that another lane of its own warp has yet to flip.
static __device__ __forceinline__ void dealloc_bits(const HeapView& h, uint32_t bid, uint32_t t,
                                                 unsigned long long bits) {
  const unsigned long long capmask = __ldg(&h.cls[t].capmask);
  const uint32_t dlim = __ldg(&h.cls[t].dlimit);
  const unsigned long long empty = ~capmask;
  const unsigned long long before = atomicAnd(h.alloc_bm + bid, ~bits);
  if ((before & bits) != bits) {  // precondition of Alg. 5.8 violated
    set_error(h, SMMO_E_BAD_HANDLE, ((unsigned long long)bid << 6) | (__ffsll((long long)bits) - 1));
    return;
  }
  int act = 0, alc = 0, fre = 0, dfr = 0;
  if (before == kAll) act += 1;  // freed the first slot of a full block
  const uint32_t fb = __popcll(before & capmask), fa = fb - __popcll(bits);
  if (fb > dlim && fa <= dlim) dfr += 1;  // became a defragmentation candidate
  if ((before & ~bits) == empty) {
    // freed the last object: try to invalidate the block (Alg. 5.11)
    for (int s = 0; s < h.bitmap_spins; ++s) {
      const unsigned long long ib = atomicOr(h.alloc_bm + bid, kAll);
      if (ib == kAll) break;                       // nothing invalidated
      if (ib == empty) { act -= 1; alc -= 1; fre += 1; dfr -= 1; break; }  // success
      const unsigned long long rb = atomicAnd(h.alloc_bm + bid, ib);  // rollback
      if (rb != kAll) act -= 1;  // a concurrent free saw a full block
      if ((rb & ib) != empty) break;               // not empty again
    }
  }
  for (int s = 0; (act | alc | fre | dfr) && s < h.bitmap_spins; ++s) {
    if (act > 0 && bm_try_set(h, bm_active(h, t), bid)) --act;
    if (act < 0 && bm_try_clear(h, bm_active(h, t), bid)) ++act;
    if (dfr > 0 && bm_try_set(h, bm_defrag(h, t), bid)) --dfr;
    if (dfr < 0 && bm_try_clear(h, bm_defrag(h, t), bid)) ++dfr;
    if (alc < 0 && bm_try_clear(h, bm_alloc(h, t), bid)) ++alc;
    if (fre > 0 && act == 0 && alc == 0 && dfr == 0 && bm_try_set(h, bm_free(), bid)) --fre;
    if (act | alc | fre | dfr) __nanosleep(32);
  }
  if (act | alc | fre | dfr)  // pending block-state changes left: act, alc, fre, dfr in bits 32..47
    set_error(h, SMMO_E_CONTENTION, kSiteDealloc | ((unsigned long long)((act & 15) | (alc & 15) << 4 |
                                                                          (fre & 15) << 8 | (dfr & 15) << 12) << 32) | bid);
}

// destroy(ptr) for a single object (Alg. 5.2 / 5.12).
__device__ __forceinline__ void smmo_delete(const HeapView& h, uint32_t handle) {
  const uint32_t bid = handle >> 6;
  if (handle == kNull || bid >= h.num_blocks) {  // never touch memory for a bad handle
    set_error(h, SMMO_E_BOUNDS, handle);
    return;
  }
  const uint32_t t = type_of(h, handle);
  if (t >= (uint32_t)h.num_classes) { set_error(h, SMMO_E_BAD_HANDLE, handle); return; }
  dealloc_bits(h, bid, t, 1ull << (handle & 63));
  // warp-aggregated free counter
  const unsigned m = __activemask();
  const unsigned same = __match_any_sync(m, t);
  if ((threadIdx.x & 31) == __ffs(same) - 1) count(h, SMMO_CTR_FREE(t), __popc(same));
}

// ---------------------------------------------------------------- allocation
// Reserves up to n free slots of block bid for class c (Block::reserve of
// Alg. 5.7, extended to several slots, with the state changes of Alg. 6.2:
// the thread that fills the block removes it from active, the one that
// takes it above dlimit removes it from the candidates).  If the block was
// re-initialised to another class the reservation is rolled back (Alg. 5.1).
static __device__ __forceinline__ unsigned long long reserve_in(const HeapView& h, uint32_t c, uint32_t bid,
                                                             int n) {
  for (int s = 0; s < h.bitmap_spins; ++s) {
    const unsigned long long cur = ld_cg(h.alloc_bm + bid);
    const unsigned long long freeb = ~cur;
    if (freeb == 0) { count(h, SMMO_CTR_RESERVE_FAIL, 1); return 0; }  // full or invalidated
    const unsigned long long pick = lowest_set_bits(freeb, (uint32_t)n);
    const unsigned long long before = atomicOr(h.alloc_bm + bid, pick);
    const unsigned long long got = pick & ~before;
    if (!got) continue;
    const uint32_t t = atomicAdd(h.block_type + bid, 0u);
    if (t < (uint32_t)h.num_classes) {
      const unsigned long long tcap = __ldg(&h.cls[t].capmask);
      const uint32_t dlim = __ldg(&h.cls[t].dlimit);
      const uint32_t fb = __popcll(before & tcap), fa = fb + __popcll(got);
      if ((before | pick) == kAll) bm_clear(h, bm_active(h, t), bid);       // filled it
      if (fb <= dlim && fa > dlim) bm_clear(h, bm_defrag(h, t), bid);       // no candidate now
    }
    if (t != c) {  // block was re-initialised to another class: roll back
      dealloc_bits(h, bid, t, got);
      return 0;
    }
    return got;
  }
  return 0;
}

// A block from the free bitmap, initialised for class c and full for the
// caller (initialize_block, Alg. 5.10: no slot is open to others until the
// caller frees what it does not use).  -1 if no block is free.
static __device__ __forceinline__ int take_fresh_block(const HeapView& h, uint32_t c, uint32_t seed) {
  const int fb = bm_clear_any(h, bm_free(), seed ^ 0x5bd1e995u);
  if (fb < 0) return -1;
  atomicExch(h.block_type + fb, c);
  __threadfence();
  atomicExch(h.alloc_bm + fb, kAll);
  bm_set(h, bm_alloc(h, c), (uint32_t)fb);
  count(h, SMMO_CTR_SLOW, 1);
  return fb;
}

// Finds room for a warp's cache: (0) near the hint (the block whose objects
// the warp is running a method on): the hint block itself if it is of class
// c and has a free slot, else a defragmentation candidate among the 64
// blocks of the hint's level-0 bitmap word, so that new objects land next to
// the objects that created them (in the cellular workloads, next to them in
// space, which keeps neighbour accesses of later do-alls coalesced); (1) any
// defragmentation candidate, i.e. a block at most dlimit full, so one
// reservation yields many slots; (2) a fresh block from the free bitmap,
// initialised full for the caller (initialize_block, Alg. 5.10, opening no
// slot to others); (3) when no block is free, any active block with room.
// Lookups retry with a new random choice (Sec. 5.3.2).  Returns the reserved
// slot bits and the block in *bid_out (kNull: the heap is exhausted).
static __device__ __forceinline__ unsigned long long refill_reserve(const HeapView& h, uint32_t c,
                                                                 uint32_t seed, uint32_t hint,
                                                                 uint32_t* bid_out) {
  if (hint < h.num_blocks) {
    if (__ldcg(h.block_type + hint) == c && ~ld_cg(h.alloc_bm + hint) != 0) {
      const unsigned long long got = reserve_in(h, c, hint, 64);
      if (got) { *bid_out = hint; return got; }
    }
    const unsigned long long w = ld_cg(bm_level(h, bm_defrag(h, c), 0) + (hint >> 6));
    if (w) {
      const uint32_t b = (hint & ~63u) + (uint32_t)nth_set_bit64(w, mix32(seed) % (uint32_t)__popcll(w));
      const unsigned long long got = b < h.num_blocks ? reserve_in(h, c, b, 64) : 0ull;
      if (got) { *bid_out = b; return got; }
    }
  }
  for (int r = 0; r < h.lookup_retries; ++r) {
    const int b = bm_try_find_set(h, bm_defrag(h, c), seed + 104729u * (uint32_t)r);
    if (b < 0) {
      if (ld_cg(bm_level(h, bm_defrag(h, c), h.nlevels - 1)) == 0) break;
      continue;
    }
    const unsigned long long got = reserve_in(h, c, (uint32_t)b, 64);
    if (got) { *bid_out = (uint32_t)b; return got; }
  }
  count(h, SMMO_CTR_LOOKUP_MISS, 1);
  const int fb = take_fresh_block(h, c, seed);
  if (fb >= 0) {
    *bid_out = (uint32_t)fb;
    return __ldg(&h.cls[c].capmask);
  }
  for (int r = 0; r < h.lookup_retries; ++r) {
    const int b = bm_try_find_set(h, bm_active(h, c), seed + 7u + 104729u * (uint32_t)r);
    if (b < 0) {
      if (ld_cg(bm_level(h, bm_active(h, c), h.nlevels - 1)) == 0) break;
      continue;
    }
    const unsigned long long got = reserve_in(h, c, (uint32_t)b, 64);
    if (got) { *bid_out = (uint32_t)b; return got; }
  }
  *bid_out = kNull;
  return 0;
}

// Per-warp allocation cache (shared memory, one slot per warp and class,
// plus the block the warp is working on as a placement hint).
// When a warp runs out of cached slots its leader refills the cache with
// every free slot of the block refill_reserve finds; later allocations of
// the same warp are served from the cached bits without touching global
// memory.  Only leader lanes of the warp touch its slot; a per-warp lock
// still guards it because two diverged lane groups of one warp may each be
// inside smmo_new at the same time (independent thread scheduling), and
// without the lock both could hand out the same cached slot.  The lock is
// uncontended unless that happens.  Slots still cached when the do-all
// kernel ends are returned with dealloc_bits, exactly like deleted objects.
struct WarpAllocCache {
  unsigned long long bits[SMMO_MAX_CLASSES];
  uint32_t bid[SMMO_MAX_CLASSES];
  uint32_t hint;
  int lock;
};
static __shared__ WarpAllocCache g_wcache[16];  // do-all CTAs have at most 16 warps
struct WarpNewBcast {  // warp_new: the cache's slots, broadcast by the leader
  unsigned long long bits;
  uint32_t bid;
};
static __shared__ WarpNewBcast g_wnew[16];

__device__ __forceinline__ void alloc_cache_init() {
  const uint32_t lane = threadIdx.x & 31;
  if (lane < SMMO_MAX_CLASSES) {
    g_wcache[threadIdx.x >> 5].bid[lane] = kNull;
    g_wcache[threadIdx.x >> 5].bits[lane] = 0;
  }
  if (lane == 0) { g_wcache[threadIdx.x >> 5].lock = 0; g_wcache[threadIdx.x >> 5].hint = kNull; }
  __syncwarp();
}

__device__ __forceinline__ void alloc_cache_flush(const HeapView& h) {
  __syncwarp();
  const uint32_t lane = threadIdx.x & 31;
  WarpAllocCache& wc = g_wcache[threadIdx.x >> 5];
  if (lane < SMMO_MAX_CLASSES && wc.bits[lane]) {
    dealloc_bits(h, wc.bid[lane], lane, wc.bits[lane]);
    wc.bits[lane] = 0;
  }
}

// Refills an empty warp-cache entry.
static __device__ __forceinline__ unsigned long long cache_refill(const HeapView& h, uint32_t c,
                                                               uint32_t seed, uint32_t* bid) {
  count(h, SMMO_CTR_REFILL, 1);
  return refill_reserve(h, c, seed, g_wcache[threadIdx.x >> 5].hint, bid);
}

// Takes up to n slots of class c from the calling warp's cache, refilling
// it when empty.  Returns the slot bits (possibly fewer or none) and the
// block in *bid (kNull: heap exhausted).
__device__ __forceinline__ unsigned long long cache_take(const HeapView& h, uint32_t c, int n,
                                                         uint32_t seed, uint32_t* bid) {
  WarpAllocCache& wc = g_wcache[threadIdx.x >> 5];
  int spins = 0;
  while (atomicCAS(&wc.lock, 0, 1) != 0) {
    if (++spins > h.bitmap_spins) { set_error(h, SMMO_E_CONTENTION, kSiteCacheLock | c); *bid = 0; return 0; }
    __nanosleep(8);
  }
  __threadfence_block();
  unsigned long long avail = wc.bits[c];
  uint32_t b = wc.bid[c];
  if (avail == 0) {
    avail = cache_refill(h, c, seed, &b);
    wc.bid[c] = b;
  }
  // keep the highest bits, hand out the n lowest
  const unsigned long long take = lowest_set_bits(avail, (uint32_t)n);
  avail ^= take;
  wc.bits[c] = b == kNull ? 0ull : avail;
  __threadfence_block();
  atomicExch(&wc.lock, 0);
  *bid = b;
  return take;
}

// new(d_allocator) T: warp-aggregated allocation of one object of class c
// per calling lane (allocation request coalescing, Alg. 5.6).  Lanes that
// call it together (the active mask) are served by one leader per round from
// the warp cache; lanes left without a slot retry with a new leader.  Only
// methods run by parallel_do may call it (it uses the warp cache above).
// Returns kNull (and records SMMO_E_DEVICE_OOM or SMMO_E_CONTENTION) if the
// heap is exhausted or the budget runs out.
__device__ __forceinline__ uint32_t smmo_new(const HeapView& h, uint32_t c) {
  if (c >= (uint32_t)h.num_classes) { set_error(h, SMMO_E_INVALID_ARG, c); return kNull; }
  const unsigned active = __activemask();
  const int lane = threadIdx.x & 31;
  const uint32_t warp_uid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t result = kNull;
  int round = 0;
  for (; round < h.alloc_retries; ++round) {
    const unsigned need = __ballot_sync(active, result == kNull);
    if (need == 0) break;
    const int leader = __ffs(need) - 1;
    unsigned long long got = 0;
    uint32_t bid = 0;
    if (lane == leader) {
      got = cache_take(h, c, __popc(need), mix32(warp_uid * 0x27d4eb2fu + (uint32_t)round), &bid);
      if (got) count(h, SMMO_CTR_ALLOC(c), __popcll(got));
      if (round) count(h, SMMO_CTR_RETRY, 1);
    }
    got = __shfl_sync(active, got, leader);
    bid = __shfl_sync(active, bid, leader);
    __syncwarp(active);  // the leader's cache update is visible to the next leader
    if (bid == kNull) {  // no free block anywhere
      if (lane == leader) set_error(h, SMMO_E_DEVICE_OOM, c);
      break;
    }
    if (result == kNull) {
      const int rank = __popc(need & ((1u << lane) - 1));
      const int slot = rank < __popcll(got) ? nth_set_bit64(got, (uint32_t)rank) : -1;
      if (slot >= 0) result = (bid << 6) | (uint32_t)slot;
    }
  }
  if (round == h.alloc_retries && result == kNull) set_error(h, SMMO_E_CONTENTION, kSiteRounds | c);
  return result;
}

// ------------------------------------------------ warp-parallel allocation
// new for a converged warp that needs `need` (1..32) objects of class c at
// once (the deferred creations below): lane i < need receives a handle.
// The warp's cache is used first; the rest is reserved in the blocks of
// class c around the warp's hint (the 64 blocks of the hint's level-0
// bitmap word, then those of the neighbouring words, 32 per round while
// slots are missing) with one block per lane and every reservation of a
// round in flight at the same time: one round of loads (allocation bitmaps and type ids),
// one round of atomicOr reservations, one round of type re-checks (a block
// re-initialised to another class in between is rolled back, Alg. 5.1),
// then the block-state changes of the blocks that became full or left the
// candidates (as reserve_in).  After the hint's own word, a round whose 32
// blocks have no free slot ends the search; if SMMO_FRESH_MIN or more slots
// are still missing the warp takes a fresh block (its surplus goes to the
// warp's cache), and a leader-at-a-time refill (smmo_new) serves the rest.
__device__ __forceinline__ uint32_t warp_new(const HeapView& h, uint32_t c, uint32_t need) {
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpAllocCache& wc = g_wcache[w];
  uint32_t result = kNull;
  // (1) the warp's cache (the warp is converged: no lane group of it is
  // inside smmo_new, so the leader may touch the cache without the lock)
  if (lane == 0) {
    const unsigned long long avail = wc.bits[c], take = lowest_set_bits(avail, need);
    wc.bits[c] = avail ^ take;
    g_wnew[w].bits = take;
    g_wnew[w].bid = wc.bid[c];
    if (take) count(h, SMMO_CTR_ALLOC(c), __popcll(take));
  }
  __syncwarp();
  const unsigned long long take = g_wnew[w].bits;
  uint32_t got_n = (uint32_t)__popcll(take);
  if (lane < got_n) result = (g_wnew[w].bid << 6) | (uint32_t)nth_set_bit64(take, lane);
  __syncwarp();
  // (2) blocks of class c near the hint, 32 per round (one per lane): the
  // two halves of the hint's level-0 bitmap word, then of the word after
  // it and of the word before it, while slots are missing
  const uint32_t hint = wc.hint;
  if (hint < h.num_blocks) {
    const int32_t w0 = (int32_t)(hint >> 6);
    for (int r = 0; r < 6 && got_n < need; ++r) {
      const int32_t wd = w0 + (r < 2 ? 0 : (r < 4 ? 1 : -1));
      if (wd < 0) continue;
      const uint32_t cand = (uint32_t)wd * 64u + (uint32_t)(r & 1) * 32u + lane;
      const uint32_t rem = need - got_n;
      const bool ok = cand < h.num_blocks && __ldcg(h.block_type + cand) == c;
      const unsigned long long freeb = ok ? ~ld_cg(h.alloc_bm + cand) : 0ull;
      const uint32_t bid = freeb ? cand : kNull;
      if (r >= SMMO_NEAR_STOP_FROM && __ballot_sync(0xFFFFFFFFu, freeb != 0ull) == 0u) break;  // full around: stop
      // the lowest free slots, in lane order, until rem are covered
      const uint32_t nf = (uint32_t)__popcll(freeb);
      uint32_t incl = nf;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
      }
      const uint32_t excl = incl - nf;
      const unsigned long long pick = excl < rem ? lowest_set_bits(freeb, rem - excl) : 0ull;
      unsigned long long got = 0;
      if (pick) {
        const unsigned long long before = atomicOr(h.alloc_bm + bid, pick);
        got = pick & ~before;
        if (got) {
          const uint32_t t = atomicAdd(h.block_type + bid, 0u);
          if (t < (uint32_t)h.num_classes) {
            const unsigned long long tcap = __ldg(&h.cls[t].capmask);
            const uint32_t dlim = __ldg(&h.cls[t].dlimit);
            const uint32_t fb = __popcll(before & tcap), fa = fb + __popcll(got);
            if ((before | got) == kAll) bm_clear(h, bm_active(h, t), bid);   // filled it
            if (fb <= dlim && fa > dlim) bm_clear(h, bm_defrag(h, t), bid);  // no candidate now
          }
          if (t != c) {  // re-initialised to another class meanwhile: roll back
            dealloc_bits(h, bid, t, got);
            got = 0;
          } else {
            count(h, SMMO_CTR_ALLOC(c), __popcll(got));
          }
        }
      }
      // concatenate the lanes' reserved slots; lane got_n + j takes number j
      const uint32_t ng = (uint32_t)__popcll(got);
      uint32_t gi = ng;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, gi, o);
        if (lane >= (uint32_t)o) gi += v;
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, gi, 31);
      const uint32_t want = lane - got_n;  // wraps for lanes already served
      uint32_t src = 0;  // first lane whose inclusive count exceeds want
#pragma unroll
      for (uint32_t step = 16; step; step >>= 1) {
        const uint32_t v = __shfl_sync(0xFFFFFFFFu, gi, src + step - 1);
        if (v <= want) src += step;
      }
      src &= 31;
      const uint32_t sb = __shfl_sync(0xFFFFFFFFu, bid, src);
      const unsigned long long sg = __shfl_sync(0xFFFFFFFFu, got, src);
      const uint32_t sexcl = __shfl_sync(0xFFFFFFFFu, gi, src) - (uint32_t)__popcll(sg);
      if (lane >= got_n && lane < need && want < total) result = (sb << 6) | (uint32_t)nth_set_bit64(sg, want - sexcl);
      got_n += total;
    }
  }
  // (3) SMMO_FRESH_MIN or more still missing (a full neighbourhood, as in a
  // birth wave): one fresh block for the warp, the surplus kept in its cache
  // (the cache is empty here: step (1) found fewer slots than needed)
  if (need - got_n >= SMMO_FRESH_MIN) {
    int fb = -1;
    if (lane == 0) fb = take_fresh_block(h, c, mix32(((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 0x9E3779B9u + got_n));
    fb = __shfl_sync(0xFFFFFFFFu, fb, 0);
    if (fb >= 0) {
      const unsigned long long capm = __ldg(&h.cls[c].capmask);
      const unsigned long long mine = lowest_set_bits(capm, need - got_n);
      const uint32_t k = (uint32_t)__popcll(mine);
      if (lane >= got_n && lane - got_n < k) result = ((uint32_t)fb << 6) | (uint32_t)nth_set_bit64(mine, lane - got_n);
      if (lane == 0) {
        wc.bits[c] = capm & ~mine;
        wc.bid[c] = (uint32_t)fb;
        count(h, SMMO_CTR_ALLOC(c), k);
      }
      got_n += k;
    }
    __syncwarp();
  }
  // (4) what is still missing, one leader at a time
  if (got_n < need && lane >= got_n && lane < need) result = smmo_new(h, c);
  __syncwarp();
  return lane < need ? result : kNull;
}

// ------------------------------------------------------- deferred creation
// A method that creates objects may defer them: defer_new(payload) appends
// a word to its warp's list in shared memory, and the do-all creates the
// objects between rounds, 32 at a time with the whole warp (one
// warp-aggregated new, Alg. 5.6, for 32 objects), passing each new object
// and its payload to M::create.  The objects exist before the do-all ends,
// as with a new inside the method, but the method itself carries no
// allocator code, and the allocation is not split into the few lanes of a
// round that create.  A method opts in by defining kDeferMax (the most
// defer_new calls one run makes), child_class(args) and create(h, args,
// child, payload); child is kNull if the heap is exhausted (the error is
// recorded).
template <class M, class = void>
struct defers { static constexpr uint32_t max = 0; };
template <class M>
struct defers<M, decltype((void)M::kDeferMax)> { static constexpr uint32_t max = M::kDeferMax; };


struct DeferList {
  uint32_t n;
  uint32_t item[32 + 32 * 2];  // < 32 left over + one round of at most 2 per lane
};
static __shared__ DeferList g_defer[16];

__device__ __forceinline__ void defer_new(uint32_t payload) {
  DeferList& d = g_defer[threadIdx.x >> 5];
  const uint32_t at = atomicAdd(&d.n, 1u);
  d.item[at] = payload;
}

// Creates the deferred objects of the calling (converged) warp in rounds of
// 32 while 32 or more wait; with all = true also the rest (fewer than 32,
// with part of the warp).
template <class M>
__device__ __forceinline__ void defer_flush_alloc(const HeapView& h, const typename M::Args& args, bool all) {
  DeferList& d = g_defer[threadIdx.x >> 5];
  const uint32_t lane = threadIdx.x & 31;
  __syncwarp();
  uint32_t n = d.n;
  while (n >= 32) {
    n -= 32;
    const uint32_t p = d.item[n + lane];
    const uint32_t child = warp_new(h, M::child_class(args), 32);
    M::create(h, args, child, p);
    __syncwarp();
  }
  if (all && n) {
    const uint32_t p = lane < n ? d.item[lane] : 0u;
    const uint32_t child = warp_new(h, M::child_class(args), n);
    if (lane < n) M::create(h, args, child, p);
    n = 0;
  }
  __syncwarp();
  if (lane == 0) d.n = n;
  __syncwarp();
}

// Deferred creation through a queue in global memory (a method with
// kQueued = true and queue(args)): instead of allocating inside the do-all,
// the warp writes its deferred payloads in chunks of 32, each with the
// block it was working on as the placement hint, and a later launch
// (create_queued_kernel) creates them, one full warp per chunk.  The do-all
// then carries no allocator code at all.  A chunk's unused tail holds kNull
// (payloads are never kNull).
struct DeferQueue {
  uint32_t* item;   // payloads, chunks of 32
  uint32_t* hint;   // per chunk: the placement hint
  uint32_t* count;  // entries written (a multiple of 32); zeroed before the do-all
  uint32_t cap;     // capacity in entries (a multiple of 32)
};
template <class M, class = void>
struct queued { static constexpr bool value = false; };
template <class M>
struct queued<M, decltype((void)M::kQueued)> { static constexpr bool value = M::kQueued; };

template <class M>
__device__ __forceinline__ void defer_flush_queue(const HeapView& h, const typename M::Args& args, bool all) {
  DeferList& d = g_defer[threadIdx.x >> 5];
  const uint32_t lane = threadIdx.x & 31;
  __syncwarp();
  const DeferQueue q = M::queue(args);
  const uint32_t hint = g_wcache[threadIdx.x >> 5].hint;
  uint32_t n = d.n;
  while (n >= 32 || (all && n)) {
    const uint32_t take = n >= 32 ? 32u : n;
    n -= take;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(q.count, 32u);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base + 32 <= q.cap) {
      q.item[base + lane] = lane < take ? d.item[n + lane] : kNull;
      if (lane == 0) q.hint[base >> 5] = hint;
    } else if (lane == 0) {
      set_error(h, SMMO_E_DEVICE_OOM, M::child_class(args));  // queue full: creations lost
    }
    __syncwarp();
  }
  if (lane == 0) d.n = n;
  __syncwarp();
}

template <class M>
__device__ __forceinline__ void defer_flush(const HeapView& h, const typename M::Args& args, bool all) {
  if constexpr (queued<M>::value) defer_flush_queue<M>(h, args, all);
  else defer_flush_alloc<M>(h, args, all);
}

// Creates the queued objects of method M: chunk k goes to warp k mod
// (warps of the grid); the warp takes its chunk's hint and creates the
// chunk's objects with one warp-parallel new.
template <class M>
__global__ void __launch_bounds__(512, SMMO_DOALL_MIN_CTAS) create_queued_kernel(HeapView h, typename M::Args args) {
  alloc_cache_init();
  const DeferQueue q = M::queue(args);
  const uint32_t total = __ldcg(q.count);
  const uint32_t chunks = (total < q.cap ? total : q.cap) >> 5;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < chunks; ch += nwarps) {
    const uint32_t p = q.item[ch * 32 + lane];
    const uint32_t need = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, p != kNull));
    if (lane == 0) g_wcache[w].hint = q.hint[ch];
    __syncwarp();
    const uint32_t child = warp_new(h, M::child_class(args), need);
    if (lane < need) M::create(h, args, child, p);
    __syncwarp();
  }
  alloc_cache_flush(h);
}

// ---------------------------------------------------------------- do-all
// Persistent do-all over the enumerated blocks (Sec. 5.2.7): the slots of
// one block are handled by consecutive threads (one warp per 32 slots, a
// "unit"), thread t of a block's group handles slot t, and a slot runs the
// method iff its bit is set in the snapshot taken at enumeration time.  Each
// warp takes one contiguous run of units (rather than every nwarps-th), so
// that consecutive units of a warp are neighbouring blocks and the warp's
// allocation cache, refilled near the current block, keeps new objects close
// to their creators.  With POLY the enumeration holds blocks of several
// classes (the concrete subclasses of one class, enumerated one after the
// other into one snapshot): every unit takes its block's class from the
// enumeration entry and passes it to the method, and every block counts as
// two units.  A method that defers its creations (defer_new) has them made
// after each unit once 32 are listed, and the rest at the end.
//
// (Packing the live slots of several blocks into full warps through a
// shared-memory queue was measured and dropped: the rounds then span two
// blocks' columns and cost more sectors and instructions than the idle
// lanes of partly full units, which these latency-bound kernels hide.)
// The enumeration entries of 32 consecutive units (at most 17 entries for
// blocks of 64 slots), one per lane, so that a unit's block and bitmap come
// from a shuffle instead of a load at the head of its chain of dependent
// loads.
struct UnitEntries {
  uint32_t e0;     // entry index held by lane 0
  uint32_t block;  // this lane's entry
  uint32_t cls;
  uint32_t lo, hi;
  __device__ __forceinline__ void load(const HeapView& h, uint32_t u0, uint32_t uend, uint32_t halves) {
    const uint32_t lane = threadIdx.x & 31;
    e0 = halves == 2 ? (u0 >> 1) : u0;
    const uint32_t elast = halves == 2 ? ((uend - 1) >> 1) : uend - 1;
    block = kNull; cls = 0; lo = hi = 0;
    if (e0 + lane <= elast) {
      const uint4 raw = __ldcg(reinterpret_cast<const uint4*>(h.R + e0 + lane));
      block = raw.x; cls = raw.y; lo = raw.z; hi = raw.w;
    }
  }
  // block, class and the unit's 32 slot bits of unit u (warp-converged)
  __device__ __forceinline__ void unit(uint32_t u, uint32_t halves, uint32_t* blk, uint32_t* c, uint32_t* bits32) const {
    const uint32_t src = (halves == 2 ? (u >> 1) : u) - e0;
    *blk = __shfl_sync(0xFFFFFFFFu, block, src);
    *c = __shfl_sync(0xFFFFFFFFu, cls, src);
    const uint32_t l = __shfl_sync(0xFFFFFFFFu, lo, src), hh = __shfl_sync(0xFFFFFFFFu, hi, src);
    *bits32 = (halves == 2 && (u & 1)) ? hh : l;
  }
};

// Marking and filtered do-alls.  A marking method (M::kMarks) returns from
// run whether the object has work in the do-all that follows over the same
// snapshot; the do-all stores the ballot of those slots per unit in
// h.umark.  A filtered method (M::kFiltered) is run only on the marked slots
// of each unit: the do-all still walks every unit and counts every object of
// the snapshot, but an object whose method would return at once (the
// marking do-all already knew that) costs no load, and the marked slots of
// consecutive units are packed into full warps, so 32 of them issue their
// loads together instead of unit after unit.  The pair behaves as the
// unfiltered pair as long as nothing re-enumerates the class in between.
template <class M, class = void>
struct marks { static constexpr bool value = false; };
template <class M>
struct marks<M, decltype((void)M::kMarks)> { static constexpr bool value = M::kMarks; };
template <class M, class = void>
struct filtered { static constexpr bool value = false; };
template <class M>
struct filtered<M, decltype((void)M::kFiltered)> { static constexpr bool value = M::kFiltered; };

// Marked slots of a filtered do-all, collected per warp until 32 can run
// at once (one per lane).
static __shared__ uint32_t g_pack[16][64];

template <class M, bool POLY, class F, class G>
__device__ __forceinline__ void for_each_unit(const HeapView& h, uint32_t c, F&& f, G&& after_unit) {
  constexpr bool kMark = marks<M>::value, kFilter = filtered<M>::value;
  static_assert(!(kFilter && POLY), "a filtered do-all runs over one class");
  const uint32_t n = __ldcg(h.rcnt);
  const uint32_t cap = POLY ? 64u : __ldg(&h.cls[c].cap);
  const uint32_t halves = cap > 32 ? 2u : 1u;
  const uint32_t units = n * halves;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  uint32_t visited = 0;
  const uint32_t per = (units + nwarps - 1) / nwarps;
  const uint32_t ub = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * per;
  const uint32_t ue = ub + per < units ? ub + per : units;
  uint32_t np = 0;  // filtered: marked slots waiting in g_pack[w] (warp-uniform)
  for (uint32_t u0 = ub; u0 < ue; u0 += 32) {
    const uint32_t uend = u0 + 32 < ue ? u0 + 32 : ue;
    UnitEntries ents;
    ents.load(h, u0, uend, halves);
    uint32_t umk = 0;
    if constexpr (kFilter) umk = u0 + lane < uend ? __ldcg(h.umark + u0 + lane) : 0u;
    for (uint32_t u = u0; u < uend; ++u) {
      uint32_t blk, ecls, bits32;
      ents.unit(u, halves, &blk, &ecls, &bits32);
      const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + lane;
      if (lane == 0) visited += __popc(bits32);
      if constexpr (kFilter) {
        // the marked slots of the unit join the warp's list; every full 32
        // of them run together, one per lane
        const uint32_t run_bits = bits32 & __shfl_sync(0xFFFFFFFFu, umk, u - u0);
        if (run_bits == 0) continue;
        if ((run_bits >> lane) & 1) g_pack[w][np + __popc(run_bits & ((1u << lane) - 1))] = (blk << 6) | slot;
        np += __popc(run_bits);
        __syncwarp();
        if (np < 32) continue;
        np -= 32;
        const uint32_t self = g_pack[w][np + lane];
        __syncwarp();
        g_wcache[w].hint = self >> 6;
        f(c, self);
        __syncwarp();
        after_unit();
      } else {
        g_wcache[w].hint = blk;
        bool mk = false;
        if ((bits32 >> lane) & 1) mk = f(POLY ? ecls : c, (blk << 6) | slot);
        __syncwarp();  // reconverge: lane groups never run different iterations
        if constexpr (kMark) {
          const uint32_t m = __ballot_sync(0xFFFFFFFFu, mk);
          if (lane == 0) h.umark[u] = m;
        }
        after_unit();
      }
    }
  }
  if constexpr (kFilter) {
    if (np) {
      const uint32_t self = lane < np ? g_pack[w][lane] : kNull;
      __syncwarp();
      g_wcache[w].hint = __shfl_sync(0xFFFFFFFFu, self, 0) >> 6;
      if (lane < np) f(c, self);
      __syncwarp();
      after_unit();
    }
  }
  if (lane == 0 && visited) count(h, SMMO_CTR_VISIT, visited);
}

template <class M, bool POLY = false>
__global__ void __launch_bounds__(512, SMMO_DOALL_MIN_CTAS) do_all_kernel(HeapView h, uint32_t c,
                                                                          typename M::Args args) {
  alloc_cache_init();
  constexpr bool kDefer = defers<M>::max > 0;
  static_assert(defers<M>::max <= 2, "defer list holds two per lane and unit");
  if (kDefer && (threadIdx.x & 31) == 0) g_defer[threadIdx.x >> 5].n = 0;
  __syncwarp();
  for_each_unit<M, POLY>(
      h, c,
      [&](uint32_t cls, uint32_t self) -> bool {
        if constexpr (marks<M>::value) {
          return M::run(h, args, cls, self);
        } else {
          M::run(h, args, cls, self);
          return false;
        }
      },
      [&]() {
        if constexpr (kDefer) {
          if (g_defer[threadIdx.x >> 5].n >= 32) defer_flush<M>(h, args, false);
        }
      });
  if constexpr (kDefer) defer_flush<M>(h, args, true);
  alloc_cache_flush(h);
}

// ------------------------------------------------------- do-all with reduce
// parallel_do_and_reduce (Sec. 3.2.2, the SMMO programming interface: the
// method's return values are combined with a binary reducer, e.g. for the
// termination test of an iterative algorithm): M::run returns a long long;
// each thread folds its values, then the warp (shuffles), the CTA (shared
// memory) and the grid (one 64-bit atomic per CTA on *out, which holds the
// identity before the launch).  Integer reducers only, so the result does
// not depend on the order of the objects.
__device__ __forceinline__ long long reduce_identity(int op) {
  switch (op) {
    case SMMO_REDUCE_MIN: return 0x7FFFFFFFFFFFFFFFll;
    case SMMO_REDUCE_MAX: return (long long)0x8000000000000000ull;
    case SMMO_REDUCE_AND: return -1ll;
    default: return 0ll;  // sum, or
  }
}

__device__ __forceinline__ long long reduce2(int op, long long x, long long y) {
  switch (op) {
    case SMMO_REDUCE_MIN: return x < y ? x : y;
    case SMMO_REDUCE_MAX: return x > y ? x : y;
    case SMMO_REDUCE_OR: return x | y;
    case SMMO_REDUCE_AND: return x & y;
    default: return (long long)((unsigned long long)x + (unsigned long long)y);  // wrapping sum
  }
}

template <class M, bool POLY = false>
__global__ void __launch_bounds__(512, SMMO_DOALL_MIN_CTAS) do_all_reduce_kernel(HeapView h, uint32_t c,
                                                                                 typename M::Args args, int op,
                                                                                 long long* out) {
  __shared__ long long part[16];
  const uint32_t lane = threadIdx.x & 31;
  alloc_cache_init();
  long long acc = reduce_identity(op);
  for_each_unit<M, POLY>(
      h, c,
      [&](uint32_t cls, uint32_t self) -> bool {
        acc = reduce2(op, acc, M::run(h, args, cls, self));
        return false;
      },
      [] {});
  alloc_cache_flush(h);
#pragma unroll
  for (int o = 16; o; o >>= 1) acc = reduce2(op, acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
  if (lane == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long v = part[0];
    for (uint32_t w = 1; w < (blockDim.x >> 5); ++w) v = reduce2(op, v, part[w]);
    switch (op) {
      case SMMO_REDUCE_MIN: atomicMin(out, v); break;
      case SMMO_REDUCE_MAX: atomicMax(out, v); break;
      case SMMO_REDUCE_OR: atomicOr((unsigned long long*)out, (unsigned long long)v); break;
      case SMMO_REDUCE_AND: atomicAnd((unsigned long long*)out, (unsigned long long)v); break;
      default: atomicAdd((unsigned long long*)out, (unsigned long long)v); break;
    }
  }
}

#endif  // __CUDACC__
}  // namespace smmo
