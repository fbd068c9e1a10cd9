// heap.cu -- heap creation, class registry, block geometry, bulk creation,
// enumeration (parallel_do), live-object export, statistics, C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "heap_internal.h"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {
thread_local int g_last_cuda = 0;

int esize(int t) {
  switch (t) {
    case SMMO_I8: case SMMO_U8: return 1;
    case SMMO_I16: case SMMO_U16: return 2;
    case SMMO_I32: case SMMO_U32: case SMMO_F32: case SMMO_HANDLE: case SMMO_INSTANCE: return 4;
    case SMMO_I64: case SMMO_U64: case SMMO_F64: return 8;
    default: return 0;
  }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace

namespace smmo {
int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SMMO_OK;
  g_last_cuda = (int)e;
  return SMMO_E_CUDA;
}

void concrete_subtree(const smmo_heap* h, int c, std::vector<int>* out) {
  if (!h->classes[c].abstract) out->push_back(c);
  for (int ch : h->classes[c].children) concrete_subtree(h, ch, out);
}
}  // namespace smmo

// =========================================================== kernels
// Fills level l of a hierarchical bitmap so that exactly the first nbits
// bits are set (initial free bitmap: every block free, Sec. 5.2.4).
__global__ void k_fill_bitmap(unsigned long long* w, uint32_t nwords, uint64_t nbits) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += gridDim.x * blockDim.x) {
    const uint64_t lo = (uint64_t)i * 64;
    unsigned long long v = 0;
    if (lo + 64 <= nbits) v = kAll;
    else if (lo < nbits) v = (1ull << (nbits - lo)) - 1;
    w[i] = v;
  }
}

// Enumeration of the allocated blocks of class c into h.R (the thesis'
// indices(), Alg. 5.5, with the iteration-bitmap snapshot fused in).  One
// warp per level-0 container (64 blocks) per round: the level-1 bit is
// tested first so empty regions of the heap are skipped without reading
// level 0; the CTA sums its eight containers' blocks and reserves their
// output slots with one atomicAdd (one per container would serialise on the
// counter), and the two halves of a container are written by the 32 lanes
// (block index, class, bitmap snapshot).
__global__ void __launch_bounds__(256) k_enumerate(HeapView h, int c) {
  __shared__ uint32_t wcnt[8], wbase[8], cbase;
  const unsigned long long* L0 = bm_level(h, bm_alloc(h, c), 0);
  const unsigned long long* L1 = h.nlevels > 1 ? bm_level(h, bm_alloc(h, c), 1) : nullptr;
  const uint32_t nw = h.level_words[0];
  // level-1 bits of the containers of one level-0 word (1 or 2 of them)
  const uint32_t per_word = 6 - h.bm_shift;
  const unsigned long long l1mask = (1ull << (1u << per_word)) - 1;
  const unsigned long long capmask = h.cls[c].capmask;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t rounds = (nw + nwarps - 1) / nwarps;  // the same in every CTA
  const unsigned lt = (1u << lane) - 1;
  uint32_t objs = 0, blks = 0;
  for (uint32_t r = 0; r < rounds; ++r) {
    const uint32_t w = r * nwarps + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    unsigned long long word = 0;
    if (w < nw) {
      const uint32_t c0 = w << per_word;  // first container of word w
      if (!L1 || ((L1[c0 >> 6] >> (c0 & 63)) & l1mask)) word = L0[w];
    }
    if (lane == 0) wcnt[warp] = (uint32_t)__popcll(word);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int i = 0; i < 8; ++i) { wbase[i] = tot; tot += wcnt[i]; }
      cbase = tot ? atomicAdd(h.rcnt, tot) : 0u;
    }
    __syncthreads();
    if (word == 0) continue;
    const uint32_t lo = (uint32_t)word, hi = (uint32_t)(word >> 32);
    const uint32_t base = cbase + wbase[warp];
    unsigned long long b0 = 0, b1 = 0;
    if ((lo >> lane) & 1) b0 = __ldcg(h.alloc_bm + w * 64 + lane) & capmask;
    if ((hi >> lane) & 1) b1 = __ldcg(h.alloc_bm + w * 64 + 32 + lane) & capmask;
    if ((lo >> lane) & 1) {
      REntry e;
      e.block = w * 64 + lane; e.cls = (uint32_t)c; e.bits = b0;
      h.R[base + __popc(lo & lt)] = e;
      objs += __popcll(b0);
    }
    if ((hi >> lane) & 1) {
      REntry e;
      e.block = w * 64 + 32 + lane; e.cls = (uint32_t)c; e.bits = b1;
      h.R[base + __popc(lo) + __popc(hi & lt)] = e;
      objs += __popcll(b1);
    }
    if (lane == 0) blks += __popcll(word);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) objs += __shfl_xor_sync(0xFFFFFFFFu, objs, o);
  if (lane == 0 && (objs | blks)) {
    count(h, SMMO_CTR_ENUM_OBJ, objs);
    count(h, SMMO_CTR_ENUM_BLK, blks);
  }
}

// First `want` free blocks in ascending order (bulk creation takes whole
// blocks).  Single CTA: chunked scan of the level-0 free containers.
__global__ void __launch_bounds__(1024) k_find_free(HeapView h, uint32_t want, uint32_t* out,
                                                    unsigned long long* found) {
  __shared__ uint32_t psum[1024];
  __shared__ uint32_t running;
  const unsigned long long* L0 = bm_level(h, bm_free(), 0);
  const uint32_t nw = h.level_words[0];
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nw; base += 1024) {
    if (running >= want) break;
    const uint32_t i = base + threadIdx.x;
    const unsigned long long w = i < nw ? L0[i] : 0ull;
    psum[threadIdx.x] = __popcll(w);
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {  // inclusive scan
      const uint32_t v = threadIdx.x >= o ? psum[threadIdx.x - o] : 0;
      __syncthreads();
      psum[threadIdx.x] += v;
      __syncthreads();
    }
    uint32_t pos = running + psum[threadIdx.x] - __popcll(w);
    unsigned long long ww = w;
    while (ww && pos < want) {
      const int b = __ffsll((long long)ww) - 1;
      ww &= ww - 1;
      out[pos++] = i * 64 + b;
    }
    __syncthreads();
    if (threadIdx.x == 1023) running += psum[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *found = running < want ? running : want;
}

// Claims the listed free blocks for class c and fills them with n objects
// in order (block j holds objects j*cap .. j*cap+cap-1).
__global__ void k_bulk_claim(HeapView h, uint32_t c, const uint32_t* list, uint32_t nb,
                             uint64_t n, uint32_t cap, unsigned long long capmask) {
  if (h.st->aux[0] < nb) {  // k_find_free found too few free blocks
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(h, SMMO_E_OOM, nb);
    return;
  }
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += gridDim.x * blockDim.x) {
    const uint32_t bid = list[j];
    if (!bm_try_clear(h, bm_free(), bid)) { set_error(h, SMMO_E_CONTENTION, bid); continue; }
    const uint64_t rem = n - (uint64_t)j * cap;
    const uint64_t fill64 = rem < cap ? rem : cap;
    const uint32_t fill = (uint32_t)fill64;
    h.block_type[bid] = c;
    const unsigned long long used = fill >= 64 ? kAll : ((1ull << fill) - 1);
    h.alloc_bm[bid] = ~capmask | used;
    bm_set(h, bm_alloc(h, c), bid);
    if (fill < cap) bm_set(h, bm_active(h, c), bid);
    if (fill <= h.cls[c].dlimit) bm_set(h, bm_defrag(h, c), bid);
  }
}

struct ColSrc {
  const void* p[SMMO_MAX_COLS];
};

__device__ __forceinline__ void copy_elem(void* dst, const void* src, uint32_t sz) {
  switch (sz) {
    case 1: *(uint8_t*)dst = *(const uint8_t*)src; break;
    case 2: *(uint16_t*)dst = *(const uint16_t*)src; break;
    case 4: *(uint32_t*)dst = *(const uint32_t*)src; break;
    default: *(uint64_t*)dst = *(const uint64_t*)src; break;
  }
}

__global__ void k_bulk_copy(HeapView h, uint32_t c, const uint32_t* list, uint64_t n,
                            ColSrc src, uint32_t ncols, uint32_t* out_handles, uint32_t nb) {
  const ClassLayout& L = h.cls[c];
  const uint32_t cap = L.cap;
  if (h.st->aux[0] < nb) return;  // too few free blocks: k_bulk_claim recorded OOM
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t bid = list[i / cap];
    const uint32_t slot = (uint32_t)(i % cap);
    uint8_t* blk = block_data(h, bid);
    for (uint32_t k = 0; k < ncols; ++k) {
      const uint32_t sz = L.col_size[k];
      if (src.p[k])
        copy_elem(blk + L.col_off[k] + (size_t)slot * sz, (const uint8_t*)src.p[k] + i * sz, sz);
    }
    if (out_handles) out_handles[i] = (bid << 6) | slot;
    if (L.inst_col >= 0) {  // an instance index must name a row of the table
      const uint32_t k = *reinterpret_cast<const uint32_t*>(blk + L.col_off[L.inst_col] + (size_t)slot * 4);
      if (k >= h.n_inst) set_error(h, SMMO_E_BOUNDS, ((unsigned long long)k << 32) | ((bid << 6) | slot));
    }
  }
}

// Expands the enumerated blocks into object handles.
__global__ void k_expand(HeapView h, uint32_t* out, uint64_t cap_out, unsigned long long* total) {
  const uint32_t n = *h.rcnt;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const REntry e = h.R[i];
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(total, (unsigned long long)__popcll(e.bits));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t half = 0; half < 2; ++half) {
      const uint32_t slot = half * 32 + lane;
      if ((e.bits >> slot) & 1) {
        const uint64_t r = base + __popcll(e.bits & ((1ull << slot) - 1));
        if (r < cap_out) out[r] = (e.block << 6) | slot;
      }
    }
  }
}

struct ColDst {
  void* p[SMMO_MAX_COLS];
  int col[SMMO_MAX_COLS];
};

__global__ void k_gather(HeapView h, const uint32_t* handles, uint64_t n, ColDst dst, int ncol) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t hd = handles[i];
    if (hd == kNull || (hd >> 6) >= h.num_blocks) { set_error(h, SMMO_E_BOUNDS, hd); continue; }
    const uint32_t t = h.block_type[hd >> 6];
    if (t >= (uint32_t)h.num_classes) { set_error(h, SMMO_E_BAD_HANDLE, hd); continue; }
    const ClassLayout& L = h.cls[t];
    const uint8_t* blk = block_data(h, hd >> 6);
    for (int k = 0; k < ncol; ++k) {
      const uint32_t sz = L.col_size[dst.col[k]];
      copy_elem((uint8_t*)dst.p[k] + i * sz, blk + L.col_off[dst.col[k]] + (size_t)(hd & 63) * sz, sz);
    }
  }
}

// Per-class live objects, blocks and free slots (fragmentation F, Sec. 6.2.2).
__global__ void __launch_bounds__(256) k_stats(HeapView h) {
  __shared__ unsigned long long live[SMMO_MAX_CLASSES], blocks[SMMO_MAX_CLASSES],
      freeslots[SMMO_MAX_CLASSES];
  if (threadIdx.x < SMMO_MAX_CLASSES) {
    live[threadIdx.x] = 0; blocks[threadIdx.x] = 0; freeslots[threadIdx.x] = 0;
  }
  __syncthreads();
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < h.num_blocks;
       b += gridDim.x * blockDim.x) {
    const uint32_t t = h.block_type[b];
    if (t < (uint32_t)h.num_classes && bm_get(h, bm_alloc(h, t), b)) {
      const ClassLayout& L = h.cls[t];
      const uint32_t f = __popcll(h.alloc_bm[b] & L.capmask);
      atomicAdd(&live[t], (unsigned long long)f);
      atomicAdd(&blocks[t], 1ull);
      atomicAdd(&freeslots[t], (unsigned long long)(L.cap - f));
    }
  }
  __syncthreads();
  if (threadIdx.x < (uint32_t)h.num_classes) {
    atomicAdd(&h.st->stat_live[threadIdx.x], live[threadIdx.x]);
    atomicAdd(&h.st->stat_blocks[threadIdx.x], blocks[threadIdx.x]);
    atomicAdd(&h.st->stat_free_slots[threadIdx.x], freeslots[threadIdx.x]);
  }
  const unsigned long long* F = bm_level(h, bm_free(), 0);
  unsigned long long fb = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < h.level_words[0];
       i += gridDim.x * blockDim.x)
    fb += __popcll(F[i]);
  if (fb) atomicAdd(&h.st->stat_free_blocks, fb);
}

// Invariant checks (see smmo_heap_check).  Counts violations into aux[2].
__global__ void k_check_levels(HeapView h, int k) {
  unsigned long long bad = 0;
  for (uint32_t l = 1; l < h.nlevels; ++l) {
    const unsigned long long* hi = bm_level(h, k, l);
    // bit i of level l for every container i of level l - 1
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < h.level_bits[l];
         i += gridDim.x * blockDim.x) {
      const bool want = bm_container(h, k, l - 1, i) != 0;
      const bool have = (hi[i >> 6] >> (i & 63)) & 1;
      if (want != have) ++bad;
    }
    // bits past the last container stay clear
    const uint32_t top = h.level_words[l] * 64;
    for (uint32_t i = h.level_bits[l] + blockIdx.x * blockDim.x + threadIdx.x; i < top;
         i += gridDim.x * blockDim.x)
      if ((hi[i >> 6] >> (i & 63)) & 1) ++bad;
  }
  if (bad) atomicAdd(&h.st->aux[2], bad);
}

__global__ void k_check_blocks(HeapView h) {
  unsigned long long bad = 0;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < h.num_blocks;
       b += gridDim.x * blockDim.x) {
    const bool fr = bm_get(h, bm_free(), b);
    int nalloc = 0, owner = -1;
    for (int c = 0; c < h.num_classes; ++c) {
      const bool a = bm_get(h, bm_alloc(h, c), b);
      const bool ac = bm_get(h, bm_active(h, c), b);
      if (a) { ++nalloc; owner = c; }
      if (ac && !a) ++bad;
    }
    if (fr && nalloc) ++bad;
    if (!fr && nalloc != 1) ++bad;
    if (nalloc == 1) {
      const ClassLayout& L = h.cls[owner];
      const unsigned long long bm = h.alloc_bm[b];
      if (h.block_type[b] != (uint32_t)owner) ++bad;
      if ((bm & ~L.capmask) != ~L.capmask) ++bad;          // padding bits set
      if ((bm & L.capmask) == 0) ++bad;                     // empty but allocated
      const bool full = bm == kAll;
      if (bm_get(h, bm_active(h, owner), b) == full) ++bad;  // active iff not full
      const bool cand = (uint32_t)__popcll(bm & L.capmask) <= L.dlimit;
      if (bm_get(h, bm_defrag(h, owner), b) != cand) ++bad;  // candidate iff fill <= dlimit
    } else {
      for (int c = 0; c < h.num_classes; ++c)
        if (bm_get(h, bm_defrag(h, c), b)) ++bad;
    }
  }
  if (bad) atomicAdd(&h.st->aux[2], bad);
}

// =========================================================== host helpers
namespace smmo {

static int launch_enumerate(smmo_heap* h, const HeapView& v, int c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(v.rcnt, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t grid = (v.level_words[0] + 7) / 8;  // one warp per container
  grid = std::max(1u, std::min(grid, (uint32_t)h->num_sms * 8));
  k_enumerate<<<grid, 256, 0, s>>>(v, c);
  return cuda_status(cudaGetLastError());
}

int enumerate(smmo_heap* h, int c, cudaStream_t s) { return launch_enumerate(h, h->view, c, s); }

static int snapshot_alloc(smmo_heap* h, Snapshot* sn) {
  if (sn->buf) return SMMO_OK;
  // M entries and the count, in one allocation
  const size_t bytes = (size_t)h->view.num_blocks * sizeof(REntry) + 16;
  cudaError_t e = cudaMalloc(&sn->buf, bytes);
  if (e != cudaSuccess) { sn->buf = nullptr; return cuda_status(e); }
  sn->view = h->view;
  sn->view.R = reinterpret_cast<REntry*>(sn->buf);
  sn->view.rcnt = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(sn->buf) +
                                              (size_t)h->view.num_blocks * sizeof(REntry));
  return SMMO_OK;
}

int Snapshot::take_subtree(smmo_heap* h, int c, cudaStream_t s) {
  if (!h->frozen) return SMMO_E_FROZEN;
  int st = snapshot_alloc(h, this);
  if (st) return st;
  cls = c;
  std::vector<int> cs;
  concrete_subtree(h, c, &cs);
  for (int k : cs)
    if (h->classes[k].layout.cap > 64) return SMMO_E_UNSUPPORTED;
  // the count is reset once: each class's blocks are appended
  cudaError_t e = cudaMemsetAsync(view.rcnt, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t grid = (view.level_words[0] + 7) / 8;
  grid = std::max(1u, std::min(grid, (uint32_t)h->num_sms * 8));
  for (int k : cs) k_enumerate<<<grid, 256, 0, s>>>(view, k);
  return cuda_status(cudaGetLastError());
}

int Snapshot::take(smmo_heap* h, int c, cudaStream_t s) {
  if (!h->frozen) return SMMO_E_FROZEN;
  int st = snapshot_alloc(h, this);
  if (st) return st;
  cls = c;
  return launch_enumerate(h, view, c, s);
}

void Snapshot::release() {
  if (buf) cudaFree(buf);
  buf = nullptr;
}

// Enumeration scratch: one REntry per block, and at least room for the
// compaction scan's per-word offsets and per-chunk totals (level-0 words
// rounded up to 1024, plus 1024), which reuse it.
static uint64_t rscratch_bytes(uint64_t M) {
  const uint64_t words = (M + 63) / 64;
  const uint64_t scan = ((words + 1023) / 1024 * 1024 + 1024) * 4;
  return std::max<uint64_t>(M * 16, scan);
}

int freeze(smmo_heap* h, cudaStream_t s) {
  if (h->frozen) return SMMO_OK;
  const int nc = (int)h->classes.size();
  if (nc == 0) return SMMO_E_UNSUPPORTED;
  // object sizes and the smallest concrete class
  int min_size = 1 << 30;
  for (auto& ci : h->classes) {
    int sz = 0, ncols = 0;
    for (auto& f : ci.fields) { sz += esize(f.elem_type) * f.count; ncols += f.count; }
    ci.object_bytes = sz;
    ci.ncols = ncols;
    if (ncols > SMMO_MAX_COLS) return SMMO_E_INVALID_ARG;
    if (!ci.abstract && sz > 0) min_size = std::min(min_size, sz);
  }
  if (min_size == (1 << 30)) return SMMO_E_UNSUPPORTED;
  uint32_t data_bytes = h->cfg.block_data_bytes ? h->cfg.block_data_bytes : 64u * (uint32_t)min_size;
  data_bytes = (uint32_t)align_up(data_bytes, 64);
  // capacity N_T: the largest N <= 64 whose 16-byte-aligned SOA columns fit
  for (auto& ci : h->classes) {
    ClassLayout& L = ci.layout;
    memset(&L, 0, sizeof(L));
    int cap = 0;
    for (int N = 64; N >= 1; --N) {
      size_t need = 0;
      for (auto& f : ci.fields)
        for (int k = 0; k < f.count; ++k) need = align_up(need, 16) + (size_t)N * esize(f.elem_type);
      if (need <= data_bytes) { cap = N; break; }
    }
    if (!ci.abstract && cap < 2) return SMMO_E_UNSUPPORTED;
    L.cap = (uint32_t)cap;
    L.ncols = (uint32_t)ci.ncols;
    L.inst_col = -1;
    L.capmask = cap >= 64 ? kAll : ((1ull << cap) - 1);
    L.dlimit = (uint32_t)((uint64_t)cap * (uint64_t)h->cfg.defrag_factor / (uint64_t)(h->cfg.defrag_factor + 1));
    size_t off = 0;
    int col = 0;
    for (auto& f : ci.fields)
      for (int k = 0; k < f.count; ++k) {
        off = align_up(off, 16);
        if (f.elem_type == SMMO_INSTANCE && L.inst_col < 0) L.inst_col = col;
        L.col_off[col] = (uint32_t)off;
        L.col_size[col] = (uint32_t)esize(f.elem_type);
        off += (size_t)cap * esize(f.elem_type);
        ++col;
      }
  }
  const size_t block_bytes = data_bytes;
  const int nbm = 1 + 3 * nc;
  // carve: state | layouts | alloc_bm | block_type | R | scratch | moved | bitmaps | unit marks | instances | data
  const size_t fixed = align_up(sizeof(DeviceState), 256) +
                       align_up(sizeof(ClassLayout) * SMMO_MAX_CLASSES, 256) + 8 * 256;
  if (h->buf_bytes <= fixed) return SMMO_E_OOM;
  // levels of F-bit containers (F = bitmap fan-out): level 0 has M bits,
  // level l + 1 one bit per container of level l, up to a level that is a
  // single container; each level is stored in whole 64-bit words
  const uint32_t fshift = h->cfg.bitmap_fanout == 32 ? 5u : 6u;
  auto bm_geom = [fshift](uint64_t M, uint32_t* lw, uint32_t* lo, uint32_t* lb, uint32_t* nl) {
    uint64_t bits = M, off = 0;
    int l = 0;
    for (;;) {
      const uint64_t w = (bits + 63) / 64;
      lw[l] = (uint32_t)w;
      lo[l] = (uint32_t)off;
      lb[l] = (uint32_t)bits;
      off += w;
      ++l;
      if (bits <= (1ull << fshift) || l == SMMO_MAX_LEVELS) break;
      bits = (bits + (1ull << fshift) - 1) >> fshift;
    }
    *nl = (uint32_t)l;
    return bits <= (1ull << fshift) ? (uint64_t)align_up(off, 32) : 0ull;  // 0: too many levels
  };
  const size_t inst_bytes = h->batch.size() * sizeof(Inst);
  auto need_bytes = [&](uint64_t M) {
    uint32_t lw[SMMO_MAX_LEVELS], lo[SMMO_MAX_LEVELS], lb[SMMO_MAX_LEVELS], nl;
    const uint64_t bw = bm_geom(M, lw, lo, lb, &nl);
    return fixed + align_up(M * 8, 256) + align_up(M * 4, 256) + align_up(rscratch_bytes(M), 256) +
           align_up(M * 4 + 1024, 256) + align_up((M + 63) / 64 * 8, 256) + align_up(bw * 8 * nbm, 256) +
           align_up(M * 8, 256) +
           align_up(inst_bytes, 256) + M * block_bytes;
  };
  uint64_t M = h->buf_bytes / (block_bytes + 48);
  M = std::min<uint64_t>(M, (1ull << 26) - 1);
  while (M > 0 && need_bytes(M) > h->buf_bytes) M -= std::max<uint64_t>(1, M / 1000);
  if (M < 2) return SMMO_E_OOM;
  HeapView& v = h->view;
  memset(&v, 0, sizeof(v));
  uint32_t lw[SMMO_MAX_LEVELS], lo[SMMO_MAX_LEVELS], lb[SMMO_MAX_LEVELS], nl;
  const uint64_t bw = bm_geom(M, lw, lo, lb, &nl);
  if (bw == 0) return SMMO_E_UNSUPPORTED;
  uint8_t* p = h->buf;
  auto take = [&](size_t bytes) { uint8_t* r = p; p += align_up(bytes, 256); return r; };
  v.st = (DeviceState*)take(sizeof(DeviceState));
  h->d_layouts = (ClassLayout*)take(sizeof(ClassLayout) * SMMO_MAX_CLASSES);
  v.cls = h->d_layouts;
  v.alloc_bm = (unsigned long long*)take(M * 8);
  v.block_type = (uint32_t*)take(M * 4);
  v.R = (REntry*)take(rscratch_bytes(M));
  v.rcnt = &v.st->rcount;
  h->d_scratch = (uint32_t*)take(M * 4 + 1024);
  h->d_moved = (unsigned long long*)take((M + 63) / 64 * 8);
  v.bitmaps = (unsigned long long*)take(bw * 8 * nbm);
  v.umark = (uint32_t*)take(M * 8);  // two 32-slot units per block
  h->d_inst = h->batch.empty() ? nullptr : (Inst*)take(inst_bytes);
  v.inst = h->d_inst;
  v.n_inst = (uint32_t)h->batch.size();
  v.data = p;
  v.block_bytes = (uint32_t)block_bytes;
  v.num_blocks = (uint32_t)M;
  v.bm_words = (uint32_t)bw;
  v.nlevels = nl;
  v.bm_shift = fshift;
  for (uint32_t l = 0; l < nl; ++l) { v.level_words[l] = lw[l]; v.level_off[l] = lo[l]; v.level_bits[l] = lb[l]; }
  v.num_classes = nc;
  v.lookup_retries = h->cfg.lookup_retries;
  v.alloc_retries = h->cfg.alloc_retries;
  v.bitmap_spins = h->cfg.bitmap_spins;
  v.debug = h->cfg.debug_checks;
  // device initialisation
  std::vector<ClassLayout> lay(SMMO_MAX_CLASSES);
  memset(lay.data(), 0, sizeof(ClassLayout) * SMMO_MAX_CLASSES);
  for (int c = 0; c < nc; ++c) lay[c] = h->classes[c].layout;
  cudaError_t e = cudaMemsetAsync(v.st, 0, sizeof(DeviceState), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_layouts, lay.data(), sizeof(ClassLayout) * SMMO_MAX_CLASSES, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.alloc_bm, 0xFF, M * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.block_type, 0xFF, M * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.bitmaps, 0, bw * 8 * nbm, s);
  std::vector<Inst> itab(h->batch.size());
  for (size_t i = 0; i < h->batch.size(); ++i) {
    const smmo_instance_desc& d = h->batch[i];
    Inst& r = itab[i];
    memset(&r, 0, sizeof(r));
    r.cell_base = (uint32_t)d.base;
    r.W = d.W; r.H = d.H; r.id = d.id;
    r.wdiv = d.W ? ~0ull / d.W + 1 : 0ull;
    r.count = (uint32_t)d.count;
    r.kind = d.kind;
    r.param[0] = d.param[0]; r.param[1] = d.param[1];
  }
  if (e == cudaSuccess && !itab.empty())
    e = cudaMemcpyAsync(h->d_inst, itab.data(), inst_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  for (uint32_t l = 0; l < nl; ++l) {  // the free bitmap: every block free
    const uint32_t grid = std::min<uint32_t>((lw[l] + 255) / 256, 4096);
    k_fill_bitmap<<<std::max(grid, 1u), 256, 0, s>>>(v.bitmaps + lo[l], lw[l], lb[l]);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  h->frozen = true;
  return SMMO_OK;
}
}  // namespace smmo

// =========================================================== method table
namespace {
struct Table {
  const smmo::MethodEntry* e;
  const int* n;
};
const Table kTables[] = {{g_methods_test, &g_methods_test_n},
                         {g_methods_wator, &g_methods_wator_n},
                         {g_methods_gol, &g_methods_gol_n},
                         {g_methods_nasch, &g_methods_nasch_n},
                         {g_methods_nbody, &g_methods_nbody_n},
                         {g_methods_bh, &g_methods_bh_n},
                         {g_methods_bfs, &g_methods_bfs_n},
                         {g_methods_structure, &g_methods_structure_n}};
}  // namespace

const smmo::MethodEntry* smmo::method_by_id(int id) {
  if (id < 0) return nullptr;
  for (const Table& t : kTables) {
    if (id < *t.n) return &t.e[id];
    id -= *t.n;
  }
  return nullptr;
}

// =========================================================== C ABI
extern "C" {

const char* smmo_status_string(int st) {
  switch (st) {
    case SMMO_OK: return "ok";
    case SMMO_E_INVALID_ARG: return "invalid argument";
    case SMMO_E_OOM: return "heap has too few free blocks";
    case SMMO_E_DEVICE_OOM: return "device new found no free block";
    case SMMO_E_CONTENTION: return "device retry budget exhausted";
    case SMMO_E_CUDA: return "CUDA error";
    case SMMO_E_TIMEOUT: return "timeout";
    case SMMO_E_BAD_HANDLE: return "bad handle (double free or foreign handle)";
    case SMMO_E_BOUNDS: return "bounds check failed";
    case SMMO_E_UNSUPPORTED: return "unsupported";
    case SMMO_E_FROZEN: return "heap geometry already fixed";
    default: return "unknown status";
  }
}

int smmo_last_cuda_error(void) { return g_last_cuda; }

void smmo_heap_config_default(smmo_heap_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->block_data_bytes = 0;
  c->lookup_retries = 5;
  c->alloc_retries = 4096;
  c->bitmap_spins = 1 << 20;
  c->threads_per_cta = 256;
  c->ctas_per_sm = 8;
  c->debug_checks = 0;
  c->defrag_factor = 1;
  c->bitmap_fanout = 64;
}

int smmo_heap_create(const smmo_heap_config* cfg, void* dev_buf, size_t buf_bytes, void* stream,
                     smmo_heap** out) {
  (void)stream;
  if (!dev_buf || !out || buf_bytes < (1u << 20) || ((uintptr_t)dev_buf & 255)) return SMMO_E_INVALID_ARG;
  smmo_heap_config c;
  smmo_heap_config_default(&c);
  if (cfg) c = *cfg;
  if (c.threads_per_cta <= 0 || c.threads_per_cta % 64 || c.threads_per_cta > 512 ||
      c.ctas_per_sm <= 0 || c.lookup_retries < 1 || c.alloc_retries < 1 || c.bitmap_spins < 1 ||
      c.defrag_factor < 1 || c.defrag_factor > 63 || (c.bitmap_fanout != 32 && c.bitmap_fanout != 64))
    return SMMO_E_INVALID_ARG;
  smmo_heap* h = new smmo_heap();
  h->cfg = c;
  h->buf = (uint8_t*)dev_buf;
  h->buf_bytes = buf_bytes;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { delete h; return smmo::cuda_status(e); }
  *out = h;
  return SMMO_OK;
}

int smmo_heap_destroy(smmo_heap* h) {
  if (!h) return SMMO_E_INVALID_ARG;
  delete h;
  return SMMO_OK;
}

int smmo_class_register(smmo_heap* h, const char* name, const smmo_field_desc* fields, int nfields,
                        int parent, int is_abstract, int* class_id) {
  if (!h || !name || nfields < 0 || (nfields > 0 && !fields)) return SMMO_E_INVALID_ARG;
  if (h->frozen) return SMMO_E_FROZEN;
  if ((int)h->classes.size() >= SMMO_MAX_CLASSES) return SMMO_E_UNSUPPORTED;
  if (parent < -1 || parent >= (int)h->classes.size()) return SMMO_E_INVALID_ARG;
  for (auto& c : h->classes)
    if (c.name == name) return SMMO_E_INVALID_ARG;
  ClassInfo ci;
  ci.name = name;
  ci.parent = parent;
  ci.abstract = is_abstract ? 1 : 0;
  std::vector<smmo_field_desc> all;
  std::vector<std::string> names;
  if (parent >= 0) { all = h->classes[parent].fields; names = h->classes[parent].field_names; }
  for (int i = 0; i < nfields; ++i) {
    smmo_field_desc f = fields[i];
    if (esize(f.elem_type) == 0 || f.count < 1) return SMMO_E_INVALID_ARG;
    all.push_back(f);
    names.push_back(f.name ? f.name : "");
  }
  if ((int)all.size() > SMMO_MAX_FIELDS) return SMMO_E_UNSUPPORTED;
  ci.fields = all;
  ci.field_names = names;
  for (size_t i = 0; i < ci.fields.size(); ++i) ci.fields[i].name = nullptr;
  const int id = (int)h->classes.size();
  h->classes.push_back(ci);
  if (parent >= 0) h->classes[parent].children.push_back(id);
  if (class_id) *class_id = id;
  return SMMO_OK;
}

int smmo_class_lookup(smmo_heap* h, const char* name, int* class_id) {
  if (!h || !name || !class_id) return SMMO_E_INVALID_ARG;
  for (size_t i = 0; i < h->classes.size(); ++i)
    if (h->classes[i].name == name) { *class_id = (int)i; return SMMO_OK; }
  return SMMO_E_INVALID_ARG;
}

int smmo_heap_freeze(smmo_heap* h) {
  if (!h) return SMMO_E_INVALID_ARG;
  return smmo::freeze(h, 0);
}

int smmo_class_info(smmo_heap* h, int c, int* nfields, int* capacity, int* object_bytes) {
  if (!h || c < 0 || c >= (int)h->classes.size()) return SMMO_E_INVALID_ARG;
  if (nfields) *nfields = (int)h->classes[c].fields.size();
  if (!h->frozen) return SMMO_E_UNSUPPORTED;
  if (capacity) *capacity = (int)h->classes[c].layout.cap;
  if (object_bytes) *object_bytes = h->classes[c].object_bytes;
  return SMMO_OK;
}

int smmo_class_layout(smmo_heap* h, int c, uint32_t* col_off, int* ncols, uint32_t* block_bytes,
                      void** data_base) {
  if (!h || c < 0 || c >= (int)h->classes.size()) return SMMO_E_INVALID_ARG;
  if (!h->frozen) return SMMO_E_UNSUPPORTED;
  const ClassInfo& ci = h->classes[c];
  if (col_off)
    for (int k = 0; k < ci.ncols; ++k) col_off[k] = ci.layout.col_off[k];
  if (ncols) *ncols = ci.ncols;
  if (block_bytes) *block_bytes = h->view.block_bytes;
  if (data_base) *data_base = h->view.data;
  return SMMO_OK;
}

int smmo_method_lookup(smmo_heap* h, const char* name, int* method_id) {
  if (!name || !method_id) return SMMO_E_INVALID_ARG;
  int base = 0;
  for (const Table& t : kTables) {
    for (int i = 0; i < *t.n; ++i)
      if (strcmp(t.e[i].name, name) == 0) {
        // a batch method reads the instance table, which this heap lacks
        if (h && h->frozen && h->batch.empty() && strncmp(name, "test.batch_", 11) == 0)
          return SMMO_E_UNSUPPORTED;
        *method_id = base + i;
        return SMMO_OK;
      }
    base += *t.n;
  }
  return SMMO_E_INVALID_ARG;
}

int smmo_batch_define(smmo_heap* h, const smmo_instance_desc* inst, int n_inst) {
  if (!h || !inst || n_inst < 1 || n_inst > (1 << 20)) return SMMO_E_INVALID_ARG;
  if (h->frozen) return SMMO_E_FROZEN;
  if (!h->batch.empty()) return SMMO_E_UNSUPPORTED;  // once per heap
  uint64_t end = 0;
  for (int i = 0; i < n_inst; ++i) {
    const smmo_instance_desc& d = inst[i];
    if (d.count > 0) {
      if (d.base < end || d.base + d.count > (1ull << 32) || d.base + d.count < d.base) return SMMO_E_INVALID_ARG;
      end = d.base + d.count;
    }
  }
  h->batch.assign(inst, inst + n_inst);
  return SMMO_OK;
}

int smmo_batch_count(smmo_heap* h, int* n_inst) {
  if (!h || !n_inst) return SMMO_E_INVALID_ARG;
  *n_inst = (int)h->batch.size();
  return SMMO_OK;
}

int smmo_bulk_new(smmo_heap* h, int c, int64_t n, const void* const* field_src,
                  smmo_handle* out_handles, int64_t* out_first_block, void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size() || n < 0) return SMMO_E_INVALID_ARG;
  if (h->classes[c].abstract) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = smmo::freeze(h, s);
  if (st) return st;
  if (n > 0) ++h->bulk_calls;
  if (out_first_block) *out_first_block = -1;
  if (n == 0) return SMMO_OK;
  const ClassInfo& ci = h->classes[c];
  const uint32_t cap = ci.layout.cap;
  const uint64_t nb64 = ((uint64_t)n + cap - 1) / cap;
  if (nb64 > h->view.num_blocks) return SMMO_E_OOM;
  const uint32_t nb = (uint32_t)nb64;
  // k_find_free leaves the number of blocks it found in aux[0]; the claim
  // and copy kernels do nothing (the claim records SMMO_E_OOM) when it is
  // short, so no host round trip is needed
  unsigned long long* found_d = &h->view.st->aux[0];
  k_find_free<<<1, 1024, 0, s>>>(h->view, nb, h->d_scratch, found_d);
  const uint32_t g1 = std::min<uint32_t>((nb + 255) / 256, 8192);
  k_bulk_claim<<<std::max(g1, 1u), 256, 0, s>>>(h->view, c, h->d_scratch, nb, (uint64_t)n, cap, ci.layout.capmask);
  ColSrc src;
  memset(&src, 0, sizeof(src));
  for (int k = 0; k < ci.ncols; ++k) src.p[k] = field_src ? field_src[k] : nullptr;
  const uint64_t g2 = std::min<uint64_t>(((uint64_t)n + 255) / 256, 65535);
  k_bulk_copy<<<(unsigned)std::max<uint64_t>(g2, 1), 256, 0, s>>>(h->view, c, h->d_scratch, (uint64_t)n, src, ci.ncols,
                                                                  out_handles, nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return smmo::cuda_status(e);
  if (!out_first_block) return SMMO_OK;
  // synchronous form: the first and last block used, and an OOM now
  unsigned long long found = 0;
  uint32_t first = 0, last = 0;
  e = cudaMemcpyAsync(&found, found_d, sizeof(found), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&first, h->d_scratch, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last, h->d_scratch + nb - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  if (found < nb) return SMMO_E_OOM;
  if (last - first == nb - 1) *out_first_block = first;
  return SMMO_OK;
}

int smmo_parallel_do(smmo_heap* h, int c, int method_id, const void* args, size_t args_bytes,
                     void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size()) return SMMO_E_INVALID_ARG;
  const smmo::MethodEntry* m = smmo::method_by_id(method_id);
  if (!m || !m->launch || args_bytes != m->args_size || (args_bytes && !args) || args_bytes > 1024)
    return SMMO_E_INVALID_ARG;
  if (!h->frozen) return SMMO_OK;  // no object exists yet
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> cls;
  smmo::concrete_subtree(h, c, &cls);
  for (int k : cls) {
    int st = smmo::enumerate(h, k, s);
    if (st) return st;
    st = m->launch(h, k, args, s);
    if (st) return st;
  }
  return SMMO_OK;
}

namespace {
__global__ void k_set_i64(long long* p, long long v) { *p = v; }
long long host_identity(int op) {
  switch (op) {
    case SMMO_REDUCE_MIN: return 0x7FFFFFFFFFFFFFFFll;
    case SMMO_REDUCE_MAX: return (long long)0x8000000000000000ull;
    case SMMO_REDUCE_AND: return -1ll;
    default: return 0ll;
  }
}
}  // namespace

int smmo_parallel_do_and_reduce(smmo_heap* h, int c, int method_id, const void* args, size_t args_bytes, int op,
                                int64_t* dev_result, void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size() || !dev_result || op < SMMO_REDUCE_SUM || op > SMMO_REDUCE_AND)
    return SMMO_E_INVALID_ARG;
  const smmo::MethodEntry* m = smmo::method_by_id(method_id);
  if (!m || !m->reduce || args_bytes != m->args_size || (args_bytes && !args) || args_bytes > 1024)
    return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  long long* out = reinterpret_cast<long long*>(dev_result);
  k_set_i64<<<1, 1, 0, s>>>(out, host_identity(op));
  int st = smmo::cuda_status(cudaGetLastError());
  if (st || !h->frozen) return st;
  std::vector<int> cls;
  smmo::concrete_subtree(h, c, &cls);
  for (int k : cls) {
    st = smmo::enumerate(h, k, s);
    if (st) return st;
    st = m->reduce(h, k, args, op, out, s);
    if (st) return st;
  }
  return SMMO_OK;
}

int smmo_enumerate_live(smmo_heap* h, int c, int include_subclasses, smmo_handle* out, int64_t cap,
                        int64_t* out_count, void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size() || cap < 0 || (cap > 0 && !out)) return SMMO_E_INVALID_ARG;
  if (out_count) *out_count = 0;
  if (!h->frozen) return SMMO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> cls;
  if (include_subclasses) smmo::concrete_subtree(h, c, &cls);
  else if (!h->classes[c].abstract) cls.push_back(c);
  unsigned long long* total = &h->view.st->aux[1];
  cudaError_t e = cudaMemsetAsync(total, 0, sizeof(*total), s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  for (int k : cls) {
    int st = smmo::enumerate(h, k, s);
    if (st) return st;
    k_expand<<<h->num_sms * 4, 256, 0, s>>>(h->view, out, (uint64_t)cap, total);
  }
  unsigned long long t = 0;
  e = cudaMemcpyAsync(&t, total, sizeof(t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  if (out_count) *out_count = (int64_t)t;
  return SMMO_OK;
}

int smmo_gather_fields(smmo_heap* h, int c, const smmo_handle* handles, int64_t n, const int* columns,
                       int ncol, void* const* dst, void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size() || n < 0 || ncol < 0 || ncol > SMMO_MAX_COLS)
    return SMMO_E_INVALID_ARG;
  if (n == 0 || ncol == 0) return SMMO_OK;
  if (!handles || !columns || !dst) return SMMO_E_INVALID_ARG;
  if (!h->frozen) return SMMO_E_UNSUPPORTED;
  ColDst d;
  memset(&d, 0, sizeof(d));
  for (int k = 0; k < ncol; ++k) {
    if (columns[k] < 0 || columns[k] >= h->classes[c].ncols || !dst[k]) return SMMO_E_INVALID_ARG;
    d.p[k] = dst[k];
    d.col[k] = columns[k];
  }
  const uint64_t g = std::min<uint64_t>(((uint64_t)n + 255) / 256, 65535);
  k_gather<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(h->view, handles, (uint64_t)n, d, ncol);
  return smmo::cuda_status(cudaGetLastError());
}

int smmo_heap_get_stats(smmo_heap* h, smmo_heap_stats* out, void* stream) {
  if (!h || !out) return SMMO_E_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->num_classes = (int)h->classes.size();
  if (!h->frozen) return SMMO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceState* st = h->view.st;
  cudaError_t e = cudaMemsetAsync(&st->stat_live, 0,
                                  sizeof(unsigned long long) * (3 * SMMO_MAX_CLASSES + 1), s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  const uint32_t g = std::min<uint32_t>((h->view.num_blocks + 255) / 256, (uint32_t)h->num_sms * 8);
  k_stats<<<std::max(g, 1u), 256, 0, s>>>(h->view);
  std::vector<unsigned char> hs(sizeof(DeviceState));
  e = cudaMemcpyAsync(hs.data(), st, sizeof(DeviceState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  const DeviceState* d = (const DeviceState*)hs.data();
  double fsum = 0, fblk = 0;
  for (int c = 0; c < out->num_classes; ++c) {
    const ClassInfo& ci = h->classes[c];
    out->live_objects[c] = (int64_t)d->stat_live[c];
    out->blocks[c] = (int64_t)d->stat_blocks[c];
    out->capacity[c] = (int)ci.layout.cap;
    out->object_bytes[c] = ci.object_bytes;
    out->fragmentation[c] = d->stat_blocks[c] ? (double)d->stat_free_slots[c] / ((double)ci.layout.cap * d->stat_blocks[c]) : 0.0;
    fsum += out->fragmentation[c] * d->stat_blocks[c];
    fblk += d->stat_blocks[c];
    for (int sh = 0; sh < SMMO_NSHARD; ++sh) {
      out->allocs[c] += (int64_t)d->ctr[sh][SMMO_CTR_ALLOC(c)];
      out->frees[c] += (int64_t)d->ctr[sh][SMMO_CTR_FREE(c)];
    }
  }
  for (int sh = 0; sh < SMMO_NSHARD; ++sh) {
    out->slow_paths += (int64_t)d->ctr[sh][SMMO_CTR_SLOW];
    out->enumerated_objects += (int64_t)d->ctr[sh][SMMO_CTR_ENUM_OBJ];
    out->enumerated_blocks += (int64_t)d->ctr[sh][SMMO_CTR_ENUM_BLK];
  }
  out->fragmentation_all = fblk ? fsum / fblk : 0.0;
  out->free_blocks = (int64_t)d->stat_free_blocks;
  out->num_blocks = h->view.num_blocks;
  out->block_bytes = (int)h->view.block_bytes;
  return SMMO_OK;
}

int smmo_heap_alloc_counters(smmo_heap* h, int64_t* out6, void* stream) {
  if (!h || !out6) return SMMO_E_INVALID_ARG;
  for (int k = 0; k < 6; ++k) out6[k] = 0;
  if (!h->frozen) return SMMO_OK;
  std::vector<unsigned long long> c(SMMO_NSHARD * SMMO_NCTR);
  cudaError_t e = cudaMemcpyAsync(c.data(), h->view.st->ctr, sizeof(unsigned long long) * c.size(),
                                  cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  const int idx[6] = {SMMO_CTR_SLOW, SMMO_CTR_RETRY, SMMO_CTR_REFILL, SMMO_CTR_LOOKUP_MISS,
                      SMMO_CTR_RESERVE_FAIL, SMMO_CTR_ENUM_BLK};
  for (int sh = 0; sh < SMMO_NSHARD; ++sh)
    for (int k = 0; k < 6; ++k) out6[k] += (int64_t)c[(size_t)sh * SMMO_NCTR + idx[k]];
  return SMMO_OK;
}

int smmo_heap_counters(smmo_heap* h, int64_t* enumerated_objects, int64_t* allocs, int64_t* frees,
                       void* stream) {
  if (!h) return SMMO_E_INVALID_ARG;
  if (enumerated_objects) *enumerated_objects = 0;
  if (allocs) *allocs = 0;
  if (frees) *frees = 0;
  if (!h->frozen) return SMMO_OK;
  std::vector<unsigned long long> c(SMMO_NSHARD * SMMO_NCTR);
  cudaError_t e = cudaMemcpyAsync(c.data(), h->view.st->ctr, sizeof(unsigned long long) * c.size(),
                                  cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  for (int sh = 0; sh < SMMO_NSHARD; ++sh) {
    const unsigned long long* r = &c[(size_t)sh * SMMO_NCTR];
    if (enumerated_objects) *enumerated_objects += (int64_t)r[SMMO_CTR_VISIT];
    for (int k = 0; k < SMMO_MAX_CLASSES; ++k) {
      if (allocs) *allocs += (int64_t)r[SMMO_CTR_ALLOC(k)];
      if (frees) *frees += (int64_t)r[SMMO_CTR_FREE(k)];
    }
  }
  return SMMO_OK;
}

int smmo_heap_check(smmo_heap* h, int64_t* violations, void* stream) {
  if (!h || !violations) return SMMO_E_INVALID_ARG;
  *violations = 0;
  if (!h->frozen) return SMMO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* bad = &h->view.st->aux[2];
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(*bad), s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  const int nbm = 1 + 3 * h->view.num_classes;
  for (int k = 0; k < nbm; ++k) k_check_levels<<<h->num_sms * 2, 256, 0, s>>>(h->view, k);
  const uint32_t g = std::min<uint32_t>((h->view.num_blocks + 255) / 256, (uint32_t)h->num_sms * 8);
  k_check_blocks<<<std::max(g, 1u), 256, 0, s>>>(h->view);
  unsigned long long v = 0;
  e = cudaMemcpyAsync(&v, bad, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  *violations = (int64_t)v;
  return SMMO_OK;
}

int smmo_heap_last_device_error(smmo_heap* h, int* code, uint64_t* detail, void* stream) {
  if (!h || !code) return SMMO_E_INVALID_ARG;
  *code = 0;
  if (detail) *detail = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  if (!h->frozen) return SMMO_OK;
  struct { int err; int pad; unsigned long long detail; } hd;
  e = cudaMemcpy(&hd, h->view.st, sizeof(hd), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  *code = hd.err;
  if (detail) *detail = hd.detail;
  return SMMO_OK;
}

int smmo_heap_sync(smmo_heap* h, void* stream, uint64_t* detail) {
  if (!h) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  if (!h->frozen) return SMMO_OK;
  struct { int err; int pad; unsigned long long detail; } hd;
  e = cudaMemcpy(&hd, h->view.st, sizeof(hd), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return smmo::cuda_status(e);
  if (detail) *detail = hd.detail;
  if (hd.err) {
    e = cudaMemset(h->view.st, 0, 16);
    if (e != cudaSuccess) return smmo::cuda_status(e);
  }
  return hd.err;
}

}  // extern "C"
