// compact.cu -- in-place parallel defragmentation of one class (CompactGpu,
// thesis Ch. 6).  A pass (Sec. 6.3.2):
//   1. candidates: allocated blocks of the class at most n/(n+1) full
//      (Sec. 6.3.1; computed here from the allocation bitmaps, the
//      alternative the thesis mentions, into the level-0 defrag bitmap) and
//      their sorted index list R (order matters, Sec. 6.3.3);
//   2. with B = floor(r/(n+1)), R[0..B-1] are sources and source s moves
//      its objects into targets R[s + i B], i = 1..n (Sec. 6.3.3);
//   3. move_objects: 64 threads per source, thread l copies the l-th object
//      of the source into the l-th free slot across its targets (Alg. 6.4);
//   4. place_forwarding_ptrs: a second kernel writes the new handle into the
//      source slot (Alg. 6.5; separate so no copy reads an overwritten slot);
//   5. block states: targets get their first m free slots marked, sources
//      become free (Sec. 6.3.6);
//   6. rewrite every HANDLE column that can refer to the class: a handle is
//      forwarded iff its block is a candidate with index < R[B] (Alg. 6.6),
//      so the forwarding slot is read only for real sources (Sec. 6.3.5).
//      The rewrite runs after the state update so that a class referring to
//      itself is rewritten in the moved copies, never in the dead sources.
// Passes repeat until at most k1 candidates remain (Sec. 6.3.7).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "heap_internal.h"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

// Candidate bitmap (level 0 of defrag[c]) of the allocated blocks of c.
__global__ void k_candidates(HeapView h, uint32_t c, uint32_t limit) {
  const unsigned long long* A = bm_level(h, bm_alloc(h, c), 0);
  unsigned long long* D = bm_level(h, bm_defrag(h, c), 0);
  const unsigned long long capmask = h.cls[c].capmask;
  const uint32_t nw = h.level_words[0];
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    unsigned long long a = A[w], d = 0;
    while (a) {
      const int b = __ffsll((long long)a) - 1;
      a &= a - 1;
      const uint32_t fill = __popcll(h.alloc_bm[w * 64 + b] & capmask);
      if (fill <= limit) d |= 1ull << b;
    }
    D[w] = d;
  }
}

// Sorted list of the set bits of a level-0 bitmap (single CTA, chunked
// prefix sum over containers).  count -> *n.
__global__ void __launch_bounds__(1024) k_sorted_list(const unsigned long long* L0, uint32_t nw,
                                                      uint32_t* out, unsigned long long* n) {
  __shared__ uint32_t psum[1024];
  __shared__ uint32_t running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nw; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const unsigned long long w = i < nw ? L0[i] : 0ull;
    psum[threadIdx.x] = __popcll(w);
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {
      const uint32_t v = threadIdx.x >= o ? psum[threadIdx.x - o] : 0;
      __syncthreads();
      psum[threadIdx.x] += v;
      __syncthreads();
    }
    uint32_t pos = running + psum[threadIdx.x] - __popcll(w);
    unsigned long long ww = w;
    while (ww) {
      const int b = __ffsll((long long)ww) - 1;
      ww &= ww - 1;
      out[pos++] = i * 64 + b;
    }
    __syncthreads();
    if (threadIdx.x == 1023) running += psum[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n = running;
}

// Target slot of the l-th object of source s (shared by the copy and the
// forwarding kernels): walks the n targets' free slots in order (Alg. 6.4).
__device__ __forceinline__ bool target_slot(const HeapView& h, const uint32_t* R, uint32_t B,
                                            uint32_t n, uint32_t s, uint32_t l, uint32_t* t_bid,
                                            uint32_t* t_oid) {
  uint32_t t_loc = l;
  for (uint32_t i = 1; i <= n; ++i) {
    const uint32_t tb = R[s + i * B];
    const unsigned long long tfree = ~h.alloc_bm[tb];
    const uint32_t nf = __popcll(tfree);
    if (t_loc < nf) {
      *t_bid = tb;
      *t_oid = (uint32_t)nth_set_bit(tfree, (int)t_loc);
      return true;
    }
    t_loc -= nf;
  }
  return false;
}

__global__ void k_move_objects(HeapView h, uint32_t c, const uint32_t* R, uint32_t B, uint32_t n) {
  const ClassLayout& L = h.cls[c];
  const uint64_t total = (uint64_t)B * 64;
  for (uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; tid < total;
       tid += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(tid / 64), l = (uint32_t)(tid % 64);
    const uint32_t sb = R[s];
    const unsigned long long sbits = h.alloc_bm[sb] & L.capmask;
    if (l >= (uint32_t)__popcll(sbits)) continue;
    uint32_t tb, to;
    if (!target_slot(h, R, B, n, s, l, &tb, &to)) { set_error(h, SMMO_E_CONTENTION, sb); continue; }
    const uint32_t so = (uint32_t)nth_set_bit(sbits, (int)l);
    const uint8_t* src = block_data(h, sb);
    uint8_t* dst = block_data(h, tb);
    for (uint32_t k = 0; k < L.ncols; ++k) {
      const uint32_t sz = L.col_size[k];
      const uint8_t* p = src + L.col_off[k] + (size_t)so * sz;
      uint8_t* q = dst + L.col_off[k] + (size_t)to * sz;
      switch (sz) {
        case 1: *q = *p; break;
        case 2: *(uint16_t*)q = *(const uint16_t*)p; break;
        case 4: *(uint32_t*)q = *(const uint32_t*)p; break;
        default: *(uint64_t*)q = *(const uint64_t*)p; break;
      }
    }
  }
}

// Forwarding handle of source slot so: a u32 at offset 4*so of the dead
// source block's data segment.
__global__ void k_place_forwarding(HeapView h, uint32_t c, const uint32_t* R, uint32_t B, uint32_t n,
                                   unsigned long long* moved) {
  const ClassLayout& L = h.cls[c];
  const uint64_t total = (uint64_t)B * 64;
  unsigned long long cnt = 0;
  for (uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; tid < total;
       tid += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(tid / 64), l = (uint32_t)(tid % 64);
    const uint32_t sb = R[s];
    const unsigned long long sbits = h.alloc_bm[sb] & L.capmask;
    if (l >= (uint32_t)__popcll(sbits)) continue;
    uint32_t tb, to;
    if (!target_slot(h, R, B, n, s, l, &tb, &to)) continue;
    const uint32_t so = (uint32_t)nth_set_bit(sbits, (int)l);
    reinterpret_cast<uint32_t*>(block_data(h, sb))[so] = (tb << 6) | to;
    ++cnt;
  }
  if (cnt) atomicAdd(moved, cnt);
}

// Block states after a pass: each target gets its first m free slots marked
// (m = objects it received), a target that filled up leaves the active
// bitmap; each source block is invalidated and becomes free.
__global__ void k_update_states(HeapView h, uint32_t c, const uint32_t* R, uint32_t B, uint32_t n) {
  const ClassLayout& L = h.cls[c];
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < B; s += gridDim.x * blockDim.x) {
    const uint32_t sb = R[s];
    uint32_t cnt = __popcll(h.alloc_bm[sb] & L.capmask);
    for (uint32_t i = 1; i <= n && cnt; ++i) {
      const uint32_t tb = R[s + i * B];
      const unsigned long long bm = h.alloc_bm[tb];
      unsigned long long tfree = ~bm, add = 0;
      while (cnt && tfree) {
        const unsigned long long low = tfree & (0ull - tfree);
        add |= low;
        tfree ^= low;
        --cnt;
      }
      h.alloc_bm[tb] = bm | add;
      if ((bm | add) == kAll) bm_clear(h, bm_active(h, c), tb);
    }
    h.alloc_bm[sb] = kAll;  // invalidated
    bm_clear(h, bm_active(h, c), sb);
    bm_clear(h, bm_alloc(h, c), sb);
    bm_set(h, bm_free(), sb);
  }
}

// Pointer rewrite over the objects of a referring class (run as a do-all,
// one thread per object): every listed HANDLE column whose value lies in a
// source block is replaced by the forwarding handle (Alg. 6.6).
struct RewriteArgs {
  const uint32_t* R;
  const unsigned long long* defrag_l0;
  uint32_t first_target;  // R[B]
  uint32_t ncols;
  uint32_t col[8];
  unsigned long long* rewritten;
};

struct Rewrite {
  using Args = RewriteArgs;
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint32_t cnt = 0;
    for (uint32_t k = 0; k < a.ncols; ++k) {
      uint32_t* p = field_ptr<uint32_t>(h, __ldg(&h.cls[c].col_off[a.col[k]]), self);
      const uint32_t v = *p;
      if (v == kNull) continue;
      const uint32_t b = v >> 6;
      if (b < a.first_target && ((a.defrag_l0[b >> 6] >> (b & 63)) & 1)) {
        *p = reinterpret_cast<const uint32_t*>(block_data(h, b))[v & 63];
        ++cnt;
      }
    }
    if (cnt) atomicAdd(a.rewritten, (unsigned long long)cnt);
  }
};

// Rebuilds the candidate bitmap defrag[c] that new and delete maintain
// (fill <= dlimit) after a compaction used its level 0 as scratch: level 0
// from the allocation bitmaps, every higher level as the OR of its
// container below.
__global__ void k_rebuild_defrag_l0(HeapView h, uint32_t c) {
  const unsigned long long* A = bm_level(h, bm_alloc(h, c), 0);
  unsigned long long* D = bm_level(h, bm_defrag(h, c), 0);
  const unsigned long long capmask = h.cls[c].capmask;
  const uint32_t lim = h.cls[c].dlimit;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < h.level_words[0]; w += gridDim.x * blockDim.x) {
    unsigned long long a = A[w], d = 0;
    while (a) {
      const int b = __ffsll((long long)a) - 1;
      a &= a - 1;
      if ((uint32_t)__popcll(h.alloc_bm[w * 64 + b] & capmask) <= lim) d |= 1ull << b;
    }
    D[w] = d;
  }
}

__global__ void k_rebuild_level(HeapView h, int k, uint32_t l) {
  const unsigned long long* lo = bm_level(h, k, l - 1);
  unsigned long long* hi = bm_level(h, k, l);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < h.level_words[l]; i += gridDim.x * blockDim.x) {
    unsigned long long v = 0;
    for (uint32_t j = 0; j < 64; ++j) {
      const uint64_t q = (uint64_t)i * 64 + j;
      if (q < h.level_words[l - 1] && lo[q]) v |= 1ull << j;
    }
    hi[i] = v;
  }
}

bool is_ancestor_or_self(const smmo_heap* h, int anc, int c) {
  for (int k = c; k >= 0; k = h->classes[k].parent)
    if (k == anc) return true;
  return false;
}

}  // namespace

extern "C" int smmo_compact(smmo_heap* h, int c, int n, int64_t k1, smmo_compact_stats* out,
                            void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size() || n < 1 || n > 63 || k1 < 0) return SMMO_E_INVALID_ARG;
  if (h->classes[c].abstract) return SMMO_E_INVALID_ARG;
  smmo_compact_stats st{};
  if (!h->frozen) { if (out) *out = st; return SMMO_OK; }
  if (h->view.block_bytes < 256) return SMMO_E_UNSUPPORTED;  // forwarding slots need 64 x 4 bytes
  cudaStream_t s = (cudaStream_t)stream;
  const ClassLayout& L = h->classes[c].layout;
  const uint32_t limit = (uint32_t)((uint64_t)L.cap * n / (n + 1));
  uint32_t* R = h->d_scratch;
  unsigned long long* aux = h->view.st->aux;  // [3] r, [4] moved, [5] rewritten
  unsigned long long* D0 = bm_level_host(h, bm_defrag(h->view, c));  // level 0 only
  const uint32_t nw = h->view.level_words[0];
  const uint32_t g = std::max(1u, std::min((nw + 255) / 256, (uint32_t)h->num_sms * 4));
  // referring (class, HANDLE columns) pairs: columns whose ref_class is c or
  // an ancestor of c, or unknown (-1)
  std::vector<std::pair<int, std::vector<int>>> refs;
  for (int u = 0; u < (int)h->classes.size(); ++u) {
    if (h->classes[u].abstract) continue;
    std::vector<int> cols;
    int col = 0;
    for (auto& f : h->classes[u].fields) {
      for (int k = 0; k < f.count; ++k, ++col)
        if (f.elem_type == SMMO_HANDLE && (f.ref_class < 0 || is_ancestor_or_self(h, f.ref_class, c)))
          cols.push_back(col);
    }
    if (!cols.empty()) refs.push_back({u, cols});
  }
  cudaError_t e = cudaSuccess;
  for (int pass = 0; pass < 1000; ++pass) {
    k_candidates<<<g, 256, 0, s>>>(h->view, c, limit);
    k_sorted_list<<<1, 1024, 0, s>>>(D0, nw, R, aux + 3);
    unsigned long long r = 0;
    e = cudaMemcpyAsync(&r, aux + 3, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    st.candidates_left = (int64_t)r;
    const uint64_t B = r / (uint64_t)(n + 1);
    if ((int64_t)r <= k1 || B == 0) break;
    uint32_t first_target = 0;
    e = cudaMemcpyAsync(&first_target, R + B, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(aux + 4, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) break;
    const unsigned gm = (unsigned)std::min<uint64_t>((B * 64 + 255) / 256, 65535);
    k_move_objects<<<gm, 256, 0, s>>>(h->view, c, R, (uint32_t)B, (uint32_t)n);
    k_place_forwarding<<<gm, 256, 0, s>>>(h->view, c, R, (uint32_t)B, (uint32_t)n, aux + 4);
    k_update_states<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>((B + 255) / 256, 4096)), 256, 0, s>>>(
        h->view, c, R, (uint32_t)B, (uint32_t)n);
    e = cudaStreamSynchronize(s);  // first_target is needed on the host
    if (e != cudaSuccess) break;
    for (auto& rc : refs) {
      RewriteArgs ra{};
      ra.R = R;
      ra.defrag_l0 = D0;
      ra.first_target = first_target;
      ra.ncols = (uint32_t)std::min<size_t>(rc.second.size(), 8);
      for (uint32_t k = 0; k < ra.ncols; ++k) ra.col[k] = (uint32_t)rc.second[k];
      ra.rewritten = aux + 5;
      int r2 = enumerate(h, rc.first, s);
      if (!r2) r2 = launch_do_all<Rewrite>(h, rc.first, &ra, s);
      if (r2) return r2;
    }
    unsigned long long mv[2] = {0, 0};
    e = cudaMemcpyAsync(mv, aux + 4, sizeof(mv), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    st.passes += 1;
    st.blocks_freed += (int64_t)B;
    st.objects_moved += (int64_t)mv[0];
    st.pointers_rewritten += (int64_t)mv[1];
  }
  // the pass used defrag[c] level 0 as scratch: restore the candidate state
  // that new and delete maintain
  k_rebuild_defrag_l0<<<g, 256, 0, s>>>(h->view, c);
  for (uint32_t l = 1; l < h->view.nlevels; ++l)
    k_rebuild_level<<<std::max(1u, std::min((h->view.level_words[l] + 255) / 256, 1024u)), 256, 0, s>>>(
        h->view, bm_defrag(h->view, c), l);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (out) *out = st;
  return cuda_status(e);
}
