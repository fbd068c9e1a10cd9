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

// Candidate scan in three kernels, one thread per block, 1024 blocks per
// CTA: (1) the candidate flag of every block (allocated to c and at most
// `limit` full, Sec. 6.3.1, from the allocation bitmaps), written as level 0
// of defrag[c] by warp ballots, and each CTA's candidate count; (2) the
// exclusive prefix over the CTAs' counts (r = the total); (3) every
// candidate written to its place in the sorted index list R.
__device__ __forceinline__ uint32_t block_exclusive_scan_1024(uint32_t v, uint32_t* sh, uint32_t* total) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (uint32_t o = 1; o < 1024; o <<= 1) {
    const uint32_t x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  const uint32_t incl = sh[threadIdx.x];
  *total = sh[1023];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(1024) k_cand_scan1(HeapView h, uint32_t c, uint32_t limit,
                                                     uint32_t* part) {
  __shared__ uint32_t wsum[32];
  const uint32_t blk = blockIdx.x * 1024 + threadIdx.x;  // grid covers every level-0 bit
  bool cand = false;
  if (blk < h.num_blocks) {
    const unsigned long long A = bm_level(h, bm_alloc(h, c), 0)[blk >> 6];
    if ((A >> (blk & 63)) & 1) cand = (uint32_t)__popcll(h.alloc_bm[blk] & h.cls[c].capmask) <= limit;
  }
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, cand);
  uint32_t* D32 = reinterpret_cast<uint32_t*>(bm_level(h, bm_defrag(h, c), 0));
  if ((threadIdx.x & 31) == 0) {
    D32[blk >> 5] = bal;  // little-endian halves of the 64-bit words
    wsum[threadIdx.x >> 5] = __popc(bal);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t t = __reduce_add_sync(0xFFFFFFFFu, wsum[threadIdx.x]);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_cand_scan2(uint32_t* part, uint32_t nparts,
                                                     unsigned long long* r) {
  __shared__ uint32_t sh[1024];
  uint32_t run = 0;
  for (uint32_t base = 0; base < nparts; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nparts ? part[i] : 0;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan_1024(v, sh, &tot);
    if (i < nparts) part[i] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) *r = run;
}

__global__ void __launch_bounds__(1024) k_cand_scan3(HeapView h, uint32_t c, const uint32_t* part,
                                                     uint32_t* R) {
  __shared__ uint32_t wsum[32];
  const uint32_t blk = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t bal = reinterpret_cast<const uint32_t*>(bm_level(h, bm_defrag(h, c), 0))[blk >> 5];
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = wsum[lane];
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= (uint32_t)o) incl += x;
    }
    wsum[lane] = incl - v;
  }
  __syncthreads();
  if ((bal >> lane) & 1) R[part[blockIdx.x] + wsum[warp] + __popc(bal & ((1u << lane) - 1))] = blk;
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
  // one atomic per warp: a counter hit by every thread serialises in L2
  cnt = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(moved, cnt);
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

// Pointer rewrite over the enumerated objects of a referring class (Alg.
// 6.6): a handle whose block is a source of this pass (a candidate with
// index below R[B]) is replaced by the forwarding handle in its source
// slot, so the forwarding slot is read only for real sources (Sec. 6.3.5).
// Like a do-all, one thread per slot of each enumerated block; each warp
// takes four units (32 slots each) at a time so that their column loads,
// bitmap tests and forwarding loads are in flight together.
struct RewriteArgs {
  const uint32_t* R;  // sorted candidates of this pass
  uint32_t B;         // number of sources
  const unsigned long long* defrag_l0;
  uint32_t ncols;
  uint32_t col_off[8];  // HANDLE columns of the referring class
  unsigned long long* rewritten;
};

__global__ void __launch_bounds__(256) k_rewrite(HeapView h, uint32_t u_cls, RewriteArgs a) {
  const uint32_t n = __ldcg(&h.st->rcount);
  const uint32_t cap = h.cls[u_cls].cap;
  const uint32_t halves = cap > 32 ? 2u : 1u, units = n * halves;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t first_target = a.R[a.B];
  uint32_t cnt = 0;
  for (uint32_t u0 = warp * 4; u0 < units; u0 += nwarps * 4) {
    uint32_t hd[4];
    bool live[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t u = u0 + k;
      live[k] = false;
      hd[k] = 0;
      if (u < units) {
        const REntry e = h.R[halves == 2 ? (u >> 1) : u];
        const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + lane;
        live[k] = (e.bits >> slot) & 1;
        hd[k] = (e.block << 6) | slot;
      }
    }
#pragma unroll
    for (uint32_t col = 0; col < 8; ++col) {  // constant indices into the parameter block
      if (col >= a.ncols) break;
      const uint32_t off = a.col_off[col];
      uint32_t v[4], nv[4];
      bool fwd[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = live[k] ? *field_ptr<uint32_t>(h, off, hd[k]) : kNull;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t b = v[k] >> 6;
        fwd[k] = v[k] != kNull && b < first_target && ((__ldg(a.defrag_l0 + (b >> 6)) >> (b & 63)) & 1);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        nv[k] = fwd[k] ? reinterpret_cast<const uint32_t*>(block_data(h, v[k] >> 6))[v[k] & 63] : 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (fwd[k]) { *field_ptr<uint32_t>(h, off, hd[k]) = nv[k]; ++cnt; }
    }
  }
  // one atomic per warp: a counter hit by every thread serialises in L2
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if (lane == 0 && cnt) atomicAdd(a.rewritten, (unsigned long long)cnt);
}

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
  const uint32_t nchunks = (nw * 64 + 1023) / 1024;  // CTAs of the scan, 1024 blocks each
  // the scan's per-CTA counts live in the enumeration scratch, which no
  // kernel of the scan's own pass uses before the rewrite re-enumerates
  uint32_t* part = reinterpret_cast<uint32_t*>(h->view.R);
  const uint32_t g = std::max(1u, std::min((nw + 255) / 256, (uint32_t)h->num_sms * 4));
  // referring (class, HANDLE columns) pairs: columns whose ref_class is c or
  // an ancestor of c, or unknown (-1)
  std::vector<std::pair<int, std::vector<uint32_t>>> refs;
  for (int u = 0; u < (int)h->classes.size(); ++u) {
    if (h->classes[u].abstract) continue;
    std::vector<uint32_t> offs;
    int col = 0;
    for (auto& f : h->classes[u].fields) {
      for (int k = 0; k < f.count; ++k, ++col)
        if (f.elem_type == SMMO_HANDLE && (f.ref_class < 0 || is_ancestor_or_self(h, f.ref_class, c)))
          offs.push_back(h->classes[u].layout.col_off[col]);
    }
    for (size_t k = 0; k < offs.size(); k += 8)
      refs.push_back({u, std::vector<uint32_t>(offs.begin() + k, offs.begin() + std::min(offs.size(), k + 8))});
  }
  cudaError_t e = cudaMemsetAsync(aux + 4, 0, 2 * sizeof(unsigned long long), s);
  // phase timing: per pass, events at the pass start, after the scan, after
  // copy and forwarding, after the state update and after the rewrite
  std::vector<cudaEvent_t> ev;
  auto mark = [&]() {
    cudaEvent_t x = nullptr;
    if (cudaEventCreate(&x) == cudaSuccess) { cudaEventRecord(x, s); ev.push_back(x); }
    else ev.push_back(nullptr);
  };
  std::vector<int> full_pass;  // 1 if the pass recorded all five events
  int status = SMMO_OK;
  for (int pass = 0; pass < 1000 && e == cudaSuccess; ++pass) {
    mark();
    k_cand_scan1<<<nchunks, 1024, 0, s>>>(h->view, c, limit, part);
    k_cand_scan2<<<1, 1024, 0, s>>>(part, nchunks, aux + 3);
    k_cand_scan3<<<nchunks, 1024, 0, s>>>(h->view, c, part, R);
    mark();
    unsigned long long r = 0;
    e = cudaMemcpyAsync(&r, aux + 3, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    st.candidates_left = (int64_t)r;
    const uint64_t B = r / (uint64_t)(n + 1);
    if ((int64_t)r <= k1 || B == 0) { full_pass.push_back(0); break; }
    const unsigned gm = (unsigned)std::min<uint64_t>((B * 64 + 255) / 256, 65535);
    k_move_objects<<<gm, 256, 0, s>>>(h->view, c, R, (uint32_t)B, (uint32_t)n);
    k_place_forwarding<<<gm, 256, 0, s>>>(h->view, c, R, (uint32_t)B, (uint32_t)n, aux + 4);
    mark();
    k_update_states<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>((B + 255) / 256, 4096)), 256, 0, s>>>(
        h->view, c, R, (uint32_t)B, (uint32_t)n);
    mark();
    for (auto& rc : refs) {
      RewriteArgs ra{};
      ra.R = R;
      ra.B = (uint32_t)B;
      ra.defrag_l0 = D0;
      ra.ncols = (uint32_t)rc.second.size();
      for (uint32_t k = 0; k < ra.ncols; ++k) ra.col_off[k] = rc.second[k];
      ra.rewritten = aux + 5;
      status = enumerate(h, rc.first, s);
      if (status) break;
      k_rewrite<<<h->num_sms * 4, 256, 0, s>>>(h->view, (uint32_t)rc.first, ra);
    }
    mark();
    full_pass.push_back(1);
    if (status) break;
    e = cudaGetLastError();
    st.passes += 1;
    st.blocks_freed += (int64_t)B;
  }
  // the pass used defrag[c] level 0 as scratch: restore the candidate state
  // that new and delete maintain
  if (e == cudaSuccess && !status) {
    k_rebuild_defrag_l0<<<g, 256, 0, s>>>(h->view, c);
    for (uint32_t l = 1; l < h->view.nlevels; ++l)
      k_rebuild_level<<<std::max(1u, std::min((h->view.level_words[l] + 255) / 256, 1024u)), 256, 0, s>>>(
          h->view, bm_defrag(h->view, c), l);
    unsigned long long mv[2] = {0, 0};
    e = cudaMemcpyAsync(mv, aux + 4, sizeof(mv), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st.objects_moved = (int64_t)mv[0];
    st.pointers_rewritten = (int64_t)mv[1];
  }
  // phase times from the events (all complete after the synchronisation)
  auto el = [&](size_t i, size_t j) -> double {
    float ms = 0.0f;
    if (j >= ev.size() || !ev[i] || !ev[j]) return 0.0;
    return cudaEventElapsedTime(&ms, ev[i], ev[j]) == cudaSuccess ? (double)ms : 0.0;
  };
  size_t k = 0;
  for (int f : full_pass) {
    st.scan_ms += el(k, k + 1);
    if (f) {
      st.copy_ms += el(k + 1, k + 2);
      st.state_ms += el(k + 2, k + 3);
      st.rewrite_ms += el(k + 3, k + 4);
      k += 5;
    } else {
      k += 2;
    }
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (out) *out = st;
  if (status) return status;
  return cuda_status(e);
}
