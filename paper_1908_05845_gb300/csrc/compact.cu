// compact.cu -- in-place parallel defragmentation of one class (CompactGpu,
// thesis Ch. 6).  A pass (Sec. 6.3.2):
//   1. candidates: allocated blocks of the class at most n/(n+1) full
//      (Sec. 6.3.1; computed here from the allocation bitmaps, the
//      alternative the thesis mentions, into the level-0 defrag bitmap) and
//      their sorted index list R (order matters, Sec. 6.3.3);
//   2. with B = floor(r/(n+1)), R[0..B-1] are sources and source s moves
//      its objects into targets R[s + i B], i = 1..n (Sec. 6.3.3);
//   3. relocate: 64 threads per source, thread l copies the l-th object of
//      the source into the l-th free slot across its targets (Alg. 6.4),
//      then, after a CTA barrier (a source's 64 threads share a CTA, so no
//      copy still reads the slot), writes the new handle into the source
//      slot as its forwarding pointer (Alg. 6.5);
//   4. block states: targets get their first m free slots marked, sources
//      become free and are marked in a "moved from" bitmap (Sec. 6.3.6).
// Passes repeat until at most k1 candidates remain (Sec. 6.3.7).  Then
//   5. one rewrite of every HANDLE column that can refer to the class: a
//      handle into a block that was a source in some pass is replaced by
//      its forwarding pointer, repeatedly while the result lies in a later
//      source (Alg. 6.6 applied to the chain of passes).
// The thesis rewrites after every pass (Sec. 6.3.5); forwarding slots of a
// freed source are never overwritten during the compaction (a free block is
// no candidate), so one rewrite that follows the chain gives the same
// handles and reads every HANDLE column once instead of once per pass.
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

// Pass control in device memory, so that passes run without a host round
// trip: ctl[0] done flag, ctl[1] passes run, ctl[2] sources freed, ctl[3]
// r of the latest scan.  Every kernel of a pass returns at once when done.
enum { CTL_DONE = 0, CTL_PASSES = 1, CTL_FREED = 2, CTL_R = 3 };

// (part and ctl may be null: the restore of the maintained candidate bitmap
// after the compaction uses this kernel with limit = dlimit.)
__global__ void __launch_bounds__(1024) k_cand_scan1(HeapView h, uint32_t c, uint32_t limit,
                                                     uint32_t* part, const unsigned long long* ctl) {
  __shared__ uint32_t wsum[32];
  if (ctl && ctl[CTL_DONE]) return;
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
  if (!part) return;
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t t = __reduce_add_sync(0xFFFFFFFFu, wsum[threadIdx.x]);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// (2) also decides the pass: r <= k1 or fewer than n + 1 candidates ends
// the compaction (Sec. 6.3.7).
__global__ void __launch_bounds__(1024) k_cand_scan2(uint32_t* part, uint32_t nparts, uint32_t n,
                                                     unsigned long long k1, unsigned long long* ctl) {
  __shared__ uint32_t sh[1024];
  if (ctl[CTL_DONE]) return;
  uint32_t run = 0;
  for (uint32_t base = 0; base < nparts; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nparts ? part[i] : 0;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan_1024(v, sh, &tot);
    if (i < nparts) part[i] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) {
    const unsigned long long B = run / (n + 1);
    ctl[CTL_R] = run;
    if (run <= k1 || B == 0) {
      ctl[CTL_DONE] = 1;
    } else {
      ctl[CTL_PASSES] += 1;
      ctl[CTL_FREED] += B;
    }
  }
}

__global__ void __launch_bounds__(1024) k_cand_scan3(HeapView h, uint32_t c, const uint32_t* part,
                                                     uint32_t* R, const unsigned long long* ctl) {
  __shared__ uint32_t wsum[32];
  if (ctl[CTL_DONE]) return;
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

// Target slot of the l-th object of source s: walks the n targets' free
// slots in order (Alg. 6.4).
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
      *t_oid = (uint32_t)nth_set_bit64(tfree, t_loc);
      return true;
    }
    t_loc -= nf;
  }
  return false;
}

// Copy and forwarding pointers of one pass.  The loop runs over CTA-sized
// chunks of (source, l) pairs so that every thread of a CTA meets the
// barrier equally often; 256 threads hold four whole sources.
__global__ void __launch_bounds__(256) k_relocate(HeapView h, uint32_t c, const uint32_t* R, uint32_t n,
                                                  const unsigned long long* ctl, unsigned long long* moved) {
  if (ctl[CTL_DONE]) return;
  const uint32_t B = (uint32_t)(ctl[CTL_R] / (n + 1));
  const ClassLayout& L = h.cls[c];
  const uint64_t total = (uint64_t)B * 64;
  uint32_t cnt = 0;
  for (uint64_t base = (uint64_t)blockIdx.x * 256; base < total; base += (uint64_t)gridDim.x * 256) {
    const uint64_t tid = base + threadIdx.x;
    bool go = false;
    uint32_t sb = 0, so = 0, tb = 0, to = 0;
    if (tid < total) {
      const uint32_t s = (uint32_t)(tid >> 6), l = (uint32_t)(tid & 63);
      sb = R[s];
      const unsigned long long sbits = h.alloc_bm[sb] & L.capmask;
      if (l < (uint32_t)__popcll(sbits)) {
        go = target_slot(h, R, B, n, s, l, &tb, &to);
        if (!go) set_error(h, SMMO_E_CONTENTION, sb);
        so = (uint32_t)nth_set_bit64(sbits, l);
      }
    }
    if (go) {
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
    __syncthreads();  // every copy out of these sources is done
    if (go) {
      reinterpret_cast<uint32_t*>(block_data(h, sb))[so] = (tb << 6) | to;
      ++cnt;
    }
    // the next chunk's sources are other blocks: no second barrier needed
  }
  // one atomic per warp: a counter hit by every thread serialises in L2
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(moved, (unsigned long long)cnt);
}

// Block states after a pass: each target gets its first m free slots marked
// (m = objects it received), a target that filled up leaves the active
// bitmap; each source block is invalidated and becomes free.
__global__ void k_update_states(HeapView h, uint32_t c, const uint32_t* R, uint32_t n,
                                const unsigned long long* ctl, unsigned long long* moved_from) {
  if (ctl[CTL_DONE]) return;
  const uint32_t B = (uint32_t)(ctl[CTL_R] / (n + 1));
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
    atomicOr(moved_from + (sb >> 6), 1ull << (sb & 63));
    h.alloc_bm[sb] = kAll;  // invalidated
    bm_clear(h, bm_active(h, c), sb);
    bm_clear(h, bm_alloc(h, c), sb);
    bm_set(h, bm_free(), sb);
  }
}

// Pointer rewrite over the enumerated objects of a referring class, once
// after all passes (Alg. 6.6 along the chain of passes): a handle whose
// block was a source is replaced by the forwarding pointer in its source
// slot, again while the result lies in a block that was a source of a later
// pass (at most one hop per pass), so the forwarding slot is read only for
// real sources (Sec. 6.3.5).  Like a do-all, one thread per slot of each
// enumerated block; each warp takes four units (32 slots each) at a time so
// that their column loads, bitmap tests and forwarding loads are in flight
// together.
struct RewriteArgs {
  const unsigned long long* moved_from;  // level-0 bitmap of the passes' sources
  uint32_t max_hops;                     // passes run
  uint32_t ncols;
  uint32_t col_off[8];  // HANDLE columns of the referring class
  unsigned long long* rewritten;
};

__device__ __forceinline__ bool was_source(const HeapView& h, const unsigned long long* mf, uint32_t v) {
  const uint32_t b = v >> 6;
  return v != kNull && b < h.num_blocks && ((__ldg(mf + (b >> 6)) >> (b & 63)) & 1);
}

__global__ void __launch_bounds__(256) k_rewrite(HeapView h, uint32_t u_cls, RewriteArgs a) {
  const uint32_t n = __ldcg(h.rcnt);
  const uint32_t cap = h.cls[u_cls].cap;
  const uint32_t halves = cap > 32 ? 2u : 1u, units = n * halves;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
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
      uint32_t v[4];
      bool fwd[4], moved[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = live[k] ? *field_ptr<uint32_t>(h, off, hd[k]) : kNull;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        fwd[k] = was_source(h, a.moved_from, v[k]);
        moved[k] = fwd[k];
      }
      for (uint32_t hop = 0; hop < a.max_hops && (fwd[0] | fwd[1] | fwd[2] | fwd[3]); ++hop) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (fwd[k]) v[k] = reinterpret_cast<const uint32_t*>(block_data(h, v[k] >> 6))[v[k] & 63];
#pragma unroll
        for (int k = 0; k < 4; ++k) fwd[k] = fwd[k] && was_source(h, a.moved_from, v[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (moved[k]) { *field_ptr<uint32_t>(h, off, hd[k]) = v[k]; ++cnt; }
    }
  }
  // one atomic per warp: a counter hit by every thread serialises in L2
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if (lane == 0 && cnt) atomicAdd(a.rewritten, (unsigned long long)cnt);
}

// Level l of a hierarchical bitmap as the OR of the containers below (the
// restore of defrag[c] after a compaction used its level 0 as scratch).
__global__ void k_rebuild_level(HeapView h, int k, uint32_t l) {
  unsigned long long* hi = bm_level(h, k, l);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < h.level_words[l]; i += gridDim.x * blockDim.x) {
    unsigned long long v = 0;
    for (uint32_t j = 0; j < 64; ++j) {  // bit q of level l: container q of level l - 1
      const uint32_t q = i * 64 + j;
      if (q < h.level_bits[l] && bm_container(h, k, l - 1, q)) v |= 1ull << j;
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
  const uint32_t nw = h->view.level_words[0];
  const uint32_t nchunks = (nw * 64 + 1023) / 1024;  // CTAs of the scan, 1024 blocks each
  // the scan's per-CTA counts live in the enumeration scratch, which is
  // unused during the passes (the rewrite enumerates after the last pass)
  uint32_t* part = reinterpret_cast<uint32_t*>(h->view.R);
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
  cudaError_t e = cudaMemsetAsync(aux, 0, 6 * sizeof(unsigned long long), s);
  unsigned long long* moved_from = h->d_moved;  // sources of all passes, one bit per block
  if (e == cudaSuccess) e = cudaMemsetAsync(moved_from, 0, (size_t)nw * 8, s);
  // passes are queued in groups of kGroup; the host looks at the control
  // block once per group (passes after the last real one return at once)
  const int kGroup = 4;
  const unsigned grel = (unsigned)h->num_sms * 8, gupd = (unsigned)h->num_sms * 4;
  int status = SMMO_OK;
  unsigned long long ctl[4] = {0, 0, 0, 0};
  // phase timing: per pass, events at the pass start, after the scan, after
  // copy and forwarding and after the state update; one set of events for a
  // group, read after the group's synchronisation and reused
  cudaEvent_t ev[4 * kGroup] = {};
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  auto el = [&](int i, int j) -> double {
    float ms = 0.0f;
    return cudaEventElapsedTime(&ms, ev[i], ev[j]) == cudaSuccess ? (double)ms : 0.0;
  };
  for (int queued = 0; queued < 1000 && e == cudaSuccess;) {
    for (int k = 0; k < kGroup; ++k, ++queued) {
      cudaEventRecord(ev[4 * k], s);
      k_cand_scan1<<<nchunks, 1024, 0, s>>>(h->view, c, limit, part, aux);
      k_cand_scan2<<<1, 1024, 0, s>>>(part, nchunks, (uint32_t)n, (unsigned long long)k1, aux);
      k_cand_scan3<<<nchunks, 1024, 0, s>>>(h->view, c, part, R, aux);
      cudaEventRecord(ev[4 * k + 1], s);
      k_relocate<<<grel, 256, 0, s>>>(h->view, c, R, (uint32_t)n, aux, aux + 4);
      cudaEventRecord(ev[4 * k + 2], s);
      k_update_states<<<gupd, 256, 0, s>>>(h->view, c, R, (uint32_t)n, aux, moved_from);
      cudaEventRecord(ev[4 * k + 3], s);
    }
    e = cudaMemcpyAsync(ctl, aux, sizeof(ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    for (int k = 0; k < kGroup; ++k) {
      st.scan_ms += el(4 * k, 4 * k + 1);
      st.copy_ms += el(4 * k + 1, 4 * k + 2);
      st.state_ms += el(4 * k + 2, 4 * k + 3);
    }
    if (ctl[0]) break;
  }
  st.passes = (int32_t)ctl[1];
  st.blocks_freed = (int64_t)ctl[2];
  st.candidates_left = (int64_t)ctl[3];
  // one rewrite along the chain of passes
  cudaEvent_t rw0 = nullptr, rw1 = nullptr;
  if (e == cudaSuccess && st.passes > 0) {
    cudaEventCreate(&rw0);
    cudaEventCreate(&rw1);
    cudaEventRecord(rw0, s);
    for (auto& rc : refs) {
      RewriteArgs ra{};
      ra.moved_from = moved_from;
      ra.max_hops = (uint32_t)st.passes;
      ra.ncols = (uint32_t)rc.second.size();
      for (uint32_t k = 0; k < ra.ncols; ++k) ra.col_off[k] = rc.second[k];
      ra.rewritten = aux + 5;
      status = enumerate(h, rc.first, s);
      if (status) break;
      k_rewrite<<<h->num_sms * 4, 256, 0, s>>>(h->view, (uint32_t)rc.first, ra);
    }
    cudaEventRecord(rw1, s);
    e = cudaGetLastError();
  }
  // the pass used defrag[c] level 0 as scratch: restore the candidate state
  // that new and delete maintain
  if (e == cudaSuccess && !status) {
    k_cand_scan1<<<nchunks, 1024, 0, s>>>(h->view, c, L.dlimit, nullptr, nullptr);
    for (uint32_t l = 1; l < h->view.nlevels; ++l)
      k_rebuild_level<<<std::max(1u, std::min((h->view.level_words[l] + 255) / 256, 1024u)), 256, 0, s>>>(
          h->view, bm_defrag(h->view, c), l);
    unsigned long long mv[2] = {0, 0};
    e = cudaMemcpyAsync(mv, aux + 4, sizeof(mv), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st.objects_moved = (int64_t)mv[0];
    st.pointers_rewritten = (int64_t)mv[1];
  }
  if (rw0 && rw1) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, rw0, rw1) == cudaSuccess) st.rewrite_ms = ms;
  }
  if (rw0) cudaEventDestroy(rw0);
  if (rw1) cudaEventDestroy(rw1);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (out) *out = st;
  if (status) return status;
  if (e == cudaSuccess) {
    // forwarding slots of this compaction stay readable until the next
    // allocation: remember where the allocation counters stand
    int64_t news = 0;
    const int cst = smmo_heap_counters(h, nullptr, &news, nullptr, stream);
    if (cst) return cst;
    h->compact_passes = (uint32_t)st.passes;
    h->compact_news = news;
    h->compact_bulks = h->bulk_calls;
  }
  return cuda_status(e);
}

namespace {
// Defragmentation candidates of class c for factor n: allocated blocks at
// most `limit` full (Sec. 6.3.1), one thread per block, warp-aggregated.
__global__ void __launch_bounds__(256) k_count_candidates(HeapView h, uint32_t c, uint32_t limit,
                                                          unsigned long long* out) {
  uint32_t cnt = 0;
  for (uint32_t blk = blockIdx.x * blockDim.x + threadIdx.x; blk < h.num_blocks; blk += gridDim.x * blockDim.x) {
    const unsigned long long A = bm_level(h, bm_alloc(h, c), 0)[blk >> 6];
    if ((A >> (blk & 63)) & 1) cnt += (uint32_t)__popcll(h.alloc_bm[blk] & h.cls[c].capmask) <= limit ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, (unsigned long long)cnt);
}
}  // namespace

extern "C" int smmo_defrag_candidates(smmo_heap* h, int c, int n, int64_t* count, void* stream) {
  if (!h || c < 0 || c >= (int)h->classes.size() || n < 1 || n > 63 || !count) return SMMO_E_INVALID_ARG;
  if (h->classes[c].abstract) return SMMO_E_INVALID_ARG;
  *count = 0;
  if (!h->frozen) return SMMO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const ClassLayout& L = h->classes[c].layout;
  const uint32_t limit = (uint32_t)((uint64_t)L.cap * n / (n + 1));
  unsigned long long* d = &h->view.st->aux[0];
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), s);
  if (e != cudaSuccess) return cuda_status(e);
  const uint32_t grid = std::max(1u, std::min((h->view.num_blocks + 255) / 256, (uint32_t)h->num_sms * 8));
  k_count_candidates<<<grid, 256, 0, s>>>(h->view, (uint32_t)c, limit, d);
  unsigned long long v = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *count = (int64_t)v;
  return SMMO_OK;
}

extern "C" int smmo_compact_if(smmo_heap* h, int c, int n, int64_t k1, int64_t k2_blocks, double k2_fraction,
                               smmo_compact_stats* out, int* ran, void* stream) {
  if (ran) *ran = 0;
  if (!h || k2_blocks < 0 || !(k2_fraction >= 0.0) || k2_fraction > 1.0) return SMMO_E_INVALID_ARG;
  int64_t cand = 0;
  int st = smmo_defrag_candidates(h, c, n, &cand, stream);
  if (st) return st;
  // k2 as a block count or a fraction of the heap's blocks, scaled by
  // n / (n + 1): a larger n makes more blocks candidates
  const double k2 = std::max((double)k2_blocks, k2_fraction * (double)h->view.num_blocks);
  if ((double)cand < k2 * n / (n + 1)) {
    if (out) {
      *out = smmo_compact_stats{};
      out->candidates_left = cand;
    }
    return SMMO_OK;
  }
  if (ran) *ran = 1;
  return smmo_compact(h, c, n, k1, out, stream);
}

namespace {
// Caller-held handles through the forwarding slots of the last compaction
// (the same chain the rewrite follows, at most one hop per pass).
__global__ void __launch_bounds__(256) k_remap(HeapView h, const unsigned long long* mf, uint32_t* hd, uint64_t n,
                                               uint32_t max_hops) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = hd[i];
    for (uint32_t hop = 0; hop < max_hops && was_source(h, mf, v); ++hop)
      v = reinterpret_cast<const uint32_t*>(block_data(h, v >> 6))[v & 63];
    hd[i] = v;
  }
}
}  // namespace

extern "C" int smmo_remap_handles(smmo_heap* h, uint32_t* handles, int64_t n, void* stream) {
  if (!h || n < 0 || (n > 0 && !handles)) return SMMO_E_INVALID_ARG;
  if (!h->frozen || h->compact_news < 0 || n == 0) return SMMO_OK;  // nothing was moved
  int64_t news = 0;
  int st = smmo_heap_counters(h, nullptr, &news, nullptr, stream);
  if (st) return st;
  if (news != h->compact_news || h->bulk_calls != h->compact_bulks) return SMMO_E_UNSUPPORTED;  // slots reused
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t grid = (uint32_t)std::min<int64_t>((n + 255) / 256, (int64_t)h->num_sms * 8);
  k_remap<<<grid, 256, 0, s>>>(h->view, h->d_moved, handles, (uint64_t)n, h->compact_passes);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}
