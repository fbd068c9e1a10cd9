// levels.cuh -- consecutive levels of a level-synchronous reducing do-all
// (the frontier BFS of Sec. 4.3 and the removal of Sec. 7.4) in one
// persistent cooperative launch.
//
// Level l is parallel_do_and_reduce(method, frontier = l) with the OR
// reducer over one saved snapshot; the levels are separated by a grid
// barrier instead of a kernel boundary, and the launch ends after the
// first level whose OR is 0 (every CTA reads the same flag after the
// barrier, so all leave together).  The result is that of one launch per
// level: a level starts after every write of the previous one is visible
// (fence, barrier, fence; the methods read the values that other CTAs
// write through L2).  The methods must not create or delete objects (the
// snapshot stays valid).  The grid is the number of CTAs that can be
// resident at once, which a cooperative launch guarantees (else it fails
// to launch); every barrier wait is bounded and records SMMO_E_TIMEOUT.
#pragma once
#include "heap_internal.h"
#include "smmo_core.cuh"

namespace smmo {

constexpr unsigned kLevelBarrierSpins = 1u << 23;  // x ~100 ns: about a second
constexpr int kLevelChunk = 4;                     // units tested at once per warp

constexpr int kLevelThreads = 1024;                // CTA size: one CTA of 32 warps per SM (fewest arrivals)
constexpr int kBarrierWords = 64;                  // arrive[0] counter, arrive[32] release word

// Barrier across the grid's CTAs: arrive[0] counts arrivals (zeroed before
// the launch); the CTA that completes the k-th barrier (its arrival makes
// the count k x gridDim.x) writes k to arrive[32], on which the others wait
// (the count and the word are in different cache lines, so the waiting
// reads do not slow the arrivals).
__device__ __forceinline__ bool grid_barrier(const HeapView& h, unsigned int* arrive, unsigned int k,
                                             unsigned spin_limit = kLevelBarrierSpins) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned int target = k * gridDim.x;
    if (atomicAdd(arrive, 1u) + 1 == target) {
      __threadfence();
      atomicExch(arrive + 32, k);
    }
    unsigned spins = 0;
    while (*(volatile unsigned int*)(arrive + 32) < k) {
      if (++spins > spin_limit) {
        ok = 0;
        set_error(h, SMMO_E_TIMEOUT, target);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Levels base .. base + K - 1 of M (M::Args has an int32 `frontier`;
// M::active(h, a, c, self) is the method's cheap test "in this level's
// frontier" (loads only), M::run the level step for such an object, which
// returns nonzero as the level's OR).  A warp tests kLevelChunk of its units at
// once (their loads are independent), then runs the method where the test
// passed; units are dealt to the warps round-robin (no allocation happens,
// so the locality of contiguous runs does not matter).  flags[k] (zeroed before the launch) receives the OR of level
// base + k.
template <class M, bool POLY>
__global__ void __launch_bounds__(kLevelThreads, 1) levels_kernel(HeapView h, uint32_t c, typename M::Args args, int32_t base,
                                                     int K, unsigned long long* flags, unsigned int* arrive) {
  __shared__ int any;
  const uint32_t n = __ldcg(h.rcnt);
  const uint32_t cap = POLY ? 64u : __ldg(&h.cls[c].cap);
  const uint32_t halves = cap > 32 ? 2u : 1u;
  const uint32_t units = n * halves;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t visited = 0;
  for (int k = 0; k < K; ++k) {
    args.frontier = base + k;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    bool mine = false;
    // units wid, wid + nwarps, ...: a frontier is often a contiguous run of
    // blocks, and striding spreads it over the warps
    for (uint32_t u0 = wid; u0 < units; u0 += kLevelChunk * nwarps) {
      uint32_t hd[kLevelChunk], cl[kLevelChunk];
      bool act[kLevelChunk];
#pragma unroll
      for (int j = 0; j < kLevelChunk; ++j) {
        const uint32_t u = u0 + j * nwarps;
        act[j] = false;
        hd[j] = kNull;
        cl[j] = c;
        if (u < units) {
          const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + lane;
          // the entries are fixed during the launch: read-only cache
          const uint4 raw = __ldg(reinterpret_cast<const uint4*>(h.R + (halves == 2 ? (u >> 1) : u)));
          REntry e;
          e.block = raw.x;
          e.cls = raw.y;
          e.bits = (unsigned long long)raw.z | ((unsigned long long)raw.w << 32);
          if (lane == 0) visited += __popcll(halves == 2 ? (e.bits >> ((u & 1) * 32)) & 0xFFFFFFFFull : e.bits);
          if ((e.bits >> slot) & 1) {
            hd[j] = (e.block << 6) | slot;
            cl[j] = POLY ? e.cls : c;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kLevelChunk; ++j) act[j] = hd[j] != kNull && M::active(h, args, cl[j], hd[j]);
#pragma unroll
      for (int j = 0; j < kLevelChunk; ++j)
        if (act[j]) mine |= M::run(h, args, cl[j], hd[j]) != 0;
      __syncwarp();
    }
    if (__any_sync(0xFFFFFFFFu, mine) && lane == 0) any = 1;
    __syncthreads();
    if (threadIdx.x == 0 && any) atomicOr(&flags[k], 1ull);
    if (!grid_barrier(h, arrive, (unsigned)(k + 1))) break;
    if (__ldcg(&flags[k]) == 0) break;  // no frontier at this level: the search is over
  }
  if (lane == 0 && visited) count(h, SMMO_CTR_VISIT, visited);
}

// Host side: one cooperative launch of up to K levels over the snapshot
// view `v` (class c, or with POLY the classes enumerated into it).
template <class M, bool POLY>
int launch_levels(smmo_heap* hp, const HeapView& v, int c, const typename M::Args& a, int32_t base, int K,
                  unsigned long long* flags, unsigned int* arrive, cudaStream_t s) {
  static int occ = 0;
  if (occ == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, levels_kernel<M, POLY>, kLevelThreads, 0) != cudaSuccess ||
        nb < 1)
      return SMMO_E_UNSUPPORTED;
    occ = nb;
  }
  const int per_sm = occ;
  cudaError_t e = cudaMemsetAsync(arrive, 0, sizeof(unsigned int) * kBarrierWords, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long) * (size_t)K, s);
  if (e != cudaSuccess) return cuda_status(e);
  HeapView hv = v;
  uint32_t cc = (uint32_t)c;
  typename M::Args args = a;
  int32_t b = base;
  int kk = K;
  void* params[] = {&hv, &cc, &args, &b, &kk, &flags, &arrive};
  e = cudaLaunchCooperativeKernel((const void*)levels_kernel<M, POLY>, dim3((unsigned)(hp->num_sms * per_sm)),
                                  dim3(kLevelThreads), params, 0, s);
  return cuda_status(e);
}

}  // namespace smmo
