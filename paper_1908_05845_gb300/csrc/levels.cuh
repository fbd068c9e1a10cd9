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
constexpr int kBarrierWords = 64;                  // 64-bit words: [0], [16] counters, [32] release

// Barrier across the grid's CTAs that also combines one bit per CTA (did
// it find a frontier object).  Level k (counted from 0 in the launch) adds
// 1 + (bit << 32) to the counter ctl[16 (k mod 2)]; the CTA whose addition
// completes the count of `ncta` CTAs sees the OR of all bits in the high
// half of the result, resets the other counter (the next level's: all CTAs
// are past the level before), and publishes ((k + 1) << 1) | OR in the
// release word ctl[32], on which the others wait.  Counters and release
// word lie in different cache lines, so the waiting reads do not slow the
// arrivals.  Returns 0 on timeout (recorded as SMMO_E_TIMEOUT), else 1,
// with the level's OR in *any_out.  ctl is zeroed before the launch.
__device__ __forceinline__ bool level_barrier(const HeapView& h, unsigned long long* ctl, unsigned int k, bool bit,
                                              unsigned int ncta, int* any_out,
                                              unsigned spin_limit = kLevelBarrierSpins) {
  __shared__ int ok, any;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned long long add = 1ull + (bit ? (1ull << 32) : 0ull);
    const unsigned long long now = atomicAdd(ctl + 16 * (k & 1), add) + add;
    if ((now & 0xFFFFFFFFull) == ncta) {
      ctl[16 * ((k + 1) & 1)] = 0ull;
      __threadfence();
      atomicExch(ctl + 32, ((unsigned long long)(k + 1) << 1) | ((now >> 32) ? 1ull : 0ull));
    }
    unsigned spins = 0;
    unsigned long long r;
    while (((r = *(volatile unsigned long long*)(ctl + 32)) >> 1) < k + 1) {
      if (++spins > spin_limit) {
        ok = 0;
        set_error(h, SMMO_E_TIMEOUT, k + 1);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    any = (int)(r & 1);
  }
  __syncthreads();
  *any_out = any;
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
                                                     int K, unsigned long long* flags, unsigned long long* ctl) {
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
    int level_or = 0;
    if (!level_barrier(h, ctl, (unsigned)k, any != 0, gridDim.x, &level_or)) break;
    if (threadIdx.x == 0 && blockIdx.x == 0 && level_or) flags[k] = 1ull;  // for the host
    if (!level_or) break;  // no frontier at this level: the search is over
  }
  if (lane == 0 && visited) count(h, SMMO_CTR_VISIT, visited);
}

// Host side: one cooperative launch of up to K levels over the snapshot
// view `v` (class c, or with POLY the classes enumerated into it).
template <class M, bool POLY>
int launch_levels(smmo_heap* hp, const HeapView& v, int c, const typename M::Args& a, int32_t base, int K,
                  unsigned long long* flags, unsigned long long* ctl, cudaStream_t s) {
  static int occ = 0;
  if (occ == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, levels_kernel<M, POLY>, kLevelThreads, 0) != cudaSuccess ||
        nb < 1)
      return SMMO_E_UNSUPPORTED;
    occ = nb;
  }
  const int per_sm = occ;
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(unsigned long long) * kBarrierWords, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long) * (size_t)K, s);
  if (e != cudaSuccess) return cuda_status(e);
  HeapView hv = v;
  uint32_t cc = (uint32_t)c;
  typename M::Args args = a;
  int32_t b = base;
  int kk = K;
  void* params[] = {&hv, &cc, &args, &b, &kk, &flags, &ctl};
  e = cudaLaunchCooperativeKernel((const void*)levels_kernel<M, POLY>, dim3((unsigned)(hp->num_sms * per_sm)),
                                  dim3(kLevelThreads), params, 0, s);
  return cuda_status(e);
}

}  // namespace smmo
