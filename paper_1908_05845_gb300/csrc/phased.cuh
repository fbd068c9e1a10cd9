// phased.cuh -- two do-alls over one snapshot in one persistent cooperative
// launch: phase 1 runs a method on every enumerated object, a grid barrier
// separates the phases, and phase 2 runs a second method on the same
// objects.  It replaces the pair parallel_do(C, prepare); parallel_do(C,
// update) of the thesis' cellular applications (Sec. 7.6: every agent
// posts its move request before any agent reads the requests) when phase 1
// creates and deletes no object of C, so one snapshot serves both.
//
// What the fusion buys on top of saving a launch: phase 1 returns one
// 32-bit word per object (the "carry"), which stays in shared memory until
// phase 2 instead of being stored to and reloaded from the object's field;
// phase 2 runs only where the carry is not M::kIdle, so objects that have
// nothing to do in the update cost no load at all.  Units (32 slots of one
// block) are processed K at a time with every load of the K units issued
// before any of them is used (the method is split into load stages and a
// compute stage), which keeps K times more independent loads in flight per
// warp than a method call per unit.
//
// Method interface (M::Args, M::P, M::U):
//   load1(h, a, c, self, P&)     loads of the object's own fields
//   load2(h, a, c, self, P&)     loads that need load1's values (gathers)
//   prepare(h, a, c, self, P&)   phase 1's compute and stores; returns the
//                                carry (kIdle: nothing to do in phase 2)
//   spill / unspill(h, a, c, self[, w])  keep the carry of a unit beyond the
//                                shared capacity in a field of the object
//   uload(h, a, c, self, w, U&)  phase 2's loads (carry w != kIdle)
//   update(h, a, c, self, w, U&) phase 2's compute and stores; may call
//                                defer_new (objects created after each
//                                K-unit round once 32 are listed, see
//                                smmo_core.cuh) and smmo_delete.
// The grid holds as many CTAs as can be resident (a cooperative launch,
// which fails instead of waiting if they cannot be); the barrier wait is
// bounded and records SMMO_E_TIMEOUT, after which phase 2 is skipped.
#pragma once
#include "heap_internal.h"
#include "levels.cuh"
#include "smmo_core.cuh"

namespace smmo {

// CTA size and the units per warp whose carries stay in shared memory
// (compile-time choices; the carries take threads x units x 4 bytes)
#ifndef SMMO_PHASED_THREADS
#define SMMO_PHASED_THREADS 256
#endif
#ifndef SMMO_CARRY_UNITS
#define SMMO_CARRY_UNITS 16
#endif
constexpr int kPhasedThreads = SMMO_PHASED_THREADS;
constexpr int kCarryUnits = SMMO_CARRY_UNITS;

// Creates the deferred objects of the calling (converged) warp, 32 at a
// time while 32 or more wait, with all = true also the rest.  Kept out of
// line: the allocator's registers then do not count against the loops of
// the phases, and the call happens once per 32 creations.
template <class M>
__device__ __noinline__ void defer_flush_call(const HeapView& h, const typename M::Args& args, bool all) {
  defer_flush<M>(h, args, all);
}

template <class M, int K, int MINB>
__global__ void __launch_bounds__(kPhasedThreads, MINB)
    phased_kernel(HeapView h, uint32_t c, typename M::Args args, unsigned long long* ctl) {
  __shared__ uint32_t carry[kPhasedThreads / 32][kCarryUnits][32];
  __shared__ uint32_t ublock[kPhasedThreads / 32][kCarryUnits];
  constexpr bool kDefer = defers<M>::max > 0;
  static_assert(defers<M>::max * K <= 2, "defer list holds two per lane and round");
  alloc_cache_init();
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (kDefer && lane == 0) g_defer[w].n = 0;
  __syncwarp();
  const uint32_t n = __ldcg(h.rcnt);
  const uint32_t cap = __ldg(&h.cls[c].cap);
  const uint32_t halves = cap > 32 ? 2u : 1u;
  const uint32_t units = n * halves;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t per = (units + nwarps - 1) / nwarps;
  const uint32_t ub = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * per;
  const uint32_t ue = ub + per < units ? ub + per : units;
  uint32_t visited = 0;

  // ---- phase 1
  for (uint32_t c0 = ub; c0 < ue; c0 += 32) {
    const uint32_t cend = c0 + 32 < ue ? c0 + 32 : ue;
    UnitEntries ents;
    ents.load(h, c0, cend, halves);
    for (uint32_t u0 = c0; u0 < cend; u0 += K) {
      uint32_t self[K];
      typename M::P p[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const uint32_t u = u0 + j;
        self[j] = kNull;
        if (u < cend) {
          uint32_t blk, ecls, bits32;
          ents.unit(u, halves, &blk, &ecls, &bits32);
          const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + lane;
          if (lane == 0) visited += __popc(bits32);
          if (u - ub < (uint32_t)kCarryUnits && lane == 0) ublock[w][u - ub] = blk;
          if ((bits32 >> lane) & 1) self[j] = (blk << 6) | slot;
        }
      }
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (self[j] != kNull) M::load1(h, args, c, self[j], p[j]);
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (self[j] != kNull) M::load2(h, args, c, self[j], p[j]);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const uint32_t u = u0 + j;
        if (u >= cend) break;
        const uint32_t cw = self[j] != kNull ? M::prepare(h, args, c, self[j], p[j]) : M::kIdle;
        if (u - ub < (uint32_t)kCarryUnits) carry[w][u - ub][lane] = cw;
        else if (self[j] != kNull) M::spill(h, args, c, self[j], cw);
      }
      __syncwarp();
    }
  }

  int dummy = 0;
  if (!level_barrier(h, ctl, 0u, false, gridDim.x, &dummy)) return;  // timed out: recorded

  // ---- phase 2
  __syncwarp();
  for (uint32_t u0 = ub; u0 < ue; u0 += K) {
    uint32_t self[K], cw[K];
    typename M::U q[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const uint32_t u = u0 + j;
      self[j] = kNull;
      cw[j] = M::kIdle;
      if (u >= ue) continue;
      const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + lane;
      if (u - ub < (uint32_t)kCarryUnits) {
        cw[j] = carry[w][u - ub][lane];
        if (cw[j] != M::kIdle) self[j] = (ublock[w][u - ub] << 6) | slot;
      } else {
        const REntry e = h.R[halves == 2 ? (u >> 1) : u];
        if ((e.bits >> slot) & 1) {
          self[j] = (e.block << 6) | slot;
          cw[j] = M::unspill(h, args, c, self[j]);
          if (cw[j] == M::kIdle) self[j] = kNull;
        }
      }
      if (lane == 0) {
        const uint32_t b = u - ub < (uint32_t)kCarryUnits ? ublock[w][u - ub] : h.R[halves == 2 ? (u >> 1) : u].block;
        g_wcache[w].hint = b;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (self[j] != kNull) M::uload(h, args, c, self[j], cw[j], q[j]);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (self[j] != kNull) M::update(h, args, c, self[j], cw[j], q[j]);
    __syncwarp();  // reconverge: the defer list is read by the whole warp
    if constexpr (kDefer) {
      if (g_defer[w].n >= 32) defer_flush_call<M>(h, args, false);
    }
  }
  if constexpr (kDefer) defer_flush_call<M>(h, args, true);
  alloc_cache_flush(h);
  // every object is visited by both phases
  if (lane == 0 && visited) count(h, SMMO_CTR_VISIT, 2ull * visited);
}

// Host side: one cooperative launch over the heap's current enumeration of
// class c, with as many CTAs per SM as can be resident, at most the heap's
// ctas_per_sm.  ctl: kBarrierWords zeroed words (the barrier's counters).
template <class M, int K, int MINB>
int launch_phased(smmo_heap* hp, int c, const typename M::Args& a, unsigned long long* ctl, cudaStream_t s) {
  static int occ = 0;
  if (occ == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, phased_kernel<M, K, MINB>, kPhasedThreads, 0) !=
            cudaSuccess || nb < 1)
      return SMMO_E_UNSUPPORTED;
    occ = nb;
  }
  const int per_sm = occ < hp->cfg.ctas_per_sm ? occ : hp->cfg.ctas_per_sm;
  HeapView hv = hp->view;
  uint32_t cc = (uint32_t)c;
  typename M::Args args = a;
  void* params[] = {&hv, &cc, &args, &ctl};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(hp->num_sms * per_sm));
  cfg.blockDim = dim3(kPhasedThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_status(cudaLaunchKernelExC(&cfg, (const void*)phased_kernel<M, K, MINB>, params));
}

}  // namespace smmo
