// wl_nbody.cu -- direct n-body with collision merge and its adjoint as an
// SMMO application (thesis Sec. 7.1 "nbody", Sec. 7.2 "collision").
//
// Class Body {x, y, z, vx, vy, vz, m, id, lx, ly, lz, lvx, lvy, lvz}; the
// last six fields hold the adjoint state.  One step (drift-kick-drift):
//   Body::drift_stage  x += v dt/2 and publish (x, m) into an id-ordered
//                      staging array (the sequential device_do of the thesis
//                      iterates over objects; here it iterates over this
//                      array in id order, which fixes the summation order);
//   force              a_i = G sum_j m_j r_ij / (|r_ij|^2 + eps^2)^{3/2}
//                      over j in id order, read tile by tile through shared
//                      memory, then v += a dt and x += v dt/2;
// and with merging (Sec. 7.2, made deterministic): restage, merge_prepare
// (a receiver takes the first lighter body within R in id order and posts
// its id with atomicMin, so the lowest receiver wins), merge_perform (a
// picked body merges into its receiver unless the receiver is itself picked,
// then deletes itself).
//
// FP32 arithmetic uses explicit round-to-nearest intrinsics in the order
//   s2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps^2))); inv = 1/(s2*sqrt(s2));
//   f = m_j*inv; a = fma(f, d, a);
// with IEEE division and square root, so results equal a sequential FP32
// evaluation in the same order bit for bit.  The self pair and freed ids
// (mass 0 in the staging array) add exactly +0 and need no branch.
//
// Adjoint (no merge, loss L = 1/2 sum m |v_T|^2, gradient w.r.t. v_0):
// checkpoints of (x, v) every `ckpt` steps; each segment is recomputed
// forward keeping the mid-step positions x1, then reversed step by step:
//   w = lambda_v + dt/2 lambda_x;  mu = dt w;
//   g_k = G sum_j H(x1_j - x1_k)(m_k mu_j - m_j mu_k),
//   H(r) = I/s^3 - 3 r r^T / s^5,  s^2 = |r|^2 + eps^2;
//   lambda_x += g;  lambda_v = w + dt/2 lambda_x.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fp32_rn.cuh"
#include "heap_internal.h"
#include "smmo.h"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

enum { CX, CY, CZ, CVX, CVY, CVZ, CM, CID, CLX, CLY, CLZ, CLVX, CLVY, CLVZ, NCOL };

struct NBodyArgs {
  float4* S;            // (x, y, z, m) by id
  float4* Sd;           // the live entries of S in id order (force partners)
  uint32_t* live;       // [0] live count; [1..] per-chunk offsets
  float4* A;            // (mu_x, mu_y, mu_z, 0) by id (adjoint)
  const float4* X1;     // mid-step (x, y, z, m) by id for the step being reversed
  uint32_t* hmap;       // handle by id
  uint32_t* tgt;        // merge receiver by id
  float* buf;           // per-id scratch (checkpoints, export)
  double* ke;           // per-id kinetic energy
  uint32_t n0;
  float G, eps2, dt, h, R2;
  uint32_t off[NCOL];
  unsigned long long* merges;
};

template <class T>
__device__ __forceinline__ T& F(const HeapView& h, uint32_t self, uint32_t off) {
  return *field_ptr<T>(h, off, self);
}

__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }

struct DriftStage {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    float& x = F<float>(hv, self, a.off[CX]);
    float& y = F<float>(hv, self, a.off[CY]);
    float& z = F<float>(hv, self, a.off[CZ]);
    x = fa(x, fm(F<float>(hv, self, a.off[CVX]), a.h));
    y = fa(y, fm(F<float>(hv, self, a.off[CVY]), a.h));
    z = fa(z, fm(F<float>(hv, self, a.off[CVZ]), a.h));
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    a.S[id] = make_float4(x, y, z, F<float>(hv, self, a.off[CM]));
    a.hmap[id] = self;
  }
};

struct Stage {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    a.S[id] = make_float4(F<float>(hv, self, a.off[CX]), F<float>(hv, self, a.off[CY]),
                          F<float>(hv, self, a.off[CZ]), F<float>(hv, self, a.off[CM]));
    a.hmap[id] = self;
    a.tgt[id] = kNull;
  }
};

// Tiled pass over all ids for the objects of class c enumerated in h.R:
// the CTA walks groups of 8 warp units (32 slots each); every thread of the
// CTA loads the shared tiles, only threads on live slots accumulate.
#define NB_TILE 256

// Coordinates bound for the branch-free square root and reciprocal: with
// |x| <= 2^18 for both bodies and eps^2 in [2^-40, 2^38], s2 lies in
// [2^-40, 2^40] and s2 sqrt(s2) in [2^-60, 2^60], the ranges on which those
// functions equal the IEEE-rounded ones.
constexpr unsigned kCoordMaxBits = 0x48800000u;  // 2^18

// One pair's weight f = m_j inv, inv = 1 / (s2 sqrt(s2)), in the fixed
// evaluation order: s2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps^2))),
// one rounding per fused multiply-add, every other operation rounded on
// its own.
template <bool FAST>
__device__ __forceinline__ float pair_f(float mj, float dx, float dy, float dz, float eps2) {
  float s2 = __fmaf_rn(dx, dx, eps2);
  s2 = __fmaf_rn(dy, dy, s2);
  s2 = __fmaf_rn(dz, dz, s2);
  const float inv = FAST ? rcp_rn_fast(fm(s2, sqrt_rn_fast(s2))) : __fdiv_rn(1.0f, fm(s2, __fsqrt_rn(s2)));
  return fm(mj, inv);
}

// Pairs whose weights are computed per round before they are accumulated:
// one body per thread leaves few warps per SM (65,536 threads), so the
// independent work of a round has to hide the latency of the square-root
// and reciprocal chains (each term keeps f and the three differences).
#ifndef SMMO_NBODY_TERMS
#define SMMO_NBODY_TERMS 16
#endif
constexpr int kForceTerms = SMMO_NBODY_TERMS;

// Sum of the pair terms of one tile into (ax, ay, az), j in increasing
// order: the weights of kForceTerms consecutive j are computed first (they
// are independent), then a = fma(f, d, a) in order, so the result is that
// of the plain loop bit for bit.
template <bool FAST>
__device__ __forceinline__ void force_tile(const float4* tile, uint32_t cnt, float xi, float yi, float zi,
                                           float eps2, float& ax, float& ay, float& az) {
  uint32_t k = 0;
  for (; k + kForceTerms <= cnt; k += kForceTerms) {
    float f[kForceTerms], dx[kForceTerms], dy[kForceTerms], dz[kForceTerms];
#pragma unroll
    for (int u = 0; u < kForceTerms; ++u) {
      const float4 p = tile[k + u];
      dx[u] = fs(p.x, xi);
      dy[u] = fs(p.y, yi);
      dz[u] = fs(p.z, zi);
      f[u] = pair_f<FAST>(p.w, dx[u], dy[u], dz[u], eps2);
    }
#pragma unroll
    for (int u = 0; u < kForceTerms; ++u) {
      ax = __fmaf_rn(f[u], dx[u], ax);
      ay = __fmaf_rn(f[u], dy[u], ay);
      az = __fmaf_rn(f[u], dz[u], az);
    }
  }
  for (; k < cnt; ++k) {
    const float4 p = tile[k];
    const float dx = fs(p.x, xi), dy = fs(p.y, yi), dz = fs(p.z, zi);
    const float f = pair_f<FAST>(p.w, dx, dy, dz, eps2);
    ax = __fmaf_rn(f, dx, ax);
    ay = __fmaf_rn(f, dy, ay);
    az = __fmaf_rn(f, dz, az);
  }
}

__device__ __forceinline__ unsigned abs_max_bits(float x, float y, float z) {
  return max(__float_as_uint(fabsf(x)), max(__float_as_uint(fabsf(y)), __float_as_uint(fabsf(z))));
}

__global__ void __launch_bounds__(256) k_force(HeapView hv, uint32_t c, NBodyArgs a) {
  __shared__ float4 tile[NB_TILE];
  __shared__ unsigned tile_max[NB_TILE / 32];
  const uint32_t n = __ldcg(hv.rcnt);
  const uint32_t cap = hv.cls[c].cap;
  const uint32_t halves = cap > 32 ? 2u : 1u;
  const uint32_t units = n * halves, groups = (units + 7) / 8;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool eps_ok = a.eps2 >= 0x1p-40f && a.eps2 <= 0x1p38f;
  for (uint32_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const uint32_t u = g * 8 + warp;
    bool live = false;
    uint32_t self = 0;
    if (u < units) {
      const REntry e = hv.R[halves == 2 ? (u >> 1) : u];
      const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + lane;
      live = (e.bits >> slot) & 1;
      self = (e.block << 6) | slot;
    }
    float xi = 0, yi = 0, zi = 0, ax = 0.0f, ay = 0.0f, az = 0.0f;
    if (live) {
      xi = F<float>(hv, self, a.off[CX]);
      yi = F<float>(hv, self, a.off[CY]);
      zi = F<float>(hv, self, a.off[CZ]);
    }
    const bool own_ok = eps_ok && abs_max_bits(xi, yi, zi) <= kCoordMaxBits;
    const uint32_t nl = __ldcg(a.live);  // partners: the live bodies in id order
    for (uint32_t base = 0; base < nl; base += NB_TILE) {
      __syncthreads();
      float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (base + threadIdx.x < nl) q = a.Sd[base + threadIdx.x];
      tile[threadIdx.x] = q;
      const unsigned wm = __reduce_max_sync(0xFFFFFFFFu, abs_max_bits(q.x, q.y, q.z));
      if (lane == 0) tile_max[warp] = wm;
      __syncthreads();
      unsigned tm = 0;
#pragma unroll
      for (int w = 0; w < NB_TILE / 32; ++w) tm = max(tm, tile_max[w]);
      const uint32_t cnt = nl - base < NB_TILE ? nl - base : NB_TILE;
      if (live) {
        if (own_ok && tm <= kCoordMaxBits) force_tile<true>(tile, cnt, xi, yi, zi, a.eps2, ax, ay, az);
        else force_tile<false>(tile, cnt, xi, yi, zi, a.eps2, ax, ay, az);
      }
    }
    if (live) {
      ax = fm(a.G, ax); ay = fm(a.G, ay); az = fm(a.G, az);
      float& vx = F<float>(hv, self, a.off[CVX]);
      float& vy = F<float>(hv, self, a.off[CVY]);
      float& vz = F<float>(hv, self, a.off[CVZ]);
      vx = fa(vx, fm(ax, a.dt));
      vy = fa(vy, fm(ay, a.dt));
      vz = fa(vz, fm(az, a.dt));
      F<float>(hv, self, a.off[CX]) = fa(xi, fm(vx, a.h));
      F<float>(hv, self, a.off[CY]) = fa(yi, fm(vy, a.h));
      F<float>(hv, self, a.off[CZ]) = fa(zi, fm(vz, a.h));
    }
  }
}

// ---- force partners: the live bodies in id order -------------------------
// The force sums over live bodies in increasing id; dead ids hold zeros in
// S (mass 0, an exact zero term).  These kernels pack the live entries of
// S, in id order, into Sd: (1) live count per chunk of 1024 ids, (2) the
// exclusive prefix over the chunks and the total, (3) every live entry to
// its place.  The sum over Sd is the sum over S without its zero terms,
// bit for bit (an accumulator that starts at +0 never becomes -0).
__global__ void __launch_bounds__(1024) k_live_count(const float4* S, uint32_t n0, uint32_t* part) {
  __shared__ uint32_t wsum[32];
  const uint32_t i = blockIdx.x * 1024 + threadIdx.x;
  const bool lv = i < n0 && S[i].w > 0.0f;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, lv);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t t = __reduce_add_sync(0xFFFFFFFFu, wsum[threadIdx.x]);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_live_scan(uint32_t* part, uint32_t nparts, uint32_t* total,
                                                    unsigned long long* pairs) {
  __shared__ uint32_t sh[1024];
  uint32_t run = 0;
  for (uint32_t base = 0; base < nparts; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nparts ? part[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {
      const uint32_t x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nparts) part[i] = run + sh[threadIdx.x] - v;
    run += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = run;
    *pairs += (unsigned long long)run * run;  // pair terms of this force pass
  }
}

__global__ void __launch_bounds__(1024) k_live_scatter(const float4* S, uint32_t n0, const uint32_t* part,
                                                       float4* Sd) {
  __shared__ uint32_t wsum[32];
  const uint32_t i = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (i < n0) v = S[i];
  const bool lv = i < n0 && v.w > 0.0f;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, lv);
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    const uint32_t c = wsum[lane];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= (uint32_t)o) incl += x;
    }
    wsum[lane] = incl - c;
  }
  __syncthreads();
  if (lv) Sd[part[blockIdx.x] + wsum[warp] + __popc(bal & ((1u << lane) - 1))] = v;
}

// ---- merge search on a hashed uniform grid (cell edge >= R) -------------
// Receiver i takes the first body j in id order with (m_j, j) < (m_i, i) and
// |x_j - x_i|^2 < R^2; the lowest receiver id wins j.  Every body j with
// |x_j - x_i| < R lies in one of the 27 cells around i's cell, so the
// smallest qualifying id over those cells is that first body.  The
// edge is R (1 + 1e-4) and cell coordinates are taken in double, so that
// neither the float distance test (which may accept |x_j - x_i| up to
// R (1 + 2^-22)) nor the rounding of x / edge can split such a pair across
// two cells apart.  Colliding hashes only add candidates, which the exact
// test rejects.
#define NB_HASH_BITS 20
#define NB_HASH (1u << NB_HASH_BITS)

__device__ __forceinline__ uint32_t cell_coord(float v, double inv_edge) {
  return (uint32_t)__double2ll_rd((double)v * inv_edge);
}

__device__ __forceinline__ uint32_t cell_hash(uint32_t cx, uint32_t cy, uint32_t cz) {
  const uint32_t h = cx * 73856093u ^ cy * 19349663u ^ cz * 83492791u;
  return (h ^ (h >> 16)) & (NB_HASH - 1);
}

struct GridArgs {
  const float4* S;
  uint32_t* cnt;    // NB_HASH counts, then fill cursors
  uint32_t* start;  // NB_HASH + 1 exclusive offsets
  uint32_t* part;   // per-CTA partial sums of the scan
  uint32_t* ids;    // n0 ids sorted by bucket
  uint32_t* tgt;
  uint32_t n0;
  float R2;
  double inv_edge;
};

__global__ void k_grid_count(GridArgs g) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n0; i += gridDim.x * blockDim.x) {
    const float4 p = g.S[i];
    if (!(p.w > 0.0f)) continue;
    atomicAdd(g.cnt + cell_hash(cell_coord(p.x, g.inv_edge), cell_coord(p.y, g.inv_edge),
                                cell_coord(p.z, g.inv_edge)), 1u);
  }
}

// exclusive scan of cnt into start: per CTA 1024 x 4 buckets
__global__ void __launch_bounds__(1024) k_grid_scan_local(GridArgs g) {
  __shared__ uint32_t sh[1024];
  const uint32_t base = blockIdx.x * 4096 + threadIdx.x * 4;
  uint32_t v[4], t = 0;
  for (int k = 0; k < 4; ++k) { v[k] = g.cnt[base + k]; t += v[k]; }
  sh[threadIdx.x] = t;
  __syncthreads();
  for (uint32_t o = 1; o < 1024; o <<= 1) {
    const uint32_t x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  uint32_t run = sh[threadIdx.x] - t;
  for (int k = 0; k < 4; ++k) { g.start[base + k] = run; run += v[k]; }
  if (threadIdx.x == 1023) g.part[blockIdx.x] = sh[1023];
}

__global__ void __launch_bounds__(256) k_grid_scan_top(GridArgs g, uint32_t nparts) {
  __shared__ uint32_t sh[256];
  const uint32_t v = threadIdx.x < nparts ? g.part[threadIdx.x] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (uint32_t o = 1; o < 256; o <<= 1) {
    const uint32_t x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  if (threadIdx.x < nparts) g.part[threadIdx.x] = sh[threadIdx.x] - v;
  if (threadIdx.x == 0) g.start[NB_HASH] = sh[255];
}

__global__ void k_grid_scatter(GridArgs g) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n0; i += gridDim.x * blockDim.x) {
    const float4 p = g.S[i];
    if (!(p.w > 0.0f)) continue;
    const uint32_t hb = cell_hash(cell_coord(p.x, g.inv_edge), cell_coord(p.y, g.inv_edge),
                                  cell_coord(p.z, g.inv_edge));
    const uint32_t pos = g.start[hb] + g.part[hb >> 12] + atomicAdd(g.cnt + hb, 1u);
    g.ids[pos] = i;
  }
}

// receiver i: smallest j in the 27 cells with (m_j, j) < (m_i, i) and
// |x_j - x_i|^2 < R^2, then atomicMin(tgt[j], i)
__global__ void k_grid_merge_prepare(GridArgs g) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n0; i += gridDim.x * blockDim.x) {
    const float4 pi = g.S[i];
    if (!(pi.w > 0.0f)) continue;
    const uint32_t cx = cell_coord(pi.x, g.inv_edge), cy = cell_coord(pi.y, g.inv_edge),
                   cz = cell_coord(pi.z, g.inv_edge);
    uint32_t pick = kNull;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const uint32_t hb = cell_hash(cx + (uint32_t)dx, cy + (uint32_t)dy, cz + (uint32_t)dz);
          const uint32_t b0 = g.start[hb] + g.part[hb >> 12];
          const uint32_t b1 = hb + 1 < NB_HASH ? g.start[hb + 1] + g.part[(hb + 1) >> 12] : g.start[NB_HASH];
          for (uint32_t q = b0; q < b1; ++q) {
            const uint32_t j = g.ids[q];
            if (j >= pick) continue;
            const float4 p = g.S[j];
            if (!(p.w < pi.w || (p.w == pi.w && j < i))) continue;
            const float ddx = fs(p.x, pi.x), ddy = fs(p.y, pi.y), ddz = fs(p.z, pi.z);
            float d2 = fm(ddx, ddx);
            d2 = fa(d2, fm(ddy, ddy));
            d2 = fa(d2, fm(ddz, ddz));
            if (d2 < g.R2) pick = j;
          }
        }
    if (pick != kNull) atomicMin(g.tgt + pick, i);
  }
}

struct MergePerform {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    const uint32_t t = a.tgt[id];
    if (t == kNull || a.tgt[t] != kNull) return;
    const uint32_t th = a.hmap[t];
    const float my = F<float>(hv, self, a.off[CM]);
    float& mt = F<float>(hv, th, a.off[CM]);
    const float nm = fa(my, mt);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float& vt = F<float>(hv, th, a.off[CVX + d]);
      const float vy = F<float>(hv, self, a.off[CVX + d]);
      vt = __fdiv_rn(fa(fm(vy, my), fm(vt, mt)), nm);
      float& xt = F<float>(hv, th, a.off[CX + d]);
      xt = __fdiv_rn(fa(F<float>(hv, self, a.off[CX + d]), xt), 2.0f);
    }
    mt = nm;
    atomicAdd(a.merges, 1ull);
    smmo_delete(hv, self);
  }
};

// id-indexed export of (x, y, z, vx, vy, vz, m) into buf (7 arrays of n0)
// and live flags into the byte array after them.
struct Export {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    for (int k = 0; k < 7; ++k) a.buf[(size_t)k * a.n0 + id] = F<float>(hv, self, a.off[k]);
    reinterpret_cast<uint8_t*>(a.buf + (size_t)7 * a.n0)[id] = 1;
  }
};

// Checkpoint save / restore of (x, v) by id into buf (6 arrays of n0).
struct SaveState {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    for (int k = 0; k < 6; ++k) a.buf[(size_t)k * a.n0 + id] = F<float>(hv, self, a.off[k]);
  }
};

struct LoadState {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    for (int k = 0; k < 6; ++k) F<float>(hv, self, a.off[k]) = a.buf[(size_t)k * a.n0 + id];
  }
};

// Loss term and adjoint initialisation at the final state:
// ke = 1/2 m |v|^2 (double), lambda_x = 0, lambda_v = m v.
struct AdjInit {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    const float m = F<float>(hv, self, a.off[CM]);
    double ke = 0;
    for (int d = 0; d < 3; ++d) {
      const float v = F<float>(hv, self, a.off[CVX + d]);
      ke += (double)v * (double)v;
      F<float>(hv, self, a.off[CLX + d]) = 0.0f;
      F<float>(hv, self, a.off[CLVX + d]) = m * v;
    }
    a.ke[id] = 0.5 * (double)m * ke;
  }
};

// First half of a reverse step: w = lambda_v + h lambda_x (kept in the
// lambda_v fields), mu = dt w published by id.
struct AdjW {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    float mu[3];
    for (int d = 0; d < 3; ++d) {
      float& lv = F<float>(hv, self, a.off[CLVX + d]);
      lv = fmaf(a.h, F<float>(hv, self, a.off[CLX + d]), lv);
      mu[d] = a.dt * lv;
    }
    a.A[id] = make_float4(mu[0], mu[1], mu[2], 0.0f);
  }
};

// Pair kernel of the reverse step (tiled like the force), then
// lambda_x += g and lambda_v = w + h lambda_x.
// Reverse-step pair sum g_k.  The sum is not bound to an evaluation order
// (its tolerance is 1e-3 against the FP64 sweep), so four lanes share one
// body, each summing every fourth id of every tile, and the four partial sums are
// combined by shuffles: 65,536 bodies then occupy four times the warps one
// lane per body would.  A CTA (8 warps) covers 64 slots (two units).
__global__ void __launch_bounds__(256, 4) k_adjoint_pair(HeapView hv, uint32_t c, NBodyArgs a) {
  __shared__ float4 tx[NB_TILE];
  __shared__ float4 tm[NB_TILE];
  const uint32_t n = __ldcg(hv.rcnt);
  const uint32_t cap = hv.cls[c].cap;
  const uint32_t halves = cap > 32 ? 2u : 1u;
  const uint32_t units = n * halves, pairs = (units + 1) / 2;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t part = lane & 3, q = warp * 8 + (lane >> 2);  // q: slot of the CTA's 64
  for (uint32_t g = blockIdx.x; g < pairs; g += gridDim.x) {
    const uint32_t u = g * 2 + (q >> 5);
    bool live = false;
    uint32_t self = 0;
    if (u < units) {
      const REntry e = hv.R[halves == 2 ? (u >> 1) : u];
      const uint32_t slot = (halves == 2 ? (u & 1) * 32 : 0) + (q & 31);
      live = (e.bits >> slot) & 1;
      self = (e.block << 6) | slot;
    }
    float4 xk = make_float4(0, 0, 0, 0), mk = make_float4(0, 0, 0, 0);
    if (live) {
      const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
      xk = a.X1[id];
      mk = a.A[id];
    }
    float gx = 0, gy = 0, gz = 0;
    for (uint32_t base = 0; base < a.n0; base += NB_TILE) {
      __syncthreads();
      if (base + threadIdx.x < a.n0) {
        tx[threadIdx.x] = a.X1[base + threadIdx.x];
        tm[threadIdx.x] = a.A[base + threadIdx.x];
      }
      __syncthreads();
      const uint32_t cnt = a.n0 - base < NB_TILE ? a.n0 - base : NB_TILE;
      if (live) {
        // lane part takes every fourth j of the tile: the four lanes of a
        // body read neighbouring float4s (distinct banks, no conflict)
        // eight terms of this lane's ids computed before they are added
        // (independent work to hide the reciprocal square root)
        uint32_t k = part;
        for (; k + 4 * (8 - 1) < cnt; k += 4 * 8) {
          float hx[8], hy[8], hz[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 p = tx[k + 4 * u], w = tm[k + 4 * u];
            const float rx = p.x - xk.x, ry = p.y - xk.y, rz = p.z - xk.z;
            const float s2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, a.eps2)));
            const float is = rsqrtf(s2);
            const float is3 = is * is * is;
            const float ux = xk.w * w.x - p.w * mk.x;
            const float uy = xk.w * w.y - p.w * mk.y;
            const float uz = xk.w * w.z - p.w * mk.z;
            const float ru = fmaf(rx, ux, fmaf(ry, uy, rz * uz));
            const float c3 = 3.0f * ru * is3 * is * is;
            hx[u] = ux * is3 - c3 * rx;
            hy[u] = uy * is3 - c3 * ry;
            hz[u] = uz * is3 - c3 * rz;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) { gx += hx[u]; gy += hy[u]; gz += hz[u]; }
        }
        for (; k < cnt; k += 4) {
          const float4 p = tx[k], w = tm[k];
            const float rx = p.x - xk.x, ry = p.y - xk.y, rz = p.z - xk.z;
            const float s2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, a.eps2)));
            const float is = rsqrtf(s2);
            const float is3 = is * is * is;
            const float ux = xk.w * w.x - p.w * mk.x;
            const float uy = xk.w * w.y - p.w * mk.y;
            const float uz = xk.w * w.z - p.w * mk.z;
            const float ru = fmaf(rx, ux, fmaf(ry, uy, rz * uz));
            const float c3 = 3.0f * ru * is3 * is * is;
          gx += ux * is3 - c3 * rx;
          gy += uy * is3 - c3 * ry;
          gz += uz * is3 - c3 * rz;
        }
      }
    }
    // combine the four lanes of a body (every lane takes part)
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      gx += __shfl_xor_sync(0xFFFFFFFFu, gx, o);
      gy += __shfl_xor_sync(0xFFFFFFFFu, gy, o);
      gz += __shfl_xor_sync(0xFFFFFFFFu, gz, o);
    }
    if (live && part == 0) {
      const float gg[3] = {a.G * gx, a.G * gy, a.G * gz};
      for (int d = 0; d < 3; ++d) {
        float& lx = F<float>(hv, self, a.off[CLX + d]);
        lx += gg[d];
        float& lv = F<float>(hv, self, a.off[CLVX + d]);
        lv = fmaf(a.h, lx, lv);
      }
    }
  }
}

struct GradOut {
  using Args = NBodyArgs;
  __device__ static void run(const HeapView& hv, const Args& a, uint32_t, uint32_t self) {
    const uint32_t id = F<int32_t>(hv, self, a.off[CID]);
    for (int d = 0; d < 3; ++d) a.buf[(size_t)id * 3 + d] = F<float>(hv, self, a.off[CLVX + d]);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_nbody[] = {
    SMMO_METHOD("nbody.drift_stage", DriftStage), SMMO_METHOD("nbody.stage", Stage),
    SMMO_METHOD("nbody.merge_perform", MergePerform), SMMO_METHOD("nbody.export", Export)};
const int g_methods_nbody_n = sizeof(g_methods_nbody) / sizeof(g_methods_nbody[0]);

struct smmo_nbody {
  smmo_heap* heap = nullptr;
  int cls = -1;
  uint32_t n0 = 0;
  smmo_nbody_params p{};
  NBodyArgs args{};
  float4* d_S = nullptr;
  float4* d_Sd = nullptr;      // live entries of d_S in id order
  uint32_t* d_live = nullptr;  // count | per-chunk offsets
  unsigned long long* d_pairs = nullptr;  // pair terms computed by the force passes
  float4* d_A = nullptr;
  uint32_t* d_hmap = nullptr;
  uint32_t* d_tgt = nullptr;
  double* d_ke = nullptr;
  unsigned long long* d_merges = nullptr;
  uint32_t* d_grid = nullptr;  // counts | start | parts | ids
  float* d_ckpt = nullptr;   // nseg x 6 x n0
  float4* d_x1 = nullptr;    // ckpt x n0
  int fw_steps = 0, fw_ckpt = 0;
  uint64_t steps_done = 0;
};

namespace {
int pdo(smmo_nbody* w, method_launch_fn fn, const NBodyArgs& a, cudaStream_t s) {
  int st = enumerate(w->heap, w->cls, s);
  if (!st) st = fn(w->heap, w->cls, &a, s);
  return st;
}

int tiled_grid(const smmo_heap* h) { return h->num_sms * 4; }

// one drift-kick-drift step (no merge); x1 (nullable) receives the mid-step
// staging array
int dkd_step(smmo_nbody* w, cudaStream_t s, float4* x1) {
  NBodyArgs a = w->args;
  cudaError_t e = cudaMemsetAsync(w->d_S, 0, sizeof(float4) * w->n0, s);
  if (e != cudaSuccess) return cuda_status(e);
  int st = pdo(w, &launch_do_all<DriftStage>, a, s);
  if (st) return st;
  if (x1) {
    e = cudaMemcpyAsync(x1, w->d_S, sizeof(float4) * w->n0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  const uint32_t nch = (w->n0 + 1023) / 1024;
  k_live_count<<<nch, 1024, 0, s>>>(w->d_S, w->n0, w->d_live + 1);
  k_live_scan<<<1, 1024, 0, s>>>(w->d_live + 1, nch, w->d_live, w->d_pairs);
  k_live_scatter<<<nch, 1024, 0, s>>>(w->d_S, w->n0, w->d_live + 1, w->d_Sd);
  k_force<<<tiled_grid(w->heap), 256, 0, s>>>(w->heap->view, w->cls, a);
  return cuda_status(cudaGetLastError());
}
}  // namespace

extern "C" {

int smmo_nbody_create(smmo_heap* heap, int64_t n, const float* const* cols,
                      const smmo_nbody_params* p, void* stream, smmo_nbody** out) {
  if (!heap || n < 1 || n > (1 << 26) || !cols || !p || !out) return SMMO_E_INVALID_ARG;
  for (int k = 0; k < 7; ++k) if (!cols[k]) return SMMO_E_INVALID_ARG;
  if (!heap->classes.empty() || heap->frozen) return SMMO_E_FROZEN;
  cudaStream_t s = (cudaStream_t)stream;
  smmo_nbody* w = new smmo_nbody();
  w->heap = heap;
  w->n0 = (uint32_t)n;
  w->p = *p;
  const char* names[NCOL] = {"x", "y", "z", "vx", "vy", "vz", "m", "id", "lx", "ly", "lz", "lvx", "lvy", "lvz"};
  smmo_field_desc f[NCOL];
  for (int k = 0; k < NCOL; ++k) f[k] = {names[k], k == CID ? SMMO_I32 : SMMO_F32, 1, -1};
  int st = smmo_class_register(heap, "Body", f, NCOL, -1, 0, &w->cls);
  if (!st) st = freeze(heap, s);
  if (st) { delete w; return st; }
  cudaError_t e = cudaMalloc(&w->d_S, sizeof(float4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_Sd, sizeof(float4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_live, sizeof(uint32_t) * (1 + ((size_t)n + 1023) / 1024));
  if (e == cudaSuccess) e = cudaMalloc(&w->d_pairs, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_pairs, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_A, sizeof(float4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_hmap, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_tgt, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_ke, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->d_merges, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&w->d_grid, sizeof(uint32_t) * (2 * (size_t)NB_HASH + 1 + 256 + (size_t)n));
  if (e == cudaSuccess) e = cudaMemsetAsync(w->d_merges, 0, sizeof(unsigned long long), s);
  int32_t* ids = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&ids, sizeof(int32_t) * n, s);
  if (e != cudaSuccess) { smmo_nbody_destroy(w); return cuda_status(e); }
  std::vector<int32_t> hid((size_t)n);
  for (int64_t i = 0; i < n; ++i) hid[i] = (int32_t)i;
  e = cudaMemcpyAsync(ids, hid.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
  float* zeros = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&zeros, sizeof(float) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(zeros, 0, sizeof(float) * n, s);
  if (e != cudaSuccess) { smmo_nbody_destroy(w); return cuda_status(e); }
  const void* src[NCOL] = {cols[0], cols[1], cols[2], cols[3], cols[4], cols[5], cols[6], ids,
                           zeros, zeros, zeros, zeros, zeros, zeros};
  st = smmo_bulk_new(heap, w->cls, n, src, nullptr, nullptr, stream);
  cudaFreeAsync(ids, s);
  cudaFreeAsync(zeros, s);
  if (st) { smmo_nbody_destroy(w); return st; }
  NBodyArgs& a = w->args;
  memset(&a, 0, sizeof(a));
  a.S = w->d_S; a.Sd = w->d_Sd; a.live = w->d_live; a.A = w->d_A; a.hmap = w->d_hmap; a.tgt = w->d_tgt; a.ke = w->d_ke;
  a.merges = w->d_merges;
  a.n0 = (uint32_t)n;
  a.G = p->G;
  a.eps2 = p->eps * p->eps;
  a.dt = p->dt;
  a.h = 0.5f * p->dt;
  a.R2 = p->merge_r * p->merge_r;
  for (int k = 0; k < NCOL; ++k) a.off[k] = heap->classes[w->cls].layout.col_off[k];
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { smmo_nbody_destroy(w); return cuda_status(e); }
  *out = w;
  return SMMO_OK;
}

int smmo_nbody_step(smmo_nbody* w, int nsteps, void* stream) {
  if (!w || nsteps < 0) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < nsteps; ++k) {
    int st = dkd_step(w, s, nullptr);
    if (st) return st;
    if (w->p.merge) {
      NBodyArgs a = w->args;
      cudaError_t e = cudaMemsetAsync(w->d_S, 0, sizeof(float4) * w->n0, s);
      if (e != cudaSuccess) return cuda_status(e);
      st = pdo(w, &launch_do_all<Stage>, a, s);
      if (st) return st;
      GridArgs g;
      g.S = w->d_S;
      g.cnt = w->d_grid;
      g.start = w->d_grid + NB_HASH;
      g.part = w->d_grid + 2 * NB_HASH + 1;
      g.ids = w->d_grid + 2 * NB_HASH + 1 + 256;
      g.tgt = w->d_tgt;
      g.n0 = w->n0;
      g.inv_edge = 1.0 / ((double)w->p.merge_r * 1.0001);
      g.R2 = a.R2;
      const unsigned gb = (unsigned)((w->n0 + 255) / 256);
      e = cudaMemsetAsync(g.cnt, 0, sizeof(uint32_t) * NB_HASH, s);
      if (e != cudaSuccess) return cuda_status(e);
      k_grid_count<<<gb, 256, 0, s>>>(g);
      k_grid_scan_local<<<NB_HASH / 4096, 1024, 0, s>>>(g);
      k_grid_scan_top<<<1, 256, 0, s>>>(g, NB_HASH / 4096);
      e = cudaMemsetAsync(g.cnt, 0, sizeof(uint32_t) * NB_HASH, s);
      if (e != cudaSuccess) return cuda_status(e);
      k_grid_scatter<<<gb, 256, 0, s>>>(g);
      k_grid_merge_prepare<<<gb, 256, 0, s>>>(g);
      st = cuda_status(cudaGetLastError());
      if (!st) st = pdo(w, &launch_do_all<MergePerform>, a, s);
      if (st) return st;
    }
    ++w->steps_done;
  }
  return SMMO_OK;
}

int smmo_nbody_export(smmo_nbody* w, float* out7, uint8_t* live, int64_t* merges, void* stream) {
  if (!w || !out7 || !live) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n0 = w->n0;
  float* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, sizeof(float) * 7 * n0 + n0, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(float) * 7 * n0 + n0, s);
  if (e != cudaSuccess) return cuda_status(e);
  NBodyArgs a = w->args;
  a.buf = buf;
  int st = pdo(w, &launch_do_all<Export>, a, s);
  if (!st) {
    e = cudaMemcpyAsync(out7, buf, sizeof(float) * 7 * n0, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(live, buf + 7 * n0, n0, cudaMemcpyDeviceToDevice, s);
    unsigned long long m = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, w->d_merges, sizeof(m), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e);
    if (merges) *merges = (int64_t)m;
  }
  cudaFreeAsync(buf, s);
  return st;
}

int smmo_nbody_forward_ckpt(smmo_nbody* w, int nsteps, int ckpt, double* loss, void* stream) {
  if (!w || nsteps < 1 || ckpt < 1 || !loss || w->p.merge) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nseg = (nsteps + ckpt - 1) / ckpt;
  const size_t n0 = w->n0;
  if (w->d_ckpt) cudaFreeAsync(w->d_ckpt, s);
  if (w->d_x1) cudaFreeAsync(w->d_x1, s);
  w->d_ckpt = nullptr;
  w->d_x1 = nullptr;
  cudaError_t e = cudaMallocAsync(&w->d_ckpt, sizeof(float) * 6 * n0 * nseg, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&w->d_x1, sizeof(float4) * n0 * ckpt, s);
  if (e != cudaSuccess) return cuda_status(e);
  w->fw_steps = nsteps;
  w->fw_ckpt = ckpt;
  NBodyArgs a = w->args;
  for (int k = 0; k < nsteps; ++k) {
    if (k % ckpt == 0) {
      a.buf = w->d_ckpt + (size_t)(k / ckpt) * 6 * n0;
      int st = pdo(w, &launch_do_all<SaveState>, a, s);
      if (st) return st;
    }
    int st = dkd_step(w, s, nullptr);
    if (st) return st;
  }
  e = cudaMemsetAsync(w->d_ke, 0, sizeof(double) * n0, s);
  if (e != cudaSuccess) return cuda_status(e);
  int st = pdo(w, &launch_do_all<AdjInit>, a, s);
  if (st) return st;
  std::vector<double> ke(n0);
  e = cudaMemcpyAsync(ke.data(), w->d_ke, sizeof(double) * n0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  double L = 0;
  for (double v : ke) L += v;  // fixed (id) order
  *loss = L;
  return SMMO_OK;
}

int smmo_nbody_backward(smmo_nbody* w, float* grad_v0, void* stream) {
  if (!w || !grad_v0 || !w->d_ckpt) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n0 = w->n0;
  const int T = w->fw_steps, ck = w->fw_ckpt, nseg = (T + ck - 1) / ck;
  NBodyArgs a = w->args;
  // adjoint fields survive LoadState (which restores x and v only)
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * ck, s1 = s0 + ck < T ? s0 + ck : T;
    a.buf = w->d_ckpt + (size_t)seg * 6 * n0;
    int st = pdo(w, &launch_do_all<LoadState>, a, s);
    if (st) return st;
    for (int k = s0; k < s1; ++k) {
      st = dkd_step(w, s, w->d_x1 + (size_t)(k - s0) * n0);
      if (st) return st;
    }
    for (int k = s1 - 1; k >= s0; --k) {
      NBodyArgs b = a;
      b.X1 = w->d_x1 + (size_t)(k - s0) * n0;
      st = pdo(w, &launch_do_all<AdjW>, b, s);
      if (st) return st;
      // one CTA per 64 ids: 1,024 CTAs at N = 65,536, all resident at once
      // on 152 SMs (at least 7 CTAs of 256 threads per SM)
      k_adjoint_pair<<<std::max<uint32_t>(1, (w->n0 + 63) / 64), 256, 0, s>>>(w->heap->view, w->cls, b);
      st = cuda_status(cudaGetLastError());
      if (st) return st;
    }
  }
  a.buf = grad_v0;
  cudaError_t e = cudaMemsetAsync(grad_v0, 0, sizeof(float) * 3 * n0, s);
  if (e != cudaSuccess) return cuda_status(e);
  return pdo(w, &launch_do_all<GradOut>, a, s);
}

int smmo_nbody_destroy(smmo_nbody* w) {
  if (!w) return SMMO_E_INVALID_ARG;
  cudaFree(w->d_S); cudaFree(w->d_Sd); cudaFree(w->d_live); cudaFree(w->d_pairs); cudaFree(w->d_A); cudaFree(w->d_hmap); cudaFree(w->d_tgt);
  cudaFree(w->d_ke); cudaFree(w->d_merges);
  if (w->d_grid) cudaFree(w->d_grid);
  if (w->d_ckpt) cudaFree(w->d_ckpt);
  if (w->d_x1) cudaFree(w->d_x1);
  delete w;
  return SMMO_OK;
}

}  // extern "C"

namespace {
// Self-test of the branch-free square root and reciprocal against the
// IEEE-rounded intrinsics on every float with bit pattern in [lo, hi].
__global__ void k_selftest_fp32_rn(uint32_t lo, uint32_t hi, unsigned long long* cnt, unsigned* first) {
  for (uint64_t u = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= hi;
       u += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((uint32_t)u);
    const bool bs = __float_as_uint(sqrt_rn_fast(x)) != __float_as_uint(__fsqrt_rn(x));
    const bool br = __float_as_uint(rcp_rn_fast(x)) != __float_as_uint(__frcp_rn(x));
    if (bs) { atomicAdd(cnt + 0, 1ull); atomicMin(first + 0, (unsigned)u); }
    if (br) { atomicAdd(cnt + 1, 1ull); atomicMin(first + 1, (unsigned)u); }
  }
}
}  // namespace

namespace {
// FP32 add/multiply throughput: eight independent chains per thread of
// x = x * m + c as a round-to-nearest multiply then add (two instructions,
// never fused), enough warps to fill every SM.  The chains stay bounded
// (m < 1) and the result is stored so that nothing is eliminated.
__global__ void __launch_bounds__(256) k_fp32_peak(float* out, int iters) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
  const float m = 0.999999f, c = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __fadd_rn(__fmul_rn(x[k], m), c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// FP32 fused multiply-add throughput: the same chains as one fused
// multiply-add each (two floating-point operations per instruction).
__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
  const float m = 0.999999f, c = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __fmaf_rn(x[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// Special-function throughput: eight independent chains per thread of the
// hardware reciprocal square root (x -> rsqrt(x) stays near 1).
__global__ void __launch_bounds__(256) k_mufu_peak(float* out, int iters) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.5f + (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("rsqrt.approx.f32 %0, %0;" : "+f"(x[k]));
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class K>
int time_peak(K kernel, int iters, double ops_per_thread_iter, double* ops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
  if (e != cudaSuccess) return cuda_status(e);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  float* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaMallocAsync(&out, sizeof(float) * (size_t)grid * 256, s);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float ms = 0.0f;
  if (e == cudaSuccess) {
    kernel<<<grid, 256, 0, s>>>(out, iters < 64 ? iters : 64);  // warm-up
    cudaEventRecord(a, s);
    kernel<<<grid, 256, 0, s>>>(out, iters);
    cudaEventRecord(b, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (out) cudaFreeAsync(out, s);
  if (e != cudaSuccess) return cuda_status(e);
  *ops_per_s = ms > 0.0f ? (double)grid * 256.0 * iters * ops_per_thread_iter / (ms * 1e-3) : 0.0;
  return SMMO_OK;
}
}  // namespace

extern "C" {

int smmo_selftest_fp32_rn(uint32_t lo_bits, uint32_t hi_bits, uint64_t* out4, void* stream) {
  if (!out4 || lo_bits > hi_bits || hi_bits >= 0x7F800000u) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* cnt = nullptr;
  unsigned* first = nullptr;
  cudaError_t e = cudaMallocAsync(&cnt, 2 * sizeof(unsigned long long) + 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_status(e);
  first = reinterpret_cast<unsigned*>(cnt + 2);
  e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(first, 0xFF, 2 * sizeof(unsigned), s);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    k_selftest_fp32_rn<<<sms * 16, 256, 0, s>>>(lo_bits, hi_bits, cnt, first);
    e = cudaGetLastError();
  }
  unsigned long long hc[2] = {0, 0};
  unsigned hf[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, first, sizeof(hf), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(cnt, s);
  if (e != cudaSuccess) return cuda_status(e);
  out4[0] = hc[0];
  out4[1] = hc[1];
  out4[2] = hf[0];
  out4[3] = hf[1];
  return SMMO_OK;
}

int smmo_measure_fp32_peak(int iters, double* ops_per_s, void* stream) {
  if (!ops_per_s || iters < 1 || iters > (1 << 20)) return SMMO_E_INVALID_ARG;
  return time_peak(k_fp32_peak, iters, 16.0, ops_per_s, (cudaStream_t)stream);
}

int smmo_measure_fma_peak(int iters, double* flops_per_s, void* stream) {
  if (!flops_per_s || iters < 1 || iters > (1 << 20)) return SMMO_E_INVALID_ARG;
  return time_peak(k_fma_peak, iters, 16.0, flops_per_s, (cudaStream_t)stream);  // 8 chains x 2 flops
}

int smmo_measure_mufu_peak(int iters, double* ops_per_s, void* stream) {
  if (!ops_per_s || iters < 1 || iters > (1 << 20)) return SMMO_E_INVALID_ARG;
  return time_peak(k_mufu_peak, iters, 8.0, ops_per_s, (cudaStream_t)stream);
}

int smmo_nbody_pairs(smmo_nbody* w, int64_t* pairs, void* stream) {
  if (!w || !pairs) return SMMO_E_INVALID_ARG;
  unsigned long long v = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&v, w->d_pairs, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *pairs = (int64_t)v;
  return SMMO_OK;
}

}  // extern "C"
