// grid_common.cuh -- helpers shared by the cellular workloads (Life, Wa-Tor):
// counter-based random draws, the instance table of a (batched) heap, and
// addressing of the statically allocated Cell objects.
#pragma once
#include <cstdint>

#include "smmo_core.cuh"

namespace smmo {

// Philox4x32-10 (Salmon et al., SC'11, Sec. 3.2 and Table 2): ten rounds of
// two 32x32->64 multiplications, high halves xored with the other counter
// words and the round key, Weyl-sequence key schedule.  draw() returns word
// 0 for key (seed lo, seed hi) and counter (step, cell, tag, inst).
__device__ __forceinline__ uint32_t philox_draw(uint64_t seed, uint32_t tag, uint32_t step,
                                                uint32_t cell, uint32_t inst) {
  uint32_t c0 = step, c1 = cell, c2 = tag, c3 = inst;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return c0;
}

// Random-stream tags of the step draws.
enum : uint32_t { TAG_FISH = 1, TAG_SHARK = 2, TAG_ROUTE = 5, TAG_BRAKE = 6 };

// Division by the invariant width W as a multiply-high (Granlund and
// Montgomery, PLDI 1994): with M = floor((2^64 - 1) / W) + 1 the product
// lc M / 2^64 exceeds lc / W by less than lc / 2^64 < 1 / W for lc < 2^32,
// too little to reach the next integer, so its floor is floor(lc / W).
__host__ __device__ inline uint64_t div_magic(uint32_t W) { return ~0ull / W + 1; }

// (x, y) of local cell lc of instance in (row-major, width W).
__device__ __forceinline__ void cell_xy(const Inst* in, uint32_t lc, uint32_t* x, uint32_t* y) {
  const uint32_t q = (uint32_t)__umul64hi((unsigned long long)lc, in->wdiv);
  *y = q;
  *x = lc - q * in->W;
}

// Instance owning global cell g: the heap's instance-table row whose cell
// range holds g (one simulation instance of a batched heap; its cells
// occupy the global range [cell_base, cell_base + W*H) of the dense Cell
// objects).
__device__ __forceinline__ const Inst* find_inst(const HeapView& h, uint32_t g) {
  return instance_at(h.inst, h.n_inst, g);
}

// The Cell objects are created by one bulk_new into consecutive blocks of
// capacity N = 2^shift (32 or 64), so cell g is object slot g % N of block
// b0 + g / N.
struct CellRef {
  uint8_t* data;
  uint32_t block_bytes;
  uint32_t b0;
  uint32_t shift;
  __device__ __forceinline__ uint8_t* blk(uint32_t g) const {
    return data + (size_t)(b0 + (g >> shift)) * block_bytes;
  }
  template <class T>
  __device__ __forceinline__ T* col(uint32_t g, uint32_t off) const {
    return reinterpret_cast<T*>(blk(g) + off) + (g & ((1u << shift) - 1));
  }
  __device__ __forceinline__ uint32_t handle(uint32_t g) const {
    return ((b0 + (g >> shift)) << 6) | (g & ((1u << shift) - 1));
  }
  __device__ __forceinline__ uint32_t cell_of(uint32_t handle) const {
    return (((handle >> 6) - b0) << shift) | (handle & 63);
  }
};

// The step counter lives in device memory so that a captured step graph
// advances it on every replay; this kernel opens a step (t <- t + 1).
static __global__ void k_step_begin(uint32_t* t) { *t += 1; }

// Torus neighbour of local cell (x, y) in direction d:
// 0 = (0,-1), 1 = (+1,0), 2 = (0,+1), 3 = (-1,0).
__device__ __forceinline__ uint32_t torus_nb4(uint32_t x, uint32_t y, uint32_t W, uint32_t H, int d) {
  uint32_t nx = x, ny = y;
  if (d == 0) ny = y == 0 ? H - 1 : y - 1;
  else if (d == 1) nx = x + 1 == W ? 0 : x + 1;
  else if (d == 2) ny = y + 1 == H ? 0 : y + 1;
  else nx = x == 0 ? W - 1 : x - 1;
  return ny * W + nx;
}

}  // namespace smmo
