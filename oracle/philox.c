/*
 * Philox4x32-10 for the oracle (test infrastructure only).
 *
 * Written from the published definition: J. K. Salmon, M. A. Moraes,
 * R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11, Sec. 3.2 (the Philox S-box: two 32x32->64 multiplications whose
 * high halves are xored with the other counter words and the round key,
 * followed by a fixed permutation) and Table 2 (multipliers 0xD2511F53 and
 * 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85, 10 rounds).
 *
 * draw() is the counter-based stream used by every random decision of the
 * workloads: key = (seed mod 2^32, seed >> 32), counter = (step, cell, tag,
 * inst), result = word 0.
 */
#include "oracle.h"

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

uint32_t orc_draw(uint64_t seed, uint32_t tag, uint32_t step, uint32_t cell,
                  uint32_t inst) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {step, cell, tag, inst};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[0];
}

void orc_draw_many(uint64_t seed, uint32_t tag, uint32_t step,
                   const uint32_t* cells, int64_t n, uint32_t inst,
                   uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_draw(seed, tag, step, cells[i], inst);
}
