/*
 * Counter-based random numbers for the oracle -- TEST INFRASTRUCTURE.
 *
 * Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter, a 2 x 32-bit
 * key, ten rounds of two 32x32->64 multiplications whose high halves are
 * xored with the other counter words and the round key, and a Weyl-sequence
 * key schedule.
 *
 * Stream layout. The paper (Sec. 2) ties each track's random stream to its
 * slot index, which makes results depend on the slot count. Here the stream
 * is tied to the track itself instead: key = (seed, event), counter =
 * (track id low, track id high, draw index / 2, 0). Draw index n uses output
 * words (0, 1) when n is even and (2, 3) when odd, as one 64-bit word
 * hi << 32 | lo. A uniform deviate is u = (floor(w / 2^12) + 1/2) * 2^-52,
 * which is exact in binary64 and lies in [2^-53, 1 - 2^-53].
 */
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void om_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

uint64_t om_raw_word(uint32_t seed, uint32_t event, uint64_t tid, uint32_t index) {
  uint32_t ctr[4] = {(uint32_t)tid, (uint32_t)(tid >> 32), index >> 1, 0u};
  uint32_t key[2] = {seed, event};
  uint32_t out[4];
  om_philox4x32_10(ctr, key, out);
  if ((index & 1u) == 0u) return ((uint64_t)out[1] << 32) | out[0];
  return ((uint64_t)out[3] << 32) | out[2];
}

double om_uniform(uint64_t w) {
  return ((double)(w >> 12) + 0.5) * 0x1p-52;
}

uint64_t om_draw_raw(om_rng* r) {
  uint64_t w = om_raw_word(r->seed, r->event, r->tid, r->ctr);
  r->ctr += 1u;
  return w;
}

double om_draw(om_rng* r) { return om_uniform(om_draw_raw(r)); }
