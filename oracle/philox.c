/*
 * philox.c -- Philox4x32-10 counter-based generator (oracle side).
 *
 * TEST INFRASTRUCTURE ONLY (see kpo.h).
 *
 * Written from the definition in Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11, Sec. 4: a 4-word, 32-bit
 * Philox bijection applied for ten rounds.  Each round multiplies words 0
 * and 2 by the two round multipliers, keeps both halves of each 64-bit
 * product, and mixes the high halves with the other two words and the
 * round key; the 2-word key is advanced by the Weyl increments between
 * rounds.  The paper itself draws controls and durations "randomly"
 * (Algorithm 2); the generator and its counter layout are this project's
 * definition so that the oracle and the device code make the same draws.
 */
#include "kpo.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void mul_hi_lo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void kpo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: add the Weyl constants */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mul_hi_lo(PHILOX_M0, x0, &hi0, &lo0);
    mul_hi_lo(PHILOX_M1, x2, &hi1, &lo1);
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void kpo_philox4x32_10_n(const uint32_t *ctr, const uint32_t key[2], uint32_t *out,
                         int64_t n) {
  for (int64_t i = 0; i < n; ++i) kpo_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}
