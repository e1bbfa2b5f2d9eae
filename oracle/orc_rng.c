/*
 * orc_rng.c -- counter-based random numbers of the CPU oracle.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64
 * multiplications by the round constants M0, M1 with a Weyl-sequence key
 * schedule (W0, W1).  Per round, with counter (c0, c1, c2, c3) and key
 * (k0, k1):  (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
 *            new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
 * then the key is bumped by (W0, W1) before the next round.
 *
 * Stream layout (the tracer's draw contract): counter = (ray id low word,
 * ray id high word, block index, instrument id), key = (seed low, seed high).
 */
#include "orc.h"

#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void block_words(uint64_t id, uint32_t instr, uint64_t seed, uint32_t block,
                        uint32_t x[4])
{
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), block, instr};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, x);
}

/* Draw j in binary64: the 64-bit word (hi << 32 | lo) made of words
 * 2(j mod 2) (lo) and 2(j mod 2)+1 (hi) of block j/2; its top 53 bits
 * times 2^-53, so u is in [0, 1) on a grid of 2^-53. */
double orc_uniform64(uint64_t id, uint32_t instr, uint64_t seed, uint32_t j)
{
  uint32_t x[4];
  block_words(id, instr, seed, j >> 1, x);
  uint32_t lo = x[2 * (j & 1u)], hi = x[2 * (j & 1u) + 1];
  uint64_t v = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(v >> 11) * 0x1.0p-53;
}

/* Draw j in binary32: word j mod 4 of block j/4; its top 24 bits times 2^-24. */
float orc_uniform32(uint64_t id, uint32_t instr, uint64_t seed, uint32_t j)
{
  uint32_t x[4];
  block_words(id, instr, seed, j >> 2, x);
  return (float)(x[j & 3u] >> 8) * 0x1.0p-24f;
}

/* ln x from IEEE operations in a fixed order (the atanh series of orc.h).
 * The reduction is exact (exponent and significand taken from the bits, a
 * halving of m); every later step is one correctly rounded operation. */
double orc_ln64(double x)
{
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  int e = (int)((b >> 52) & 0x7ffu) - 1023;
  const uint64_t mb = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  double m;
  memcpy(&m, &mb, sizeof m);
  if (m > 1.4142135623730951) { m = m * 0.5; e += 1; }
  const double f = (m - 1.0) / (m + 1.0);
  const double f2 = f * f;
  double p = 1.0 / 21.0;
  for (int k = 9; k >= 0; k--) p = p * f2 + 1.0 / (double)(2 * k + 1);
  return (double)e * 0.6931471805599453 + 2.0 * f * p;
}

float orc_ln32(float x)
{
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  int e = (int)((b >> 23) & 0xffu) - 127;
  const uint32_t mb = (b & 0x007fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mb, sizeof m);
  if (m > (float)1.4142135623730951) { m = m * 0.5f; e += 1; }
  const float f = (m - 1.0f) / (m + 1.0f);
  const float f2 = f * f;
  float p = 1.0f / 11.0f;
  for (int k = 4; k >= 0; k--) p = p * f2 + 1.0f / (float)(2 * k + 1);
  return (float)e * (float)0.6931471805599453 + 2.0f * f * p;
}
