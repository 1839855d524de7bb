/*
 * Oracle random numbers and track ids -- TEST INFRASTRUCTURE (see oracle.h).
 *
 * Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4-word counter and
 * a 2-word key; each of the 10 rounds multiplies words 0 and 2 by the two round
 * multipliers, keeps both halves of the 64-bit products and mixes the high
 * halves with the other words and the key; the key is advanced by the two Weyl
 * constants between rounds.  The paper's AdePT keeps a per-track RNG state
 * (Sec. 5, the photon RNG-state field); the toy model replaces it by this
 * stateless generator keyed by (seed, event) and countered by (id, step, block).
 *
 * The SplitMix64 finalizer (Steele, Lea, Flood, OOPSLA 2014) derives secondary
 * track ids.
 */
#include "oracle.h"

#define PHILOX_MUL0 0xD2511F53u
#define PHILOX_MUL1 0xCD9E8D57u
#define PHILOX_WEYL0 0x9E3779B9u
#define PHILOX_WEYL1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_WEYL0;
      k1 += PHILOX_WEYL1;
    }
    uint64_t p0 = (uint64_t)PHILOX_MUL0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_MUL1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u = ((x >> 8) + 1) * 2^-24, in (0, 1]; exact in FP32. */
float oracle_u01(uint32_t x) {
  return (float)((x >> 8) + 1u) * (1.0f / 16777216.0f);
}

uint64_t oracle_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Secondary with ordinal k (0..3) created at the parent's track-local step s. */
uint64_t oracle_secondary_id(uint64_t parent, uint32_t step, uint32_t ordinal) {
  uint64_t tag = ((uint64_t)step << 2) | (uint64_t)(ordinal & 3u) | (1ull << 62);
  return oracle_mix64(parent ^ oracle_mix64(tag));
}

/* Array form: out[4 i + j] for counters ctr[4 i + j], one key. */
void oracle_philox_n(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, size_t n) {
  for (size_t i = 0; i < n; ++i) oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}
