/*
 * Oracle of the served workload's operand generator (test infrastructure
 * only; never linked into the library).
 *
 * Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC 2011): a 128-bit counter of four
 * 32-bit words and a 64-bit key of two words; each of the ten rounds
 * multiplies words 0 and 2 by two fixed 32-bit constants into 64-bit
 * products, and the new counter is (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
 * hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is advanced by two Weyl
 * constants before every round after the first.
 *
 * Element i of operand o of request q under seed s: the counter is
 * (i, o, q mod 2^32, q div 2^32), the key (s mod 2^32, s div 2^32), and the
 * element is v mod p for v = x0 + 2^32 x1 + 2^64 x2 + 2^96 x3, reduced here
 * with unsigned __int128 % p.
 */
#include <stdint.h>

typedef unsigned __int128 u128;

static const uint64_t kPrimes[3] = {998244353ull, 2013265921ull,
                                    0xFFFFFFFF00000001ull};

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = (uint64_t)M0 * c0;
    const uint64_t p1 = (uint64_t)M1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

int orc_gen_operand(int id, uint64_t seed, uint64_t request,
                    uint32_t operand, uint64_t n, uint64_t *out) {
  if (id < 0 || id > 2) return 1;
  const uint64_t p = kPrimes[id];
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint64_t i = 0; i < n; ++i) {
    const uint32_t ctr[4] = {(uint32_t)i, operand, (uint32_t)request,
                             (uint32_t)(request >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    const u128 v = (u128)x[0] | ((u128)x[1] << 32) | ((u128)x[2] << 64) |
                   ((u128)x[3] << 96);
    out[i] = (uint64_t)(v % p);
  }
  return 0;
}
