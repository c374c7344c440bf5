// Host-side helpers shared by the C-ABI translation units: the primes'
// parameters, exact modular arithmetic for tables and plans, and small
// utilities.  Host code only (no kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tftgb {

typedef unsigned __int128 u128;

struct PrimeInfo {
  uint64_t p;
  int K;
  uint64_t g;
  uint32_t w;  // element bytes
};

const PrimeInfo kPrimes[3] = {
    {998244353ull, 23, 3, 4},
    {2013265921ull, 27, 31, 4},
    {0xFFFFFFFF00000001ull, 32, 7, 8},
};

inline uint64_t mulm(uint64_t a, uint64_t b, uint64_t p) {
  return (uint64_t)(((u128)a * b) % p);
}
inline uint64_t powm(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulm(r, a, p);
    a = mulm(a, a, p);
    e >>= 1;
  }
  return r;
}
inline uint64_t rev_bits(uint64_t s, int k) {
  uint64_t o = 0;
  for (int i = 0; i < k; i++) {
    o = (o << 1) | (s & 1);
    s >>= 1;
  }
  return o;
}
// omega_s = omega_[K]^(rev_K s)
inline uint64_t omega_s(const PrimeInfo& pr, uint64_t s) {
  uint64_t top = powm(pr.g, (pr.p - 1) >> pr.K, pr.p);
  return powm(top, rev_bits(s, pr.K), pr.p);
}
// twiddle form: Montgomery (x 2^32) for the 32-bit primes, identity otherwise
inline uint64_t to_tw(const PrimeInfo& pr, uint64_t x) {
  if (pr.w == 8) return x % pr.p;
  return (uint64_t)((((u128)(x % pr.p)) << 32) % pr.p);
}

inline int ceil_log2(uint64_t n) {
  int l = 0;
  while ((1ull << l) < n) ++l;
  return l;
}

inline bool valid_prime(int prime) { return prime >= 0 && prime < 3; }

// Largest transform length the two-pass plan handles.
inline uint64_t max_supported(const PrimeInfo& pr) {
  return pr.w == 8 ? (1ull << 25) : (1ull << 27);
}

// Choose the plan for length n (see tft_internal.h).  Returns false if n is

// RAII switch to the context's device.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
      cudaSetDevice(prev);
  }
};

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

inline bool overlap(const void* a, uint64_t abytes, const void* b, uint64_t bbytes) {
  const uintptr_t a0 = (uintptr_t)a, a1 = a0 + abytes;
  const uintptr_t b0 = (uintptr_t)b, b1 = b0 + bbytes;
  return a0 < b1 && b0 < a1;
}

}  // namespace tftgb
