// Device-side operand generator for served workloads.
//
// Element i of operand o (0 = a, 1 = b) of request q under seed s is the
// residue mod p of the 128-bit output of Philox4x32-10 (Salmon, Moraes,
// Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011)
// with counter (i, o, q mod 2^32, q div 2^32) and key (s mod 2^32,
// s div 2^32); the four output words x0..x3 form
// v = x0 + 2^32 x1 + 2^64 x2 + 2^96 x3.  This is not part of the transform:
// it lets a served request carry only (q, na, nb) while its operands are
// produced in device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "field.cuh"
#include "tft_internal.h"

namespace tftgb {

namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;  // round multipliers
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;  // key schedule increments
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr int kGenThreads = 256;
constexpr int kGenPerThread = 4;
constexpr uint64_t kGenChunk = (uint64_t)kGenThreads * kGenPerThread;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// v mod p for the 128-bit v of the four words.
template <int PRIME>
__device__ __forceinline__ uint64_t reduce_words(uint4 x);

template <>
__device__ __forceinline__ uint64_t reduce_words<2>(uint4 x) {
  const uint64_t lo = (uint64_t)x.x | ((uint64_t)x.y << 32);
  const uint64_t hi = (uint64_t)x.z | ((uint64_t)x.w << 32);
  return Goldilocks::canon(Goldilocks::reduce128(lo, hi));
}

template <uint64_t P>
__device__ __forceinline__ uint64_t horner32(uint4 x) {
  // most significant word first; each step keeps acc < p < 2^31
  uint64_t acc = x.w % P;
  acc = ((acc << 32) | x.z) % P;
  acc = ((acc << 32) | x.y) % P;
  return ((acc << 32) | x.x) % P;
}
template <>
__device__ __forceinline__ uint64_t reduce_words<0>(uint4 x) {
  return horner32<998244353ull>(x);
}
template <>
__device__ __forceinline__ uint64_t reduce_words<1>(uint4 x) {
  return horner32<2013265921ull>(x);
}

template <int PRIME>
__device__ __forceinline__ void gen_store(void* dst, uint64_t i,
                                          uint64_t v) {
  if (PRIME == 2)
    reinterpret_cast<uint64_t*>(dst)[i] = v;
  else
    reinterpret_cast<uint32_t*>(dst)[i] = (uint32_t)v;
}

template <int PRIME>
__device__ __forceinline__ void gen_chunk(void* dst, uint64_t n,
                                          uint64_t request, uint32_t operand,
                                          uint64_t seed, uint64_t first) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int j = 0; j < kGenPerThread; ++j) {
    const uint64_t i = first + (uint64_t)j * kGenThreads + threadIdx.x;
    if (i < n) {
      const uint4 c = make_uint4((uint32_t)i, operand, (uint32_t)request,
                                 (uint32_t)(request >> 32));
      gen_store<PRIME>(dst, i, reduce_words<PRIME>(philox4x32_10(c, k0, k1)));
    }
  }
}

// All operands of a table, chunk by chunk (chunk -> descriptor by a
// binary search over the prefix chunk_base).
template <int PRIME>
__global__ void __launch_bounds__(kGenThreads)
k_gen_table(const GenDesc* __restrict__ d, uint32_t nd, uint64_t chunks,
            uint64_t seed) {
  for (uint64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
    uint32_t lo = 0, hi = nd;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (d[mid].chunk_base <= ch)
        lo = mid;
      else
        hi = mid;
    }
    const GenDesc q = d[lo];
    gen_chunk<PRIME>(reinterpret_cast<void*>(q.dst), q.n, q.request,
                     q.operand, seed, (ch - q.chunk_base) * kGenChunk);
  }
}

// Both operands of one request (blockIdx.y = operand).
template <int PRIME>
__global__ void __launch_bounds__(kGenThreads)
k_gen_pair(void* a, uint64_t na, void* b, uint64_t nb, uint64_t request,
           uint64_t seed) {
  void* dst = blockIdx.y ? b : a;
  const uint64_t n = blockIdx.y ? nb : na;
  for (uint64_t first = (uint64_t)blockIdx.x * kGenChunk; first < n;
       first += (uint64_t)gridDim.x * kGenChunk)
    gen_chunk<PRIME>(dst, n, request, blockIdx.y, seed, first);
}

uint32_t grid_for(uint64_t chunks, int nsm) {
  const uint64_t cap = (uint64_t)nsm * 8;
  return (uint32_t)(chunks < cap ? (chunks ? chunks : 1) : cap);
}

}  // namespace

uint64_t gen_chunks(uint64_t n) { return (n + kGenChunk - 1) / kGenChunk; }

cudaError_t launch_gen_table(int prime, const GenDesc* d, uint32_t nd,
                             uint64_t chunks, uint64_t seed, int nsm,
                             cudaStream_t s) {
  if (!nd || !chunks) return cudaSuccess;
  const uint32_t grid = grid_for(chunks, nsm);
  switch (prime) {
    case 0: k_gen_table<0><<<grid, kGenThreads, 0, s>>>(d, nd, chunks, seed); break;
    case 1: k_gen_table<1><<<grid, kGenThreads, 0, s>>>(d, nd, chunks, seed); break;
    case 2: k_gen_table<2><<<grid, kGenThreads, 0, s>>>(d, nd, chunks, seed); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gen_pair(int prime, void* a, uint64_t na, void* b,
                            uint64_t nb, uint64_t request, uint64_t seed,
                            int nsm, cudaStream_t s) {
  const uint64_t ch = gen_chunks(na > nb ? na : nb);
  const dim3 grid(grid_for(ch, nsm), 2);
  switch (prime) {
    case 0: k_gen_pair<0><<<grid, kGenThreads, 0, s>>>(a, na, b, nb, request, seed); break;
    case 1: k_gen_pair<1><<<grid, kGenThreads, 0, s>>>(a, na, b, nb, request, seed); break;
    case 2: k_gen_pair<2><<<grid, kGenThreads, 0, s>>>(a, na, b, nb, request, seed); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tftgb
