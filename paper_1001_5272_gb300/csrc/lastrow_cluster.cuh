// The ragged last row without global scratch (tft_forward_noscratch,
// tft_inverse_noscratch).
//
// With n = a R + b, b > 0, block a of the network (the last row) has as
// inputs, for the short columns q >= b, the values E_q = C_q(omega_a) of the
// column polynomials C_q(x) = sum_{t < a} X_{q + tR} x^t at omega_a -- the
// row/column form of the odd-child evaluations that Algorithm 1 adds to an
// unpaired element and Algorithm 2 subtracts (Sections 3 and 4).  The other
// transforms keep the R - b values E_q in an R-word scratch between the
// column pass and the last row.  Here one thread-block cluster computes
// them where they are needed: each of its CTAs evaluates the polynomials of
// a share of the short columns by Horner's rule straight from the buffer --
// the raw coefficients before the short columns are transformed (forward),
// the recovered coefficients after they are inverted (inverse) -- into its
// own shared memory; the leading CTA gathers the whole row through
// distributed shared memory and runs the row: the first b outputs of block a
// (forward, the pruned network) or the generalized block inverse with the
// known outputs at q < b and the known inputs E_q at q >= b (inverse).
// Nothing outside the n-word buffer is written or read.
#pragma once
#include <cooperative_groups.h>

#include "engine.cuh"

namespace tftgb {

// CTAs per cluster (the portable maximum).
constexpr int kLastRowCluster = 8;

// Short columns per CTA for a row of 2^lr with b long columns.
__host__ __device__ inline uint32_t lastrow_cluster_share(int lr, uint64_t b) {
  const uint32_t nshort = (1u << lr) - (uint32_t)b;
  return (nshort + kLastRowCluster - 1) / kLastRowCluster;
}

// Shared layout: E slice (share words, 16-byte aligned) | Z (R) | W (R/2) |
// Wih (R/2) | L (R/2).
template <class T>
__host__ __device__ inline size_t lastrow_cluster_smem(int lr, uint64_t b) {
  const size_t R = (size_t)1 << lr;
  const size_t share = lastrow_cluster_share(lr, b);
  const size_t head = (share * sizeof(T) + 15) & ~(size_t)15;
  return head + sizeof(T) * (R + 3 * (R / 2));
}

template <class F, bool INV>
__global__ void __cluster_dims__(kLastRowCluster, 1, 1) __launch_bounds__(512)
k_lastrow_cluster(typename F::T* X, int lr, uint64_t a, uint64_t b,
                  typename F::T omega_a_tw, RootTable<typename F::T> rt) {
  namespace cg = cooperative_groups;
  using T = typename F::T;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  {
    const T* src = reinterpret_cast<const T*>(&rt);
    T* dst = reinterpret_cast<T*>(&s_rt);
    constexpr int nwords = sizeof(RootTable<T>) / sizeof(T);
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const uint32_t R = 1u << lr;
  const uint32_t share = lastrow_cluster_share(lr, b);
  const unsigned rank = cluster.block_rank();
  T* Es = reinterpret_cast<T*>(smem_raw);
  // E_q, q in this CTA's share of [b, R): sum_{t < a} X_{q + tR} omega_a^t
  // as four interleaved Horner chains in omega_a^4 (independent chains keep
  // several loads and products in flight), combined by omega_a^j.
  const T w1 = omega_a_tw;
  const T w2 = F::mul_tw(w1, w1);
  const T w3 = F::mul_tw(w2, w1);
  const T w4 = F::mul_tw(w2, w2);
  const uint64_t groups = (a + 3) / 4;
  for (uint32_t j = threadIdx.x; j < share; j += blockDim.x) {
    const uint64_t q = b + (uint64_t)rank * share + j;
    T e = T(0);
    if (q < R) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (uint64_t g = groups; g-- > 0;) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t t = 4 * g + k;
          const T c = t < a ? X[q + t * R] : T(0);
          acc[k] = F::add(F::mul_tw(acc[k], w4), c);
        }
      }
      e = F::add(F::add(acc[0], F::mul_tw(acc[1], w1)),
                 F::add(F::mul_tw(acc[2], w2), F::mul_tw(acc[3], w3)));
      e = F::canon(e);
    }
    Es[j] = e;
  }
  cluster.sync();  // every share is in its CTA's shared memory
  const size_t head = ((size_t)share * sizeof(T) + 15) & ~(size_t)15;
  T* Z = reinterpret_cast<T*>(smem_raw + head);
  if (rank == 0) {
    // the row's inputs: q < b from the buffer, q >= b from the shares
    for (uint32_t q = threadIdx.x; q < R; q += blockDim.x) {
      if (q < b) {
        Z[q] = X[a * R + q];
      } else {
        const uint32_t i = q - (uint32_t)b;
        Z[q] = *cluster.map_shared_rank(Es + (i % share), i / share);
      }
    }
  }
  cluster.sync();  // the shares have been read; the other CTAs may exit
  if (rank != 0) return;
  T* W = Z + R;
  T* Wih = W + R / 2;
  T* L = Wih + R / 2;
  build_base_tables<F>(W, INV ? Wih : nullptr, lr, s_rt);  // ends in a barrier
  RowTw<F> tw{W, Wih, L, &s_rt, a, lr};
  if (!INV) {
    fwd_pruned<F>(Z, 0, 0, lr, (uint32_t)b, tw);
  } else {
    inv_block<F>(Z, 0, 0, lr, (uint32_t)b, tw);
  }
  for (uint32_t q = threadIdx.x; q < b; q += blockDim.x)
    X[a * R + q] = F::canon(Z[q]);
}

}  // namespace tftgb
