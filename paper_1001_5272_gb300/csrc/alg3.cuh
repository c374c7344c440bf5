// Kernels of the space-restricted product (Algorithm 3, Section 5): the
// folding step, the pointwise product of a chunk, and the tail block.
//
// Folding.  For a chunk [q, q + L) with L | q, coefficient j < L of
// A(omega_q x) mod (x^L - 1) is sum_t A_{j + tL} omega_q^{j + tL}; a forward
// transform of length L of those L coefficients gives A(omega_q omega_s) =
// A(omega_{q+s}) for s < L (disjoint bits, as in the proof of Proposition
// 5.1).  Each thread folds 4 coefficients j, j + 256, ...: omega_q^j from the
// binary powers omega_q^{2^b} (kernel parameter), then one multiply per
// term by omega_q^L = omega_q^{2^ell}.
#pragma once
#include "field.cuh"

namespace tftgb {

// omega_q^{2^b}, b <= 32, in twiddle form (a product of twiddles is a
// twiddle: mul_tw keeps the form).
template <class T>
struct FoldPowers {
  T w[33];
};

constexpr int kFoldThreads = 256;
constexpr int kFoldPerThread = 4;

// blockIdx.y selects the operand: (dst0, src0, n0) or (dst1, src1, n1).
template <class F>
__global__ void __launch_bounds__(kFoldThreads)
k_fold(typename F::T* dst0, const typename F::T* src0, uint64_t n0,
       typename F::T* dst1, const typename F::T* src1, uint64_t n1,
       uint64_t L, int ell, FoldPowers<typename F::T> fp) {
  using T = typename F::T;
  T* dst = blockIdx.y ? dst1 : dst0;
  const T* src = blockIdx.y ? src1 : src0;
  const uint64_t n = blockIdx.y ? n1 : n0;
  const T wL = fp.w[ell];
  const T wstep = fp.w[8];  // omega_q^256 between a thread's coefficients
  const uint64_t span = (uint64_t)kFoldThreads * kFoldPerThread;
  for (uint64_t base = (uint64_t)blockIdx.x * span; base < L;
       base += (uint64_t)gridDim.x * span) {
    const uint64_t j0 = base + threadIdx.x;
    // omega_q^{j0} from the binary powers
    T w = F::one_tw();
    {
      uint64_t bits = j0;
      int b = 0;
      while (bits) {
        if (bits & 1) w = F::mul_tw(w, fp.w[b]);
        bits >>= 1;
        ++b;
      }
    }
#pragma unroll
    for (int k = 0; k < kFoldPerThread; ++k) {
      const uint64_t j = j0 + (uint64_t)k * kFoldThreads;
      if (j < L) {
        T acc = 0;
        T wt = w;
        for (uint64_t i = j; i < n; i += L) {
          acc = F::add(acc, F::mul_tw(src[i], wt));
          wt = F::mul_tw(wt, wL);
        }
        dst[j] = F::canon(acc);
      }
      w = F::mul_tw(w, wstep);
    }
  }
}

// X[i] = X[i] * Y[i], i < L (a chunk's pointwise product, C^ = A^ B^).
template <class F>
__global__ void __launch_bounds__(256)
k_chunk_mul(typename F::T* X, const typename F::T* Y, uint64_t L) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L;
       i += (uint64_t)gridDim.x * blockDim.x)
    X[i] = F::canon(F::mul_data(X[i], Y[i]));
}

// Tail block [Q, Q + M): for positions s in [lo, hi) set X_s = S_{s-Q}
// (mul = 0) or X_s = X_s * S_{s-Q} (mul = 1).
template <class F>
__global__ void __launch_bounds__(256)
k_tail(typename F::T* X, const typename F::T* S, uint64_t Q, uint64_t lo,
       uint64_t hi, int mul) {
  for (uint64_t s = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
       s < hi; s += (uint64_t)gridDim.x * blockDim.x) {
    const typename F::T v = S[s - Q];
    X[s] = mul ? F::canon(F::mul_data(X[s], v)) : v;
  }
}

}  // namespace tftgb
