// Kernels of the space-restricted product (Algorithm 3, Section 5): the
// folding step, the pointwise product of a chunk, and the tail block.
//
// Folding.  For a chunk [q, q + L) with L | q, coefficient j < L of
// A(omega_q x) mod (x^L - 1) is sum_t A_{j + tL} omega_q^{j + tL}; a forward
// transform of length L of those L coefficients gives A(omega_q omega_s) =
// A(omega_{q+s}) for s < L (disjoint bits, as in the proof of Proposition
// 5.1).  Twiddles omega_q^e come from the binary powers omega_q^{2^b}
// (kernel parameter).
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

// A CTA of 8 warps folds 32 * 8 / G consecutive coefficients, G = 2^glog
// <= 8 warps per coefficient block: lane l of warp w takes coefficient
// j = j0 + (w / G) * 32 + l and the terms i = j + gL + t G L, t = 0, 1, ...,
// with g = w mod G, so every load reads 32 consecutive words; the G partial
// sums of a coefficient are added through shared memory.  Short chunks
// (small L, many terms per coefficient) thus still fill the GPU.  A lane's
// sum omega_q^{j + gL} sum_t src_i (omega_q^{GL})^t is taken by Horner's
// rule from the last term down (one multiply per term); omega_q^{j + gL} =
// omega_q^{base of the warp} * omega_q^l, the first carried from iteration
// to iteration, the second from a 32-entry table.  blockIdx.y selects the operand:
// (dst0, src0, n0) or (dst1, src1, n1).
template <class F>
__global__ void __launch_bounds__(kFoldThreads)
k_fold(typename F::T* dst0, const typename F::T* src0, uint64_t n0,
       typename F::T* dst1, const typename F::T* src1, uint64_t n1,
       uint64_t L, int ell, int glog, FoldPowers<typename F::T> fp) {
  using T = typename F::T;
  __shared__ T part[kFoldThreads];
  __shared__ T lanepow[32];
  T* dst = blockIdx.y ? dst1 : dst0;
  const T* src = blockIdx.y ? src1 : src0;
  const uint64_t n = blockIdx.y ? n1 : n0;
  const uint32_t G = 1u << glog;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t g = warp & (G - 1u);
  const uint32_t jw = warp >> glog;          // coefficient block in the CTA
  const uint64_t per_cta = (uint64_t)32 * (8u >> glog);
  const T wstep = fp.w[ell + glog];          // omega_q^{L G}
  const uint64_t stride = (uint64_t)G << ell;
  if (threadIdx.x < 32) {
    T v = F::one_tw();
    for (int b = 0; b < 5; ++b)
      if ((threadIdx.x >> b) & 1) v = F::mul_tw(v, fp.w[b]);
    lanepow[threadIdx.x] = v;
  }
  __syncthreads();
  // omega_q^e for the warp's first coefficient block e = j0 + 32 jw + g L
  // and the step omega_q^{gridDim per_cta} between its iterations, each as a
  // product over the exponent's set bits taken across the warp's lanes
  // (lane b contributes omega_q^{2^b} or 1; five shuffle rounds multiply)
  auto warp_pow = [&](uint64_t e) {
    T v = ((e >> lane) & 1) ? fp.w[lane] : F::one_tw();
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
      v = F::mul_tw(v, (T)__shfl_xor_sync(0xffffffffu, v, o));
    return v;  // e < 2^32: lanes 0..31 cover every bit
  };
  T base = warp_pow((uint64_t)blockIdx.x * per_cta + (uint64_t)jw * 32 +
                    ((uint64_t)g << ell));
  const T bstep = warp_pow((uint64_t)gridDim.x * per_cta);
  for (uint64_t j0 = (uint64_t)blockIdx.x * per_cta; j0 < L;
       j0 += (uint64_t)gridDim.x * per_cta, base = F::mul_tw(base, bstep)) {
    const uint64_t jbase = j0 + (uint64_t)jw * 32;
    const uint64_t j = jbase + lane;
    const uint64_t i0 = j + ((uint64_t)g << ell);
    T acc = 0;
    if (j < L && i0 < n) {
      // terms t = nt - 1 down to 0, eight loads in flight at a time
      uint64_t nt = (n - 1 - i0) / stride + 1;
      while (nt >= 8) {
        T v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = src[i0 + (nt - 1 - k) * stride];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = F::add(F::mul_tw(acc, wstep), v[k]);
        nt -= 8;
      }
      for (; nt > 0; --nt)
        acc = F::add(F::mul_tw(acc, wstep), src[i0 + (nt - 1) * stride]);
      acc = F::mul_tw(acc, F::mul_tw(base, lanepow[lane]));
    }
    if (G > 1) {
      part[threadIdx.x] = acc;
      __syncthreads();
      if (g == 0) {
        for (uint32_t k = 1; k < G; ++k)
          acc = F::add(acc, part[threadIdx.x + 32 * k]);
      }
      __syncthreads();
    }
    if (g == 0 && j < L) dst[j] = F::canon(acc);
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
