// Shared-memory transform engine: the radix-2 network of Algorithm 1 run
// level by level over a tile held in shared memory.
//
// The network.  For a buffer Z of length 2^l and level r = l-1, ..., 0, the
// pair (y, y + 2^r) with bit r of y clear is replaced by
//     (Z_y + theta Z_{y+2^r},  Z_y - theta Z_{y+2^r}),  theta = omega_{2 (y >> (r+1))}.
// In Algorithm 1 the node S = (q, r) pairs S_{2j} = X_{q + 2j 2^r} with
// S_{2j+1} = X_{q + (2j+1) 2^r} under theta = omega_{2j} (eq. (1)); with
// y = q + 2j 2^r and q < 2^r we get j = y >> (r+1), so the loop above performs
// exactly those butterflies, node by node, level by level.  Run on x padded
// with zeros to 2^l it yields F(omega_s) at position s (Section 2.2), i.e. the
// first n outputs are the TFT of length n (the TFT is the truncation of the
// length-2^l transform, Section 1.2).  Shared memory is the work area of one
// CTA; the global buffer is never padded.
//
// A tile holds C = 2^clog interleaved columns, element (t, c) at
// Z[(t << slog) + c] with slog >= clog; all columns run the same control
// flow.
//
// Three routines:
//   fwd_pruned   the network restricted to the butterflies that feed outputs
//                < n_out: at level r only rows t < ceil(n_out / 2^{r+1}) 2^{r+1}.
//   inv_full     the exact inverse of the full network (levels 0 .. l-1):
//                (X, Y) -> ((X + Y) / 2, theta^{-1} (X - Y) / 2), the
//                butterfly of Algorithm 2 (Section 4).
//   inv_block    the inverse when only the first m outputs are known and the
//                inputs at rows >= m are known (zero for a plain ITFT).  The
//                top level of a block [B, B + 2^l) splits it into halves; if
//                m >= 2^{l-1} the lower half's outputs are all known and are
//                inverted in full, the upper half's known inputs are rewritten
//                as inputs of the upper sub-network, and the problem recurses
//                on the upper half; otherwise the lower half's inputs at rows
//                >= m are formed from known values and the problem recurses on
//                the lower half.  Unwinding applies the top-level inverse.
//                Flattened: phase A inverts, all at once, the dyadic blocks of
//                m (the full lower halves); then a descent and an ascent of
//                one level each.  This plays the role of Algorithm 2's
//                odd-length corrections: it recovers the coefficients from
//                exactly the n known transform values.
#pragma once
#include "field.cuh"

namespace tftgb {

// Twiddle source for a standalone transform (a column, or a small transform):
// theta(r, j) = omega_{2j} = W[j], theta^{-1}/2 = Wih[j].
template <class F>
struct ColTw {
  using T = typename F::T;
  // no per-level table: consecutive levels that stay inside one warp's rows
  // need only a warp barrier between them
  static constexpr bool kWarpSync = true;
  const T* W;
  const T* Wih;
  __device__ __forceinline__ void prep_fwd(int, uint32_t) const {}
  __device__ __forceinline__ void prep_inv(int, uint32_t) const {}
  __device__ __forceinline__ T fwd(int, uint32_t j) const { return W[j]; }
  __device__ __forceinline__ T invh(int, uint32_t j) const { return Wih[j]; }
  __device__ __forceinline__ T fwd_direct(int, uint32_t j) const { return W[j]; }
  __device__ __forceinline__ T invh_direct(int, uint32_t j) const {
    return Wih[j];
  }
};

// Twiddle source for block rho (of size 2^lr) of a longer network: positions
// y = rho 2^lr + y' so theta(r, j') = omega_{2((rho 2^lr + y') >> (r+1))}
//   = omega_{rho 2^{lr-r}} * omega_{2 j'}     (disjoint bits, Section 5's
//                                             omega_q omega_i = omega_{q+i})
// The row factor u_r = omega_{rho 2^{lr-r}} is the product of omega_[b+lr-r+1]
// over the set bits b of rho (omega_{2^e} = omega_[e+1]).  prep_* builds the
// level's table L[j'] = u_r W[j'] (or u_r^{-1} Wih[j']) in shared memory.
template <class F>
struct RowTw {
  using T = typename F::T;
  static constexpr bool kWarpSync = false;  // prep_* rebuilds L per level
  const T* W;
  const T* Wih;
  T* L;                 // shared scratch of 2^{lr-1} entries
  const RootTable<T>* rt;
  uint64_t rho;
  int lr;

  __device__ __forceinline__ T ufwd(int r) const {
    T u = rt->one_tw;
    uint64_t bits = rho;
    int b = 0;
    while (bits) {
      if (bits & 1) u = F::mul_tw(u, rt->w[b + lr - r + 1]);
      bits >>= 1;
      ++b;
    }
    return u;
  }
  __device__ __forceinline__ T uinv(int r) const {
    T u = rt->one_tw;
    uint64_t bits = rho;
    int b = 0;
    while (bits) {
      if (bits & 1) u = F::mul_tw(u, rt->winv[b + lr - r + 1]);
      bits >>= 1;
      ++b;
    }
    return u;
  }
  // Twiddle-form product of two twiddle-form values.  For Montgomery fields
  // mul_tw(a~, b~) = a b 2^32 = (a b)~; for Goldilocks the form is canonical.
  __device__ __forceinline__ void prep_fwd(int r, uint32_t count) const {
    __syncthreads();  // previous readers of L are done
    if (rho == 0) {
      for (uint32_t j = threadIdx.x; j < count; j += blockDim.x) L[j] = W[j];
    } else {
      const T u = ufwd(r);
      for (uint32_t j = threadIdx.x; j < count; j += blockDim.x)
        L[j] = F::mul_tw(u, W[j]);
    }
    __syncthreads();
  }
  __device__ __forceinline__ void prep_inv(int r, uint32_t count) const {
    __syncthreads();
    if (rho == 0) {
      for (uint32_t j = threadIdx.x; j < count; j += blockDim.x) L[j] = Wih[j];
    } else {
      const T u = uinv(r);
      for (uint32_t j = threadIdx.x; j < count; j += blockDim.x)
        L[j] = F::mul_tw(u, Wih[j]);
    }
    __syncthreads();
  }
  __device__ __forceinline__ T fwd(int, uint32_t j) const { return L[j]; }
  __device__ __forceinline__ T invh(int, uint32_t j) const { return L[j]; }
  __device__ __forceinline__ T fwd_direct(int r, uint32_t j) const {
    return rho == 0 ? W[j] : F::mul_tw(ufwd(r), W[j]);
  }
  __device__ __forceinline__ T invh_direct(int r, uint32_t j) const {
    return rho == 0 ? Wih[j] : F::mul_tw(uinv(r), Wih[j]);
  }
};

// Build W[j] = omega_{2j} and Wih[j] = omega_{2j}^{-1} / 2 for j < 2^{l-1}
// (twiddle form) by doubling: omega_{2(j + 2^e)} = omega_{2j} omega_[e+2]
// for j < 2^e.  Ends with a barrier.
template <class F>
__device__ void build_base_tables(typename F::T* W, typename F::T* Wih, int l,
                                  const RootTable<typename F::T>& rt) {
  using T = typename F::T;
  if (l < 1) {
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    W[0] = rt.one_tw;
    if (Wih) Wih[0] = rt.half_tw;
  }
  __syncthreads();
  for (int e = 0; e + 1 < l; ++e) {
    const uint32_t half = 1u << e;
    const T step = rt.w[e + 2];
    const T stepi = rt.winv[e + 2];
    for (uint32_t j = threadIdx.x; j < half; j += blockDim.x) {
      W[j + half] = F::mul_tw(W[j], step);
      if (Wih) Wih[j + half] = F::mul_tw(Wih[j], stepi);
    }
    __syncthreads();
  }
}

template <class F, class Tw>
__device__ void fwd_pruned(typename F::T* Z, int clog, int slog, int l,
                           uint32_t n_out, const Tw& tw) {
  using T = typename F::T;
  const uint32_t C = 1u << clog;
  for (int r = l - 1; r >= 0; --r) {
    const uint32_t blk = 1u << (r + 1);
    uint32_t lim = ((n_out + blk - 1) >> (r + 1)) << (r + 1);
    if (lim > (1u << l)) lim = 1u << l;
    tw.prep_fwd(r, lim >> (r + 1));
    const uint32_t npairs = (lim >> 1) << clog;
    const uint32_t mask = (1u << r) - 1;
    for (uint32_t pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
      const uint32_t c = pi & (C - 1);
      const uint32_t tp = pi >> clog;
      const uint32_t t = ((tp >> r) << (r + 1)) | (tp & mask);
      const T th = tw.fwd(r, t >> (r + 1));
      T* pu = Z + ((size_t)t << slog) + c;
      T* pw = pu + ((size_t)1 << (r + slog));
      const T u = *pu;
      const T m = F::mul_tw(*pw, th);
      *pu = F::add(u, m);
      *pw = F::sub(u, m);
    }
    // A warp's pairs pi in [32 w, 32 w + 32) (+ multiples of the block)
    // cover rows [64 w, 64 w + 64) >> clog of every column at each level r
    // with 2^r <= 32 >> clog, so levels r and r - 1 then exchange data only
    // inside the warp.
    if (Tw::kWarpSync && r >= 1 && r <= 5 - clog)
      __syncwarp();
    else
      __syncthreads();
  }
}

// Inverse butterflies of levels 0 .. top-1 on rows [0, lim_r) where lim_r is
// given per level by the functor; used by inv_full (lim = 2^l) and phase A.
// wsync: the next level (r + 1) stays inside each warp's rows (see
// fwd_pruned), so a warp barrier ends this one.
template <class F, class Tw>
__device__ __forceinline__ void inv_level(typename F::T* Z, int clog, int slog,
                                          int r, uint32_t lim, const Tw& tw,
                                          bool wsync = false) {
  using T = typename F::T;
  const uint32_t C = 1u << clog;
  tw.prep_inv(r, lim >> (r + 1));
  const uint32_t npairs = (lim >> 1) << clog;
  const uint32_t mask = (1u << r) - 1;
  for (uint32_t pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
    const uint32_t c = pi & (C - 1);
    const uint32_t tp = pi >> clog;
    const uint32_t t = ((tp >> r) << (r + 1)) | (tp & mask);
    const T th = tw.invh(r, t >> (r + 1));
    T* pu = Z + ((size_t)t << slog) + c;
    T* pw = pu + ((size_t)1 << (r + slog));
    const T X = *pu, Y = *pw;
    *pu = F::half(F::add(X, Y));
    *pw = F::mul_tw(F::sub(X, Y), th);
  }
  if (wsync)
    __syncwarp();
  else
    __syncthreads();
}

template <class F, class Tw>
__device__ void inv_full(typename F::T* Z, int clog, int slog, int l,
                         const Tw& tw) {
  for (int r = 0; r < l; ++r)
    inv_level<F>(Z, clog, slog, r, 1u << l, tw,
                 Tw::kWarpSync && r + 1 < l && r + 1 <= 5 - clog);
}

// Levels 1..5 of inv_block's descent and ascent for one column (clog = 0):
// below level 6 both stay inside the 32-row block of m0 (rows base + lane,
// base = m0 rounded down to a multiple of 32), so warp 0 runs them with one
// row per lane and level l pairing lanes lane and lane ^ 2^(l-1) by
// shuffles, with no barrier between levels; the operations are those of
// inv_block's own levels.  Returns nothing; the caller's barrier follows.
template <class F, class Tw>
__device__ __forceinline__ void inv_block_low_warp(typename F::T* Z, int slog,
                                                   uint32_t m0, const Tw& tw) {
  using T = typename F::T;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t base = m0 & ~31u;
  T* z = Z + ((size_t)(base + lane) << slog);
  T x = *z;
  int lstop = 0;
#pragma unroll 1
  for (int l = 5; l >= 1; --l) {
    const uint32_t low = m0 & ((1u << l) - 1);
    if (low == 0) {
      lstop = l;
      break;
    }
    const uint32_t B = m0 & ~((1u << l) - 1);
    const uint32_t h = 1u << (l - 1);
    const T th = tw.fwd_direct(l - 1, B >> l);
    const bool upc = low >= h;
    const uint32_t j0 = upc ? low - h : low;
    const T y = __shfl_xor_sync(0xffffffffu, x, h);
    const bool in = (lane & ~((1u << l) - 1)) == B - base &&
                    (lane & (h - 1)) >= j0;
    const bool upper = (lane & h) != 0;
    if (in && upc && upper) {
      const T t = F::mul_tw(x, th);
      x = F::sub(F::sub(y, t), t);
    } else if (in && !upc && !upper) {
      x = F::add(x, F::mul_tw(y, th));
    }
  }
#pragma unroll 1
  for (int l = lstop + 1; l <= 5; ++l) {
    const uint32_t low = m0 & ((1u << l) - 1);
    const uint32_t B = m0 & ~((1u << l) - 1);
    const uint32_t h = 1u << (l - 1);
    const bool up = low >= h;
    const T th = up ? tw.invh_direct(l - 1, B >> l) : tw.fwd_direct(l - 1, B >> l);
    const T y = __shfl_xor_sync(0xffffffffu, x, h);
    const bool in = (lane & ~((1u << l) - 1)) == B - base;
    const bool upper = (lane & h) != 0;
    if (in && up) {
      x = upper ? F::mul_tw(F::sub(y, x), th) : F::half(F::add(x, y));
    } else if (in && !upper) {
      x = F::sub(x, F::mul_tw(y, th));
    }
  }
  *z = x;
}

// Generalized inverse on the padded block of 2^l0 rows: rows < m0 hold known
// outputs, rows >= m0 hold known inputs.  On return every row < 2^l0 holds
// the network's input.
template <class F, class Tw>
__device__ void inv_block(typename F::T* Z, int clog, int slog, int l0,
                          uint32_t m0, const Tw& tw) {
  using T = typename F::T;
  const uint32_t C = 1u << clog;
  if (m0 == 0) return;
  if (m0 == (1u << l0)) {
    inv_full<F>(Z, clog, slog, l0, tw);
    return;
  }
  // Phase A: the full lower halves met on the way down are the dyadic blocks
  // of m0; at level r they cover rows [0, floor(m0 / 2^{r+1}) 2^{r+1}).
  for (int r = 0; r < l0; ++r) {
    const uint32_t lim = (m0 >> (r + 1)) << (r + 1);
    if (lim == 0) break;  // lim is non-increasing in r
    const bool next = r + 1 < l0 && (m0 >> (r + 2)) != 0;
    inv_level<F>(Z, clog, slog, r, lim, tw,
                 Tw::kWarpSync && next && r + 1 <= 5 - clog);
  }
  // Descent: levels l = l0 .. 1 while m0 mod 2^l != 0.  The block at level
  // l starts at row B = m0 with its low l bits cleared; m = m0 mod 2^l.
  // With one column, levels 1..5 go to inv_block_low_warp.
  const int wl = (clog == 0 && l0 >= 5) ? 5 : 0;
  int lstop = 0;
  bool stopped = false;
  for (int l = l0; l > wl; --l) {
    const uint32_t low = m0 & ((1u << l) - 1);
    if (low == 0) {
      lstop = l;
      stopped = true;
      break;
    }
    const uint32_t B = m0 & ~((1u << l) - 1);
    const uint32_t h = 1u << (l - 1);
    const T th = tw.fwd_direct(l - 1, B >> l);
    if (low >= h) {
      // upper inputs: Q_j = P_j - 2 theta in_{h+j} for j in [low - h, h)
      const uint32_t j0 = low - h;
      const uint32_t cnt = (h - j0) << clog;
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t c = i & (C - 1);
        const uint32_t j = j0 + (i >> clog);
        T* pl = Z + ((size_t)(B + j) << slog) + c;
        T* pu = Z + ((size_t)(B + h + j) << slog) + c;
        const T t = F::mul_tw(*pu, th);
        *pu = F::sub(F::sub(*pl, t), t);
      }
    } else {
      // lower inputs: P_j = in_j + theta in_{h+j} for j in [low, h)
      const uint32_t cnt = (h - low) << clog;
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t c = i & (C - 1);
        const uint32_t j = low + (i >> clog);
        T* pl = Z + ((size_t)(B + j) << slog) + c;
        T* pu = Z + ((size_t)(B + h + j) << slog) + c;
        *pl = F::add(*pl, F::mul_tw(*pu, th));
      }
    }
    __syncthreads();
  }
  if (!stopped && wl > 0) {
    if (m0 & 31u) {
      if (threadIdx.x < 32) inv_block_low_warp<F>(Z, slog, m0, tw);
      __syncthreads();
    }
    lstop = wl;
  }
  // Ascent: the same levels bottom-up.
  for (int l = lstop + 1; l <= l0; ++l) {
    const uint32_t low = m0 & ((1u << l) - 1);
    const uint32_t B = m0 & ~((1u << l) - 1);
    const uint32_t h = 1u << (l - 1);
    const uint32_t cnt = h << clog;
    if (low >= h) {
      const T thi = tw.invh_direct(l - 1, B >> l);
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t c = i & (C - 1);
        const uint32_t j = i >> clog;
        T* pl = Z + ((size_t)(B + j) << slog) + c;
        T* pu = Z + ((size_t)(B + h + j) << slog) + c;
        const T X = *pl, Y = *pu;
        *pl = F::half(F::add(X, Y));
        *pu = F::mul_tw(F::sub(X, Y), thi);
      }
    } else {
      const T th = tw.fwd_direct(l - 1, B >> l);
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t c = i & (C - 1);
        const uint32_t j = i >> clog;
        T* pl = Z + ((size_t)(B + j) << slog) + c;
        T* pu = Z + ((size_t)(B + h + j) << slog) + c;
        *pl = F::sub(*pl, F::mul_tw(*pu, th));
      }
    }
    __syncthreads();
  }
}

}  // namespace tftgb
