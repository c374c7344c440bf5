// Register-blocked stages of the network for full power-of-two blocks.
//
// A block of R = 2^lr positions (one row of the row/column split, i.e. block
// rho of the global network) is processed in stages of L <= 4 levels.  In a
// stage covering levels r_lo + L - 1 .. r_lo, a "unit" is the 2^L positions
//     p(u, i) = ((u >> r_lo) << (r_lo + L)) | (i << r_lo) | (u mod 2^r_lo),
// i < 2^L, held in the registers of one thread.  In the remainder view of the
// network (level r reduces modulo x^{2^r} - omega_{2 (y >> (r+1))}, eq. (1)),
// such a unit holds the coefficients of g(z), z = x^{2^r_lo}, that must be
// evaluated at the 2^L points omega_{B 2^L + s'} = omega_{B 2^L} omega_{s'}
// (disjoint bits), where B = y >> (r_lo + L) is the unit's block index.  So a
// stage is: multiply element i by zeta^i with zeta = omega_{B 2^L} (the
// "twist"), then run the constant 2^L-point network whose twiddles
// omega_{2k}, k < 2^{L-1}, are the same for every unit.  B splits into the
// row's part and a local part, zeta = omega_{rho 2^{lr - r_lo}} *
// omega_{B_local 2^L}; the first factor is one value per stage and row, the
// second comes from a small per-CTA table (at most ~R/15 entries).
//
// The inverse stage undoes this up to a factor 2^L: the inverse constant
// network (levels in increasing order, butterfly (X, Y) -> (X + Y,
// omega_{2k}^{-1} (X - Y)), twice Algorithm 2's butterfly) and then the
// untwist by zeta^{-i}.  Every level doubles every entry, so a whole inverse
// of 2^k positions returns 2^k times the input; the factor 2^-k is applied
// once, by a single multiply per entry at the end of the transform (or of a
// block), instead of a halving in every butterfly.
//
// Shared memory holds a block with an XOR swizzle, phys(p) = p ^ ((p >> 4)
// & 15), so that every stage's access pattern (unit-strided or contiguous)
// touches distinct banks per half-warp.
#pragma once
#include "field.cuh"

namespace tftgb {

__device__ __forceinline__ uint32_t swz(uint32_t p) {
  return p ^ ((p >> 4) & 15u);
}

// One element from global to shared memory by an asynchronous copy
// (cp.async, 4 or 8 bytes): the load holds no register and a thread can
// have all of its copies in flight; cp_async_wait_all() waits for the
// thread's own copies (a barrier then publishes them to the CTA).
template <class T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d),
                 "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Stage descriptor: levels [r_lo, r_lo + L).
struct StageDesc {
  int r_lo;
  int L;
  int tl_off;  // offset of this stage's local twist table (2^{lr-r_lo-L})
};

// Stages of a block of 2^lr positions, forward order (highest levels first).
// Rows: the first stage takes lr mod 4 levels (or 4), then stages of 4 down
// to 0.  Columns (balanced): the fewest stages, ceil(c / 4), with the levels
// spread as evenly as possible and the wider stages first -- the first
// stage reads global memory, and a wide one keeps more loads in flight per
// unit, while no stage is left with one or two levels when three fit (a
// narrow stage pays a shared-memory round trip and a unit's overhead for
// few butterflies).
struct StagePlan {
  int n;
  StageDesc s[5];
  int tl_total;
};

__host__ __device__ inline StagePlan make_stage_plan(int lr,
                                                     bool balanced = false) {
  StagePlan sp;
  sp.n = 0;
  const int nst = (lr + 3) / 4;
  int r = lr;
  int off = 0;
  for (int i = 0; r > 0; ++i) {
    int L;
    if (balanced)
      L = lr / nst + (i < lr % nst ? 1 : 0);
    else
      L = i == 0 ? (lr % 4 ? lr % 4 : 4) : 4;
    if (L > r) L = r;
    sp.s[sp.n].r_lo = r - L;
    sp.s[sp.n].L = L;
    sp.s[sp.n].tl_off = off;
    off += 1 << (lr - (r - L) - L);  // entries: 2^{lr - r_lo - L}
    ++sp.n;
    r -= L;
  }
  sp.tl_total = off;
  return sp;
}

// Per-CTA constants of the stage engine, in shared memory.
template <class T>
struct StageConsts {
  T c[8];    // omega_{2k}, k < 8 (twiddle form)
  T cu[8];   // omega_{2k}^{-1} (twiddle form)
  T sc;      // 2^-lr (twiddle form): the row kernels' inverse scale
};

// 2^-j in twiddle form: (1/2)^j by repeated squaring of the twiddle form of
// 1/2 (mul_tw of two twiddle-form values is the twiddle form of their
// product).
template <class F>
__device__ __forceinline__ typename F::T pow2_inv(
    int j, const RootTable<typename F::T>& rt) {
  typename F::T v = rt.one_tw, base = rt.half_tw;
  for (; j; j >>= 1) {
    if (j & 1) v = F::mul_tw(v, base);
    base = F::mul_tw(base, base);
  }
  return v;
}

// The stage constants from the root table (cu[k] = 2 (omega_{2k}^{-1} / 2)).
template <class F>
__device__ __forceinline__ void fill_stage_consts(
    StageConsts<typename F::T>* K, const RootTable<typename F::T>& rt,
    int lr) {
  for (int i = threadIdx.x; i < 8; i += blockDim.x) {
    K->c[i] = rt.c16[i];
    K->cu[i] = F::add(rt.c16i[i], rt.c16i[i]);
  }
  if (threadIdx.x == 0) K->sc = pow2_inv<F>(lr, rt);
}

// Build the local twist tables TL[m] = omega_{m 2^L} and TLi (inverses) for
// every stage: product of omega_[b + L + 1] over the set bits b of m.
template <class F>
__device__ void build_stage_tables(typename F::T* TL, typename F::T* TLi,
                                   const StagePlan& sp, int lr,
                                   const RootTable<typename F::T>& rt) {
  using T = typename F::T;
  for (int si = 0; si < sp.n; ++si) {
    const int L = sp.s[si].L;
    const int cnt = 1 << (lr - sp.s[si].r_lo - L);
    for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
      T v = rt.one_tw, vi = rt.one_tw;
      int bits = m, b = 0;
      while (bits) {
        if (bits & 1) {
          v = F::mul_tw(v, rt.w[b + L + 1]);
          vi = F::mul_tw(vi, rt.winv[b + L + 1]);
        }
        bits >>= 1;
        ++b;
      }
      TL[sp.s[si].tl_off + m] = v;
      TLi[sp.s[si].tl_off + m] = vi;
    }
  }
}

// omega_{rho 2^e} and its inverse: product of omega_[b + e + 1] over the set
// bits b of rho (omega_{2^j} = omega_[j+1]).
template <class F>
__device__ __forceinline__ typename F::T row_factor(
    uint64_t rho, int e, const RootTable<typename F::T>& rt, bool inverse) {
  typename F::T v = rt.one_tw;
  int b = 0;
  while (rho) {
    if (rho & 1) v = F::mul_tw(v, inverse ? rt.winv[b + e + 1] : rt.w[b + e + 1]);
    rho >>= 1;
    ++b;
  }
  return v;
}

// Powers zeta^i, i < 2^L (pw[0] is not used: the twist skips element 0).
template <class F, int L>
__device__ __forceinline__ void powers(typename F::T (&pw)[1 << L],
                                       typename F::T zeta) {
  pw[1] = zeta;
#pragma unroll
  for (int i = 2; i < (1 << L); ++i)
    pw[i] = (i & 1) ? F::mul_tw(pw[i - 1], zeta)
                    : F::mul_tw(pw[i / 2], pw[i / 2]);
}

// The network constant's multiply for a runtime k folded to a compile-time
// one (the networks' loops are unrolled, so k is a constant per butterfly).
template <class F, bool INV>
__device__ __forceinline__ typename F::T net_mul_k(int k, typename F::T w,
                                                   typename F::T c) {
  switch (k) {
    case 1: return F::template net_mul<1, INV>(w, c);
    case 2: return F::template net_mul<2, INV>(w, c);
    case 3: return F::template net_mul<3, INV>(w, c);
    case 4: return F::template net_mul<4, INV>(w, c);
    case 5: return F::template net_mul<5, INV>(w, c);
    case 6: return F::template net_mul<6, INV>(w, c);
    default: return F::template net_mul<7, INV>(w, c);
  }
}

// TOPCOPY: the upper half of the unit's inputs is known to be zero, so the
// top level's butterflies (u, 0) -> (u, u) are copies.  Each butterfly
// brings its second term m (a product, or for k = 0 the entry itself) to
// [0, p) first, so that the sum and the difference need a single carry
// correction (F::add_c, F::sub_c); for the 32-bit fields these are the
// plain operations.  A constant -2^s (F::net_neg) exchanges the sum and
// the difference.
template <class F, int L, bool TOPCOPY = false>
__device__ __forceinline__ void cnet_fwd(typename F::T (&x)[1 << L],
                                         const StageConsts<typename F::T>& K) {
  using T = typename F::T;
#pragma unroll
  for (int d = L - 1; d >= 0; --d) {
#pragma unroll
    for (int i = 0; i < (1 << L); ++i) {
      if (i & (1 << d)) continue;
      if (TOPCOPY && d == L - 1) {
        x[i + (1 << d)] = x[i];
        continue;
      }
      const int k = i >> (d + 1);
      const T w = x[i + (1 << d)];
      const T m =
          F::canon_fast(k == 0 ? w : net_mul_k<F, false>(k, w, K.c[k]));
      const T u = x[i];
      if (k != 0 && F::net_neg(k, false)) {
        x[i] = F::sub_c(u, m);
        x[i + (1 << d)] = F::add_c(u, m);
      } else {
        x[i] = F::add_c(u, m);
        x[i + (1 << d)] = F::sub_c(u, m);
      }
    }
  }
}

// Inverse constant network without the halvings: returns 2^L times the
// inputs of cnet_fwd.  For a constant -2^s the difference is taken the
// other way round, Y - X.
template <class F, int L>
__device__ __forceinline__ void cnet_inv2(typename F::T (&x)[1 << L],
                                          const StageConsts<typename F::T>& K) {
  using T = typename F::T;
#pragma unroll
  for (int d = 0; d < L; ++d) {
#pragma unroll
    for (int i = 0; i < (1 << L); ++i) {
      if (i & (1 << d)) continue;
      const int k = i >> (d + 1);
      const T X = x[i], Y = F::canon_fast(x[i + (1 << d)]);
      x[i] = F::add_c(X, Y);
      if (k == 0) {
        x[i + (1 << d)] = F::sub_c(X, Y);
      } else if (F::net_neg(k, true)) {
        x[i + (1 << d)] = net_mul_k<F, true>(k, F::sub(Y, X), K.cu[k]);
      } else {
        x[i + (1 << d)] = net_mul_k<F, true>(k, F::sub_c(X, Y), K.cu[k]);
      }
    }
  }
}

template <class F, int L>
__device__ __forceinline__ void twist(typename F::T (&x)[1 << L],
                                      typename F::T zeta) {
  typename F::T pw[1 << L];
  powers<F, L>(pw, zeta);
#pragma unroll
  for (int i = 1; i < (1 << L); ++i) x[i] = F::mul_tw(x[i], pw[i]);
}

// Dispatch a runtime stage width L in [1, 4] to a compile-time LL.
#define TFT_STAGE_SWITCH(L, ...)                                \
  switch (L) {                                                  \
    case 1: { constexpr int LL = 1; __VA_ARGS__; } break;       \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break;       \
    case 3: { constexpr int LL = 3; __VA_ARGS__; } break;       \
    default: { constexpr int LL = 4; __VA_ARGS__; } break;      \
  }

// Unit geometry of a stage.
__device__ __forceinline__ uint32_t unit_pos(uint32_t u, int r_lo, int L,
                                             int i) {
  return ((u >> r_lo) << (r_lo + L)) | ((uint32_t)i << r_lo) |
         (u & ((1u << r_lo) - 1));
}

}  // namespace tftgb
