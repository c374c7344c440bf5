// Field arithmetic for the three NTT primes (device side).
//
// The paper works over any ring R in which 2 is not a zero-divisor and that
// has the 2^k-th roots of unity it needs (Section 2.1).  The library
// instantiates R = Z/p for
//   p = 998244353        = 119 * 2^23 + 1   (uint32 storage, Montgomery form)
//   p = 2013265921       =  15 * 2^27 + 1   (uint32 storage, Montgomery form)
//   p = 2^64 - 2^32 + 1                      (uint64 storage, direct reduction)
//
// Data elements in global memory are always canonical residues in [0, p)
// (inside a transform the 64-bit field keeps values in [0, 2^64), see
// Goldilocks; F::canon is applied at every store).  Twiddles are kept
// in a per-field "twiddle form" that makes mul_tw(x, w) return x * w mod p:
//   * 32-bit primes: w~ = w * 2^32 mod p and mul_tw is one Montgomery REDC of
//     the 64-bit product (x * w~ * 2^-32 = x * w), canonical;
//   * 2^64 - 2^32 + 1: w~ = w and mul_tw reduces the 128-bit product using
//     2^64 = 2^32 - 1 and 2^96 = -1 (mod p), into [0, 2^64).
#pragma once
#include <stdint.h>

#ifndef TFT_HD
#define TFT_HD __host__ __device__ __forceinline__
#endif

namespace tftgb {

// ---------------------------------------------------------------------------
// p = 2^64 - 2^32 + 1
// ---------------------------------------------------------------------------
struct Goldilocks {
  using T = uint64_t;
  static constexpr uint64_t P = 0xFFFFFFFF00000001ull;
  static constexpr uint64_t EPS = 0xFFFFFFFFull;  // 2^64 mod p
  static constexpr uint64_t HALF = 0x7FFFFFFF80000001ull;  // (p + 1) / 2
  static constexpr int K = 32;                     // two-adicity
  static constexpr int ID = 2;

  // Values inside a transform are kept in [0, 2^64) ("lazy": congruent to
  // the residue, not necessarily below p); canon() maps them to [0, p) and
  // every store to global memory goes through it.  The carry chains below
  // use 2^64 = EPS (mod p): a carry out of bit 63 is worth EPS, a borrow
  // costs EPS.

  // a + b for any a, b < 2^64.  After one carry the wrapped sum is at most
  // 2^64 - 2, and adding EPS can carry again only if it was >= p; the
  // second wrapped value is then below 2^32, so a third carry cannot occur.
  static __device__ __forceinline__ T add(T a, T b) {
    uint32_t s0, s1, m;
    asm("add.cc.u32 %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32 %2, 0, 0;\n\t"
        "sub.u32 %2, 0, %2;\n\t"
        "add.cc.u32 %0, %0, %2;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.u32 %2, 0, 0;\n\t"
        "sub.u32 %2, 0, %2;\n\t"
        "add.cc.u32 %0, %0, %2;\n\t"
        "addc.u32 %1, %1, 0;"
        : "=&r"(s0), "=&r"(s1), "=&r"(m)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b),
          "r"((uint32_t)(b >> 32)));
    return ((uint64_t)s1 << 32) | s0;
  }
  // a - b for any a, b < 2^64 (a borrow is repaid by subtracting EPS; a
  // second borrow, possible only when b >= p, leaves a value near 2^64, so
  // the second repayment cannot borrow).
  static __device__ __forceinline__ T sub(T a, T b) {
    uint32_t d0, d1, m;
    asm("sub.cc.u32 %0, %3, %5;\n\t"
        "subc.cc.u32 %1, %4, %6;\n\t"
        "subc.u32 %2, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, %2;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 %2, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, %2;\n\t"
        "subc.u32 %1, %1, 0;"
        : "=&r"(d0), "=&r"(d1), "=&r"(m)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b),
          "r"((uint32_t)(b >> 32)));
    return ((uint64_t)d1 << 32) | d0;
  }
  // x = lo + 2^64 (hl + 2^32 hh)  ==  lo - hh + (2^32 - 1) hl  (mod p), for
  // any 128-bit x; result in [0, 2^64).  t = lo - hh (a borrow costs EPS;
  // t stays positive because lo - hh > -2^32), then t + (2^32 - 1) hl on the
  // multiply-add pipe (mad.lo.cc / madc.hi.cc, which keeps the ALU pipe,
  // the busier one in the butterflies, free for the carry chains) with one
  // carry worth EPS (t + (2^32 - 1) hl - 2^64 < 2^64 - 2^33, so adding EPS
  // cannot carry).
  static __device__ __forceinline__ T reduce128(uint64_t lo, uint64_t hi) {
    uint32_t t0, t1, m, c;
    asm("sub.cc.u32 %0, %4, %7;\n\t"
        "subc.cc.u32 %1, %5, 0;\n\t"
        "subc.u32 %2, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, %2;\n\t"
        "subc.u32 %1, %1, 0;\n\t"
        "mad.lo.cc.u32 %0, %6, 0xffffffff, %0;\n\t"
        "madc.hi.cc.u32 %1, %6, 0xffffffff, %1;\n\t"
        "addc.u32 %3, 0, 0;\n\t"
        "sub.u32 %3, 0, %3;\n\t"
        "add.cc.u32 %0, %0, %3;\n\t"
        "addc.u32 %1, %1, 0;"
        : "=&r"(t0), "=&r"(t1), "=&r"(m), "=&r"(c)
        : "r"((uint32_t)lo), "r"((uint32_t)(lo >> 32)), "r"((uint32_t)hi),
          "r"((uint32_t)(hi >> 32)));
    return ((uint64_t)t1 << 32) | t0;
  }
  // [0, 2^64) -> [0, p): x >= p exactly when the high word is 2^32 - 1 and
  // the low word is not 0, and then x - p has high word 0 and low word
  // x0 - 1 (two predicated instructions instead of a 64-bit compare and
  // subtract).
  static __device__ __forceinline__ T canon_fast(T x) {
    uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    asm("{\n\t.reg .pred q;\n\t"
        "setp.eq.u32 q, %1, 0xffffffff;\n\t"
        "setp.ne.and.u32 q, %0, 0, q;\n\t"
        "@q sub.u32 %0, %0, 1;\n\t"
        "@q mov.u32 %1, 0;\n\t}"
        : "+r"(x0), "+r"(x1));
    return ((uint64_t)x1 << 32) | x0;
  }
  // a + b for a < 2^64 and b < p: a + b < 2^64 + p, so after a carry the
  // wrapped sum is below p and adding EPS cannot carry again.
  static __device__ __forceinline__ T add_c(T a, T b) {
    uint32_t s0, s1, m;
    asm("add.cc.u32 %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32 %2, 0, 0;\n\t"
        "sub.u32 %2, 0, %2;\n\t"
        "add.cc.u32 %0, %0, %2;\n\t"
        "addc.u32 %1, %1, 0;"
        : "=&r"(s0), "=&r"(s1), "=&r"(m)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b),
          "r"((uint32_t)(b >> 32)));
    return ((uint64_t)s1 << 32) | s0;
  }
  // a - b for a < 2^64 and b < p: after a borrow the wrapped difference is
  // above 2^64 - p = EPS, so subtracting EPS cannot borrow again.
  static __device__ __forceinline__ T sub_c(T a, T b) {
    uint32_t d0, d1, m;
    asm("sub.cc.u32 %0, %3, %5;\n\t"
        "subc.cc.u32 %1, %4, %6;\n\t"
        "subc.u32 %2, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, %2;\n\t"
        "subc.u32 %1, %1, 0;"
        : "=&r"(d0), "=&r"(d1), "=&r"(m)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b),
          "r"((uint32_t)(b >> 32)));
    return ((uint64_t)d1 << 32) | d0;
  }
  // The 128-bit product by 32-bit limbs, schoolbook, with the partial
  // products' sums folded into multiply-add carry chains (four low and four
  // high 32 x 32 products, one carry add), then reduce128.  Measured on the
  // calibration kernel against the 64-bit mul.lo / mul.hi pair: 35.3 instead
  // of 40.6 multiply-pipe cycles and 20.4 instead of 23.3 instructions per
  // warp-wide modular multiply.
  static __device__ __forceinline__ T mul(T a, T b) {
    uint32_t r0, r1, r2, r3;
    asm("mul.lo.u32 %0, %4, %6;\n\t"
        "mul.hi.u32 %1, %4, %6;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.u32 %2, %4, %7, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, 0, 0;\n\t"
        "mad.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, %3;"
        : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b),
          "r"((uint32_t)(b >> 32)));
    return reduce128(((uint64_t)r1 << 32) | r0, ((uint64_t)r3 << 32) | r2);
  }
  static __device__ __forceinline__ T mul_tw(T a, T w) { return mul(a, w); }
  // x 2^S for 0 < S < 64: the 128-bit product is (x << S, x >> (64 - S)),
  // reduced without a multiplication.
  template <int S>
  static __device__ __forceinline__ T mul_pow2(T x) {
    return reduce128(x << S, x >> (64 - S));
  }
  // The constants of the 16-point network, omega_{2k} for k < 8, are powers
  // of 2 under the library's root convention (omega_[32] = 7^((p-1)/2^32)):
  // omega_{2k} = 2^{e_k}, e = 0, 48, 120, 168, 156, 12, 84, 132 (mod 192,
  // 2^96 = -1), i.e. +-2^s with s < 96; so are their inverses.  Where
  // s < 64 the network multiplies by a shift and a reduction (no 64 x 64
  // product, which would load the multiply pipe); kNet*Shift = 0 means the
  // ordinary multiply by the table's constant, and kNet*Neg that the
  // constant is -2^s, so the caller exchanges the sum and the difference.
  // (The host checks these against the root table, check_constants.)
  static constexpr int kNetShift[8] = {0, 48, 24, 0, 60, 12, 0, 36};
  static constexpr int kNetInvShift[8] = {0, 48, 0, 24, 36, 0, 12, 60};
  static constexpr unsigned kNetNegMask = 0x94;     // k = 2, 4, 7: -2^s
  static constexpr unsigned kNetInvNegMask = 0x42;  // k = 1, 6
  template <int Kk, bool INV>
  static __device__ __forceinline__ T net_mul(T w, T c) {
    constexpr int sh = INV ? kNetInvShift[Kk] : kNetShift[Kk];
    if constexpr (sh > 0)
      return mul_pow2<sh>(w);
    else
      return mul(w, c);
  }
  static __host__ __device__ constexpr bool net_neg(int k, bool inv) {
    return (((inv ? kNetInvNegMask : kNetNegMask) >> k) & 1u) != 0;
  }
  static __device__ __forceinline__ T mul_data(T a, T b) { return mul(a, b); }
  // a / 2 for any a < 2^64: (a - 1) / 2 + (p + 1) / 2 = (a + p) / 2 < 2^64
  // when a is odd.
  static TFT_HD T half(T a) { return (a >> 1) + ((a & 1) ? HALF : 0); }
  static TFT_HD T canon(T a) { return a >= P ? a - P : a; }
  static TFT_HD T one_tw() { return 1; }
};

// Goldilocks with the product as the 64-bit mul.lo / mul.hi pair: the
// arithmetic of the scratch-free inverse's cluster kernel (Horner chains
// and the row's generalized inverse in one CTA), which measured 0.34 ms
// slower with the carry-chain product above (its forward measured faster
// with it and keeps it).
struct GoldilocksWide : Goldilocks {
  static __device__ __forceinline__ T mul(T a, T b) {
    return reduce128(a * b, __umul64hi(a, b));
  }
  static __device__ __forceinline__ T mul_tw(T a, T w) { return mul(a, w); }
  static __device__ __forceinline__ T mul_data(T a, T b) { return mul(a, b); }
};

// The field type the scratch-free inverse's cluster kernel is instantiated
// with.
template <class F>
struct ClusterField {
  using type = F;
};
template <>
struct ClusterField<Goldilocks> {
  using type = GoldilocksWide;
};

// ---------------------------------------------------------------------------
// 32-bit primes in Montgomery form with R = 2^32.
//   PINV = -p^{-1} mod 2^32, R2 = 2^64 mod p, ONE = 2^32 mod p.
// ---------------------------------------------------------------------------
template <uint32_t P_, uint32_t PINV_, uint32_t R2_, uint32_t ONE_, int K_,
          int ID_>
struct Mont32 {
  using T = uint32_t;
  static constexpr uint32_t P = P_;
  static constexpr uint32_t PINV = PINV_;
  static constexpr uint32_t R2 = R2_;
  static constexpr uint32_t ONE = ONE_;
  static constexpr int K = K_;
  static constexpr int ID = ID_;

  static TFT_HD T add(T a, T b) {
    T s = a + b;  // < 2p < 2^32
    return s >= P ? s - P : s;
  }
  static TFT_HD T sub(T a, T b) { return a >= b ? a - b : a - b + P; }
  // t < p * 2^32  ->  t * 2^-32 mod p, canonical
  static TFT_HD T redc(uint64_t t) {
    const uint32_t m = (uint32_t)t * PINV;
    const uint64_t u = (t + (uint64_t)m * P) >> 32;  // < 2p, no overflow
    return (T)(u >= P ? u - P : u);
  }
  static TFT_HD T mul_tw(T a, T w) { return redc((uint64_t)a * w); }
  static TFT_HD T mul_data(T a, T b) {
    return redc((uint64_t)redc((uint64_t)a * b) * R2);
  }
  static TFT_HD T half(T a) { return (a + ((a & 1) ? P : 0)) >> 1; }
  static TFT_HD T canon(T a) { return a; }  // always canonical
  // the butterfly forms of Goldilocks (canonical second operand): values
  // here are always canonical, so they are the plain operations
  static TFT_HD T canon_fast(T a) { return a; }
  static TFT_HD T add_c(T a, T b) { return add(a, b); }
  static TFT_HD T sub_c(T a, T b) { return sub(a, b); }
  // the 16-point network multiplies by the table's constants here
  template <int Kk, bool INV>
  static __device__ __forceinline__ T net_mul(T w, T c) {
    return mul_tw(w, c);
  }
  static __host__ __device__ constexpr bool net_neg(int, bool) {
    return false;
  }
  static TFT_HD T one_tw() { return ONE; }
};

// -p^{-1} mod 2^32, 2^64 mod p and 2^32 mod p for the two 32-bit primes
// (checked on the host at context creation).
using P998 = Mont32<998244353u, 998244351u, 932051910u, 301989884u, 23, 0>;
using P2013 = Mont32<2013265921u, 2013265919u, 1172168163u, 268435454u, 27, 1>;

// Root table passed by value to every kernel: omega_[j] (Section 2.2) in
// twiddle form, and omega_[j]^{-1} / 2 in twiddle form, for j <= K.
template <class T>
struct RootTable {
  T w[33];       // omega_[j]
  T winv[33];    // omega_[j]^{-1}
  T half_tw;     // 1/2 in twiddle form
  T one_tw;      // 1 in twiddle form
  T c16[8];      // omega_{2k}, k < 8: the twiddles of a 16-point network
  T c16i[8];     // omega_{2k}^{-1} / 2
};

}  // namespace tftgb
