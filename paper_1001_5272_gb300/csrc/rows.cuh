// Row kernels on the register-blocked stage engine (stages.cuh).
//
// A row rho < a is block rho (2^LR positions) of the global network, so its
// LR levels are run as stages with the twist zeta = omega_{rho 2^{LR-r_lo}} *
// omega_{B_local 2^L}.  Each row is handled by R/16 threads holding 16
// elements each; a CTA holds G = blockDim / (R/16) rows at a time.  The
// kernels are persistent over rows and specialized on LR: the first stage
// takes L0 = LR mod 4 levels (4 if that is 0), the others 4.
#pragma once
#include "stages.cuh"

// Resident CTAs per SM asked of the 256-thread row kernels, per element
// width (the register cap follows: 3 -> 80, 4 -> 64 registers per thread;
// measured best on GB300 for the 64-bit and 32-bit fields respectively).
#ifndef TFT_ROW_MIN_CTAS_64
#define TFT_ROW_MIN_CTAS_64 3
#endif
#ifndef TFT_ROW_MIN_CTAS_32
#define TFT_ROW_MIN_CTAS_32 4
#endif

namespace tftgb {

// Row geometry: TPR threads per row, each holding EPT = R / TPR elements
// (16, one unit of the widest stage; more when the row is longer than
// 16 * TMAX), G rows per CTA of THREADS threads.  The fused product rows
// keep one unit per thread (TMAX = 1024); the forward and inverse rows cap
// a row at 256 threads so that several CTAs share an SM.
template <int LR, int TMAX = 1024>
struct RowGeom {
  static constexpr uint32_t R = 1u << LR;
  static constexpr int TPR =
      (int)((R >> 4) < (uint32_t)TMAX ? (R >> 4) : TMAX);  // threads per row
  static constexpr int EPT = (int)(R / TPR);              // elements / thread
  static constexpr int THREADS = TPR < 256 ? 256 : TPR;   // per CTA
  static constexpr int G = THREADS / TPR;                 // rows per CTA
  // CTAs per SM asked of 256-thread CTAs holding W-byte elements
  template <int W>
  static constexpr int min_ctas() {
    return THREADS <= 256 ? (W == 8 ? TFT_ROW_MIN_CTAS_64 : TFT_ROW_MIN_CTAS_32)
                          : 1;
  }
  static constexpr int L0 = LR % 4 ? LR % 4 : 4;          // first stage
  static constexpr int NST = 1 + (LR - L0) / 4;           // stages
  // r_lo of stage si (stage 0 covers the top L0 levels)
  static __host__ __device__ constexpr int r_lo(int si) {
    return LR - L0 - 4 * si;
  }
};

// Shared layout of the row kernels:
//   K (StageConsts) | RF[G][2][5] | TL[tl] | TLi[tl] | Z[NB][G][R]
template <class T>
struct RowSmem {
  StageConsts<T>* K;
  T* RF;  // RF[(g * 2 + inv) * 5 + stage]
  T* TL;
  T* TLi;
  T* Z;
  __device__ RowSmem(unsigned char* raw, int G, int tl) {
    K = reinterpret_cast<StageConsts<T>*>(raw);
    T* p = reinterpret_cast<T*>(raw + sizeof(StageConsts<T>));
    RF = p;
    p += G * 10;
    TL = p;
    p += tl;
    TLi = p;
    p += tl;
    uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
    Z = reinterpret_cast<T*>(a);
  }
};

// Words between consecutive rows in shared memory.  With 32-bit elements
// and rows of 2^8 (16 threads per row) a warp spans two rows; a 16-word gap
// puts the second row's banks in the other half, so the two rows of a warp
// never collide.
template <class T>
__host__ __device__ constexpr size_t row_stride(int lr) {
  return ((size_t)1 << lr) + (sizeof(T) == 4 && lr <= 8 ? 16 : 0);
}

template <class T>
__host__ __device__ inline size_t row_smem_bytes(int lr, int G, int nbuf) {
  const StagePlan sp = make_stage_plan(lr);
  size_t b = sizeof(StageConsts<T>) + sizeof(T) * (G * 10 + 2 * sp.tl_total);
  b = (b + 15) & ~(size_t)15;
  return b + sizeof(T) * ((size_t)nbuf * G * row_stride<T>(lr));
}

template <class F>
__device__ void copy_roots(RootTable<typename F::T>* s_rt,
                           const RootTable<typename F::T>& rt) {
  using T = typename F::T;
  const T* s = reinterpret_cast<const T*>(&rt);
  T* d = reinterpret_cast<T*>(s_rt);
  for (int i = threadIdx.x; i < (int)(sizeof(rt) / sizeof(T)); i += blockDim.x)
    d[i] = s[i];
}

template <class F>
__device__ void row_setup(RowSmem<typename F::T>& S, const StagePlan& sp,
                          int lr, const RootTable<typename F::T>& rt) {
  fill_stage_consts<F>(S.K, rt, lr);
  build_stage_tables<F>(S.TL, S.TLi, sp, lr, rt);
  __syncthreads();
}

// Row factors of row rho for every stage: RF = omega_{rho 2^{lr - r_lo}}.
template <class F>
__device__ __forceinline__ void row_factors(RowSmem<typename F::T>& S,
                                            const StagePlan& sp, int lr,
                                            int g, int t, uint64_t rho,
                                            const RootTable<typename F::T>& rt) {
  if (t < 2 * sp.n) {
    const int si = t % sp.n;
    const bool inv = t >= sp.n;
    S.RF[(g * 2 + (inv ? 1 : 0)) * 5 + si] =
        row_factor<F>(rho, lr - sp.s[si].r_lo, rt, inv);
  }
}

// One forward stage on one operand of one row.  SRC_GLOBAL: read from Grow
// (the row in global memory), else from the swizzled shared row.
template <class F, int L, bool SRC_GLOBAL>
__device__ __forceinline__ void fwd_stage(typename F::T* Zrow,
                                          const typename F::T* Grow, int r_lo,
                                          int t, int Tpr, typename F::T RF,
                                          const typename F::T* TLs,
                                          const StageConsts<typename F::T>& K,
                                          int ept = 16) {
  using T = typename F::T;
  constexpr int U = 1 << L;
#pragma unroll 1
  for (int v = 0; v < (ept >> L); ++v) {
    const uint32_t u = (uint32_t)(v * Tpr + t);
    T x[U];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint32_t p = unit_pos(u, r_lo, L, i);
      x[i] = SRC_GLOBAL ? Grow[p] : Zrow[swz(p)];
    }
    twist<F, L>(x, F::mul_tw(RF, TLs[u >> r_lo]));
    cnet_fwd<F, L>(x, K);
#pragma unroll
    for (int i = 0; i < U; ++i) Zrow[swz(unit_pos(u, r_lo, L, i))] = x[i];
  }
}

// One forward stage on both operands of the product (same rows, same twist):
// the powers of zeta are computed once; operand B is processed after A has
// been stored (the empty asm with a memory clobber keeps the compiler from
// overlapping the two units, which would double the live registers).
template <class F, int L, bool SRC_GLOBAL>
__device__ __noinline__ void fwd_stage_ab(
    typename F::T* ZA, const typename F::T* GA, typename F::T* ZB,
    const typename F::T* GB, int r_lo, int t, int Tpr, typename F::T RF,
    const typename F::T* TLs, const StageConsts<typename F::T>& K,
    int ept = 16) {
  using T = typename F::T;
  constexpr int U = 1 << L;
#pragma unroll 1
  for (int v = 0; v < (ept >> L); ++v) {
    const uint32_t u = (uint32_t)(v * Tpr + t);
    T pw[U];
    powers<F, L>(pw, F::mul_tw(RF, TLs[u >> r_lo]));
#pragma unroll
    for (int op = 0; op < 2; ++op) {
      T* Zrow = op ? ZB : ZA;
      const T* Grow = op ? GB : GA;
      T x[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const uint32_t p = unit_pos(u, r_lo, L, i);
        x[i] = SRC_GLOBAL ? Grow[p] : Zrow[swz(p)];
      }
#pragma unroll
      for (int i = 1; i < U; ++i) x[i] = F::mul_tw(x[i], pw[i]);
      cnet_fwd<F, L>(x, K);
#pragma unroll
      for (int i = 0; i < U; ++i) Zrow[swz(unit_pos(u, r_lo, L, i))] = x[i];
      asm volatile("" ::: "memory");
    }
  }
}

// One inverse stage (2^L times the exact inverse, see cnet_inv2).
// DST_GLOBAL: write to Grow instead of the shared row; with SPLIT, positions
// p >= bsplit go to Galt[p] instead; with SCALE, multiply by K.sc = 2^-lr
// first (the last stage of a row's inverse).
template <class F, int L, bool DST_GLOBAL, bool SPLIT = false,
          bool SCALE = false>
__device__ __forceinline__ void inv_stage(typename F::T* Zrow,
                                          typename F::T* Grow, int r_lo, int t,
                                          int Tpr, typename F::T RFi,
                                          const typename F::T* TLis,
                                          const StageConsts<typename F::T>& K,
                                          int ept = 16, uint32_t bsplit = 0,
                                          typename F::T* Galt = nullptr) {
  using T = typename F::T;
  constexpr int U = 1 << L;
#pragma unroll 1
  for (int v = 0; v < (ept >> L); ++v) {
    const uint32_t u = (uint32_t)(v * Tpr + t);
    T x[U];
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = Zrow[swz(unit_pos(u, r_lo, L, i))];
    cnet_inv2<F, L>(x, K);
    twist<F, L>(x, F::mul_tw(RFi, TLis[u >> r_lo]));
    if (SCALE) {
#pragma unroll
      for (int i = 0; i < U; ++i) x[i] = F::mul_tw(x[i], K.sc);
    }
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint32_t p = unit_pos(u, r_lo, L, i);
      if (DST_GLOBAL && SPLIT)
        (p < bsplit ? Grow : Galt)[p] = F::canon(x[i]);
      else if (DST_GLOBAL)
        Grow[p] = F::canon(x[i]);
      else
        Zrow[swz(p)] = x[i];
    }
  }
}

// Common prologue of the row kernels: root table, constants, tables.
#define TFT_ROW_PROLOGUE(NBUF) TFT_ROW_PROLOGUE_G(NBUF, RowGeom<LR>)
#define TFT_ROW_PROLOGUE_G(NBUF, ...)                                   \
  using T = typename F::T;                                              \
  using Geo = __VA_ARGS__;                                              \
  extern __shared__ __align__(16) unsigned char smem_raw[];             \
  __shared__ RootTable<T> s_rt;                                         \
  copy_roots<F>(&s_rt, rt);                                             \
  __syncthreads();                                                      \
  constexpr uint32_t R = Geo::R;                                        \
  constexpr int Tpr = Geo::TPR;                                         \
  constexpr int G = Geo::G;                                             \
  const int g = threadIdx.x / Tpr, t = threadIdx.x % Tpr;               \
  const StagePlan sp = make_stage_plan(LR);                             \
  RowSmem<T> S(smem_raw, G, sp.tl_total);                               \
  row_setup<F>(S, sp, LR, s_rt);

// ---------------------------------------------------------------------------
// Forward rows rho < a.  The a rows at X are rows rho_off .. rho_off + a - 1
// of the row/column view (rho_off > 0 for a block of rows held apart, as a
// rank of a sharded transform holds them): the row factors use the global
// row index.
// ---------------------------------------------------------------------------
template <class F, int LR>
__global__ void __launch_bounds__(RowGeom<LR, 256>::THREADS, RowGeom<LR, 256>::template min_ctas<sizeof(typename F::T)>())
k_row_fwd2(typename F::T* X, uint64_t a, uint64_t rho_off,
           RootTable<typename F::T> rt) {
  TFT_ROW_PROLOGUE_G(1, RowGeom<LR, 256>)
  T* Zrow = S.Z + g * row_stride<T>(LR);
  for (uint64_t rho0 = (uint64_t)blockIdx.x * G; rho0 < a;
       rho0 += (uint64_t)gridDim.x * G) {
    const uint64_t rho = rho0 + g;
    const bool active = rho < a;
    if (active) row_factors<F>(S, sp, LR, g, t, rho_off + rho, s_rt);
    __syncthreads();
    T* Grow = X + rho * R;
    if (active)
      fwd_stage<F, Geo::L0, true>(Zrow, Grow, Geo::r_lo(0), t, Tpr,
                                  S.RF[(g * 2) * 5], S.TL + sp.s[0].tl_off,
                                  *S.K, Geo::EPT);
    __syncthreads();
#pragma unroll 1
    for (int si = 1; si < Geo::NST; ++si) {
      if (active)
        fwd_stage<F, 4, false>(Zrow, Grow, Geo::r_lo(si), t, Tpr,
                               S.RF[(g * 2) * 5 + si],
                               S.TL + sp.s[si].tl_off, *S.K, Geo::EPT);
      __syncthreads();
    }
    if (active)
      for (uint32_t q = t; q < R; q += Tpr) Grow[q] = F::canon(Zrow[swz(q)]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Inverse rows rho < a (rows rho_off + rho of the view, as above).
// ---------------------------------------------------------------------------
template <class F, int LR>
__global__ void __launch_bounds__(RowGeom<LR, 256>::THREADS, RowGeom<LR, 256>::template min_ctas<sizeof(typename F::T)>())
k_row_inv2(typename F::T* X, uint64_t a, uint64_t rho_off,
           RootTable<typename F::T> rt) {
  TFT_ROW_PROLOGUE_G(1, RowGeom<LR, 256>)
  T* Zrow = S.Z + g * row_stride<T>(LR);
  for (uint64_t rho0 = (uint64_t)blockIdx.x * G; rho0 < a;
       rho0 += (uint64_t)gridDim.x * G) {
    const uint64_t rho = rho0 + g;
    const bool active = rho < a;
    T* Grow = X + rho * R;
    if (active) {
      row_factors<F>(S, sp, LR, g, t, rho_off + rho, s_rt);
      // asynchronous copies: all of the thread's positions in flight
      for (uint32_t q = t; q < R; q += Tpr) cp_async_elem(Zrow + swz(q), Grow + q);
      cp_async_wait_all();
    }
    __syncthreads();
#pragma unroll 1
    for (int si = Geo::NST - 1; si >= 1; --si) {
      if (active)
        inv_stage<F, 4, false>(Zrow, Grow, Geo::r_lo(si), t, Tpr,
                               S.RF[(g * 2 + 1) * 5 + si],
                               S.TLi + sp.s[si].tl_off, *S.K, Geo::EPT);
      __syncthreads();
    }
    if (active)
      inv_stage<F, Geo::L0, true, false, true>(Zrow, Grow, Geo::r_lo(0), t,
                                               Tpr, S.RF[(g * 2 + 1) * 5],
                                               S.TLi + sp.s[0].tl_off, *S.K,
                                               Geo::EPT);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Fused product rows: forward row network of A' and B', pointwise product,
// inverse row network, result written over A'.  The inverse is left scaled
// by 2^lr (cnet_inv2): the inverse column pass removes that factor together
// with its own.  Requires LR >= 8 (at least two stages).  row_mul_body
// processes, for every row slot g of the CTA, row rho_g (GA, GB: that row of
// A' and B' in global memory); inactive slots only take part in the
// barriers.  A row whose positions q >= bsplit lie beyond the buffers (the
// last row of a product transform of length rounded up to a multiple of R)
// reads those positions from EAg / EBg and writes them back to EAg.
// ---------------------------------------------------------------------------
template <class F, int LR>
__device__ __forceinline__ void row_mul_body(
    RowSmem<typename F::T>& S, const StagePlan& sp, int g, int t,
    bool active, uint64_t rho, typename F::T* GA,
    const typename F::T* GB, const RootTable<typename F::T>& s_rt,
    uint32_t bsplit = 0xffffffffu, typename F::T* EAg = nullptr,
    const typename F::T* EBg = nullptr) {
  using T = typename F::T;
  using Geo = RowGeom<LR>;
  constexpr uint32_t R = Geo::R;
  constexpr int Tpr = Geo::TPR;
  constexpr int G = Geo::G;
  static_assert(Geo::NST >= 2, "fused row pass needs two stages");
  T* ZA = S.Z + g * row_stride<T>(LR);
  T* ZB = S.Z + (G + g) * row_stride<T>(LR);
  constexpr int last = Geo::NST - 1;  // r_lo = 0, L = 4
  if (active) row_factors<F>(S, sp, LR, g, t, rho, s_rt);
  __syncthreads();
  // the split is needed again by the last stage: parked in shared memory
  // so that it holds no registers across the stages
  __shared__ uint32_t s_bsplit[G];
  __shared__ T* s_ealt[G];
  if (active && t == 0) {
    s_bsplit[g] = bsplit;
    s_ealt[g] = EAg;
  }
  // both rows to shared memory (coalesced), then the first stage from
  // there: reading the first stage straight from global memory lets the
  // scheduler overlap the two operands' loads and spill registers.  The
  // loads are asynchronous copies straight into the swizzled rows, all of a
  // thread's in flight at once without holding registers.
  if (active) {
    for (uint32_t q = t; q < R; q += Tpr) {
      const bool mem = q < bsplit;  // bsplit >= R for a full row
      cp_async_elem(ZA + swz(q), mem ? GA + q : EAg + q);
      cp_async_elem(ZB + swz(q), mem ? GB + q : EBg + q);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  if (active) {
    const T RF = S.RF[(g * 2) * 5];
    const T* TLs = S.TL + sp.s[0].tl_off;
    fwd_stage_ab<F, Geo::L0, false>(ZA, GA, ZB, GB, Geo::r_lo(0), t, Tpr,
                                    RF, TLs, *S.K);
  }
  __syncthreads();
#pragma unroll 1
  for (int si = 1; si < last; ++si) {
    if (active) {
      const T RF = S.RF[(g * 2) * 5 + si];
      const T* TLs = S.TL + sp.s[si].tl_off;
      fwd_stage_ab<F, 4, false>(ZA, GA, ZB, GB, Geo::r_lo(si), t, Tpr, RF,
                                TLs, *S.K);
    }
    __syncthreads();
  }
  // last forward stage (r_lo = 0, L = 4), the pointwise product and the
  // first inverse stage.  64-bit elements: fwd_stage_ab, then each thread
  // reads back only the 16 entries it has just written (no barrier needed)
  // for the product and the inverse stage; reusing fwd_stage_ab keeps the
  // kernel's code smaller, which measured faster.  32-bit elements: all
  // three in registers on one unit (their code is smaller; measured faster).
  if (active) {
    const T RFi = S.RF[(g * 2 + 1) * 5 + last];
    const T* TLis = S.TLi + sp.s[last].tl_off;
    const uint32_t u = (uint32_t)t;  // one unit per thread
    T xa[16];
    if constexpr (sizeof(T) == 8) {
      fwd_stage_ab<F, 4, false>(ZA, GA, ZB, GB, 0, t, Tpr,
                                S.RF[(g * 2) * 5 + last],
                                S.TL + sp.s[last].tl_off, *S.K);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        xa[i] = F::mul_data(ZA[swz(u * 16 + i)], ZB[swz(u * 16 + i)]);
    } else {
      T xb[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        xa[i] = ZA[swz(u * 16 + i)];
        xb[i] = ZB[swz(u * 16 + i)];
      }
      // twist both operands with one running power
      const T zeta = F::mul_tw(S.RF[(g * 2) * 5 + last],
                               (S.TL + sp.s[last].tl_off)[u]);
      T zp = zeta;
#pragma unroll
      for (int i = 1; i < 16; ++i) {
        xa[i] = F::mul_tw(xa[i], zp);
        xb[i] = F::mul_tw(xb[i], zp);
        if (i < 15) zp = F::mul_tw(zp, zeta);
      }
      cnet_fwd<F, 4>(xa, *S.K);
      cnet_fwd<F, 4>(xb, *S.K);
#pragma unroll
      for (int i = 0; i < 16; ++i) xa[i] = F::mul_data(xa[i], xb[i]);
    }
    cnet_inv2<F, 4>(xa, *S.K);
    twist<F, 4>(xa, F::mul_tw(RFi, TLis[u]));
#pragma unroll
    for (int i = 0; i < 16; ++i) ZA[swz(u * 16 + i)] = xa[i];
  }
  __syncthreads();
#pragma unroll 1
  for (int si = last - 1; si >= 1; --si) {
    if (active)
      inv_stage<F, 4, false>(ZA, GA, Geo::r_lo(si), t, Tpr,
                             S.RF[(g * 2 + 1) * 5 + si],
                             S.TLi + sp.s[si].tl_off, *S.K);
    __syncthreads();
  }
  if (active) {
    const uint32_t bs = s_bsplit[g];
    if (bs >= R)
      inv_stage<F, Geo::L0, true>(ZA, GA, Geo::r_lo(0), t, Tpr,
                                  S.RF[(g * 2 + 1) * 5],
                                  S.TLi + sp.s[0].tl_off, *S.K);
    else
      inv_stage<F, Geo::L0, true, true>(ZA, GA, Geo::r_lo(0), t, Tpr,
                                        S.RF[(g * 2 + 1) * 5],
                                        S.TLi + sp.s[0].tl_off, *S.K, 16, bs,
                                        s_ealt[g]);
  }
  __syncthreads();
}

// Rows 0 .. a - 1 of the product, and with b > 0 also row a in full: the
// product's transforms then have length (a + 1) R >= r, and the positions
// a R + q, q >= b, past the r-word buffers live in EA / EB (R words each;
// the forward column pass leaves them there).
template <class F, int LR>
__global__ void __launch_bounds__(RowGeom<LR>::THREADS, RowGeom<LR>::template min_ctas<sizeof(typename F::T)>())
k_row_mul2(typename F::T* out, const typename F::T* __restrict__ work,
           typename F::T* EA, const typename F::T* EB, uint64_t a, uint64_t b,
           RootTable<typename F::T> rt) {
  TFT_ROW_PROLOGUE(2)
  const uint64_t nrows = a + (b > 0 ? 1 : 0);
  for (uint64_t rho0 = (uint64_t)blockIdx.x * G; rho0 < nrows;
       rho0 += (uint64_t)gridDim.x * G) {
    const uint64_t rho = rho0 + g;
    row_mul_body<F, LR>(S, sp, g, t, rho < nrows, rho, out + rho * R,
                        work + rho * R, s_rt,
                        rho == a ? (uint32_t)b : 0xffffffffu, EA, EB);
  }
}

// ---------------------------------------------------------------------------
// The ragged last row of a forward transform (block a, first b outputs) on
// the stage engine: the full forward network of block a, whose inputs are
// the long columns' last entries (q < b, in the buffer) and E_q (q >= b,
// scratch).  Only outputs q < b are stored, over the row's first b words.
// (Products run their transforms at a length that has no ragged row.)
// ---------------------------------------------------------------------------
template <class F, int LR>
__global__ void __launch_bounds__(RowGeom<LR>::THREADS, RowGeom<LR>::template min_ctas<sizeof(typename F::T)>())
k_row_last2(typename F::T* GA, const typename F::T* __restrict__ E,
            uint64_t a, uint64_t b, RootTable<typename F::T> rt) {
  TFT_ROW_PROLOGUE(1)
  // one row (GA = row a of the view): slot 0 of the first CTA
  const bool active = blockIdx.x == 0 && g == 0;
  T* ZA = S.Z + g * row_stride<T>(LR);
  constexpr int last = Geo::NST - 1;
  if (active) {
    row_factors<F>(S, sp, LR, g, t, a, s_rt);
    for (uint32_t q = t; q < R; q += Tpr) ZA[swz(q)] = q < b ? GA[q] : E[q];
  }
  __syncthreads();
#pragma unroll 1
  for (int si = 0; si < last; ++si) {
    if (active) {
      const T RF = S.RF[(g * 2) * 5 + si];
      const T* TLs = S.TL + sp.s[si].tl_off;
      const int r_lo = Geo::r_lo(si);
      if (si == 0)
        fwd_stage<F, Geo::L0, false>(ZA, GA, r_lo, t, Tpr, RF, TLs, *S.K);
      else
        fwd_stage<F, 4, false>(ZA, GA, r_lo, t, Tpr, RF, TLs, *S.K);
    }
    __syncthreads();
  }
  if (active) {
    const T RF = S.RF[(g * 2) * 5 + last];
    const T* TLs = S.TL + sp.s[last].tl_off;
    const uint32_t u = (uint32_t)t;  // 16 consecutive outputs per thread
    T xa[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) xa[i] = ZA[swz(u * 16 + i)];
    twist<F, 4>(xa, F::mul_tw(RF, TLs[u]));
    cnet_fwd<F, 4>(xa, *S.K);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (u * 16 + i < b) GA[u * 16 + i] = F::canon(xa[i]);
  }
}

// Dispatch a runtime lr in [8, 12] (the batched large class) to LR.
#define TFT_LR_DISPATCH_BATCH(lr, ...)                           \
  switch (lr) {                                                  \
    case 8: { constexpr int LR = 8; __VA_ARGS__; } break;        \
    case 9: { constexpr int LR = 9; __VA_ARGS__; } break;        \
    case 10: { constexpr int LR = 10; __VA_ARGS__; } break;      \
    case 11: { constexpr int LR = 11; __VA_ARGS__; } break;      \
    default: { constexpr int LR = 12; __VA_ARGS__; } break;      \
  }

// Dispatch a runtime lr in [8, 14] to a compile-time LR.
#define TFT_LR_DISPATCH(lr, ...)                        \
  switch (lr) {                                         \
    case 8: { constexpr int LR = 8; __VA_ARGS__; } break; \
    case 9: { constexpr int LR = 9; __VA_ARGS__; } break; \
    case 10: { constexpr int LR = 10; __VA_ARGS__; } break; \
    case 11: { constexpr int LR = 11; __VA_ARGS__; } break; \
    case 12: { constexpr int LR = 12; __VA_ARGS__; } break; \
    case 13: { constexpr int LR = 13; __VA_ARGS__; } break; \
    default: { constexpr int LR = 14; __VA_ARGS__; } break; \
  }

}  // namespace tftgb
