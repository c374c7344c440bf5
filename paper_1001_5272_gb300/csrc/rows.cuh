// Row kernels on the register-blocked stage engine (stages.cuh).
//
// A row rho < a is block rho (2^lr positions) of the global network, so its
// lr levels are run as stages with the twist zeta = omega_{rho 2^{lr-r_lo}} *
// omega_{B_local 2^L}.  Each row is handled by R/16 threads holding 16
// elements each; a CTA holds G = blockDim / (R/16) rows at a time.  The
// kernels are persistent over rows.
#pragma once
#include "stages.cuh"

namespace tftgb {

// Shared layout of the row kernels (after the static root table copy):
//   K (StageConsts) | RF[G][2][5] | TL[tl] | TLi[tl] | Z[NB][G][R]
template <class T>
struct RowSmem {
  StageConsts<T>* K;
  T* RF;    // RF[(g * 2 + inv) * 5 + stage]
  T* TL;
  T* TLi;
  T* Z;
  __device__ RowSmem(unsigned char* raw, int G, int tl, uint32_t R, int nbuf) {
    K = reinterpret_cast<StageConsts<T>*>(raw);
    T* p = reinterpret_cast<T*>(raw + sizeof(StageConsts<T>));
    RF = p;
    p += G * 10;
    TL = p;
    p += tl;
    TLi = p;
    p += tl;
    // align the data to 16 bytes
    uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
    Z = reinterpret_cast<T*>(a);
    (void)R;
    (void)nbuf;
  }
};

template <class T>
__host__ __device__ inline size_t row_smem_bytes(int lr, int G, int nbuf) {
  const StagePlan sp = make_stage_plan(lr);
  size_t b = sizeof(StageConsts<T>) + sizeof(T) * (G * 10 + 2 * sp.tl_total);
  b = (b + 15) & ~(size_t)15;
  return b + sizeof(T) * ((size_t)nbuf * G << lr);
}

template <class F>
__device__ void row_setup(RowSmem<typename F::T>& S, const StagePlan& sp,
                          int lr, const RootTable<typename F::T>& rt) {
  for (int i = threadIdx.x; i < 8; i += blockDim.x) {
    S.K->c[i] = rt.c16[i];
    S.K->ci[i] = rt.c16i[i];
  }
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
// (row in global memory), else from the swizzled shared row.
template <class F, int L, bool SRC_GLOBAL>
__device__ __forceinline__ void fwd_stage(typename F::T* Zrow,
                                          const typename F::T* Grow, int r_lo,
                                          int t, int Tpr,
                                          typename F::T RF,
                                          const typename F::T* TLs,
                                          const StageConsts<typename F::T>& K) {
  using T = typename F::T;
  constexpr int U = 1 << L;
#pragma unroll 1
  for (int v = 0; v < (16 >> L); ++v) {
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

// One inverse stage.  DST_GLOBAL: write to Grow instead of the shared row.
template <class F, int L, bool DST_GLOBAL>
__device__ __forceinline__ void inv_stage(typename F::T* Zrow,
                                          typename F::T* Grow, int r_lo, int t,
                                          int Tpr, typename F::T RFi,
                                          const typename F::T* TLis,
                                          const StageConsts<typename F::T>& K) {
  using T = typename F::T;
  constexpr int U = 1 << L;
#pragma unroll 1
  for (int v = 0; v < (16 >> L); ++v) {
    const uint32_t u = (uint32_t)(v * Tpr + t);
    T x[U];
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = Zrow[swz(unit_pos(u, r_lo, L, i))];
    cnet_inv<F, L>(x, K);
    twist<F, L>(x, F::mul_tw(RFi, TLis[u >> r_lo]));
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint32_t p = unit_pos(u, r_lo, L, i);
      if (DST_GLOBAL)
        Grow[p] = x[i];
      else
        Zrow[swz(p)] = x[i];
    }
  }
}

#define TFT_STAGE_SWITCH(L, CALL)          \
  switch (L) {                             \
    case 1: { constexpr int LL = 1; CALL; } break; \
    case 2: { constexpr int LL = 2; CALL; } break; \
    case 3: { constexpr int LL = 3; CALL; } break; \
    default: { constexpr int LL = 4; CALL; } break; \
  }

// ---------------------------------------------------------------------------
// Forward rows rho < a.
// ---------------------------------------------------------------------------
template <class F, int MAXT>
__global__ void __launch_bounds__(MAXT)
k_row_fwd2(typename F::T* X, int lr, uint64_t a, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  {
    const T* src = reinterpret_cast<const T*>(&rt);
    T* dst = reinterpret_cast<T*>(&s_rt);
    for (int i = threadIdx.x; i < (int)(sizeof(rt) / sizeof(T)); i += blockDim.x)
      dst[i] = src[i];
  }
  __syncthreads();
  const uint32_t R = 1u << lr;
  const int Tpr = (int)(R >> 4);
  const int G = blockDim.x / Tpr;
  const int g = threadIdx.x / Tpr, t = threadIdx.x % Tpr;
  const StagePlan sp = make_stage_plan(lr);
  RowSmem<T> S(smem_raw, G, sp.tl_total, R, 1);
  row_setup<F>(S, sp, lr, s_rt);
  T* Zrow = S.Z + ((size_t)g << lr);
  for (uint64_t rho0 = (uint64_t)blockIdx.x * G; rho0 < a;
       rho0 += (uint64_t)gridDim.x * G) {
    const uint64_t rho = rho0 + g;
    const bool active = rho < a;
    if (active) row_factors<F>(S, sp, lr, g, t, rho, s_rt);
    __syncthreads();
    T* Grow = X + rho * R;
    for (int si = 0; si < sp.n; ++si) {
      if (active) {
        const T RF = S.RF[(g * 2) * 5 + si];
        const T* TLs = S.TL + sp.s[si].tl_off;
        const int r_lo = sp.s[si].r_lo;
        if (si == 0) {
          TFT_STAGE_SWITCH(sp.s[si].L, (fwd_stage<F, LL, true>(
                                           Zrow, Grow, r_lo, t, Tpr, RF, TLs,
                                           *S.K)));
        } else {
          TFT_STAGE_SWITCH(sp.s[si].L, (fwd_stage<F, LL, false>(
                                           Zrow, Grow, r_lo, t, Tpr, RF, TLs,
                                           *S.K)));
        }
      }
      __syncthreads();
    }
    if (active)
      for (uint32_t q = t; q < R; q += Tpr) Grow[q] = Zrow[swz(q)];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Inverse rows rho < a.
// ---------------------------------------------------------------------------
template <class F, int MAXT>
__global__ void __launch_bounds__(MAXT)
k_row_inv2(typename F::T* X, int lr, uint64_t a, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  {
    const T* src = reinterpret_cast<const T*>(&rt);
    T* dst = reinterpret_cast<T*>(&s_rt);
    for (int i = threadIdx.x; i < (int)(sizeof(rt) / sizeof(T)); i += blockDim.x)
      dst[i] = src[i];
  }
  __syncthreads();
  const uint32_t R = 1u << lr;
  const int Tpr = (int)(R >> 4);
  const int G = blockDim.x / Tpr;
  const int g = threadIdx.x / Tpr, t = threadIdx.x % Tpr;
  const StagePlan sp = make_stage_plan(lr);
  RowSmem<T> S(smem_raw, G, sp.tl_total, R, 1);
  row_setup<F>(S, sp, lr, s_rt);
  T* Zrow = S.Z + ((size_t)g << lr);
  for (uint64_t rho0 = (uint64_t)blockIdx.x * G; rho0 < a;
       rho0 += (uint64_t)gridDim.x * G) {
    const uint64_t rho = rho0 + g;
    const bool active = rho < a;
    T* Grow = X + rho * R;
    if (active) {
      row_factors<F>(S, sp, lr, g, t, rho, s_rt);
      for (uint32_t q = t; q < R; q += Tpr) Zrow[swz(q)] = Grow[q];
    }
    __syncthreads();
    for (int si = sp.n - 1; si >= 0; --si) {
      if (active) {
        const T RFi = S.RF[(g * 2 + 1) * 5 + si];
        const T* TLis = S.TLi + sp.s[si].tl_off;
        const int r_lo = sp.s[si].r_lo;
        if (si == 0) {
          TFT_STAGE_SWITCH(sp.s[si].L, (inv_stage<F, LL, true>(
                                           Zrow, Grow, r_lo, t, Tpr, RFi,
                                           TLis, *S.K)));
        } else {
          TFT_STAGE_SWITCH(sp.s[si].L, (inv_stage<F, LL, false>(
                                           Zrow, Grow, r_lo, t, Tpr, RFi,
                                           TLis, *S.K)));
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Fused product rows rho < a: forward row network of A' (in out) and B' (in
// work), pointwise product, inverse row network, result to out.  The last
// forward stage, the product and the first inverse stage share one unit in
// registers.
// ---------------------------------------------------------------------------
template <class F, int MAXT>
__global__ void __launch_bounds__(MAXT)
k_row_mul2(typename F::T* out, const typename F::T* __restrict__ work, int lr,
           uint64_t a, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  {
    const T* src = reinterpret_cast<const T*>(&rt);
    T* dst = reinterpret_cast<T*>(&s_rt);
    for (int i = threadIdx.x; i < (int)(sizeof(rt) / sizeof(T)); i += blockDim.x)
      dst[i] = src[i];
  }
  __syncthreads();
  const uint32_t R = 1u << lr;
  const int Tpr = (int)(R >> 4);
  const int G = blockDim.x / Tpr;
  const int g = threadIdx.x / Tpr, t = threadIdx.x % Tpr;
  const StagePlan sp = make_stage_plan(lr);
  RowSmem<T> S(smem_raw, G, sp.tl_total, R, 2);
  row_setup<F>(S, sp, lr, s_rt);
  T* ZA = S.Z + ((size_t)g << lr);
  T* ZB = S.Z + ((size_t)(G + g) << lr);
  const int last = sp.n - 1;  // the stage with r_lo = 0 (always L = 4)
  for (uint64_t rho0 = (uint64_t)blockIdx.x * G; rho0 < a;
       rho0 += (uint64_t)gridDim.x * G) {
    const uint64_t rho = rho0 + g;
    const bool active = rho < a;
    if (active) row_factors<F>(S, sp, lr, g, t, rho, s_rt);
    __syncthreads();
    T* GA = out + rho * R;
    const T* GB = work + rho * R;
    // forward stages before the last, both operands
    for (int si = 0; si < last; ++si) {
      if (active) {
        const T RF = S.RF[(g * 2) * 5 + si];
        const T* TLs = S.TL + sp.s[si].tl_off;
        const int r_lo = sp.s[si].r_lo;
        if (si == 0) {
          TFT_STAGE_SWITCH(sp.s[si].L, (fwd_stage<F, LL, true>(
                                           ZA, GA, r_lo, t, Tpr, RF, TLs,
                                           *S.K)));
          TFT_STAGE_SWITCH(sp.s[si].L, (fwd_stage<F, LL, true>(
                                           ZB, GB, r_lo, t, Tpr, RF, TLs,
                                           *S.K)));
        } else {
          TFT_STAGE_SWITCH(sp.s[si].L, (fwd_stage<F, LL, false>(
                                           ZA, GA, r_lo, t, Tpr, RF, TLs,
                                           *S.K)));
          TFT_STAGE_SWITCH(sp.s[si].L, (fwd_stage<F, LL, false>(
                                           ZB, GB, r_lo, t, Tpr, RF, TLs,
                                           *S.K)));
        }
      }
      __syncthreads();
    }
    // last forward stage (r_lo = 0, L = 4) + product + first inverse stage
    if (active) {
      const T RF = S.RF[(g * 2) * 5 + last];
      const T RFi = S.RF[(g * 2 + 1) * 5 + last];
      const T* TLs = S.TL + sp.s[last].tl_off;
      const T* TLis = S.TLi + sp.s[last].tl_off;
      const bool from_global = last == 0;
      const uint32_t u = (uint32_t)t;  // one unit per thread
      T xa[16], xb[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const uint32_t p = u * 16 + i;
        xa[i] = from_global ? GA[p] : ZA[swz(p)];
        xb[i] = from_global ? GB[p] : ZB[swz(p)];
      }
      {
        T pw[16];
        powers<F, 4>(pw, F::mul_tw(RF, TLs[u]));
#pragma unroll
        for (int i = 1; i < 16; ++i) {
          xa[i] = F::mul_tw(xa[i], pw[i]);
          xb[i] = F::mul_tw(xb[i], pw[i]);
        }
      }
      cnet_fwd<F, 4>(xa, *S.K);
      cnet_fwd<F, 4>(xb, *S.K);
#pragma unroll
      for (int i = 0; i < 16; ++i) xa[i] = F::mul_data(xa[i], xb[i]);
      cnet_inv<F, 4>(xa, *S.K);
      twist<F, 4>(xa, F::mul_tw(RFi, TLis[u]));
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (last == 0)
          GA[u * 16 + i] = xa[i];
        else
          ZA[swz(u * 16 + i)] = xa[i];
      }
    }
    __syncthreads();
    // remaining inverse stages
    for (int si = last - 1; si >= 0; --si) {
      if (active) {
        const T RFi = S.RF[(g * 2 + 1) * 5 + si];
        const T* TLis = S.TLi + sp.s[si].tl_off;
        const int r_lo = sp.s[si].r_lo;
        if (si == 0) {
          TFT_STAGE_SWITCH(sp.s[si].L, (inv_stage<F, LL, true>(
                                           ZA, GA, r_lo, t, Tpr, RFi, TLis,
                                           *S.K)));
        } else {
          TFT_STAGE_SWITCH(sp.s[si].L, (inv_stage<F, LL, false>(
                                           ZA, GA, r_lo, t, Tpr, RFi, TLis,
                                           *S.K)));
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace tftgb
