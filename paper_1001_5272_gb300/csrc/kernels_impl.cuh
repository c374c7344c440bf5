// CUDA kernels of the in-place TFT / ITFT / TFT product for sm_103a.
//
// Decomposition (the L1 x L2 row/column split the paper credits to the
// cache-friendly TFT, Section 1.3).  Fix R = 2^lr and write n = a R + b,
// 0 <= b < R.  Column q (q < R) is C_q(x) = sum_t X_{q + tR} x^t, of length
// a + 1 if q < b ("long") and a otherwise ("short"), so that
//     F(x) = sum_q x^q C_q(x^R),
//     F(omega_{rho R + j}) = sum_q omega_{rho R + j}^q C_q(omega_rho)
// because omega_s^R = omega_{s >> lr} and omega_{rho R} omega_j =
// omega_{rho R + j} (disjoint bits, Section 5).  Hence
//   1. column pass: TFT of every column (its own TFT of length a or a+1,
//      written back in place at stride R); short columns also need
//      E_q = C_q(omega_a), which has no slot in the buffer and goes to an
//      R-word scratch;
//   2. row pass: every full row rho < a runs the last lr levels of the
//      network (block rho of the global network) in place;
//   3. last row rho = a: the first b outputs of block a, whose inputs are
//      the long columns' last entries and E_q.
// The inverse runs the same steps backwards: inverse rows; inverse short
// columns (ITFT of length a) and E_q by Horner; the last row by the
// generalized block inverse with known inputs E_q at q >= b; inverse long
// columns (length a + 1).  Global memory holds the n-word buffer plus the
// R-word scratch; every transform works in shared memory.  The product on
// rows of at least 2^8 runs its transforms at length (a + 1) R instead (any
// length >= r determines the product), so it has no ragged row: every
// column has length a + 1 and row a is a full row whose positions past r
// live in the R-word scratch (Launch::polymul).
#pragma once
#include <cuda_runtime.h>

#include "engine.cuh"
#include "alg3.cuh"
#include "batch.cuh"
#include "cols.cuh"
#include "lastrow_cluster.cuh"
#include "rows.cuh"
#include "tft_internal.h"

namespace tftgb {

template <class F>
__device__ __forceinline__ void load_roots(RootTable<typename F::T>* s_rt,
                                           const RootTable<typename F::T>& rt) {
  using T = typename F::T;
  const T* src = reinterpret_cast<const T*>(&rt);
  T* dst = reinterpret_cast<T*>(s_rt);
  constexpr int nwords = sizeof(RootTable<T>) / sizeof(T);
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Small transforms: the whole transform of length n <= 2^l in one CTA.
// ---------------------------------------------------------------------------
template <class F, bool INV>
__global__ void __launch_bounds__(512)
k_small(typename F::T* __restrict__ x, uint32_t n, int l,
        RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  load_roots<F>(&s_rt, rt);
  T* Z = reinterpret_cast<T*>(smem_raw);
  const uint32_t N = 1u << l;
  T* W = Z + N;
  T* Wih = W + (N > 1 ? N / 2 : 1);
  build_base_tables<F>(W, INV ? Wih : nullptr, l, s_rt);
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
    Z[i] = i < n ? x[i] : T(0);
  __syncthreads();
  ColTw<F> tw{W, Wih};
  if (!INV)
    fwd_pruned<F>(Z, 0, 0, l, n, tw);
  else
    inv_block<F>(Z, 0, 0, l, n, tw);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = F::canon(Z[i]);
}

// Small TFT product: r = na + nb - 1 <= 2^l, both operands in one CTA.
// The two operands are interleaved as the two columns of one tile.
template <class F>
__global__ void __launch_bounds__(512)
k_small_mul(const typename F::T* __restrict__ a, uint32_t na,
            const typename F::T* __restrict__ b, uint32_t nb,
            typename F::T* __restrict__ out, int l,
            RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  load_roots<F>(&s_rt, rt);
  const uint32_t N = 1u << l;
  const uint32_t r = na + nb - 1;
  T* Z = reinterpret_cast<T*>(smem_raw);  // 2 N: (t, 0) = A, (t, 1) = B
  T* W = Z + 2 * N;
  T* Wih = W + (N > 1 ? N / 2 : 1);
  build_base_tables<F>(W, Wih, l, s_rt);
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
    Z[2 * i] = i < na ? a[i] : T(0);
    Z[2 * i + 1] = i < nb ? b[i] : T(0);
  }
  __syncthreads();
  ColTw<F> tw{W, Wih};
  fwd_pruned<F>(Z, 1, 1, l, r, tw);
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
    Z[2 * i] = i < r ? F::mul_data(Z[2 * i], Z[2 * i + 1]) : T(0);
  __syncthreads();
  inv_block<F>(Z, 0, 1, l, r, tw);
  for (uint32_t i = threadIdx.x; i < r; i += blockDim.x)
    out[i] = F::canon(Z[2 * i]);
}

// ---------------------------------------------------------------------------
// Row pass (forward), persistent over rows.  Rows rho < a are full blocks of
// the network; if b > 0 the last row rho = a is processed first (by CTA 0)
// from the long columns' last entries (q < b) and E (q >= b), and only its
// first b outputs are computed and stored.
// ---------------------------------------------------------------------------
template <class F>
__global__ void __launch_bounds__(512)
k_row_fwd(typename F::T* X, const typename F::T* __restrict__ E, int lr,
          uint64_t a, uint64_t b, int only_last, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  load_roots<F>(&s_rt, rt);
  const uint32_t R = 1u << lr;
  T* Z = reinterpret_cast<T*>(smem_raw);
  T* W = Z + R;
  T* L = W + R / 2;
  build_base_tables<F>(W, nullptr, lr, s_rt);
  // only_last: just the ragged last row (the full rows run elsewhere)
  const uint64_t nrows = only_last ? 1 : a + (b > 0 ? 1 : 0);
  for (uint64_t it = blockIdx.x; it < nrows; it += gridDim.x) {
    const uint64_t rho =
        only_last ? a : ((b > 0) ? (it == 0 ? a : it - 1) : it);
    const bool last = rho == a;
    T* row = X + rho * R;
    for (uint32_t q = threadIdx.x; q < R; q += blockDim.x)
      Z[q] = (!last || q < b) ? row[q] : E[q];
    __syncthreads();
    RowTw<F> tw{W, nullptr, L, &s_rt, rho, lr};
    const uint32_t nout = last ? (uint32_t)b : R;
    fwd_pruned<F>(Z, 0, 0, lr, nout, tw);
    for (uint32_t q = threadIdx.x; q < nout; q += blockDim.x)
      row[q] = F::canon(Z[q]);
    __syncthreads();
  }
}

// Row pass (inverse) over the full rows rho < a.
template <class F>
__global__ void __launch_bounds__(512)
k_row_inv(typename F::T* X, int lr, uint64_t a, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  load_roots<F>(&s_rt, rt);
  const uint32_t R = 1u << lr;
  T* Z = reinterpret_cast<T*>(smem_raw);
  T* W = Z + R;
  T* Wih = W + R / 2;
  T* L = Wih + R / 2;
  build_base_tables<F>(W, Wih, lr, s_rt);
  for (uint64_t rho = blockIdx.x; rho < a; rho += gridDim.x) {
    T* row = X + rho * R;
    for (uint32_t q = threadIdx.x; q < R; q += blockDim.x) Z[q] = row[q];
    __syncthreads();
    RowTw<F> tw{W, Wih, L, &s_rt, rho, lr};
    inv_full<F>(Z, 0, 0, lr, tw);
    for (uint32_t q = threadIdx.x; q < R; q += blockDim.x)
      row[q] = F::canon(Z[q]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Fused product row pass, persistent over rows.  For a full row rho < a the
// two column-transformed operands (A' in out, B' in work) are interleaved as
// a two-column tile, both run the forward row network, are multiplied
// pointwise (C^_s = A^_s B^_s), and the product runs the inverse row network;
// the result goes back to out.  The last row (rho = a, first b outputs) only
// gets the forward half and the pointwise product: its inverse needs the
// inverse column pass first.
// ---------------------------------------------------------------------------
template <class F>
__global__ void __launch_bounds__(512)
k_row_mul(typename F::T* out, const typename F::T* __restrict__ work,
          const typename F::T* __restrict__ EA,
          const typename F::T* __restrict__ EB, int lr, uint64_t a, uint64_t b,
          int only_last, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  load_roots<F>(&s_rt, rt);
  const uint32_t R = 1u << lr;
  T* Z = reinterpret_cast<T*>(smem_raw);  // 2R
  T* W = Z + 2 * R;
  T* Wih = W + R / 2;
  T* L = Wih + R / 2;
  build_base_tables<F>(W, Wih, lr, s_rt);
  const uint64_t nrows = only_last ? 1 : a + (b > 0 ? 1 : 0);
  for (uint64_t it = blockIdx.x; it < nrows; it += gridDim.x) {
    const uint64_t rho =
        only_last ? a : ((b > 0) ? (it == 0 ? a : it - 1) : it);
    const bool last = rho == a;
    T* orow = out + rho * R;
    const T* wrow = work + rho * R;
    for (uint32_t q = threadIdx.x; q < R; q += blockDim.x) {
      const bool mem = !last || q < b;
      Z[2 * q] = mem ? orow[q] : EA[q];
      Z[2 * q + 1] = mem ? wrow[q] : EB[q];
    }
    __syncthreads();
    RowTw<F> tw{W, Wih, L, &s_rt, rho, lr};
    const uint32_t nout = last ? (uint32_t)b : R;
    fwd_pruned<F>(Z, 1, 1, lr, nout, tw);
    for (uint32_t q = threadIdx.x; q < nout; q += blockDim.x)
      Z[2 * q] = F::mul_data(Z[2 * q], Z[2 * q + 1]);
    __syncthreads();
    if (!last) inv_full<F>(Z, 0, 1, lr, tw);
    for (uint32_t q = threadIdx.x; q < nout; q += blockDim.x)
      orow[q] = F::canon(Z[2 * q]);
    __syncthreads();
  }
}

// Many single-CTA transforms of uneven lengths in one launch: each CTA
// takes table entries blockIdx.x, blockIdx.x + gridDim.x, ... and runs the
// whole transform of each (the k_small body) in shared memory sized for
// the largest.
template <class F, bool INV>
__global__ void __launch_bounds__(512)
k_small_batch(const XformDesc* __restrict__ d, uint32_t count,
              RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  load_roots<F>(&s_rt, rt);
  T* Z = reinterpret_cast<T*>(smem_raw);
  for (uint32_t p = blockIdx.x; p < count; p += gridDim.x) {
    const XformDesc q = d[p];
    const int l = (int)q.l;
    const uint32_t N = 1u << l, n = q.n;
    T* x = reinterpret_cast<T*>(q.x);
    T* W = Z + N;
    T* Wih = W + (N > 1 ? N / 2 : 1);
    __syncthreads();  // the previous transform is done with shared memory
    build_base_tables<F>(W, INV ? Wih : nullptr, l, s_rt);
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
      Z[i] = i < n ? x[i] : T(0);
    __syncthreads();
    ColTw<F> tw{W, Wih};
    if (!INV)
      fwd_pruned<F>(Z, 0, 0, l, n, tw);
    else
      inv_block<F>(Z, 0, 0, l, n, tw);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
      x[i] = F::canon(Z[i]);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <class F>
static size_t smem_small(int l, bool inv) {
  const size_t N = 1ull << l;
  return (N + 2 * (N > 1 ? N / 2 : 1)) * sizeof(typename F::T);
}
template <class F>
static size_t smem_small_mul(int l) {
  const size_t N = 1ull << l;
  return (2 * N + 2 * (N > 1 ? N / 2 : 1)) * sizeof(typename F::T);
}
template <class F>
static size_t smem_col(int c, int clog, bool inv) {
  const size_t N = 1ull << c;
  size_t tab = inv ? 2 * (N > 1 ? N / 2 : 1) : (N > 1 ? N / 2 : 1);
  if (inv && tab < 512) tab = 512;  // the Horner reduction reuses it
  return ((N << clog) + tab) * sizeof(typename F::T);
}
template <class F>
static size_t smem_row(int lr, int kind) {
  const size_t R = 1ull << lr;
  switch (kind) {
    case 0: return (R + R / 2 + R / 2) * sizeof(typename F::T);      // fwd
    case 1: return (R + 3 * (R / 2)) * sizeof(typename F::T);        // inv
    default: return (2 * R + 3 * (R / 2)) * sizeof(typename F::T);   // mul
  }
}

// Allow each kernel the device's opt-in shared memory minus its own static
// shared memory (the per-CTA copy of the root table).
template <class F>
static cudaError_t set_smem(const void* fn, size_t optin) {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, fn);
  if (e != cudaSuccess) return e;
  const size_t dyn = optin > at.sharedSizeBytes ? optin - at.sharedSizeBytes : 0;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dyn);
  if (e != cudaSuccess) return e;
  // prefer the largest shared-memory carve-out, so that as many CTAs as
  // the registers allow can also fit their tiles
  return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// Launch with the optional hook around it (H and s in scope).
#define TFT_LAUNCH(kind, ...)                        \
  do {                                               \
    if (H) H->before(H->user, (kind), s);            \
    __VA_ARGS__;                                     \
    if (H) H->after(H->user, (kind), s);             \
  } while (0)
#define TFT_LAUNCH_ON(kind, strm, ...)               \
  do {                                               \
    if (H) H->before(H->user, (kind), (strm));       \
    __VA_ARGS__;                                     \
    if (H) H->after(H->user, (kind), (strm));        \
  } while (0)

template <class F>
struct Launch {
  using T = typename F::T;
  using RT = RootTable<T>;

#define TFT_PREP_LR(LRV)                                                   \
  do {                                                                     \
    if ((e = set_smem<F>((const void*)k_row_fwd2<F, LRV>, mx))) return e;  \
    if ((e = set_smem<F>((const void*)k_row_inv2<F, LRV>, mx))) return e;  \
    if ((e = set_smem<F>((const void*)k_row_mul2<F, LRV>, mx))) return e;  \
    if ((e = set_smem<F>((const void*)k_row_last2<F, LRV>, mx))) return e; \
  } while (0)

  static cudaError_t prepare(size_t mx) {
    cudaError_t e;
    if ((e = set_smem<F>((const void*)k_col_fwd2<F, 256>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_col_inv2<F, 256>, mx))) return e;

    if ((e = set_smem<F>((const void*)k_small<F, false>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_small<F, true>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_small_batch<F, false>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_small_batch<F, true>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_small_mul<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_row_fwd<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_row_inv<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_row_mul<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_lastrow_inv2<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_lastrow_cluster<F, false>, mx)))
      return e;
    if ((e = set_smem<F>(
             (const void*)k_lastrow_cluster<typename ClusterField<F>::type,
                                            true>,
             mx)))
      return e;
    TFT_PREP_LR(8);
    TFT_PREP_LR(9);
    TFT_PREP_LR(10);
    TFT_PREP_LR(11);
    TFT_PREP_LR(12);
    TFT_PREP_LR(13);
    TFT_PREP_LR(14);
    return cudaSuccess;
  }

  // Full rows run on the register-blocked engine (rows.cuh) when lr >= 8:
  // R/16 threads per row, at least 256 threads per CTA.
  static bool use_v2(const Plan& P) { return P.lr >= 8; }
  template <class K>
  static uint32_t v2_grid(K kernel, int threads, size_t smem, uint64_t a,
                          int G, int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const uint64_t units = (a + G - 1) / G;
    const uint64_t cap = (uint64_t)nsm * per_sm;
    return (uint32_t)(units < cap ? units : cap);
  }

  static cudaError_t rows_fwd_v2(T* x, const Plan& P, const RT& rt, int nsm,
                                 cudaStream_t s, const LaunchHook* H) {
    TFT_LR_DISPATCH(P.lr, {
      using Geo = RowGeom<LR, 256>;
      const size_t sm = row_smem_bytes<T>(LR, Geo::G, 1);
      const uint32_t grid =
          v2_grid(k_row_fwd2<F, LR>, Geo::THREADS, sm, P.a, Geo::G, nsm);
      TFT_LAUNCH(K_ROW_FWD, k_row_fwd2<F, LR><<<grid, Geo::THREADS, sm, s>>>(
                                x, P.a, 0, rt));
    });
    return cudaGetLastError();
  }
  static cudaError_t rows_inv_v2(T* x, const Plan& P, const RT& rt, int nsm,
                                 cudaStream_t s, const LaunchHook* H) {
    TFT_LR_DISPATCH(P.lr, {
      using Geo = RowGeom<LR, 256>;
      const size_t sm = row_smem_bytes<T>(LR, Geo::G, 1);
      const uint32_t grid =
          v2_grid(k_row_inv2<F, LR>, Geo::THREADS, sm, P.a, Geo::G, nsm);
      TFT_LAUNCH(K_ROW_INV, k_row_inv2<F, LR><<<grid, Geo::THREADS, sm, s>>>(
                                x, P.a, 0, rt));
    });
    return cudaGetLastError();
  }
  static cudaError_t rows_mul_v2(T* out, const T* work, T* EA, const T* EB,
                                 const Plan& P, const RT& rt, int nsm,
                                 cudaStream_t s, const LaunchHook* H) {
    TFT_LR_DISPATCH(P.lr, {
      using Geo = RowGeom<LR>;
      const size_t sm = row_smem_bytes<T>(LR, Geo::G, 2);
      const uint32_t grid =
          v2_grid(k_row_mul2<F, LR>, Geo::THREADS, sm,
                  P.a + (P.b > 0 ? 1 : 0), Geo::G, nsm);
      TFT_LAUNCH(K_ROW_MUL, k_row_mul2<F, LR><<<grid, Geo::THREADS, sm, s>>>(
                                out, work, EA, EB, P.a, P.b, rt));
    });
    return cudaGetLastError();
  }

  // Forward column pass on the stage engine: C = 2^clog columns per CTA,
  // 16 elements per thread and stage, at most 256 threads.
  static cudaError_t cols_fwd_v2(const T* src, uint64_t n_src, T* dst, T* E,
                                 const Plan& P, const RT& rt, int nsm,
                                 cudaStream_t s, const LaunchHook* H) {
    const uint32_t R = 1u << P.lr;
    const int cl = set_clog(P, R, nsm);
    const uint32_t C = 1u << cl;
    const uint64_t units = (uint64_t)C << (P.c > 4 ? P.c - 4 : 0);
    const int th = units >= 256 ? 256 : (units < 32 ? 32 : (int)units);
    const size_t sm = col_smem_bytes<T>(P.c, cl);
    TFT_LAUNCH(K_COL_FWD, k_col_fwd2<F, 256><<<(R + C - 1) / C, th, sm, s>>>(
                              src, n_src, dst, E, P.lr, P.a, P.b, P.c, cl, 0,
                              R, rt));
    return cudaGetLastError();
  }

  // Run `launch(stream)` for the ragged last row on the side stream, forked
  // after the work already queued on s; join() makes s wait for it.
  struct SideRow {
    const AuxStreams* aux;
    cudaStream_t s;
    cudaStream_t side() const { return aux ? aux->side : s; }
    void fork() const {
      if (aux) {
        cudaEventRecord(aux->fork, s);
        cudaStreamWaitEvent(aux->side, aux->fork, 0);
      }
    }
    void join() const {
      if (aux) {
        cudaEventRecord(aux->join, aux->side);
        cudaStreamWaitEvent(s, aux->join, 0);
      }
    }
  };

  static cudaError_t forward(T* x, uint64_t n, const Plan& P, T* E,
                             const RT& rt, int nsm, cudaStream_t s,
                             const LaunchHook* H, const AuxStreams* aux) {
    if (P.small) {
      TFT_LAUNCH(K_SMALL, k_small<F, false><<<1, 512,
                                              smem_small<F>(P.l, false), s>>>(
                              x, (uint32_t)n, P.l, rt));
      return cudaGetLastError();
    }
    cols_fwd_v2(x, n, x, E, P, rt, nsm, s, H);
    if (!use_v2(P)) {
      const uint64_t rows = P.a + (P.b ? 1 : 0);
      const uint32_t grid =
          (uint32_t)(rows < (uint64_t)nsm * P.row_ctas_per_sm
                         ? rows
                         : (uint64_t)nsm * P.row_ctas_per_sm);
      TFT_LAUNCH(K_ROW_FWD,
                 k_row_fwd<F><<<grid, 512, smem_row<F>(P.lr, 0), s>>>(
                     x, E, P.lr, P.a, P.b, 0, rt));
      return cudaGetLastError();
    }
    const SideRow side{aux, s};
    if (P.b > 0) {
      side.fork();
      cudaStream_t s2 = side.side();
      TFT_LR_DISPATCH(P.lr, {
        using Geo = RowGeom<LR>;
        TFT_LAUNCH_ON(K_LASTROW_FWD, s2,
                      (k_row_last2<F, LR><<<1, Geo::THREADS,
                                            row_smem_bytes<T>(LR, Geo::G, 1),
                                            s2>>>(x + P.a * (1ull << LR), E,
                                                  P.a, P.b, rt)));
      });
    }
    cudaError_t e = rows_fwd_v2(x, P, rt, nsm, s, H);
    if (P.b > 0) side.join();
    return e != cudaSuccess ? e : cudaGetLastError();
  }

  // Columns per tile for an inverse column set of `cols` columns: the
  // plan's, halved while the set would give fewer tiles than SMs (the long
  // columns are often a small set).
  static int set_clog(const Plan& P, uint32_t cols, int nsm) {
    int cl = P.clog;
    while (cl > 0 && ((cols + (1u << cl) - 1) >> cl) < (uint32_t)nsm) --cl;
    return cl;
  }

  // in_scale_log: the rows' inverse left its factor 2^lr in x (the fused
  // product rows); 0 when the rows are exact.
  static cudaError_t inverse_tail(T* x, const Plan& P, T* E, T omega_a_tw,
                                  int in_scale_log, const RT& rt, int nsm,
                                  cudaStream_t s, const LaunchHook* H) {
    const uint32_t R = 1u << P.lr;
    // short columns q in [b, R): length a, and E_q = C_q(omega_a)
    if (P.a > 0 && P.b < R) {
      const uint32_t qb = (uint32_t)P.b;
      const int cl = set_clog(P, R - qb, nsm);
      const uint32_t C = 1u << cl;
      TFT_LAUNCH(K_COL_INV,
                 k_col_inv2<F, 256><<<(R - qb + C - 1) / C, 256,
                                      col_smem_bytes<T>(P.c, cl), s>>>(
                     x, E, P.lr, (uint32_t)P.a, P.c, cl, qb, R,
                     P.b > 0 ? 1 : 0, omega_a_tw, in_scale_log, rt, ~0ull,
                     nullptr));
    }
    if (P.b > 0) {
      TFT_LAUNCH(K_LASTROW_INV,
                 k_lastrow_inv2<F><<<1, 512, col_smem_bytes<T>(P.lr, 0), s>>>(
                     x + P.a * (uint64_t)R, E, P.lr, P.a, P.b, rt));
      const uint32_t qe = (uint32_t)P.b;
      const int cl = set_clog(P, qe, nsm);
      const uint32_t C = 1u << cl;
      TFT_LAUNCH(K_COL_INV,
                 k_col_inv2<F, 256><<<(qe + C - 1) / C, 256,
                                      col_smem_bytes<T>(P.c, cl), s>>>(
                     x, E, P.lr, (uint32_t)(P.a + 1), P.c, cl, 0, qe, 0,
                     omega_a_tw, in_scale_log, rt, ~0ull, nullptr));
    }
    return cudaGetLastError();
  }

  static cudaError_t small_batch(const XformDesc* d, uint32_t count, int lmax,
                                 bool inv, const RT& rt, int nsm,
                                 cudaStream_t s, const LaunchHook* H) {
    if (count == 0) return cudaSuccess;
    const size_t sm = smem_small<F>(lmax, inv);
    if (inv) {
      const uint32_t grid =
          persistent_grid(k_small_batch<F, true>, 512, sm, count, nsm);
      TFT_LAUNCH(K_SMALL,
                 k_small_batch<F, true><<<grid, 512, sm, s>>>(d, count, rt));
    } else {
      const uint32_t grid =
          persistent_grid(k_small_batch<F, false>, 512, sm, count, nsm);
      TFT_LAUNCH(K_SMALL,
                 k_small_batch<F, false><<<grid, 512, sm, s>>>(d, count, rt));
    }
    return cudaGetLastError();
  }

  // ---- pieces of a transform held in parts (a sharded transform) ---------
  // A part holds a block of W = 2^{Pc.lr} adjacent columns of the R-wide
  // view, (a + 1) x W words at row stride W, and/or a run of full rows.
  // Pc is the transform's plan with lr = log2 W and b = the block's long
  // columns (the column transforms do not depend on which columns they
  // are, so the block is a column pass of its own).
  //   dir 0: forward columns, long and short, E[j] = C_j(omega_a) for the
  //          short ones (want_E);
  //   dir 1, which 0: inverse of the short columns (length a), with E;
  //   dir 1, which 1: inverse of the long columns (length a + 1, row a
  //          already holding the last row's inverse).
  static cudaError_t shard_cols(int dir, int which, T* blk, const Plan& Pc,
                                T* E, int want_E, T omega_a_tw, const RT& rt,
                                int nsm, cudaStream_t s, const LaunchHook* H) {
    const uint32_t W = 1u << Pc.lr;
    if (dir == 0 && want_E && Pc.b == 0) {
      // every column of the block is short but the transform has a ragged
      // row: the column pass produces row a (C_q(omega_a), the padded
      // transform's output there) only for long columns, so run the block
      // as all-long columns whose row-a inputs are zero (positions >= a W
      // read as zero) and take E from the block's row a
      Plan P2 = Pc;
      P2.b = W;
      cudaError_t e = cols_fwd_v2(blk, Pc.a * (uint64_t)W, blk, nullptr, P2,
                                  rt, nsm, s, H);
      if (e != cudaSuccess) return e;
      return cudaMemcpyAsync(E, blk + Pc.a * (uint64_t)W, W * sizeof(T),
                             cudaMemcpyDeviceToDevice, s);
    }
    if (dir == 0)
      return cols_fwd_v2(blk, Pc.a * (uint64_t)W + Pc.b, blk, want_E ? E
                                                                       : nullptr,
                         Pc, rt, nsm, s, H);
    if (which == 0) {
      if (Pc.a == 0 || Pc.b >= W) return cudaSuccess;
      const uint32_t qb = (uint32_t)Pc.b;
      const int cl = set_clog(Pc, W - qb, nsm);
      const uint32_t C = 1u << cl;
      TFT_LAUNCH(K_COL_INV,
                 k_col_inv2<F, 256><<<(W - qb + C - 1) / C, 256,
                                      col_smem_bytes<T>(Pc.c, cl), s>>>(
                     blk, E, Pc.lr, (uint32_t)Pc.a, Pc.c, cl, qb, W, want_E,
                     omega_a_tw, 0, rt, ~0ull, nullptr));
      return cudaGetLastError();
    }
    if (Pc.b == 0) return cudaSuccess;
    const uint32_t qe = (uint32_t)Pc.b;
    const int cl = set_clog(Pc, qe, nsm);
    const uint32_t C = 1u << cl;
    TFT_LAUNCH(K_COL_INV,
               k_col_inv2<F, 256><<<(qe + C - 1) / C, 256,
                                    col_smem_bytes<T>(Pc.c, cl), s>>>(
                   blk, nullptr, Pc.lr, (uint32_t)(Pc.a + 1), Pc.c, cl, 0, qe,
                   0, omega_a_tw, 0, rt, ~0ull, nullptr));
    return cudaGetLastError();
  }
  // count full rows of 2^lr words at `rows`, rows rho_off .. of the view
  static cudaError_t shard_rows(int dir, T* rows, uint64_t count,
                                uint64_t rho_off, int lr, const RT& rt,
                                int nsm, cudaStream_t s, const LaunchHook* H) {
    if (count == 0) return cudaSuccess;
    TFT_LR_DISPATCH(lr, {
      using Geo = RowGeom<LR, 256>;
      const size_t sm = row_smem_bytes<T>(LR, Geo::G, 1);
      if (dir == 0) {
        const uint32_t grid =
            v2_grid(k_row_fwd2<F, LR>, Geo::THREADS, sm, count, Geo::G, nsm);
        TFT_LAUNCH(K_ROW_FWD,
                   k_row_fwd2<F, LR><<<grid, Geo::THREADS, sm, s>>>(
                       rows, count, rho_off, rt));
      } else {
        const uint32_t grid =
            v2_grid(k_row_inv2<F, LR>, Geo::THREADS, sm, count, Geo::G, nsm);
        TFT_LAUNCH(K_ROW_INV,
                   k_row_inv2<F, LR><<<grid, Geo::THREADS, sm, s>>>(
                       rows, count, rho_off, rt));
      }
    });
    return cudaGetLastError();
  }
  // the ragged last row (row a, b outputs) from an R-word row and E
  static cudaError_t shard_last(int dir, T* row, const T* E, uint64_t a,
                                uint64_t b, int lr, const RT& rt,
                                cudaStream_t s, const LaunchHook* H) {
    if (b == 0) return cudaSuccess;
    if (dir == 0) {
      TFT_LR_DISPATCH(lr, {
        using Geo = RowGeom<LR>;
        TFT_LAUNCH(K_LASTROW_FWD,
                   (k_row_last2<F, LR><<<1, Geo::THREADS,
                                         row_smem_bytes<T>(LR, Geo::G, 1),
                                         s>>>(row, E, a, b, rt)));
      });
    } else {
      TFT_LAUNCH(K_LASTROW_INV,
                 k_lastrow_inv2<F><<<1, 512, col_smem_bytes<T>(lr, 0), s>>>(
                     row, E, lr, a, b, rt));
    }
    return cudaGetLastError();
  }

  // ---- transforms without global scratch ---------------------------------
  // Forward column pass over columns [q0, q1) with b_arg as the plan's b
  // (b_arg = 0: columns of length a, no row a), no E.
  static cudaError_t cols_fwd_range(T* x, uint64_t n, const Plan& P,
                                    uint64_t b_arg, uint32_t q0, uint32_t q1,
                                    const RT& rt, int nsm, cudaStream_t s,
                                    const LaunchHook* H) {
    const int cl = set_clog(P, q1 - q0, nsm);
    const uint32_t C = 1u << cl;
    const uint64_t units = (uint64_t)C << (P.c > 4 ? P.c - 4 : 0);
    const int th = units >= 256 ? 256 : (units < 32 ? 32 : (int)units);
    TFT_LAUNCH(K_COL_FWD,
               k_col_fwd2<F, 256><<<(q1 - q0 + C - 1) / C, th,
                                    col_smem_bytes<T>(P.c, cl), s>>>(
                   x, n, x, nullptr, P.lr, P.a, b_arg, P.c, cl, q0, q1, rt));
    return cudaGetLastError();
  }
  static cudaError_t lastrow_cluster(T* x, const Plan& P, T omega_a_tw,
                                     bool inv, const RT& rt, cudaStream_t s,
                                     const LaunchHook* H) {
    const size_t sm = lastrow_cluster_smem<T>(P.lr, P.b);
    if (inv)
      TFT_LAUNCH(K_LASTROW_INV,
                 (k_lastrow_cluster<typename ClusterField<F>::type, true>
                  <<<kLastRowCluster, 512, sm, s>>>(
                     x, P.lr, P.a, P.b, omega_a_tw, rt)));
    else
      TFT_LAUNCH(K_LASTROW_FWD,
                 (k_lastrow_cluster<F, false><<<kLastRowCluster, 512, sm, s>>>(
                     x, P.lr, P.a, P.b, omega_a_tw, rt)));
    return cudaGetLastError();
  }
  // Forward TFT touching no memory but x: long columns (their row a in
  // place), the last row from the raw short columns (lastrow_cluster.cuh),
  // the short columns (length a), the full rows.
  static cudaError_t forward_zs(T* x, uint64_t n, const Plan& P, T omega_a_tw,
                                const RT& rt, int nsm, cudaStream_t s,
                                const LaunchHook* H) {
    if (P.small || P.b == 0)  // no ragged row: the plain forward uses no E
      return forward(x, n, P, nullptr, rt, nsm, s, H, nullptr);
    const uint32_t R = 1u << P.lr;
    cudaError_t e = cols_fwd_range(x, n, P, P.b, 0, (uint32_t)P.b, rt, nsm,
                                   s, H);
    if (e == cudaSuccess) e = lastrow_cluster(x, P, omega_a_tw, false, rt, s, H);
    if (e == cudaSuccess)
      e = cols_fwd_range(x, n, P, 0, (uint32_t)P.b, R, rt, nsm, s, H);
    if (e != cudaSuccess) return e;
    if (use_v2(P)) return rows_fwd_v2(x, P, rt, nsm, s, H);
    const uint32_t grid = (uint32_t)(P.a < (uint64_t)nsm * P.row_ctas_per_sm
                                         ? P.a
                                         : (uint64_t)nsm * P.row_ctas_per_sm);
    TFT_LAUNCH(K_ROW_FWD, k_row_fwd<F><<<grid, 512, smem_row<F>(P.lr, 0), s>>>(
                              x, nullptr, P.lr, P.a, 0, 0, rt));
    return cudaGetLastError();
  }
  // Inverse TFT touching no memory but x: full rows, short columns, the
  // last row with E_q from the recovered short columns, long columns.
  static cudaError_t inverse_zs(T* x, uint64_t n, const Plan& P, T omega_a_tw,
                                const RT& rt, int nsm, cudaStream_t s,
                                const LaunchHook* H) {
    if (P.small || P.b == 0)  // no ragged row: the plain inverse uses no E
      return inverse(x, n, P, nullptr, omega_a_tw, rt, nsm, s, H);
    const uint32_t R = 1u << P.lr;
    if (use_v2(P)) {
      cudaError_t e = rows_inv_v2(x, P, rt, nsm, s, H);
      if (e != cudaSuccess) return e;
    } else {
      const uint32_t grid = (uint32_t)(P.a < (uint64_t)nsm * P.row_ctas_per_sm
                                           ? P.a
                                           : (uint64_t)nsm * P.row_ctas_per_sm);
      TFT_LAUNCH(K_ROW_INV,
                 k_row_inv<F><<<grid, 512, smem_row<F>(P.lr, 1), s>>>(
                     x, P.lr, P.a, rt));
    }
    const uint32_t qb = (uint32_t)P.b;
    {
      const int cl = set_clog(P, R - qb, nsm);
      const uint32_t C = 1u << cl;
      TFT_LAUNCH(K_COL_INV,
                 k_col_inv2<F, 256><<<(R - qb + C - 1) / C, 256,
                                      col_smem_bytes<T>(P.c, cl), s>>>(
                     x, nullptr, P.lr, (uint32_t)P.a, P.c, cl, qb, R, 0,
                     omega_a_tw, 0, rt, ~0ull, nullptr));
    }
    cudaError_t e = lastrow_cluster(x, P, omega_a_tw, true, rt, s, H);
    if (e != cudaSuccess) return e;
    {
      const int cl = set_clog(P, qb, nsm);
      const uint32_t C = 1u << cl;
      TFT_LAUNCH(K_COL_INV,
                 k_col_inv2<F, 256><<<(qb + C - 1) / C, 256,
                                      col_smem_bytes<T>(P.c, cl), s>>>(
                     x, nullptr, P.lr, (uint32_t)(P.a + 1), P.c, cl, 0, qb, 0,
                     omega_a_tw, 0, rt, ~0ull, nullptr));
    }
    return cudaGetLastError();
  }

  static cudaError_t inverse(T* x, uint64_t n, const Plan& P, T* E,
                             T omega_a_tw, const RT& rt, int nsm,
                             cudaStream_t s, const LaunchHook* H) {
    if (P.small) {
      TFT_LAUNCH(K_SMALL, k_small<F, true><<<1, 512, smem_small<F>(P.l, true),
                                             s>>>(x, (uint32_t)n, P.l, rt));
      return cudaGetLastError();
    }
    if (P.a > 0 && use_v2(P)) {
      cudaError_t e = rows_inv_v2(x, P, rt, nsm, s, H);
      if (e != cudaSuccess) return e;
    } else if (P.a > 0) {
      const uint32_t grid = (uint32_t)(P.a < (uint64_t)nsm * P.row_ctas_per_sm
                                           ? P.a
                                           : (uint64_t)nsm * P.row_ctas_per_sm);
      TFT_LAUNCH(K_ROW_INV,
                 k_row_inv<F><<<grid, 512, smem_row<F>(P.lr, 1), s>>>(
                     x, P.lr, P.a, rt));
    }
    return inverse_tail(x, P, E, omega_a_tw, 0, rt, nsm, s, H);
  }

  static cudaError_t polymul(const T* a, uint64_t na, const T* b, uint64_t nb,
                             T* out, const Plan& P, T* work, T* EA, T* EB,
                             T omega_a_tw, const RT& rt, int nsm,
                             cudaStream_t s, const LaunchHook* H,
                             const AuxStreams* aux) {
    if (P.small) {
      TFT_LAUNCH(K_SMALL_MUL,
                 k_small_mul<F><<<1, 512, smem_small_mul<F>(P.l), s>>>(
                     a, (uint32_t)na, b, (uint32_t)nb, out, P.l, rt));
      return cudaGetLastError();
    }
    {
      // the two operands' column passes are independent: B's runs on the
      // side stream next to A's
      const SideRow side{aux, s};
      side.fork();
      cols_fwd_v2(b, nb, work, EB, P, rt, nsm, side.side(), H);
      cols_fwd_v2(a, na, out, EA, P, rt, nsm, s, H);
      side.join();
    }
    if (!use_v2(P)) {
      const uint64_t rows = P.a + (P.b ? 1 : 0);
      const uint32_t grid =
          (uint32_t)(rows < (uint64_t)nsm * P.row_ctas_per_sm
                         ? rows
                         : (uint64_t)nsm * P.row_ctas_per_sm);
      TFT_LAUNCH(K_ROW_MUL,
                 k_row_mul<F><<<grid, 512, smem_row<F>(P.lr, 2), s>>>(
                     out, work, EA, EB, P.lr, P.a, P.b, 0, rt));
      return inverse_tail(out, P, EA, omega_a_tw, 0, rt, nsm, s, H);
    }
    // The product's transforms have length (a + 1) R when b > 0 (r rounded
    // up to a multiple of R; a TFT of any length >= r determines the
    // product): the forward column pass already produced every column's
    // entry in row a, with the positions past r in EA / EB.  The row pass
    // then treats row a as a full row, and the inverse is one column pass of
    // length a + 1 over all columns; no ragged last row, no E_q, no long
    // column pass.
    cudaError_t e = rows_mul_v2(out, work, EA, EB, P, rt, nsm, s, H);
    if (e != cudaSuccess) return e;
    if (P.b == 0)
      return inverse_tail(out, P, EA, omega_a_tw, P.lr, rt, nsm, s, H);
    const uint32_t R = 1u << P.lr;
    const int cl = set_clog(P, R, nsm);
    const uint32_t C = 1u << cl;
    TFT_LAUNCH(K_COL_INV,
               k_col_inv2<F, 256><<<(R + C - 1) / C, 256,
                                    col_smem_bytes<T>(P.c, cl), s>>>(
                   out, nullptr, P.lr, (uint32_t)(P.a + 1), P.c, cl, 0, R, 0,
                   omega_a_tw, P.lr, rt, P.a * (uint64_t)R + P.b, EA));
    return cudaGetLastError();
  }
  // Persistent grid: the SMs times the resident CTAs of `kernel`.
  template <class K>
  static uint32_t persistent_grid(K kernel, int threads, size_t smem,
                                  uint64_t tasks, int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const uint64_t cap = (uint64_t)nsm * per_sm;
    return (uint32_t)(tasks < cap ? (tasks ? tasks : 1) : cap);
  }

  static cudaError_t prepare_batch(size_t mx) {
    cudaError_t e;
    if ((e = set_smem<F>((const void*)k_small_mul_batch<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_col_fwd_batch<F>, mx))) return e;
    if ((e = set_smem<F>((const void*)k_col_inv_batch<F>, mx))) return e;
#define TFT_PREP_BATCH_LR(LRV)                                             \
  if ((e = set_smem<F>((const void*)k_row_mul_batch<F, LRV>, mx))) return e;
    TFT_PREP_BATCH_LR(8)
    TFT_PREP_BATCH_LR(9)
    TFT_PREP_BATCH_LR(10)
    TFT_PREP_BATCH_LR(11)
    TFT_PREP_BATCH_LR(12)
#undef TFT_PREP_BATCH_LR
    return cudaSuccess;
  }

  // A planned batch: the small class on the side stream, the three phases
  // of the large class on the caller's stream.
  static cudaError_t batch(const BatchLaunch& B, const RT& rt, int nsm,
                           cudaStream_t s, const LaunchHook* H,
                           const AuxStreams* aux) {
    const SideRow side{aux, s};
    if (B.ns) {
      side.fork();
      cudaStream_t s2 = side.side();
      const size_t sm = smem_small_mul<F>(B.lmax);
      const uint32_t grid =
          persistent_grid(k_small_mul_batch<F>, 512, sm, B.ns, nsm);
      TFT_LAUNCH_ON(K_SMALL_MUL, s2,
                    (k_small_mul_batch<F><<<grid, 512, sm, s2>>>(
                        (const BatchSmall*)B.small, B.ns, B.lmax, rt)));
    }
    if (B.nl) {
      const BatchLarge* d = (const BatchLarge*)B.large;
      const uint32_t R = 1u << B.lr;
      const size_t smc = col_smem_bytes<T>(B.cmax, B.clog);
      // the products are sorted by column height: when the shorter ones'
      // tiles let more CTAs reside per SM, their column passes run as a
      // launch of their own with the smaller tiles
      // a schedule may give that class its own tile width (clog_lo)
      uint32_t nlo = 0;
      size_t smlo = smc;
      if (B.nl_lo > 0 && B.nl_lo < B.nl) {
        const size_t sm1 = col_smem_bytes<T>(B.cmax_lo, B.clog_lo);
        int o0 = 0, o1 = 0;
        if (B.clog_lo != B.clog ||
            (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &o0, k_col_fwd_batch<F>, 256, smc) == cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &o1, k_col_fwd_batch<F>, 256, sm1) == cudaSuccess &&
             o1 > o0)) {
          nlo = B.nl_lo;
          smlo = sm1;
        }
      }
      auto col_fwd = [&](const BatchLarge* dd, uint32_t np, size_t sm,
                         int cl) {
        const uint64_t tasks = (uint64_t)np * 2 * (R >> cl);
        TFT_LAUNCH(K_COL_FWD,
                   (k_col_fwd_batch<F><<<persistent_grid(k_col_fwd_batch<F>,
                                                         256, sm, tasks, nsm),
                                         256, sm, s>>>(dd, np, B.lr, cl,
                                                       rt)));
      };
      auto col_inv = [&](const BatchLarge* dd, uint32_t np, size_t sm,
                         int cl) {
        const uint64_t tasks = (uint64_t)np * (R >> cl);
        TFT_LAUNCH(K_COL_INV,
                   (k_col_inv_batch<F><<<persistent_grid(k_col_inv_batch<F>,
                                                         256, sm, tasks, nsm),
                                         256, sm, s>>>(dd, np, tasks, B.lr,
                                                       cl, rt)));
      };
      if (nlo) col_fwd(d, nlo, smlo, B.clog_lo);
      col_fwd(d + nlo, B.nl - nlo, smc, B.clog);
      TFT_LR_DISPATCH_BATCH(B.lr, {
        using Geo = RowGeom<LR>;
        // the row prefix goes to shared memory when its values fit 32 bits
        // and the extra bytes cost no resident CTA
        const size_t smr0 = row_smem_bytes<T>(LR, Geo::G, 2);
        const size_t smr1 = smr0 + 4 * (size_t)B.nl;
        int occ0 = 0, occ1 = 0;
        const int cache =
            B.total_rows < (1ull << 32) &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ0, k_row_mul_batch<F, LR>, Geo::THREADS, smr0) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ1, k_row_mul_batch<F, LR>, Geo::THREADS, smr1) ==
                cudaSuccess &&
            occ1 >= occ0 && occ1 > 0;
        const size_t smr = cache ? smr1 : smr0;
        const uint64_t slots = (B.total_rows + Geo::G - 1) / Geo::G;
        TFT_LAUNCH(K_ROW_MUL,
                   (k_row_mul_batch<F, LR><<<persistent_grid(
                                                 k_row_mul_batch<F, LR>,
                                                 Geo::THREADS, smr, slots,
                                                 nsm),
                                             Geo::THREADS, smr, s>>>(
                       d, B.nl, B.total_rows, cache, rt)));
      });
      if (nlo) col_inv(d, nlo, smlo, B.clog_lo);
      col_inv(d + nlo, B.nl - nlo, smc, B.clog);
    }
    if (B.ns) side.join();
    return cudaGetLastError();
  }
};

// Shared-memory bytes of each kernel for a plan (used by the planner).
template <class F>
static PlanSmem smem_of(const Plan& P) {
  PlanSmem m{};
  if (P.small) {
    m.col = smem_small<F>(P.l, true);
    m.row = smem_small_mul<F>(P.l);
    return m;
  }
  m.col = smem_col<F>(P.c, P.clog, true);
  m.row = smem_row<F>(P.lr, 2);
  return m;
}

// ---------------------------------------------------------------------------
// Launchers of the space-restricted product's kernels (alg3.cuh)
// ---------------------------------------------------------------------------
static inline uint32_t flat_grid(uint64_t work, uint64_t per_block, int nsm) {
  const uint64_t blocks = (work + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)nsm * 8;
  return (uint32_t)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

template <class F>
static cudaError_t launch_fold(void* d0, const void* s0, uint64_t n0,
                               void* d1, const void* s1, uint64_t n1,
                               uint64_t L, int ell, const void* powers,
                               int nsm, cudaStream_t s) {
  using T = typename F::T;
  // warps per coefficient block (1, 2, 4 or 8): enough threads to fill
  // the GPU, at least two terms per lane
  const uint64_t nmax = n0 > n1 ? n0 : n1;
  const uint64_t target = (uint64_t)nsm * 2048;
  int glog = 0;
  while (glog < 3 && (L << glog) < target && ((nmax / L) >> glog) >= 2)
    ++glog;
  const uint64_t per_cta = (uint64_t)32 * (8u >> glog);
  const uint64_t blocks = (L + per_cta - 1) / per_cta;
  const uint64_t cap = (uint64_t)nsm * 8;
  const dim3 grid((uint32_t)(blocks < cap ? blocks : cap), d1 ? 2 : 1);
  k_fold<F><<<grid, kFoldThreads, 0, s>>>(
      (T*)d0, (const T*)s0, n0, (T*)d1, (const T*)s1, n1, L, ell, glog,
      *(const FoldPowers<T>*)powers);
  return cudaGetLastError();
}

template <class F>
static cudaError_t launch_chunk_mul(void* X, const void* Y, uint64_t L,
                                   int nsm, cudaStream_t s) {
  using T = typename F::T;
  k_chunk_mul<F><<<flat_grid(L, 256, nsm), 256, 0, s>>>((T*)X, (const T*)Y,
                                                         L);
  return cudaGetLastError();
}

template <class F>
static cudaError_t launch_tail(void* X, const void* S, uint64_t Q,
                               uint64_t lo, uint64_t hi, int mul, int nsm,
                               cudaStream_t s) {
  using T = typename F::T;
  if (hi <= lo) return cudaSuccess;
  k_tail<F><<<flat_grid(hi - lo, 256, nsm), 256, 0, s>>>(
      (T*)X, (const T*)S, Q, lo, hi, mul);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-field entry points, defined once per field in kernels_<field>.cu
// (one translation unit per field so that they compile in parallel).
// ---------------------------------------------------------------------------
#define TFT_DEFINE_FIELD_ENTRIES(F, NAME)                                     \
  cudaError_t NAME##_prepare(size_t optin) {                                  \
    return Launch<F>::prepare(optin);                                         \
  }                                                                           \
  cudaError_t NAME##_forward(void* x, uint64_t n, const Plan& P, void* E,     \
                             const void* rt, int nsm, cudaStream_t s,         \
                             const LaunchHook* hook, const AuxStreams* aux) { \
    return Launch<F>::forward((F::T*)x, n, P, (F::T*)E,                       \
                              *(const RootTable<F::T>*)rt, nsm, s, hook,      \
                              aux);                                           \
  }                                                                           \
  cudaError_t NAME##_inverse(void* x, uint64_t n, const Plan& P, void* E,     \
                             uint64_t omega_a_tw, const void* rt, int nsm,    \
                             cudaStream_t s, const LaunchHook* hook) {        \
    return Launch<F>::inverse((F::T*)x, n, P, (F::T*)E, (F::T)omega_a_tw,     \
                              *(const RootTable<F::T>*)rt, nsm, s, hook);     \
  }                                                                           \
  cudaError_t NAME##_polymul(const void* a, uint64_t na, const void* b,       \
                             uint64_t nb, void* out, const Plan& P,           \
                             void* work, void* EA, void* EB,                  \
                             uint64_t omega_a_tw, const void* rt, int nsm,    \
                             cudaStream_t s, const LaunchHook* hook,          \
                             const AuxStreams* aux) {                         \
    return Launch<F>::polymul((const F::T*)a, na, (const F::T*)b, nb,         \
                              (F::T*)out, P, (F::T*)work, (F::T*)EA,          \
                              (F::T*)EB, (F::T)omega_a_tw,                    \
                              *(const RootTable<F::T>*)rt, nsm, s, hook,      \
                              aux);                                           \
  }                                                                           \
  PlanSmem NAME##_plan_smem(const Plan& P) { return smem_of<F>(P); }        \
  cudaError_t NAME##_forward_zs(void* x, uint64_t n, const Plan& P,           \
                                uint64_t omega_a_tw, const void* rt, int nsm, \
                                cudaStream_t s, const LaunchHook* hook) {     \
    return Launch<F>::forward_zs((F::T*)x, n, P, (F::T)omega_a_tw,            \
                                 *(const RootTable<F::T>*)rt, nsm, s, hook);  \
  }                                                                           \
  cudaError_t NAME##_inverse_zs(void* x, uint64_t n, const Plan& P,           \
                                uint64_t omega_a_tw, const void* rt, int nsm, \
                                cudaStream_t s, const LaunchHook* hook) {     \
    return Launch<F>::inverse_zs((F::T*)x, n, P, (F::T)omega_a_tw,            \
                                 *(const RootTable<F::T>*)rt, nsm, s, hook);  \
  }                                                                           \
  cudaError_t NAME##_small_batch(const void* d, uint32_t count, int lmax,     \
                                 int inverse, const void* rt, int nsm,        \
                                 cudaStream_t s, const LaunchHook* hook) {    \
    return Launch<F>::small_batch((const XformDesc*)d, count, lmax,           \
                                  inverse != 0, *(const RootTable<F::T>*)rt,  \
                                  nsm, s, hook);                              \
  }                                                                           \
  cudaError_t NAME##_shard_cols(int dir, int which, void* blk, const Plan& Pc, \
                                void* E, int want_E, uint64_t omega_a_tw,     \
                                const void* rt, int nsm, cudaStream_t s,      \
                                const LaunchHook* hook) {                     \
    return Launch<F>::shard_cols(dir, which, (F::T*)blk, Pc, (F::T*)E,        \
                                 want_E, (F::T)omega_a_tw,                    \
                                 *(const RootTable<F::T>*)rt, nsm, s, hook);  \
  }                                                                           \
  cudaError_t NAME##_shard_rows(int dir, void* rows, uint64_t count,          \
                                uint64_t rho_off, int lr, const void* rt,     \
                                int nsm, cudaStream_t s,                      \
                                const LaunchHook* hook) {                     \
    return Launch<F>::shard_rows(dir, (F::T*)rows, count, rho_off, lr,        \
                                 *(const RootTable<F::T>*)rt, nsm, s, hook);  \
  }                                                                           \
  cudaError_t NAME##_shard_last(int dir, void* row, const void* E, uint64_t a, \
                                uint64_t b, int lr, const void* rt,           \
                                cudaStream_t s, const LaunchHook* hook) {     \
    return Launch<F>::shard_last(dir, (F::T*)row, (const F::T*)E, a, b, lr,   \
                                 *(const RootTable<F::T>*)rt, s, hook);       \
  }

#define TFT_DEFINE_FIELD_BATCH(F, NAME)                                       \
  cudaError_t NAME##_fold(void* d0, const void* s0, uint64_t n0, void* d1,    \
                          const void* s1, uint64_t n1, uint64_t L, int ell,   \
                          const void* powers, int nsm, cudaStream_t s) {      \
    return launch_fold<F>(d0, s0, n0, d1, s1, n1, L, ell, powers, nsm, s);    \
  }                                                                           \
  cudaError_t NAME##_chunk_mul(void* X, const void* Y, uint64_t L, int nsm,   \
                               cudaStream_t s) {                              \
    return launch_chunk_mul<F>(X, Y, L, nsm, s);                              \
  }                                                                           \
  cudaError_t NAME##_tail(void* X, const void* S, uint64_t Q, uint64_t lo,    \
                          uint64_t hi, int mul, int nsm, cudaStream_t s) {    \
    return launch_tail<F>(X, S, Q, lo, hi, mul, nsm, s);                      \
  }                                                                           \
  cudaError_t NAME##_prepare_batch(size_t optin) {                            \
    return Launch<F>::prepare_batch(optin);                                   \
  }                                                                           \
  cudaError_t NAME##_batch(const BatchLaunch& B, const void* rt, int nsm,     \
                           cudaStream_t s, const LaunchHook* hook,            \
                           const AuxStreams* aux) {                           \
    return Launch<F>::batch(B, *(const RootTable<F::T>*)rt, nsm, s, hook,     \
                            aux);                                             \
  }

}  // namespace tftgb
