// Batched TFT products: many independent products in a handful of launches.
//
// Products are split into two size classes by r = na + nb - 1:
//   small (r <= 2^small_log): one CTA holds both operands in shared memory
//          (the single-CTA product), one product per task;
//   large: the row/column split with one row length R = 2^lr for the whole
//          class (a_p, b_p, c_p per product), run as three phase launches
//          over all large products: forward columns of both operands, fused
//          rows, inverse columns.  As in the single product, a product with
//          b_p > 0 runs its transforms at length (a_p + 1) R: row a_p is a
//          full row whose positions past r_p live in EA / EB, and every
//          column's inverse has length a_p + 1.
// Every kernel is persistent over its flattened task list (task -> product
// by a prefix table), so one launch per phase covers the whole batch and the
// launch sequence can be captured into one CUDA graph.
#pragma once
#include "cols.cuh"
#include "engine.cuh"
#include "rows.cuh"

namespace tftgb {

struct BatchSmall {
  uint64_t a, b, out;  // device pointers
  uint32_t na, nb;
  uint32_t l;          // log2 of the padded length (r <= 2^l)
  uint32_t pad;
};

struct BatchLarge {
  uint64_t a, b, out, work, EA, EB;  // device pointers
  uint64_t na, nb;
  uint32_t A;                        // a_p = r >> lr (full rows)
  uint32_t Bm;                       // b_p = r mod R (last row length)
  uint32_t c;                        // columns padded to 2^c
  uint32_t pad;
  uint64_t row_base;                 // prefix of the row counts a_p + [b_p > 0]
};

// Largest p with base(p) <= x over a non-decreasing prefix (binary search).
template <class Get>
__device__ __forceinline__ uint32_t find_product(uint32_t n, uint64_t x,
                                                 Get base) {
  uint32_t lo = 0, hi = n;  // invariant: base(lo) <= x < base(hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (base(mid) <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Small class: one product per CTA at a time (single-CTA product of
// kernels_impl.cuh: operands interleaved as two columns, pruned forward
// network, pointwise product, generalized block inverse).
// ---------------------------------------------------------------------------
template <class F>
__global__ void __launch_bounds__(512)
k_small_mul_batch(const BatchSmall* __restrict__ d, uint32_t n, int lmax,
                  RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  stage_roots<F>(&s_rt, rt);
  const uint32_t NMAX = 1u << lmax;
  T* Z = reinterpret_cast<T*>(smem_raw);  // 2 NMAX
  T* W = Z + 2 * NMAX;
  T* Wih = W + (NMAX > 1 ? NMAX / 2 : 1);
  for (uint32_t p = blockIdx.x; p < n; p += gridDim.x) {
    const BatchSmall q = d[p];
    const int l = (int)q.l;
    const uint32_t N = 1u << l;
    const uint32_t r = q.na + q.nb - 1;
    const T* A = reinterpret_cast<const T*>(q.a);
    const T* B = reinterpret_cast<const T*>(q.b);
    T* out = reinterpret_cast<T*>(q.out);
    __syncthreads();  // the previous product is done with shared memory
    build_base_tables<F>(W, Wih, l, s_rt);
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
      Z[2 * i] = i < q.na ? A[i] : T(0);
      Z[2 * i + 1] = i < q.nb ? B[i] : T(0);
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
}

// ---------------------------------------------------------------------------
// Large class, phase 1: forward column pass of both operands of every
// product.  Task = (product, operand, column tile of C columns).
// ---------------------------------------------------------------------------
template <class F>
__global__ void TFT_COL_LAUNCH_BOUNDS(256, typename F::T)
k_col_fwd_batch(const BatchLarge* __restrict__ d, uint32_t nl, int lr,
                int clog, RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  stage_roots<F>(&s_rt, rt);
  const uint32_t R = 1u << lr;
  const uint32_t tiles = R >> clog;
  const uint64_t total = (uint64_t)nl * 2 * tiles;
  for (uint64_t task = blockIdx.x; task < total; task += gridDim.x) {
    const uint32_t p = (uint32_t)(task / (2 * tiles));
    const uint32_t o = (uint32_t)((task / tiles) & 1);
    const uint32_t j = (uint32_t)(task % tiles);
    const BatchLarge q = d[p];
    const T* src = reinterpret_cast<const T*>(o ? q.b : q.a);
    T* dst = reinterpret_cast<T*>(o ? q.work : q.out);
    T* E = reinterpret_cast<T*>(o ? q.EB : q.EA);
    col_fwd_tile<F, true>(smem_raw, s_rt, src, o ? q.nb : q.na, dst, E, lr,
                          q.A, q.Bm, (int)q.c, clog, j << clog, R);
  }
}

// Phase 2: fused rows, all rows of all products flattened (row a_p of a
// product with b_p > 0 reads and writes its positions past r_p in EA / EB).
// With cache_prefix the CTA first copies the row prefix (32-bit) into the
// shared memory after the row buffers, so that a row's product is a binary
// search in shared memory rather than a chain of dependent global loads.
template <class F, int LR>
__global__ void __launch_bounds__(RowGeom<LR>::THREADS, RowGeom<LR>::template min_ctas<sizeof(typename F::T)>())
k_row_mul_batch(const BatchLarge* __restrict__ d, uint32_t nl,
                uint64_t total_rows, int cache_prefix,
                RootTable<typename F::T> rt) {
  TFT_ROW_PROLOGUE(2)
  uint32_t* s_rb = reinterpret_cast<uint32_t*>(
      smem_raw + row_smem_bytes<T>(LR, G, 2));
  if (cache_prefix) {
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x)
      s_rb[i] = (uint32_t)d[i].row_base;
    __syncthreads();
  }
  for (uint64_t row0 = (uint64_t)blockIdx.x * G; row0 < total_rows;
       row0 += (uint64_t)gridDim.x * G) {
    const uint64_t row = row0 + g;
    const bool active = row < total_rows;
    uint64_t rho = 0;
    T* GA = nullptr;
    const T* GB = nullptr;
    uint32_t bsplit = 0xffffffffu;
    T* EA = nullptr;
    const T* EB = nullptr;
    if (active) {
      const uint32_t p =
          cache_prefix
              ? find_product(nl, row,
                             [&](uint32_t i) { return (uint64_t)s_rb[i]; })
              : find_product(nl, row,
                             [&](uint32_t i) { return d[i].row_base; });
      rho = row - d[p].row_base;
      GA = reinterpret_cast<T*>(d[p].out) + rho * R;
      GB = reinterpret_cast<const T*>(d[p].work) + rho * R;
      if (rho == d[p].A) {
        bsplit = d[p].Bm;
        EA = reinterpret_cast<T*>(d[p].EA);
        EB = reinterpret_cast<const T*>(d[p].EB);
      }
    }
    row_mul_body<F, LR>(S, sp, g, t, active, rho, GA, GB, s_rt, bsplit, EA,
                        EB);
  }
}

// Phase 3: inverse columns, all R columns of every product, of length
// a_p + [b_p > 0].  Every product has R / C tiles: task = p (R / C) + j.
template <class F>
__global__ void TFT_COL_LAUNCH_BOUNDS(256, typename F::T)
k_col_inv_batch(const BatchLarge* __restrict__ d, uint32_t nl,
                uint64_t total, int lr, int clog,
                RootTable<typename F::T> rt) {
  using T = typename F::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<T> s_rt;
  stage_roots<F>(&s_rt, rt);
  const uint32_t R = 1u << lr;
  const uint32_t C = 1u << clog;
  for (uint64_t task = blockIdx.x; task < total; task += gridDim.x) {
    const uint32_t p = (uint32_t)(task >> (lr - clog));
    const BatchLarge q = d[p];
    const uint32_t j = (uint32_t)(task & ((1u << (lr - clog)) - 1));
    const uint64_t r = (uint64_t)q.A * R + q.Bm;
    col_inv_tile<F, false>(smem_raw, s_rt, reinterpret_cast<T*>(q.out),
                           nullptr, lr,
                    q.A + (q.Bm > 0 ? 1u : 0u), (int)q.c, clog, j * C, R, 0,
                    T(0), lr, r, reinterpret_cast<const T*>(q.EA));
  }
}

}  // namespace tftgb
