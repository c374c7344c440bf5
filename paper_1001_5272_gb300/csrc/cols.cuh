// Column kernels on the register-blocked stage engine (stages.cuh).
//
// A column tile holds C = 2^clog adjacent columns of the R-wide matrix view,
// each padded to 2^c rows, row-major in shared memory: element (t, c) at
// Z[tswz(t) * C + c].  tswz permutes rows inside each 16-row group by
// XOR-ing the low 4 - clog bits of t with t >> 4, so that a warp touching C
// columns of several 16-row groups hits distinct banks.  Every column is its
// own transform (twiddles independent of the column), so a stage's twist is
// omega_{B 2^L} with B the unit's block index inside the column: the row
// factor of the row kernels is 1 here.
#pragma once
#include "stages.cuh"

// Resident CTAs per SM asked of the 256-thread column kernels, per element
// width (3 -> 80, 4 -> 64 registers per thread; measured best on GB300).
#ifndef TFT_COL_MIN_CTAS_64
#define TFT_COL_MIN_CTAS_64 3
#endif
#ifndef TFT_COL_MIN_CTAS_32
#define TFT_COL_MIN_CTAS_32 4
#endif
#define TFT_COL_LAUNCH_BOUNDS(NT, T)                                  \
  __launch_bounds__(NT, sizeof(T) == 8 ? TFT_COL_MIN_CTAS_64          \
                                       : TFT_COL_MIN_CTAS_32)

namespace tftgb {

__device__ __forceinline__ uint32_t tswz(uint32_t t, int clog) {
  return clog >= 4 ? t : t ^ ((t >> 4) & ((1u << (4 - clog)) - 1));
}

// Shared layout of the column kernels:
//   K (StageConsts) | TL[tl] | TLi[tl] | Z[2^c * C]
template <class T>
struct ColSmem {
  StageConsts<T>* K;
  T* TL;
  T* TLi;
  T* Z;
  __device__ ColSmem(unsigned char* raw, int tl) {
    K = reinterpret_cast<StageConsts<T>*>(raw);
    T* p = reinterpret_cast<T*>(raw + sizeof(StageConsts<T>));
    TL = p;
    p += tl;
    TLi = p;
    p += tl;
    uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
    Z = reinterpret_cast<T*>(a);
  }
};

// (the tile area holds at least 256 words: the inverse kernel reuses it for
// its Horner reduction)
template <class T>
__host__ __device__ inline size_t col_smem_bytes(int c, int clog) {
  const StagePlan sp = make_stage_plan(c, true);
  size_t b = sizeof(StageConsts<T>) + sizeof(T) * 2 * sp.tl_total;
  b = (b + 15) & ~(size_t)15;
  const size_t tile = (size_t)1 << (c + clog);
  return b + sizeof(T) * (tile < 256 ? 256 : tile);
}

// One forward stage over all units of a column tile.  FIRST: inputs from
// global memory (positions >= n_src and rows >= rows are zero); LAST: outputs
// to global memory (rows t < a to dst, row a to dst or E).  TZ (first stage
// only): the operand has no entries in the upper half of the padded column
// (rows >= 2^{c-1}), so the stage's top level is a copy and those inputs are
// not loaded.  PWT: the stage's twist powers come from PW by block,
// PW[16 B + i] = TLs[B]^i, shared by the 16 C units of each block.
template <class F, int L, bool FIRST, bool LAST, bool TZ = false,
          bool PWT = false>
__device__ __forceinline__ void col_fwd_stage(
    typename F::T* Z, const typename F::T* src, uint64_t n_src,
    typename F::T* dst, typename F::T* E, uint64_t R, uint64_t a, uint64_t b,
    uint32_t rows, int c, int clog, uint32_t q0, uint32_t q_end, int r_lo,
    const typename F::T* TLs, const StageConsts<typename F::T>& K,
    const typename F::T* PW = nullptr) {
  using T = typename F::T;
  constexpr int U = 1 << L;
  const uint32_t C = 1u << clog;
  // rows still needed once this stage is done: < ceil(rows / 2^r_lo) 2^r_lo
  const uint32_t need = ((rows + (1u << r_lo) - 1) >> r_lo) << r_lo;
  const uint32_t units = 1u << (c - L + clog);
  // a unit whose block starts at or past `need` is skipped
  auto live = [&](uint32_t u) {
    return (((u >> clog) >> r_lo) << (r_lo + L)) < need;
  };
  auto load = [&](uint32_t u, T(&x)[U]) {
    const uint32_t cc = u & (C - 1);
    const uint32_t ut = u >> clog;
    const uint64_t q = (uint64_t)q0 + cc;
    const bool colok = q < q_end;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint32_t t = unit_pos(ut, r_lo, L, i);
      if (FIRST) {
        const uint64_t pos = q + (uint64_t)t * R;
        x[i] = (!(TZ && i >= U / 2) && colok && t < rows && pos < n_src)
                   ? src[pos]
                   : T(0);
      } else {
        x[i] = Z[(tswz(t, clog) << clog) + cc];
      }
    }
  };
  auto compute_store = [&](uint32_t u, T(&x)[U]) {
    const uint32_t cc = u & (C - 1);
    const uint32_t ut = u >> clog;
    const uint64_t q = (uint64_t)q0 + cc;
    const bool colok = q < q_end;
    // the first stage's block index is 0: zeta = 1, no twist
    if (!FIRST) {
      if constexpr (PWT) {
        const T* pw = PW + 16 * (ut >> r_lo);
#pragma unroll
        for (int i = 1; i < U; ++i) x[i] = F::mul_tw(x[i], pw[i]);
      } else {
        twist<F, L>(x, TLs[ut >> r_lo]);
      }
    }
    cnet_fwd<F, L, FIRST && TZ>(x, K);
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint32_t t = unit_pos(ut, r_lo, L, i);
      if (LAST) {
        if (colok && t < rows) {
          if (t < a)
            dst[q + (uint64_t)t * R] = F::canon(x[i]);
          else if (q < b)
            dst[q + a * R] = F::canon(x[i]);
          else
            E[q] = F::canon(x[i]);
        }
      } else {
        Z[(tswz(t, clog) << clog) + cc] = x[i];
      }
    }
  };
#pragma unroll 1
  for (uint32_t u = threadIdx.x; u < units; u += blockDim.x) {
    if (!live(u)) continue;
    T x[U];
    load(u, x);
    compute_store(u, x);
  }
}

// ---------------------------------------------------------------------------
// Forward column pass.  Rows produced: `rows` = a (+1 if b > 0).  Inputs at
// positions >= n_src are the operand's zero extension.  A unit whose whole
// block lies at or beyond the rows the later stages need is skipped (the
// pruned network of engine.cuh, at stage granularity).  The last stage
// writes straight to global memory: rows t < a to dst, row a to dst for long
// columns (q < b) and to E for short ones.
// ---------------------------------------------------------------------------
template <class F, bool PWTAB = false>
__device__ void col_fwd_tile(unsigned char* smem_raw,
                             const RootTable<typename F::T>& s_rt,
                             const typename F::T* src, uint64_t n_src,
                             typename F::T* dst, typename F::T* E, int lr,
                             uint64_t a, uint64_t b, int c, int clog,
                             uint32_t q0, uint32_t q_end) {
  using T = typename F::T;
  __syncthreads();  // the previous tile is done with shared memory
  const StagePlan sp = make_stage_plan(c, true);
  ColSmem<T> S(smem_raw, sp.tl_total);
  fill_stage_consts<F>(S.K, s_rt, c);
  build_stage_tables<F>(S.TL, S.TLi, sp, c, s_rt);
  __syncthreads();
  // PWTAB: the second stage's twist powers by block when it has at most 32
  // blocks (the later stages have too many blocks for a table).  Each table
  // row serves the 16 C units of its block, so it pays on wide tiles (the
  // batched products' 32-column tiles: forward columns 4% faster); on the
  // single transforms' 2- and 4-column tiles it measured slower.
  __shared__ T s_pw[PWTAB ? 32 * 16 : 1];
  const bool pw1 =
      PWTAB && sp.n >= 2 && (c - sp.s[1].r_lo - sp.s[1].L) <= 5;
  if (pw1) {
    const T* TL1 = S.TL + sp.s[1].tl_off;
    const int cnt = 16 << (c - sp.s[1].r_lo - sp.s[1].L);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      T z = TL1[e >> 4], v = s_rt.one_tw;
      for (int t = e & 15; t; t >>= 1) {
        if (t & 1) v = F::mul_tw(v, z);
        z = F::mul_tw(z, z);
      }
      s_pw[e] = v;
    }
    __syncthreads();
  }
  const uint64_t R = 1ull << lr;
  const uint32_t rows = (uint32_t)(a + (b > 0 ? 1 : 0));
  // the operand's rows (the longest column's) all below 2^{c-1}: the top
  // level is a copy (the first stage covers it)
  const bool tz = c >= 1 && ((n_src + R - 1) >> lr) <= (1ull << (c - 1));
  for (int si = 0; si < sp.n; ++si) {
    const int r_lo = sp.s[si].r_lo;
    const T* TLs = S.TL + sp.s[si].tl_off;
    const bool first = si == 0, last = si == sp.n - 1;
#define TFT_COL_FWD_CALL(FI, LA, TZ, PWT)                                   \
  TFT_STAGE_SWITCH(sp.s[si].L,                                              \
                   (col_fwd_stage<F, LL, FI, LA, TZ, PWT>(                  \
                       S.Z, src, n_src, dst, E, R, a, b, rows, c, clog, q0, \
                       q_end, r_lo, TLs, *S.K, s_pw)))
    const bool pw = si == 1 && pw1;
    if (first && last) {
      if (tz) {
        TFT_COL_FWD_CALL(true, true, true, false);
      } else {
        TFT_COL_FWD_CALL(true, true, false, false);
      }
    } else if (first) {
      if (tz) {
        TFT_COL_FWD_CALL(true, false, true, false);
      } else {
        TFT_COL_FWD_CALL(true, false, false, false);
      }
    } else if (last) {
      if (PWTAB && pw) {
        TFT_COL_FWD_CALL(false, true, false, PWTAB);
      } else {
        TFT_COL_FWD_CALL(false, true, false, false);
      }
    } else {
      if (PWTAB && pw) {
        TFT_COL_FWD_CALL(false, false, false, PWTAB);
      } else {
        TFT_COL_FWD_CALL(false, false, false, false);
      }
    }
#undef TFT_COL_FWD_CALL
    __syncthreads();
  }
}

// Per-CTA copy of the root table (kernel parameters are not addressable
// without a local copy).
template <class F>
__device__ __forceinline__ void stage_roots(RootTable<typename F::T>* s_rt,
                                            const RootTable<typename F::T>& rt) {
  using T = typename F::T;
  const T* s = reinterpret_cast<const T*>(&rt);
  T* d = reinterpret_cast<T*>(s_rt);
  for (int i = threadIdx.x; i < (int)(sizeof(rt) / sizeof(T)); i += blockDim.x)
    d[i] = s[i];
  __syncthreads();
}

template <class F, int MAXT>
__global__ void TFT_COL_LAUNCH_BOUNDS(MAXT, typename F::T)
k_col_fwd2(const typename F::T* src, uint64_t n_src, typename F::T* dst,
           typename F::T* __restrict__ E, int lr, uint64_t a, uint64_t b,
           int c, int clog, uint32_t q_begin, uint32_t q_end,
           RootTable<typename F::T> rt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<typename F::T> s_rt;
  stage_roots<F>(&s_rt, rt);
  col_fwd_tile<F>(smem_raw, s_rt, src, n_src, dst, E, lr, a, b, c, clog,
                  q_begin + blockIdx.x * (1u << clog), q_end);
}

// omega_{2j} (twiddle form) as the product of omega_[b+2] over the set bits b
// of j (omega_{2^{b+1}} = omega_[b+2]); inverse: the inverse roots times 1/2.
template <class F>
__device__ __forceinline__ typename F::T col_theta(
    uint32_t j, const RootTable<typename F::T>& rt, bool inv_half) {
  typename F::T v = inv_half ? rt.half_tw : rt.one_tw;
  int b = 0;
  while (j) {
    if (j & 1) v = F::mul_tw(v, inv_half ? rt.winv[b + 2] : rt.w[b + 2]);
    j >>= 1;
    ++b;
  }
  return v;
}

// One unit of an inverse stage (levels r_lo .. r_lo + L - 1) of the full
// inverse network of the dyadic block [off, off + 2^k) of the tile: unit u
// of the block covers column u mod C.  The block is block off >> k of the
// column's network, so the stage twist is omega_{(off >> k) 2^{k - r_lo}} *
// omega_{B_local 2^L} (inverted here, RFi is the first factor's inverse).
// The stage returns 2^L times its exact inverse (cnet_inv2); the stage that
// reaches the block's top level (top) also carries the block's whole factor
// 2^-k (times any scale its inputs carry).  At the top stage B_local = 0 for
// every unit of the block, so its twist and scale are one per-block table,
// top_tab[i] = 2^-k RFi^i, instead of the powers of zeta per unit.
template <class F, int L>
__device__ __forceinline__ void col_inv_unit(
    typename F::T* Z, int clog, uint32_t off, int r_lo, uint32_t u,
    typename F::T RFi, const typename F::T* TL16i,
    const StageConsts<typename F::T>& K, bool top,
    const typename F::T* top_tab) {
  using T = typename F::T;
  constexpr int U = 1 << L;
  const uint32_t cc = u & ((1u << clog) - 1);
  const uint32_t ut = u >> clog;
  T x[U];
#pragma unroll
  for (int i = 0; i < U; ++i) {
    const uint32_t t = off + unit_pos(ut, r_lo, L, i);
    x[i] = Z[(tswz(t, clog) << clog) + cc];
  }
  cnet_inv2<F, L>(x, K);
  if (top) {
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = F::mul_tw(x[i], top_tab[i]);
  } else {
    // only the 4-level stages below a block's top have B_local != 0
    const uint32_t bl = ut >> r_lo;
    twist<F, L>(x, L == 4 && bl ? F::mul_tw(RFi, TL16i[bl]) : RFi);
  }
#pragma unroll
  for (int i = 0; i < U; ++i) {
    const uint32_t t = off + unit_pos(ut, r_lo, L, i);
    Z[(tswz(t, clog) << clog) + cc] = x[i];
  }
}

// All units of width L of stage j across the dyadic blocks whose stage j has
// that width, flattened over the CTA's threads.
template <class F, int L>
__device__ __forceinline__ void col_inv_stage_flat(
    typename F::T* Z, int clog, int r_lo, int j, int nb, const int* bk,
    const uint32_t* boff, const typename F::T* rfi, const typename F::T* ttab,
    const typename F::T* TL16i, const StageConsts<typename F::T>& K) {
  uint32_t total = 0;
  for (int i = 0; i < nb; ++i) {
    const int w = bk[i] - r_lo;
    if (w > 0 && (w >= 4 ? 4 : w) == L) total += 1u << (bk[i] - L + clog);
  }
#pragma unroll 1
  for (uint32_t ug = threadIdx.x; ug < total; ug += blockDim.x) {
    uint32_t u = ug;
    int i = 0;
    for (; i < nb; ++i) {
      const int w = bk[i] - r_lo;
      if (w <= 0 || (w >= 4 ? 4 : w) != L) continue;
      const uint32_t cnt = 1u << (bk[i] - L + clog);
      if (u < cnt) break;
      u -= cnt;
    }
    col_inv_unit<F, L>(Z, clog, boff[i], r_lo, u, rfi[j * 14 + i], TL16i, K,
                       bk[i] - r_lo == L, ttab + 16 * i);
  }
}

// ---------------------------------------------------------------------------
// Inverse column pass over columns [q_begin, q_end), all of length m (a for
// short columns, a + 1 for long ones), padded to 2^c in shared memory: the
// generalized block inverse of engine.cuh (phase A: the full inverses of the
// dyadic blocks of m; then one descent and one ascent), with phase A on the
// stage engine.  With want_E also E_q = C_q(omega_a) by a parallel Horner
// rule (omega_a in twiddle form).  Positions q + t R >= split lie past the
// buffer: they are read from Ealt[q] and not stored (a product transform
// whose length is rounded up to a multiple of R; its coefficients there are
// zero).  The tile's inputs may carry a factor 2^in_scale_log (the product's
// row pass leaves its inverse unscaled), removed here with the blocks' own
// factors.
//
// LASTROW: the tile is the ragged last row instead, one "column" of 2^c
// contiguous words (lr = 0, clog = 0, m = b) that is block gblk = a of the
// length-2^k network: every butterfly's twiddle takes the block's global
// index ((gblk << c) + offset) >> level, and the known inputs at t >= m are
// Ealt[t] (the short columns' E_t) instead of zero.
// ---------------------------------------------------------------------------
template <class F, bool ASYNC_LOAD = true, bool LASTROW = false>
__device__ void col_inv_tile(unsigned char* smem_raw,
                             const RootTable<typename F::T>& s_rt,
                             typename F::T* X, typename F::T* E, int lr,
                             uint32_t m, int c, int clog, uint32_t q0,
                             uint32_t q_end, int want_E,
                             typename F::T omega_a_tw, int in_scale_log,
                             uint64_t split = ~0ull,
                             const typename F::T* Ealt = nullptr,
                             uint64_t gblk = 0) {
  using T = typename F::T;
  __syncthreads();  // the previous tile is done with shared memory
  // stage tables for 4-level stages: TL16[m'] = omega_{16 m'}, m' < 2^{c-4}
  const StagePlan sp = make_stage_plan(c, true);
  ColSmem<T> S(smem_raw, sp.tl_total);
  fill_stage_consts<F>(S.K, s_rt, c);
  const uint32_t n16 = c > 4 ? 1u << (c - 4) : 1u;
  T* TL16i = S.TLi;  // n16 <= tl_total entries (the last stage's table)
  for (uint32_t j = threadIdx.x; j < n16; j += blockDim.x) {
    T v = s_rt.one_tw;
    uint32_t bits = j;
    int b = 0;
    while (bits) {
      if (bits & 1) v = F::mul_tw(v, s_rt.winv[b + 5]);  // omega_{16 2^b}
      bits >>= 1;
      ++b;
    }
    TL16i[j] = v;
  }
  const uint32_t C = 1u << clog;
  const uint64_t R = 1ull << lr;
  const uint32_t N = 1u << c;
  T* Z = S.Z;
  // descent and ascent twiddles, one serial product per level, computed by
  // separate threads while the tile loads: s_thd[l] = omega_{2 (m >> l)},
  // s_tha[l] the same or (if the ascent's level l is an up step) its
  // inverse over 2
  __shared__ T s_thd[16], s_tha[16];
  if (threadIdx.x >= 32 && threadIdx.x < 32 + 2 * 16) {
    const int l = (threadIdx.x - 32) & 15;
    const bool asc = threadIdx.x >= 48;
    if (l >= 1 && l <= c) {
      const uint32_t low = m & ((1u << l) - 1);
      const bool up = asc && low >= (1u << (l - 1));
      T th;
      if constexpr (LASTROW) {
        th = row_factor<F>((gblk << (c - l)) + (m >> l), 1, s_rt, up);
        if (up) th = F::mul_tw(th, s_rt.half_tw);
      } else {
        th = col_theta<F>(m >> l, s_rt, up);
      }
      if (asc)
        s_tha[l] = th;
      else
        s_thd[l] = th;
    }
  }
  // the tile; positions outside the columns or past m are zero.
  // ASYNC_LOAD: asynchronous copies (every load of the thread in flight at
  // once, no registers held; measured faster for the single transforms);
  // otherwise eight loads in flight per thread through registers (measured
  // faster for the batched products' short columns)
  const uint32_t nld = N << clog;
  if constexpr (LASTROW) {
#pragma unroll 4
    for (uint32_t t = threadIdx.x; t < N; t += blockDim.x)
      cp_async_elem(Z + tswz(t, 0), t < m ? X + t : Ealt + t);
    cp_async_wait_all();
  } else if constexpr (ASYNC_LOAD) {
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < nld; i += blockDim.x) {
      const uint32_t t = i >> clog, cc = i & (C - 1);
      const uint64_t q = (uint64_t)q0 + cc;
      const uint64_t pos = q + (uint64_t)t * R;
      T* z = Z + (tswz(t, clog) << clog) + cc;
      if (q < q_end && t < m)
        cp_async_elem(z, pos < split ? X + pos : Ealt + q);
      else
        *z = T(0);
    }
    cp_async_wait_all();
  } else {
#pragma unroll 1
    for (uint32_t i0 = threadIdx.x; i0 < nld; i0 += 8 * blockDim.x) {
      T v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t i = i0 + k * blockDim.x;
        const uint32_t t = i >> clog, cc = i & (C - 1);
        const uint64_t q = (uint64_t)q0 + cc;
        const uint64_t pos = q + (uint64_t)t * R;
        v[k] = (i < nld && q < q_end && t < m)
                   ? (pos < split ? X[pos] : Ealt[q])
                   : T(0);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t i = i0 + k * blockDim.x;
        if (i < nld) Z[(tswz(i >> clog, clog) << clog) + (i & (C - 1))] = v[k];
      }
    }
  }
  __syncthreads();
  // ---- phase A: full inverse of every dyadic block of m ------------------
  // The blocks are the set bits k of m (sizes 2^k, decreasing, at increasing
  // offsets); m = 2^c is the single block of the whole column.  Stage j
  // covers levels 4j .. 4j + 3 (fewer at a block's top); blocks are
  // independent, so the units of all blocks are processed together and one
  // barrier separates stage indices.
  __shared__ int s_bk[14];
  __shared__ uint32_t s_boff[14];
  __shared__ T s_rfi[4 * 14];
  __shared__ T s_bsc[14];
  __shared__ T s_ttab[14 * 16];
  __shared__ int s_nb;
  if (threadIdx.x == 0) {
    int nb = 0;
    uint32_t off = 0;
    for (int k = c; k >= 1; --k) {
      const bool block = (k == c) ? (m == N) : (((m >> k) & 1u) != 0);
      if (!block) continue;
      s_bk[nb] = k;
      s_boff[nb] = off;
      ++nb;
      off += 1u << k;
    }
    s_nb = nb;
  }
  __syncthreads();
  const int nb = s_nb;
  const int nst = (c + 3) / 4;
  // row factors per (stage, block), then each block's scale 2^-(k + in)
  for (int e = threadIdx.x; e < (nst + 1) * nb; e += blockDim.x) {
    const int jj = e / nb, i = e % nb;
    const int k = s_bk[i];
    if (jj == nst)
      s_bsc[i] = pow2_inv<F>(k + in_scale_log, s_rt);
    else
      s_rfi[jj * 14 + i] =
          k > 4 * jj
              ? row_factor<F>(LASTROW ? ((gblk << c) + s_boff[i]) >> k
                                      : (uint64_t)(s_boff[i] >> k),
                              k - 4 * jj, s_rt, true)
              : s_rt.one_tw;
  }
  // an odd m leaves a block of one entry (row m - 1), which has no network
  // but still carries the inputs' scale
  if ((m & 1u) && in_scale_log > 0 && threadIdx.x < (1u << clog)) {
    T* z = Z + (tswz(m - 1, clog) << clog) + threadIdx.x;
    *z = F::mul_tw(*z, pow2_inv<F>(in_scale_log, s_rt));
  }
  __syncthreads();
  // each block's top-stage table: 2^-(k + in) RFi^t, t < 16, with RFi the
  // row factor of the block's top stage (stage (k - 1) / 4)
  for (int e = threadIdx.x; e < 16 * nb; e += blockDim.x) {
    const int i = e >> 4;
    T z = s_rfi[((s_bk[i] - 1) >> 2) * 14 + i], v = s_bsc[i];
    for (int t = e & 15; t; t >>= 1) {
      if (t & 1) v = F::mul_tw(v, z);
      z = F::mul_tw(z, z);
    }
    s_ttab[e] = v;
  }
  __syncthreads();
  for (int jj = 0; jj < nst; ++jj) {
    const int r_lo = 4 * jj;
    col_inv_stage_flat<F, 4>(Z, clog, r_lo, jj, nb, s_bk, s_boff, s_rfi,
                             s_ttab, TL16i, *S.K);
    col_inv_stage_flat<F, 3>(Z, clog, r_lo, jj, nb, s_bk, s_boff, s_rfi,
                             s_ttab, TL16i, *S.K);
    col_inv_stage_flat<F, 2>(Z, clog, r_lo, jj, nb, s_bk, s_boff, s_rfi,
                             s_ttab, TL16i, *S.K);
    col_inv_stage_flat<F, 1>(Z, clog, r_lo, jj, nb, s_bk, s_boff, s_rfi,
                             s_ttab, TL16i, *S.K);
    __syncthreads();
  }
  // ---- descent and ascent (one level each) -------------------------------
  if (m != N) {
    int lstop = 0;
    for (int l = c; l >= 1; --l) {
      const uint32_t low = m & ((1u << l) - 1);
      if (low == 0) {
        lstop = l;
        break;
      }
      const uint32_t B = m & ~((1u << l) - 1);
      const uint32_t h = 1u << (l - 1);
      const T th = s_thd[l];
      const uint32_t j0 = low >= h ? low - h : low;
      const uint32_t cnt = (h - j0) << clog;
#pragma unroll 4
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t cc = i & (C - 1);
        const uint32_t jj = j0 + (i >> clog);
        T* pl = Z + (tswz(B + jj, clog) << clog) + cc;
        T* pu = Z + (tswz(B + h + jj, clog) << clog) + cc;
        if (low >= h) {
          const T tt = F::mul_tw(*pu, th);
          *pu = F::sub(F::sub(*pl, tt), tt);
        } else {
          *pl = F::add(*pl, F::mul_tw(*pu, th));
        }
      }
      __syncthreads();
    }
    for (int l = lstop + 1; l <= c; ++l) {
      const uint32_t low = m & ((1u << l) - 1);
      const uint32_t B = m & ~((1u << l) - 1);
      const uint32_t h = 1u << (l - 1);
      const uint32_t cnt = h << clog;
      const bool up = low >= h;
      const T th = s_tha[l];
#pragma unroll 4
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t cc = i & (C - 1);
        const uint32_t jj = i >> clog;
        T* pl = Z + (tswz(B + jj, clog) << clog) + cc;
        T* pu = Z + (tswz(B + h + jj, clog) << clog) + cc;
        if (up) {
          const T Xv = *pl, Yv = *pu;
          *pl = F::half(F::add(Xv, Yv));
          *pu = F::mul_tw(F::sub(Xv, Yv), th);
        } else {
          *pl = F::sub(*pl, F::mul_tw(*pu, th));
        }
      }
      __syncthreads();
    }
  }
  // ---- store and E ---------------------------------------------------------
#pragma unroll 4
  for (uint32_t i = threadIdx.x; i < (m << clog); i += blockDim.x) {
    const uint32_t t = i >> clog, cc = i & (C - 1);
    const uint64_t q = (uint64_t)q0 + cc;
    const uint64_t pos = q + (uint64_t)t * R;
    if (q < q_end && pos < split)
      X[pos] = F::canon(Z[(tswz(t, clog) << clog) + cc]);
  }
  if (want_E) {
    const uint32_t tpc = blockDim.x >> clog;  // threads per column
    const uint32_t cc = threadIdx.x & (C - 1);
    const uint32_t kk = threadIdx.x >> clog;
    const uint32_t chunk = (m + tpc - 1) / tpc;
    const uint32_t t0 = kk * chunk;
    const uint32_t t1 = t0 + chunk < m ? t0 + chunk : m;
    T acc = 0;
    for (uint32_t t = t1; t > t0; --t)
      acc = F::add(F::mul_tw(acc, omega_a_tw),
                   Z[(tswz(t - 1, clog) << clog) + cc]);
    if (t0 < m) {
      T pw = s_rt.one_tw, base = omega_a_tw;
      for (uint32_t e = t0; e; e >>= 1) {
        if (e & 1) pw = F::mul_tw(pw, base);
        base = F::mul_tw(base, base);
      }
      acc = F::mul_tw(acc, pw);
    } else {
      acc = 0;
    }
    __syncthreads();
    T* part = Z;  // the tile is no longer needed
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
      T sacc = 0;
      for (uint32_t k2 = 0; k2 < tpc; ++k2)
        sacc = F::add(sacc, part[(k2 << clog) + threadIdx.x]);
      const uint64_t q = (uint64_t)q0 + threadIdx.x;
      if (q < q_end) E[q] = F::canon(sacc);
    }
  }
}

template <class F, int MAXT>
__global__ void TFT_COL_LAUNCH_BOUNDS(MAXT, typename F::T)
k_col_inv2(typename F::T* X, typename F::T* __restrict__ E, int lr,
           uint32_t m, int c, int clog, uint32_t q_begin, uint32_t q_end,
           int want_E, typename F::T omega_a_tw, int in_scale_log,
           RootTable<typename F::T> rt, uint64_t split,
           const typename F::T* Ealt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<typename F::T> s_rt;
  stage_roots<F>(&s_rt, rt);
  col_inv_tile<F>(smem_raw, s_rt, X, E, lr, m, c, clog,
                  q_begin + blockIdx.x * (1u << clog), q_end, want_E,
                  omega_a_tw, in_scale_log, split, Ealt);
}

// Inverse of the ragged last row (one CTA): block a of the network, outputs
// known at q < b (in row) and inputs at q >= b (E_q = C_q(omega_a)); writes
// the b recovered inputs (the long columns' last transform values) over the
// outputs.  The generalized block inverse of the column tiles on one
// contiguous 2^lr-word column whose twiddles carry the row index a.
template <class F>
__global__ void __launch_bounds__(512)
k_lastrow_inv2(typename F::T* row, const typename F::T* __restrict__ E,
               int lr, uint64_t a, uint64_t b, RootTable<typename F::T> rt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RootTable<typename F::T> s_rt;
  stage_roots<F>(&s_rt, rt);
  col_inv_tile<F, true, true>(smem_raw, s_rt, row, nullptr, 0, (uint32_t)b,
                              lr, 0, 0, 1, 0, s_rt.one_tw, 0, ~0ull, E, a);
}

}  // namespace tftgb
