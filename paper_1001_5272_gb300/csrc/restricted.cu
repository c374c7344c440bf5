// The space-restricted product (Algorithm 3, Section 5) on the device:
// C = AB written into the r-word output buffer with no r-sized work area
// (include/tft.h: tft_polymul_restricted).  Host orchestration; the kernels
// are the field translation units' folding / chunk / tail kernels and the
// library's forward and inverse transforms.
//
// As in Algorithm 3, chunk [q, q + L) with L the largest power of two such
// that q + 2L <= r receives A^_{q..q+L-1} (fold of A(omega_q x) mod x^L - 1,
// then a forward transform of length L), [q + L, q + 2L) receives B^ the
// same way, and the chunk's pointwise product overwrites [q, q + L).  The
// loop runs while L > 2^16.  What remains, [q, r) with r - q < 2^18
// (including the last position r - 1, which Algorithm 3 evaluates by
// Horner), is produced from aligned blocks [Q, Q + M) of M = 2^18 positions
// (fewer when r is smaller): the fold of A(omega_Q x) mod x^M - 1 and a
// forward transform of length M in the context's fixed scratch give A^ on
// the whole block, which is copied to the tail positions; B^ likewise is
// multiplied in.  (Each short chunk would cost a fold over all of A and B
// and two small, latency-bound transforms; one or two tail blocks replace
// the chunks below 2^17.)  The auxiliary device memory is the context's
// fixed scratch (2^18 + 2^14 words) whatever r is.  Finally the in-place
// inverse transform of length r recovers C.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "alg3.cuh"
#include "ctx.h"

using namespace tftgb;

namespace {

int floor_log2(uint64_t x) {
  int l = -1;
  while (x) {
    x >>= 1;
    ++l;
  }
  return l;
}

// omega_q^{2^b}, b <= 32, in twiddle form, laid out as FoldPowers<T>.
void fold_powers(const PrimeInfo& pr, uint64_t q, unsigned char* out) {
  uint64_t w = omega_s(pr, q);
  for (int b = 0; b <= 32; ++b) {
    const uint64_t tw = to_tw(pr, w);
    if (pr.w == 8)
      memcpy(out + 8 * b, &tw, 8);
    else {
      const uint32_t t32 = (uint32_t)tw;
      memcpy(out + 4 * b, &t32, 4);
    }
    w = mulm(w, w, pr.p);
  }
}

constexpr int kChunkLogMin = 16;  // chunks with L > 2^16 use the buffer
constexpr int kTailLog = 18;      // tail blocks of 2^18 positions

// The chunk loop of Algorithm 3 for an output of r positions: the (q, L)
// pairs processed in the output buffer, in order, and the first tail
// position.  Returns the number of chunks (at most 64).
int chunk_schedule(uint64_t r, uint64_t* qs, uint64_t* Ls, uint64_t* tail) {
  uint64_t q = 0;
  int count = 0;
  while (q + 1 < r) {
    const int ell = floor_log2(r - q) - 1;  // floor(lg(r - q)) - 1
    if (ell <= kChunkLogMin) break;
    qs[count] = q;
    Ls[count] = 1ull << ell;
    ++count;
    q += 1ull << ell;
  }
  *tail = q;
  return count;
}

}  // namespace

tft_status tft_restricted_schedule(uint64_t r, uint64_t* q, uint64_t* L,
                                   uint32_t capacity, uint32_t* count,
                                   uint64_t* tail_start) {
  if (r == 0 || !count || !tail_start) return TFT_EINVAL;
  uint64_t qs[64], Ls[64], tail = 0;
  const int n = chunk_schedule(r, qs, Ls, &tail);
  if ((uint32_t)n > capacity || (n && (!q || !L))) return TFT_ERANGE;
  for (int i = 0; i < n; ++i) {
    q[i] = qs[i];
    L[i] = Ls[i];
  }
  *count = (uint32_t)n;
  *tail_start = tail;
  return TFT_OK;
}

tft_status tft_polymul_restricted(tft_ctx* ctx, const void* a, uint64_t na,
                                  const void* b, uint64_t nb, void* out,
                                  void* stream) {
  if (!ctx || !a || !b || !out || na == 0 || nb == 0) return TFT_EINVAL;
  if (!aligned16(a) || !aligned16(b) || !aligned16(out)) return TFT_EINVAL;
  const uint64_t r = na + nb - 1;
  const PrimeInfo& pr = ctx->pr;
  const size_t w = pr.w;
  if (overlap(out, r * w, a, na * w) || overlap(out, r * w, b, nb * w))
    return TFT_EINVAL;
  Plan Pr;
  if (!make_plan(ctx->prime, r, &Pr)) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* X = (unsigned char*)out;
  unsigned char* scratch = (unsigned char*)ctx->scratch;
  static_assert(((size_t)1 << kTailLog) + ((size_t)1 << 14) <= kCtxScratchWords,
                "tail block and row scratch must fit the context scratch");
  void* E = scratch + ((size_t)1 << kTailLog) * w;  // after the tail block
  alignas(16) unsigned char powers[33 * 8];
  const LaunchHook& H = ctx->hook;
  cudaError_t e = cudaSuccess;
  auto fold = [&](void* d0, void* d1, uint64_t L, int ell, uint64_t q) {
    fold_powers(pr, q, powers);
    H.before(H.user, K_FOLD, s);
    e = launch_fold(ctx->prime, d0, a, na, d1, d1 ? b : nullptr,
                    d1 ? nb : 0, L, ell, powers, ctx->nsm, s);
    H.after(H.user, K_FOLD, s);
    return e == cudaSuccess;
  };
  // ---- chunks in the output buffer -----------------------------------------
  uint64_t qs[64], Ls[64], q = 0;
  const int nchunks = chunk_schedule(r, qs, Ls, &q);
  for (int ci = 0; ci < nchunks; ++ci) {
    const uint64_t L = Ls[ci];
    const int ell = floor_log2(L);
    const uint64_t qc = qs[ci];
    Plan PL;
    if (!make_plan(ctx->prime, L, &PL)) return TFT_ERANGE;
    void* XA = X + qc * w;
    void* XB = X + (qc + L) * w;
    if (!fold(XA, XB, L, ell, qc)) return from_cuda(ctx, e);
    // the two chunk transforms are independent: B's on the context's side
    // stream, forked after the fold and joined before the product (b = 0 for
    // a power-of-two length, so neither transform uses E)
    const AuxStreams& ax = ctx->aux;
    e = cudaEventRecord(ax.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ax.side, ax.fork, 0);
    if (e == cudaSuccess)
      e = launch_forward(ctx->prime, XB, L, PL, E, ctx->rt, ctx->nsm,
                         ax.side, &H, nullptr);
    if (e == cudaSuccess)
      e = launch_forward(ctx->prime, XA, L, PL, E, ctx->rt, ctx->nsm, s, &H,
                         nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(ax.join, ax.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ax.join, 0);
    if (e != cudaSuccess) return from_cuda(ctx, e);
    H.before(H.user, K_FOLD, s);
    e = launch_chunk_mul(ctx->prime, XA, XB, L, ctx->nsm, s);
    H.after(H.user, K_FOLD, s);
    if (e != cudaSuccess) return from_cuda(ctx, e);
  }
  // ---- tail blocks in the fixed scratch ------------------------------------
  if (q < r) {
    int mlog = kTailLog;
    while (mlog > 0 && (1ull << (mlog - 1)) >= r) --mlog;  // M >= r suffices
    const uint64_t M = 1ull << mlog;
    Plan PM;
    if (!make_plan(ctx->prime, M, &PM)) return TFT_ERANGE;
    for (uint64_t Q = q & ~(M - 1); Q < r; Q += M) {
      const uint64_t lo = Q > q ? Q : q;
      const uint64_t hi = Q + M < r ? Q + M : r;
      for (int op = 0; op < 2; ++op) {
        fold_powers(pr, Q, powers);
        H.before(H.user, K_FOLD, s);
        e = launch_fold(ctx->prime, scratch, op ? b : a, op ? nb : na,
                        nullptr, nullptr, 0, M, mlog, powers, ctx->nsm, s);
        H.after(H.user, K_FOLD, s);
        if (e == cudaSuccess)
          e = launch_forward(ctx->prime, scratch, M, PM, E, ctx->rt,
                             ctx->nsm, s, &H, &ctx->aux);
        if (e == cudaSuccess) {
          H.before(H.user, K_FOLD, s);
          e = launch_tail(ctx->prime, X, scratch, Q, lo, hi, op, ctx->nsm,
                          s);
          H.after(H.user, K_FOLD, s);
        }
        if (e != cudaSuccess) return from_cuda(ctx, e);
      }
    }
  }
  // ---- inverse transform of length r ----------------------------------------
  return from_cuda(
      ctx, launch_inverse(ctx->prime, X, r, Pr, scratch,
                          Pr.small ? 0 : to_tw(pr, omega_s(pr, Pr.a)),
                          ctx->rt, ctx->nsm, s, &H));
}
