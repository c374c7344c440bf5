// C ABI of the batched product (include/tft.h: tft_ctx_reserve_batch,
// tft_batch_plan, tft_batch_run, tft_polymul_batch, tft_batch_work_words)
// and the batch description shared with the request server.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ctx.h"

using namespace tftgb;

namespace tftgb {

BatchSchedule batch_schedule(const PrimeInfo& pr,
                             const tft_batch_params* params) {
  // small class in one CTA up to 2^13 words (u32) / 2^12 (u64); the large
  // class on rows of 2^9 (u32) / 2^10 (u64) with 16 / 4 columns per tile
  BatchSchedule S = pr.w == 8 ? BatchSchedule{12, 10, 2, -1}
                              : BatchSchedule{13, 9, 4, -1};
  if (params) {
    if (params->small_log) S.small_log = (int)params->small_log;
    if (params->lr) S.lr = (int)params->lr;
    if (params->clog_plus1) S.clog = (int)params->clog_plus1 - 1;
    if (params->clog_lo_plus1) S.clog_lo = (int)params->clog_lo_plus1 - 1;
  }
  return S;
}

bool batch_schedule_valid(const PrimeInfo& pr, const BatchSchedule& S) {
  const int small_max = pr.w == 8 ? 12 : 13;
  return S.lr >= 8 && S.lr <= 12 && S.small_log >= S.lr &&
         S.small_log <= small_max && S.clog >= 0 && S.clog <= 5 &&
         S.clog <= S.lr && S.clog_lo >= -1 && S.clog_lo <= 5 &&
         S.clog_lo <= S.lr;
}

uint64_t batch_product_work_words(const PrimeInfo& pr, const BatchSchedule& S,
                                  uint64_t na, uint64_t nb) {
  const uint64_t r = na + nb - 1;
  if (r <= (1ull << S.small_log)) return 0;
  const uint64_t align = 16 / pr.w;
  const uint64_t R = 1ull << S.lr;
  auto up = [&](uint64_t x) { return (x + align - 1) / align * align; };
  return up(r) + 2 * up(R);
}

tft_status batch_describe(const PrimeInfo& pr, const BatchSchedule& S,
                          const tft_polymul_desc* descs, uint32_t count,
                          void* const* work_of, void* work_base,
                          uint64_t work_cap, size_t optin,
                          std::vector<BatchSmall>* hs,
                          std::vector<BatchLarge>* hl, BatchLaunch* B) {
  if (!batch_schedule_valid(pr, S)) return TFT_EINVAL;
  const size_t w = pr.w;
  const int c_max = pr.w == 8 ? 12 : 13;
  const uint64_t R = 1ull << S.lr;
  const uint32_t C = 1u << S.clog;
  const uint64_t align = 16 / w;
  hs->clear();
  hl->clear();
  uint64_t work_off = 0;  // words
  int lmax = 0, cmax = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const tft_polymul_desc& d = descs[i];
    if (!d.a || !d.b || !d.out || d.na == 0 || d.nb == 0) return TFT_EINVAL;
    if (!aligned16(d.a) || !aligned16(d.b) || !aligned16(d.out))
      return TFT_EINVAL;
    const uint64_t r = d.na + d.nb - 1;
    if (overlap(d.out, r * w, d.a, d.na * w) ||
        overlap(d.out, r * w, d.b, d.nb * w))
      return TFT_EINVAL;
    if (r <= (1ull << S.small_log)) {
      BatchSmall q;
      q.a = (uint64_t)d.a;
      q.b = (uint64_t)d.b;
      q.out = (uint64_t)d.out;
      q.na = (uint32_t)d.na;
      q.nb = (uint32_t)d.nb;
      q.l = (uint32_t)ceil_log2(r);
      q.pad = 0;
      lmax = std::max(lmax, (int)q.l);
      hs->push_back(q);
      continue;
    }
    BatchLarge q;
    memset(&q, 0, sizeof(q));
    q.A = (uint32_t)(r >> S.lr);
    q.Bm = (uint32_t)(r & (R - 1));
    const uint64_t rows = q.A + (q.Bm ? 1 : 0);
    if (rows > (1ull << c_max)) return TFT_ERANGE;
    q.c = (uint32_t)ceil_log2(rows);
    cmax = std::max(cmax, (int)q.c);
    q.a = (uint64_t)d.a;
    q.b = (uint64_t)d.b;
    q.out = (uint64_t)d.out;
    q.na = d.na;
    q.nb = d.nb;
    // work area: B' (r words) then EA and EB (R words each), 16-byte slots
    unsigned char* base;
    if (work_of) {
      base = (unsigned char*)work_of[i];
      if (!base || !aligned16(base)) return TFT_EINVAL;
    } else {
      const uint64_t need = batch_product_work_words(pr, S, d.na, d.nb);
      if (work_off + need > work_cap) return TFT_ERANGE;
      base = (unsigned char*)work_base + work_off * w;
      work_off += need;
    }
    const uint64_t r_up = (r + align - 1) / align * align;
    const uint64_t R_up = (R + align - 1) / align * align;
    q.work = (uint64_t)base;
    q.EA = (uint64_t)(base + r_up * w);
    q.EB = (uint64_t)(base + (r_up + R_up) * w);
    hl->push_back(q);
  }
  // the column tile of the longest large product must fit in shared memory
  // next to the kernel's static copy of the root table
  if (!hl->empty()) {
    const size_t need = w == 8 ? col_smem_bytes<uint64_t>(cmax, S.clog)
                               : col_smem_bytes<uint32_t>(cmax, S.clog);
    if (need + sizeof(RootTable<uint64_t>) + 256 > optin) return TFT_ERANGE;
  }
  // small products largest first (the persistent CTAs then balance better)
  std::sort(hs->begin(), hs->end(),
            [](const BatchSmall& x, const BatchSmall& y) {
              return x.na + x.nb > y.na + y.nb;
            });
  // large products by column height, so that the column passes can run the
  // shorter columns in smaller tiles (more resident CTAs) than the tallest
  std::stable_sort(hl->begin(), hl->end(),
                   [](const BatchLarge& x, const BatchLarge& y) {
                     return x.c < y.c;
                   });
  uint32_t nl_lo = 0;
  int cmax_lo = 0;
  for (const BatchLarge& q : *hl)
    if ((int)q.c < cmax) {
      ++nl_lo;
      cmax_lo = std::max(cmax_lo, (int)q.c);
    }
  // the shorter-column class's tiles with their own width must fit too
  if (nl_lo > 0 && S.clog_lo >= 0) {
    const size_t need = w == 8 ? col_smem_bytes<uint64_t>(cmax_lo, S.clog_lo)
                               : col_smem_bytes<uint32_t>(cmax_lo, S.clog_lo);
    if (need + sizeof(RootTable<uint64_t>) + 256 > optin) return TFT_ERANGE;
  }
  // rows a_p (+ the full row a_p when b_p > 0); all R columns inverted,
  // R / C tiles per product
  uint64_t rows_acc = 0;
  for (BatchLarge& q : *hl) {
    q.row_base = rows_acc;
    rows_acc += q.A + (q.Bm ? 1 : 0);
  }
  const uint64_t ci_acc = (uint64_t)hl->size() * (R / C);
  memset(B, 0, sizeof(*B));
  B->nl = (uint32_t)hl->size();
  B->ns = (uint32_t)hs->size();
  B->lmax = lmax;
  B->lr = S.lr;
  B->clog = S.clog;
  B->clog_lo = S.clog_lo >= 0 ? S.clog_lo : S.clog;
  B->cmax = cmax;
  B->nl_lo = nl_lo;
  B->cmax_lo = cmax_lo;
  B->total_rows = rows_acc;
  B->ci_tiles = ci_acc;
  return TFT_OK;
}

}  // namespace tftgb

namespace {

tft_status device_optin(tft_ctx* ctx, size_t* optin) {
  int v = 0;
  if (note(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  ctx->device)) != cudaSuccess)
    return TFT_ECUDA;
  *optin = (size_t)v;
  return TFT_OK;
}

}  // namespace

tft_status tft_ctx_reserve_batch(tft_ctx* ctx, uint32_t max_products,
                                 uint64_t work_words) {
  if (!ctx || max_products == 0) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  if (ctx->batch_tab) dev_free(ctx->batch_tab);
  if (ctx->batch_work) dev_free(ctx->batch_work);
  ctx->batch_tab = ctx->batch_work = nullptr;
  ctx->batch_ready = 0;
  ctx->batch_tab_bytes =
      (uint64_t)max_products * (sizeof(BatchLarge) + sizeof(BatchSmall)) +
      256;
  if (dev_malloc((void**)&ctx->batch_tab, ctx->batch_tab_bytes) != cudaSuccess) {
    ctx->batch_tab = nullptr;
    return TFT_ENOMEM;
  }
  ctx->batch_work_words = work_words;
  if (work_words &&
      dev_malloc((void**)&ctx->batch_work, work_words * ctx->pr.w) != cudaSuccess) {
    dev_free(ctx->batch_tab);
    ctx->batch_tab = ctx->batch_work = nullptr;
    return TFT_ENOMEM;
  }
  ctx->batch_max = max_products;
  return TFT_OK;
}

tft_status tft_batch_plan(tft_ctx* ctx, const tft_polymul_desc* descs,
                          uint32_t count, const tft_batch_params* params) {
  if (!ctx || (!descs && count)) return TFT_EINVAL;
  if (!ctx->batch_tab) return TFT_EINVAL;
  if (count > ctx->batch_max) return TFT_ERANGE;
  ctx->batch_ready = 0;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  size_t optin = 0;
  tft_status st = device_optin(ctx, &optin);
  if (st != TFT_OK) return st;
  std::vector<BatchSmall> hs;
  std::vector<BatchLarge> hl;
  BatchLaunch B;
  st = batch_describe(ctx->pr, batch_schedule(ctx->pr, params), descs, count,
                      nullptr, ctx->batch_work, ctx->batch_work_words, optin,
                      &hs, &hl, &B);
  if (st != TFT_OK) return st;
  unsigned char* tab = (unsigned char*)ctx->batch_tab;
  const size_t lbytes = hl.size() * sizeof(BatchLarge);
  const size_t sbytes = hs.size() * sizeof(BatchSmall);
  const size_t soff = (lbytes + 255) & ~(size_t)255;
  if (lbytes && cudaMemcpy(tab, hl.data(), lbytes, cudaMemcpyHostToDevice) !=
                    cudaSuccess)
    return from_cuda(ctx, cudaErrorUnknown);
  if (sbytes && cudaMemcpy(tab + soff, hs.data(), sbytes,
                           cudaMemcpyHostToDevice) != cudaSuccess)
    return from_cuda(ctx, cudaErrorUnknown);
  B.large = tab;
  B.small = tab + soff;
  ctx->batch = B;
  ctx->batch_ready = 1;
  return TFT_OK;
}

tft_status tft_batch_run(tft_ctx* ctx, void* stream) {
  if (!ctx) return TFT_EINVAL;
  if (!ctx->batch_ready) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  return from_cuda(ctx, launch_batch(ctx->prime, ctx->batch, ctx->rt,
                                     ctx->nsm, (cudaStream_t)stream,
                                     &ctx->hook, &ctx->aux));
}

tft_status tft_polymul_batch(tft_ctx* ctx, const tft_polymul_desc* descs,
                             uint32_t count, const tft_batch_params* params,
                             void* stream) {
  tft_status st = tft_batch_plan(ctx, descs, count, params);
  if (st != TFT_OK) return st;
  return tft_batch_run(ctx, stream);
}

tft_status tft_batch_work_words(tft_prime prime, const tft_polymul_desc* descs,
                                uint32_t count, const tft_batch_params* params,
                                uint64_t* words) {
  if (!valid_prime((int)prime) || (!descs && count) || !words)
    return TFT_EINVAL;
  const PrimeInfo& pr = kPrimes[(int)prime];
  const BatchSchedule S = batch_schedule(pr, params);
  uint64_t total = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (descs[i].na == 0 || descs[i].nb == 0) return TFT_EINVAL;
    total += batch_product_work_words(pr, S, descs[i].na, descs[i].nb);
  }
  *words = total;
  return TFT_OK;
}
