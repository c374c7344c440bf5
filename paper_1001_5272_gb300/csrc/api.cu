// C ABI (include/tft.h): argument checking, planning, context management.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ctx.h"
#include "field.cuh"

using namespace tftgb;

namespace tftgb {

// Choose the plan for length n (see tft_internal.h).  Returns false if n is
// beyond the supported range.
bool make_plan(int prime, uint64_t n, Plan* out) {
  const PrimeInfo& pr = kPrimes[prime];
  Plan P;
  memset(&P, 0, sizeof(P));
  const int small_l = pr.w == 8 ? 12 : 13;
  const int lr_max = pr.w == 8 ? 13 : 14;
  const int c_max = pr.w == 8 ? 12 : 13;
  if (n == 0 || n > max_supported(pr)) return false;
  if (n <= (1ull << small_l)) {
    P.small = 1;
    P.l = ceil_log2(n);
    P.row_ctas_per_sm = 1;
    *out = P;
    return true;
  }
  const int lg = ceil_log2(n);
  int lr = (lg + 1) / 2;
  if (lr < 6) lr = 6;
  if (lr > lr_max) lr = lr_max;
  // column rows: a, plus one row for the long columns' last entries and the
  // short columns' E_q when b > 0
  auto col_rows = [&](int lrr) {
    return (n >> lrr) + ((n & ((1ull << lrr) - 1)) ? 1 : 0);
  };
  while (col_rows(lr) > (1ull << c_max)) {
    if (++lr > lr_max) return false;
  }
  P.lr = lr;
  P.a = n >> lr;
  P.b = n & ((1ull << lr) - 1);
  P.c = ceil_log2(col_rows(lr));
  // columns per CTA: the most (<= 16, <= R) whose tile fits ~100 KB, so that
  // two column CTAs share an SM
  const size_t budget = 100 * 1024;
  int clog = 0;
  while (clog < 4 && (1 << (clog + 1)) <= (1 << lr)) {
    Plan Q = P;
    Q.clog = clog + 1;
    if (plan_smem(prime, Q).col > budget) break;
    ++clog;
  }
  P.clog = clog;
  const size_t srow = plan_smem(prime, P).row;
  int per_sm = (int)((228 * 1024) / (srow + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  P.row_ctas_per_sm = per_sm;
  *out = P;
  return true;
}


}  // namespace tftgb


namespace {

// Release everything a (possibly partly built) context owns.
void ctx_release(tft_ctx* c) {
  for (int i = 0; i < kProfSlots; ++i) {
    if (c->prof[i].start) cudaEventDestroy(c->prof[i].start);
    if (c->prof[i].stop) cudaEventDestroy(c->prof[i].stop);
  }
  if (c->aux.fork) cudaEventDestroy(c->aux.fork);
  if (c->aux.join) cudaEventDestroy(c->aux.join);
  if (c->aux.side) cudaStreamDestroy(c->aux.side);
  if (c->stage) dev_free(c->stage);
  if (c->work) dev_free(c->work);
  if (c->scratch) dev_free(c->scratch);
  if (c->batch_tab) dev_free(c->batch_tab);
  if (c->batch_work) dev_free(c->batch_work);
  free(c);
}

}  // namespace

namespace {

void build_root_table(tft_ctx* c) {
  const PrimeInfo& pr = c->pr;
  const uint64_t top = powm(pr.g, (pr.p - 1) >> pr.K, pr.p);
  uint64_t w[33], wi[33];
  for (int j = 0; j <= 32; ++j) {
    if (j > pr.K) {
      w[j] = wi[j] = 0;
      continue;
    }
    uint64_t v = top;
    for (int i = 0; i < pr.K - j; ++i) v = mulm(v, v, pr.p);
    w[j] = v;
    wi[j] = powm(v, pr.p - 2, pr.p);
  }
  const uint64_t half = (pr.p + 1) / 2;
  // 16-point network twiddles omega_{2k} = omega_s at s = 2k, k < 8
  uint64_t c16[8], c16i[8];
  for (int k = 0; k < 8; ++k) {
    c16[k] = omega_s(pr, 2 * k);
    c16i[k] = mulm(powm(c16[k], pr.p - 2, pr.p), half, pr.p);
  }
  if (pr.w == 8) {
    RootTable<uint64_t> t;
    for (int j = 0; j <= 32; ++j) {
      t.w[j] = to_tw(pr, w[j]);
      t.winv[j] = to_tw(pr, wi[j]);
    }
    t.half_tw = to_tw(pr, half);
    t.one_tw = to_tw(pr, 1);
    for (int k = 0; k < 8; ++k) {
      t.c16[k] = to_tw(pr, c16[k]);
      t.c16i[k] = to_tw(pr, c16i[k]);
    }
    memcpy(c->rt, &t, sizeof(t));
  } else {
    RootTable<uint32_t> t;
    for (int j = 0; j <= 32; ++j) {
      t.w[j] = (uint32_t)to_tw(pr, w[j]);
      t.winv[j] = (uint32_t)to_tw(pr, wi[j]);
    }
    t.half_tw = (uint32_t)to_tw(pr, half);
    t.one_tw = (uint32_t)to_tw(pr, 1);
    for (int k = 0; k < 8; ++k) {
      t.c16[k] = (uint32_t)to_tw(pr, c16[k]);
      t.c16i[k] = (uint32_t)to_tw(pr, c16i[k]);
    }
    memcpy(c->rt, &t, sizeof(t));
  }
}

// The Montgomery constants compiled into field.cuh must match the moduli.
bool check_constants() {
  auto chk = [](uint32_t p, uint32_t pinv, uint32_t r2, uint32_t one) {
    return (uint32_t)(p * pinv) == 0xFFFFFFFFu &&
           r2 == (uint32_t)(((u128)1 << 64) % p) &&
           one == (uint32_t)(((uint64_t)1 << 32) % p);
  };
  if (!chk(P998::P, P998::PINV, P998::R2, P998::ONE) ||
      !chk(P2013::P, P2013::PINV, P2013::R2, P2013::ONE))
    return false;
  // the 16-point network's constants of 2^64 - 2^32 + 1 that the kernels
  // apply as +-2^s by shifts must be the root table's omega_{2k} (and their
  // inverses)
  const PrimeInfo& g = kPrimes[2];
  for (int k = 1; k < 8; ++k) {
    const uint64_t c = omega_s(g, 2 * k);
    const uint64_t ci = powm(c, g.p - 2, g.p);
    for (int inv = 0; inv < 2; ++inv) {
      const int sh = inv ? Goldilocks::kNetInvShift[k] : Goldilocks::kNetShift[k];
      if (sh == 0) continue;
      const uint64_t v = powm(2, (uint64_t)sh, g.p);
      const uint64_t want = Goldilocks::net_neg(k, inv != 0) ? g.p - v : v;
      if ((inv ? ci : c) != want) return false;
    }
  }
  return true;
}

std::mutex g_prep_mu;
bool g_prepared[3][64] = {};

thread_local const char* g_last_cuda_error = "no error";

}  // namespace

namespace tftgb {

cudaError_t note(cudaError_t e) {
  if (e != cudaSuccess) g_last_cuda_error = cudaGetErrorName(e);
  return e;
}

namespace {
std::mutex g_alloc_mu;
int64_t g_alloc_fail_after = -1;  // allocations to pass before one fails
int64_t g_live_allocs = 0;

// true: this allocation is to fail (the injected failure is used up)
bool inject_failure() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (g_alloc_fail_after < 0) return false;
  if (g_alloc_fail_after == 0) {
    g_alloc_fail_after = -1;
    return true;
  }
  --g_alloc_fail_after;
  return false;
}
void count_alloc(int64_t d) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_live_allocs += d;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (inject_failure()) return note(cudaErrorMemoryAllocation);
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return note(e);
  }
  count_alloc(1);
  return e;
}

void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  count_alloc(-1);
}

cudaError_t host_malloc_pinned(void** p, size_t bytes) {
  *p = nullptr;
  if (inject_failure()) return note(cudaErrorMemoryAllocation);
  const cudaError_t e = cudaMallocHost(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return note(e);
  }
  count_alloc(1);
  return e;
}

void host_free_pinned(void* p) {
  if (!p) return;
  cudaFreeHost(p);
  count_alloc(-1);
}

tft_status from_cuda(tft_ctx* ctx, cudaError_t e) {
  if (e == cudaSuccess) return TFT_OK;
  note(e);
  if (ctx) ctx->sticky = TFT_ECUDA;
  return TFT_ECUDA;
}

}  // namespace tftgb

namespace {


void prof_drain(tft_ctx* c) {
  for (int i = 0; i < c->prof_pending; ++i) {
    float ms = 0.f;
    if (cudaEventSynchronize(c->prof[i].stop) == cudaSuccess &&
        cudaEventElapsedTime(&ms, c->prof[i].start, c->prof[i].stop) ==
            cudaSuccess) {
      c->prof_ms[c->prof[i].kind] += ms;
      c->prof_count[c->prof[i].kind] += 1;
    }
  }
  c->prof_pending = 0;
}

void hook_before(void* user, int kind, cudaStream_t s) {
  tft_ctx* c = (tft_ctx*)user;
  if (!c->prof_on) return;
  if (c->prof_pending == kProfSlots) prof_drain(c);
  cudaEventRecord(c->prof[c->prof_pending].start, s);
  (void)kind;
}

void hook_after(void* user, int kind, cudaStream_t s) {
  tft_ctx* c = (tft_ctx*)user;
  c->launches++;
  if (!c->prof_on) return;
  ProfSlot& sl = c->prof[c->prof_pending];
  cudaEventRecord(sl.stop, s);
  sl.kind = kind;
  c->prof_pending++;
}

tft_status check_transform_args(tft_ctx* ctx, const void* x, uint64_t n,
                                uint32_t k) {
  if (!ctx || !x) return TFT_EINVAL;
  if (n == 0) return TFT_EINVAL;
  if ((int)k > ctx->pr.K) return TFT_EINVAL;
  if (k < 64 && n > (1ull << k)) return TFT_EINVAL;
  if (!aligned16(x)) return TFT_EINVAL;
  if (n > ctx->max_len) return TFT_ERANGE;
  return TFT_OK;
}


// One staging slot: max_len words rounded up to 256 bytes.
size_t stage_slot_bytes(const tft_ctx* ctx) {
  return (ctx->max_len * ctx->pr.w + 255) & ~(size_t)255;
}

uint64_t omega_a_tw(tft_ctx* ctx, const Plan& P) {
  return to_tw(ctx->pr, omega_s(ctx->pr, P.a));
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for tft_forward_noalloc: a fixed array in device memory instead of
// a context.  Its capacity covers the scratch of every plan the library makes
// (one row of at most 2^14 words), whatever n is.
// ---------------------------------------------------------------------------
constexpr size_t kNoallocScratchWords = (size_t)1 << 14;  // 128 KiB
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoallocScratchWords];

namespace {

// Once per (prime, device), with that device current: read the SM count
// and set the kernels' shared-memory limits for `prime`.  Host state only;
// no device memory is touched.
std::mutex g_devinfo_mu;
int g_devinfo_nsm[64];

tft_status device_prepare(int prime, int dev, int* nsm_out) {
  if (dev < 0 || dev >= 64) return TFT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(g_devinfo_mu);
    if (g_devinfo_nsm[dev] == 0) {
      int nsm = 0;
      if (note(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount,
                                      dev)) != cudaSuccess)
        return TFT_ECUDA;
      g_devinfo_nsm[dev] = nsm;
    }
    *nsm_out = g_devinfo_nsm[dev];
  }
  std::lock_guard<std::mutex> lk2(g_prep_mu);
  if (!g_prepared[prime][dev]) {
    int optin = 0;
    if (note(cudaDeviceGetAttribute(&optin,
                                    cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                    dev)) != cudaSuccess)
      return TFT_ECUDA;
    if (note(prepare_kernels(prime, (size_t)optin)) != cudaSuccess)
      return TFT_ECUDA;
    g_prepared[prime][dev] = true;
  }
  return TFT_OK;
}

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];  // device address of g_noalloc_scratch per device

// Once per device, with that device current: resolve the array's device
// address (the host-side name is only a stand-in), then the device set-up
// above.
tft_status noalloc_setup(int prime, int dev, void** scratch, int* nsm) {
  if (dev < 0 || dev >= 64) return TFT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (note(cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
        return TFT_ECUDA;
      g_noalloc_addr[dev] = p;
    }
    *scratch = g_noalloc_addr[dev];
  }
  return device_prepare(prime, dev, nsm);
}

}  // namespace

extern "C" {

void tft_debug_fail_allocation(int64_t n) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_fail_after = n < 0 ? -1 : n;
}

int64_t tft_debug_live_allocations(void) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_live_allocs;
}

tft_status tft_forward_noalloc(tft_prime prime, void* x, uint64_t n,
                               uint32_t k, void* stream) {
  if (!valid_prime((int)prime) || !x || n == 0) return TFT_EINVAL;
  const PrimeInfo& pr = kPrimes[(int)prime];
  if ((int)k > pr.K || (k < 64 && n > (1ull << k))) return TFT_EINVAL;
  if (!aligned16(x)) return TFT_EINVAL;
  Plan P;
  if (!make_plan((int)prime, n, &P)) return TFT_ERANGE;
  const uint64_t need_words = P.small ? 0 : (1ull << P.lr);
  if (need_words * pr.w > sizeof(g_noalloc_scratch)) return TFT_ERANGE;
  int dev = -1;
  if (note(cudaGetDevice(&dev)) != cudaSuccess) return TFT_ECUDA;
  void* scratch = nullptr;
  int nsm = 0;
  tft_status st = noalloc_setup((int)prime, dev, &scratch, &nsm);
  if (st != TFT_OK) return st;
  // The root table is built on the stack; nothing is allocated.
  tft_ctx tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.pr = pr;
  build_root_table(&tmp);
  cudaError_t e = launch_forward((int)prime, x, n, P, scratch, tmp.rt, nsm,
                                 (cudaStream_t)stream, nullptr, nullptr);
  if (e != cudaSuccess) {
    note(e);
    return TFT_ECUDA;
  }
  return TFT_OK;
}

static tft_status noscratch_transform(tft_prime prime, void* x, uint64_t n,
                                      uint32_t k, void* stream, bool inv) {
  if (!valid_prime((int)prime) || !x || n == 0) return TFT_EINVAL;
  const PrimeInfo& pr = kPrimes[(int)prime];
  if ((int)k > pr.K || (k < 64 && n > (1ull << k))) return TFT_EINVAL;
  if (!aligned16(x)) return TFT_EINVAL;
  Plan P;
  if (!make_plan((int)prime, n, &P)) return TFT_ERANGE;
  int dev = -1;
  if (note(cudaGetDevice(&dev)) != cudaSuccess) return TFT_ECUDA;
  int nsm = 0;
  tft_status st = device_prepare((int)prime, dev, &nsm);
  if (st != TFT_OK) return st;
  // The root table is built on the stack; nothing is allocated and no
  // device memory but x is read or written.
  tft_ctx tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.pr = pr;
  build_root_table(&tmp);
  const uint64_t wa = P.small ? 0 : to_tw(pr, omega_s(pr, P.a));
  cudaError_t e =
      inv ? launch_inverse_zs((int)prime, x, n, P, wa, tmp.rt, nsm,
                              (cudaStream_t)stream, nullptr)
          : launch_forward_zs((int)prime, x, n, P, wa, tmp.rt, nsm,
                              (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) {
    note(e);
    return TFT_ECUDA;
  }
  return TFT_OK;
}

tft_status tft_forward_noscratch(tft_prime prime, void* x, uint64_t n,
                                 uint32_t k, void* stream) {
  return noscratch_transform(prime, x, n, k, stream, false);
}

tft_status tft_inverse_noscratch(tft_prime prime, void* x, uint64_t n,
                                 uint32_t k, void* stream) {
  return noscratch_transform(prime, x, n, k, stream, true);
}

tft_status tft_ctx_create(tft_prime prime, int device, uint64_t max_len,
                          uint32_t flags, tft_ctx** out) {
  if (!out) return TFT_EINVAL;
  *out = nullptr;
  if (!valid_prime((int)prime) || max_len == 0 || device < 0)
    return TFT_EINVAL;
  if (!check_constants()) return TFT_EINVAL;
  const PrimeInfo& pr = kPrimes[(int)prime];
  if (max_len > max_supported(pr)) return TFT_ERANGE;
  int ndev = 0;
  if (note(cudaGetDeviceCount(&ndev)) != cudaSuccess) return TFT_ECUDA;
  if (device >= ndev) return TFT_EINVAL;
  DeviceGuard g(device);
  if (!g.ok) return TFT_ECUDA;
  {
    std::lock_guard<std::mutex> lk(g_prep_mu);
    if (device < 64 && !g_prepared[(int)prime][device]) {
      int optin = 0;
      if (note(cudaDeviceGetAttribute(&optin,
                                      cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                      device)) != cudaSuccess)
        return TFT_ECUDA;
      if (note(prepare_kernels((int)prime, (size_t)optin)) != cudaSuccess)
        return TFT_ECUDA;
      g_prepared[(int)prime][device] = true;
    }
  }
  tft_ctx* c = (tft_ctx*)calloc(1, sizeof(tft_ctx));
  if (!c) return TFT_ENOMEM;
  c->prime = (int)prime;
  c->device = device;
  c->max_len = max_len;
  c->flags = flags;
  c->pr = pr;
  c->sticky = TFT_OK;
  if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount,
                             device) != cudaSuccess) {
    free(c);
    return TFT_ECUDA;
  }
  build_root_table(c);
  c->hook.before = hook_before;
  c->hook.after = hook_after;
  c->hook.user = c;
  for (int i = 0; i < kProfSlots; ++i) {
    if (note(cudaEventCreate(&c->prof[i].start)) != cudaSuccess ||
        note(cudaEventCreate(&c->prof[i].stop)) != cudaSuccess) {
      ctx_release(c);
      return TFT_ECUDA;
    }
  }
  if (note(cudaStreamCreateWithFlags(&c->aux.side, cudaStreamNonBlocking)) !=
          cudaSuccess ||
      note(cudaEventCreateWithFlags(&c->aux.fork, cudaEventDisableTiming)) !=
          cudaSuccess ||
      note(cudaEventCreateWithFlags(&c->aux.join, cudaEventDisableTiming)) !=
          cudaSuccess) {
    ctx_release(c);
    return TFT_ECUDA;
  }
  const size_t w = pr.w;
  if (dev_malloc((void**)&c->scratch, kCtxScratchWords * w) != cudaSuccess ||
      dev_malloc((void**)&c->work, max_len * w) != cudaSuccess) {
    ctx_release(c);
    return TFT_ENOMEM;
  }
  if (flags & TFT_CTX_HOST_STAGING) {
    if (dev_malloc((void**)&c->stage, 3 * stage_slot_bytes(c)) != cudaSuccess) {
      ctx_release(c);
      return TFT_ENOMEM;
    }
  }
  *out = c;
  return TFT_OK;
}

tft_status tft_ctx_destroy(tft_ctx* ctx) {
  if (!ctx) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  ctx_release(ctx);
  return TFT_OK;
}

tft_status tft_forward(tft_ctx* ctx, void* x, uint64_t n, uint32_t k,
                       void* stream) {
  tft_status st = check_transform_args(ctx, x, n, k);
  if (st != TFT_OK) return st;
  Plan P;
  if (!make_plan(ctx->prime, n, &P)) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  return from_cuda(ctx, launch_forward(ctx->prime, x, n, P, ctx->scratch,
                                       ctx->rt, ctx->nsm,
                                       (cudaStream_t)stream, &ctx->hook,
                                       &ctx->aux));
}

tft_status tft_inverse(tft_ctx* ctx, void* X, uint64_t n, uint32_t k,
                       void* stream) {
  tft_status st = check_transform_args(ctx, X, n, k);
  if (st != TFT_OK) return st;
  Plan P;
  if (!make_plan(ctx->prime, n, &P)) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  return from_cuda(ctx, launch_inverse(ctx->prime, X, n, P, ctx->scratch,
                                       P.small ? 0 : omega_a_tw(ctx, P),
                                       ctx->rt, ctx->nsm,
                                       (cudaStream_t)stream, &ctx->hook));
}

tft_status tft_transform_batch(tft_ctx* ctx, int inverse,
                               const tft_transform_desc* descs,
                               uint32_t count, void* stream) {
  if (!ctx || (!descs && count)) return TFT_EINVAL;
  if (count == 0) return TFT_OK;
  const size_t w = ctx->pr.w;
  std::vector<XformDesc> small;
  std::vector<std::pair<uintptr_t, uint64_t>> spans;
  small.reserve(count);
  spans.reserve(count);
  int lmax = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const tft_transform_desc& d = descs[i];
    if (!d.x || d.n == 0 || !aligned16(d.x)) return TFT_EINVAL;
    if (d.n > ctx->max_len) return TFT_ERANGE;
    Plan P;
    if (!make_plan(ctx->prime, d.n, &P)) return TFT_ERANGE;
    spans.push_back({(uintptr_t)d.x, d.n * w});
    if (P.small) {
      small.push_back(XformDesc{(uint64_t)d.x, (uint32_t)d.n, (uint32_t)P.l});
      if (P.l > lmax) lmax = P.l;
    }
  }
  // the buffers must not overlap (each is transformed in place)
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); ++i)
    if (spans[i - 1].first + spans[i - 1].second > spans[i].first)
      return TFT_EINVAL;
  if (!small.empty() &&
      (!ctx->batch_tab || small.size() > ctx->batch_max ||
       small.size() * sizeof(XformDesc) > ctx->batch_tab_bytes))
    return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (!small.empty()) {
    // the table goes into the batch reservation (a product plan there is
    // dropped); pageable source: the copy is staged before the call returns
    ctx->batch_ready = 0;
    cudaError_t e = cudaMemcpyAsync(ctx->batch_tab, small.data(),
                                    small.size() * sizeof(XformDesc),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_small_batch(ctx->prime, ctx->batch_tab,
                             (uint32_t)small.size(), lmax, inverse ? 1 : 0,
                             ctx->rt, ctx->nsm, s, &ctx->hook);
    if (e != cudaSuccess) return from_cuda(ctx, e);
  }
  // the longer transforms one after another on the stream (they share the
  // context's scratch)
  for (uint32_t i = 0; i < count; ++i) {
    const tft_transform_desc& d = descs[i];
    Plan P;
    make_plan(ctx->prime, d.n, &P);
    if (P.small) continue;
    cudaError_t e =
        inverse ? launch_inverse(ctx->prime, d.x, d.n, P, ctx->scratch,
                                 omega_a_tw(ctx, P), ctx->rt, ctx->nsm, s,
                                 &ctx->hook)
                : launch_forward(ctx->prime, d.x, d.n, P, ctx->scratch,
                                 ctx->rt, ctx->nsm, s, &ctx->hook, &ctx->aux);
    if (e != cudaSuccess) return from_cuda(ctx, e);
  }
  return TFT_OK;
}

// The plan of a transform of length n held in `parts` parts, and the
// column block plan of part `part` (row stride W = R / parts, b = the
// block's long columns).
static tft_status shard_plans(tft_ctx* ctx, uint64_t n, uint32_t parts,
                              uint32_t part, Plan* P, Plan* Pc) {
  if (!ctx || n == 0 || parts == 0 || (parts & (parts - 1)) ||
      part >= parts)
    return TFT_EINVAL;
  if (!make_plan(ctx->prime, n, P)) return TFT_ERANGE;
  if (P->small || P->lr < 8) return TFT_EINVAL;
  int lp = 0;
  while ((1u << lp) < parts) ++lp;
  if (lp > P->lr) return TFT_EINVAL;
  *Pc = *P;
  Pc->lr = P->lr - lp;
  const uint64_t W = 1ull << Pc->lr;
  const uint64_t q0 = (uint64_t)part * W;
  Pc->b = P->b > q0 ? (P->b - q0 < W ? P->b - q0 : W) : 0;
  return TFT_OK;
}

tft_status tft_shard_columns(tft_ctx* ctx, int inverse, int which,
                             void* block, uint64_t n, uint32_t parts,
                             uint32_t part, void* E, void* stream) {
  Plan P, Pc;
  tft_status st = shard_plans(ctx, n, parts, part, &P, &Pc);
  if (st != TFT_OK) return st;
  if (!block || !aligned16(block) || (E && !aligned16(E))) return TFT_EINVAL;
  if (inverse && which != 0 && which != 1) return TFT_EINVAL;
  const uint64_t W = 1ull << Pc.lr;
  // E is read or written for the block's short columns when the transform
  // has a ragged last row
  const int want_E = P.b > 0 && Pc.b < W && (!inverse || which == 0);
  if (want_E && !E) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  return from_cuda(ctx, launch_shard_cols(ctx->prime, inverse ? 1 : 0, which,
                                          block, Pc, E, want_E,
                                          omega_a_tw(ctx, P), ctx->rt,
                                          ctx->nsm, (cudaStream_t)stream,
                                          &ctx->hook));
}

tft_status tft_shard_rows(tft_ctx* ctx, int inverse, void* rows, uint64_t n,
                          uint64_t rho_begin, uint64_t count, void* stream) {
  Plan P, Pc;
  tft_status st = shard_plans(ctx, n, 1, 0, &P, &Pc);
  if (st != TFT_OK) return st;
  if ((count && (!rows || !aligned16(rows))) || rho_begin + count > P.a)
    return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  return from_cuda(ctx, launch_shard_rows(ctx->prime, inverse ? 1 : 0, rows,
                                          count, rho_begin, P.lr, ctx->rt,
                                          ctx->nsm, (cudaStream_t)stream,
                                          &ctx->hook));
}

tft_status tft_shard_last_row(tft_ctx* ctx, int inverse, void* row,
                              const void* E, uint64_t n, void* stream) {
  Plan P, Pc;
  tft_status st = shard_plans(ctx, n, 1, 0, &P, &Pc);
  if (st != TFT_OK) return st;
  if (P.b == 0) return TFT_OK;  // no ragged row
  if (!row || !E || !aligned16(row) || !aligned16(E)) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  return from_cuda(ctx, launch_shard_last(ctx->prime, inverse ? 1 : 0, row, E,
                                          P.a, P.b, P.lr, ctx->rt,
                                          (cudaStream_t)stream, &ctx->hook));
}

tft_status tft_polymul(tft_ctx* ctx, const void* a, uint64_t na,
                       const void* b, uint64_t nb, void* out, void* stream) {
  if (!ctx || !a || !b || !out || na == 0 || nb == 0) return TFT_EINVAL;
  if (!aligned16(a) || !aligned16(b) || !aligned16(out)) return TFT_EINVAL;
  const uint64_t r = na + nb - 1;
  const size_t w = ctx->pr.w;
  if (overlap(out, r * w, a, na * w) || overlap(out, r * w, b, nb * w))
    return TFT_EINVAL;
  if (r > ctx->max_len) return TFT_ERANGE;
  Plan P;
  if (!make_plan(ctx->prime, r, &P)) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  unsigned char* s = (unsigned char*)ctx->scratch;
  void* EA = s;
  void* EB = s + (1ull << 14) * w;
  return from_cuda(ctx, launch_polymul(ctx->prime, a, na, b, nb, out, P,
                                       ctx->work, EA, EB,
                                       P.small ? 0 : omega_a_tw(ctx, P),
                                       ctx->rt, ctx->nsm,
                                       (cudaStream_t)stream, &ctx->hook,
                                       &ctx->aux));
}

tft_status tft_polymul_padded(tft_ctx* ctx, const void* a, uint64_t na,
                              const void* b, uint64_t nb, void* out,
                              void* scratch, void* stream) {
  if (!ctx || !a || !b || !out || !scratch || na == 0 || nb == 0)
    return TFT_EINVAL;
  if (!aligned16(a) || !aligned16(b) || !aligned16(out) ||
      !aligned16(scratch))
    return TFT_EINVAL;
  const uint64_t r = na + nb - 1;
  const size_t w = ctx->pr.w;
  const uint64_t N = 1ull << ceil_log2(r);
  if (overlap(out, r * w, a, na * w) || overlap(out, r * w, b, nb * w) ||
      overlap(scratch, 2 * N * w, a, na * w) ||
      overlap(scratch, 2 * N * w, b, nb * w) ||
      overlap(scratch, 2 * N * w, out, r * w))
    return TFT_EINVAL;
  Plan P;
  if (!make_plan(ctx->prime, N, &P)) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  unsigned char* sc = (unsigned char*)scratch;
  unsigned char* e = (unsigned char*)ctx->scratch;
  cudaStream_t s = (cudaStream_t)stream;
  // both operands zero-extended to N (implicitly, by the column pass), the
  // length-N transforms, pointwise product and inverse; then the first r
  // coefficients (the rest are zero) to out
  cudaError_t err = launch_polymul(ctx->prime, a, na, b, nb, sc, P,
                                   sc + N * w, e, e + (1ull << 14) * w,
                                   P.small ? 0 : omega_a_tw(ctx, P), ctx->rt,
                                   ctx->nsm, s, &ctx->hook, &ctx->aux);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(out, sc, r * w, cudaMemcpyDeviceToDevice, s);
  return from_cuda(ctx, err);
}

static tft_status host_transform(tft_ctx* ctx, void* xh, uint64_t n,
                                 uint32_t k, void* stream, bool inv) {
  if (!ctx || !xh) return TFT_EINVAL;
  if (!(ctx->flags & TFT_CTX_HOST_STAGING) || !ctx->stage) return TFT_EINVAL;
  if (n == 0) return TFT_EINVAL;
  if (n > ctx->max_len) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = n * ctx->pr.w;
  if (cudaMemcpyAsync(ctx->stage, xh, bytes, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return from_cuda(ctx, cudaErrorUnknown);
  tft_status st = inv ? tft_inverse(ctx, ctx->stage, n, k, stream)
                      : tft_forward(ctx, ctx->stage, n, k, stream);
  if (st != TFT_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  if (cudaMemcpyAsync(xh, ctx->stage, bytes, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return from_cuda(ctx, cudaErrorUnknown);
  return from_cuda(ctx, cudaStreamSynchronize(s));
}

tft_status tft_forward_host(tft_ctx* ctx, void* x_host, uint64_t n,
                            uint32_t k, void* stream) {
  return host_transform(ctx, x_host, n, k, stream, false);
}

tft_status tft_inverse_host(tft_ctx* ctx, void* X_host, uint64_t n,
                            uint32_t k, void* stream) {
  return host_transform(ctx, X_host, n, k, stream, true);
}

tft_status tft_polymul_host(tft_ctx* ctx, const void* a_host, uint64_t na,
                            const void* b_host, uint64_t nb, void* out_host,
                            void* stream) {
  if (!ctx || !a_host || !b_host || !out_host || na == 0 || nb == 0)
    return TFT_EINVAL;
  if (!(ctx->flags & TFT_CTX_HOST_STAGING) || !ctx->stage) return TFT_EINVAL;
  const uint64_t r = na + nb - 1;
  if (r > ctx->max_len) return TFT_ERANGE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  const size_t w = ctx->pr.w;
  // staging layout: [out][a][b], each max_len words rounded up to 256 bytes
  unsigned char* base = (unsigned char*)ctx->stage;
  const size_t slot = stage_slot_bytes(ctx);
  void* dout = base;
  void* da = base + slot;
  void* db = base + 2 * slot;
  cudaStream_t s = (cudaStream_t)stream;
  // a is copied first; b follows on the side stream, where its column pass
  // will run, so that a's column pass overlaps b's copy
  const AuxStreams& ax = ctx->aux;
  if (cudaMemcpyAsync(da, a_host, na * w, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaEventRecord(ax.fork, s) != cudaSuccess ||
      cudaStreamWaitEvent(ax.side, ax.fork, 0) != cudaSuccess ||
      cudaMemcpyAsync(db, b_host, nb * w, cudaMemcpyHostToDevice, ax.side) !=
          cudaSuccess)
    return from_cuda(ctx, cudaErrorUnknown);
  Plan P;
  if (make_plan(ctx->prime, r, &P) && P.small) {
    // the single-CTA product reads both operands on s
    if (cudaEventRecord(ax.join, ax.side) != cudaSuccess ||
        cudaStreamWaitEvent(s, ax.join, 0) != cudaSuccess)
      return from_cuda(ctx, cudaErrorUnknown);
  }
  tft_status st = tft_polymul(ctx, da, na, db, nb, dout, stream);
  if (st != TFT_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  if (cudaMemcpyAsync(out_host, dout, r * w, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return from_cuda(ctx, cudaErrorUnknown);
  return from_cuda(ctx, cudaStreamSynchronize(s));
}

tft_status tft_footprint(tft_prime prime, uint64_t n, uint32_t k, int op,
                         uint64_t* inplace_bytes, uint64_t* padded_bytes) {
  if (!valid_prime((int)prime) || !inplace_bytes || !padded_bytes || n == 0)
    return TFT_EINVAL;
  const PrimeInfo& pr = kPrimes[(int)prime];
  if (k == 0) k = (uint32_t)ceil_log2(n);
  if ((int)k > pr.K || (k < 64 && n > (1ull << k))) return TFT_EINVAL;
  Plan P;
  if (!make_plan((int)prime, n, &P)) return TFT_ERANGE;
  const uint64_t w = pr.w;
  const uint64_t R = P.small ? 0 : (1ull << P.lr);
  if (op == 0) {
    *inplace_bytes = (n + (P.b ? R : 0)) * w;
    *padded_bytes = (1ull << k) * w;
  } else if (op == 1) {
    *inplace_bytes = (2 * n + (P.small ? 0 : 2 * R)) * w;
    *padded_bytes = 2 * (1ull << k) * w;
  } else {
    return TFT_EINVAL;
  }
  return TFT_OK;
}

tft_status tft_describe_plan(tft_prime prime, uint64_t n, int64_t out[8]) {
  if (!valid_prime((int)prime) || !out) return TFT_EINVAL;
  Plan P;
  if (!make_plan((int)prime, n, &P)) return TFT_ERANGE;
  out[0] = P.small;
  out[1] = P.l;
  out[2] = P.lr;
  out[3] = P.c;
  out[4] = P.clog;
  out[5] = (int64_t)P.a;
  out[6] = (int64_t)P.b;
  out[7] = P.row_ctas_per_sm;
  return TFT_OK;
}

uint32_t tft_element_bytes(tft_prime prime) {
  return valid_prime((int)prime) ? kPrimes[(int)prime].w : 0;
}

tft_status tft_last_error(tft_ctx* ctx) {
  if (!ctx) return TFT_EINVAL;
  if (ctx->sticky != TFT_OK) return ctx->sticky;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaPeekAtLastError();
  return e == cudaSuccess ? TFT_OK : TFT_ECUDA;
}

tft_status tft_profile_enable(tft_ctx* ctx, int enable) {
  if (!ctx) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  prof_drain(ctx);
  for (int k = 0; k < K_NUM_KINDS; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_count[k] = 0;
  }
  ctx->prof_on = enable ? 1 : 0;
  return TFT_OK;
}

tft_status tft_profile_read(tft_ctx* ctx, double* ms, uint64_t* launches) {
  if (!ctx || !ms || !launches) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  prof_drain(ctx);
  for (int k = 0; k < K_NUM_KINDS; ++k) {
    ms[k] = ctx->prof_ms[k];
    launches[k] = ctx->prof_count[k];
  }
  return TFT_OK;
}

const char* tft_kernel_name(int kind) {
  static const char* names[K_NUM_KINDS] = {
      "k_small",   "k_small_mul",   "k_col_fwd",     "k_row_fwd",
      "k_row_inv", "k_col_inv",     "k_lastrow_inv", "k_row_mul",
      "k_lastrow_fwd", "k_lastrow_mul", "k_gen", "k_fold"};
  return (kind >= 0 && kind < K_NUM_KINDS) ? names[kind] : "unknown";
}

uint64_t tft_launch_count(tft_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* tft_last_cuda_error(void) { return g_last_cuda_error; }

const char* tft_status_string(tft_status s) {
  switch (s) {
    case TFT_OK: return "ok";
    case TFT_EINVAL: return "invalid argument";
    case TFT_ERANGE: return "size out of range";
    case TFT_ENOMEM: return "out of device memory";
    case TFT_ECUDA: return "CUDA error";
    case TFT_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

}  // extern "C"
