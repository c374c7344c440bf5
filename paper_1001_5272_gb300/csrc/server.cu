// Served products: a request stream run through the batched product with
// continuous batching and admission by in-place bytes (include/tft.h:
// tft_server_*), the one-by-one comparison path, the device operand
// generator's C entry point, and the host-side device-memory arena the
// server allocates from.  Host code; the kernels it launches live in the
// field translation units and gen.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "ctx.h"

using namespace tftgb;

// ---------------------------------------------------------------------------
// Arena: first-fit allocation of byte ranges of [0, size) in multiples of
// `align`, with free ranges coalesced on release.  Pure host bookkeeping (the
// server maps offsets onto one device allocation).
// ---------------------------------------------------------------------------
struct tft_arena {
  uint64_t size = 0;
  uint64_t align = 256;
  uint64_t used = 0;
  uint64_t peak = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> length
  std::map<uint64_t, uint64_t> live_;  // offset -> length

  void init(uint64_t sz, uint64_t al) {
    align = al;
    size = sz / al * al;
    used = peak = 0;
    free_.clear();
    live_.clear();
    if (size) free_[0] = size;
  }
  uint64_t round(uint64_t b) const { return (b + align - 1) / align * align; }
  bool alloc(uint64_t bytes, uint64_t* off) {
    const uint64_t need = round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const uint64_t o = it->first, len = it->second;
      free_.erase(it);
      if (len > need) free_[o + need] = len - need;
      live_[o] = need;
      used += need;
      if (used > peak) peak = used;
      *off = o;
      return true;
    }
    return false;
  }
  bool release(uint64_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    uint64_t o = off, len = it->second;
    live_.erase(it);
    used -= len;
    auto nx = free_.lower_bound(o);
    if (nx != free_.end() && nx->first == o + len) {  // merge right
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {  // merge left
      auto pv = std::prev(nx);
      if (pv->first + pv->second == o) {
        o = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[o] = len;
    return true;
  }
};

tft_status tft_arena_create(uint64_t size, uint64_t align, tft_arena** out) {
  if (!out || align == 0 || (align & (align - 1)) || size < align)
    return TFT_EINVAL;
  tft_arena* a = new (std::nothrow) tft_arena();
  if (!a) return TFT_ENOMEM;
  a->init(size, align);
  *out = a;
  return TFT_OK;
}

tft_status tft_arena_destroy(tft_arena* a) {
  if (!a) return TFT_EINVAL;
  delete a;
  return TFT_OK;
}

tft_status tft_arena_alloc(tft_arena* a, uint64_t bytes, uint64_t* offset) {
  if (!a || !offset) return TFT_EINVAL;
  return a->alloc(bytes, offset) ? TFT_OK : TFT_ENOMEM;
}

tft_status tft_arena_free(tft_arena* a, uint64_t offset) {
  if (!a) return TFT_EINVAL;
  return a->release(offset) ? TFT_OK : TFT_EINVAL;
}

tft_status tft_arena_usage(tft_arena* a, uint64_t* used, uint64_t* peak,
                           uint64_t* free_ranges) {
  if (!a) return TFT_EINVAL;
  if (used) *used = a->used;
  if (peak) *peak = a->peak;
  if (free_ranges) *free_ranges = a->free_.size();
  return TFT_OK;
}

// ---------------------------------------------------------------------------
// Generator entry point
// ---------------------------------------------------------------------------
tft_status tft_generate(tft_ctx* ctx, uint64_t seed, uint64_t request,
                        uint32_t operand, void* out, uint64_t n,
                        void* stream) {
  // the element index is one 32-bit counter word
  if (!ctx || !out || n == 0 || n > (1ull << 32) || operand > 1)
    return TFT_EINVAL;
  if (!aligned16(out)) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->hook.before(ctx->hook.user, K_GEN, s);
  const cudaError_t e =
      operand ? launch_gen_pair(ctx->prime, nullptr, 0, out, n, request, seed,
                                ctx->nsm, s)
              : launch_gen_pair(ctx->prime, out, n, nullptr, 0, request, seed,
                                ctx->nsm, s);
  ctx->hook.after(ctx->hook.user, K_GEN, s);
  return from_cuda(ctx, e);
}

// ---------------------------------------------------------------------------
// Request footprint
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kBlockAlign = 256;

uint64_t up256(uint64_t b) { return (b + kBlockAlign - 1) & ~(kBlockAlign - 1); }

// Layout of one request's block: a | b | out | work (work only for the
// row/column class), each part 256-byte aligned.
struct ReqLayout {
  uint64_t a, b, out, work, total;
};

ReqLayout request_layout(const PrimeInfo& pr, const BatchSchedule& S,
                         uint64_t na, uint64_t nb) {
  ReqLayout L;
  const uint64_t r = na + nb - 1;
  L.a = 0;
  L.b = L.a + up256(na * pr.w);
  L.out = L.b + up256(nb * pr.w);
  L.work = L.out + up256(r * pr.w);
  L.total = L.work + up256(batch_product_work_words(pr, S, na, nb) * pr.w);
  return L;
}

}  // namespace

tft_status tft_request_bytes(tft_prime prime, uint64_t na, uint64_t nb,
                             const tft_batch_params* params, uint64_t* bytes) {
  if (!valid_prime((int)prime) || na == 0 || nb == 0 || !bytes)
    return TFT_EINVAL;
  const PrimeInfo& pr = kPrimes[(int)prime];
  const BatchSchedule S = batch_schedule(pr, params);
  if (!batch_schedule_valid(pr, S)) return TFT_EINVAL;
  *bytes = request_layout(pr, S, na, nb).total;
  return TFT_OK;
}

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------
namespace {

constexpr int kSlots = 2;  // batches in flight

struct Slot {
  void* dtab = nullptr;     // device tables (GenDesc | BatchLarge | BatchSmall)
  void* htab = nullptr;     // pinned staging of the same bytes
  size_t tab_bytes = 0;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<uint64_t> reqs;   // request indices
  std::vector<uint64_t> blocks; // arena offsets
};

}  // namespace

struct tft_server {
  tft_ctx* ctx = nullptr;
  BatchSchedule S{};
  uint32_t max_batch = 0;
  size_t optin = 0;
  void* base = nullptr;      // device arena
  tft_arena arena;
  cudaStream_t stream = nullptr;
  AuxStreams aux{};
  cudaEvent_t t0 = nullptr;
  Slot slot[kSlots];
};

namespace {

void server_release(tft_server* s) {
  for (Slot& sl : s->slot) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.htab) host_free_pinned(sl.htab);
    if (sl.dtab) dev_free(sl.dtab);
  }
  if (s->t0) cudaEventDestroy(s->t0);
  if (s->aux.fork) cudaEventDestroy(s->aux.fork);
  if (s->aux.join) cudaEventDestroy(s->aux.join);
  if (s->aux.side) cudaStreamDestroy(s->aux.side);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->base) dev_free(s->base);
  delete s;
}

size_t table_bytes(uint32_t max_batch) {
  return up256(2ull * max_batch * sizeof(GenDesc)) +
         up256((uint64_t)max_batch * sizeof(BatchLarge)) +
         up256((uint64_t)max_batch * sizeof(BatchSmall));
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0)
      .count();
}

}  // namespace

tft_status tft_server_create(tft_ctx* ctx, uint64_t budget_bytes,
                             uint32_t max_batch,
                             const tft_batch_params* params,
                             tft_server** out) {
  if (!ctx || !out || max_batch == 0 || budget_bytes < kBlockAlign)
    return TFT_EINVAL;
  const BatchSchedule S = batch_schedule(ctx->pr, params);
  if (!batch_schedule_valid(ctx->pr, S)) return TFT_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return TFT_ECUDA;
  tft_server* s = new (std::nothrow) tft_server();
  if (!s) return TFT_ENOMEM;
  s->ctx = ctx;
  s->S = S;
  s->max_batch = max_batch;
  int optin = 0;
  if (note(cudaDeviceGetAttribute(&optin,
                                  cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  ctx->device)) != cudaSuccess) {
    server_release(s);
    return TFT_ECUDA;
  }
  s->optin = (size_t)optin;
  s->arena.init(budget_bytes, kBlockAlign);
  if (dev_malloc((void**)&s->base, s->arena.size) != cudaSuccess) {
    s->base = nullptr;
    server_release(s);
    return TFT_ENOMEM;
  }
  const size_t tb = table_bytes(max_batch);
  bool ok = note(cudaStreamCreateWithFlags(&s->stream,
                                           cudaStreamNonBlocking)) ==
                cudaSuccess &&
            note(cudaStreamCreateWithFlags(&s->aux.side,
                                           cudaStreamNonBlocking)) ==
                cudaSuccess &&
            note(cudaEventCreateWithFlags(&s->aux.fork,
                                          cudaEventDisableTiming)) ==
                cudaSuccess &&
            note(cudaEventCreateWithFlags(&s->aux.join,
                                          cudaEventDisableTiming)) ==
                cudaSuccess &&
            note(cudaEventCreate(&s->t0)) == cudaSuccess;
  for (Slot& sl : s->slot) {
    if (!ok) break;
    sl.tab_bytes = tb;
    ok = dev_malloc((void**)&sl.dtab, tb) == cudaSuccess &&
         host_malloc_pinned((void**)&sl.htab, tb) == cudaSuccess &&
         note(cudaEventCreate(&sl.done)) == cudaSuccess;
  }
  if (!ok) {
    server_release(s);
    return TFT_ENOMEM;
  }
  *out = s;
  return TFT_OK;
}

tft_status tft_server_destroy(tft_server* s) {
  if (!s) return TFT_EINVAL;
  DeviceGuard g(s->ctx->device);
  cudaStreamSynchronize(s->stream);
  server_release(s);
  return TFT_OK;
}

namespace {

// Launch one batch of admitted requests on slot sl: operand generation,
// the batched product, optional copies of kept results, completion event.
tft_status launch_slot(tft_server* s, Slot& sl, const tft_request* reqs,
                       uint64_t seed, void* const* keep,
                       tft_server_stats* st) {
  tft_ctx* ctx = s->ctx;
  const PrimeInfo& pr = ctx->pr;
  const uint32_t n = (uint32_t)sl.reqs.size();
  unsigned char* base = (unsigned char*)s->base;
  // descriptors
  std::vector<tft_polymul_desc> descs(n);
  std::vector<void*> work(n);
  unsigned char* h = (unsigned char*)sl.htab;
  GenDesc* gd = (GenDesc*)h;
  uint64_t chunks = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const tft_request& q = reqs[sl.reqs[i]];
    const ReqLayout L = request_layout(pr, s->S, q.na, q.nb);
    unsigned char* blk = base + sl.blocks[i];
    descs[i] = {blk + L.a, q.na, blk + L.b, q.nb, blk + L.out};
    work[i] = blk + L.work;
    for (uint32_t o = 0; o < 2; ++o) {
      GenDesc& d = gd[2 * i + o];
      d.dst = (uint64_t)(o ? blk + L.b : blk + L.a);
      d.n = o ? q.nb : q.na;
      d.request = q.id;
      d.operand = o;
      d.pad = 0;
      d.chunk_base = chunks;
      chunks += gen_chunks(d.n);
    }
  }
  std::vector<BatchSmall> hs;
  std::vector<BatchLarge> hl;
  BatchLaunch B;
  tft_status stt = batch_describe(pr, s->S, descs.data(), n, work.data(),
                                  nullptr, 0, s->optin, &hs, &hl, &B);
  if (stt != TFT_OK) return stt;
  const size_t off_l = up256(2ull * s->max_batch * sizeof(GenDesc));
  const size_t off_s = off_l + up256((uint64_t)s->max_batch *
                                     sizeof(BatchLarge));
  if (!hl.empty()) memcpy(h + off_l, hl.data(), hl.size() * sizeof(BatchLarge));
  if (!hs.empty()) memcpy(h + off_s, hs.data(), hs.size() * sizeof(BatchSmall));
  const size_t bytes = off_s + hs.size() * sizeof(BatchSmall);
  unsigned char* d = (unsigned char*)sl.dtab;
  B.large = d + off_l;
  B.small = d + off_s;
  cudaError_t e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice,
                                  s->stream);
  if (e != cudaSuccess) return from_cuda(ctx, e);
  ctx->hook.before(ctx->hook.user, K_GEN, s->stream);
  e = launch_gen_table(ctx->prime, (const GenDesc*)d, 2 * n, chunks, seed,
                       ctx->nsm, s->stream);
  ctx->hook.after(ctx->hook.user, K_GEN, s->stream);
  if (e != cudaSuccess) return from_cuda(ctx, e);
  e = launch_batch(ctx->prime, B, ctx->rt, ctx->nsm, s->stream, &ctx->hook,
                   &s->aux);
  if (e != cudaSuccess) return from_cuda(ctx, e);
  if (keep) {
    for (uint32_t i = 0; i < n; ++i) {
      void* dst = keep[sl.reqs[i]];
      if (!dst) continue;
      const tft_request& q = reqs[sl.reqs[i]];
      e = cudaMemcpyAsync(dst, descs[i].out, (q.na + q.nb - 1) * pr.w,
                          cudaMemcpyDeviceToDevice, s->stream);
      if (e != cudaSuccess) return from_cuda(ctx, e);
    }
  }
  e = cudaEventRecord(sl.done, s->stream);
  if (e != cudaSuccess) return from_cuda(ctx, e);
  sl.busy = true;
  if (st) {
    st->batches++;
    if (n > st->max_batch) st->max_batch = n;
  }
  return TFT_OK;
}

// Retire slot sl if its batch has completed (or wait for it when `wait`).
// Returns 1 if retired, 0 if still running, -1 on a CUDA error.
int retire_slot(tft_server* s, Slot& sl, double* done_s, bool wait,
                tft_server_stats* st) {
  if (!sl.busy) return 0;
  cudaError_t e = wait ? cudaEventSynchronize(sl.done)
                       : cudaEventQuery(sl.done);
  if (e == cudaErrorNotReady) return 0;
  if (e != cudaSuccess) {
    note(e);
    return -1;
  }
  float ms = 0.f;
  if (note(cudaEventElapsedTime(&ms, s->t0, sl.done)) != cudaSuccess)
    return -1;
  for (uint64_t i : sl.reqs) {
    if (done_s) done_s[i] = ms / 1e3;
  }
  for (uint64_t b : sl.blocks) s->arena.release(b);
  if (st) st->completed += sl.reqs.size();
  sl.reqs.clear();
  sl.blocks.clear();
  sl.busy = false;
  return 1;
}

tft_status replay_batched(tft_server* s, const tft_request* reqs,
                          uint64_t count, uint64_t seed, double* done_s,
                          void* const* keep, tft_server_stats* st,
                          std::chrono::steady_clock::time_point h0) {
  const PrimeInfo& pr = s->ctx->pr;
  std::deque<uint64_t> pending;
  uint64_t next = 0;      // next request to arrive
  uint64_t completed = 0;
  int turn = 0;           // slot to fill next (batches complete in order)
  while (completed < count) {
    const double t = now_s(h0);
    while (next < count && reqs[next].arrival_s <= t) pending.push_back(next++);
    // retire finished batches in launch order
    for (int k = 0; k < kSlots; ++k) {
      Slot& sl = s->slot[(turn + k) % kSlots];
      const uint64_t nreq = sl.reqs.size();
      const int r = retire_slot(s, sl, done_s, false, st);
      if (r < 0) return TFT_ECUDA;
      if (r > 0) completed += nreq;
    }
    Slot& sl = s->slot[turn];
    if (!sl.busy && !pending.empty()) {
      // admit in arrival order while the requests fit in the budget
      while (!pending.empty() && sl.reqs.size() < s->max_batch) {
        const tft_request& q = reqs[pending.front()];
        uint64_t off;
        if (!s->arena.alloc(request_layout(pr, s->S, q.na, q.nb).total, &off))
          break;
        sl.reqs.push_back(pending.front());
        sl.blocks.push_back(off);
        pending.pop_front();
      }
      if (!sl.reqs.empty()) {
        const tft_status r = launch_slot(s, sl, reqs, seed, keep, st);
        if (r != TFT_OK) return r;
        turn = (turn + 1) % kSlots;
      } else if (!s->slot[(turn + 1) % kSlots].busy) {
        return TFT_ERANGE;  // nothing in flight and the head cannot fit
      }
    }
  }
  return TFT_OK;
}

tft_status replay_one_by_one(tft_server* s, const tft_request* reqs,
                             uint64_t count, uint64_t seed, double* done_s,
                             void* const* keep, tft_server_stats* st,
                             std::chrono::steady_clock::time_point h0) {
  tft_ctx* ctx = s->ctx;
  const PrimeInfo& pr = ctx->pr;
  uint64_t mna = 1, mnb = 1, mr = 1;
  for (uint64_t i = 0; i < count; ++i) {
    if (reqs[i].na > mna) mna = reqs[i].na;
    if (reqs[i].nb > mnb) mnb = reqs[i].nb;
    if (reqs[i].na + reqs[i].nb - 1 > mr) mr = reqs[i].na + reqs[i].nb - 1;
  }
  if (mr > ctx->max_len) return TFT_ERANGE;
  // operand and result buffers from the arena, reused in stream order
  uint64_t oa = 0, ob = 0, oo = 0;
  const bool ga = s->arena.alloc(mna * pr.w, &oa);
  const bool gb = ga && s->arena.alloc(mnb * pr.w, &ob);
  const bool go = gb && s->arena.alloc(mr * pr.w, &oo);
  if (!go) {
    if (gb) s->arena.release(ob);
    if (ga) s->arena.release(oa);
    return TFT_ERANGE;
  }
  unsigned char* base = (unsigned char*)s->base;
  void* A = base + oa;
  void* Bv = base + ob;
  void* O = base + oo;
  // a ring of completion events
  const uint64_t ring = 1024;
  std::vector<cudaEvent_t> ev(ring, nullptr);
  tft_status res = TFT_OK;
  for (auto& x : ev) {
    if (note(cudaEventCreate(&x)) != cudaSuccess) {
      res = TFT_ECUDA;
      break;
    }
  }
  uint64_t issued = 0, retired = 0;
  auto retire = [&](bool wait) -> bool {
    while (retired < issued) {
      cudaEvent_t e = ev[retired % ring];
      cudaError_t q = wait ? cudaEventSynchronize(e) : cudaEventQuery(e);
      if (q == cudaErrorNotReady) return true;
      if (q != cudaSuccess) {
        note(q);
        return false;
      }
      float ms = 0.f;
      if (note(cudaEventElapsedTime(&ms, s->t0, e)) != cudaSuccess)
        return false;
      if (done_s) done_s[retired] = ms / 1e3;
      retired++;
      if (st) st->completed++;
      if (wait) wait = false;  // one forced retirement frees a ring entry
    }
    return true;
  };
  while (res == TFT_OK && retired < count) {
    if (issued < count && reqs[issued].arrival_s <= now_s(h0)) {
      if (issued - retired == ring && !retire(true)) {
        res = TFT_ECUDA;
        break;
      }
      const tft_request& q = reqs[issued];
      ctx->hook.before(ctx->hook.user, K_GEN, s->stream);
      cudaError_t e = launch_gen_pair(ctx->prime, A, q.na, Bv, q.nb, q.id,
                                      seed, ctx->nsm, s->stream);
      ctx->hook.after(ctx->hook.user, K_GEN, s->stream);
      if (e != cudaSuccess) {
        res = from_cuda(ctx, e);
        break;
      }
      res = tft_polymul(ctx, A, q.na, Bv, q.nb, O, s->stream);
      if (res != TFT_OK) break;
      if (keep && keep[issued]) {
        e = cudaMemcpyAsync(keep[issued], O, (q.na + q.nb - 1) * pr.w,
                            cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) {
          res = from_cuda(ctx, e);
          break;
        }
      }
      if (cudaEventRecord(ev[issued % ring], s->stream) != cudaSuccess) {
        res = TFT_ECUDA;
        break;
      }
      issued++;
      if (st) st->batches++;
    }
    if (!retire(false)) res = TFT_ECUDA;
  }
  cudaStreamSynchronize(s->stream);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  s->arena.release(oo);
  s->arena.release(ob);
  s->arena.release(oa);
  return res;
}

}  // namespace

tft_status tft_server_replay(tft_server* s, const tft_request* reqs,
                             uint64_t count, uint64_t seed, int mode,
                             double* done_s, void* const* keep,
                             tft_server_stats* stats) {
  if (!s || (!reqs && count) || (mode != TFT_SERVE_BATCHED &&
                                 mode != TFT_SERVE_ONE_BY_ONE))
    return TFT_EINVAL;
  const PrimeInfo& pr = s->ctx->pr;
  for (uint64_t i = 0; i < count; ++i) {
    const tft_request& q = reqs[i];
    if (q.na == 0 || q.nb == 0 || q.na > (1ull << 32) || q.nb > (1ull << 32))
      return TFT_EINVAL;
    if (i && q.arrival_s < reqs[i - 1].arrival_s) return TFT_EINVAL;
    if (keep && keep[i] && !aligned16(keep[i])) return TFT_EINVAL;
    if (mode == TFT_SERVE_BATCHED &&
        s->arena.round(request_layout(pr, s->S, q.na, q.nb).total) >
            s->arena.size)
      return TFT_ERANGE;
  }
  tft_server_stats local;
  memset(&local, 0, sizeof(local));
  DeviceGuard g(s->ctx->device);
  if (!g.ok) return TFT_ECUDA;
  const uint64_t launches0 = s->ctx->launches;
  s->arena.peak = s->arena.used;
  // time origin: the device event t0, taken with the host clock once it
  // has completed
  if (note(cudaStreamSynchronize(s->stream)) != cudaSuccess ||
      note(cudaEventRecord(s->t0, s->stream)) != cudaSuccess ||
      note(cudaEventSynchronize(s->t0)) != cudaSuccess)
    return TFT_ECUDA;
  const auto h0 = std::chrono::steady_clock::now();
  tft_status r = mode == TFT_SERVE_BATCHED
                     ? replay_batched(s, reqs, count, seed, done_s, keep,
                                      &local, h0)
                     : replay_one_by_one(s, reqs, count, seed, done_s, keep,
                                         &local, h0);
  if (r != TFT_OK) {
    // drain whatever is in flight before returning the error
    cudaStreamSynchronize(s->stream);
    for (Slot& sl : s->slot) {
      for (uint64_t b : sl.blocks) s->arena.release(b);
      sl.reqs.clear();
      sl.blocks.clear();
      sl.busy = false;
    }
    return r;
  }
  local.wall_s = now_s(h0);
  local.peak_bytes = s->arena.peak;
  local.launches = s->ctx->launches - launches0;
  if (stats) *stats = local;
  return TFT_OK;
}
