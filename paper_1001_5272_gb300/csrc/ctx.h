// The context object behind the C ABI's tft_ctx handle, and the helpers
// that the C-ABI translation units share.  Host code only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/tft.h"
#include "batch.cuh"
#include "host_common.h"
#include "tft_internal.h"

namespace tftgb {

// A context's fixed device scratch, in elements: the E rows of transforms
// and products (2^14 words each at most) and, for the space-restricted
// product, one tail block of 2^18 points plus one row.
constexpr size_t kCtxScratchWords = ((size_t)1 << 18) + ((size_t)1 << 14);

constexpr int kProfSlots = 64;

struct ProfSlot {
  cudaEvent_t start;
  cudaEvent_t stop;
  int kind;
};

}  // namespace tftgb

struct tft_ctx {
  using PrimeInfo = tftgb::PrimeInfo;
  using ProfSlot = tftgb::ProfSlot;
  using LaunchHook = tftgb::LaunchHook;
  using AuxStreams = tftgb::AuxStreams;
  using BatchLaunch = tftgb::BatchLaunch;
  int prime;
  int device;
  int nsm;
  uint64_t max_len;
  uint32_t flags;
  PrimeInfo pr;
  alignas(16) unsigned char rt[sizeof(tftgb::RootTable<uint64_t>)];
  void* scratch;     // kCtxScratchWords: E / EA, EB; restricted tail
  void* work;        // max_len words (products)
  void* stage;       // 3 * max_len words (host-buffer entry points)
  tft_status sticky;
  // launch accounting and optional per-kernel timing
  uint64_t launches;
  int prof_on;
  int prof_pending;
  ProfSlot prof[tftgb::kProfSlots];
  double prof_ms[tftgb::K_NUM_KINDS];
  uint64_t prof_count[tftgb::K_NUM_KINDS];
  LaunchHook hook;
  AuxStreams aux;    // side stream + fork/join events
  // batched products (tft_ctx_reserve_batch / tft_batch_plan)
  void* batch_tab;         // device descriptor tables
  uint64_t batch_tab_bytes;
  void* batch_work;        // work area of the large products
  uint64_t batch_work_words;
  uint32_t batch_max;      // products per plan
  BatchLaunch batch;       // the current plan
  int batch_ready;
};

namespace tftgb {

// Record a CUDA error for tft_last_cuda_error; returns e.
cudaError_t note(cudaError_t e);
// Every device and pinned-host allocation of the library goes through these
// (tft_debug_fail_allocation injects a failure here; the live count shows
// leaks).  A failed allocation leaves *p null and clears the runtime's
// last-error state, so a later launch check does not report it again.
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t host_malloc_pinned(void** p, size_t bytes);
void host_free_pinned(void* p);
// TFT_OK on success; otherwise records e, marks the context and returns
// TFT_ECUDA.
tft_status from_cuda(tft_ctx* ctx, cudaError_t e);
// The single-call plan for length n (false: n beyond the supported range).
bool make_plan(int prime, uint64_t n, Plan* out);

// Batch schedule with the library defaults filled in.
struct BatchSchedule {
  int small_log, lr, clog;
  int clog_lo;  // tile width of the shorter-column class; -1: clog
};
BatchSchedule batch_schedule(const PrimeInfo& pr,
                             const tft_batch_params* params);
bool batch_schedule_valid(const PrimeInfo& pr, const BatchSchedule& S);
// Elements of work area a product of the row/column class needs (B', EA,
// EB in 16-byte slots); 0 for the single-CTA class.
uint64_t batch_product_work_words(const PrimeInfo& pr, const BatchSchedule& S,
                                  uint64_t na, uint64_t nb);
// Classify and describe a batch.  The work area of large product i starts at
// work_of[i] when work_of is given, else products take consecutive slots of
// [work_base, work_base + work_cap words).  Fills the host tables (small
// products sorted largest first) and the launch description, whose table
// pointers are left for the caller to set.  optin: the device's opt-in
// shared memory per block.
tft_status batch_describe(const PrimeInfo& pr, const BatchSchedule& S,
                          const tft_polymul_desc* descs, uint32_t count,
                          void* const* work_of, void* work_base,
                          uint64_t work_cap, size_t optin,
                          std::vector<BatchSmall>* hs,
                          std::vector<BatchLarge>* hl, BatchLaunch* B);

}  // namespace tftgb
