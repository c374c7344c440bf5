// Internal interface between the C-ABI layer (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tftgb {

// Kernel kinds, for launch counting and per-kernel timing (the numbering is
// part of the C ABI: tft_kernel_name / tft_profile_read).
enum KernelKind {
  K_SMALL = 0,
  K_SMALL_MUL = 1,
  K_COL_FWD = 2,
  K_ROW_FWD = 3,
  K_ROW_INV = 4,
  K_COL_INV = 5,
  K_LASTROW_INV = 6,
  K_ROW_MUL = 7,
  K_LASTROW_FWD = 8,   // ragged last row of a forward transform
  K_LASTROW_MUL = 9,   // reserved: products run their last row in the row pass
  K_GEN = 10,          // served-request operand generator
  K_FOLD = 11,         // space-restricted product: folding, chunk products
  K_NUM_KINDS = 12
};

// Called around every kernel launch (may be null).
struct LaunchHook {
  void (*before)(void* user, int kind, cudaStream_t s);
  void (*after)(void* user, int kind, cudaStream_t s);
  void* user;
};

// Execution plan for one transform length.
//   small = 1: the whole transform in one CTA, padded in shared memory to 2^l.
//   small = 0: n = a 2^lr + b; columns padded to 2^c in shared memory, C =
//              2^clog columns per CTA; row kernels persistent with
//              row_ctas_per_sm CTAs per SM.
struct Plan {
  int small;
  int l;
  int lr;
  int c;
  int clog;
  uint64_t a;
  uint64_t b;
  int row_ctas_per_sm;
};

struct PlanSmem {
  size_t col;
  size_t row;
};

cudaError_t prepare_kernels(int prime, size_t optin_smem);
PlanSmem plan_smem(int prime, const Plan& P);

// A second stream and two events owned by a context: independent pieces of a
// call (the ragged last row next to the full rows) run concurrently, forked
// from and joined back into the caller's stream.  Null: run serially.
struct AuxStreams {
  cudaStream_t side;
  cudaEvent_t fork;
  cudaEvent_t join;
};

// One transform of a batch of single-CTA transforms (device table entry).
struct XformDesc {
  uint64_t x;  // device pointer
  uint32_t n;  // length
  uint32_t l;  // padded length 2^l >= n
};

// A planned batch of products (tables already on the device).
struct BatchLaunch {
  const void* small;   // BatchSmall[ns] on the device
  uint32_t ns;
  int lmax;            // largest small-class log length
  const void* large;   // BatchLarge[nl] on the device
  uint32_t nl;
  int lr;              // row length of the large class
  int clog;            // columns per tile
  int clog_lo;         // columns per tile of the shorter-column class
  int cmax;            // largest column log length
  uint32_t nl_lo;      // large products (first, sorted by c) with c < cmax
  int cmax_lo;         // their largest column log length
  uint64_t total_rows; // sum of a_p + [b_p > 0]
  uint64_t ci_tiles;   // inverse column tiles
};

cudaError_t launch_batch(int prime, const BatchLaunch& B, const void* rt,
                         int nsm, cudaStream_t s, const LaunchHook* hook,
                         const AuxStreams* aux);

// Operand generator of served requests (gen.cu): one descriptor per
// (request, operand); chunk_base is the prefix of gen_chunks(n).
struct GenDesc {
  uint64_t dst;         // device pointer
  uint64_t n;           // elements
  uint64_t request;
  uint64_t chunk_base;
  uint32_t operand;     // 0 = a, 1 = b
  uint32_t pad;
};
uint64_t gen_chunks(uint64_t n);
cudaError_t launch_gen_table(int prime, const GenDesc* d, uint32_t nd,
                             uint64_t chunks, uint64_t seed, int nsm,
                             cudaStream_t s);
cudaError_t launch_gen_pair(int prime, void* a, uint64_t na, void* b,
                            uint64_t nb, uint64_t request, uint64_t seed,
                            int nsm, cudaStream_t s);

// Space-restricted product (Algorithm 3): folding of both operands of a
// chunk (d1 = null: one operand), a chunk's pointwise product, and the tail
// block's copy / product.  `powers` points at 33 words omega_q^{2^b} in
// twiddle form (host memory, passed by value to the kernel).
cudaError_t launch_fold(int prime, void* d0, const void* s0, uint64_t n0,
                        void* d1, const void* s1, uint64_t n1, uint64_t L,
                        int ell, const void* powers, int nsm, cudaStream_t s);
cudaError_t launch_chunk_mul(int prime, void* X, const void* Y, uint64_t L,
                             int nsm, cudaStream_t s);
cudaError_t launch_tail(int prime, void* X, const void* S, uint64_t Q,
                        uint64_t lo, uint64_t hi, int mul, int nsm,
                        cudaStream_t s);

cudaError_t launch_forward(int prime, void* x, uint64_t n, const Plan& P,
                           void* E, const void* rt, int nsm, cudaStream_t s,
                           const LaunchHook* hook, const AuxStreams* aux);
cudaError_t launch_inverse(int prime, void* x, uint64_t n, const Plan& P,
                           void* E, uint64_t omega_a_tw, const void* rt,
                           int nsm, cudaStream_t s, const LaunchHook* hook);
// Forward / inverse TFT that read and write nothing but x (the ragged last
// row from a thread-block cluster, lastrow_cluster.cuh).
cudaError_t launch_forward_zs(int prime, void* x, uint64_t n, const Plan& P,
                              uint64_t omega_a_tw, const void* rt, int nsm,
                              cudaStream_t s, const LaunchHook* hook);
cudaError_t launch_inverse_zs(int prime, void* x, uint64_t n, const Plan& P,
                              uint64_t omega_a_tw, const void* rt, int nsm,
                              cudaStream_t s, const LaunchHook* hook);
// Single-CTA transforms of a batch, one persistent launch (lmax: the
// largest l of the table).
cudaError_t launch_small_batch(int prime, const void* d, uint32_t count,
                               int lmax, int inverse, const void* rt, int nsm,
                               cudaStream_t s, const LaunchHook* hook);
// Pieces of a transform held in parts (kernels_impl.cuh, Launch::shard_*).
cudaError_t launch_shard_cols(int prime, int dir, int which, void* blk,
                              const Plan& Pc, void* E, int want_E,
                              uint64_t omega_a_tw, const void* rt, int nsm,
                              cudaStream_t s, const LaunchHook* hook);
cudaError_t launch_shard_rows(int prime, int dir, void* rows, uint64_t count,
                              uint64_t rho_off, int lr, const void* rt,
                              int nsm, cudaStream_t s, const LaunchHook* hook);
cudaError_t launch_shard_last(int prime, int dir, void* row, const void* E,
                              uint64_t a, uint64_t b, int lr, const void* rt,
                              cudaStream_t s, const LaunchHook* hook);
cudaError_t launch_polymul(int prime, const void* a, uint64_t na,
                           const void* b, uint64_t nb, void* out,
                           const Plan& P, void* work, void* EA, void* EB,
                           uint64_t omega_a_tw, const void* rt, int nsm,
                           cudaStream_t s, const LaunchHook* hook,
                           const AuxStreams* aux);

}  // namespace tftgb
