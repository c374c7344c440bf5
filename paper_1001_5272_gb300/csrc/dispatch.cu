// Prime dispatch: forwards each launcher to the field's translation unit.
#include "tft_internal.h"

namespace tftgb {

#define TFT_FIELD_DECLS(NAME)                                                 \
  cudaError_t NAME##_prepare(size_t optin);                                   \
  cudaError_t NAME##_forward(void* x, uint64_t n, const Plan& P, void* E,     \
                             const void* rt, int nsm, cudaStream_t s,         \
                             const LaunchHook* hook, const AuxStreams* aux);  \
  cudaError_t NAME##_inverse(void* x, uint64_t n, const Plan& P, void* E,     \
                             uint64_t omega_a_tw, const void* rt, int nsm,    \
                             cudaStream_t s, const LaunchHook* hook);         \
  cudaError_t NAME##_polymul(const void* a, uint64_t na, const void* b,       \
                             uint64_t nb, void* out, const Plan& P,           \
                             void* work, void* EA, void* EB,                  \
                             uint64_t omega_a_tw, const void* rt, int nsm,    \
                             cudaStream_t s, const LaunchHook* hook,          \
                             const AuxStreams* aux);                          \
  PlanSmem NAME##_plan_smem(const Plan& P);                                   \
  cudaError_t NAME##_forward_zs(void* x, uint64_t n, const Plan& P,           \
                                uint64_t omega_a_tw, const void* rt, int nsm, \
                                cudaStream_t s, const LaunchHook* hook);      \
  cudaError_t NAME##_inverse_zs(void* x, uint64_t n, const Plan& P,           \
                                uint64_t omega_a_tw, const void* rt, int nsm, \
                                cudaStream_t s, const LaunchHook* hook);      \
  cudaError_t NAME##_small_batch(const void* d, uint32_t count, int lmax,     \
                                 int inverse, const void* rt, int nsm,        \
                                 cudaStream_t s, const LaunchHook* hook);     \
  cudaError_t NAME##_shard_cols(int dir, int which, void* blk, const Plan& Pc, \
                                void* E, int want_E, uint64_t omega_a_tw,     \
                                const void* rt, int nsm, cudaStream_t s,      \
                                const LaunchHook* hook);                      \
  cudaError_t NAME##_shard_rows(int dir, void* rows, uint64_t count,          \
                                uint64_t rho_off, int lr, const void* rt,     \
                                int nsm, cudaStream_t s,                      \
                                const LaunchHook* hook);                      \
  cudaError_t NAME##_shard_last(int dir, void* row, const void* E, uint64_t a, \
                                uint64_t b, int lr, const void* rt,           \
                                cudaStream_t s, const LaunchHook* hook);      \
  cudaError_t NAME##_batch(const BatchLaunch& B, const void* rt, int nsm,   \
                           cudaStream_t s, const LaunchHook* hook,          \
                           const AuxStreams* aux);                          \
  cudaError_t NAME##_prepare_batch(size_t optin);                            \
  cudaError_t NAME##_fold(void* d0, const void* s0, uint64_t n0, void* d1,    \
                          const void* s1, uint64_t n1, uint64_t L, int ell,   \
                          const void* powers, int nsm, cudaStream_t s);       \
  cudaError_t NAME##_chunk_mul(void* X, const void* Y, uint64_t L, int nsm,   \
                               cudaStream_t s);                               \
  cudaError_t NAME##_tail(void* X, const void* S, uint64_t Q, uint64_t lo,    \
                          uint64_t hi, int mul, int nsm, cudaStream_t s);

TFT_FIELD_DECLS(p998)
TFT_FIELD_DECLS(p2013)
TFT_FIELD_DECLS(gold)

#define TFT_BY_PRIME(prime, CALL0, CALL1, CALL2) \
  switch (prime) {                               \
    case 0: return CALL0;                        \
    case 1: return CALL1;                        \
    case 2: return CALL2;                        \
    default: return cudaErrorInvalidValue;       \
  }

cudaError_t prepare_kernels(int prime, size_t optin) {
  cudaError_t e;
  switch (prime) {
    case 0: e = p998_prepare(optin); break;
    case 1: e = p2013_prepare(optin); break;
    case 2: e = gold_prepare(optin); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  TFT_BY_PRIME(prime, p998_prepare_batch(optin), p2013_prepare_batch(optin),
               gold_prepare_batch(optin));
}

cudaError_t launch_forward(int prime, void* x, uint64_t n, const Plan& P,
                           void* E, const void* rt, int nsm, cudaStream_t s,
                           const LaunchHook* hook, const AuxStreams* aux) {
  TFT_BY_PRIME(prime, p998_forward(x, n, P, E, rt, nsm, s, hook, aux),
               p2013_forward(x, n, P, E, rt, nsm, s, hook, aux),
               gold_forward(x, n, P, E, rt, nsm, s, hook, aux));
}

cudaError_t launch_inverse(int prime, void* x, uint64_t n, const Plan& P,
                           void* E, uint64_t omega_a_tw, const void* rt,
                           int nsm, cudaStream_t s, const LaunchHook* hook) {
  TFT_BY_PRIME(prime, p998_inverse(x, n, P, E, omega_a_tw, rt, nsm, s, hook),
               p2013_inverse(x, n, P, E, omega_a_tw, rt, nsm, s, hook),
               gold_inverse(x, n, P, E, omega_a_tw, rt, nsm, s, hook));
}

cudaError_t launch_forward_zs(int prime, void* x, uint64_t n, const Plan& P,
                              uint64_t omega_a_tw, const void* rt, int nsm,
                              cudaStream_t s, const LaunchHook* hook) {
  TFT_BY_PRIME(prime, p998_forward_zs(x, n, P, omega_a_tw, rt, nsm, s, hook),
               p2013_forward_zs(x, n, P, omega_a_tw, rt, nsm, s, hook),
               gold_forward_zs(x, n, P, omega_a_tw, rt, nsm, s, hook));
}

cudaError_t launch_inverse_zs(int prime, void* x, uint64_t n, const Plan& P,
                              uint64_t omega_a_tw, const void* rt, int nsm,
                              cudaStream_t s, const LaunchHook* hook) {
  TFT_BY_PRIME(prime, p998_inverse_zs(x, n, P, omega_a_tw, rt, nsm, s, hook),
               p2013_inverse_zs(x, n, P, omega_a_tw, rt, nsm, s, hook),
               gold_inverse_zs(x, n, P, omega_a_tw, rt, nsm, s, hook));
}

cudaError_t launch_polymul(int prime, const void* a, uint64_t na,
                           const void* b, uint64_t nb, void* out,
                           const Plan& P, void* work, void* EA, void* EB,
                           uint64_t omega_a_tw, const void* rt, int nsm,
                           cudaStream_t s, const LaunchHook* hook,
                           const AuxStreams* aux) {
  TFT_BY_PRIME(prime,
               p998_polymul(a, na, b, nb, out, P, work, EA, EB, omega_a_tw,
                            rt, nsm, s, hook, aux),
               p2013_polymul(a, na, b, nb, out, P, work, EA, EB, omega_a_tw,
                             rt, nsm, s, hook, aux),
               gold_polymul(a, na, b, nb, out, P, work, EA, EB, omega_a_tw,
                            rt, nsm, s, hook, aux));
}

cudaError_t launch_batch(int prime, const BatchLaunch& B, const void* rt,
                         int nsm, cudaStream_t s, const LaunchHook* hook,
                         const AuxStreams* aux) {
  TFT_BY_PRIME(prime, p998_batch(B, rt, nsm, s, hook, aux),
               p2013_batch(B, rt, nsm, s, hook, aux),
               gold_batch(B, rt, nsm, s, hook, aux));
}

PlanSmem plan_smem(int prime, const Plan& P) {
  switch (prime) {
    case 0: return p998_plan_smem(P);
    case 1: return p2013_plan_smem(P);
    default: return gold_plan_smem(P);
  }
}

cudaError_t launch_fold(int prime, void* d0, const void* s0, uint64_t n0,
                        void* d1, const void* s1, uint64_t n1, uint64_t L,
                        int ell, const void* powers, int nsm,
                        cudaStream_t s) {
  TFT_BY_PRIME(prime,
               p998_fold(d0, s0, n0, d1, s1, n1, L, ell, powers, nsm, s),
               p2013_fold(d0, s0, n0, d1, s1, n1, L, ell, powers, nsm, s),
               gold_fold(d0, s0, n0, d1, s1, n1, L, ell, powers, nsm, s));
}

cudaError_t launch_chunk_mul(int prime, void* X, const void* Y, uint64_t L,
                             int nsm, cudaStream_t s) {
  TFT_BY_PRIME(prime, p998_chunk_mul(X, Y, L, nsm, s),
               p2013_chunk_mul(X, Y, L, nsm, s),
               gold_chunk_mul(X, Y, L, nsm, s));
}

cudaError_t launch_tail(int prime, void* X, const void* S, uint64_t Q,
                        uint64_t lo, uint64_t hi, int mul, int nsm,
                        cudaStream_t s) {
  TFT_BY_PRIME(prime, p998_tail(X, S, Q, lo, hi, mul, nsm, s),
               p2013_tail(X, S, Q, lo, hi, mul, nsm, s),
               gold_tail(X, S, Q, lo, hi, mul, nsm, s));
}

cudaError_t launch_small_batch(int prime, const void* d, uint32_t count,
                               int lmax, int inverse, const void* rt, int nsm,
                               cudaStream_t s, const LaunchHook* hook) {
  TFT_BY_PRIME(prime,
               p998_small_batch(d, count, lmax, inverse, rt, nsm, s, hook),
               p2013_small_batch(d, count, lmax, inverse, rt, nsm, s, hook),
               gold_small_batch(d, count, lmax, inverse, rt, nsm, s, hook));
}

cudaError_t launch_shard_cols(int prime, int dir, int which, void* blk,
                              const Plan& Pc, void* E, int want_E,
                              uint64_t omega_a_tw, const void* rt, int nsm,
                              cudaStream_t s, const LaunchHook* hook) {
  TFT_BY_PRIME(prime,
               p998_shard_cols(dir, which, blk, Pc, E, want_E, omega_a_tw, rt,
                               nsm, s, hook),
               p2013_shard_cols(dir, which, blk, Pc, E, want_E, omega_a_tw,
                                rt, nsm, s, hook),
               gold_shard_cols(dir, which, blk, Pc, E, want_E, omega_a_tw, rt,
                               nsm, s, hook));
}

cudaError_t launch_shard_rows(int prime, int dir, void* rows, uint64_t count,
                              uint64_t rho_off, int lr, const void* rt,
                              int nsm, cudaStream_t s,
                              const LaunchHook* hook) {
  TFT_BY_PRIME(prime,
               p998_shard_rows(dir, rows, count, rho_off, lr, rt, nsm, s,
                               hook),
               p2013_shard_rows(dir, rows, count, rho_off, lr, rt, nsm, s,
                                hook),
               gold_shard_rows(dir, rows, count, rho_off, lr, rt, nsm, s,
                               hook));
}

cudaError_t launch_shard_last(int prime, int dir, void* row, const void* E,
                              uint64_t a, uint64_t b, int lr, const void* rt,
                              cudaStream_t s, const LaunchHook* hook) {
  TFT_BY_PRIME(prime, p998_shard_last(dir, row, E, a, b, lr, rt, s, hook),
               p2013_shard_last(dir, row, E, a, b, lr, rt, s, hook),
               gold_shard_last(dir, row, E, a, b, lr, rt, s, hook));
}

}  // namespace tftgb
