/*
 * tft.h -- C ABI of the GB300 in-place truncated Fourier transform library.
 *
 * What it computes (Harvey & Roche, "An in-place truncated Fourier transform
 * and applications to polynomial multiplication", 2010):
 *
 *   Ring (Section 2.1): Z/p for one of three primes p = c 2^K + 1; 2 is
 *   invertible and primitive 2^k-th roots exist for every k <= K.
 *
 *   Roots (Section 2.2): compatible primitive roots omega_[k],
 *   omega_[k+1]^2 = omega_[k].  The paper leaves the choice open; this
 *   library fixes omega_[K] = g^((p-1)/2^K) with the generator g below and
 *   omega_[k] = omega_[K]^(2^(K-k)).  Then omega_s = omega_[K]^(rev_K s).
 *
 *     prime                 storage  K   g    omega_[K]
 *     998244353             uint32   23  3    15311432
 *     2013265921            uint32   27  31   440564289
 *     2^64 - 2^32 + 1       uint64   32  7    1753635133440165772
 *
 *   TFT (Section 2.2, Algorithm 1): for x_0..x_{n-1} (coefficients of F,
 *   deg F < n) the transform overwrites x with F^_s = F(omega_s), s < n.
 *   The output is in this bit-reversed-root order, not natural DFT order.
 *   It equals the first n outputs of the length-2^k transform of x padded
 *   with zeros for any n <= 2^k (Section 1.2); with compatible roots it does
 *   not depend on k, which is therefore only validated.
 *
 *   ITFT (Section 4, Algorithm 2): the inverse map, in place.
 *
 *   Product (Sections 1.2 and 5): C = A B of length r = na + nb - 1 by a TFT
 *   of both zero-extended operands, the pointwise product C^_s = A^_s B^_s,
 *   and an ITFT.
 *
 * Elements are canonical residues in [0, p): uint32_t for the two 32-bit
 * primes, uint64_t for 2^64 - 2^32 + 1.  Inputs outside [0, p) are not
 * checked and give unspecified (but memory-safe) results.  All arithmetic is
 * exact; results are bit-for-bit those of the definitions above.
 *
 * Memory: transforms run in place on the caller's n-word device buffer; the
 * context owns a fixed scratch of 2^18 + 2^14 words (rows of at most 2^14
 * words for transforms and products, one 2^18-point block for the
 * space-restricted product) plus, for products, one r-word work buffer, all
 * reserved when the context is created.  No call allocates device memory;
 * tft_forward_noscratch and tft_inverse_noscratch use none beyond x.
 *
 * Errors: argument errors are returned synchronously and nothing is
 * launched.  Launch failures return TFT_ECUDA.  Kernels run asynchronously
 * on the given stream; faults that surface later are reported by
 * tft_last_error() after the stream has been synchronized.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Calls on one context must not overlap on the GPU: the
 * context's scratch is shared by every call (use one context per concurrent
 * stream).
 */
#ifndef TFT_GB300_H
#define TFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tft_prime {
  TFT_P998244353 = 0,  /* 119 * 2^23 + 1, uint32 elements */
  TFT_P2013265921 = 1, /*  15 * 2^27 + 1, uint32 elements */
  TFT_PGOLDILOCKS = 2  /* 2^64 - 2^32 + 1, uint64 elements */
} tft_prime;

typedef enum tft_status {
  TFT_OK = 0,
  TFT_EINVAL = 1,   /* bad argument: null or misaligned pointer, n = 0,
                       n > 2^k, k > K, aliasing output, unknown prime */
  TFT_ERANGE = 2,   /* size beyond this context's max_len or the supported
                       maximum (2^25 words for 2^64-2^32+1, 2^27 otherwise) */
  TFT_ENOMEM = 3,   /* device allocation failed (context creation only) */
  TFT_ECUDA = 4,    /* a CUDA runtime call or launch failed */
  TFT_ETIMEOUT = 5  /* a bounded device-side wait expired */
} tft_status;

typedef struct tft_ctx tft_ctx;

/* Context-creation flags. */
#define TFT_CTX_HOST_STAGING 1u /* also reserve device staging buffers for
                                   the *_host entry points (3 max_len words) */

/*
 * Create a context for `prime` on CUDA device `device`.  Transforms of length
 * n <= max_len and products with r = na + nb - 1 <= max_len are accepted.
 * Reserves the root table, the fixed scratch and (products) a max_len-word
 * work buffer on the device.  On success *out owns them until
 * tft_ctx_destroy.  Errors: TFT_EINVAL (bad prime/device/out, max_len = 0),
 * TFT_ERANGE (max_len beyond the supported maximum), TFT_ENOMEM, TFT_ECUDA.
 */
tft_status tft_ctx_create(tft_prime prime, int device, uint64_t max_len,
                          uint32_t flags, tft_ctx** out);

/* Free a context (waits for nothing: synchronize its streams first). */
tft_status tft_ctx_destroy(tft_ctx* ctx);

/*
 * tft(x, n, k): in-place forward TFT, Algorithm 1 (Section 3).
 *   x      device pointer, n elements, 16-byte aligned; overwritten with
 *          F^_s = F(omega_s), s < n.
 *   n      1 <= n <= 2^k and n <= max_len.
 *   k      log2 of the transform size the caller has in mind, n <= 2^k,
 *          k <= K(prime).  The result does not depend on k.
 */
tft_status tft_forward(tft_ctx* ctx, void* x, uint64_t n, uint32_t k,
                       void* stream);

/*
 * itft(X, n, k): in-place inverse TFT, Algorithm 2 (Section 4).  Same
 * arguments as tft_forward; X holds F^_0..F^_{n-1} and is overwritten with
 * F_0..F_{n-1}.
 */
tft_status tft_inverse(tft_ctx* ctx, void* X, uint64_t n, uint32_t k,
                       void* stream);

/*
 * polymul(a, b): out = a * b mod p (Section 5; TFT of both operands,
 * pointwise product, ITFT).  The transforms have length r rounded up to a
 * multiple of the plan's row length R (any length >= r determines the
 * product); the fewer than R positions past r live in the context's
 * scratch.
 *   a, b   device pointers, na and nb elements (read only; may alias each
 *          other), 16-byte aligned.
 *   out    device pointer, r = na + nb - 1 elements, 16-byte aligned, must
 *          not overlap a or b.
 * Uses the context's r-word work buffer.  Errors as above.
 */
tft_status tft_polymul(tft_ctx* ctx, const void* a, uint64_t na,
                       const void* b, uint64_t nb, void* out, void* stream);

/*
 * Padded power-of-two product, for comparison with the TFT product (the
 * zero-padded FFT the TFT improves on, Section 1.2): both operands
 * zero-extended to N = 2^ceil(lg r), transforms of length N, pointwise
 * product, inverse of length N, then the first r coefficients copied to
 * out.  scratch: 2N device words (16-byte aligned, not overlapping the
 * other buffers) holding the two padded transforms.  For N at most the
 * single-CTA size (2^13 words, 2^12 for 2^64 - 2^32 + 1) the single-CTA
 * kernel pads inside shared memory, as tft_polymul does.  Errors as
 * tft_polymul; TFT_ERANGE if N exceeds the supported length.
 */
tft_status tft_polymul_padded(tft_ctx* ctx, const void* a, uint64_t na,
                              const void* b, uint64_t nb, void* out,
                              void* scratch, void* stream);

/*
 * Space-restricted product (Algorithm 3, Section 5): the same result as
 * tft_polymul, computed in the output buffer alone.  Chunks [q, q + L) of
 * the output (L the largest power of two with q + 2L <= r) receive the
 * transforms of A and of B at the points omega_{q..q+L-1}, obtained by
 * folding A(omega_q x) and B(omega_q x) modulo x^L - 1 and a forward
 * transform of length L; the chunk's pointwise product overwrites the first
 * half; the last positions (fewer than 2^18) come from aligned blocks of
 * 2^18 points evaluated in the context's fixed scratch; then the in-place
 * inverse transform of length r.  Device memory beyond out: the context's
 * fixed scratch only (no r-word work area), so out may be as long as the
 * library supports (r <= 2^25 for 2^64 - 2^32 + 1, r <= min(2^K, 2^27)
 * for the 32-bit primes) whatever the context's max_len.  Arguments and
 * errors as tft_polymul.
 */
tft_status tft_polymul_restricted(tft_ctx* ctx, const void* a, uint64_t na,
                                  const void* b, uint64_t nb, void* out,
                                  void* stream);
/* The chunk sequence tft_polymul_restricted follows for an output of r
 * positions (host only): *count pairs (q[i], L[i]) in processing order --
 * Algorithm 3's loop, stopped before the first chunk with L <= 2^16 -- and
 * *tail_start, the first position produced by the tail blocks.  TFT_ERANGE
 * if more than `capacity` chunks (64 always suffice). */
tft_status tft_restricted_schedule(uint64_t r, uint64_t* q, uint64_t* L,
                                   uint32_t capacity, uint32_t* count,
                                   uint64_t* tail_start);

/*
 * Batched products: many independent polymul(a, b) calls (Section 5's
 * product, each exactly as tft_polymul computes it) in a few launches.
 *
 * Products with r = na + nb - 1 <= 2^small_log run one per CTA entirely in
 * shared memory; the others use the row/column split with one row length
 * 2^lr for all of them, in three phases that each cover every large
 * product (forward columns, fused rows, inverse columns; a column phase is
 * two launches when the shorter columns fit smaller tiles).  Each launch is
 * persistent over its task list.
 *
 * Usage: tft_ctx_reserve_batch once (reserves the descriptor tables for up
 * to max_products and a work area of work_words elements: each large
 * product needs r + 2 * 2^lr elements of it, see tft_batch_work_words);
 * tft_batch_plan for a set of products (validates, classifies, uploads the
 * tables; synchronous, not capturable); tft_batch_run to launch the planned
 * batch on a stream (launches only, so it can be captured into a CUDA
 * graph and replayed; the operands may change between runs, the pointers
 * and lengths may not).  tft_polymul_batch = plan + run.
 *
 * Each descriptor: a, b (device, read only, na, nb >= 1 elements), out
 * (device, r elements, not overlapping a or b); 16-byte aligned.  Errors:
 * TFT_EINVAL (bad descriptor or parameters, no reservation), TFT_ERANGE
 * (more products than reserved, work area too small, or a product too long
 * for the row length: its 2^c column rows, c = ceil(log2(ceil(r / 2^lr))),
 * must satisfy c <= 13 (32-bit primes) or 12 (2^64 - 2^32 + 1), and a tile
 * of 2^(c + clog) elements must fit in the device's shared memory -- with
 * 16 columns of 4-byte elements that is c <= 11, i.e. r <= 2^(lr + 11)).
 */
typedef struct tft_polymul_desc {
  const void* a;
  uint64_t na;
  const void* b;
  uint64_t nb;
  void* out;
} tft_polymul_desc;

/* Batch schedule; 0 in a field means the default (32-bit primes:
 * small_log 13, lr 9, 16 columns per tile; 2^64 - 2^32 + 1: 12, 10, 4).
 * Constraints: 8 <= lr <= 12, lr <= small_log <= 13 (12 for 64-bit
 * elements), columns per tile 2^(clog_plus1 - 1) <= 32.  clog_lo_plus1:
 * the column tile width of the size class whose columns are shorter than
 * the batch's tallest (its column passes run as launches of their own),
 * 2^(clog_lo_plus1 - 1) <= 32 columns; 0 = the same as clog_plus1. */
typedef struct tft_batch_params {
  uint32_t small_log;
  uint32_t lr;
  uint32_t clog_plus1;
  uint32_t clog_lo_plus1;
} tft_batch_params;

tft_status tft_ctx_reserve_batch(tft_ctx* ctx, uint32_t max_products,
                                 uint64_t work_words);
tft_status tft_batch_work_words(tft_prime prime, const tft_polymul_desc* descs,
                                uint32_t count, const tft_batch_params* params,
                                uint64_t* words);
tft_status tft_batch_plan(tft_ctx* ctx, const tft_polymul_desc* descs,
                          uint32_t count, const tft_batch_params* params);
tft_status tft_batch_run(tft_ctx* ctx, void* stream);
tft_status tft_polymul_batch(tft_ctx* ctx, const tft_polymul_desc* descs,
                             uint32_t count, const tft_batch_params* params,
                             void* stream);

/*
 * Device operand generator (not part of the paper's method: it lets a
 * served request carry only its identifier and lengths).  Writes n residues
 * of operand `operand` (0 = a, 1 = b) of request `request` under `seed` to
 * the device buffer out (16-byte aligned, n elements of the context's
 * prime): element i is v mod p for the 128-bit output
 * v = x0 + 2^32 x1 + 2^64 x2 + 2^96 x3 of Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw, SC 2011) with counter (i, operand, request mod 2^32,
 * request div 2^32) and key (seed mod 2^32, seed div 2^32).  Asynchronous
 * on `stream`.  Errors: TFT_EINVAL (null or misaligned out, n = 0 or
 * n > 2^32, operand > 1).
 */
tft_status tft_generate(tft_ctx* ctx, uint64_t seed, uint64_t request,
                        uint32_t operand, void* out, uint64_t n, void* stream);

/*
 * Device bytes one served request occupies while in flight (its in-place
 * footprint, the unit of the server's admission budget): a (na), b (nb) and
 * the product (na + nb - 1 elements), plus the row/column class's work area
 * (B' and two rows, as tft_batch_work_words), each part rounded up to 256
 * bytes.  Host only.
 */
tft_status tft_request_bytes(tft_prime prime, uint64_t na, uint64_t nb,
                             const tft_batch_params* params, uint64_t* bytes);

/*
 * Arena: the server's device-memory bookkeeping, exposed so that its
 * policy can be checked without a device.  First-fit allocation of byte
 * ranges of [0, size) in multiples of `align` (a power of two), free ranges
 * merged on release.  Host only; offsets, not pointers.
 * tft_arena_alloc returns TFT_ENOMEM when no free range is large enough;
 * tft_arena_free takes an offset returned by tft_arena_alloc (TFT_EINVAL
 * otherwise).  tft_arena_usage: bytes in use, the peak since creation, and
 * the number of free ranges.
 */
typedef struct tft_arena tft_arena;
tft_status tft_arena_create(uint64_t size, uint64_t align, tft_arena** out);
tft_status tft_arena_destroy(tft_arena* arena);
tft_status tft_arena_alloc(tft_arena* arena, uint64_t bytes,
                           uint64_t* offset);
tft_status tft_arena_free(tft_arena* arena, uint64_t offset);
tft_status tft_arena_usage(tft_arena* arena, uint64_t* used, uint64_t* peak,
                           uint64_t* free_ranges);

/*
 * Served products: a stream of requests, each the product of two operands
 * produced by tft_generate, answered through the batched product with
 * continuous batching.
 *
 * tft_server_create reserves budget_bytes of device memory (the admission
 * budget), its own stream and two descriptor tables of max_batch products
 * (two batches in flight).  The server borrows ctx (which must outlive it)
 * for the roots, the launch counting and, in one-by-one mode, the
 * single-call product; the batched mode uses `params` as its schedule.
 *
 * tft_server_replay runs `count` requests open loop: request i becomes
 * available reqs[i].arrival_s seconds after the start (arrival times
 * non-decreasing).  Mode TFT_SERVE_BATCHED: whenever one of the two batch
 * slots is free, every available request is admitted in arrival order while
 * its tft_request_bytes fit in the budget (at most max_batch per batch), and
 * the admitted requests' operands are generated and multiplied as one
 * batch; a request's memory is released when its batch completes.  Mode
 * TFT_SERVE_ONE_BY_ONE: each request, as it arrives, is generated and
 * multiplied by itself with tft_polymul on the server's stream (the plain
 * path, for comparison).  done_s[i] (optional) receives the completion time
 * of request i in seconds from the start, measured by CUDA events; where
 * keep[i] is non-null (optional array), the product of request i (na + nb
 * - 1 elements) is copied there before its memory is released.  The call
 * returns when every request has completed; stats (optional) summarise the
 * run.  Errors: TFT_EINVAL (bad request, unsorted arrivals, misaligned
 * keep), TFT_ERANGE (a request larger than the budget, or, one by one,
 * longer than the context's max_len), TFT_ECUDA.
 */
typedef struct tft_server tft_server;
typedef struct tft_request {
  uint64_t id;        /* generator counter of the operands */
  uint64_t na;
  uint64_t nb;
  double arrival_s;   /* scheduled arrival, seconds from the start */
} tft_request;
typedef struct tft_server_stats {
  uint64_t completed;
  uint64_t batches;     /* batches launched (one by one: requests) */
  uint64_t max_batch;   /* most requests in one batch */
  uint64_t peak_bytes;  /* most budget bytes in use at once */
  uint64_t launches;    /* kernels launched */
  double wall_s;        /* host time from the start to the last completion */
} tft_server_stats;
#define TFT_SERVE_BATCHED 0
#define TFT_SERVE_ONE_BY_ONE 1
tft_status tft_server_create(tft_ctx* ctx, uint64_t budget_bytes,
                             uint32_t max_batch,
                             const tft_batch_params* params,
                             tft_server** out);
tft_status tft_server_destroy(tft_server* server);
tft_status tft_server_replay(tft_server* server, const tft_request* reqs,
                             uint64_t count, uint64_t seed, int mode,
                             double* done_s, void* const* keep,
                             tft_server_stats* stats);

/*
 * tft_forward_noalloc: the in-place forward TFT of tft_forward, for callers
 * that must not allocate device memory and so cannot create a context --
 * for example a serving loop whose device memory is fully reserved at
 * start-up and that may not call cudaMalloc (which can synchronize the
 * device and stall other streams) while requests are in flight, or code
 * running inside an allocator callback that cannot re-enter the allocator.
 * The paper has no counterpart to this entry point; it is a deployment aid.
 *   x, n, k, stream  as in tft_forward (x a 16-byte aligned device pointer
 *                    on the calling thread's current device).
 * Scratch: instead of a context, the call uses one fixed array of 2^14
 * eight-byte words (128 KiB) in the library's static device memory.  Every
 * GPU on which the library is loaded holds that array until the process
 * exits.  Its size covers every length the library accepts:
 * n <= 2^25 for 2^64 - 2^32 + 1 and n <= min(2^K, 2^27) for the two 32-bit
 * primes; longer n returns TFT_ERANGE (and n > 2^k or k > K returns
 * TFT_EINVAL) without launching anything.
 * Set-up: the first call on each device resolves the array's device address
 * and configures the kernels for that device (no allocation); make that
 * first call before capturing any stream on that device.
 * Sharing: all calls on a device use the same array, which keeps whatever
 * the previous call left; each call writes every scratch word it reads, so
 * nothing needs clearing.  Calls whose work overlaps on the GPU (different
 * streams, or different host threads without ordering) race on the array;
 * order them on one stream.
 * Never calls cudaMalloc, cudaFree or any allocating routine.
 */
tft_status tft_forward_noalloc(tft_prime prime, void* x, uint64_t n,
                               uint32_t k, void* stream);

/*
 * tft_forward_noscratch / tft_inverse_noscratch: the in-place forward and
 * inverse TFT of tft_forward and tft_inverse (the same results, bit for
 * bit) reading and writing no device memory but the n-word buffer x: no
 * context, no scratch array, no allocation (Propositions 3.2 and 4.2 bound
 * the paper's own auxiliary space by O(1) cells).  The other transforms keep
 * the ragged last row's inputs E_q = C_q(omega_a) of the short columns in an
 * R-word scratch; here one cluster of 8 CTAs evaluates them by Horner's rule
 * straight from the buffer (the raw short columns before the forward
 * transforms them, the recovered ones after the inverse has) and runs the
 * last row from its shared memory -- extra work of about one multiply per
 * coefficient of the short columns, and a serial step between the column
 * launches.
 *   x, n, k, stream  as in tft_forward (x a 16-byte aligned device pointer
 *                    on the calling thread's current device).
 * Errors: as tft_forward, without the context's max_len (n up to 2^25 for
 * 2^64 - 2^32 + 1, min(2^K, 2^27) otherwise).  The first call for a
 * prime on a device reads the device's SM count and sets the kernels'
 * shared-memory limits (host state behind a lock, no allocation); make it
 * before capturing any stream on that device.  Calls may overlap freely on
 * the GPU: they share no device memory.
 */
tft_status tft_forward_noscratch(tft_prime prime, void* x, uint64_t n,
                                 uint32_t k, void* stream);
tft_status tft_inverse_noscratch(tft_prime prime, void* x, uint64_t n,
                                 uint32_t k, void* stream);

/*
 * Host-buffer variants: the same operations on HOST buffers.  Each call
 * copies the inputs to the context's staging buffers (cudaMemcpyAsync on
 * `stream`), runs the transform or product there, copies the result back and
 * synchronizes `stream` before returning.  Pinned host memory gives full
 * copy bandwidth.  Requires a context created with TFT_CTX_HOST_STAGING.
 */
tft_status tft_forward_host(tft_ctx* ctx, void* x_host, uint64_t n,
                            uint32_t k, void* stream);
tft_status tft_inverse_host(tft_ctx* ctx, void* X_host, uint64_t n,
                            uint32_t k, void* stream);
tft_status tft_polymul_host(tft_ctx* ctx, const void* a_host, uint64_t na,
                            const void* b_host, uint64_t nb, void* out_host,
                            void* stream);

/*
 * Device memory footprint of one operation, next to a padded power-of-two
 * NTT (van der Hoeven's TFT and the plain NTT both work in a 2^k buffer,
 * Section 1.2).
 *   op = 0 (transform, either direction): *inplace_bytes = n words + the
 *          context scratch the plan uses; *padded_bytes = 2^k words.
 *   op = 1 (product, n = r = na + nb - 1, k = ceil(lg r) if 0 is passed):
 *          *inplace_bytes = out (r words) + work (r words) + scratch;
 *          *padded_bytes = two 2^k-word buffers.
 * Pure host computation; no device is touched.
 */
tft_status tft_footprint(tft_prime prime, uint64_t n, uint32_t k, int op,
                         uint64_t* inplace_bytes, uint64_t* padded_bytes);

/*
 * Execution plan chosen for length n (host only), for diagnostics and
 * benchmarks: out[0] = 1 if the single-CTA path is used, out[1] = its log2
 * padded length; out[2] = lr (rows of 2^lr), out[3] = c (columns padded to
 * 2^c), out[4] = log2 columns per CTA, out[5] = a, out[6] = b,
 * out[7] = row CTAs per SM.  Returns TFT_ERANGE when n is unsupported.
 */
tft_status tft_describe_plan(tft_prime prime, uint64_t n, int64_t out[8]);

/* Bytes per element: 4 or 8. 0 for an unknown prime. */
uint32_t tft_element_bytes(tft_prime prime);

/* Sticky device-side status of a context (TFT_OK, TFT_ECUDA, TFT_ETIMEOUT).
 * Call after synchronizing the context's streams. */
tft_status tft_last_error(tft_ctx* ctx);

/* Static description of a status code. */
const char* tft_status_string(tft_status s);

/* Name of the CUDA error behind the calling thread's last TFT_ECUDA
 * ("no error" if none); a static string. */
const char* tft_last_cuda_error(void);

/*
 * Launch accounting and per-kernel timing.  Every kernel the library
 * launches is counted per context (tft_launch_count).  With profiling
 * enabled the library also records a CUDA event pair on the call's stream
 * around each launch; tft_profile_read (after the streams are synchronized)
 * returns, per kernel kind 0 .. TFT_NUM_KERNEL_KINDS-1, the summed duration
 * in milliseconds and the number of timed launches since the last
 * tft_profile_enable (which resets the totals).  Kind names come from
 * tft_kernel_name; a kind names a kernel family (a column pass, a row pass,
 * the ragged last row, ...).  Launches on the context's side stream run
 * concurrently with the main stream, so their durations can include time
 * spent waiting for an SM.  Profiling must be off while a stream is being captured
 * into a CUDA graph.
 */
#define TFT_NUM_KERNEL_KINDS 12
tft_status tft_profile_enable(tft_ctx* ctx, int enable);
tft_status tft_profile_read(tft_ctx* ctx, double* ms, uint64_t* launches);
const char* tft_kernel_name(int kind);
uint64_t tft_launch_count(tft_ctx* ctx);

/*
 * tft_transform_batch: the in-place forward (inverse = 0, Algorithm 1) or
 * inverse (inverse = 1, Algorithm 2) TFT of every buffer of a batch of
 * uneven lengths -- results bit for bit those of tft_forward / tft_inverse
 * on each buffer alone.  The transforms short enough for one CTA (2^12
 * words for 2^64 - 2^32 + 1, 2^13 otherwise) run in one persistent launch,
 * one CTA per transform at a time; the longer ones follow one after another
 * on `stream` on the row/column path (they share the context's scratch).
 *   descs   count entries {x, n}: 16-byte aligned device buffers that do
 *           not overlap, 1 <= n <= the context's max_len
 * The table of the short transforms goes into the context's batch
 * reservation (tft_ctx_reserve_batch with at least that many products;
 * work_words may be 0) and replaces a product batch planned there.
 * Errors: TFT_EINVAL for a null, misaligned or overlapping buffer or n = 0;
 * TFT_ERANGE for n beyond max_len or a reservation too small.
 */
typedef struct tft_transform_desc {
  void* x;
  uint64_t n;
} tft_transform_desc;
tft_status tft_transform_batch(tft_ctx* ctx, int inverse,
                               const tft_transform_desc* descs,
                               uint32_t count, void* stream);

/*
 * Pieces of a transform held in parts -- the data plane of a transform
 * sharded over several GPUs (one part per rank).  The library's transforms
 * of length n = a R + b (R = 2^lr, the split tft_describe_plan reports;
 * requires a plan that is not single-CTA, with lr >= 8) are the row/column
 * form of Algorithms 1 and 2, the split that Section 1.3 credits to the
 * cache-friendly TFT: column q holds x_{q + tR}, t <= a (long, q < b) or
 * t < a (short); every column is its own TFT, full row rho < a is block rho
 * of the length-2^k network, and the ragged last row (row a, b outputs)
 * needs E_q = C_q(omega_a) of the short columns.  With P = parts (a power
 * of two, P <= R) and W = R / P, part p holds
 *   - column block p: columns [p W, (p + 1) W) as an (a + 1) x W array at
 *     row stride W, element (t, j) = x_{pW + j + tR}; its long columns are
 *     j < b_p = min(max(b - p W, 0), W), and row a is used only for them;
 *   - E_p: W words, the block's share of E (entries j >= b_p);
 *   - full rows [rho_p, rho_{p+1}), rho_p = p a / P (integer division):
 *     positions rho R .. rho R + R - 1 of the transform, R words each;
 *   - for the last part, the ragged row: an R-word row buffer (first b
 *     words) with the R-word E gathered from all parts.
 * Forward TFT: tft_shard_columns(inverse 0) on every block; the caller
 * moves block rows to the parts owning them (an all-to-all) and gathers
 * the long columns' row a and every E_p into the last part's row and E;
 * tft_shard_rows(0) on every part's rows; tft_shard_last_row(0) on the last
 * part.  Inverse: tft_shard_rows(1); move rows back into column blocks;
 * tft_shard_columns(1, which 0) (short columns, writes E_p); gather E and
 * tft_shard_last_row(1) on the last part, whose row then holds the long
 * columns' entries of row a; scatter them into the blocks;
 * tft_shard_columns(1, which 1) (long columns).  Results are bit for bit
 * those of tft_forward / tft_inverse.
 *   inverse   0 forward, 1 inverse; which (inverse columns only): 0 the
 *             block's short columns, 1 its long ones
 *   block, rows, row, E   16-byte aligned device pointers as above (E may
 *             be NULL where the block has no short columns or b = 0)
 *   rho_begin, count      the part's rows rho_begin .. + count - 1 (< a)
 * Errors: TFT_EINVAL for a bad argument (parts not a power of two, part >=
 * parts, a single-CTA plan, rows beyond a); TFT_ERANGE for n beyond the
 * supported maximum.  No call allocates; the context's scratch is unused.
 */
tft_status tft_shard_columns(tft_ctx* ctx, int inverse, int which,
                             void* block, uint64_t n, uint32_t parts,
                             uint32_t part, void* E, void* stream);
tft_status tft_shard_rows(tft_ctx* ctx, int inverse, void* rows, uint64_t n,
                          uint64_t rho_begin, uint64_t count, void* stream);
tft_status tft_shard_last_row(tft_ctx* ctx, int inverse, void* row,
                              const void* E, uint64_t n, void* stream);

/*
 * Allocation-failure injection (a testing aid; the paper has no
 * counterpart).  Every device and pinned-host allocation the library makes
 * (context creation, tft_ctx_reserve_batch, tft_server_create) goes through
 * one host-side wrapper.  tft_debug_fail_allocation(n) makes the allocation
 * after the next n successful ones fail once, as if the device were out of
 * memory, without calling CUDA (n < 0 switches it off); the failing call
 * returns TFT_ENOMEM after releasing what it had allocated.
 * tft_debug_live_allocations returns how many of the library's allocations
 * are currently held, so that a test can check that a failed call leaked
 * nothing.  Neither touches the GPU.
 */
void tft_debug_fail_allocation(int64_t n);
int64_t tft_debug_live_allocations(void);

/*
 * tft_calibrate: measurement aid for the roofline (the paper has no
 * counterpart).  Launches one calibration kernel of `blocks` CTAs of 256
 * threads on `stream`: kind 0 runs eight independent chains of the context
 * field's modular multiply per thread (the multiply every butterfly uses),
 * kind 1 chains of 32-bit multiply-adds, kind 2 chains of 32-bit XORs, kind 3
 * the stage engine's 16-point unit (twist and constant network), each
 * `iters` times in registers.  Pipe counters of a profiler divided by *ops
 * give the cost of one operation in instructions and pipe cycles; the
 * caller's CUDA-event time around the launch gives the rate.
 *   out        device buffer of at least blocks * 256 * 8 bytes, 16-byte
 *              aligned; receives one meaningless word per thread
 *   ops        (may be NULL) operations per launch: modmuls, multiply-adds,
 *              XORs, or butterflies (32 per unit)
 * Errors: TFT_EINVAL for a null or small buffer, kind outside 0..3, zero
 * blocks or iterations; TFT_ECUDA if the launch fails.
 */
tft_status tft_calibrate(tft_ctx* ctx, int kind, uint32_t iters,
                         uint32_t blocks, void* out, uint64_t out_bytes,
                         void* stream, uint64_t* ops);

#ifdef __cplusplus
}
#endif

#endif /* TFT_GB300_H */
