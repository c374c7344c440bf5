// Calibration kernels for the roofline (include/tft.h: tft_calibrate).
//
// The roofline of a transform kernel is the slower of its algorithmic bytes
// at the HBM bandwidth and its algorithmic modular multiplies at the
// multiply pipe's rate.  How many multiply-pipe cycles one modular multiply
// of a field costs is a property of the instruction sequence the compiler
// emits for it (a 64 x 64-bit product and its reduction for 2^64 - 2^32 + 1,
// a Montgomery REDC for the 32-bit primes), so it is measured rather than
// assumed: these kernels run long chains of independent operations in
// registers, with no memory traffic inside the loop, so that a profiler's
// pipe counters divided by the operation count give the cost per operation,
// and the CUDA-event time gives the rate the GPU reaches.
//
//   kind 0  modular multiply chains of the field (F::mul_tw, eight
//           independent chains per thread)
//   kind 1  32-bit multiply-add chains (mad.lo.u32): the multiply pipe's
//           lane rate
//   kind 2  32-bit XOR chains: the integer ALU pipe's lane rate
//   kind 3  the stage engine's 16-point unit (twist by the powers of a
//           per-thread zeta, then the constant 16-point network), the
//           butterfly rate in registers
//
// Every kernel writes one word per thread so that nothing is optimized
// away; the result values are meaningless.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ctx.h"
#include "stages.cuh"

using namespace tftgb;

namespace {

constexpr int kCalibThreads = 256;

template <class F>
__global__ void __launch_bounds__(kCalibThreads)
k_calib_modmul(typename F::T* out, uint32_t iters) {
  using T = typename F::T;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T x[8], w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = (T)((tid * 0x9E3779B97F4A7C15ull + (uint64_t)j) % F::P);
    w[j] = (T)((tid * 77u + (uint64_t)j * 0x5bd1e995u + 3u) % F::P);
  }
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = F::mul_tw(x[j], w[j]);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= x[j];
  out[tid] = s;
}

__global__ void __launch_bounds__(kCalibThreads)
k_calib_mad32(uint32_t* out, uint32_t iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = tid + (uint32_t)j;
  const uint32_t a = tid | 1u, b = tid * 3u;
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(a), "r"(b));
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= x[j];
  out[tid] = s;
}

__global__ void __launch_bounds__(kCalibThreads)
k_calib_xor32(uint32_t* out, uint32_t iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8], y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = tid + (uint32_t)j;
    y[j] = tid ^ ((uint32_t)j * 77u);
  }
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      asm volatile("xor.b32 %0, %0, %1;" : "+r"(x[j]) : "r"(y[j]));
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= x[j];
  out[tid] = s;
}

template <class F>
__global__ void __launch_bounds__(kCalibThreads)
k_calib_unit(typename F::T* out, uint32_t iters, RootTable<typename F::T> rt) {
  using T = typename F::T;
  __shared__ StageConsts<T> K;
  fill_stage_consts<F>(&K, rt, 4);
  __syncthreads();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i)
    x[i] = (T)((tid * 0x9E3779B97F4A7C15ull + (uint64_t)i * 0x1234567ull) %
               F::P);
  T zeta = (T)((tid + 12345u) % F::P);
#pragma unroll 1
  for (uint32_t it = 0; it < iters; ++it) {
    twist<F, 4>(x, zeta);
    cnet_fwd<F, 4>(x, K);
    zeta = F::canon(x[3]);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) s ^= F::canon(x[i]);
  out[tid] = s;
}

template <class F>
cudaError_t launch_calib(int kind, uint32_t iters, void* out, uint32_t blocks,
                         const unsigned char* rt_raw, cudaStream_t st) {
  using T = typename F::T;
  switch (kind) {
    case 0:
      k_calib_modmul<F><<<blocks, kCalibThreads, 0, st>>>((T*)out, iters);
      break;
    case 1:
      k_calib_mad32<<<blocks, kCalibThreads, 0, st>>>((uint32_t*)out, iters);
      break;
    case 2:
      k_calib_xor32<<<blocks, kCalibThreads, 0, st>>>((uint32_t*)out, iters);
      break;
    default: {
      RootTable<T> rt;
      memcpy(&rt, rt_raw, sizeof(rt));
      k_calib_unit<F><<<blocks, kCalibThreads, 0, st>>>((T*)out, iters, rt);
      break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" tft_status tft_calibrate(tft_ctx* ctx, int kind, uint32_t iters,
                                    uint32_t blocks, void* out,
                                    uint64_t out_bytes, void* stream,
                                    uint64_t* ops) {
  if (!ctx || !out || kind < 0 || kind > 3 || blocks == 0 || iters == 0)
    return TFT_EINVAL;
  if (!aligned16(out) || out_bytes < (uint64_t)blocks * kCalibThreads * 8)
    return TFT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (ctx->prime) {
    case 0: e = launch_calib<P998>(kind, iters, out, blocks, ctx->rt, st); break;
    case 1: e = launch_calib<P2013>(kind, iters, out, blocks, ctx->rt, st); break;
    default:
      e = launch_calib<Goldilocks>(kind, iters, out, blocks, ctx->rt, st);
      break;
  }
  if (e != cudaSuccess) {
    note(e);
    return TFT_ECUDA;
  }
  ++ctx->launches;
  if (ops) {
    // operations per launch: modmuls, mads or xors (8 chains per thread),
    // or butterflies (32 per 16-point unit)
    const uint64_t per = kind == 3 ? 32 : 8;
    *ops = (uint64_t)blocks * kCalibThreads * iters * per;
  }
  return TFT_OK;
}
