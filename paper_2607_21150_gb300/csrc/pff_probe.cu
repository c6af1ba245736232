// Pipe-rate probes: dependent multiply-add chains that keep one arithmetic
// pipe of every SM busy, so that the roofline of an ALU-bound kernel can be
// stated against a rate measured on the same GPU and at the same clocks as
// the kernel (the FP64 Jacobian action is bound by the FP64 pipe).
//
//   PFF_PROBE_DFMA  FP64 fused multiply-add (DFMA), 2 flop each
//   PFF_PROBE_FFMA  FP32 fused multiply-add (FFMA), 2 flop each
//   PFF_PROBE_DMMA  FP64 warp matrix multiply-accumulate mma.sync m8n8k4
//                   (the only FP64 tensor-core instruction; tcgen05 has no
//                   FP64 kind), 2 * 8 * 8 * 4 = 512 flop per warp instruction
//   PFF_PROBE_CVT   double -> float -> double conversion instructions (two
//                   per step; counted as operations): on GB300 they run at
//                   the FP64 rate, which is why the kernels that move FP64
//                   work onto the FP32 pipes convert by integer operations
//
// Every thread (warp, for DMMA) runs kChains independent chains of `iters`
// steps, so the pipe sees kChains operations in flight per thread; the FMA
// chains converge to a fixed point, the DMMA accumulators grow linearly, and
// the final sums are stored so that no step is dead code.
#include "../../include/pff.h"

#include <cuda_runtime.h>

#include "pff_internal.h"

namespace pff {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;  // chain steps per loop trip (keeps loop overhead off the issue slots)

__global__ void k_probe_dfma(long long iters, double a, double b, double* sink) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = 1e-3 * (threadIdx.x + c);
  for (long long it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_ffma(long long iters, double a, double b, double* sink) {
  float acc[kChains];
  const float af = (float)a, bf = (float)b;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = 1e-3f * (threadIdx.x + c);
  for (long long it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], af, bf);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// mma.sync.aligned.m8n8k4.row.col.f64: A 8x4 (one double per thread), B 4x8
// (one double per thread), C = D 8x8 (two doubles per thread).
__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void k_probe_dmma(long long iters, double a, double b, double* sink) {
  double d[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 1e-3 * (threadIdx.x + c);
  // every step adds the same product A B (entries 4 * a/4 * b) to D, so the
  // accumulators grow linearly and stay finite for any iteration count used
  const double av = a * 0.25, bv = b;
  for (long long it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) dmma(d[c][0], d[c][1], av, bv);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_cvt(long long iters, double a, double b, double* sink) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = a + b * (threadIdx.x + c);
  for (long long it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = (double)__double2float_rn(acc[c]);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace pff

extern "C" int pff_probe_pipe(int kind, int64_t iters, int blocks, int threads, double* sink, double* flops,
                              void* stream) {
  using namespace pff;
  if (iters < 1 || iters % kUnroll != 0 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 ||
      !sink || !flops)
    return set_last_error(PFF_ERR_INVALID,
                          "pff_probe_pipe: need iters >= 1 (a multiple of 4), blocks >= 1, 32 <= threads <= 1024 "
                          "(multiple of 32), sink and flops");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double per_thread = (double)iters * kChains;
  const double nthreads = (double)blocks * threads;
  // chain multiplier and addend: a fixed point x = b / (1 - a) keeps every chain bounded
  const double a = 0.5, b = 0.25;
  switch (kind) {
    case PFF_PROBE_DFMA:
      k_probe_dfma<<<blocks, threads, 0, st>>>(iters, a, b, sink); note_launch();
      *flops = 2.0 * per_thread * nthreads;
      break;
    case PFF_PROBE_FFMA:
      k_probe_ffma<<<blocks, threads, 0, st>>>(iters, a, b, sink); note_launch();
      *flops = 2.0 * per_thread * nthreads;
      break;
    case PFF_PROBE_DMMA:
      k_probe_dmma<<<blocks, threads, 0, st>>>(iters, a, b, sink); note_launch();
      *flops = 512.0 * per_thread * (nthreads / 32.0);
      break;
    case PFF_PROBE_CVT:
      k_probe_cvt<<<blocks, threads, 0, st>>>(iters, a, b, sink); note_launch();
      *flops = 2.0 * per_thread * nthreads;
      break;
    default:
      return set_last_error(PFF_ERR_INVALID, "pff_probe_pipe: unknown probe kind");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(PFF_ERR_CUDA, cudaGetErrorString(e));
  return PFF_OK;
}
