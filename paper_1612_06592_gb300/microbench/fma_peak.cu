// FP32 FMA throughput of one GB300 (the ALU roofline's denominator).
//
// Every thread runs CH independent multiply-add chains for `iters` rounds of
// 16 steps; the chains never depend on one another, so with enough warps per
// scheduler the FMA pipe, not latency, sets the rate.  Two forms:
//   variant 0: scalar FFMA  (fmaf; 2 FLOP per lane and instruction),
//   variant 1: packed FFMA2 (__ffma2_rn on float2; 4 FLOP per lane and
//              instruction: two independent fused multiply-adds).
// Comparing them shows whether the packed instruction doubles the lane rate or
// only halves the instructions issued for the same rate.  The result is
// written only when it equals an impossible value, which keeps the chains
// alive without a store per step.
#include <cuda_runtime.h>

namespace {

constexpr int CH = 8;
constexpr int UNROLL = 16;

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float a, float b) {
  float acc[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) acc[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < CH; ++i) acc[i] = fmaf(acc[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += acc[i];
  if (s == -1.2345e30f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ffma2(float* out, int iters, float a, float b) {
  float2 acc[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i)
    acc[i] = make_float2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)(threadIdx.x + i));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < CH; ++i) acc[i] = __ffma2_rn(acc[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += acc[i].x + acc[i].y;
  if (s == -1.2345e30f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// FLOP one launch performs: blocks * threads * iters * UNROLL * CH multiply-adds
// per lane, 2 FLOP each (FFMA) or 4 (FFMA2).
double mb_fma_flop(int variant, int blocks, int threads, int iters) {
  const double fma = (double)blocks * threads * iters * UNROLL * CH;
  return fma * (variant == 1 ? 4.0 : 2.0);
}

// Launches variant (0 FFMA, 1 FFMA2) `reps` times on the current device after
// one warm-up launch and returns the mean CUDA-event time in *ms (0 on
// success, the cudaError otherwise).  `out` is a device buffer of blocks *
// threads floats (never written in practice).  threads <= 256.
int mb_fma_run(int variant, int blocks, int threads, int iters, int reps, float* out,
               double* ms) {
  if (variant < 0 || variant > 1 || blocks < 1 || threads < 32 || threads > 256 || iters < 1 ||
      reps < 1 || !out || !ms)
    return (int)cudaErrorInvalidValue;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return (int)e;
  const float a = 0.9999999f, b = 1e-7f;
  auto launch = [&]() {
    if (variant == 0)
      k_ffma<<<blocks, threads>>>(out, iters, a, b);
    else
      k_ffma2<<<blocks, threads>>>(out, iters, a, b);
    return cudaGetLastError();
  };
  e = launch();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  *ms = (double)t / reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (int)e;
}

}  // extern "C"
