// Streaming HBM bandwidth at a given read/write mix (the context of the
// beamformer's HBM roofline).
//
// Every input float4 is read once and written `fan` times, to `fan` output
// arrays of the input's size, so a launch moves n (1 + fan) 16-byte words:
// fan = 1 is a plain copy (the driver's copy-bandwidth measurement), fan = 4
// the beamformer's mix (6.14 GB of station samples read, 25.6 GB of beam rows
// written: 1 : 4.2).  Grid-stride loop, two words in flight per thread, the
// grid a multiple of the SM count; no arithmetic.
#include <cuda_runtime.h>

namespace {

__global__ void __launch_bounds__(512) k_mix(const float4* __restrict__ in,
                                             float4* __restrict__ out, long long n, int fan) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const bool two = i + stride < n;
    const float4 a = in[i];
    const float4 b = two ? in[i + stride] : a;
    for (int r = 0; r < fan; ++r) {
      out[r * n + i] = a;
      if (two) out[r * n + i + stride] = b;
    }
  }
}

}  // namespace

extern "C" {

// Launches the mix `reps` times on the current device after one warm-up launch
// over n float4 of `in` into fan * n float4 of `out` (device buffers) and
// returns the mean CUDA-event time in *ms (0 on success, the cudaError
// otherwise).  blocks: the grid (e.g. 4 per SM).
int mb_mix_run(const void* in, void* out, long long n, int fan, int blocks, int reps,
               double* ms) {
  if (!in || !out || !ms || n < 1 || fan < 1 || fan > 16 || blocks < 1 || reps < 1)
    return (int)cudaErrorInvalidValue;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return (int)e;
  auto launch = [&]() {
    k_mix<<<blocks, 512>>>(static_cast<const float4*>(in), static_cast<float4*>(out), n, fan);
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
