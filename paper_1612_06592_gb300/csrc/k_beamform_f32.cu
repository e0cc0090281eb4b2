// Beamforming + de-dispersion, plain FP32 form (Sec. 3, first and third
// paragraphs):
//     beam[j = (b,t,pol)][k][m] = D[k,t] * sum_s w[k,b,s] * x[pol][k][m][s]
// as FP32 fused multiply-adds; int8/int16 samples are exact in FP32.
//
// One thread block handles (pol, subband k, 128 consecutive frames): the
// station samples of the tile are read once from HBM (contiguous, S*2 values
// per frame) into shared memory as [station][frame] complex floats, the
// weights of a chunk of 32 beams as [beam][station].  Each thread owns one
// frame and 4 beams at a time (16 FMAs per station and beam quad).  Beams are
// written as rows of consecutive frames, i.e. coalesced.  The block's partial
// sum of |beam|^2 (the Parseval noise estimate, |D| = 1) goes to
// power_part[j][k][tile] in a fixed reduction order (deterministic).
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int FT = 128;        // frames per block (= threads)
constexpr int BC = 32;         // beams per weight chunk
constexpr int BR = 4;          // beams per register block

template <typename T2>
__global__ void __launch_bounds__(FT) k_beamform_f32(
    const T2* __restrict__ x, long long pol_stride, const float2* __restrict__ w,
    const float2* __restrict__ dd, int S, int P, int K, int B, int Tr, long long F, long long row,
    float2* __restrict__ beams, float* __restrict__ power_part, int n_ftiles, int pol0) {
  extern __shared__ float2 smem[];
  float2* xs = smem;                 // [S][FT]
  float2* ws = smem + S * FT;        // [BC][S]
  __shared__ float red[FT / 32][BC];

  const int tile = blockIdx.x, k = blockIdx.y, pol = pol0 + (int)blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long f0 = (long long)tile * FT;
  const long long f = f0 + tid;
  const bool valid = f < F;

  // station samples of this (pol, k) and frame tile -> xs[s][frame]
  const T2* xk = x + (long long)pol * pol_stride + ((long long)k * F + f0) * S;
  const int nvalid = (int)min((long long)(FT), (long long)(F - f0));
  for (int e = tid; e < FT * S; e += FT) {
    const int fr = e / S, s = e - fr * S;
    float2 v = make_float2(0.f, 0.f);
    if (fr < nvalid) {
      const T2 q = xk[e];
      v = make_float2((float)q.x, (float)q.y);
    }
    xs[s * FT + fr] = v;
  }

  for (int b0 = 0; b0 < B; b0 += BC) {
    const int nb = min(BC, B - b0);
    __syncthreads();   // xs ready / previous chunk's ws and red consumed
    const float2* wk = w + ((long long)k * B + b0) * S;
    for (int e = tid; e < nb * S; e += FT) ws[e] = wk[e];
    __syncthreads();
    for (int bb = 0; bb < nb; bb += BR) {
      float2 acc[BR];
#pragma unroll
      for (int i = 0; i < BR; ++i) acc[i] = make_float2(0.f, 0.f);
      for (int s = 0; s < S; ++s) {
        const float2 xv = xs[s * FT + tid];
#pragma unroll
        for (int i = 0; i < BR; ++i) {
          const float2 wv = ws[min(bb + i, nb - 1) * S + s];
          acc[i].x = fmaf(wv.x, xv.x, acc[i].x);
          acc[i].x = fmaf(-wv.y, xv.y, acc[i].x);
          acc[i].y = fmaf(wv.x, xv.y, acc[i].y);
          acc[i].y = fmaf(wv.y, xv.x, acc[i].y);
        }
      }
#pragma unroll
      for (int i = 0; i < BR; ++i) {
        const int b = b0 + bb + i;
        if (bb + i >= nb) break;
        float pw = valid ? acc[i].x * acc[i].x + acc[i].y * acc[i].y : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, off);
        if (lane == 0) red[warp][bb + i] = pw;
        if (valid) {
          for (int t = 0; t < Tr; ++t) {
            const float2 d = dd[k * Tr + t];
            const float2 v = make_float2(d.x * acc[i].x - d.y * acc[i].y,
                                         d.x * acc[i].y + d.y * acc[i].x);
            const long long j = ((long long)b * Tr + t) * P + pol;
            beams[(j * K + k) * row + kPrefix + f] = v;
          }
        }
      }
    }
    __syncthreads();
    if (tid < nb) {
      float pw = 0.f;
#pragma unroll
      for (int wi = 0; wi < FT / 32; ++wi) pw += red[wi][tid];
      const int b = b0 + tid;
      for (int t = 0; t < Tr; ++t) {
        const long long j = ((long long)b * Tr + t) * P + pol;
        power_part[(j * K + k) * n_ftiles + tile] = pw;
      }
    }
  }
}

}  // namespace

int beamform_f32_frame_tile() { return FT; }


size_t f32_smem(const Shape& sh) { return (size_t)(sh.S * FT + BC * sh.S) * sizeof(float2); }

cudaError_t init_f32_attributes(const Shape& sh) {
  cudaError_t e = cudaFuncSetAttribute(k_beamform_f32<char2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32_smem(sh));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_beamform_f32<short2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)f32_smem(sh));
}

cudaError_t launch_beamform_f32(const lp_plan& p, const void* x, long long pol_stride,
                                cudaStream_t s, PolSel ps) {
  const auto& sh = p.shape;
  const int ntile = (int)((sh.F + FT - 1) / FT);
  const dim3 grid(ntile, sh.K, ps.npol ? ps.npol : sh.P);
  const size_t smem = f32_smem(sh);
  if (p.cfg.input_dtype == LP_INPUT_INT8) {
    k_beamform_f32<char2><<<grid, FT, smem, s>>>((const char2*)x, pol_stride, p.buf.w32, p.buf.dd,
                                                 sh.S, sh.P, sh.K, sh.B, sh.Tr, sh.F, p.row(),
                                                 p.buf.beams, p.buf.power_part, ntile, ps.pol0);
  } else {
    k_beamform_f32<short2><<<grid, FT, smem, s>>>((const short2*)x, pol_stride, p.buf.w32,
                                                  p.buf.dd, sh.S, sh.P, sh.K, sh.B, sh.Tr, sh.F,
                                                  p.row(), p.buf.beams, p.buf.power_part, ntile, ps.pol0);
  }
  return cudaGetLastError();
}

}  // namespace lp
