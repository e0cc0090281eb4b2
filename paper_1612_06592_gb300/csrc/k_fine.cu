// Fine-resolution de-dispersion in the channel domain (Sec. 3, third paragraph).
//
// The beamformer applies the STEC phase at each subband centre.  The rest of
// the phase inside subband k, psi(nu_k + dnu) = phi(nu_k + dnu) - phi(nu_k)
// = A dnu (1/nu_ref^2 - 1/((nu_k + dnu) nu_k)) cycles (mostly a delay of a
// fraction of a frame), is a filter along the subband's frames, whose
// frequency is the frame-rate frequency f = dnu / (fs / M) in [-1/2, 1/2):
//     R(f) = exp(-2 pi i (psi(f fs / M) + 8 f))          (8 frames of delay),
//     r[q] = w_k[q] (1/1024) sum_j R(f_j) exp(+2 pi i f_j q),  q < 17,
// f_j = (j + 1/2)/1024 - 1/2, w_k a Kaiser window (beta 4) centred on the
// subband's first-order delay c_k = 8 + A (fs/M) (1/nu_ref^2 - 1/nu_k^2) with
// half-width min(c_k, 16 - c_k).  The filter is causal, so a frame needs the
// 16 frames before it, which the beam rows hold in their prefix.
//
// k_fine_taps: one warp per (subband, trial); FP64 arguments and sums.
// k_fine: one 4-warp block per (stream, subband, 1024 frames) (the index
// arithmetic of a block is four 32-bit divisions); the frames (and the 16
// before them) are copied by cp.async, all at once, into shared memory in
// rows of 8 frames padded to 20 words, so that both the 16-byte copies and
// each thread's 16-byte reads of three consecutive rows are conflict-free; a
// thread filters 8 consecutive
// frames from a 24-frame window in registers, two packed FFMA2 per tap and
// frame with the taps as (r.re, r.re, -r.im, r.im).  HBM-bound: 8 bytes in and
// 8 out per bin-frame, 136 FLOP.
#include <algorithm>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int FN_NTH = 128;                     // threads per block
constexpr int FN_FPT = 8;                       // frames per thread
constexpr int FN_FT = FN_NTH * FN_FPT;          // frames per block
constexpr int FN_ROWW = 20;                     // words per 8-frame shared-memory row
constexpr int FN_ROWS = (FN_FT + kPrefix) / 8;  // rows: the tile and the 16 frames before

__global__ void __launch_bounds__(128) k_fine_taps(const double* __restrict__ tec, int K, int Tr,
                                                   int first_bin, double nu_ref,
                                                   float4* __restrict__ taps) {
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (wid >= (long long)K * Tr) return;                  // whole warps leave together
  const int t = (int)(wid % Tr), k = (int)(wid / Tr);
  const double dnu_sb = kFs / kM;
  const double nu = kNu0 + (double)(first_bin + k) * dnu_sb;
  const double a = kKappa * tec[t] * kTecu / kC;
  const double slope = 1.0 / (nu_ref * nu_ref);
  double re[kFineTaps], im[kFineTaps];
#pragma unroll
  for (int q = 0; q < kFineTaps; ++q) re[q] = im[q] = 0.0;
  for (int j = lane; j < kFineGrid; j += 32) {
    const double f = ((double)j + 0.5) / kFineGrid - 0.5;
    const double dnu = f * dnu_sb;
    const double cyc = a * dnu * (slope - 1.0 / ((nu + dnu) * nu)) + kFineDelay * f;
#pragma unroll
    for (int q = 0; q < kFineTaps; ++q) {
      const double x = f * q - cyc;                      // exp(+2 pi i (f q - cyc))
      double sn, cs;
      sincospi(2.0 * (x - rint(x)), &sn, &cs);
      re[q] += cs;
      im[q] += sn;
    }
  }
#pragma unroll
  for (int q = 0; q < kFineTaps; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      re[q] += __shfl_xor_sync(0xffffffffu, re[q], off);
      im[q] += __shfl_xor_sync(0xffffffffu, im[q], off);
    }
  }
  const double c = kFineDelay + a * dnu_sb * (slope - 1.0 / (nu * nu));
  const double hw = fmin(c, (kFineTaps - 1) - c);
  const double i0b = bessel_i0_series(kFineBeta);
#pragma unroll
  for (int q = 0; q < kFineTaps; ++q) {
    if (lane != q) continue;
    const double u = (q - c) / hw;
    const double w = bessel_i0_series(kFineBeta * sqrt(fmax(1.0 - u * u, 0.0))) / i0b;
    const float rr = (float)(w * re[q] / kFineGrid), ri = (float)(w * im[q] / kFineGrid);
    taps[wid * kFineTaps + q] = make_float4(rr, rr, -ri, ri);
  }
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// grid: x = frame tile, y = launch row (stream jj, bin k) - row0; 32-bit index
// arithmetic (rows < 2^32), the stream map only when it is not the identity
__global__ void __launch_bounds__(FN_NTH) k_fine(const float2* __restrict__ beams,
                                                 float2* __restrict__ out,
                                                 const float4* __restrict__ taps, unsigned K,
                                                 unsigned Tr, unsigned P, long long F,
                                                 long long row, unsigned pol0, unsigned npol,
                                                 unsigned row0) {
  __shared__ __align__(16) float tile[FN_ROWS * FN_ROWW];
  __shared__ float4 tp[kFineTaps];
  const unsigned rr = row0 + blockIdx.y;
  const unsigned jj = rr / K, k = rr - jj * K;
  const unsigned j = npol == P ? jj : (jj / npol) * P + pol0 + jj % npol;
  const unsigned t = (j / P) % Tr;
  const long long m0 = (long long)blockIdx.x * FN_FT;
  const int nval = (int)min((long long)FN_FT, F - m0);       // a multiple of 8
  const long long base = ((long long)j * K + k) * row + kPrefix + m0;   // frame m0 of the row
  // frames [m0 - 16, m0 + nval) as 16-byte pairs (rows and prefix are even),
  // all copies in flight at once
  const float4* src = reinterpret_cast<const float4*>(beams + base - kPrefix);
  for (int i = threadIdx.x; i < (nval + kPrefix) / 2; i += FN_NTH)
    cp_async16(&tile[(i >> 2) * FN_ROWW + (i & 3) * 4], src + i);
  if (threadIdx.x < kFineTaps)
    cp_async16(&tp[threadIdx.x], taps + ((long long)k * Tr + t) * kFineTaps + threadIdx.x);
  cp_async_wait_all();
  __syncthreads();
  const int m = threadIdx.x * FN_FPT;                        // my first frame in the tile
  if (m >= nval) return;
  // x[i] = frame m - 16 + i (tile rows threadIdx.x .. threadIdx.x + 2)
  float2 x[24], xs[24];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(&tile[(threadIdx.x + r) * FN_ROWW + 4 * c]);
      x[8 * r + 2 * c] = make_float2(v.x, v.y);
      x[8 * r + 2 * c + 1] = make_float2(v.z, v.w);
    }
  }
#pragma unroll
  for (int i = 0; i < 24; ++i) xs[i] = make_float2(x[i].y, x[i].x);
  float2 acc[FN_FPT];
#pragma unroll
  for (int i = 0; i < FN_FPT; ++i) acc[i] = make_float2(0.f, 0.f);
  // out[m + i] = sum_q r[q] in[m + i - q] = sum_q r[q] x[16 + i - q]
#pragma unroll
  for (int q = 0; q < kFineTaps; ++q) {
    const float4 w = tp[q];                                  // broadcast
    const float2 w0 = make_float2(w.x, w.y), w1 = make_float2(w.z, w.w);
#pragma unroll
    for (int i = 0; i < FN_FPT; ++i)
      acc[i] = fma2(w1, xs[16 + i - q], fma2(w0, x[16 + i - q], acc[i]));
  }
  float4* dst = reinterpret_cast<float4*>(out + base + m);
#pragma unroll
  for (int i = 0; i < FN_FPT / 2; ++i)
    dst[i] = make_float4(acc[2 * i].x, acc[2 * i].y, acc[2 * i + 1].x, acc[2 * i + 1].y);
}

}  // namespace

cudaError_t launch_fine_taps(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const long long warps = (long long)sh.K * sh.Tr;
  k_fine_taps<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, s>>>(
      p.buf.tec, sh.K, sh.Tr, p.cfg.first_bin, p.nu_ref, p.buf.fine_taps);
  return cudaGetLastError();
}

cudaError_t launch_fine(const lp_plan& p, cudaStream_t s, PolSel ps) {
  const auto& sh = p.shape;
  const int npol = ps.npol ? ps.npol : sh.P;
  const unsigned n_tiles = (unsigned)((sh.F + FN_FT - 1) / FN_FT);
  const long long rows = (long long)sh.J() / sh.P * npol * sh.K;
  for (long long r0 = 0; r0 < rows; r0 += 65535) {            // grid y is at most 65535
    const dim3 grid(n_tiles, (unsigned)std::min<long long>(65535, rows - r0));
    k_fine<<<grid, FN_NTH, 0, s>>>(p.buf.beams, p.buf.beams_fine, p.buf.fine_taps, sh.K, sh.Tr,
                                   sh.P, sh.F, p.row(), ps.pol0, npol, (unsigned)r0);
  }
  return cudaGetLastError();
}

}  // namespace lp
