// Beamforming + de-dispersion, plain FP32 form (Sec. 3, first and third
// paragraphs):
//     beam[j = (b,t,pol)][k][m] = D[k,t] * sum_s w[k,b,s] * x[pol][k][m][s]
// as FP32 fused multiply-adds; int8/int16 samples are exact in FP32.
//
// One thread block (4 warps) handles (pol, subband k, 256 consecutive frames);
// each thread owns two consecutive frames.  The tile's station samples are read
// once from HBM (contiguous, [frame][station]) into shared memory in their
// input form, station-major with a padded row, so that a thread reads both of
// its frames of one station in one conflict-free access; the weights of up to
// 64 beams at a time sit in shared memory as (w_re, w_re, -w_im, w_im).  A
// complex multiply-add is then two packed FFMA2 per frame,
//     (acc_re, acc_im) += (w_re, w_re) * (x_re, x_im) + (-w_im, w_im) * (x_im, x_re),
// a thread keeps BB beams x 2 frames of accumulators (BB = 4, 8 or 16, chosen
// by the GEMM autotuner; 8 by default) and every weight is one
// shared-memory broadcast for 4 FFMA2.  Beams are written as 16-byte pairs of
// frames, coalesced.  Each warp's partial of |beam|^2 over its 64 frames (the
// Parseval noise estimate, |D| = 1) goes to power_part[j][k][64-frame tile] in
// a fixed reduction order (deterministic).
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int FT = 256;          // frames per block
constexpr int NTH = 128;         // threads per block, two frames each
constexpr int FW = 64;           // frames per warp = noise-partial tile
constexpr int FTP = FT + 2;      // padded station row of the sample tile
constexpr int BCH = 64;          // beams whose weights sit in shared memory

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// two consecutive frames of one station: int8 or int16 complex pairs
template <typename T2> struct Pair2;
template <> struct Pair2<char2> { using T = char4; };
template <> struct Pair2<short2> { using T = short4; };

template <typename T2, int BB>
__global__ void __launch_bounds__(NTH, 3) k_beamform_f32(
    const T2* __restrict__ x, long long pol_stride, const float2* __restrict__ w,
    const float2* __restrict__ dd, int S, int P, int K, int B, int Tr, long long F, long long row,
    float2* __restrict__ beams, float* __restrict__ power_part, int n_ftiles, int pol0,
    int bch) {
  using T4 = typename Pair2<T2>::T;
  extern __shared__ float4 smem4[];
  float4* ws = smem4;                                        // [bch][S]
  T2* xs = reinterpret_cast<T2*>(ws + bch * S);              // [S][FTP]

  const int tile = blockIdx.x, k = blockIdx.y, pol = pol0 + (int)blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long f0 = (long long)tile * FT;
  const int nvalid = (int)min((long long)FT, F - f0);

  // station samples of this (pol, k) and frame tile -> xs[s][frame]; the
  // (frame, station) of sample e is carried from one e to the next (e += NTH)
  const T2* xk = x + (long long)pol * pol_stride + ((long long)k * F + f0) * S;
  {
    int fr = tid / S, st = tid - fr * S;
    const int dq = NTH / S, dr = NTH - dq * S;
    for (int e = tid; e < FT * S; e += NTH) {
      T2 v;
      v.x = 0;
      v.y = 0;
      if (fr < nvalid) v = xk[e];
      xs[st * FTP + fr] = v;
      st += dr;
      fr += dq;
      if (st >= S) {
        st -= S;
        ++fr;
      }
    }
  }

  const int fl = 2 * tid;                                    // my frames fl, fl + 1
  const bool va = fl < nvalid, vb = fl + 1 < nvalid;
  const int ptile = tile * (FT / FW) + warp;                 // my warp's noise tile
  const bool ptile_ok = (long long)ptile * FW < F;
  for (int b0 = 0; b0 < B; b0 += bch) {
    const int nb = min(bch, B - b0);
    __syncthreads();   // samples ready / previous weights consumed
    const float2* wk = w + ((long long)k * B + b0) * S;
    for (int e = tid; e < nb * S; e += NTH) {
      const float2 v = wk[e];
      ws[e] = make_float4(v.x, v.x, -v.y, v.y);
    }
    __syncthreads();
    for (int bb = 0; bb < nb; bb += BB) {
      float2 acc[BB][2];
#pragma unroll
      for (int i = 0; i < BB; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int st = 0; st < S; ++st) {
        const T4 q = *reinterpret_cast<const T4*>(xs + st * FTP + fl);
        const float2 xa = make_float2((float)q.x, (float)q.y);
        const float2 xb = make_float2((float)q.z, (float)q.w);
        const float2 xas = make_float2(xa.y, xa.x), xbs = make_float2(xb.y, xb.x);
#pragma unroll
        for (int i = 0; i < BB; ++i) {
          const float4 wv = ws[min(bb + i, nb - 1) * S + st];   // broadcast
          const float2 w0 = make_float2(wv.x, wv.y), w1 = make_float2(wv.z, wv.w);
          acc[i][0] = fma2(w1, xas, fma2(w0, xa, acc[i][0]));
          acc[i][1] = fma2(w1, xbs, fma2(w0, xb, acc[i][1]));
        }
      }
#pragma unroll
      for (int i = 0; i < BB; ++i) {
        if (bb + i >= nb) break;                             // uniform
        const int b = b0 + bb + i;
        float pw = (va ? fmaf(acc[i][0].x, acc[i][0].x, acc[i][0].y * acc[i][0].y) : 0.f) +
                   (vb ? fmaf(acc[i][1].x, acc[i][1].x, acc[i][1].y * acc[i][1].y) : 0.f);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pw += __shfl_xor_sync(0xffffffffu, pw, off);
        for (int t = 0; t < Tr; ++t) {
          const float2 d = dd[k * Tr + t];
          const float2 u = acc[i][0], v = acc[i][1];
          const long long j = ((long long)b * Tr + t) * P + pol;
          float2* dst = beams + (j * K + k) * row + kPrefix + f0 + fl;
          if (vb)
            *reinterpret_cast<float4*>(dst) =
                make_float4(d.x * u.x - d.y * u.y, d.x * u.y + d.y * u.x,
                            d.x * v.x - d.y * v.y, d.x * v.y + d.y * v.x);
          else if (va)
            *dst = make_float2(d.x * u.x - d.y * u.y, d.x * u.y + d.y * u.x);
          if (lane == 0 && ptile_ok) power_part[(j * K + k) * n_ftiles + ptile] = pw;
        }
      }
    }
  }
}

}  // namespace

int beamform_f32_frame_tile() { return FW; }

// beams with weights in shared memory at a time, and the block's shared memory
int f32_bch(const Shape& sh) { return sh.B < BCH ? sh.B : BCH; }
size_t f32_smem(const Shape& sh, size_t sample_bytes) {
  return (size_t)f32_bch(sh) * sh.S * sizeof(float4) + (size_t)sh.S * FTP * sample_bytes;
}

template <typename T2, int BB>
cudaError_t set_f32_attr(const Shape& sh) {
  return raise_smem_limit((const void*)k_beamform_f32<T2, BB>, f32_smem(sh, sizeof(T2)));
}

cudaError_t init_f32_attributes(const Shape& sh) {
  cudaError_t e = set_f32_attr<char2, 8>(sh);
  if (e == cudaSuccess) e = set_f32_attr<char2, 16>(sh);
  if (e == cudaSuccess) e = set_f32_attr<char2, 4>(sh);
  if (e == cudaSuccess) e = set_f32_attr<short2, 8>(sh);
  if (e == cudaSuccess) e = set_f32_attr<short2, 16>(sh);
  if (e == cudaSuccess) e = set_f32_attr<short2, 4>(sh);
  return e;
}

template <typename T2, int BB>
void launch_f32(const lp_plan& p, const void* x, long long pol_stride, cudaStream_t s,
                PolSel ps) {
  const auto& sh = p.shape;
  const int nblk = (int)((sh.F + FT - 1) / FT);
  const dim3 grid(nblk, sh.K, ps.npol ? ps.npol : sh.P);
  k_beamform_f32<T2, BB><<<grid, NTH, f32_smem(sh, sizeof(T2)), s>>>(
      (const T2*)x, pol_stride, p.buf.w32, p.buf.dd, sh.S, sh.P, sh.K, sh.B, sh.Tr, sh.F, p.row(),
      p.buf.beams, p.buf.power_part, p.n_ftiles_bf, ps.pol0, f32_bch(sh));
}

// beams per accumulator pass of each configuration (the first is the default)
constexpr int kF32Beams[3] = {8, 16, 4};

template <typename T2>
void launch_f32_bb(const lp_plan& p, const void* x, long long pol_stride, cudaStream_t s,
                   PolSel ps) {
  const int bb = p.gemm_cfg >= 0 && p.gemm_cfg < 3 ? kF32Beams[p.gemm_cfg] : kF32Beams[0];
  if (bb == 16)
    launch_f32<T2, 16>(p, x, pol_stride, s, ps);
  else if (bb == 4)
    launch_f32<T2, 4>(p, x, pol_stride, s, ps);
  else
    launch_f32<T2, 8>(p, x, pol_stride, s, ps);
}

cudaError_t launch_beamform_f32(const lp_plan& p, const void* x, long long pol_stride,
                                cudaStream_t s, PolSel ps) {
  if (p.cfg.input_dtype == LP_INPUT_INT8)
    launch_f32_bb<char2>(p, x, pol_stride, s, ps);
  else
    launch_f32_bb<short2>(p, x, pol_stride, s, ps);
  return cudaGetLastError();
}

int tc_configs(const Shape& sh, int esz, int* desc, int max);

int beamform_gemm_configs(const lp_plan& p, int* desc, int max) {
  if (p.cfg.precision == LP_PREC_FP16)
    return tc_configs(p.shape, p.cfg.input_dtype == LP_INPUT_INT8 ? 1 : 2, desc, max);
  int n = 0;
  for (int i = 0; i < 3 && n < max; ++i, ++n) {
    desc[2 * n] = kF32Beams[i];
    desc[2 * n + 1] = 0;
  }
  return n;
}

}  // namespace lp
