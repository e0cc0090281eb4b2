// PPF inversion by windowed LSMR (Sec. 3, second paragraph): the inverse FFT
// of each frame, then the sparse system H x = y solved with LSMR (Fong and
// Saunders 2011).  H is the PPF's window; it splits into one banded Toeplitz
// system per phase p along the frames,
//     y_m[p] = sum_{t<16} a_p[t] x_p[m - 15 + t],   a_p[t] = h[t M + p],
// h the prototype (sum h = 1).  A block is solved window by window: window w
// takes the 272 equations of frames [256 w - 16, 256 w + 256) over the 287
// unknowns x_p[q], q in [256 w - 31, 256 w + 256), and keeps q in
// [256 w - 16, 256 w + 240), the unknowns all 16 of whose equations lie in the
// window; the output of a block lags its frames by 16 (sample (m - 16) M + p).
//
// The right-hand sides, the inverse DFT of every frame written phase-major
// zt[stream][p][frame + 16] (a phase's frames contiguous), come from the
// synthesis kernel's DFT role (launch_ippf_zt).
// k_lsmr: one warp per (stream, phase, window); lane l owns elements
// [9 l, 9 l + 9) of every vector.  A v and A^T u read a 24-element window of
// the other vector from shared memory once and slide the 16 taps over it in
// registers (complex x real tap = one packed FFMA2); norms by warp reduction;
// the scalar recurrences run redundantly in every lane.  FP32 throughout.
// k_lsmr_sigma / k_lsmr_trigger: the series' noise level per (stream, phase)
// (its gain depends on the phase's system) with the running update of the FIR
// path, and the threshold with warp-ballot compaction.
#include <algorithm>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int LS_W = 256;                      // unknowns kept per window
constexpr int LS_ROWS = LS_W + kPrefix;        // 272 equations
constexpr int LS_COLS = LS_ROWS + kTaps - 1;   // 287 unknowns
constexpr int LS_PER = 9;                      // elements per lane (32 * 9 >= 287)
constexpr int LS_WARPS = 4;                    // warps (phases) per block (3 blocks per SM)
constexpr int LS_PAD = 16;                     // zero guard before / after a vector in smem
constexpr int kLsmrLag = kPrefix;              // output row i is frame i - 16 of the block

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(LS_WARPS * 32, 3) k_lsmr(const float2* __restrict__ zt,
                                                        const double* __restrict__ proto,
                                                        const double* __restrict__ sums,
                                                        long long nfr, int n_win,
                                                        int iters, long long j0,
                                                        float2* __restrict__ out,
                                                        long long o_stream, long long o_phase,
                                                        long long o_frame) {
  __shared__ float2 us[LS_WARPS][LS_PAD + LS_ROWS + LS_PAD + 16];
  __shared__ float2 vs[LS_WARPS][LS_COLS + LS_PAD + 16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = (blockIdx.x % (kM / LS_WARPS)) * LS_WARPS + warp;
  const int w = blockIdx.x / (kM / LS_WARPS);
  const long long j = j0 + blockIdx.y;
  float2* u_s = us[warp];
  float2* v_s = vs[warp];
  // taps of this phase, (a, a) pairs
  float2 a[kTaps];
  const double inv_sum = 1.0 / sums[0];
#pragma unroll
  for (int t = 0; t < kTaps; ++t) {
    const float at = (float)(proto[t * kM + p] * inv_sum);
    a[t] = make_float2(at, at);
  }
  const int e0 = LS_PER * lane;                              // my elements e0 .. e0 + 8
  // guards and tails of the shared vectors are zero
  for (int i = lane; i < LS_PAD + LS_ROWS + LS_PAD + 16; i += 32) u_s[i] = make_float2(0.f, 0.f);
  for (int i = lane; i < LS_COLS + LS_PAD + 16; i += 32) v_s[i] = make_float2(0.f, 0.f);
  __syncwarp();

  // right-hand side: equations e = frames w W - 16 + e = zt positions w W + e
  const float2* b = zt + (j * kM + p) * nfr + (long long)w * LS_W;
  float2 u[LS_PER], v[LS_PER], h[LS_PER], hb[LS_PER], x[LS_PER];
  const float2 zero = make_float2(0.f, 0.f);
  float2 part = zero;
#pragma unroll
  for (int i = 0; i < LS_PER; ++i) {
    const int e = e0 + i;
    u[i] = e < LS_ROWS ? b[e] : zero;
    part = fma2(u[i], u[i], part);
  }
  // a norm from its sum of squares ss by one reciprocal square root: returns
  // 1 / norm (1 for a zero norm, which then leaves the vector unchanged)
  auto inv_norm = [](float ss, float& nrm) {
    const float r = ss > 0.f ? rsqrtf(ss) : 1.f;
    nrm = ss > 0.f ? ss * r : 0.f;
    return r;
  };
  float beta;
  const float rb0 = inv_norm(warp_sum(part.x + part.y), beta);
  // u <- u r, v <- v r (r = 1 / norm); packed FMUL2
  auto norm_u = [&](float r) {
    const float2 r2 = make_float2(r, r);
#pragma unroll
    for (int i = 0; i < LS_PER; ++i) u[i] = __fmul2_rn(u[i], r2);
  };
  auto norm_v = [&](float r) {
    const float2 r2 = make_float2(r, r);
#pragma unroll
    for (int i = 0; i < LS_PER; ++i) v[i] = __fmul2_rn(v[i], r2);
  };
  // A^T u - c v, into v; returns the new sum of squares
  auto rmatvec = [&](float c) {
#pragma unroll
    for (int i = 0; i < LS_PER; ++i)
      if (e0 + i < LS_ROWS) u_s[LS_PAD + e0 + i] = u[i];
    __syncwarp();
    // unknown n = e0 + i takes u[n - t], t < 16: window u[e0 - 15 .. e0 + 8]
    float2 win[LS_PER + kTaps - 1];
#pragma unroll
    for (int i = 0; i < LS_PER + kTaps - 1; ++i) win[i] = u_s[LS_PAD + e0 - (kTaps - 1) + i];
    const float2 mc = make_float2(-c, -c);
    float2 pt = zero;
#pragma unroll
    for (int i = 0; i < LS_PER; ++i) {
      float2 acc = __fmul2_rn(mc, v[i]);
#pragma unroll
      for (int t = 0; t < kTaps; ++t) acc = fma2(a[t], win[i + (kTaps - 1) - t], acc);
      v[i] = e0 + i < LS_COLS ? acc : zero;
      pt = fma2(v[i], v[i], pt);
    }
    __syncwarp();
    return warp_sum(pt.x + pt.y);
  };
  // A v - c u, into u; returns the new sum of squares
  auto matvec = [&](float c) {
#pragma unroll
    for (int i = 0; i < LS_PER; ++i)
      if (e0 + i < LS_COLS) v_s[e0 + i] = v[i];
    __syncwarp();
    // equation e = e0 + i takes v[e + t], t < 16: window v[e0 .. e0 + 23]
    float2 win[LS_PER + kTaps - 1];
#pragma unroll
    for (int i = 0; i < LS_PER + kTaps - 1; ++i) win[i] = v_s[e0 + i];
    const float2 mc = make_float2(-c, -c);
    float2 pt = zero;
#pragma unroll
    for (int i = 0; i < LS_PER; ++i) {
      float2 acc = __fmul2_rn(mc, u[i]);
#pragma unroll
      for (int t = 0; t < kTaps; ++t) acc = fma2(a[t], win[i + t], acc);
      u[i] = e0 + i < LS_ROWS ? acc : zero;
      pt = fma2(u[i], u[i], pt);
    }
    __syncwarp();
    return warp_sum(pt.x + pt.y);
  };

#pragma unroll
  for (int i = 0; i < LS_PER; ++i) {
    v[i] = zero;
    h[i] = zero;
    hb[i] = zero;
    x[i] = zero;
  }
  // The scalar recurrences run on reciprocals: every norm and both rotations'
  // lengths come from one reciprocal square root each, and the quotients of
  // the updates are products with the kept reciprocals 1 / rho, 1 / rhobar
  // (the warp's dependent chain between two products with A is then a few
  // multiplications long instead of several divisions).
  if (beta > 0.f) {
    norm_u(rb0);
    float alpha;
    float ra = inv_norm(rmatvec(0.f), alpha);
    if (alpha > 0.f) {
      norm_v(ra);
      float alphabar = alpha, zetabar = alpha * beta;
      float irho = 1.f, irhobar = 1.f, cbar = 1.f, sbar = 0.f;   // rho = rhobar = 1
#pragma unroll
      for (int i = 0; i < LS_PER; ++i) h[i] = v[i];
      for (int it = 0; it < iters; ++it) {
        // continue the bidiagonalisation
        norm_u(inv_norm(matvec(alpha), beta));
        ra = inv_norm(rmatvec(beta), alpha);
        norm_v(ra);
        // rotation P_k: rho = |(alphabar, beta)|
        const float irho_old = irho;
        const float q = fmaf(alphabar, alphabar, beta * beta);
        irho = rsqrtf(q);
        const float rho = q * irho;
        const float c = alphabar * irho, s = beta * irho;
        const float theta = s * alpha;
        alphabar = c * alpha;
        // rotation Pbar_k: rhobar = |(cbar rho, theta)|
        const float irhobar_old = irhobar;
        const float thetabar = sbar * rho;
        const float cr = cbar * rho;
        const float qb = fmaf(cr, cr, theta * theta);
        irhobar = rsqrtf(qb);
        cbar = cr * irhobar;
        sbar = theta * irhobar;
        const float zeta = cbar * zetabar;
        zetabar = -sbar * zetabar;
        // update h, hbar, x
        const float f1 = thetabar * rho * (irho_old * irhobar_old);
        const float f2 = zeta * (irho * irhobar);
        const float f3 = theta * irho;
        const float2 m1 = make_float2(-f1, -f1), p2 = make_float2(f2, f2),
                     m3 = make_float2(-f3, -f3);
#pragma unroll
        for (int i = 0; i < LS_PER; ++i) {
          hb[i] = fma2(m1, hb[i], h[i]);
          x[i] = fma2(p2, hb[i], x[i]);
          h[i] = fma2(m3, h[i], v[i]);
        }
      }
    }
  }
  // keep unknowns 15 .. 15 + W - 1: output frames w W .. w W + W - 1; frame i
  // of phase p of stream j at out[j o_stream + p o_phase + i o_frame]
  float2* ob = out + j * o_stream + (long long)p * o_phase + (long long)w * LS_W * o_frame;
#pragma unroll
  for (int i = 0; i < LS_PER; ++i) {
    const int n = e0 + i;
    if (n >= kTaps - 1 && n < kTaps - 1 + LS_W) ob[(long long)(n - (kTaps - 1)) * o_frame] = x[i];
  }
}

// Noise level of the LSMR series per (stream, phase): one warp per row of F
// samples (contiguous, phase-major), FP64 sum of |x|^2 / 2 in a fixed order,
// then the running update of the FIR path.
__global__ void __launch_bounds__(256) k_lsmr_sigma(const float2* __restrict__ xhat, long long F,
                                                    double alpha, double k_sigma,
                                                    const long long* __restrict__ blk,
                                                    double* __restrict__ sigma2,
                                                    float* __restrict__ theta2, long long rows) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;   // j * M + p
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;                                     // whole warps
  const float2* row = xhat + r * F;
  // 8 loads in flight per lane (F is a multiple of 256), partial sums in FP32
  // over 8 samples, FP64 across them
  double acc = 0.0;
  for (long long i0 = lane; i0 < F; i0 += 32 * 8) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(row + i0 + 32 * u);
    float part = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) part = fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, part));
    acc += (double)part;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) {
    const double pi = 0.5 * acc / (double)F;
    const double s2 = *blk == 0 ? pi : (1.0 - alpha) * sigma2[r] + alpha * pi;
    sigma2[r] = s2;
    theta2[r] = (float)(k_sigma * k_sigma * s2);
  }
}

// Trigger on the LSMR series: |x|^2 > theta2[j][p] for samples n >= 0,
// n = (block F + i - 16) M + p; warp-ballot compaction into the trigger list.
__global__ void __launch_bounds__(256) k_lsmr_trigger(const float2* __restrict__ xhat, long long F,
                                                      const float* __restrict__ theta2,
                                                      float k_sigma,
                                                      const long long* __restrict__ blk, int P,
                                                      int Tr, long long j0,
                                                      TriggerRec* __restrict__ trig,
                                                      unsigned long long* __restrict__ count,
                                                      long long cap) {
  const int p = blockIdx.y;
  const long long j = j0 + blockIdx.z;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long long r = j * kM + p;
  const float th2 = theta2[r];
  const long long n = (*blk * F + i - kLsmrLag) * kM + p;
  bool hit = false;
  float e2 = 0.f;
  if (i < F) {
    const float2 v = xhat[r * F + i];
    e2 = v.x * v.x + v.y * v.y;
    hit = n >= 0 && e2 > th2;
  }
  const unsigned mask = __ballot_sync(0xffffffffu, hit);
  if (!mask) return;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (hit) {
    const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    if ((long long)idx < cap) {
      TriggerRec rec;
      rec.n = n;
      rec.pol = (int)(j % P);
      rec.tec = (int)((j / P) % Tr);
      rec.beam = (int)(j / ((long long)P * Tr));
      rec.stream = (int)j;
      rec.env = sqrtf(e2);
      rec.sigma = sqrtf(th2) / k_sigma;
      trig[idx] = rec;
    }
  }
}

}  // namespace

int lsmr_window() { return LS_W; }

cudaError_t launch_lsmr(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const long long nfr = sh.F + kPrefix;
  const long long J = sh.J();
  cudaError_t e = launch_ippf_zt(p, s);
  if (e != cudaSuccess) return e;
  // the recovered series: phase-major (xhat, for the per-phase level and trigger),
  // or, when the full-rate filter follows, straight into its sample-major series
  // rows after the 2048 history samples
  const bool rows = p.cfg.fullrate_dedisp != 0;
  float2* out = rows ? p.buf.ufull + kFrTaps : p.buf.xhat;
  const long long o_stream = rows ? fullrate_row(p) : kM * sh.F;
  const long long o_phase = rows ? 1 : sh.F;
  const long long o_frame = rows ? kM : 1;
  for (long long j0 = 0; j0 < J; j0 += 65535) {             // grid y is at most 65535
    const unsigned nj = (unsigned)std::min<long long>(65535, J - j0);
    const int n_win = (int)(sh.F / LS_W);
    k_lsmr<<<dim3((unsigned)(kM / LS_WARPS * n_win), nj), LS_WARPS * 32, 0, s>>>(
        p.buf.zt, p.buf.proto, p.buf.filter_sums, nfr, n_win, p.cfg.lsmr_iters, j0, out,
        o_stream, o_phase, o_frame);
  }
  return cudaGetLastError();
}

cudaError_t launch_lsmr_trigger(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const long long rows = (long long)sh.J() * kM;
  k_lsmr_sigma<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(
      p.buf.xhat, sh.F, p.cfg.sigma_alpha, p.cfg.k_sigma, p.buf.blk, p.buf.lsmr_sigma2,
      p.buf.lsmr_theta2, rows);
  for (long long j0 = 0; j0 < sh.J(); j0 += 65535) {
    const unsigned nj = (unsigned)std::min<long long>(65535, sh.J() - j0);
    k_lsmr_trigger<<<dim3((unsigned)((sh.F + 255) / 256), kM, nj), 256, 0, s>>>(
        p.buf.xhat, sh.F, p.buf.lsmr_theta2, (float)p.cfg.k_sigma, p.buf.blk, sh.P, sh.Tr, j0,
        p.buf.trig, p.buf.trig_count, p.cfg.trigger_cap);
  }
  return cudaGetLastError();
}

}  // namespace lp
