// Full-rate de-dispersion of the synthesised 200 MHz series (Sec. 3, third
// paragraph: the STEC phase applied to the spectrum of the time series at full
// resolution), as a streaming filter after the inversion:
//
//     v[o] = sum_{l < 2048} h[l] u[o - l]       (u: a stream's analytic series)
//
// h: the response exp(-2 pi i phi(nu)) (nu = 100 MHz + f fs for f >= 0, 1 for
// f < 0) sampled on 8192 frequencies and inverted, kept over the delays
// -1024 .. 1023 with a Tukey window (flat within 768 of zero delay, half-cosine
// tapers beyond) and delayed by 1024 samples, so pulses appear one frame later.
// The whole STEC phase is applied here; the beamformer's per-subband phase is
// then 1.
//
// k_fullrate, overlap-save: a stream's series row holds 2048 samples of the
// previous block, then the block's F * 1024 samples.  Segment s covers row
// samples [6144 s, 6144 s + 8192): one 8192-point FFT, the product with the
// taps' spectrum, an inverse FFT; positions 2048 .. 8191 of the result are the
// block's outputs 6144 s .. 6144 s + 6143 (no wrap-around reaches them).  The
// envelope |v| is compared with the stream's threshold and triggers are
// compacted by warp ballots, as in the synthesis kernel; Re v is the stored
// time series.  After the LSMR inversion (the paper's order) the filter reads
// the recovered series (k_lsmr writes it sample-major into the series rows)
// and writes v back phase-major for the LSMR path's per-phase noise level and
// trigger.
//
// The FFT: decimation in frequency, radices 16 x 16 x 16 x 2, in place in
// shared memory.  A thread owns 16 values per pass (a 16-point DFT in
// registers by radix-2 stages with constant twiddles); positions are padded by
// 2 per 32 so that the half-warps' 8-byte accesses of every pass fall on
// distinct banks; the last radix-2 step pairs neighbouring lanes by shuffles.
// The spectrum stays in digit-reversed order (position 512 k1 + 32 k2 + 2 k3
// + k4 holds frequency k1 + 16 k2 + 256 k3 + 4096 k4): the taps' spectrum is
// stored in the same order, per thread and value, and the inverse transform
// runs the same network backwards (decimation in time, conjugate twiddles),
// ending in natural order.  1/8192 is folded into the taps' spectrum.
//
// Set-up (per STEC set, FP64): the response on the 8192-point grid, the taps by
// a direct inverse transform, the window, and the taps' spectrum by a direct
// transform, rounded to FP32 once.
#include "lp_internal.cuh"

#include <algorithm>
#include <cstdint>

namespace lp {
namespace {

constexpr int FR_NT = 512;                  // threads per block, 16 values each
constexpr int FR_N = kFrN;                  // 8192-point transforms
constexpr int FR_V = kFrN - kFrTaps;        // 6144 outputs per segment
static_assert(FR_N == 16 * FR_NT, "16 values per thread");

// padded shared-memory position of transform position i
__host__ __device__ constexpr int frp(int i) { return i + 2 * (i >> 5); }
constexpr int FR_SMEM = (frp(FR_N - 1) + 1) * (int)sizeof(float4);

// One transform position of the block's two segments: re = (re_a, re_b),
// im = (im_a, im_b), so every packed FP32 instruction does the same step for
// both segments.
struct CP {
  float2 re, im;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

__device__ __forceinline__ CP cadd(CP a, CP b) { return CP{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP csub(CP a, CP b) { return CP{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// a * w, w = (c, c, s, s) for the complex factor c + i s
__device__ __forceinline__ CP cmul(CP a, float4 w) {
  const float2 c = make_float2(w.x, w.y), s = make_float2(w.z, w.w);
  return CP{fma2(a.re, c, mul2(a.im, make_float2(-s.x, -s.y))), fma2(a.re, s, mul2(a.im, c))};
}
// a * conj(w)
__device__ __forceinline__ CP cmulc(CP a, float4 w) {
  const float2 c = make_float2(w.x, w.y), s = make_float2(w.z, w.w);
  return CP{fma2(a.re, c, mul2(a.im, s)), fma2(a.im, c, mul2(a.re, make_float2(-s.x, -s.y)))};
}
// the factor c + i s stored as (c, s), widened to the packed pairs
__device__ __forceinline__ float4 wide(float2 w) { return make_float4(w.x, w.x, w.y, w.y); }
__device__ __forceinline__ CP cmul_const(CP a, float c, float s) {    // a * (c + i s)
  return CP{fma2(a.re, bc(c), mul2(a.im, bc(-s))), fma2(a.re, bc(s), mul2(a.im, bc(c)))};
}

// a * exp(S 2 pi i e / 16) for e in [0, 8) (a constant after unrolling).
template <int S>
__device__ __forceinline__ CP rot16(CP a, int e) {
  constexpr float r = 0.70710678118654752440f;
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
  constexpr float fs = (float)S;
  switch (e) {
    case 0: return a;
    case 1: return cmul_const(a, c1, fs * s1);
    case 2:   // (re - S im, im + S re) / sqrt 2
      return fs > 0 ? CP{mul2(sub2(a.re, a.im), bc(r)), mul2(add2(a.im, a.re), bc(r))}
                    : CP{mul2(add2(a.re, a.im), bc(r)), mul2(sub2(a.im, a.re), bc(r))};
    case 3: return cmul_const(a, s1, fs * c1);
    case 4:   // S i
      return fs > 0 ? CP{make_float2(-a.im.x, -a.im.y), a.re}
                    : CP{a.im, make_float2(-a.re.x, -a.re.y)};
    case 5: return cmul_const(a, -s1, fs * c1);
    case 6:   // (-re - S im, -im + S re) / sqrt 2
      return fs > 0 ? CP{mul2(add2(a.re, a.im), bc(-r)), mul2(sub2(a.re, a.im), bc(r))}
                    : CP{mul2(sub2(a.im, a.re), bc(r)), mul2(add2(a.re, a.im), bc(-r))};
    default: return cmul_const(a, -c1, fs * s1);
  }
}

__host__ __device__ constexpr int br4(int i) {
  return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3);
}

// v[k] <- sum_r v[r] exp(S 2 pi i r k / 16): radix-2 decimation in frequency,
// then the bit reversal (register renaming).
template <int S>
__device__ __forceinline__ void dft16(CP (&v)[16]) {
#pragma unroll
  for (int span = 8; span >= 1; span >>= 1) {
#pragma unroll
    for (int st = 0; st < 16; st += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const CP a = v[st + j], b = v[st + j + span];
        v[st + j] = cadd(a, b);
        v[st + j + span] = rot16<S>(csub(a, b), j * (8 / span));
      }
    }
  }
  CP o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) o[br4(i)] = v[i];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// The radix-2 step across the lane pair (t, t ^ 1): lane b keeps
// y0 + (-1)^b y1 (y_b: lane b's value); its own inverse up to the factor 2.
__device__ __forceinline__ float2 shfl2(float2 v) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ void pair_step(CP (&v)[16], int b) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const CP p{shfl2(v[k].re), shfl2(v[k].im)};
    v[k] = b ? csub(p, v[k]) : cadd(v[k], p);
  }
}

// exp(-2 pi i k / 32) for lane parity b (1 for b = 0), k in [0, 16): (c, c, s, s)
__device__ __forceinline__ float4 w32(int k, int b) {
  constexpr float c[16] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                           0.83146961230254523708f, 0.70710678118654752440f,
                           0.55557023301960222474f, 0.38268343236508977173f,
                           0.19509032201612826785f, 0.0f, -0.19509032201612826785f,
                           -0.38268343236508977173f, -0.55557023301960222474f,
                           -0.70710678118654752440f, -0.83146961230254523708f,
                           -0.92387953251128675613f, -0.98078528040323044913f};
  constexpr float s[16] = {0.0f, 0.19509032201612826785f, 0.38268343236508977173f,
                           0.55557023301960222474f, 0.70710678118654752440f,
                           0.83146961230254523708f, 0.92387953251128675613f,
                           0.98078528040323044913f, 1.0f, 0.98078528040323044913f,
                           0.92387953251128675613f, 0.83146961230254523708f,
                           0.70710678118654752440f, 0.55557023301960222474f,
                           0.38268343236508977173f, 0.19509032201612826785f};
  const float cc = b ? c[k] : 1.0f, ss = b ? -s[k] : 0.0f;
  return make_float4(cc, cc, ss, ss);
}

struct FullrateArgs {
  const float2* u;          // [J][u_row]: 2048 history samples, then the block
  long long u_row;
  long long F;              // frames of the block
  long long nseg;           // segments per stream
  const float2* hd;         // [Tr][16][512]: taps' spectrum / N as (re, im)
  const float2* tw1;        // [16][512] exp(-2 pi i b k / 8192) as (c, s)
  const float2* tw2;        // [16][32]  exp(-2 pi i b k / 512)
  const float* theta;
  const float* theta2;
  const long long* blk;
  float* y;                 // [J][F M] Re v, or null
  float2* vph;              // LSMR chain: [J][M][F] v phase-major (no trigger here), or null
  TriggerRec* trig;
  unsigned long long* count;
  long long cap;
  float k_sigma;
  int lag;                  // frames between a block's first output and its first frame
  int jj0;                  // first launch stream of this launch (grids of at most 65535)
  int P, Tr, pol0, npol;
};

// Trigger compaction of one output of each lane (hit: above threshold).
__device__ __forceinline__ void emit(bool hit, float e2, long long n, int j, int tr,
                                     const FullrateArgs& a) {
  const unsigned mask = __ballot_sync(0xffffffffu, hit);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long at = 0;
  if (lane == leader) at = atomicAdd(a.count, (unsigned long long)__popc(mask));
  at = __shfl_sync(0xffffffffu, at, leader);
  if (hit) {
    const unsigned long long idx = at + __popc(mask & ((1u << lane) - 1u));
    if ((long long)idx < a.cap) {
      TriggerRec rec;
      rec.n = n;
      rec.pol = j % a.P;
      rec.tec = tr;
      rec.beam = j / (a.P * a.Tr);
      rec.stream = j;
      rec.env = sqrtf(e2);
      rec.sigma = a.theta[j] / a.k_sigma;
      a.trig[idx] = rec;
    }
  }
}

// One block: segments 2 x and 2 x + 1 of stream y (the second may lie past the
// block's end: it then reads zeros and emits nothing).  OUT: 0 trigger, 1
// trigger and Re v, 2 (LSMR chain) v stored phase-major, no trigger.
template <int OUT>
__global__ void __launch_bounds__(FR_NT, 1) k_fullrate(const __grid_constant__ FullrateArgs a) {
  extern __shared__ float4 xs[];
  const int t = threadIdx.x;
  const int j = (int)sel_stream(a.jj0 + blockIdx.y, a.P, a.pol0, a.npol);
  const int tr = (j / a.P) % a.Tr;
  const long long base = (long long)blockIdx.x * (2 * FR_V);   // row index of segment a's sample 0
  const float2* __restrict__ ua = a.u + (long long)j * a.u_row + base + t;
  const long long rem = a.u_row - base - t;                     // row samples left from ua
  CP v[16];

  // ---- forward pass 1: blocks of 8192, stride 512 (thread t: position t + 512 r)
  if (rem >= FR_V + FR_N) {                                     // both segments inside the row
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 x0 = __ldg(ua + 512 * r), x1 = __ldg(ua + FR_V + 512 * r);
      v[r] = CP{make_float2(x0.x, x1.x), make_float2(x0.y, x1.y)};
    }
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 z = make_float2(0.f, 0.f);
      const float2 x0 = 512 * r < rem ? __ldg(ua + 512 * r) : z;
      const float2 x1 = FR_V + 512 * r < rem ? __ldg(ua + FR_V + 512 * r) : z;
      v[r] = CP{make_float2(x0.x, x1.x), make_float2(x0.y, x1.y)};
    }
  }
  dft16<-1>(v);
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], wide(__ldg(a.tw1 + k * 512 + t)));
#pragma unroll
  for (int k = 0; k < 16; ++k)
    xs[frp(t + 512 * k)] = make_float4(v[k].re.x, v[k].re.y, v[k].im.x, v[k].im.y);
  __syncthreads();
  // ---- pass 2: blocks of 512, stride 32
  const int b2 = t & 31, o2 = (t >> 5) * 512 + b2;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float4 q = xs[frp(o2 + 32 * r)];
    v[r] = CP{make_float2(q.x, q.y), make_float2(q.z, q.w)};
  }
  dft16<-1>(v);
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], wide(__ldg(a.tw2 + k * 32 + b2)));
#pragma unroll
  for (int k = 0; k < 16; ++k)
    xs[frp(o2 + 32 * k)] = make_float4(v[k].re.x, v[k].re.y, v[k].im.x, v[k].im.y);
  __syncthreads();
  // ---- pass 3: blocks of 32, stride 2; pass 4: pairs across neighbouring lanes
  const int b3 = t & 1, o3 = (t >> 1) * 32 + b3;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float4 q = xs[frp(o3 + 2 * r)];
    v[r] = CP{make_float2(q.x, q.y), make_float2(q.z, q.w)};
  }
  dft16<-1>(v);
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], w32(k, b3));
  pair_step(v, b3);
  // ---- the product with the taps' spectrum (same order, same for both segments)
  const float2* hd = a.hd + (long long)tr * FR_N + t;
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = cmul(v[k], wide(__ldg(hd + k * FR_NT)));
  // ---- inverse: passes 4, 3, 2, 1 backwards
  pair_step(v, b3);
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmulc(v[k], w32(k, b3));
  dft16<1>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r)
    xs[frp(o3 + 2 * r)] = make_float4(v[r].re.x, v[r].re.y, v[r].im.x, v[r].im.y);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float4 q = xs[frp(o2 + 32 * k)];
    v[k] = CP{make_float2(q.x, q.y), make_float2(q.z, q.w)};
  }
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmulc(v[k], wide(__ldg(a.tw2 + k * 32 + b2)));
  dft16<1>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r)
    xs[frp(o2 + 32 * r)] = make_float4(v[r].re.x, v[r].re.y, v[r].im.x, v[r].im.y);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float4 q = xs[frp(t + 512 * k)];
    v[k] = CP{make_float2(q.x, q.y), make_float2(q.z, q.w)};
  }
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmulc(v[k], wide(__ldg(a.tw1 + k * 512 + t)));
  dft16<1>(v);

  // ---- v[r] = result at position t + 512 r of both segments; positions >= 2048
  // are outputs base + (segment) 6144 + t + 512 (r - 4)
  const long long FM = a.F * kM;
  const long long o0 = base + t - 2048;                      // output index of position t + 512 * 0
  if constexpr (OUT == 2) {
    // output o = i M + p goes to row (j, p), column i.  The two segments are the
    // 12 frames i0 .. i0 + 11 (i0 = base / 1024); they are staged in shared
    // memory as [phase][12 frames] (rows of 13 pairs: the half-warps' stores hit
    // distinct banks) so that each phase's 12 frames leave as 96 contiguous bytes
    // (F is a multiple of 256 under the LSMR inversion: 16-byte aligned stores)
    float2* stg = reinterpret_cast<float2*>(xs);
    constexpr int RS = 13;
    __syncthreads();                                          // xs read by every thread
#pragma unroll
    for (int r = 4; r < 16; ++r) {
      const int ph = t + 512 * ((r - 4) & 1), f = (r - 4) >> 1;
      stg[ph * RS + f] = make_float2(v[r].re.x, v[r].im.x);
      stg[ph * RS + f + 6] = make_float2(v[r].re.y, v[r].im.y);
    }
    __syncthreads();
    const long long i0 = base >> 10;
    const int nf = (int)min(12LL, a.F - i0);                  // frames of the block left
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ph = t + 512 * h;
      float2* dst = a.vph + ((long long)j * kM + ph) * a.F + i0;
      const float2* src = stg + ph * RS;
      if (nf == 12) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float2 x0 = src[2 * q], x1 = src[2 * q + 1];
          reinterpret_cast<float4*>(dst)[q] = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
      } else {
        for (int f = 0; f < nf; ++f) dst[f] = src[f];
      }
    }
    return;
  }
  const long long n_first = (*a.blk * a.F - a.lag) * (long long)kM;
  const float2 th2 = bc(a.theta2[j]);
  float* yj = OUT == 1 ? a.y + (long long)j * FM : nullptr;
  // A block whose 12288 outputs all lie inside the block and at or after the
  // stream's first sample needs no per-value checks: it stores, and leaves
  // unless one of a warp's values crosses the threshold.
  const bool whole = base + 2 * FR_V <= FM && n_first + base >= 0;
  if (whole) {
    bool hit = false;
#pragma unroll
    for (int r = 4; r < 16; ++r) {
      if constexpr (OUT == 1) {
        yj[o0 + 512 * r] = v[r].re.x;
        yj[o0 + 512 * r + FR_V] = v[r].re.y;
      }
      const float2 e2 = fma2(v[r].re, v[r].re, mul2(v[r].im, v[r].im));
      hit = hit || e2.x > th2.x || e2.y > th2.y;
    }
    if (!__any_sync(0xffffffffu, hit)) return;
  }
#pragma unroll
  for (int r = 4; r < 16; ++r) {
    const long long oa = o0 + 512 * r, ob = oa + FR_V;
    const bool ina = oa < FM, inb = ob < FM;
    if (OUT == 1 && !whole) {
      if (ina) yj[oa] = v[r].re.x;
      if (inb) yj[ob] = v[r].re.y;
    }
    const float2 e2 = fma2(v[r].re, v[r].re, mul2(v[r].im, v[r].im));
    const bool ha = ina && e2.x > th2.x && n_first + oa >= 0;
    const bool hb = inb && e2.y > th2.y && n_first + ob >= 0;
    if (__any_sync(0xffffffffu, ha || hb)) {
      emit(ha, e2.x, n_first + oa, j, tr, a);
      emit(hb, e2.y, n_first + ob, j, tr, a);
    }
  }
}

// The last 2048 samples of every series row become the next block's history
// (rows of at least 2048 block samples: the ranges do not overlap).
__global__ void k_fullrate_shift(float2* __restrict__ u, long long u_row, long long FM, int P,
                                 int pol0, int npol, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long j = sel_stream(i / kFrTaps, P, pol0, npol);
  // (rows of at least 2048 block samples: source and destination do not overlap)
  const int l = (int)(i % kFrTaps);
  float2* row = u + j * u_row;
  row[l] = row[FM + l];
}

// ---- set-up, FP64 ----------------------------------------------------------
// E[m] = exp(+2 pi i m / N); H[m] = exp(-2 pi i phi(nu_m)) for m < N/2 (nu_m =
// 100 MHz + m fs / N), 1 above; the FFT twiddle tables (as (c, s) pairs).
__global__ void k_fr_tables(const double* __restrict__ tec, int t, double nu_ref,
                            double2* __restrict__ H, double2* __restrict__ E,
                            float2* __restrict__ tw1, float2* __restrict__ tw2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= FR_N) return;
  double s, c;
  sincospi(2.0 * (double)i / FR_N, &s, &c);
  E[i] = make_double2(c, s);
  if (i < FR_N / 2) {
    const double nu = kNu0 + (double)i * (kFs / FR_N);
    const double a = kKappa * tec[t] * kTecu / kC;
    const double dnu = nu - nu_ref;
    const double cyc = a * (dnu * dnu) / (nu * nu_ref * nu_ref);
    const double r = cyc - rint(cyc);
    sincospi(2.0 * r, &s, &c);
    H[i] = make_double2(c, -s);
  } else {
    H[i] = make_double2(1.0, 0.0);
  }
  {
    const int k = i / 512, b = i % 512;        // i < 16 * 512 = N
    const int e = (b * k) % FR_N;
    sincospi(2.0 * (double)e / FR_N, &s, &c);
    tw1[i] = make_float2((float)c, (float)-s);
  }
  if (i < 16 * 32) {
    const int k = i / 32, b = i % 32;
    const int e = (b * k) % 512;
    sincospi(2.0 * (double)e / 512.0, &s, &c);
    tw2[i] = make_float2((float)c, (float)-s);
  }
}

// h[l] = w(l - D) (1/N) sum_m H[m] E[(m (l - D)) mod N], l < 2048, D = 1024;
// w(d) = 1 for |d| <= 768, (1 + cos(pi (|d| - 768) / 256)) / 2 beyond.
__global__ void k_fr_taps(const double2* __restrict__ H, const double2* __restrict__ E,
                          double2* __restrict__ h) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= kFrTaps) return;
  const int d = l - kFrDelay;
  const int dm = ((d % FR_N) + FR_N) % FR_N;
  double re = 0.0, im = 0.0;
  int m = 0;
  for (int q = 0; q < FR_N; ++q) {
    const double2 a = H[q], e = E[m];
    re = fma(a.x, e.x, fma(-a.y, e.y, re));
    im = fma(a.x, e.y, fma(a.y, e.x, im));
    m += dm;
    if (m >= FR_N) m -= FR_N;
  }
  const double half = 0.5 * kFrFlat, ramp = 0.5 * (kFrTaps - kFrFlat);
  const double ad = fabs((double)d);
  const double w = ad <= half ? 1.0 : 0.5 * (1.0 + cospi(fmin(ad - half, ramp) / ramp));
  h[l] = make_double2(re * w / FR_N, im * w / FR_N);
}

// The taps' spectrum / N in the kernel's order: entry (k, t) is frequency
// K = k1 + 16 k2 + 256 k + 4096 b (t = 2 (16 k1 + k2) + b).
__global__ void k_fr_spectrum(const double2* __restrict__ h, const double2* __restrict__ E,
                              float2* __restrict__ hd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= FR_N) return;
  const int k = i / FR_NT, t = i % FR_NT, B = t >> 1, b = t & 1;
  const int K = (B >> 4) + 16 * (B & 15) + 256 * k + 4096 * b;
  double re = 0.0, im = 0.0;
  int m = 0;
  for (int l = 0; l < kFrTaps; ++l) {
    const double2 a = h[l], e = E[m];        // a * conj(e)
    re = fma(a.x, e.x, fma(a.y, e.y, re));
    im = fma(a.y, e.x, fma(-a.x, e.y, im));
    m += K;
    if (m >= FR_N) m -= FR_N;
  }
  hd[i] = make_float2((float)(re / FR_N), (float)(im / FR_N));
}

}  // namespace

long long fullrate_row(const lp_plan& p) { return kFrTaps + p.shape.F * kM; }

size_t fullrate_table_bytes() {
  return sizeof(float2) * (16 * 512 + 16 * 32);
}

cudaError_t init_fullrate_attributes() {
  cudaError_t e = raise_smem_limit((const void*)k_fullrate<0>, FR_SMEM);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)k_fullrate<1>, FR_SMEM);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)k_fullrate<2>, FR_SMEM);
  return e;
}

cudaError_t launch_fullrate_taps(const lp_plan& p, cudaStream_t s) {
  const Buffers& b = p.buf;
  float2* tw2 = b.fr_tw + 16 * 512;
  for (int t = 0; t < p.shape.Tr; ++t) {
    k_fr_tables<<<FR_N / 256, 256, 0, s>>>(b.tec, t, p.nu_ref, b.fr_H, b.fr_E, b.fr_tw, tw2);
    k_fr_taps<<<kFrTaps / 128, 128, 0, s>>>(b.fr_H, b.fr_E, b.fr_h);
    k_fr_spectrum<<<FR_N / 128, 128, 0, s>>>(b.fr_h, b.fr_E, b.fr_hd + (size_t)t * FR_N);
  }
  return cudaGetLastError();
}

cudaError_t launch_fullrate(const lp_plan& p, cudaStream_t s, PolSel ps) {
  const Buffers& b = p.buf;
  const int npol = ps.npol ? ps.npol : p.shape.P;
  FullrateArgs a;
  a.u = b.ufull;
  a.u_row = fullrate_row(p);
  a.F = p.shape.F;
  a.nseg = (p.shape.F * kM + FR_V - 1) / FR_V;
  a.hd = b.fr_hd;
  a.tw1 = b.fr_tw;
  a.tw2 = b.fr_tw + 16 * 512;
  a.theta = b.theta;
  a.theta2 = b.theta2;
  a.blk = b.blk;
  const bool lsmr = p.cfg.inversion == LP_INV_LSMR;
  a.y = lsmr ? nullptr : b.y;
  a.vph = lsmr ? b.xhat : nullptr;
  a.lag = lsmr ? kPrefix : kHist;
  a.trig = b.trig;
  a.count = b.trig_count;
  a.cap = (long long)p.cfg.trigger_cap;
  a.k_sigma = (float)p.cfg.k_sigma;
  a.P = p.shape.P;
  a.Tr = p.shape.Tr;
  a.pol0 = ps.pol0;
  a.npol = npol;
  const long long FM = p.shape.F * kM;
  const int streams = p.shape.J() / p.shape.P * npol;
  for (int jj0 = 0; jj0 < streams; jj0 += 65535) {        // grid y is at most 65535
    a.jj0 = jj0;
    const dim3 grid((unsigned)((a.nseg + 1) / 2), (unsigned)std::min(65535, streams - jj0));
    if (a.vph)
      k_fullrate<2><<<grid, FR_NT, FR_SMEM, s>>>(a);
    else if (a.y)
      k_fullrate<1><<<grid, FR_NT, FR_SMEM, s>>>(a);
    else
      k_fullrate<0><<<grid, FR_NT, FR_SMEM, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_fullrate_shift(const lp_plan& p, cudaStream_t s, PolSel ps) {
  const int npol = ps.npol ? ps.npol : p.shape.P;
  const long long n = (long long)p.shape.J() / p.shape.P * npol * kFrTaps;
  k_fullrate_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      p.buf.ufull, fullrate_row(p), p.shape.F * kM, p.shape.P, ps.pol0, npol, n);
  return cudaGetLastError();
}

}  // namespace lp
