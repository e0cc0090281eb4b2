// Phase tables and the synthesis filter (set-up work, run once per
// lp_set_weights / lp_set_tec / lp_plan_bind_workspace).
//
//  * Beam weights (Sec. 3, first paragraph): w[k,b,s] = exp(-2 pi i cyc),
//    cyc = nu_k (r_s . s_b) / c, up to ~10^3 cycles.  The cycle count is formed
//    in FP64, reduced to r = cyc - rint(cyc) in [-1/2, 1/2] in FP64, and only
//    then rounded to FP32 for sincospif, so the FP32 phase error stays ~1e-7.
//  * De-dispersion (Sec. 3, third paragraph): D[k,t] = exp(-2 pi i phi),
//    phi = A_t (nu_k - nu_ref)^2 / (nu_k nu_ref^2), A_t = kappa STEC_t / c.  The
//    factored form has no cancellation; FP64 keeps phi exact to ~1e-13 cycles.
//  * Synthesis filter: g[n] = (2/M) M^2 h[n], h the Kaiser-windowed sinc
//    (beta = 9, zeros every M samples) normalised to sum 1; the factor 2/M is
//    the analytic inverse FFT's scale folded in.  The same set-up kernel
//    writes the 32 x 32 twiddles exp(+2 pi i p1 l / 1024) of the inverse DFT,
//    each as (cos, cos, sin, sin) so that one 16-byte load gives the
//    broadcast pairs for two frames.
#include "lp_internal.cuh"

namespace lp {
namespace {

// One block of 1024 threads builds the whole 16384-tap filter deterministically.
__global__ void __launch_bounds__(1024) k_prototype(double beta, double* __restrict__ proto,
                                                    double* __restrict__ sums,
                                                    float* __restrict__ g,
                                                    float4* __restrict__ tw1024) {
  constexpr int L = kM * kTaps;
  __shared__ double red_h[1024];
  __shared__ double red_h2[1024];
  const double i0b = bessel_i0_series(beta);
  double sh = 0.0, sh2 = 0.0;
  // the lower half, mirrored: h[L-1-n] = h[n] holds exactly
  for (int n = threadIdx.x; n < L / 2; n += blockDim.x) {
    const double xs = ((double)n - 0.5 * (L - 1)) / kM;
    const double sinc = (xs == 0.0) ? 1.0 : sinpi(xs) / (M_PI * xs);
    const double t = 2.0 * n / (L - 1) - 1.0;
    const double arg = fmax(1.0 - t * t, 0.0);
    const double h = sinc * bessel_i0_series(beta * sqrt(arg)) / i0b;
    proto[n] = h;
    proto[L - 1 - n] = h;
    sh += 2.0 * h;
    sh2 += 2.0 * h * h;
  }
  __syncthreads();
  red_h[threadIdx.x] = sh;
  red_h2[threadIdx.x] = sh2;
  __syncthreads();
  for (int off = 512; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      red_h[threadIdx.x] += red_h[threadIdx.x + off];
      red_h2[threadIdx.x] += red_h2[threadIdx.x + off];
    }
    __syncthreads();
  }
  const double total = red_h[0];
  if (threadIdx.x == 0) {
    sums[0] = total;
    sums[1] = red_h2[0];
  }
  const double scale = 2.0 * kM / total;   // (2/M) * M^2 / sum(h)
  for (int n = threadIdx.x; n < L; n += blockDim.x) g[n] = (float)(proto[n] * scale);
  // twiddles of the 32 x 32 inverse DFT: tw[p1][l] = exp(+2 pi i p1 l / 1024)
  {
    const int i = threadIdx.x;
    double sn, cs;
    sincospi((double)((i >> 5) * (i & 31)) / 512.0, &sn, &cs);
    tw1024[i] = make_float4((float)cs, (float)cs, (float)sn, (float)sn);
  }
}

__global__ void k_weights(const double* __restrict__ enu, const double* __restrict__ dir,
                          int K, int B, int S, int first_bin, float2* __restrict__ w) {
  const long long total = (long long)K * B * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i % S);
    const int b = (int)((i / S) % B);
    const int k = (int)(i / ((long long)S * B));
    const double nu = kNu0 + (double)(first_bin + k) * (kFs / kM);
    const double dot = enu[3 * s] * dir[3 * b] + enu[3 * s + 1] * dir[3 * b + 1] +
                       enu[3 * s + 2] * dir[3 * b + 2];
    const double cyc = nu * dot / kC;
    const double r = cyc - rint(cyc);
    float sn, cs;
    sincospif(2.0f * (float)r, &sn, &cs);
    w[i] = make_float2(cs, -sn);           // exp(-2 pi i cyc)
  }
}

__global__ void k_dedisp(const double* __restrict__ tec, int K, int Tr, int first_bin,
                         double nu_ref, int unit, float2* __restrict__ dd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K * Tr) return;
  if (unit) {                              // full-rate mode: the phase is applied later
    dd[i] = make_float2(1.f, 0.f);
    return;
  }
  const int t = i % Tr;
  const int k = i / Tr;
  const double nu = kNu0 + (double)(first_bin + k) * (kFs / kM);
  const double a = kKappa * tec[t] * kTecu / kC;
  const double dnu = nu - nu_ref;
  const double cyc = a * (dnu * dnu) / (nu * nu_ref * nu_ref);
  const double r = cyc - rint(cyc);
  float sn, cs;
  sincospif(2.0f * (float)r, &sn, &cs);
  dd[i] = make_float2(cs, -sn);            // exp(-2 pi i phi)
}

}  // namespace

cudaError_t launch_prototype(const lp_plan& p, cudaStream_t s) {
  k_prototype<<<1, 1024, 0, s>>>(p.cfg.kaiser_beta, p.buf.proto, p.buf.filter_sums, p.buf.g,
                                 p.buf.tw1024);
  return cudaGetLastError();
}

cudaError_t launch_weights(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const long long total = (long long)sh.K * sh.B * sh.S;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  k_weights<<<blocks, 256, 0, s>>>(p.buf.station_enu, p.buf.beam_dir, sh.K, sh.B, sh.S,
                                   p.cfg.first_bin, p.buf.w32);
  return cudaGetLastError();
}

cudaError_t launch_dedisp(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const int n = sh.K * sh.Tr;
  k_dedisp<<<(n + 255) / 256, 256, 0, s>>>(p.buf.tec, sh.K, sh.Tr, p.cfg.first_bin, p.nu_ref,
                                            p.cfg.fullrate_dedisp ? 1 : 0, p.buf.dd);
  return cudaGetLastError();
}

}  // namespace lp
