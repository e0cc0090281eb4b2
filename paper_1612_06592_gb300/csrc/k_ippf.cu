// Inverse polyphase filter bank + envelope trigger (Sec. 2 last paragraph,
// Sec. 3 second paragraph, Fig. 1), and the per-block noise level.
//
// k_ippf: one thread block owns one stream j and a run of output frames
// [m0, m1).  It walks frames m0-16 .. m1-1 in batches of 8 (one per warp):
//   1. the batch's beam bins (8 frames x K bins, frames contiguous per bin
//      row) are copied into a zero-padded 512-bin stage with cp.async while
//      the previous batch's FIR runs;
//   2. each warp takes the 1024-point inverse DFT of one frame,
//        z[p] = sum_k c[k] exp(+2 pi i k p / 1024),  c nonzero only in the
//      selected bins (< 512), as 32 x 32: a register-resident 32-point DFT
//      over k = 32 k1 + lane (upper half of the inputs zero), the twiddle
//      exp(2 pi i lane p1 / 1024), a transpose through shared memory and a
//      second 32-point DFT; the result lands in a 24-frame ring in shared
//      memory (three groups of 8 frames, addressed by group base pointers);
//   3. every thread owns 4 output phases p and computes, for the 8 new frames,
//        u_m[p] = sum_{t<16} g[t M + p] z_{m-t}[p]     (g holds the 2/M scale),
//      y = Re u (optionally stored), |u|^2 against theta^2; warps vote and
//      compact the (rare) samples above threshold into the trigger list.
// The first 16 frames of a run only fill the FIR history (16/frames_per_cta
// of extra inverse DFTs).  FP32 throughout.
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int NT = 256;            // threads per block
constexpr int NW = NT / 32;        // warps = frames per batch
constexpr int RING = 24;           // 3 groups of 8 frames: 15 history + 8 new fit
constexpr int SK = 516;            // stage row: 512 bins + pad, 2*SK = 8 mod 32 banks
constexpr int PPT = kM / NT;       // output phases per thread

__host__ __device__ constexpr int br5(int i) {
  return ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
}

// cos(2 pi e / 32) for any integer e.
__host__ __device__ constexpr float cos32v(int e) {
  constexpr float q[9] = {1.0f,
                          0.98078528040323044913f,
                          0.92387953251128675613f,
                          0.83146961230254523708f,
                          0.70710678118654752440f,
                          0.55557023301960222474f,
                          0.38268343236508977173f,
                          0.19509032201612826785f,
                          0.0f};
  e &= 31;
  return e <= 8 ? q[e] : e <= 16 ? -q[16 - e] : e <= 24 ? -q[e - 16] : q[32 - e];
}
__host__ __device__ constexpr float sin32v(int e) { return cos32v(e - 8); }

// d * exp(+2 pi i E / 32), with the trivial rotations spelled out.
template <int E>
__device__ __forceinline__ float2 rot32(float2 d) {
  constexpr int e = E & 31;
  if constexpr (e == 0) {
    return d;
  } else if constexpr (e == 8) {
    return make_float2(-d.y, d.x);
  } else if constexpr (e == 16) {
    return make_float2(-d.x, -d.y);
  } else if constexpr (e == 24) {
    return make_float2(d.y, -d.x);
  } else if constexpr (e == 4) {
    constexpr float r = 0.70710678118654752440f;
    return make_float2((d.x - d.y) * r, (d.x + d.y) * r);
  } else if constexpr (e == 12) {
    constexpr float r = 0.70710678118654752440f;
    return make_float2(-(d.x + d.y) * r, (d.x - d.y) * r);
  } else {
    constexpr float c = cos32v(e), s = sin32v(e);
    return make_float2(fmaf(d.x, c, -d.y * s), fmaf(d.x, s, d.y * c));
  }
}

#define LP_ROT_CASE(n) case n: return rot32<n>(d);
__device__ __forceinline__ float2 rot32_rt(float2 d, int e) {
  switch (e & 31) {
    LP_ROT_CASE(0) LP_ROT_CASE(1) LP_ROT_CASE(2) LP_ROT_CASE(3) LP_ROT_CASE(4)
    LP_ROT_CASE(5) LP_ROT_CASE(6) LP_ROT_CASE(7) LP_ROT_CASE(8) LP_ROT_CASE(9)
    LP_ROT_CASE(10) LP_ROT_CASE(11) LP_ROT_CASE(12) LP_ROT_CASE(13) LP_ROT_CASE(14)
    LP_ROT_CASE(15) LP_ROT_CASE(16) LP_ROT_CASE(17) LP_ROT_CASE(18) LP_ROT_CASE(19)
    LP_ROT_CASE(20) LP_ROT_CASE(21) LP_ROT_CASE(22) LP_ROT_CASE(23) LP_ROT_CASE(24)
    LP_ROT_CASE(25) LP_ROT_CASE(26) LP_ROT_CASE(27) LP_ROT_CASE(28) LP_ROT_CASE(29)
    LP_ROT_CASE(30) LP_ROT_CASE(31)
  }
  return d;
}
#undef LP_ROT_CASE

// Radix-2 decimation-in-frequency stages of a 32-point DFT with kernel
// exp(+2 pi i k n / 32), from half-size SPAN0 down to 1.  Natural-order
// input, bit-reversed output: v[i] = X[br5(i)].
template <int SPAN0>
__device__ __forceinline__ void dif32_from(float2 (&v)[32]) {
#pragma unroll
  for (int span = SPAN0; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < 32; start += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 a = v[start + j], b = v[start + j + span];
        v[start + j] = make_float2(a.x + b.x, a.y + b.y);
        v[start + j + span] = rot32_rt(make_float2(a.x - b.x, a.y - b.y), j * (16 / span));
      }
    }
  }
}

// 32-point DFT whose inputs 16..31 are zero: the first stage is a rotation.
__device__ __forceinline__ void dft32_halfzero(float2 (&v)[32]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j + 16] = rot32_rt(v[j], j);
  dif32_from<8>(v);
}

__device__ __forceinline__ void dft32(float2 (&v)[32]) { dif32_from<16>(v); }

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Stage the beam bins of CTA frames r0 .. r0+7 into stage[f][first_bin + k]
// (asynchronous copies; frames outside the run are zeroed).
__device__ __forceinline__ void stage_batch(float2* stage, const float2* __restrict__ brow, int K,
                                            int first_bin, long long row, long long m0, int r0,
                                            int nfr, int tid) {
  for (int e = tid; e < K * NW; e += NT) {
    const int k = e >> 3, f = e & 7;
    float2* dst = stage + f * SK + first_bin + k;
    if (r0 + f < nfr && m0 + r0 + f < row)
      cp_async8(dst, brow + (long long)k * row + r0 + f);
    else
      *dst = make_float2(0.f, 0.f);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(NT, 1) k_ippf(
    const float2* __restrict__ beams, int K, int first_bin, long long F, long long row,
    int frames_per_cta, const float* __restrict__ g, const float2* __restrict__ tw,
    const float* __restrict__ theta, const float* __restrict__ theta2, float k_sigma,
    long long n_first, int frame_min_trigger, int P, int Tr, float* __restrict__ y,
    TriggerRec* __restrict__ trig, unsigned long long* __restrict__ trig_count,
    long long trig_cap) {
  extern __shared__ float2 smem[];
  float2* ring = smem;                      // [3 groups][8 frames][1024]
  float2* stage = ring + RING * kM;         // [8 frames][SK], bins 0..511

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j = blockIdx.y;
  const long long m0 = (long long)blockIdx.x * frames_per_cta;
  const long long m1 = min((long long)(m0 + frames_per_cta), (long long)(F));
  const int nout = (int)(m1 - m0);
  const int nfr = nout + kPrefix;          // frames run through the inverse DFT
  const int nbatch = (nfr + NW - 1) / NW;
  const float2* brow = beams + (long long)j * K * row + m0;   // position of frame m0-16

  // bins outside the selection stay zero for the whole run
  for (int i = tid; i < NW * SK; i += NT) stage[i] = make_float2(0.f, 0.f);
  __syncthreads();
  stage_batch(stage, brow, K, first_bin, row, m0, 0, nfr, tid);

  float gr[PPT][kTaps];
#pragma unroll
  for (int q = 0; q < PPT; ++q)
#pragma unroll
    for (int t = 0; t < kTaps; ++t) gr[q][t] = g[t * kM + tid + q * NT];

  const float th2 = theta2[j];
  float* yj = y ? y + (long long)j * F * kM : nullptr;

  for (int bi = 0; bi < nbatch; ++bi) {
    const int r0 = bi * NW;
    const int gi = bi % 3;
    cp_async_wait_all();
    __syncthreads();   // stage of this batch landed; previous FIR is done with the ring
    // inverse DFT of frame r0+warp into ring group gi, slot warp
    {
      float2* slot = ring + (gi * NW + warp) * kM;
      const float2* st = stage + warp * SK + lane;
      float2 v[32];
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) v[k1] = st[32 * k1];
      dft32_halfzero(v);                  // v[i] = T[p1 = br5(i)]
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int p1 = br5(i);
        const float2 t = __ldg(tw + p1 * 32 + lane);
        const float2 a = v[i];
        slot[lane * 32 + (p1 ^ lane)] =
            make_float2(fmaf(a.x, t.x, -a.y * t.y), fmaf(a.x, t.y, a.y * t.x));
      }
      __syncwarp();
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) v[k2] = slot[k2 * 32 + (lane ^ k2)];
      __syncwarp();
      dft32(v);                           // v[i] = z[lane + 32 br5(i)]
#pragma unroll
      for (int i = 0; i < 32; ++i) slot[lane + 32 * br5(i)] = v[i];
    }
    __syncthreads();   // ring group gi written; stage consumed
    if (bi + 1 < nbatch) stage_batch(stage, brow, K, first_bin, row, m0, r0 + NW, nfr, tid);
    if (r0 + NW <= kPrefix) continue;     // history-only batch (uniform)

    // synthesis FIR + envelope threshold for frames r0 .. r0+7.  History frames
    // r0-15 .. r0-9 sit in group gi+1 (slots 1..7), r0-8 .. r0-1 in group gi+2.
    const float2* ga = ring + (((gi + 1) % 3) * NW) * kM + tid;
    const float2* gb = ring + (((gi + 2) % 3) * NW) * kM + tid;
    const float2* gc = ring + (gi * NW) * kM + tid;
    unsigned vmask = 0;                    // frames of the batch that are output frames
#pragma unroll
    for (int f = 0; f < NW; ++f) {
      const int r = r0 + f;
      const long long m = m0 - kPrefix + r;
      if (r >= kPrefix && r < nfr && m >= frame_min_trigger) vmask |= 1u << f;
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      float2 zw[kHist + NW];
#pragma unroll
      for (int w = 0; w < 7; ++w) zw[w] = ga[(w + 1) * kM + q * NT];
#pragma unroll
      for (int w = 0; w < NW; ++w) zw[7 + w] = gb[w * kM + q * NT];
#pragma unroll
      for (int w = 0; w < NW; ++w) zw[15 + w] = gc[w * kM + q * NT];
      float e2v[NW];
      unsigned hm = 0;
#pragma unroll
      for (int f = 0; f < NW; ++f) {
        float ur = 0.f, ui = 0.f;
#pragma unroll
        for (int t = 0; t < kTaps; ++t) {
          ur = fmaf(gr[q][t], zw[f + kHist - t].x, ur);
          ui = fmaf(gr[q][t], zw[f + kHist - t].y, ui);
        }
        if (yj) {
          const int r = r0 + f;
          if (r >= kPrefix && r < nfr) yj[(m0 - kPrefix + r) * kM + tid + q * NT] = ur;
        }
        e2v[f] = fmaf(ur, ur, ui * ui);
        hm |= (e2v[f] > th2 ? 1u : 0u) << f;
      }
      hm &= vmask;
      if (__any_sync(0xffffffffu, hm != 0)) {   // rare: compact this phase's hits
        const int p = tid + q * NT;
#pragma unroll
        for (int f = 0; f < NW; ++f) {
          const bool hit = (hm >> f) & 1u;
          const unsigned mask = __ballot_sync(0xffffffffu, hit);
          if (!mask) continue;
          const int leader = __ffs(mask) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(trig_count, (unsigned long long)__popc(mask));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (hit) {
            const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
            if ((long long)idx < trig_cap) {
              TriggerRec rec;
              rec.n = n_first + (m0 - kPrefix + r0 + f) * kM + p;
              rec.pol = j % P;
              rec.tec = (j / P) % Tr;
              rec.beam = j / (P * Tr);
              rec.stream = j;
              rec.env = sqrtf(e2v[f]);
              rec.sigma = theta[j] / k_sigma;
              trig[idx] = rec;
            }
          }
        }
      }
    }
  }
}

// Block noise power and running sigma (one block of 256 threads per stream).
// Pi = (2 G2 / M^3) * (1/F) * sum_{m,k} |beam|^2, G2 = sum g^2 = M^4 sum h^2 / (sum h)^2;
// s2 = Pi (first block) or (1 - alpha) s2 + alpha Pi; theta = k_sigma sqrt(s2).
__global__ void __launch_bounds__(256) k_sigma(const float* __restrict__ part, int n_per_stream,
                                               const double* __restrict__ sums, long long F,
                                               double alpha, double k_sigma, int first_block,
                                               double* __restrict__ sigma2,
                                               float* __restrict__ theta,
                                               float* __restrict__ theta2) {
  __shared__ double red[256];
  const int j = blockIdx.x;
  const float* pj = part + (long long)j * n_per_stream;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n_per_stream; i += 256) acc += (double)pj[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = (double)kM;
    const double g2 = m * m * m * m * sums[1] / (sums[0] * sums[0]);
    const double pi = 2.0 * g2 / (m * m * m) * red[0] / (double)F;
    const double s2 = first_block ? pi : (1.0 - alpha) * sigma2[j] + alpha * pi;
    sigma2[j] = s2;
    const double th = k_sigma * sqrt(s2);
    theta[j] = (float)th;
    theta2[j] = (float)(th * th);
  }
}

// Carry the last 16 frames of every (stream, bin) row into the row prefix.
__global__ void k_history_shift(float2* __restrict__ beams, long long rows, long long F,
                                long long row) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows * kPrefix) return;
  const long long r = i / kPrefix;
  const int f = (int)(i % kPrefix);
  beams[r * row + f] = beams[r * row + F + f];
}

size_t ippf_smem_bytes() { return (size_t)(RING * kM + NW * SK) * sizeof(float2); }

}  // namespace

int ippf_default_frames_per_cta(const Shape& sh) {
  // enough blocks for several waves on 152 SMs, few history frames per block
  long long fpc = 512;
  while (fpc > 64 && (long long)sh.J() * ((sh.F + fpc - 1) / fpc) < 152LL * 8) fpc /= 2;
  return (int)fpc;
}

cudaError_t launch_ippf(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const int fpc = p.frames_per_cta;
  const dim3 grid((unsigned)((sh.F + fpc - 1) / fpc), (unsigned)sh.J());
  const size_t smem = ippf_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_ippf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long n_first = (p.block_index * sh.F - kHist) * (long long)kM;
  // samples n < 0 (frames m < 15 of the first block) never trigger
  const int frame_min_trigger = p.block_index == 0 ? kHist : 0;
  k_ippf<<<grid, NT, smem, s>>>(p.buf.beams, sh.K, p.cfg.first_bin, sh.F, sh.row(), fpc, p.buf.g,
                                p.buf.tw1024, p.buf.theta, p.buf.theta2, (float)p.cfg.k_sigma,
                                n_first, frame_min_trigger, sh.P, sh.Tr, p.buf.y, p.buf.trig,
                                p.buf.trig_count, p.cfg.trigger_cap);
  return cudaGetLastError();
}

cudaError_t launch_sigma(const lp_plan& p, bool first_block, cudaStream_t s) {
  const auto& sh = p.shape;
  k_sigma<<<sh.J(), 256, 0, s>>>(p.buf.power_part, sh.K * p.n_ftiles_bf, p.buf.filter_sums, sh.F,
                                 p.cfg.sigma_alpha, p.cfg.k_sigma, first_block ? 1 : 0,
                                 p.buf.sigma2, p.buf.theta, p.buf.theta2);
  return cudaGetLastError();
}

cudaError_t launch_history_shift(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const long long rows = (long long)sh.J() * sh.K;
  const long long n = rows * kPrefix;
  k_history_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.buf.beams, rows, sh.F, sh.row());
  return cudaGetLastError();
}

}  // namespace lp
