// Inverse polyphase filter bank + envelope trigger (Sec. 2 last paragraph,
// Sec. 3 second paragraph, Fig. 1), and the per-block noise level.
//
// k_ippf: one thread block (16 warps) owns one stream j and a run of output
// frames [m0, m1).  It walks frames m0-16 .. m1-1 in batches of 8:
//   1. the batch's beam bins (8 frames x K bins, frames contiguous per bin
//      row) are copied into a zero-padded 512-bin stage with cp.async while
//      the previous batch's FIR runs;
//   2. two warps take the 1024-point inverse DFT of one frame,
//        z[p] = sum_k c[k] exp(+2 pi i k p / 1024),  c nonzero only in the
//      selected bins (< 512), as 32 x 32: a 32-point DFT over k = 32 k1 + lane
//      whose inputs 16..31 are zero, the twiddle exp(2 pi i lane p1 / 1024), a
//      transpose through shared memory and a second 32-point DFT.  Each
//      32-point DFT is split between the two warps by output parity (two
//      16-point DFTs of the folded inputs).  z lands in a 24-frame ring in
//      shared memory (three groups of 8 frames, addressed by group pointers);
//   3. every thread owns the output phases p = t and p' = 1023 - t, which share
//      one set of 16 taps (g[n] = g[L-1-n] gives g_t[p'] = g_{15-t}[p]), and
//      computes for the 8 new frames
//        u_m[p] = sum_{t<16} g[t M + p] z_{m-t}[p]     (g holds the 2/M scale),
//      y = Re u (optionally stored) and |u|^2 against theta^2; the warps vote
//      and compact the (rare) samples above threshold into the trigger list.
// The first 16 frames of a run only fill the FIR history (16/frames_per_cta
// of extra inverse DFTs).  FP32 throughout.
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int NT = 512;            // threads per block
constexpr int NW = NT / 32;        // 16 warps
constexpr int FB = 8;              // frames per batch (two warps per frame)
constexpr int RING = 24;           // 3 groups of 8 frames: 15 history + 8 new fit
constexpr int SK = 516;            // stage row: 512 bins + pad, 2*SK = 8 mod 32 banks

__host__ __device__ constexpr int br4(int i) {
  return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3);
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

__device__ __forceinline__ float2 badd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 bsub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// 16-point DFT with kernel exp(+2 pi i k n / 16), radix-2 decimation in
// frequency: natural-order input, bit-reversed output v[i] = X[br4(i)].
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int span = 8; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < 16; start += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 a = v[start + j], b = v[start + j + span];
        v[start + j] = badd(a, b);
        // exp(+2 pi i j / (2 span)) = exp(+2 pi i (16 j / span) / 32)
        v[start + j + span] = rot32_rt(bsub(a, b), j * (16 / span));
      }
    }
  }
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
// Barrier for the two warps (64 threads) of one frame.
__device__ __forceinline__ void pair_sync(int id) {
  asm volatile("bar.sync %0, 64;\n" ::"r"(id) : "memory");
}

// Staging of the beam bins of CTA frames r0 .. r0+7 into stage[f][first_bin + k]
// (asynchronous copies).  Thread t always copies frame f = t & 7 of bins
// k = t/8 + 64 i, so its source and destination advance by constants.
struct Stager {
  const float2* src;      // bin t/8, frame t&7 of CTA frame 0
  float2* dst;            // stage[t&7][first_bin + t/8]
  long long src_step;     // 64 rows
  int n;                  // bins this thread copies
  int f;                  // its frame within the batch
};

__device__ __forceinline__ Stager make_stager(float2* stage, const float2* brow, int K,
                                              int first_bin, long long row, int tid) {
  Stager st;
  st.f = tid & 7;
  const int k0 = tid >> 3;
  st.src = brow + (long long)k0 * row + st.f;
  st.dst = stage + st.f * SK + first_bin + k0;
  st.src_step = 64 * row;
  st.n = k0 < K ? (K - k0 + 63) / 64 : 0;
  return st;
}

__device__ __forceinline__ void stage_batch(const Stager& st, long long m0, long long row, int r0,
                                            int nfr) {
  const bool live = r0 + st.f < nfr && m0 + r0 + st.f < row;
  const float2* src = st.src + r0;
#pragma unroll 4
  for (int i = 0; i < st.n; ++i) {
    if (live)
      cp_async8(st.dst + 64 * i, src + i * st.src_step);
    else
      st.dst[64 * i] = make_float2(0.f, 0.f);
  }
  cp_async_commit();
}

// Packed FP32 pairs (one instruction for both components of a complex value).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 t) {
  return make_float2(fmaf(a.x, t.x, -a.y * t.y), fmaf(a.x, t.y, a.y * t.x));
}

// One warp's half of the 32 x 32 inverse DFT of a frame: HALF = 0 computes
// the even outputs of both 32-point stages, HALF = 1 the odd ones.
template <int HALF>
__device__ __forceinline__ void frame_dft(float2* slot, const float2* st,
                                          const float2* __restrict__ tw, int lane, int pair_id) {
  float2 v[16];
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = st[32 * k1];
  if constexpr (HALF) {
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = rot32_rt(v[k1], k1);
  }
  dft16(v);                               // v[i] = T[p1 = 2 br4(i) + HALF]
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int p1 = 2 * br4(i) + HALF;
    slot[lane * 32 + (p1 ^ lane)] = cmul(v[i], __ldg(tw + p1 * 32 + lane));
  }
  pair_sync(pair_id);
  float2 u[16];
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const float2 a = slot[k2 * 32 + (lane ^ k2)];
    const float2 b = slot[(k2 + 16) * 32 + (lane ^ (k2 + 16))];
    if constexpr (HALF)
      u[k2] = rot32_rt(bsub(a, b), k2);
    else
      u[k2] = badd(a, b);
  }
  pair_sync(pair_id);                     // both warps read the slot before it is overwritten
  dft16(u);                               // u[i] = z[lane + 32 (2 br4(i) + HALF)]
#pragma unroll
  for (int i = 0; i < 16; ++i) slot[lane + 32 * (2 * br4(i) + HALF)] = u[i];
}

// FIR over the batch for one output phase; TAP_REV selects g_{15-t} (the
// mirror phase).  Fills e2v = |u|^2 and returns its maximum over the batch.
template <bool TAP_REV, bool WRITE_Y>
__device__ __forceinline__ float fir_phase(const float2 (&gq)[kTaps], const float2* ga,
                                           const float2* gb, const float2* gc, int off,
                                           float* yrow, unsigned ymask, float (&e2v)[FB]) {
  float2 zw[kHist + FB];
#pragma unroll
  for (int w = 0; w < 7; ++w) zw[w] = ga[(w + 1) * kM + off];
#pragma unroll
  for (int w = 0; w < FB; ++w) zw[7 + w] = gb[w * kM + off];
#pragma unroll
  for (int w = 0; w < FB; ++w) zw[15 + w] = gc[w * kM + off];
  float emax = 0.f;
#pragma unroll
  for (int f = 0; f < FB; ++f) {
    float2 u = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < kTaps; ++t)   // both components per instruction, tap (g, g)
      u = __ffma2_rn(TAP_REV ? gq[kTaps - 1 - t] : gq[t], zw[f + kHist - t], u);
    if constexpr (WRITE_Y) {
      if ((ymask >> f) & 1u) yrow[f * kM + off] = u.x;
    }
    e2v[f] = fmaf(u.x, u.x, u.y * u.y);
    emax = fmaxf(emax, e2v[f]);          // frames outside the run are filtered later
  }
  return emax;
}

template <bool WRITE_Y>
__device__ __forceinline__ void fir_batch(const float2 (&gq)[kTaps], const float2* ga,
                                          const float2* gb, const float2* gc, int tid, int lane,
                                          float* yrow, unsigned ymask, unsigned vmask, float th2,
                                          long long n_row0, int j, int P, int Tr, float sig,
                                          TriggerRec* trig, unsigned long long* trig_count,
                                          long long trig_cap);

__device__ __forceinline__ void emit_triggers(const float (&e2v)[FB], unsigned vmask, float th2,
                                              int lane, int p, long long n_row0, int j, int P,
                                              int Tr, float sig, TriggerRec* trig,
                                              unsigned long long* trig_count, long long trig_cap) {
#pragma unroll
  for (int f = 0; f < FB; ++f) {
    const bool hit = ((vmask >> f) & 1u) && e2v[f] > th2;
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
        rec.n = n_row0 + (long long)f * kM + p;
        rec.pol = j % P;
        rec.tec = (j / P) % Tr;
        rec.beam = j / (P * Tr);
        rec.stream = j;
        rec.env = sqrtf(e2v[f]);
        rec.sigma = sig;
        trig[idx] = rec;
      }
    }
  }
}

template <bool WRITE_Y>
__device__ __forceinline__ void fir_batch(const float2 (&gq)[kTaps], const float2* ga,
                                          const float2* gb, const float2* gc, int tid, int lane,
                                          float* yrow, unsigned ymask, unsigned vmask, float th2,
                                          long long n_row0, int j, int P, int Tr, float sig,
                                          TriggerRec* trig, unsigned long long* trig_count,
                                          long long trig_cap) {
  float e2v[FB];
  {
    const float em = fir_phase<false, WRITE_Y>(gq, ga, gb, gc, tid, yrow, ymask, e2v);
    if (__any_sync(0xffffffffu, em > th2))
      emit_triggers(e2v, vmask, th2, lane, tid, n_row0, j, P, Tr, sig, trig, trig_count,
                    trig_cap);
  }
  {
    const int p = kM - 1 - tid;
    const float em = fir_phase<true, WRITE_Y>(gq, ga, gb, gc, p, yrow, ymask, e2v);
    if (__any_sync(0xffffffffu, em > th2))
      emit_triggers(e2v, vmask, th2, lane, p, n_row0, j, P, Tr, sig, trig, trig_count,
                    trig_cap);
  }
}

__global__ void __launch_bounds__(NT, 1) k_ippf(
    const float2* __restrict__ beams, int K, int first_bin, long long F, long long row,
    int frames_per_cta, const float* __restrict__ g, const float2* __restrict__ tw,
    const float* __restrict__ theta, const float* __restrict__ theta2, float k_sigma,
    const long long* __restrict__ blk, long long F_total, long long f_base, int P, int Tr,
    float* __restrict__ y,
    TriggerRec* __restrict__ trig, unsigned long long* __restrict__ trig_count,
    long long trig_cap) {
  extern __shared__ float2 smem[];
  float2* ring = smem;                      // [3 groups][8 frames][1024]
  float2* stage = ring + RING * kM;         // [8 frames][SK], bins 0..511

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int fr = warp >> 1, half = warp & 1;   // frame of the batch, output parity
  const int j = blockIdx.y;
  const long long m0 = (long long)blockIdx.x * frames_per_cta;
  const long long m1 = min((long long)(m0 + frames_per_cta), (long long)(F));
  const int nout = (int)(m1 - m0);
  const int nfr = nout + kPrefix;          // frames run through the inverse DFT
  const int nbatch = (nfr + FB - 1) / FB;
  const float2* brow = beams + (long long)j * K * row + m0;   // position of frame m0-16

  // bins outside the selection stay zero for the whole run
  for (int i = tid; i < FB * SK; i += NT) stage[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const Stager stg = make_stager(stage, brow, K, first_bin, row, tid);
  stage_batch(stg, m0, row, 0, nfr);

  float2 gq[kTaps];                        // taps (g, g) of phase tid (mirrored for 1023 - tid)
#pragma unroll
  for (int t = 0; t < kTaps; ++t) {
    const float gt = g[t * kM + tid];
    gq[t] = make_float2(gt, gt);
  }
  const float th2 = theta2[j];
  // this launch covers block frames [f_base, f_base + F) (one chunk, or the block)
  float* yj = y ? y + ((long long)j * F_total + f_base) * kM : nullptr;
  // block i of the stream starts at sample (i F - 15) M; samples n < 0 (frames
  // m < 15 of the first block) never trigger
  const long long bidx = *blk;
  const long long n_first = (bidx * F_total + f_base - kHist) * (long long)kM;
  const int frame_min_trigger = (bidx == 0 && f_base == 0) ? kHist : 0;

  for (int bi = 0; bi < nbatch; ++bi) {
    const int r0 = bi * FB;
    const int gi = bi % 3;
    cp_async_wait_all();
    __syncthreads();   // stage of this batch landed; previous FIR is done with the ring
    // inverse DFT of frame r0+fr by warps (2 fr, 2 fr + 1) into ring group gi, slot fr
    {
      float2* slot = ring + (gi * FB + fr) * kM;
      const float2* st = stage + fr * SK + lane;
      if (half)
        frame_dft<1>(slot, st, tw, lane, 1 + fr);
      else
        frame_dft<0>(slot, st, tw, lane, 1 + fr);
    }
    __syncthreads();   // ring group gi written; stage consumed
    if (bi + 1 < nbatch) stage_batch(stg, m0, row, r0 + FB, nfr);
    if (r0 + FB <= kPrefix) continue;     // history-only batch (uniform)

    // synthesis FIR + envelope threshold for frames r0 .. r0+7.  History frames
    // r0-15 .. r0-9 sit in group gi+1 (slots 1..7), r0-8 .. r0-1 in group gi+2.
    const float2* ga = ring + (((gi + 1) % 3) * FB) * kM;
    const float2* gb = ring + (((gi + 2) % 3) * FB) * kM;
    const float2* gc = ring + (gi * FB) * kM;
    unsigned vmask = 0;                    // output frames of the batch that may trigger
    unsigned ymask = 0;                    // output frames of the batch
#pragma unroll
    for (int f = 0; f < FB; ++f) {
      const int r = r0 + f;
      const long long m = m0 - kPrefix + r;
      if (r >= kPrefix && r < nfr) {
        ymask |= 1u << f;
        if (m >= frame_min_trigger) vmask |= 1u << f;
      }
    }
    const long long m_row0 = m0 - kPrefix + r0;             // frame of batch row 0
    float* yrow = yj ? yj + m_row0 * kM : nullptr;
    const long long n_row0 = n_first + m_row0 * kM;
    if (yrow)
      fir_batch<true>(gq, ga, gb, gc, tid, lane, yrow, ymask, vmask, th2, n_row0, j, P, Tr,
                      theta[j] / k_sigma, trig, trig_count, trig_cap);
    else
      fir_batch<false>(gq, ga, gb, gc, tid, lane, yrow, ymask, vmask, th2, n_row0, j, P, Tr,
                       theta[j] / k_sigma, trig, trig_count, trig_cap);
  }
}

// Block noise power and running sigma (one block of 256 threads per stream).
// Pi = (2 G2 / M^3) * (1/F) * sum_{m,k} |beam|^2, G2 = sum g^2 = M^4 sum h^2 / (sum h)^2;
// s2 = Pi (first block) or (1 - alpha) s2 + alpha Pi; theta = k_sigma sqrt(s2).
__global__ void __launch_bounds__(256) k_sigma(const float* __restrict__ part, int n_per_stream,
                                               const double* __restrict__ sums, long long F,
                                               double alpha, double k_sigma,
                                               const long long* __restrict__ blk,
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
    const double s2 = *blk == 0 ? pi : (1.0 - alpha) * sigma2[j] + alpha * pi;
    sigma2[j] = s2;
    const double th = k_sigma * sqrt(s2);
    theta[j] = (float)th;
    theta2[j] = (float)(th * th);
  }
}

// Carry the last 16 frames of every (stream, bin) row into the row prefix and
// advance the device block counter.
__global__ void k_history_shift(float2* __restrict__ beams, long long rows, long long F,
                                long long row, long long* __restrict__ blk, int advance) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i == 0 && advance) *blk += 1;
  if (i >= rows * kPrefix) return;
  const long long r = i / kPrefix;
  const int f = (int)(i % kPrefix);
  beams[r * row + f] = beams[r * row + F + f];
}

size_t ippf_smem_bytes() { return (size_t)(RING * kM + FB * SK) * sizeof(float2); }

}  // namespace

cudaError_t init_f32_attributes(const Shape& sh);
cudaError_t init_tc_attributes(const Shape& sh);

int ippf_default_frames_per_cta(const Shape& sh) {
  // enough blocks for several waves on 152 SMs, few history frames per block
  long long fpc = 512;
  while (fpc > 64 && (long long)sh.J() * ((sh.F + fpc - 1) / fpc) < 152LL * 8) fpc /= 2;
  return (int)fpc;
}

cudaError_t init_ippf_attributes() {
  return cudaFuncSetAttribute(k_ippf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ippf_smem_bytes());
}

cudaError_t launch_ippf(const lp_plan& p, const Chunk& c, cudaStream_t s) {
  const auto& sh = p.shape;
  const int fpc = p.frames_per_cta;
  const dim3 grid((unsigned)((c.nf + fpc - 1) / fpc), (unsigned)sh.J());
  k_ippf<<<grid, NT, ippf_smem_bytes(), s>>>(p.buf.beams, sh.K, p.cfg.first_bin, c.nf, p.row(), fpc,
                                             p.buf.g, p.buf.tw1024, p.buf.theta, p.buf.theta2,
                                             (float)p.cfg.k_sigma, p.buf.blk, sh.F, c.f_base, sh.P,
                                             sh.Tr, p.buf.y, p.buf.trig, p.buf.trig_count,
                                             p.cfg.trigger_cap);
  return cudaGetLastError();
}

cudaError_t launch_sigma(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  k_sigma<<<sh.J(), 256, 0, s>>>(p.buf.power_part, sh.K * p.n_ftiles_bf, p.buf.filter_sums, sh.F,
                                 p.cfg.sigma_alpha, p.cfg.k_sigma, p.buf.blk, p.buf.sigma2,
                                 p.buf.theta, p.buf.theta2);
  return cudaGetLastError();
}

cudaError_t launch_history_shift(const lp_plan& p, const Chunk& c, cudaStream_t s) {
  const auto& sh = p.shape;
  const long long rows = (long long)sh.J() * sh.K;
  const long long n = rows * kPrefix;
  k_history_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.buf.beams, rows, c.nf, p.row(),
                                                              p.buf.blk, c.last ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t init_kernel_attributes(const Shape& sh) {
  cudaError_t e = init_ippf_attributes();
  if (e == cudaSuccess) e = init_f32_attributes(sh);
  if (e == cudaSuccess) e = init_tc_attributes(sh);
  return e;
}

}  // namespace lp
