// Inverse polyphase filter bank + envelope trigger (Sec. 2 last paragraph,
// Sec. 3 second paragraph, Fig. 1), and the per-block noise level.
//
// k_ippf: one thread block owns one stream j and a run of output frames
// [m0, m1) and walks frames m0-16 .. m1-1 in batches of 8 (four frame pairs).
// Its 16 warps have two roles that run concurrently on a double-buffered ring:
//
//  * DFT warps 0..7 (two per frame pair) take, from a zero-padded 512-bin
//    stage of the batch's beam bins, the 1024-point inverse DFT
//        z[p] = sum_k c[k] exp(+2 pi i k p / 1024),  c nonzero only in the
//    selected bins (< 512), as 32 x 32 with k = 32 k1 + k2, p = p1 + 32 p2.
//    Every value is a pair of frames, so each packed FP32 instruction (FADD2 /
//    FMUL2 / FFMA2) does the same step for both frames.  Warp h = warp mod 2
//    owns the outputs p1 = h (mod 2) of the first 32-point stage (a 16-point
//    DFT of the 16 nonzero inputs k1 < 16, pre-rotated by exp(+2 pi i k1 h/32))
//    and p2 = h (mod 2) of the second (the inputs folded as
//    (a + (-1)^h b) exp(+2 pi i k2 h / 32), then a 16-point DFT).  Between the
//    stages come the twiddle exp(+2 pi i k2 p1 / 1024) and a transpose through
//    the pair's ring slots (16-byte granules, column XOR-swizzled by row mod 8:
//    free of bank conflicts both ways, addresses affine in the unrolled index).
//    The DFT warps stop before the last radix-2 stage and leave each butterfly
//    pair (a, b) of outputs P and P + 512 in the ring as two granules.
//  * FIR warps 8..15: thread t owns the butterfly partners (t, t + 512) and
//    (511 - t, 1023 - t): it forms z = a + b and a - b and filters the four
//    phases.  The taps (as (g, g) pairs, four sets) and the last 16 frames of
//    z of each phase live in the thread's own tensor-memory columns
//    (tcgen05.ld / tcgen05.st), so the ring holds only the batch in flight and
//    each granule is read once from shared memory.  Per phase it computes
//        u_m[p] = sum_{t<16} g[t M + p] z_{m-t}[p]     (g holds the 2/M scale),
//    y = Re u (optionally stored) and |u|^2 against theta^2; the warps vote
//    and compact the (rare) samples above threshold into the trigger list.
//
// The roles hand batches over with named barriers: "ready[s]" (DFT warps
// arrive, FIR warps wait) for ring buffer s, and "free[s]" (the reverse): ring
// buffer s has been read, and stage buffer s holds the bins of the batch after
// next, which the FIR warps copy (16-byte cp.async) while they filter.
// The first 16 frames of a run only fill the FIR history (16 extra inverse DFTs
// per run).  Runs: either frames_per_cta frames of one stream per block, or the
// balanced tiling (one block per SM walking an equal contiguous range of the
// streams' frames, a piece per stream it crosses), which leaves no tail wave and
// pays the 16 history frames once per piece.  FP32 throughout.
//
// OUT selects what the FIR warps do with z: 0 trigger, 1 trigger and y = Re u,
// 2 (full-rate mode) u stored, no trigger, 3 (LSMR inversion) no filter: the
// inverse DFT itself, scaled by 2/M, stored phase-major (a phase's 8 frames of a
// batch are 64 contiguous bytes, two 32-byte stores) as the right-hand sides of the
// LSMR systems.
#include "lp_internal.cuh"

#include <algorithm>
#include <cstdint>

namespace lp {
namespace {

constexpr int NT = 512;            // threads per block
constexpr int NDFT = 256;          // threads of the DFT role (warps 0..7)
constexpr int FB = 8;              // frames per batch (four pairs, two warps each)
constexpr int NPAIR = FB / 2;
constexpr int SPAIR = 514;         // stage granules per frame pair: 512 bins + pad
constexpr int TMEM_COLS = 512;
// named barriers (0 is __syncthreads)
constexpr int BAR_PAIR = 1;        // 1..4: the two warps of a frame pair
constexpr int BAR_READY = 6;       // 6, 7: ring buffer s written
constexpr int BAR_FREE = 8;        // 8, 9: ring buffer s read, stage buffer s loaded
// tensor-memory columns of a FIR thread (256 per thread: two FIR warps per
// lane quarter)
constexpr int TC_TAPS = 0;         // 4 x 32: (g, g) of each of the four phases
constexpr int TC_HIST = 128;       // 4 x 32: 16 frames (re, im) of each phase

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

// Packed FP32 pairs: one instruction for the same operation on two frames.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

// One complex value of a frame pair: re = (re_a, re_b), im = (im_a, im_b).
struct CP {
  float2 re, im;
};

__device__ __forceinline__ CP cadd(CP a, CP b) { return CP{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP csub(CP a, CP b) { return CP{sub2(a.re, b.re), sub2(a.im, b.im)}; }

// a * exp(+2 pi i E / 32), the trivial and 45-degree rotations spelled out.
template <int E>
__device__ __forceinline__ CP rot32(CP a) {
  constexpr int e = E & 31;
  constexpr float r = 0.70710678118654752440f;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 8) {
    return CP{make_float2(-a.im.x, -a.im.y), a.re};
  } else if constexpr (e == 16) {
    return CP{make_float2(-a.re.x, -a.re.y), make_float2(-a.im.x, -a.im.y)};
  } else if constexpr (e == 24) {
    return CP{a.im, make_float2(-a.re.x, -a.re.y)};
  } else if constexpr (e == 4) {
    return CP{mul2(sub2(a.re, a.im), bc(r)), mul2(add2(a.re, a.im), bc(r))};
  } else if constexpr (e == 12) {
    return CP{mul2(add2(a.re, a.im), bc(-r)), mul2(sub2(a.re, a.im), bc(r))};
  } else if constexpr (e == 20) {
    return CP{mul2(sub2(a.im, a.re), bc(r)), mul2(add2(a.re, a.im), bc(-r))};
  } else if constexpr (e == 28) {
    return CP{mul2(add2(a.re, a.im), bc(r)), mul2(sub2(a.im, a.re), bc(r))};
  } else {
    constexpr float c = cos32v(e), s = sin32v(e);
    return CP{fma2(a.re, bc(c), mul2(a.im, bc(-s))), fma2(a.re, bc(s), mul2(a.im, bc(c)))};
  }
}

// Butterfly (a, b) -> (a + b, (a - b) exp(+2 pi i E / 32)); the factor i is
// taken by swapping the subtraction's operands.
template <int E>
__device__ __forceinline__ void bfly(CP& a, CP& b) {
  const CP s = cadd(a, b);
  if constexpr ((E & 31) == 8)
    b = CP{sub2(b.im, a.im), sub2(a.re, b.re)};
  else
    b = rot32<E>(csub(a, b));
  a = s;
}

#define LP_CASE(n) case n: return rot32<n>(a);
__device__ __forceinline__ CP rot32_rt(CP a, int e) {   // e is a constant after unrolling
  switch (e & 31) {
    LP_CASE(0) LP_CASE(1) LP_CASE(2) LP_CASE(3) LP_CASE(4) LP_CASE(5) LP_CASE(6) LP_CASE(7)
    LP_CASE(8) LP_CASE(9) LP_CASE(10) LP_CASE(11) LP_CASE(12) LP_CASE(13) LP_CASE(14)
    LP_CASE(15) LP_CASE(16) LP_CASE(17) LP_CASE(18) LP_CASE(19) LP_CASE(20) LP_CASE(21)
    LP_CASE(22) LP_CASE(23) LP_CASE(24) LP_CASE(25) LP_CASE(26) LP_CASE(27) LP_CASE(28)
    LP_CASE(29) LP_CASE(30) LP_CASE(31)
  }
  return a;
}
#undef LP_CASE
#define LP_CASE(n) case n: bfly<n>(a, b); return;
__device__ __forceinline__ void bfly_rt(CP& a, CP& b, int e) {
  switch (e & 31) {
    LP_CASE(0) LP_CASE(2) LP_CASE(4) LP_CASE(6) LP_CASE(8) LP_CASE(10) LP_CASE(12) LP_CASE(14)
  }
}
#undef LP_CASE

// Radix-2 decimation-in-frequency stages of the 16-point DFT with kernel
// exp(+2 pi i k q / 16), from half-size SPAN down to 2; the last stage (twiddle
// 1) is left to the caller.  After all stages v[i] = X[br4(i)].
template <int SPAN>
__device__ __forceinline__ void dft16_stages(CP (&v)[16]) {
#pragma unroll
  for (int span = SPAN; span >= 2; span >>= 1) {
#pragma unroll
    for (int start = 0; start < 16; start += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) bfly_rt(v[start + j], v[start + j + span], j * (16 / span));
    }
  }
}

int ippf_num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 152;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src));
}
// 32-byte store (address 32-byte aligned)
__device__ __forceinline__ void st_global_v8(float* p, const float (&v)[8]) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}

// ---- tensor memory (used here as per-thread storage, no MMA) ----
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32]) {
  uint32_t (&u)[32] = reinterpret_cast<uint32_t(&)[32]>(r);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]),
        "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]),
        "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&r)[16]) {
  const uint32_t (&u)[16] = reinterpret_cast<const uint32_t(&)[16]>(r);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};\n" ::"r"(taddr),
      "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]),
      "r"(u[8]), "r"(u[9]), "r"(u[10]), "r"(u[11]), "r"(u[12]), "r"(u[13]), "r"(u[14]),
      "r"(u[15]));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Staging of the beam bins of CTA frames r0 .. r0+7 into
// stage[pair][first_bin + k] (16-byte copies of a frame pair: re_a, im_a,
// re_b, im_b).  FIR thread t copies pair t & 3 of bins k = t/4 + 64 i, so four
// neighbouring threads read the 64 contiguous bytes of one bin row and the
// shared-memory granules of a quarter warp fall in distinct banks.
struct Stager {
  const float2* src;      // bin t/4, frame 2 (t&3) of CTA frame 0
  int dst;                // granule offset of stage[t&3][first_bin + t/4]
  long long src_step;     // 64 rows
  int n;                  // bins this thread copies
  int f;                  // first frame of its pair within the batch
};

__device__ __forceinline__ Stager make_stager(const float2* brow, int K, int first_bin,
                                              long long row, int tid) {
  Stager st;
  const int q = tid & 3;
  const int k0 = tid >> 2;
  st.f = 2 * q;
  st.src = brow + (long long)k0 * row + st.f;
  st.dst = q * SPAIR + first_bin + k0;
  st.src_step = 64 * row;
  st.n = k0 < K ? (K - k0 + 63) / 64 : 0;
  return st;
}

__device__ __forceinline__ void stage_batch(const Stager& st, float4* stage, bool live, int r0) {
  const float2* src = st.src + r0;
  float4* dst = stage + st.dst;
#pragma unroll 4
  for (int i = 0; i < st.n; ++i) {
    if (live)
      cp_async16(dst + 64 * i, src + i * st.src_step);
    else
      dst[64 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_async_commit();
}

// Inverse DFT of one frame pair by its two warps; H = warp mod 2.
//   slot: the pair's 2 x 1024 float2 ring slots (frame a, then frame b), also
//         the 32 x 32 granule transpose buffer between the stages;
//   st:   stage[pair] + lane.
template <int H>
__device__ __forceinline__ void pair_dft(float2* slot, const float4* st,
                                         const float4* __restrict__ tw, int lane, int bar_id) {
  float4* tb = reinterpret_cast<float4*>(slot);
  CP v[16];
  // ---- stage 1 (k2 = lane): T[p1] = sum_{k1<16} c[32 k1 + lane] w32^(k1 p1), p1 = 2 q + H,
  // a 16-point DFT of d[k1] = c[k1] w32^(k1 H).  Its first stage is taken in
  // scalar form straight from the stage's (re_a, im_a, re_b, im_b) granules,
  // which regroups them into frame pairs at no extra cost:
  //   H = 0: (c_k + c_{k+8},  (c_k - c_{k+8}) w32^(2k))
  //   H = 1: ((c_k + i c_{k+8}) w32^k,  (c_k - i c_{k+8}) w32^(3k))
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 a = st[32 * k], b = st[32 * (k + 8)];
    if constexpr (H == 0) {
      const CP sm{make_float2(a.x + b.x, a.z + b.z), make_float2(a.y + b.y, a.w + b.w)};
      const CP df{make_float2(a.x - b.x, a.z - b.z), make_float2(a.y - b.y, a.w - b.w)};
      v[k] = sm;
      v[k + 8] = rot32_rt(df, 2 * k);
    } else {
      const CP sm{make_float2(a.x - b.y, a.z - b.w), make_float2(a.y + b.x, a.w + b.z)};
      const CP df{make_float2(a.x + b.y, a.z + b.w), make_float2(a.y - b.x, a.w - b.z)};
      v[k] = rot32_rt(sm, k);
      v[k + 8] = rot32_rt(df, 3 * k);
    }
  }
  dft16_stages<4>(v);
#pragma unroll
  for (int i = 0; i < 16; i += 2) bfly<0>(v[i], v[i + 1]);
  {
    // twiddle exp(+2 pi i lane p1 / 1024); granule (p1 & 24) + ((p1 & 7) ^ (lane & 7))
    const int l7 = lane & 7;
    float4* row = tb + lane * 32;
    float4* wb[4] = {row + ((0 + H) ^ l7), row + ((2 + H) ^ l7), row + ((4 + H) ^ l7),
                     row + ((6 + H) ^ l7)};
    const float4* twl = tw + H * 32 + lane;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int q = br4(i);
      const float4 t = __ldg(twl + q * 64);
      const float2 c = make_float2(t.x, t.y), s = make_float2(t.z, t.w);
      const float2 re = fma2(v[i].re, c, mul2(v[i].im, make_float2(-s.x, -s.y)));
      const float2 im = fma2(v[i].re, s, mul2(v[i].im, c));
      wb[q & 3][8 * (q >> 2)] = make_float4(re.x, re.y, im.x, im.y);
    }
  }
  bar_sync(bar_id, 64);
  // ---- stage 2 (p1 = lane): inputs T'[k2][lane], folded by output parity H
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float4* r = tb + (lane ^ (k & 7)) + 32 * k;
    const float4 a = r[0], b = r[512];                  // rows k and k + 16
    const CP ca{make_float2(a.x, a.y), make_float2(a.z, a.w)};
    const CP cb{make_float2(b.x, b.y), make_float2(b.z, b.w)};
    v[k] = H ? rot32_rt(csub(ca, cb), k) : cadd(ca, cb);
  }
  bar_sync(bar_id, 64);                  // both warps have read the transpose
  dft16_stages<8>(v);
  // The last butterfly stage is left to the FIR warps: outputs p2 and p2 + 16
  // (p2 = 2 br4(2m) + H, phases P = lane + 32 p2 and P + 512) are a + b and
  // a - b of a = v[2m], b = v[2m + 1], stored as granules P and P + 512.
  float4* zg = tb + lane + 32 * H;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int o = 64 * br4(2 * m);
    const CP a = v[2 * m], b = v[2 * m + 1];
    zg[o] = make_float4(a.re.x, a.re.y, a.im.x, a.im.y);
    zg[o + 512] = make_float4(b.re.x, b.re.y, b.im.x, b.im.y);
  }
}

// Per-batch context of the FIR role.
struct FirCtx {
  float th2;
  unsigned ymask;          // output frames of the batch (time-series store)
  float* yrow;             // y of batch row 0 (or null)
  float2* urow;            // u of batch row 0 (full-rate mode)
};

// The CTA's stream (index within its plan, sigma, plan), kept in shared memory
// for the rare trigger path.
struct StreamInfo {
  int j;
  float sig;
  const IppfPlan* plan;
  int nfr, r_trig;         // frames of the run, first run row that may trigger
  long long n_first, m0;   // sample index of block frame -15, phase 0; first output frame
};

// Bits [lo, hi) of an 8-bit frame mask (lo, hi clamped to [0, 8]).
__device__ __forceinline__ unsigned frame_bits(int lo, int hi) {
  lo = max(0, min(lo, FB));
  hi = max(lo, min(hi, FB));
  return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Batch r0 of the run (rows r0 .. r0 + 7): the frames that may trigger and the
// sample origin follow from the run's constants in shared memory.
__device__ __noinline__ void emit_triggers(const float (&e2v)[FB], float th2, int p, int r0,
                                           const StreamInfo* si) {
  const int lane = threadIdx.x & 31;
  const IppfPlan& o = *si->plan;
  const unsigned vmask = frame_bits(kPrefix - r0, si->nfr - r0) & frame_bits(si->r_trig - r0, FB);
  const long long n_row0 = si->n_first + (si->m0 - kPrefix + r0) * kM;
  const int j = si->j;
  const float sig = si->sig;
  const int P = o.P, Tr = o.Tr;
#pragma unroll
  for (int f = 0; f < FB; ++f) {
    const bool hit = ((vmask >> f) & 1u) && e2v[f] > th2;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (!mask) continue;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(o.count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (hit) {
      const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
      if ((long long)idx < o.cap) {
        TriggerRec rec;
        rec.n = n_row0 + (long long)f * kM + p;
        rec.pol = j % P;
        rec.tec = (j / P) % Tr;
        rec.beam = j / (P * Tr);
        rec.stream = j;
        rec.env = sqrtf(e2v[f]);
        rec.sigma = sig;
        o.trig[idx] = rec;
      }
    }
  }
}

// FIR of one phase over one batch.  hist: the phase's 16 history slots (frame
// r at slot r mod 16, (re, im) in consecutive columns); zn: the 8 new frames.
// ODD selects where the 15 history frames r0-15 .. r0-1 sit (r0 mod 16 = 8 ODD).
// OUT: 0 trigger, 1 trigger and y = Re u, 2 (full-rate mode) u stored, no trigger.
template <int ODD, int OUT>
__device__ __forceinline__ void fir_phase(const float2 (&gq)[kTaps], const float (&hist)[32],
                                          const float2 (&zn)[FB], int p, int r0, const FirCtx& c,
                                          const StreamInfo* si) {
  float2 w[kHist + FB];
#pragma unroll
  for (int i = 0; i < kHist; ++i) {
    const int slot = (ODD ? 9 + i : 1 + i) & 15;
    w[i] = make_float2(hist[2 * slot], hist[2 * slot + 1]);
  }
#pragma unroll
  for (int f = 0; f < FB; ++f) w[kHist + f] = zn[f];
  if constexpr (OUT == 2) {
#pragma unroll
    for (int f = 0; f < FB; ++f) {
      float2 u = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < kTaps; ++t) u = __ffma2_rn(gq[t], w[f + kHist - t], u);
      if ((c.ymask >> f) & 1u) c.urow[f * kM + p] = u;
    }
    return;
  }
  float e2v[FB];
  float emax = 0.f;
#pragma unroll
  for (int f = 0; f < FB; ++f) {
    float2 u = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < kTaps; ++t)   // both components per instruction, tap (g, g)
      u = __ffma2_rn(gq[t], w[f + kHist - t], u);
    if constexpr (OUT == 1)  // (in a group, plans without a stored series have no row)
      if (c.yrow && ((c.ymask >> f) & 1u)) c.yrow[f * kM + p] = u.x;
    e2v[f] = fmaf(u.x, u.x, u.y * u.y);
    emax = fmaxf(emax, e2v[f]);         // frames outside the run are filtered by vmask
  }
  if (__any_sync(0xffffffffu, emax > c.th2)) {
    // the rare trigger path gets its own copy, so that e2v stays in registers
    float e2c[FB];
#pragma unroll
    for (int f = 0; f < FB; ++f) e2c[f] = e2v[f];
    emit_triggers(e2c, c.th2, p, r0, si);
  }
}

// One phase of the FIR role for batch r0: its 8 new frames zn, history from
// tensor memory; the new frames then replace the history slots r0 mod 16 ...
template <int OUT>
__device__ __forceinline__ void fir_one(const float2 (&gq)[kTaps], uint32_t thist,
                                        const float2 (&zn)[FB], int p, int r0, bool outputs,
                                        const FirCtx& c, const StreamInfo* si) {
  if (outputs) {
    float hist[32];
    tmem_ld32(thist, hist);
    tmem_wait_ld();
    if (r0 & 8)
      fir_phase<1, OUT>(gq, hist, zn, p, r0, c, si);
    else
      fir_phase<0, OUT>(gq, hist, zn, p, r0, c, si);
  }
  // the 8 new frames fill 16 consecutive history columns: one store
  tmem_st16(thist + 2 * (r0 & 8), reinterpret_cast<const float(&)[16]>(zn[0]));
}

// One launch covers the streams of a.n plans (one plan, or a group of plans
// fused into one launch): blockIdx.y counts the launch streams of plan 0, then
// plan 1, ...; every plan has its own beam rows, thresholds, block counter and
// trigger list, and all share the frame range and the tiling.  GROUP = false:
// one plan, whose parameters are then read at fixed offsets of the parameter
// block (no indexed lookup on the single-plan path).
template <bool GROUP, int OUT>
__global__ void __launch_bounds__(NT, 1) k_ippf(
    const __grid_constant__ IppfArgsN<GROUP ? kMaxGroup : 1> a) {
  extern __shared__ float4 smem4[];
  float2* ring = reinterpret_cast<float2*>(smem4);      // [2 buffers][8 frames][1024]
  float4* stage = smem4 + FB * kM;                        // [2 buffers][4 pairs][SPAIR]
  __shared__ uint32_t tmem_slot;
  __shared__ StreamInfo sinfo;
  // the run's row origin and copy limit, re-read by the FIR threads every batch
  // (kept out of their registers)
  __shared__ const float2* s_brow;
  __shared__ int s_live_lim;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // The block's work, in the launch's (stream, frame) space: frames_per_cta
  // > 0: run blockIdx.x of frames_per_cta frames of stream blockIdx.y;
  // frames_per_cta == 0 (balanced): one contiguous range of every stream's
  // frames in turn, split evenly over the grid in multiples of 8 frames, so
  // that every block does the same work and a block's pieces are at most a few
  // streams' runs (each piece pays the 16 history frames once).
  const long long F = a.F, row = a.row;
  // the range walked so far lives in shared memory (no registers held across
  // the roles' loops): [s_pos, s_end)
  __shared__ long long s_pos, s_end;
  if (tid == 0) {
    long long pos, end;
    if (a.frames_per_cta > 0) {
      pos = (long long)blockIdx.y * F + (long long)blockIdx.x * a.frames_per_cta;
      end = min(pos + a.frames_per_cta, ((long long)blockIdx.y + 1) * F);
    } else {
      const long long total = (long long)a.nstreams * F;
      const long long per = ((total + gridDim.x - 1) / gridDim.x + FB - 1) / FB * FB;
      pos = min(total, (long long)blockIdx.x * per);
      end = min(total, pos + per);
    }
    s_pos = pos;
    s_end = end;
  }
  __syncthreads();
  for (;;) {
    const long long pos = s_pos, end = s_end;
    if (pos >= end) break;
    const int sid = (int)(pos / F);            // launch stream of this piece
    const long long m0 = pos % F;
    const long long m1 = min(F, m0 + (end - pos));
    int pi = 0;
    if constexpr (GROUP)
      while (pi + 1 < a.n && sid >= a.pl[pi].stream_end) ++pi;
    const IppfPlan& pl = a.pl[GROUP ? pi : 0];
    const int jj = sid - (GROUP && pi ? a.pl[pi - 1].stream_end : 0);
    const int j = (int)sel_stream(jj, pl.P, a.pol0, a.npol);
    const int K = pl.K, first_bin = pl.first_bin;
    const float2* __restrict__ beams = pl.beams;
    const float4* __restrict__ tw = pl.tw;
    const int nout = (int)(m1 - m0);
    const int nfr = nout + kPrefix;          // frames run through the inverse DFT
    const int nbatch = (nfr + FB - 1) / FB;

    if (tid == 0) sinfo = StreamInfo{j, pl.theta[j] / pl.k_sigma, &pl, 0, 0, 0, 0};
    // bins outside the selection stay zero for the whole piece
    for (int i = tid; i < 2 * NPAIR * SPAIR; i += NT) stage[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    if (tid == 0) s_pos = pos + (m1 - m0);     // every thread has read s_pos: the next piece
    // the FIR threads stage the bins (thread tid - NDFT); batches 0 and 1 now
    const float2* brow = beams + (long long)j * K * row + m0;   // position of frame m0-16
    const Stager stg = make_stager(brow, K, first_bin, row, tid - NDFT);
    // a pair is copied when both its frames are in the run and inside the row
    const int live_lim = (int)min((long long)nfr, row - m0);
    if (warp >= NDFT / 32) {
      stage_batch(stg, stage, stg.f + 1 < live_lim, 0);
      stage_batch(stg, stage + NPAIR * SPAIR, FB + stg.f + 1 < live_lim, FB);
      cp_async_wait_all();
    }
    if (tid == 0) {
      s_brow = brow;
      s_live_lim = live_lim;
    }
    __syncthreads();

    if (warp < NDFT / 32) {
      // ===================== DFT role =====================
      const int pr = warp >> 1, h = warp & 1;     // frame pair of the batch, output parity
      for (int bi = 0; bi < nbatch; ++bi) {
        const int s = bi & 1;
        // ring buffer s read by the FIR role, stage buffer s loaded with batch bi
        if (bi >= 2) bar_sync(BAR_FREE + s, NT);
        float2* slot = ring + (s * FB + 2 * pr) * kM;
        const float4* st = stage + s * NPAIR * SPAIR + pr * SPAIR + lane;
        if (h)
          pair_dft<1>(slot, st, tw, lane, BAR_PAIR + pr);
        else
          pair_dft<0>(slot, st, tw, lane, BAR_PAIR + pr);
        bar_arrive(BAR_READY + s, NT);
      }
    } else {
      // ===================== FIR role =====================
      // thread ft owns the butterfly partners (ft, ft + 512) and (511 - ft, 1023 - ft)
      const int ft = tid - NDFT;
      const uint32_t tbase = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 256u * ((warp - 8) >> 2);
      // taps (g, g) of the four phases into tensor memory (not in the LSMR
      // mode, which does not filter)
  #pragma unroll 1
      for (int ph = 0; ph < (OUT == 3 ? 0 : 4); ++ph) {
        const int p = (ph & 2 ? kM / 2 - 1 - ft : ft) + (ph & 1 ? kM / 2 : 0);
        float tq[32];
  #pragma unroll
        for (int t = 0; t < kTaps; ++t) {
          const float gt = pl.g[t * kM + p];
          tq[2 * t] = gt;
          tq[2 * t + 1] = gt;
        }
        tmem_st16(tbase + TC_TAPS + 32 * ph, reinterpret_cast<const float(&)[16]>(tq[0]));
        tmem_st16(tbase + TC_TAPS + 32 * ph + 16, reinterpret_cast<const float(&)[16]>(tq[16]));
      }
      tmem_wait_st();
      FirCtx c;
      c.th2 = pl.theta2[j];
      const long long F_total = a.F_total, f_base = a.f_base;
      // this launch covers block frames [f_base, f_base + F) (one chunk, or the block)
      float* yj = OUT == 1 && pl.y ? pl.y + ((long long)j * F_total + f_base) * kM : nullptr;
      // full-rate mode: the series row of the stream (history first)
      float2* uj = OUT == 2 ? pl.u + (long long)j * pl.u_row + kFrTaps + f_base * kM : nullptr;
      // LSMR mode: the stream's phase rows of u_row positions each; batch row r
      // of the run is position m0 + r (frame m0 - 16 + r), written once: rows
      // r >= 16, and the prefix rows of a stream's first run
      float2* zj = OUT == 3 ? pl.u + (long long)j * kM * pl.u_row : nullptr;
      const int r_lo = m0 == 0 ? 0 : kPrefix;
      // block i of the stream starts at sample (i F - 15) M; samples n < 0 (frames
      // m < 15 of the first block) never trigger
      const long long bidx = *pl.blk;
      const long long n_first = (bidx * F_total + f_base - kHist) * (long long)kM;
      const int frame_min_trigger = (bidx == 0 && f_base == 0) ? kHist : 0;
      // run row r (frame m0 - 16 + r) is an output for r in [16, nfr) and may
      // trigger for r >= r_trig
      const int r_trig = (int)max((long long)kPrefix, frame_min_trigger + kPrefix - m0);
      if (tid == NDFT) {   // read by the trigger path after the first ready barrier
        sinfo.nfr = nfr;
        sinfo.r_trig = r_trig;
        sinfo.n_first = n_first;
        sinfo.m0 = m0;
      }
      for (int bi = 0; bi < nbatch; ++bi) {
        const int s = bi & 1, r0 = bi * FB;
        bar_sync(BAR_READY + s, NT);       // ring buffer s holds batch bi
        // stage buffer s is free again: bins of batch bi + 2
        if (bi + 2 < nbatch) {
          const Stager st = make_stager(s_brow, K, first_bin, row, ft);
          stage_batch(st, stage + s * NPAIR * SPAIR, (bi + 2) * FB + st.f + 1 < s_live_lim,
                      (bi + 2) * FB);
        }
        const float4* zr = reinterpret_cast<const float4*>(ring + s * FB * kM);
        const bool outputs = r0 >= kPrefix;
        c.ymask = frame_bits(kPrefix - r0, nfr - r0);
        const long long m_row0 = m0 - kPrefix + r0;             // frame of batch row 0
        c.yrow = yj ? yj + m_row0 * kM : nullptr;
        if constexpr (OUT == 2) c.urow = uj + m_row0 * kM;
  #pragma unroll 1
        for (int bp = 0; bp < 2; ++bp) {
          const int pb = bp ? kM / 2 - 1 - ft : ft;
          // last butterfly: z[pb] = a + b, z[pb + 512] = a - b, for both frames of
          // each pair (granule = re_a, re_b, im_a, im_b)
          float2 za[FB], zb[FB];
  #pragma unroll
          for (int q = 0; q < FB / 2; ++q) {
            const float4 a = zr[q * kM + pb], b = zr[q * kM + pb + kM / 2];
            za[2 * q] = make_float2(a.x + b.x, a.z + b.z);
            za[2 * q + 1] = make_float2(a.y + b.y, a.w + b.w);
            zb[2 * q] = make_float2(a.x - b.x, a.z - b.z);
            zb[2 * q + 1] = make_float2(a.y - b.y, a.w - b.w);
          }
          if constexpr (OUT == 3) {
            constexpr float sc = 2.0f / kM;           // a power of two: exact
            const bool all = r0 >= r_lo && r0 + FB <= nfr;
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float2* z = h ? zb : za;
              float2* dst = zj + (long long)(pb + h * (kM / 2)) * pl.u_row + m0 + r0;
              if (all) {
                // two 32-byte stores: u_row is a multiple of 16 (block_len a
                // multiple of 256) and m0 + r0 of 8, so dst is 64-byte aligned
  #pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                  float o[8];
  #pragma unroll
                  for (int f = 0; f < 4; ++f) {
                    o[2 * f] = z[4 * hf + f].x * sc;
                    o[2 * f + 1] = z[4 * hf + f].y * sc;
                  }
                  st_global_v8(reinterpret_cast<float*>(dst) + 8 * hf, o);
                }
              } else {
  #pragma unroll
                for (int f = 0; f < FB; ++f)
                  if (r0 + f >= r_lo && r0 + f < nfr)
                    dst[f] = make_float2(z[f].x * sc, z[f].y * sc);
              }
            }
            continue;
          }
  #pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int ph = 2 * bp + h;
            float tq[32];
            tmem_ld32(tbase + TC_TAPS + 32 * ph, tq);
            tmem_wait_ld();
            float2 gq[kTaps];
  #pragma unroll
            for (int t = 0; t < kTaps; ++t) gq[t] = make_float2(tq[2 * t], tq[2 * t + 1]);
            fir_one<OUT>(gq, tbase + TC_HIST + 32 * ph, h ? zb : za, pb + h * (kM / 2), r0,
                         outputs, c, &sinfo);
          }
        }
        tmem_wait_st();                    // history slots written before the next batch reads them
        if (bi + 2 < nbatch) {
          cp_async_wait_all();             // this thread's copies of batch bi + 2 landed
          bar_arrive(BAR_FREE + s, NT);
        }
      }
    }
    // both roles are done with the ring, the stage buffers and sinfo
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// Block noise power and running sigma (one block of 256 threads per stream;
// the streams of a.n plans, plan 0's first).
// Pi = (2 G2 / M^3) * (1/F) * sum_{m,k} |beam|^2, G2 = sum g^2 = M^4 sum h^2 / (sum h)^2;
// s2 = Pi (first block) or (1 - alpha) s2 + alpha Pi; theta = k_sigma sqrt(s2).
__global__ void __launch_bounds__(256) k_sigma(const __grid_constant__ SigmaArgs a) {
  __shared__ double red[256];
  int pi = 0;
  while (pi + 1 < a.n && (int)blockIdx.x >= a.pl[pi].stream_end) ++pi;
  const SigmaPlan& pl = a.pl[pi];
  const int jj = (int)blockIdx.x - (pi ? a.pl[pi - 1].stream_end : 0);
  const long long j = sel_stream(jj, pl.P, a.pol0, a.npol);
  const int n_per_stream = pl.n_per_stream;
  const float* pj = pl.part + j * n_per_stream;
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
    const double g2 = m * m * m * m * pl.sums[1] / (pl.sums[0] * pl.sums[0]);
    const double pw = 2.0 * g2 / (m * m * m) * red[0] / (double)a.F;
    const double s2 = *pl.blk == 0 ? pw : (1.0 - pl.alpha) * pl.sigma2[j] + pl.alpha * pw;
    pl.sigma2[j] = s2;
    const double th = pl.k_sigma * sqrt(s2);
    pl.theta[j] = (float)th;
    pl.theta2[j] = (float)(th * th);
    if (pl.count && jj == 0) *pl.count = 0;
  }
}

// Carry the last 16 frames of every (stream, bin) row into the row prefix and
// advance the device block counter: the last 16 frames of each row become the
// next block's prefix, in the beam rows and (fine de-dispersion) in the
// filtered rows.  Elements of plan 0's rows first, then plan 1's, ...
__global__ void k_history_shift(const __grid_constant__ ShiftArgs a) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int pi = 0;
  while (pi + 1 < a.n && i >= a.pl[pi].elem_end) ++pi;
  const ShiftPlan& pl = a.pl[pi];
  const long long i0 = pi ? a.pl[pi - 1].elem_end : 0;
  if (i == i0 && a.advance) *pl.blk += 1;
  if (i >= pl.elem_end) return;
  const long long rr = (i - i0) / kPrefix;      // launch row of the plan: stream jj, bin k
  const int f = (int)((i - i0) % kPrefix);
  const long long r = sel_stream(rr / pl.K, pl.P, a.pol0, a.npol) * pl.K + rr % pl.K;
  const long long row = a.row, F = a.F;
  pl.beams[r * row + f] = pl.beams[r * row + F + f];
  if (pl.fine) pl.fine[r * row + f] = pl.fine[r * row + F + f];
}

size_t ippf_smem_bytes() {
  return (size_t)2 * FB * kM * sizeof(float2) + (size_t)2 * NPAIR * SPAIR * sizeof(float4);
}

}  // namespace

cudaError_t init_f32_attributes(const Shape& sh);
cudaError_t init_tc_attributes(const Shape& sh);

cudaError_t init_ippf_attributes() {
  const void* k[6] = {(const void*)k_ippf<false, 0>, (const void*)k_ippf<false, 1>,
                      (const void*)k_ippf<false, 2>, (const void*)k_ippf<false, 3>,
                      (const void*)k_ippf<true, 0>, (const void*)k_ippf<true, 1>};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = raise_smem_limit(k[i], ippf_smem_bytes());
  return e;
}

IppfPlan ippf_plan(const lp_plan& p) {
  IppfPlan q{};
  q.beams = synth_rows(p);
  q.g = p.buf.g;
  q.tw = p.buf.tw1024;
  q.theta = p.buf.theta;
  q.theta2 = p.buf.theta2;
  q.blk = p.buf.blk;
  q.y = p.buf.y;
  q.u = p.buf.ufull;
  q.u_row = p.buf.ufull ? fullrate_row(p) : 0;
  q.trig = p.buf.trig;
  q.count = p.buf.trig_count;
  q.cap = (long long)p.cfg.trigger_cap;
  q.k_sigma = (float)p.cfg.k_sigma;
  q.K = p.shape.K;
  q.first_bin = p.cfg.first_bin;
  q.P = p.shape.P;
  q.Tr = p.shape.Tr;
  return q;
}

// Plans plans[0..n) (same block length, chunking and tiling) in one launch.
cudaError_t launch_ippf_plans(const lp_plan* const* plans, int n, const Chunk& c, cudaStream_t s,
                              PolSel ps) {
  const lp_plan& p0 = *plans[0];
  const int fpc = p0.frames_per_cta;
  const int npol = ps.npol ? ps.npol : p0.shape.P;
  IppfArgs a;
  a.F = c.nf;
  a.row = p0.row();
  a.F_total = p0.shape.F;
  a.f_base = c.f_base;
  a.frames_per_cta = fpc;
  a.pol0 = ps.pol0;
  a.npol = npol;
  a.n = n;
  int streams = 0;
  for (int i = 0; i < n; ++i) {
    a.pl[i] = ippf_plan(*plans[i]);
    streams += plans[i]->shape.J() / plans[i]->shape.P * npol;
    a.pl[i].stream_end = streams;
  }
  a.nstreams = streams;
  // balanced tiling (frames_per_cta 0): one block per SM (one fits), or one per
  // 8 frames of work if there is less
  const long long work8 = ((long long)streams * c.nf + FB - 1) / FB;
  const dim3 grid = fpc > 0 ? dim3((unsigned)((c.nf + fpc - 1) / fpc), (unsigned)streams)
                            : dim3((unsigned)std::min<long long>(ippf_num_sms(), work8), 1u);
  if (n == 1) {
    IppfArgsN<1> a1;
    a1.F = a.F;
    a1.row = a.row;
    a1.F_total = a.F_total;
    a1.f_base = a.f_base;
    a1.frames_per_cta = a.frames_per_cta;
    a1.nstreams = a.nstreams;
    a1.pol0 = a.pol0;
    a1.npol = a.npol;
    a1.n = 1;
    a1.pl[0] = a.pl[0];
    if (a1.pl[0].u)
      k_ippf<false, 2><<<grid, NT, ippf_smem_bytes(), s>>>(a1);
    else if (a1.pl[0].y)
      k_ippf<false, 1><<<grid, NT, ippf_smem_bytes(), s>>>(a1);
    else
      k_ippf<false, 0><<<grid, NT, ippf_smem_bytes(), s>>>(a1);
  } else {
    bool any_y = false;
    for (int i = 0; i < n; ++i) any_y = any_y || a.pl[i].y;
    if (any_y)
      k_ippf<true, 1><<<grid, NT, ippf_smem_bytes(), s>>>(a);
    else
      k_ippf<true, 0><<<grid, NT, ippf_smem_bytes(), s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_ippf(const lp_plan& p, const Chunk& c, cudaStream_t s, PolSel ps) {
  const lp_plan* one = &p;
  return launch_ippf_plans(&one, 1, c, s, ps);
}

// The LSMR right-hand sides: the inverse DFT of every frame of the block and of
// the 16 before it, zt[j][p][frame + 16] = (2/M) z_frame[p], by the synthesis
// kernel's DFT role in its balanced tiling (OUT = 3: no filter, no trigger).
cudaError_t launch_ippf_zt(const lp_plan& p, cudaStream_t s) {
  IppfArgsN<1> a;
  a.F = p.shape.F;
  a.row = p.row();
  a.F_total = p.shape.F;
  a.f_base = 0;
  a.frames_per_cta = 0;
  a.pol0 = 0;
  a.npol = p.shape.P;
  a.n = 1;
  a.pl[0] = ippf_plan(p);
  a.pl[0].y = nullptr;
  a.pl[0].u = p.buf.zt;
  a.pl[0].u_row = p.shape.F + kPrefix;
  const int streams = p.shape.J();
  a.nstreams = streams;
  a.pl[0].stream_end = streams;
  const long long work8 = ((long long)streams * a.F + FB - 1) / FB;
  const dim3 grid((unsigned)std::min<long long>(ippf_num_sms(), work8), 1u);
  k_ippf<false, 3><<<grid, NT, ippf_smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sigma_plans(const lp_plan* const* plans, int n, bool zero_counts,
                               cudaStream_t s, PolSel ps) {
  const lp_plan& p0 = *plans[0];
  const int npol = ps.npol ? ps.npol : p0.shape.P;
  SigmaArgs a;
  a.F = p0.shape.F;
  a.pol0 = ps.pol0;
  a.npol = npol;
  a.n = n;
  int streams = 0;
  for (int i = 0; i < n; ++i) {
    const lp_plan& p = *plans[i];
    SigmaPlan& q = a.pl[i];
    q.part = p.buf.power_part;
    q.sums = p.buf.filter_sums;
    q.blk = p.buf.blk;
    q.sigma2 = p.buf.sigma2;
    q.theta = p.buf.theta;
    q.theta2 = p.buf.theta2;
    q.count = zero_counts ? p.buf.trig_count : nullptr;
    q.alpha = p.cfg.sigma_alpha;
    q.k_sigma = p.cfg.k_sigma;
    q.n_per_stream = p.shape.K * p.n_ftiles_bf;
    q.P = p.shape.P;
    streams += p.shape.J() / p.shape.P * npol;
    q.stream_end = streams;
  }
  k_sigma<<<streams, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sigma(const lp_plan& p, cudaStream_t s, PolSel ps) {
  const lp_plan* one = &p;
  return launch_sigma_plans(&one, 1, false, s, ps);
}

cudaError_t launch_history_shift_plans(const lp_plan* const* plans, int n, const Chunk& c,
                                       cudaStream_t s, PolSel ps) {
  const lp_plan& p0 = *plans[0];
  const int npol = ps.npol ? ps.npol : p0.shape.P;
  ShiftArgs a;
  a.F = c.nf;
  a.row = p0.row();
  a.advance = c.last && ps.pol0 + npol == p0.shape.P ? 1 : 0;
  a.pol0 = ps.pol0;
  a.npol = npol;
  a.n = n;
  long long elems = 0;
  for (int i = 0; i < n; ++i) {
    const lp_plan& p = *plans[i];
    ShiftPlan& q = a.pl[i];
    q.beams = p.buf.beams;
    q.fine = p.buf.beams_fine;
    q.blk = p.buf.blk;
    q.K = p.shape.K;
    q.P = p.shape.P;
    elems += (long long)p.shape.J() / p.shape.P * npol * p.shape.K * kPrefix;
    q.elem_end = elems;
  }
  k_history_shift<<<(unsigned)((elems + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_history_shift(const lp_plan& p, const Chunk& c, cudaStream_t s, PolSel ps) {
  const lp_plan* one = &p;
  return launch_history_shift_plans(&one, 1, c, s, ps);
}

cudaError_t init_fullrate_attributes();

cudaError_t init_kernel_attributes(const Shape& sh) {
  cudaError_t e = init_ippf_attributes();
  if (e == cudaSuccess) e = init_fullrate_attributes();
  if (e == cudaSuccess) e = init_f32_attributes(sh);
  if (e == cudaSuccess) e = init_tc_attributes(sh);
  return e;
}

}  // namespace lp
