// Beamforming + de-dispersion on the 5th-generation tensor cores (FP16 form).
//
// Sec. 3, first and third paragraphs:
//     beam[j = (b,t,pol)][k][m] = D[k,t] * sum_s w[k,b,s] * x[pol][k][m][s].
// Per subband k this is a complex GEMM; in real form
//     C[2b+c][m] = sum_{kd < 2S} A_k[2b+c][kd] * X[m][kd],   kd = 2s + (re, im),
// with rows 2b = Re, 2b+1 = Im of beam b and
//     A[2b][2s] = w_re, A[2b][2s+1] = -w_im, A[2b+1][2s] = w_im, A[2b+1][2s+1] = w_re.
// The int8 samples are exact in FP16; each weight is split into an FP16 high
// part and an FP16 low part (w - hi), and both products accumulate in FP32 in
// tensor memory, which keeps the weight error near 1e-7 (one FP16 part alone
// would leave ~1.5e-4 relative error in the beams).  int16 samples v are split
// as v = 256 h + l (h = v >> 8 in [-128, 127], l = v & 255), and 256 h and l
// are both exact in FP16: two B images, four products per K step.
//
// Work items: (subband k, beam tile of 64 beams, pol, chunk of 2048 frames),
// eight 256-frame tiles each.  One persistent block per SM walks a contiguous
// item range as a warp-specialised pipeline:
//   warp 0      producer: cp.async.bulk copies of each tile's samples
//               (256 frames x 2S contiguous int8 or int16) into a ring of stages, and of
//               the A images (hi and lo weights, pre-arranged by k_weights_tc)
//               whenever (k, beam tile) changes;
//   warps 2-9   converters: int8 -> FP16 in the canonical K-major no-swizzle
//               layout (8-row x 16-byte core matrices), a ring of B stages.
//               A byte b becomes the FP16 number 1024 + (b ^ 0x80) by placing
//               it under the exponent pattern of 1024 (byte permute), and one
//               packed subtraction of 1152 leaves b exactly (int16: the high
//               byte so, then times 256; the low byte as 1024 + l minus 1024);
//   warp 1      MMA: one thread issues 2 * 2S/16 (int16: 4 * 2S/16) tcgen05.mma (M = 128, N = 256,
//               K = 16) into one of two 256-column TMEM accumulators and
//               commits to mbarriers that free the B stage and publish the
//               accumulator;
//   warps 10-17 epilogue: two warps per 32-lane TMEM quarter (one per column
//               half) read the accumulator with tcgen05.ld, pair Re/Im lanes
//               by shuffle, multiply by D[k,t], sum |beam|^2 per chunk, and
//               stage 16-beam x 16-frame boxes (128-byte swizzle) that a TMA
//               tensor store (cp.async.bulk.tensor, 5-D map over
//               [beam][trial][pol][k][frame]) writes to the beam rows.
// The epilogue of tile i, the MMAs of tile i+1, the conversion of tile i+2
// and the copies of tiles i+3.. overlap.  Every mbarrier wait is bounded and
// watches a block-wide abort flag: on timeout the block raises the device
// error word, waits (bounded) for its copies in flight, frees its TMEM and
// returns.
#include <cuda.h>

#include <cstring>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int NT = 576;          // 18 warps: producer, MMA, 8 converters, 8 epilogue
constexpr int TM = 128;          // M rows per tile: 64 beams x (re, im)
constexpr int TN = 256;          // frames per MMA tile
constexpr int CHUNK = 2048;      // frames per work item (one noise partial sum)
constexpr int TMEM_COLS = 512;   // two 256-column accumulators
constexpr long long WAIT_LIMIT = 1LL << 24;   // bounded mbarrier polls
constexpr int W_PROD = 0, W_MMA = 1, W_CONV0 = 2, N_CONV = 8, W_EPI0 = 10, N_EPI = 8;
constexpr int MAX_S8 = 3, MAX_SB = 2;
constexpr int STG_BOX = 16 * 128;             // staged output box: 16 beams x 16 frames x 8 B
constexpr int STG_BYTES = N_EPI * 2 * STG_BOX; // two boxes per epilogue warp

__host__ __device__ constexpr int kpad(int S) { return (2 * S + 15) / 16 * 16; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   smem_u32(dst)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar)));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups; descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B FP16
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Byte offset of element (row, kd) in a K-major no-swizzle tile of KP columns.
__host__ __device__ inline uint32_t core_off(int row, int kd, int KP) {
  return (uint32_t)((row >> 3) * (KP / 8) * 128 + (kd >> 3) * 128 + (row & 7) * 16 + (kd & 7) * 2);
}

// Eight int8 samples -> eight FP16 (exact): byte b -> bits 0x6400 | (b ^ 0x80)
// = 1024 + b + 128, then minus 1152 (0x6480).
__device__ __forceinline__ uint4 i8x8_to_f16x8(uint2 q) {
  const uint32_t u0 = q.x ^ 0x80808080u, u1 = q.y ^ 0x80808080u;
  const uint32_t r[4] = {__byte_perm(u0, 0x64646464u, 0x4140), __byte_perm(u0, 0x64646464u, 0x4342),
                         __byte_perm(u1, 0x64646464u, 0x4140), __byte_perm(u1, 0x64646464u, 0x4342)};
  const __half2 bias = __half2half2(__ushort_as_half((unsigned short)0x6480));
  uint32_t o[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&r[i]), bias);
    o[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// Eight int16 samples (16 bytes) -> the FP16 images of 256 h and of l,
// v = 256 h + l: the high byte h as above (then times 256, exact), the low
// byte l (0..255) as 1024 + l minus 1024.
__device__ __forceinline__ void i16x8_to_f16x8x2(uint4 q, uint4& hi, uint4& lo) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  const __half2 b_hi = __half2half2(__ushort_as_half((unsigned short)0x6480));
  const __half2 b_lo = __half2half2(__ushort_as_half((unsigned short)0x6400));
  const __half2 s256 = __half2half2(__ushort_as_half((unsigned short)0x5C00));
  uint32_t oh[4], ol[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t ph = __byte_perm(w[i] ^ 0x80808080u, 0x64646464u, 0x4341);
    const uint32_t pl = __byte_perm(w[i], 0x64646464u, 0x4240);
    const __half2 h = __hmul2(__hsub2(*reinterpret_cast<const __half2*>(&ph), b_hi), s256);
    const __half2 l = __hsub2(*reinterpret_cast<const __half2*>(&pl), b_lo);
    oh[i] = *reinterpret_cast<const uint32_t*>(&h);
    ol[i] = *reinterpret_cast<const uint32_t*>(&l);
  }
  hi = make_uint4(oh[0], oh[1], oh[2], oh[3]);
  lo = make_uint4(ol[0], ol[1], ol[2], ol[3]);
}

// A-operand images: [k][beam tile][hi/lo][TM x KP] FP16 in the layout above.
__global__ void k_weights_tc(const float2* __restrict__ w32, int K, int B, int S, int n_mt,
                             __half* __restrict__ wtc) {
  const int KP = kpad(S);
  const long long per_tile = (long long)TM * KP;
  const long long total = (long long)K * n_mt * per_tile;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kd = (int)(i % KP);
    const int row = (int)((i / KP) % TM);
    const long long km = i / per_tile;          // k * n_mt + mt
    const int mt = (int)(km % n_mt);
    const int k = (int)(km / n_mt);
    const int b = mt * (TM / 2) + (row >> 1);
    float val = 0.f;
    if (b < B && kd < 2 * S) {
      const float2 w = w32[((long long)k * B + b) * S + (kd >> 1)];
      const int comp = row & 1, c = kd & 1;
      val = comp == 0 ? (c == 0 ? w.x : -w.y) : (c == 0 ? w.y : w.x);
    }
    const __half hi = __float2half_rn(val);
    const __half lo = __float2half_rn(val - __half2float(hi));
    __half* base = wtc + km * 2 * per_tile;
    const uint32_t off = core_off(row, kd, KP) / 2;
    base[off] = hi;
    base[per_tile + off] = lo;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// TMA store of one staged box to the beam rows (5-D map [beam][trial][pol][k][frame]).
__device__ __forceinline__ void tma_store_box(const CUtensorMap* map, const void* src, int frame,
                                              int k, int pol, int t, int beam) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(frame), "r"(k), "r"(pol), "r"(t), "r"(beam), "r"(smem_u32(src))
      : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// At most N committed bulk stores may still be reading shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// Bounded wait on an mbarrier phase; gives up when the block aborts.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  long long polls = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (++polls > WAIT_LIMIT) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// Per-plan part of a launch: the plan's input view, weights, tables and
// outputs.  One launch serves one plan, or a group of plans (lp_group) on
// different subband ranges and beams of one station block.
struct TcPlan {
  const int8_t* x;          // pol slabs [K][F][S][2] (int8 or int16), pol_stride complex samples apart
  long long pol_stride;
  const __half* wtc;        // A images
  const float2* dd;         // [K][Tr]
  float* power_part;        // [J][K][n_chunks]
  int K, B, Tr, n_mt;
  long long item_end;       // items of plans 0 .. this one
  long long km0;            // group-wide index of the plan's first (subband, beam tile)
};

struct TcArgs {
  int* err;                 // device error word (of the first plan)
  int S, P, n_chunks;
  long long F, row;         // frames of this launch, beam-row length (chunk + prefix)
  long long F_in, f_base;   // input frames per subband row, first input frame of the launch
  int chunk_base, n_chunks_total;   // noise-partial chunk index offset, chunks per block
  int write_beams, write_power;
  int pol0, npol;           // polarisations of this launch: pol0 .. pol0 + npol - 1
  long long n_items;
  int n_s8, n_sb;           // pipeline depths (int8 ring, FP16 ring)
  int n;                    // plans
  TcPlan pl[kMaxGroup];
  CUtensorMap maps[kMaxGroup];   // TMA map of each plan's beam rows
};

// The tile sequence every role walks: items [it0, it1) of the launch (plan 0's
// items, then plan 1's, ...), 256-frame tiles each.  GROUP = false: one plan
// (index 0 throughout; no plan lookups on the single-plan path).
template <bool GROUP>
struct TileSeq {
  long long it, it1, n0, f_hi, p_begin;
  int n_chunks, P, pidx;
  long long F;
  const TcArgs* a;
  __device__ void start(const TcArgs* args, int nc, int npol, long long f, long long b0,
                        long long b1) {
    a = args;
    it = b0; it1 = b1; n_chunks = nc; P = npol; F = f;
    pidx = 0;
    p_begin = 0;
    if (it < it1) set_item();
  }
  __device__ void set_item() {
    if constexpr (GROUP) {
      while (it >= a->pl[pidx].item_end) {
        p_begin = a->pl[pidx].item_end;
        ++pidx;
      }
    }
    const long long chunk = local() % n_chunks;
    n0 = chunk * CHUNK;
    f_hi = min(F, n0 + CHUNK);
  }
  __device__ long long local() const { return GROUP ? it - p_begin : it; }
  __device__ bool valid() const { return it < it1; }
  __device__ int chunk() const { return (int)(local() % n_chunks); }
  __device__ int pol() const { return (int)((local() / n_chunks) % P); }
  // (subband, beam tile) within the plan, and its group-wide index
  __device__ long long km() const { return local() / ((long long)n_chunks * P); }
  __device__ long long kmg() const {
    if constexpr (GROUP) return a->pl[pidx].km0 + km();
    return km();
  }
  __device__ bool last_of_item() const { return n0 + TN >= f_hi; }
  __device__ void next() {
    n0 += TN;
    if (n0 >= f_hi) {
      ++it;
      if (it < it1) set_item();
    }
  }
};

// X16: int16 input (two B images per stage: 256 h, then l).
template <bool GROUP, bool X16>
__global__ void __launch_bounds__(NT, 1) k_beamform_tc(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int ESZ = X16 ? 2 : 1;               // bytes per real sample value
  const int KP = kpad(a.S);
  const int nkg = KP / 8;
  const uint32_t a_bytes = TM * KP * 2;          // one of hi / lo
  const uint32_t img_bytes = TN * KP * 2;        // one FP16 B image
  const uint32_t b_bytes = img_bytes * ESZ;      // one B stage
  const uint32_t t8_bytes = TN * 2 * a.S * ESZ;  // input tile
  // output staging boxes, aligned to 1024 bytes of the shared window (128-byte swizzle)
  unsigned char* stg = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);
  unsigned char* sa = stg + STG_BYTES;           // A hi, A lo
  unsigned char* s8 = sa + 2 * a_bytes;          // int8 ring
  unsigned char* sbuf = s8 + a.n_s8 * t8_bytes;  // FP16 ring
  __shared__ uint64_t full8[MAX_S8], empty8[MAX_S8], fullB[MAX_SB], emptyB[MAX_SB];
  __shared__ uint64_t tfull[2], tempty[2], a_full, a_empty;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < a.n_s8; ++i) { mbar_init(&full8[i], 1); mbar_init(&empty8[i], 32 * N_CONV); }
    for (int i = 0; i < a.n_sb; ++i) { mbar_init(&fullB[i], 32 * N_CONV); mbar_init(&emptyB[i], 1); }
    for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], 32 * N_EPI); }
    mbar_init(&a_full, 1);
    mbar_init(&a_empty, 1);
    abort_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  volatile int* abort_p = &abort_flag;

  const long long per = (a.n_items + gridDim.x - 1) / gridDim.x;
  const long long it0 = blockIdx.x * per;
  const long long it1 = min(a.n_items, it0 + per);
  TileSeq<GROUP> q;
  q.start(&a, a.n_chunks, a.npol, a.F, it0, it1);
  // the current item's plan (plan 0 at a fixed parameter offset on the single-plan path)
  auto plan = [&]() -> const TcPlan& { return a.pl[GROUP ? q.pidx : 0]; };

  if (warp == W_PROD) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0, aph = 0;
      long long cur_km = -1;
      uint32_t issued = 0, last_par = 0;        // per stage: copy issued, its phase parity
      bool a_issued = false;
      for (; q.valid(); q.next()) {
        const TcPlan& pl = plan();
        const long long km = q.km(), kmg = q.kmg();
        if (kmg != cur_km) {
          if (cur_km >= 0) {
            if (!wait_phase(&a_empty, aph, abort_p)) break;
            aph ^= 1u;
          }
          mbar_expect_tx(&a_full, 2 * a_bytes);
          bulk_g2s(sa, pl.wtc + km * 2 * (long long)TM * KP, 2 * a_bytes, &a_full);
          a_issued = true;
          cur_km = kmg;
        }
        if (!wait_phase(&empty8[st], ph ^ 1u, abort_p)) break;
        const int k = (int)(km / pl.n_mt);
        const int nvalid = (int)min((long long)TN, q.f_hi - q.n0);
        const int8_t* src =
            pl.x + 2 * ESZ * ((q.pol() + a.pol0) * pl.pol_stride +
                              ((long long)k * a.F_in + a.f_base + q.n0) * a.S);
        const uint32_t bytes = (uint32_t)nvalid * 2 * ESZ * a.S;
        mbar_expect_tx(&full8[st], bytes);
        bulk_g2s(s8 + st * t8_bytes, src, bytes, &full8[st]);
        issued |= 1u << st;
        last_par = (last_par & ~(1u << st)) | (ph << st);
        if (++st == a.n_s8) { st = 0; ph ^= 1u; }
      }
      if (*abort_p) {
        // let the copies already issued land before the block's memory goes
        for (int i = 0; i < a.n_s8; ++i) {
          if (!((issued >> i) & 1u)) continue;
          long long polls = 0;
          while (!mbar_try_wait(&full8[i], (last_par >> i) & 1u) && ++polls < WAIT_LIMIT) {
          }
        }
        if (a_issued) {
          long long polls = 0;
          // the last A copy completes the a_full phase of parity aph
          while (!mbar_try_wait(&a_full, aph) && ++polls < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == W_MMA) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int sb = 0, acc = 0;
      uint32_t phb = 0, pha = 0, aph = 0;
      long long cur_km = -1;
      const uint32_t idesc = idesc_f16(TM, TN);
      const uint32_t sbo = nkg * 128;
      const uint32_t a0 = smem_u32(sa);
      int last_acc = -1;
      uint32_t last_par = 0;
      for (; q.valid(); q.next()) {
        const long long km = q.kmg();
        if (km != cur_km) {
          if (cur_km >= 0) mma_commit(&a_empty);   // old A free once its MMAs finish
          if (!wait_phase(&a_full, aph, abort_p)) break;
          aph ^= 1u;
          cur_km = km;
        }
        if (!wait_phase(&fullB[sb], phb, abort_p)) break;
        if (!wait_phase(&tempty[acc], pha ^ 1u, abort_p)) break;
        tc_fence_after();
        const uint32_t b0 = smem_u32(sbuf + sb * b_bytes);
        const uint32_t d = tmem + acc * TN;
        for (int ks = 0; ks < KP / 16; ++ks) {
#pragma unroll
          for (int im = 0; im < ESZ; ++im) {
            const uint64_t bd = smem_desc(b0 + im * img_bytes + ks * 256, 128, sbo);
            mma_f16(d, smem_desc(a0 + ks * 256, 128, sbo), bd, idesc, ks + im > 0 ? 1u : 0u);
            mma_f16(d, smem_desc(a0 + a_bytes + ks * 256, 128, sbo), bd, idesc, 1u);
          }
        }
        mma_commit(&emptyB[sb]);
        mma_commit(&tfull[acc]);
        last_acc = acc;
        last_par = pha;
        if (++sb == a.n_sb) { sb = 0; phb ^= 1u; }
        if (++acc == 2) { acc = 0; pha ^= 1u; }
      }
      if (last_acc >= 0) {
        // the tensor core must be done with shared and tensor memory before exit
        long long polls = 0;
        while (!mbar_try_wait(&tfull[last_acc], last_par) && ++polls < WAIT_LIMIT) {
        }
      }
    }
  } else if (warp < W_EPI0) {
    // ---------------- converters (N_CONV warps) ----------------
    const int cw = warp - W_CONV0;              // converter warp 0..N_CONV-1
    const int n_sub = lane & 7, c_sub = lane >> 3;
    const int n_cg = (nkg + 3) / 4;             // groups of four 8-sample K chunks
    int st = 0, sb = 0;
    uint32_t ph = 0, phb = 0;
    for (; q.valid(); q.next()) {
      if (!wait_phase(&full8[st], ph, abort_p)) break;
      if (!wait_phase(&emptyB[sb], phb ^ 1u, abort_p)) break;
      const unsigned char* src = s8 + st * t8_bytes;
      unsigned char* dst = sbuf + sb * b_bytes;
      // one step converts frames 8 ng + n_sub, K chunk 4 cg + c_sub (8 samples);
      // warp cw takes the frame groups ng = cw (mod N_CONV)
      for (int cg = 0; cg < n_cg; ++cg) {
        const int c = cg * 4 + c_sub;
        if (c >= nkg) continue;
        const bool in = 8 * c < 2 * a.S;        // K padding converts to zeros
        const unsigned char* sp = src + n_sub * (2 * ESZ * a.S) + 8 * ESZ * c;
        unsigned char* dp = dst + core_off(n_sub, 8 * c, KP);
        if constexpr (X16) {
#pragma unroll 4
          for (int ng = cw; ng < TN / 8; ng += N_CONV) {
            uint4 hi = make_uint4(0, 0, 0, 0), lo = hi;
            if (in) i16x8_to_f16x8x2(*reinterpret_cast<const uint4*>(sp + ng * 32 * a.S), hi, lo);
            *reinterpret_cast<uint4*>(dp + ng * (KP / 8) * 128) = hi;
            *reinterpret_cast<uint4*>(dp + img_bytes + ng * (KP / 8) * 128) = lo;
          }
        } else {
#pragma unroll 4
          for (int ng = cw; ng < TN / 8; ng += N_CONV) {
            uint4 h8 = make_uint4(0, 0, 0, 0);
            if (in) h8 = i8x8_to_f16x8(*reinterpret_cast<const uint2*>(sp + ng * 16 * a.S));
            *reinterpret_cast<uint4*>(dp + ng * (KP / 8) * 128) = h8;
          }
        }
      }
      fence_proxy_async();
      mbar_arrive(&fullB[sb]);
      mbar_arrive(&empty8[st]);
      if (++st == a.n_s8) { st = 0; ph ^= 1u; }
      if (++sb == a.n_sb) { sb = 0; phb ^= 1u; }
    }
  } else {
    // ---------------- epilogue (256 threads) ----------------
    const int ew = warp - W_EPI0;               // 0..7
    const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31
    const int col_half = ew >> 2;
    const int rb = (quarter * 32 + lane) >> 1;  // beam in tile
    const bool odd = lane & 1;
    int acc = 0;
    uint32_t pha = 0;
    float pw = 0.f;
    for (; q.valid(); q.next()) {
      if (!wait_phase(&tfull[acc], pha, abort_p)) break;
      tc_fence_after();
      const int pol = q.pol() + a.pol0;
      const TcPlan& pl = plan();
      const CUtensorMap* out_map = &a.maps[GROUP ? q.pidx : 0];
      const long long km = q.km();
      const int k = (int)(km / pl.n_mt), mt = (int)(km % pl.n_mt);
      const int b = mt * (TM / 2) + rb;
      const bool beam_ok = b < pl.B;
      const long long f_hi = q.f_hi, n0 = q.n0;
      const uint32_t lane_addr =
          tmem + acc * TN + ((uint32_t)(quarter * 32) << 16) + col_half * (TN / 2);
      const float2 d0 = pl.dd[k * pl.Tr];
      const int rloc = lane >> 1;                // beam row inside the warp's 16-beam box
      for (int c0 = 0; c0 < TN / 2; c0 += 32) {
        uint32_t r[2][16];
        tmem_ld16(lane_addr + c0, r[0]);
        tmem_ld16(lane_addr + c0 + 16, r[1]);
        tmem_ld_wait();
        // both 16-frame boxes of the 32-column step are staged, then one proxy
        // fence and one warp sync cover both TMA stores (the fences, not the
        // stores, were the epilogue's cost)
        float2 bvh[2][8];
        long long fbh[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float recv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            recv[i] = __shfl_xor_sync(0xffffffffu,
                                      __uint_as_float(odd ? r[h][i] : r[h][i + 8]), 1);
          const long long fb = n0 + col_half * (TN / 2) + c0 + 16 * h;
          fbh[h] = fb;
          // frames of this lane's half inside the launch: all 8 except in the
          // last tile of an item (warp-uniform test first); partials of beams
          // beyond B are never stored
          const int nin = fb + 16 <= f_hi ? 8 : (int)max(0LL, min(8LL, f_hi - fb - (odd ? 8 : 0)));
#pragma unroll
          for (int i = 0; i < 8; ++i) {   // even lane: (Re, Im) of frames 0-7, odd: 8-15
            bvh[h][i] = odd ? make_float2(recv[i], __uint_as_float(r[h][i + 8]))
                            : make_float2(__uint_as_float(r[h][i]), recv[i]);
            if (i < nin) pw = fmaf(bvh[h][i].x, bvh[h][i].x, fmaf(bvh[h][i].y, bvh[h][i].y, pw));
          }
        }
        if (fbh[0] < f_hi && a.write_beams) {
          for (int t = 0; t < pl.Tr; ++t) {
            const float2 dv = t == 0 ? d0 : pl.dd[k * pl.Tr + t];
            if (lane == 0) bulk_wait_read<0>();   // earlier stores have read both boxes
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; ++h) {       // 16-byte chunk c of row rloc, 128B swizzle
              unsigned char* box = stg + (ew * 2 + h) * STG_BOX;
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float2 u = bvh[h][2 * i], w = bvh[h][2 * i + 1];
                const int c = (odd ? 4 : 0) + i;
                *reinterpret_cast<float4*>(box + rloc * 128 + ((c ^ (rloc & 7)) << 4)) =
                    make_float4(dv.x * u.x - dv.y * u.y, dv.x * u.y + dv.y * u.x,
                                dv.x * w.x - dv.y * w.y, dv.x * w.y + dv.y * w.x);
              }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
              tma_store_box(out_map, stg + (ew * 2) * STG_BOX, (int)(kPrefix + fbh[0]), k, pol,
                            t, mt * (TM / 2) + quarter * 16);
              if (fbh[1] < f_hi)
                tma_store_box(out_map, stg + (ew * 2 + 1) * STG_BOX, (int)(kPrefix + fbh[1]), k,
                              pol, t, mt * (TM / 2) + quarter * 16);
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      if (++acc == 2) { acc = 0; pha ^= 1u; }
      if (q.last_of_item()) {
        // noise partial of the chunk and column half: lanes 2r, 2r+1 hold the
        // two halves of beam rb; k_sigma adds the two column halves
        pw += __shfl_xor_sync(0xffffffffu, pw, 1);
        if (beam_ok && !odd && a.write_power) {
          for (int t = 0; t < pl.Tr; ++t) {
            const long long j = ((long long)b * pl.Tr + t) * a.P + pol;
            pl.power_part[(j * pl.K + k) * (2LL * a.n_chunks_total) +
                         2 * (a.chunk_base + q.chunk()) + col_half] = pw;
          }
        }
        pw = 0.f;
      }
    }
    if (lane == 0) bulk_wait_all();     // staged boxes read and written before exit
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 152;
}

}  // namespace

int beamform_tc_frame_tile() { return TN; }
// noise partials per (stream, subband): two column halves per 2048-frame chunk
int beamform_tc_partials(long long F) { return 2 * (int)((F + CHUNK - 1) / CHUNK); }

size_t beamform_tc_weight_bytes(const Shape& sh) {
  const int n_mt = (sh.B + TM / 2 - 1) / (TM / 2);
  return (size_t)sh.K * n_mt * 2 * TM * kpad(sh.S) * sizeof(__half);
}

cudaError_t launch_weights_tc(const lp_plan& p, cudaStream_t s) {
  const auto& sh = p.shape;
  const int n_mt = (sh.B + TM / 2 - 1) / (TM / 2);
  const long long total = (long long)sh.K * n_mt * TM * kpad(sh.S);
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
  k_weights_tc<<<blocks, 256, 0, s>>>(p.buf.w32, sh.K, sh.B, sh.S, n_mt, p.buf.wtc);
  return cudaGetLastError();
}

// Pipeline depths that fit the 227 KB of shared memory: A (hi + lo), input
// stages, FP16 stages; esz = bytes per real input value (1: int8, 2: int16).
void tc_depths(const Shape& sh, int esz, int* n_s8, int* n_sb) {
  const size_t limit = 227 * 1024 - 2048 - STG_BYTES - 1024;
  const size_t KP = kpad(sh.S);
  const size_t a = 2 * TM * KP * 2, t8 = (size_t)TN * 2 * sh.S * esz, b = TN * KP * 2 * esz;
  *n_sb = a + 2 * b + t8 <= limit ? 2 : 1;
  *n_s8 = 1;
  while (*n_s8 < MAX_S8 && a + *n_sb * b + (*n_s8 + 1) * t8 <= limit) ++*n_s8;
}

// 5-D map of the beam rows for the epilogue's TMA stores: element = one complex
// FP32 (8 bytes); dims (frame position, k, pol, trial, beam); box 16 x 1 x 1 x 1 x 16
// with 128-byte swizzle.
cudaError_t encode_beams_map(lp_plan& p) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<Encode>(fn);
  }
  const auto& sh = p.shape;
  const cuuint64_t row = (cuuint64_t)p.row() * 8;
  const cuuint64_t dims[5] = {(cuuint64_t)p.row(), (cuuint64_t)sh.K, (cuuint64_t)sh.P,
                              (cuuint64_t)sh.Tr, (cuuint64_t)sh.B};
  const cuuint64_t strides[4] = {row, row * sh.K, row * sh.K * sh.P, row * sh.K * sh.P * sh.Tr};
  const cuuint32_t box[5] = {16, 1, 1, 1, 16};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = encode(reinterpret_cast<CUtensorMap*>(p.beams_map),
                            CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, p.buf.beams, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t tc_smem_for(const Shape& sh, int esz, int n8, int nb) {
  const size_t KP = kpad(sh.S);
  // at least 120 KB: one block per SM (it takes all 512 TMEM columns)
  return std::max<size_t>(1024 + STG_BYTES + 2 * TM * KP * 2 + (size_t)n8 * TN * 2 * sh.S * esz +
                              (size_t)nb * TN * KP * 2 * esz,
                          120 * 1024);
}

// (input stages, FP16 stages) that fit the shared memory, deepest first
int tc_configs(const Shape& sh, int esz, int* desc, int max) {
  const size_t limit = 227 * 1024 - 2048 - STG_BYTES - 1024;
  const size_t KP = kpad(sh.S);
  const size_t a = 2 * TM * KP * 2, t8 = (size_t)TN * 2 * sh.S * esz, b = TN * KP * 2 * esz;
  int n = 0;
  for (int nb = MAX_SB; nb >= 1; --nb)
    for (int n8 = MAX_S8; n8 >= 1; --n8)
      if (a + nb * b + n8 * t8 <= limit && n < max) {
        desc[2 * n] = n8;
        desc[2 * n + 1] = nb;
        ++n;
      }
  return n;
}

size_t tc_smem(const Shape& sh, int esz) {  // the largest configuration
  int desc[2 * MAX_S8 * MAX_SB];
  const int n = tc_configs(sh, esz, desc, MAX_S8 * MAX_SB);
  size_t m = 0;
  for (int i = 0; i < n; ++i)
    m = std::max(m, tc_smem_for(sh, esz, desc[2 * i], desc[2 * i + 1]));
  return m;
}

cudaError_t init_tc_attributes(const Shape& sh) {
  cudaError_t e = raise_smem_limit((const void*)k_beamform_tc<false, false>, tc_smem(sh, 1));
  if (e == cudaSuccess) e = raise_smem_limit((const void*)k_beamform_tc<true, false>, tc_smem(sh, 1));
  if (e == cudaSuccess) e = raise_smem_limit((const void*)k_beamform_tc<false, true>, tc_smem(sh, 2));
  if (e == cudaSuccess) e = raise_smem_limit((const void*)k_beamform_tc<true, true>, tc_smem(sh, 2));
  return e;
}

// Plans plans[0..n) (same stations, polarisations, block length and chunking;
// the first plan's ring depths), plan i reading its pol slabs at xs[i], in one
// launch.
cudaError_t launch_beamform_tc_plans(const lp_plan* const* plans, const void* const* xs,
                                     long long pol_stride, int n, const Chunk& c, cudaStream_t s,
                                     PolSel ps) {
  const lp_plan& p0 = *plans[0];
  const auto& sh = p0.shape;
  TcArgs a;
  a.err = p0.buf.err;
  a.S = sh.S;
  a.P = sh.P;
  a.n_chunks = (int)((c.nf + CHUNK - 1) / CHUNK);
  a.F = c.nf;
  a.row = p0.row();
  a.F_in = sh.F;
  a.f_base = c.f_base;
  a.chunk_base = (int)(c.f_base / CHUNK);
  a.n_chunks_total = (int)((sh.F + CHUNK - 1) / CHUNK);
  a.write_beams = c.write_beams ? 1 : 0;
  a.write_power = c.write_power ? 1 : 0;
  a.pol0 = ps.pol0;
  a.npol = ps.npol ? ps.npol : sh.P;
  a.n = n;
  long long items = 0, kms = 0;
  for (int i = 0; i < n; ++i) {
    const lp_plan& p = *plans[i];
    TcPlan& q = a.pl[i];
    q.x = static_cast<const int8_t*>(xs[i]);
    q.pol_stride = pol_stride;
    q.wtc = p.buf.wtc;
    q.dd = p.buf.dd;
    q.power_part = p.buf.power_part;
    q.K = p.shape.K;
    q.B = p.shape.B;
    q.Tr = p.shape.Tr;
    q.n_mt = (p.shape.B + TM / 2 - 1) / (TM / 2);
    q.km0 = kms;
    kms += (long long)q.K * q.n_mt;
    items += (long long)q.K * q.n_mt * a.npol * a.n_chunks;
    q.item_end = items;
    std::memcpy(&a.maps[i], p.beams_map, sizeof(CUtensorMap));
  }
  a.n_items = items;
  const bool x16 = p0.cfg.input_dtype == LP_INPUT_INT16;
  const int esz = x16 ? 2 : 1;
  tc_depths(sh, esz, &a.n_s8, &a.n_sb);
  if (p0.gemm_cfg >= 0) {                      // autotuned depths
    int desc[2 * MAX_S8 * MAX_SB];
    const int nc = tc_configs(sh, esz, desc, MAX_S8 * MAX_SB);
    if (p0.gemm_cfg < nc) {
      a.n_s8 = desc[2 * p0.gemm_cfg];
      a.n_sb = desc[2 * p0.gemm_cfg + 1];
    }
  }
  const long long grid = std::min<long long>(a.n_items, (long long)num_sms());
  const size_t smem = tc_smem_for(sh, esz, a.n_s8, a.n_sb);
  if (n == 1 && !x16)
    k_beamform_tc<false, false><<<(unsigned)grid, NT, smem, s>>>(a);
  else if (!x16)
    k_beamform_tc<true, false><<<(unsigned)grid, NT, smem, s>>>(a);
  else if (n == 1)
    k_beamform_tc<false, true><<<(unsigned)grid, NT, smem, s>>>(a);
  else
    k_beamform_tc<true, true><<<(unsigned)grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_beamform_tc(const lp_plan& p, const void* x, long long pol_stride,
                               const Chunk& c, cudaStream_t s, PolSel ps) {
  const lp_plan* one = &p;
  return launch_beamform_tc_plans(&one, &x, pol_stride, 1, c, s, ps);
}

}  // namespace lp
