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
// would leave ~1.5e-4 relative error in the beams).
//
// Work items: (subband k, beam tile of 64 beams, pol, chunk of 2048 frames).
// A persistent grid of 2 blocks per SM walks contiguous item ranges, so the
// A tiles (hi and lo, 128 x 2S FP16 each, pre-arranged by k_weights_tc) are
// loaded once per (k, beam tile).  Per 256-frame tile: 128 threads convert the
// int8 samples (256 frames x 2S contiguous bytes, fetched into registers while
// the previous tile's MMA and epilogue ran) into the canonical K-major,
// no-swizzle FP16 layout (8-row x 16-byte core matrices), one thread issues
// 2 * 2S/16 tcgen05.mma (M = 128, N = 256, K = 16, FP32 accumulator in 256
// TMEM columns) and commits to an mbarrier; then the eight warps (two per
// 32-lane TMEM quarter, one per column half) read TMEM with tcgen05.ld, pair
// Re/Im lanes by shuffle, multiply by D[k,t] and write 64-byte runs of the
// [stream][k][frame] beam rows.
// Every mbarrier wait is bounded: on timeout the block raises the device
// error word, frees its TMEM and returns.
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int NT = 256;          // threads per block: 2 warps per 32-lane TMEM quarter
constexpr int TM = 128;          // M rows per tile: 64 beams x (re, im)
constexpr int TN = 256;          // frames per MMA tile
constexpr int CHUNK = 2048;      // frames per work item (one noise partial sum)
constexpr int TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1LL << 22;   // bounded mbarrier polls
constexpr int MAXR = TN * 16 / NT;             // prefetch entries per thread (2S <= 128)

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

struct TcArgs {
  const int8_t* x;          // pol slabs [K][F][S][2], pol_stride complex samples apart
  long long pol_stride;
  const __half* wtc;        // A images
  const float2* dd;         // [K][Tr]
  float2* beams;            // [J][K][row]
  float* power_part;        // [J][K][n_chunks]
  int* err;                 // device error word
  int S, P, K, B, Tr, n_mt, n_chunks;
  long long F, row;
  long long n_items;
};

__global__ void __launch_bounds__(NT, 2) k_beamform_tc(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int KP = kpad(a.S);
  const int nkg = KP / 8;
  const uint32_t a_bytes = TM * KP * 2;          // one of hi / lo
  const uint32_t b_bytes = TN * KP * 2;
  unsigned char* sa = smem;                      // hi, then lo
  unsigned char* sb = smem + 2 * a_bytes;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float pw_half[2][TM / 2];   // noise partials of the two column halves

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);
  if (tid == 0) mbar_init(&mbar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_f16(TM, TN);
  uint32_t phase = 0;

  const long long per = (a.n_items + gridDim.x - 1) / gridDim.x;
  const long long it0 = blockIdx.x * per;
  const long long it1 = min(a.n_items, it0 + per);
  long long cur_km = -1;

  // accumulator row of this thread (TMEM lane quarter warp & 3) and the half
  // of the 256 columns it drains (warp >> 2); beam-in-tile rb, Re/Im = lane & 1
  const int quarter = warp & 3, col_half = warp >> 2;
  const int trow = quarter * 32 + lane;
  const int rb = trow >> 1;
  const bool odd = lane & 1;

  // Samples of the next tile, loaded into registers while the current tile's
  // MMA and epilogue run: 8 int8 (one core-matrix row) per entry.
  uint2 q[MAXR];
  auto prefetch = [&](long long it, long long n0) {
    const int chunk = (int)(it % a.n_chunks);
    const int pol = (int)((it / a.n_chunks) % a.P);
    const int k = (int)((it / ((long long)a.n_chunks * a.P)) / a.n_mt);
    const long long f_hi = min(a.F, (long long)(chunk + 1) * CHUNK);
    const int nvalid = (int)min((long long)TN, f_hi - n0);
    const int8_t* xk = a.x + 2 * (pol * a.pol_stride + ((long long)k * a.F + n0) * a.S);
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      const int e = tid + NT * r;
      const int c = e / TN, n = e - c * TN;   // 8 consecutive threads: 8 rows
      q[r] = make_uint2(0, 0);
      if (e < TN * nkg && n < nvalid && 8 * c < 2 * a.S)
        q[r] = __ldg(reinterpret_cast<const uint2*>(xk + n * (2LL * a.S) + 8 * c));
    }
  };

  long long it = it0;
  long long n0 = it < it1 ? (long long)(it % a.n_chunks) * CHUNK : 0;
  if (it < it1) prefetch(it, n0);
  float pw = 0.f;
  while (it < it1) {
    const int chunk = (int)(it % a.n_chunks);
    const int pol = (int)((it / a.n_chunks) % a.P);
    const long long km = it / ((long long)a.n_chunks * a.P);
    const int mt = (int)(km % a.n_mt);
    const int k = (int)(km / a.n_mt);
    const long long f_hi = min(a.F, (long long)(chunk + 1) * CHUNK);
    const int b = mt * (TM / 2) + rb;
    const bool beam_ok = b < a.B;
    if (km != cur_km) {
      // A images of (k, mt): 2 * a_bytes contiguous bytes -> shared memory
      const uint4* src = reinterpret_cast<const uint4*>(a.wtc + km * 2 * (long long)TM * KP);
      uint4* dst = reinterpret_cast<uint4*>(sa);
      for (uint32_t i = tid; i < 2 * a_bytes / 16; i += NT) dst[i] = src[i];
      cur_km = km;
    }
    // 1. int8 samples -> FP16 K-major core-matrix layout
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      const int e = tid + NT * r;
      if (e < TN * nkg) {
        const int c = e / TN, n = e - c * TN;
        const char4 lo4 = *reinterpret_cast<const char4*>(&q[r].x);
        const char4 hi4 = *reinterpret_cast<const char4*>(&q[r].y);
        __half2 p0 = __floats2half2_rn((float)lo4.x, (float)lo4.y);
        __half2 p1 = __floats2half2_rn((float)lo4.z, (float)lo4.w);
        __half2 p2 = __floats2half2_rn((float)hi4.x, (float)hi4.y);
        __half2 p3 = __floats2half2_rn((float)hi4.z, (float)hi4.w);
        *reinterpret_cast<uint4*>(sb + core_off(n, 8 * c, KP)) =
            make_uint4(*reinterpret_cast<uint32_t*>(&p0), *reinterpret_cast<uint32_t*>(&p1),
                       *reinterpret_cast<uint32_t*>(&p2), *reinterpret_cast<uint32_t*>(&p3));
      }
    }
    fence_proxy_async();
    __syncthreads();
    // 2. one thread issues the MMAs: hi and lo weights against the same samples
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
      const uint32_t sbo = nkg * 128;
      for (int ks = 0; ks < KP / 16; ++ks) {
        const uint64_t bd = smem_desc(b0 + ks * 256, 128, sbo);
        mma_f16(tmem, smem_desc(a0 + ks * 256, 128, sbo), bd, idesc, ks > 0 ? 1u : 0u);
        mma_f16(tmem, smem_desc(a0 + a_bytes + ks * 256, 128, sbo), bd, idesc, 1u);
      }
      mma_commit(&mbar);
    }
    // 3. next tile's samples into registers (in flight during the MMA and epilogue)
    long long nit = it, nn0 = n0 + TN;
    if (nn0 >= f_hi) {
      nit = it + 1;
      nn0 = (long long)(nit % a.n_chunks) * CHUNK;
    }
    if (nit < it1) prefetch(nit, nn0);
    // 4. wait for the accumulator (bounded)
    bool failed = false;
    long long polls = 0;
    while (!mbar_try_wait(&mbar, phase)) {
      if (++polls > WAIT_LIMIT) {
        failed = true;
        break;
      }
    }
    phase ^= 1u;
    failed = __syncthreads_or(failed) != 0;   // every thread takes the same branch
    if (failed) {
      if (tid == 0) atomicExch(a.err, 1);
      break;
    }
    tc_fence_after();
    // 5. epilogue: this warp's 128 columns, 32 per TMEM wait; per 16 columns the
    //    even lane writes frames 0-7 and the odd lane frames 8-15
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + col_half * (TN / 2);
    const float2 d0 = a.dd[k * a.Tr];
    for (int c0 = 0; c0 < TN / 2; c0 += 32) {
      uint32_t r[2][16];
      tmem_ld16(lane_addr + c0, r[0]);
      tmem_ld16(lane_addr + c0 + 16, r[1]);
      tmem_ld_wait();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float recv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)   // even lane sends Re 8-15, odd lane sends Im 0-7
          recv[i] = __shfl_xor_sync(0xffffffffu,
                                    __uint_as_float(odd ? r[h][i] : r[h][i + 8]), 1);
        const long long f0 = n0 + col_half * (TN / 2) + c0 + 16 * h + (odd ? 8 : 0);
        if (beam_ok && f0 < f_hi) {
          float2 bv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            bv[i] = odd ? make_float2(recv[i], __uint_as_float(r[h][i + 8]))
                        : make_float2(__uint_as_float(r[h][i]), recv[i]);
            if (f0 + i < f_hi) pw = fmaf(bv[i].x, bv[i].x, fmaf(bv[i].y, bv[i].y, pw));
          }
          const bool full = f0 + 8 <= f_hi;
          for (int t = 0; t < a.Tr; ++t) {
            const float2 d = t == 0 ? d0 : a.dd[k * a.Tr + t];
            const long long j = ((long long)b * a.Tr + t) * a.P + pol;
            float2* dst = a.beams + (j * a.K + k) * a.row + kPrefix + f0;
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              v[i] = make_float2(d.x * bv[i].x - d.y * bv[i].y, d.x * bv[i].y + d.y * bv[i].x);
            if (full) {
              float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
              for (int i = 0; i < 4; ++i)
                d4[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
            } else {
              for (int i = 0; i < 8 && f0 + i < f_hi; ++i) dst[i] = v[i];
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // TMEM drained and B tile free before the next tile
    if (nit != it) {
      // noise partial of the finished chunk: lanes 2r, 2r+1 of the two column
      // halves hold the four parts of beam rb; two-term sums are order-free
      pw += __shfl_xor_sync(0xffffffffu, pw, 1);
      if (!odd) pw_half[col_half][rb] = pw;
      __syncthreads();
      if (beam_ok && !odd && col_half == 0) {
        const float tot = pw_half[0][rb] + pw_half[1][rb];
        for (int t = 0; t < a.Tr; ++t) {
          const long long j = ((long long)b * a.Tr + t) * a.P + pol;
          a.power_part[(j * a.K + k) * a.n_chunks + chunk] = tot;
        }
      }
      pw = 0.f;
    }
    it = nit;
    n0 = nn0;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 152;
}

}  // namespace

int beamform_tc_frame_tile() { return CHUNK; }

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

size_t tc_smem(const Shape& sh) {
  // at least 80 KB so that no more than two blocks (2 x 256 TMEM columns) share an SM
  return std::max<size_t>((size_t)(2 * TM + TN) * kpad(sh.S) * 2, 80 * 1024);
}

cudaError_t init_tc_attributes(const Shape& sh) {
  return cudaFuncSetAttribute(k_beamform_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem(sh));
}

cudaError_t launch_beamform_tc(const lp_plan& p, const void* x, long long pol_stride,
                               cudaStream_t s) {
  const auto& sh = p.shape;
  TcArgs a;
  a.x = static_cast<const int8_t*>(x);
  a.pol_stride = pol_stride;
  a.wtc = p.buf.wtc;
  a.dd = p.buf.dd;
  a.beams = p.buf.beams;
  a.power_part = p.buf.power_part;
  a.err = p.buf.err;
  a.S = sh.S;
  a.P = sh.P;
  a.K = sh.K;
  a.B = sh.B;
  a.Tr = sh.Tr;
  a.n_mt = (sh.B + TM / 2 - 1) / (TM / 2);
  a.n_chunks = (int)((sh.F + CHUNK - 1) / CHUNK);
  a.F = sh.F;
  a.row = sh.row();
  a.n_items = (long long)sh.K * a.n_mt * sh.P * a.n_chunks;
  const long long grid = std::min<long long>(a.n_items, 2LL * num_sms());
  k_beamform_tc<<<(unsigned)grid, NT, tc_smem(sh), s>>>(a);
  return cudaGetLastError();
}

}  // namespace lp
