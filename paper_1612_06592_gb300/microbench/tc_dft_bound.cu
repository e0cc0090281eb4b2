// Lower bound of the inverse DFT on the 5th-generation tensor cores.
//
// The synthesis kernel's 1024-point inverse DFT is two 32-point stages
// (k = 32 k1 + k2, p = p1 + 32 p2; 16 nonzero k1 because the selected bins lie
// below 512).  On tcgen05 each stage is a GEMM with the DFT matrix as the
// shared operand, frames as the M dimension and the complex values in real
// form:
//   stage 1, per k2:  [128 frames x 32 (k1 re/im)] x [32 x 64 (p1 re/im)],
//   stage 2, per p1:  [128 frames x 64 (k2 re/im)] x [64 x 64 (p2 re/im)]
// (the twiddle exp(2 pi i k2 p1 / 1024) folded into the stage-2 matrix of each
// p1).  FP16 operands need a high and a low part of data and matrix (three
// products) to keep the FP32-level accuracy the pipeline states, so a tile of
// 128 frames of one stream takes 32 x 2 x 3 + 32 x 4 x 3 = 576 MMAs of
// M = 128, N = 64, K = 16.
//
// This kernel issues exactly that MMA sequence, operands read from shared
// memory, accumulators in tensor memory, and nothing else: no loads of data,
// no conversions into FP16 parts, no twiddles, no transposes, no epilogue.
// Its time is therefore a lower bound on any tensor-core form of the two
// stages.  A second shape (N = 256, the same FLOP in a quarter of the MMAs)
// shows how much of that time the narrow N of the DFT costs.  One block per
// SM, one thread issues; every wait is bounded and reports through *err.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int TMEM_COLS = 512;
constexpr long long WAIT_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no-swizzle shared-memory matrix descriptor (8-row x 16-byte core
// matrices; lbo: step between the two core matrices of a K = 16 slice, sbo:
// step between 8-row groups; descriptor version 1 at bit 46).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, FP16 A and B, K-major.
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar)));
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Shared-memory layout: 3 data tiles (hi and lo parts, 128 rows x 64 K each =
// 16 KB per part), the stage-1 and stage-2 matrices (hi and lo), each K = 16
// slice of a tile stored as its own run of core matrices.
constexpr int A_PART = 128 * 64 * 2;          // 16 KB: 128 rows x 64 K
constexpr int A_TILES = 3;
constexpr int B1_PART = 64 * 32 * 2;          // stage 1: 64 N x 32 K
constexpr int B2_PART = 64 * 64 * 2;          // stage 2: 64 N x 64 K
constexpr int BW_PART = 256 * 64 * 2;         // the N = 256 comparison shape
constexpr int SMEM = A_TILES * 2 * A_PART + 2 * B1_PART + 2 * B2_PART + 2 * BW_PART + 1024;

// Byte offset of K-slice ks of a tile part with `rows` rows.
__device__ __forceinline__ uint32_t slice(int rows, int ks) { return (uint32_t)(ks * rows * 32); }

// shape 0: the DFT sequence (576 MMAs of N = 64 per tile); shape 1: the same
// FLOP as 144 MMAs of N = 256.
__global__ void __launch_bounds__(128, 1) k_tc_dft_bound(int shape, int tiles, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* base = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (SMEM - 1024) / 16; i += 128)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&done)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // zeros visible to the MMAs
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t a0 = smem_u32(base);
  const uint32_t b1 = a0 + A_TILES * 2 * A_PART;
  const uint32_t b2 = b1 + 2 * B1_PART;
  const uint32_t bw = b2 + 2 * B2_PART;
  if (tid == 0) {
    const uint32_t id64 = idesc(128, 64), id256 = idesc(128, 256);
    int a_t = 0;
    for (int t = 0; t < tiles; ++t) {
      if (shape == 0) {
        // stage 1: per k2, K = 32 (two slices), three products
        for (int k2 = 0; k2 < 32; ++k2) {
          const uint32_t ah = a0 + (uint32_t)(a_t * 2 * A_PART), al = ah + A_PART;
          const uint32_t d = tmem + (uint32_t)((k2 & 7) * 64);
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t bh = sdesc(b1 + slice(64, ks), 128, 256);
            const uint64_t bl = sdesc(b1 + B1_PART + slice(64, ks), 128, 256);
            mma(d, sdesc(ah + slice(128, ks), 128, 256), bh, id64, ks > 0);
            mma(d, sdesc(ah + slice(128, ks), 128, 256), bl, id64, 1);
            mma(d, sdesc(al + slice(128, ks), 128, 256), bh, id64, 1);
          }
          a_t = a_t + 1 == A_TILES ? 0 : a_t + 1;
        }
        // stage 2: per p1, K = 64 (four slices), three products
        for (int p1 = 0; p1 < 32; ++p1) {
          const uint32_t ah = a0 + (uint32_t)(a_t * 2 * A_PART), al = ah + A_PART;
          const uint32_t d = tmem + (uint32_t)((p1 & 7) * 64);
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t bh = sdesc(b2 + slice(64, ks), 128, 256);
            const uint64_t bl = sdesc(b2 + B2_PART + slice(64, ks), 128, 256);
            mma(d, sdesc(ah + slice(128, ks), 128, 256), bh, id64, ks > 0);
            mma(d, sdesc(ah + slice(128, ks), 128, 256), bl, id64, 1);
            mma(d, sdesc(al + slice(128, ks), 128, 256), bh, id64, 1);
          }
          a_t = a_t + 1 == A_TILES ? 0 : a_t + 1;
        }
      } else {
        // the same FLOP per tile with N = 256: 48 groups of three K = 16 products
        for (int g = 0; g < 48; ++g) {
          const uint32_t ah = a0 + (uint32_t)(a_t * 2 * A_PART), al = ah + A_PART;
          const uint32_t d = tmem + (uint32_t)((g & 1) * 256);
          const int ks = g & 3;
          const uint64_t bh = sdesc(bw + slice(256, ks), 128, 256);
          const uint64_t bl = sdesc(bw + BW_PART + slice(256, ks), 128, 256);
          mma(d, sdesc(ah + slice(128, ks), 128, 256), bh, id256, ks > 0);
          mma(d, sdesc(ah + slice(128, ks), 128, 256), bl, id256, 1);
          mma(d, sdesc(al + slice(128, ks), 128, 256), bh, id256, 1);
          if ((g & 3) == 3) a_t = a_t + 1 == A_TILES ? 0 : a_t + 1;
        }
      }
    }
    commit(&done);
    long long polls = 0;
    while (!try_wait(&done, 0)) {
      if (++polls > WAIT_LIMIT) {
        atomicExch(err, 1);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TMEM_COLS));
}

}  // namespace

extern "C" {

// MMAs (M = 128, K = 16) per 128-frame tile of one stream and their N.
int mb_tc_dft_mmas_per_tile(int shape) { return shape == 0 ? 576 : 144; }
int mb_tc_dft_n(int shape) { return shape == 0 ? 64 : 256; }

// Runs `shape` with `tiles` tiles per block on every SM of the current device,
// `reps` times after a warm-up launch; mean CUDA-event time in *ms.  err: a
// device int (set to 1 if a bounded wait gave up).  Returns the cudaError.
int mb_tc_dft_run(int shape, int tiles, int reps, int* err, double* ms) {
  if ((shape != 0 && shape != 1) || tiles < 1 || reps < 1 || !err || !ms)
    return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_dft_bound, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t e0, e1;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return (int)e;
  k_tc_dft_bound<<<sms, 128, SMEM>>>(shape, tiles, err);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    k_tc_dft_bound<<<sms, 128, SMEM>>>(shape, tiles, err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  *ms = (double)t / reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (int)e;
}

}  // extern "C"
