// lp_process_block_noalloc: one block of the FP32 pipeline for callers that
// cannot allocate device memory.
//
// Some callers run where cudaMalloc is not available to them: code inside a
// host process that forbids device allocation after start-up (a real-time
// loop with a fixed memory budget, or a plug-in of a framework that owns the
// device heap and hands out only the buffers it has planned).  They cannot
// bind a plan workspace.  This entry point keeps everything it needs besides
// the caller's inputs and outputs (phase tables, synthesis filter, the beam
// intermediate, noise partial sums) in one file-scope device array of
// LP_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
// the process exits.  It treats the block as the first block of a stream
// (zero synthesis history), so it needs no state between calls.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; the call clears what must start at zero (the history prefix of
// the beam rows, the block counter and the trigger counter).  Calls whose GPU
// work overlaps (different streams, or host threads) race on the array and
// must be serialised by the caller.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress, with that device current) and
// caches it; make that first call before any stream capture.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lp_internal.cuh"

static __device__ __align__(256) unsigned char g_lp_noalloc_scratch[LP_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_addr_mu;
void* g_addr[128] = {};

// Device address of the scratch array on the current device (looked up once
// per device; host code must never hand the symbol itself to a kernel).
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_lp_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

lp_status report(char* err, size_t errlen, lp_status st, const char* msg) {
  if (err && errlen) snprintf(err, errlen, "%s", msg);
  return st;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" lp_status lp_process_block_noalloc(
    int stations, int pols, int subbands, int beams, int tec_trials, int64_t block_len,
    const lp_config* cfg, const double* station_enu_m, const double* beam_dir,
    const double* tec_tecu, const void* x, float* y, double* sigma2, lp_trigger* triggers,
    int64_t trigger_cap, unsigned long long* trigger_count, void* stream, char* err,
    size_t errlen) {
  char msg[256];
  if (stations < 1 || stations > 64 || pols < 1 || pols > 2 || subbands < 1 || subbands > 511 ||
      beams < 1 || beams > 1024 || tec_trials < 1 || tec_trials > 64 || block_len < 16 ||
      block_len > (1 << 22) || block_len % 8 != 0)
    return report(err, errlen, LP_ERR_ARG, "shape out of range (same limits as lp_plan_create)");
  if (!cfg || !station_enu_m || !beam_dir || !tec_tecu || !x || !y)
    return report(err, errlen, LP_ERR_ARG, "null argument");
  if (cfg->precision != LP_PREC_FP32)
    return report(err, errlen, LP_ERR_ARG, "the no-allocation entry point runs the FP32 form only");
  if (cfg->fine_dedisp || cfg->fullrate_dedisp || cfg->inversion != LP_INV_FIR)
    return report(err, errlen, LP_ERR_ARG, "the no-allocation entry point runs the FIR synthesis "
                  "without fine or full-rate de-dispersion");
  if (trigger_cap < 0 || (trigger_cap > 0 && !triggers))
    return report(err, errlen, LP_ERR_ARG, "bad trigger buffer");
  for (int i = 0; i < beams; ++i) {
    const double* d = beam_dir + 3 * i;
    if (!(std::fabs(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - 1.0) < 1e-6))
      return report(err, errlen, LP_ERR_ARG, "beam directions must be unit vectors");
  }

  // a plan on the stack: the ordinary configuration checks, no workspace
  lp_plan p;
  p.shape = lp::Shape{stations, pols, subbands, beams, tec_trials, (long long)block_len};
  lp_config c = *cfg;
  c.store_timeseries = 1;
  c.host_input = 0;
  c.trigger_cap = trigger_cap > 0 ? trigger_cap : 1;
  c.chunk_frames = 0;
  c.stream_blocks = 0;
  if (lp_plan_configure(&p, &c) != LP_OK) return report(err, errlen, LP_ERR_ARG, p.err.c_str());
  p.cfg.trigger_cap = trigger_cap;

  // carve the scratch array: tables, filter, beam rows, partial sums, counter
  const auto& sh = p.shape;
  const size_t J = (size_t)sh.J();
  size_t off = 0;
  size_t o_enu = off; off = up256(off + sizeof(double) * 3 * sh.S);
  size_t o_dir = off; off = up256(off + sizeof(double) * 3 * sh.B);
  size_t o_tec = off; off = up256(off + sizeof(double) * sh.Tr);
  size_t o_w = off;   off = up256(off + sizeof(float2) * (size_t)sh.K * sh.B * sh.S);
  size_t o_dd = off;  off = up256(off + sizeof(float2) * (size_t)sh.K * sh.Tr);
  size_t o_pr = off;  off = up256(off + sizeof(double) * lp::kM * lp::kTaps);
  size_t o_g = off;   off = up256(off + sizeof(float) * lp::kM * lp::kTaps);
  size_t o_fs = off;  off = up256(off + sizeof(double) * 2);
  size_t o_tw = off;  off = up256(off + sizeof(float4) * lp::kM);
  size_t o_bm = off;  off = up256(off + sizeof(float2) * J * sh.K * p.row());
  size_t o_pp = off;  off = up256(off + sizeof(float) * J * sh.K * p.n_ftiles_bf);
  size_t o_s2 = off;  off = up256(off + sizeof(double) * J);
  size_t o_th = off;  off = up256(off + sizeof(float) * J);
  size_t o_t2 = off;  off = up256(off + sizeof(float) * J);
  size_t o_tc = off;  off = up256(off + sizeof(unsigned long long));
  size_t o_er = off;  off = up256(off + sizeof(int));
  size_t o_bk = off;  off = up256(off + sizeof(long long));
  if (off > (size_t)LP_NOALLOC_SCRATCH_BYTES) {
    snprintf(msg, sizeof msg,
             "this shape needs %zu bytes of scratch; the static buffer holds %zu bytes",
             off, (size_t)LP_NOALLOC_SCRATCH_BYTES);
    return report(err, errlen, LP_ERR_ARG, msg);
  }

  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(err, errlen, LP_ERR_CUDA, cudaGetErrorString(e));
  // every device argument: device (or managed) memory of the current device,
  // aligned to its element; refused before anything touches the GPU
  const size_t x_align = c.input_dtype == LP_INPUT_INT8 ? 2 : 4;   // one complex sample
  const struct {
    const void* ptr;
    size_t align;
    const char* name;
  } args[] = {{x, x_align, "x"},
              {y, sizeof(float), "y"},
              {sigma2, sizeof(double), "sigma2"},
              {triggers, 8, "triggers"},
              {trigger_count, sizeof(unsigned long long), "trigger_count"}};
  for (const auto& a : args) {
    if (!a.ptr) continue;
    if (reinterpret_cast<uintptr_t>(a.ptr) % a.align) {
      snprintf(msg, sizeof msg, "%s must be %zu-byte aligned", a.name, a.align);
      return report(err, errlen, LP_ERR_ARG, msg);
    }
    cudaPointerAttributes attr;
    e = cudaPointerGetAttributes(&attr, a.ptr);
    if (e != cudaSuccess) return report(err, errlen, LP_ERR_CUDA, cudaGetErrorString(e));
    if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
        attr.device != dev) {
      snprintf(msg, sizeof msg, "%s must be device or managed memory of the current device",
               a.name);
      return report(err, errlen, LP_ERR_ARG, msg);
    }
  }
  void* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return report(err, errlen, LP_ERR_CUDA, cudaGetErrorString(e));

  char* b = static_cast<char*>(base);
  auto& buf = p.buf;
  buf.station_enu = (double*)(b + o_enu);
  buf.beam_dir = (double*)(b + o_dir);
  buf.tec = (double*)(b + o_tec);
  buf.w32 = (float2*)(b + o_w);
  buf.wtc = nullptr;
  buf.dd = (float2*)(b + o_dd);
  buf.proto = (double*)(b + o_pr);
  buf.g = (float*)(b + o_g);
  buf.filter_sums = (double*)(b + o_fs);
  buf.tw1024 = (float4*)(b + o_tw);
  buf.beams = (float2*)(b + o_bm);
  buf.power_part = (float*)(b + o_pp);
  buf.sigma2 = sigma2 ? sigma2 : (double*)(b + o_s2);
  buf.theta = (float*)(b + o_th);
  buf.theta2 = (float*)(b + o_t2);
  buf.trig_count = trigger_count ? trigger_count : (unsigned long long*)(b + o_tc);
  buf.trig = reinterpret_cast<lp::TriggerRec*>(triggers);
  buf.y = y;
  buf.staging = nullptr;
  buf.err = (int*)(b + o_er);
  buf.blk = (long long*)(b + o_bk);
  p.device = dev;
  p.block_index = 0;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
#define NA_CUDA(call)                                                              \
  do {                                                                             \
    const cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return report(err, errlen, LP_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)
  // what must start at zero: zero history (beam rows), the block counter (a
  // first block) and the trigger counter
  NA_CUDA(lp::init_kernel_attributes(p.shape));
  NA_CUDA(cudaMemsetAsync(buf.beams, 0, o_pp - o_bm, s));
  NA_CUDA(cudaMemsetAsync(buf.blk, 0, sizeof(long long), s));
  NA_CUDA(cudaMemsetAsync(buf.trig_count, 0, sizeof(unsigned long long), s));
  NA_CUDA(cudaMemcpyAsync(buf.station_enu, station_enu_m, sizeof(double) * 3 * sh.S,
                          cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(buf.beam_dir, beam_dir, sizeof(double) * 3 * sh.B,
                          cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(buf.tec, tec_tecu, sizeof(double) * sh.Tr, cudaMemcpyHostToDevice, s));
  NA_CUDA(lp::launch_prototype(p, s));
  NA_CUDA(lp::launch_weights(p, s));
  NA_CUDA(lp::launch_dedisp(p, s));
  NA_CUDA(lp::launch_beamform_f32(p, x, (long long)sh.K * sh.F * sh.S, s));
  NA_CUDA(lp::launch_sigma(p, s));
  lp::Chunk whole;
  whole.nf = sh.F;
  NA_CUDA(lp::launch_ippf(p, whole, s));
#undef NA_CUDA
  return LP_OK;
}
