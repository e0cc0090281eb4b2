// C ABI of the lunar-pulse pipeline: plan life cycle, workspace carving,
// argument checks and the per-block launch sequence.  See include/lp.h for
// the contract of every entry point.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "lp_internal.cuh"

using lp::kM;

cudaError_t lp::raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

namespace {

lp_status fail(lp_plan* p, lp_status st, const char* fmt, ...) {
  if (p) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    p->err = buf;
  }
  return st;
}

#define LP_CUDA(plan, call)                                                        \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(plan, LP_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                             \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carve the workspace.  With base == nullptr only the size is computed.
size_t carve(lp_plan& p, char* base) {
  const auto& sh = p.shape;
  const long long J = sh.J();
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = align_up(off, 256);
    char* ptr = base ? base + off : nullptr;
    off += bytes;
    return ptr;
  };
  auto& b = p.buf;
  b.station_enu = (double*)take(sizeof(double) * 3 * sh.S);
  b.beam_dir = (double*)take(sizeof(double) * 3 * sh.B);
  b.tec = (double*)take(sizeof(double) * sh.Tr);
  b.w32 = (float2*)take(sizeof(float2) * (size_t)sh.K * sh.B * sh.S);
  b.wtc = p.cfg.precision == LP_PREC_FP16 ? (__half*)take(lp::beamform_tc_weight_bytes(sh)) : nullptr;
  b.dd = (float2*)take(sizeof(float2) * (size_t)sh.K * sh.Tr);
  b.proto = (double*)take(sizeof(double) * kM * lp::kTaps);
  b.g = (float*)take(sizeof(float) * kM * lp::kTaps);
  b.tw1024 = (float4*)take(sizeof(float4) * kM);
  b.filter_sums = (double*)take(sizeof(double) * 2);
  b.beams = (float2*)take(sizeof(float2) * (size_t)J * sh.K * p.row());
  const bool fine = p.cfg.fine_dedisp != 0;
  b.beams_fine = fine ? (float2*)take(sizeof(float2) * (size_t)J * sh.K * p.row()) : nullptr;
  b.fine_taps = fine ? (float4*)take(sizeof(float4) * (size_t)sh.K * sh.Tr * lp::kFineTaps)
                     : nullptr;
  const bool lsmr = p.cfg.inversion == LP_INV_LSMR;
  b.zt = lsmr ? (float2*)take(sizeof(float2) * (size_t)J * kM * (sh.F + lp::kPrefix)) : nullptr;
  b.xhat = lsmr ? (float2*)take(sizeof(float2) * (size_t)J * kM * sh.F) : nullptr;
  b.lsmr_sigma2 = lsmr ? (double*)take(sizeof(double) * (size_t)J * kM) : nullptr;
  b.lsmr_theta2 = lsmr ? (float*)take(sizeof(float) * (size_t)J * kM) : nullptr;
  b.power_part = (float*)take(sizeof(float) * (size_t)J * sh.K * p.n_ftiles_bf);
  b.sigma2 = (double*)take(sizeof(double) * J);
  b.theta = (float*)take(sizeof(float) * J);
  b.theta2 = (float*)take(sizeof(float) * J);
  b.trig_count = (unsigned long long*)take(sizeof(unsigned long long));
  b.err = (int*)take(sizeof(int));
  b.blk = (long long*)take(sizeof(long long));
  b.trig = (lp::TriggerRec*)take(sizeof(lp::TriggerRec) * (size_t)p.cfg.trigger_cap);
  // streaming blocks: a second trigger list (and below a second staging buffer)
  const bool two = p.cfg.stream_blocks != 0;
  p.trig_buf[0] = b.trig;
  p.count_buf[0] = b.trig_count;
  p.count_buf[1] = two ? (unsigned long long*)take(sizeof(unsigned long long)) : nullptr;
  p.trig_buf[1] =
      two ? (lp::TriggerRec*)take(sizeof(lp::TriggerRec) * (size_t)p.cfg.trigger_cap) : nullptr;
  b.y = p.cfg.store_timeseries ? (float*)take(sizeof(float) * (size_t)J * sh.F * kM) : nullptr;
  const bool fr = p.cfg.fullrate_dedisp != 0;
  b.ufull = fr ? (float2*)take(sizeof(float2) * (size_t)J * (lp::kFrTaps + (size_t)sh.F * kM))
               : nullptr;
  b.fr_hd = fr ? (float2*)take(sizeof(float2) * (size_t)sh.Tr * lp::kFrN) : nullptr;
  b.fr_tw = fr ? (float2*)take(lp::fullrate_table_bytes()) : nullptr;
  b.fr_h = fr ? (double2*)take(sizeof(double2) * lp::kFrTaps) : nullptr;
  b.fr_H = fr ? (double2*)take(sizeof(double2) * lp::kFrN) : nullptr;
  b.fr_E = fr ? (double2*)take(sizeof(double2) * lp::kFrN) : nullptr;
  const size_t in_bytes = (size_t)sh.P * sh.K * sh.F * sh.S * 2 *
                          (p.cfg.input_dtype == LP_INPUT_INT8 ? 1 : 2);
  b.staging = p.cfg.host_input ? (void*)take(in_bytes) : nullptr;
  p.staging_buf[0] = b.staging;
  p.staging_buf[1] = p.cfg.host_input && two ? (void*)take(in_bytes) : nullptr;
  return align_up(off, 256);
}

size_t input_bytes(const lp_plan& p) {
  const auto& sh = p.shape;
  return (size_t)sh.P * sh.K * sh.F * sh.S * 2 * (p.cfg.input_dtype == LP_INPUT_INT8 ? 1 : 2);
}

lp_status need_bound(lp_plan* p) {
  if (!p) return LP_ERR_ARG;
  if (!p->bound) return fail(p, LP_ERR_STATE, "workspace not bound");
  return LP_OK;
}

lp_status set_device(lp_plan* p) {
  int cur = -1;
  LP_CUDA(p, cudaGetDevice(&cur));
  if (cur != p->device) LP_CUDA(p, cudaSetDevice(p->device));
  return LP_OK;
}

lp_status sync_last(lp_plan* p) {
  LP_CUDA(p, cudaStreamSynchronize(p->last_stream));
  LP_CUDA(p, cudaGetLastError());
  int err = 0;
  LP_CUDA(p, cudaMemcpy(&err, p->buf.err, sizeof err, cudaMemcpyDeviceToHost));
  if (err) {
    LP_CUDA(p, cudaMemset(p->buf.err, 0, sizeof err));
    return fail(p, LP_ERR_TIMEOUT, "a bounded device wait gave up (tensor-core beamformer)");
  }
  return LP_OK;
}

// Record the start / end event of a stage for the current block (profiling).
void prof_mark(lp_plan* p, int stage, int end, cudaStream_t s, int part = 0) {
  if (!p->profiling || !p->prof) return;
  const int slot = p->prof_n % lp_plan::kProfSlots;
  cudaEvent_t& ev = p->prof->ev[slot][stage][part][end];
  if (!ev) cudaEventCreate(&ev);
  cudaEventRecord(ev, s);
  if (end) p->prof->used[slot][stage][part] = true;
}

int stream_of(const lp_plan* p, int beam, int tec, int pol) {
  const auto& sh = p->shape;
  if (beam < 0 || beam >= sh.B || tec < 0 || tec >= sh.Tr || pol < 0 || pol >= sh.P) return -1;
  return (beam * sh.Tr + tec) * sh.P + pol;
}

}  // namespace

extern "C" {

void lp_config_default(lp_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->input_dtype = LP_INPUT_INT8;
  c->precision = LP_PREC_FP32;
  c->first_bin = 12;
  c->taps = 16;
  c->kaiser_beta = 9.0;
  c->k_sigma = 6.0;
  c->sigma_alpha = 0.25;
  c->nu_ref_hz = 0.0;
  c->trigger_cap = 1 << 20;
  c->store_timeseries = 0;
  c->host_input = 0;
  c->frames_per_cta = 0;
  c->use_graph = 0;
  c->chunk_frames = 0;
  c->fine_dedisp = 0;
  c->inversion = LP_INV_FIR;
  c->lsmr_iters = 25;
  c->stream_blocks = 0;
  c->fullrate_dedisp = 0;
}

lp_status lp_plan_create(lp_plan** out, int stations, int pols, int subbands, int beams,
                         int tec_trials, int64_t block_len) {
  if (!out) return LP_ERR_ARG;
  *out = nullptr;
  if (stations < 1 || stations > 64 || pols < 1 || pols > 2 || subbands < 1 || subbands > 511 ||
      beams < 1 || beams > 1024 || tec_trials < 1 || tec_trials > 64 || block_len < 16 ||
      block_len > (1 << 22) || block_len % 8 != 0)
    return LP_ERR_ARG;
  lp_plan* p = new (std::nothrow) lp_plan();
  if (!p) return LP_ERR_OOM;
  p->shape = lp::Shape{stations, pols, subbands, beams, tec_trials, (long long)block_len};
  lp_config_default(&p->cfg);
  *out = p;
  return LP_OK;
}

lp_status lp_plan_configure(lp_plan* p, const lp_config* c) {
  if (!p || !c) return LP_ERR_ARG;
  if (p->bound) return fail(p, LP_ERR_STATE, "configure after bind");
  const auto& sh = p->shape;
  if (c->input_dtype != LP_INPUT_INT8 && c->input_dtype != LP_INPUT_INT16)
    return fail(p, LP_ERR_ARG, "input_dtype must be LP_INPUT_INT8 or LP_INPUT_INT16");
  if (c->precision != LP_PREC_FP32 && c->precision != LP_PREC_FP16)
    return fail(p, LP_ERR_ARG, "precision must be LP_PREC_FP32 or LP_PREC_FP16");
  if (c->precision == LP_PREC_FP16 && sh.S % 4 != 0)
    return fail(p, LP_ERR_ARG, "the FP16 tensor-core form needs a multiple of 4 stations");
  if (c->first_bin < 1 || c->first_bin + sh.K > lp::kBins)
    return fail(p, LP_ERR_ARG, "bins [%d, %d) must lie inside [1, 512)", c->first_bin,
                c->first_bin + sh.K);
  if (c->taps != lp::kTaps) return fail(p, LP_ERR_ARG, "taps must be 16");
  if (!(c->kaiser_beta >= 0.0 && c->kaiser_beta <= 50.0))
    return fail(p, LP_ERR_ARG, "kaiser_beta out of range");
  if (!(c->k_sigma > 0.0)) return fail(p, LP_ERR_ARG, "k_sigma must be positive");
  if (!(c->sigma_alpha > 0.0 && c->sigma_alpha <= 1.0))
    return fail(p, LP_ERR_ARG, "sigma_alpha must be in (0, 1]");
  if (c->trigger_cap < 1 || c->trigger_cap > (1LL << 32))
    return fail(p, LP_ERR_ARG, "trigger_cap out of range");
  if (c->frames_per_cta != 0 && (c->frames_per_cta < 8 || c->frames_per_cta % 8 != 0))
    return fail(p, LP_ERR_ARG, "frames_per_cta must be 0 or a positive multiple of 8");
  if (c->fine_dedisp != 0 && c->fine_dedisp != 1)
    return fail(p, LP_ERR_ARG, "fine_dedisp must be 0 or 1");
  if (c->inversion != LP_INV_FIR && c->inversion != LP_INV_LSMR)
    return fail(p, LP_ERR_ARG, "inversion must be LP_INV_FIR or LP_INV_LSMR");
  if (c->inversion == LP_INV_LSMR) {
    if (sh.F % lp::lsmr_window() != 0)
      return fail(p, LP_ERR_ARG, "LSMR inversion needs block_len a multiple of %d",
                  lp::lsmr_window());
    if (c->lsmr_iters < 1 || c->lsmr_iters > 1000)
      return fail(p, LP_ERR_ARG, "lsmr_iters must be in [1, 1000]");
    if (c->chunk_frames != 0)
      return fail(p, LP_ERR_ARG, "LSMR inversion does not combine with chunk_frames");
  }
  if (c->fine_dedisp && c->chunk_frames != 0)
    return fail(p, LP_ERR_ARG, "fine_dedisp does not combine with chunk_frames");
  if (c->stream_blocks != 0 && c->stream_blocks != 1)
    return fail(p, LP_ERR_ARG, "stream_blocks must be 0 or 1");
  if (c->fullrate_dedisp != 0 && c->fullrate_dedisp != 1)
    return fail(p, LP_ERR_ARG, "fullrate_dedisp must be 0 or 1");
  if (c->fullrate_dedisp && (c->chunk_frames != 0 || c->fine_dedisp || c->stream_blocks))
    return fail(p, LP_ERR_ARG, "fullrate_dedisp does not combine with chunk_frames, fine_dedisp "
                "or stream_blocks");
  if (c->stream_blocks && c->use_graph)
    return fail(p, LP_ERR_ARG, "stream_blocks does not combine with use_graph");
  if (c->chunk_frames != 0) {
    if (c->precision != LP_PREC_FP16)
      return fail(p, LP_ERR_ARG, "chunk_frames needs the FP16 form");
    if (c->chunk_frames < lp::beamform_tc_frame_tile() ||
        c->chunk_frames % lp::beamform_tc_frame_tile() != 0 || sh.F % c->chunk_frames != 0)
      return fail(p, LP_ERR_ARG, "chunk_frames must be a multiple of %d that divides block_len",
                  lp::beamform_tc_frame_tile());
  }
  p->cfg = *c;
  p->fc = c->chunk_frames && c->chunk_frames < sh.F ? c->chunk_frames : sh.F;
  p->frames_per_cta = c->frames_per_cta;      // 0: the balanced tiling
  p->n_ftiles_bf = c->precision == LP_PREC_FP16
                       ? lp::beamform_tc_partials(sh.F)
                       : (int)((sh.F + lp::beamform_f32_frame_tile() - 1) /
                               lp::beamform_f32_frame_tile());
  const double nu_lo = lp::kNu0 + c->first_bin * (lp::kFs / kM);
  const double nu_hi = lp::kNu0 + (c->first_bin + sh.K - 1) * (lp::kFs / kM);
  p->nu_ref = c->nu_ref_hz > 0 ? c->nu_ref_hz : 0.5 * (nu_lo + nu_hi);
  p->configured = true;
  return LP_OK;
}

lp_status lp_plan_workspace_bytes(const lp_plan* p, size_t* bytes) {
  if (!p || !bytes) return LP_ERR_ARG;
  if (!p->configured) return LP_ERR_STATE;
  lp_plan tmp = *p;
  *bytes = carve(tmp, nullptr);
  return LP_OK;
}

lp_status lp_plan_bind_workspace(lp_plan* p, void* dev, size_t bytes, void* stream) {
  if (!p) return LP_ERR_ARG;
  if (!p->configured) return fail(p, LP_ERR_STATE, "configure before bind");
  if (!dev || (reinterpret_cast<uintptr_t>(dev) & 255u))
    return fail(p, LP_ERR_ARG, "workspace must be a 256-byte aligned device pointer");
  lp_plan tmp = *p;
  const size_t need = carve(tmp, nullptr);
  if (bytes < need) return fail(p, LP_ERR_OOM, "workspace %zu bytes < %zu needed", bytes, need);
  cudaPointerAttributes attr;
  LP_CUDA(p, cudaPointerGetAttributes(&attr, dev));
  if (attr.type != cudaMemoryTypeDevice)
    return fail(p, LP_ERR_ARG, "workspace is not device memory");
  p->device = attr.device;
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  p->ws = dev;
  p->ws_bytes = bytes;
  carve(*p, static_cast<char*>(dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LP_CUDA(p, lp::init_kernel_attributes(p->shape));
  if (p->cfg.precision == LP_PREC_FP16) LP_CUDA(p, lp::encode_beams_map(*p));
  LP_CUDA(p, cudaMemsetAsync(dev, 0, need, s));
  LP_CUDA(p, lp::launch_prototype(*p, s));
  p->last_stream = s;
  p->bound = true;
  p->block_index = 0;
  return LP_OK;
}

lp_status lp_set_weights(lp_plan* p, const double* enu, const double* dir, void* stream) {
  if (lp_status st = need_bound(p)) return st;
  if (!enu || !dir) return fail(p, LP_ERR_ARG, "null geometry");
  const auto& sh = p->shape;
  for (int b = 0; b < sh.B; ++b) {
    const double n2 = dir[3 * b] * dir[3 * b] + dir[3 * b + 1] * dir[3 * b + 1] +
                      dir[3 * b + 2] * dir[3 * b + 2];
    if (!(std::fabs(n2 - 1.0) < 1e-6)) return fail(p, LP_ERR_ARG, "beam %d is not a unit vector", b);
  }
  for (int i = 0; i < 3 * sh.S; ++i)
    if (!std::isfinite(enu[i])) return fail(p, LP_ERR_ARG, "station position not finite");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // pageable host memory: the copy is complete for the host on return
  LP_CUDA(p, cudaMemcpyAsync(p->buf.station_enu, enu, sizeof(double) * 3 * sh.S,
                             cudaMemcpyHostToDevice, s));
  LP_CUDA(p, cudaMemcpyAsync(p->buf.beam_dir, dir, sizeof(double) * 3 * sh.B,
                             cudaMemcpyHostToDevice, s));
  LP_CUDA(p, lp::launch_weights(*p, s));
  if (p->cfg.precision == LP_PREC_FP16) LP_CUDA(p, lp::launch_weights_tc(*p, s));
  p->last_stream = s;
  p->weights_set = true;
  return LP_OK;
}

lp_status lp_set_tec(lp_plan* p, const double* tec, void* stream) {
  if (lp_status st = need_bound(p)) return st;
  if (!tec) return fail(p, LP_ERR_ARG, "null tec");
  const auto& sh = p->shape;
  for (int t = 0; t < sh.Tr; ++t)
    if (!std::isfinite(tec[t]) || std::fabs(tec[t]) > 1e4)
      return fail(p, LP_ERR_ARG, "tec[%d] out of range", t);
  if (p->cfg.fine_dedisp) {
    // the fine filter's taps hold subband delays within 4 frames of its centre
    const double dnu_sb = lp::kFs / kM;
    for (int t = 0; t < sh.Tr; ++t)
      for (int k : {0, sh.K - 1}) {
        const double nu = lp::kNu0 + (p->cfg.first_bin + k) * dnu_sb;
        const double a = lp::kKappa * tec[t] * lp::kTecu / lp::kC;
        const double d = a * dnu_sb * (1.0 / (p->nu_ref * p->nu_ref) - 1.0 / (nu * nu));
        if (std::fabs(d) > 4.0)
          return fail(p, LP_ERR_ARG, "tec[%d]: subband delay %.2f frames exceeds the fine "
                      "filter's 4-frame range", t, d);
      }
  }
  if (p->cfg.fullrate_dedisp) {
    // the full-rate taps' window holds group delays within 768 samples of the
    // reference delay over the whole 100-200 MHz band
    for (int t = 0; t < sh.Tr; ++t)
      for (double nu : {lp::kNu0, lp::kFs}) {
        const double a = lp::kKappa * tec[t] * lp::kTecu / lp::kC;
        const double d = a * (1.0 / (nu * nu) - 1.0 / (p->nu_ref * p->nu_ref)) * lp::kFs;
        if (std::fabs(d) > 0.5 * lp::kFrFlat)
          return fail(p, LP_ERR_ARG, "tec[%d]: group delay %.0f samples exceeds the full-rate "
                      "filter's %d-sample range", t, d, lp::kFrFlat / 2);
      }
  }
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LP_CUDA(p, cudaMemcpyAsync(p->buf.tec, tec, sizeof(double) * sh.Tr, cudaMemcpyHostToDevice, s));
  LP_CUDA(p, lp::launch_dedisp(*p, s));
  if (p->cfg.fine_dedisp) LP_CUDA(p, lp::launch_fine_taps(*p, s));
  if (p->cfg.fullrate_dedisp) LP_CUDA(p, lp::launch_fullrate_taps(*p, s));
  p->last_stream = s;
  p->tec_set = true;
  return LP_OK;
}

namespace {

enum Tune { kTuneNone = 0, kTuneSynth = 1, kTuneGemm = 2 };

extern "C++" {
// Mean CUDA-event time of runs 2-4 of launch() on s (the first run warms up).
template <class Launch>
cudaError_t time_launch(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, Launch&& launch,
                        double* ms_mean) {
  double ms_sum = 0.0;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) ms_sum += ms;
  }
  *ms_mean = ms_sum / 3.0;
  return e;
}

// Runs launch() under each of n settings (set(i) selects one) while timing it,
// keeps the fastest and runs it once more, so that what the launch leaves in
// device memory is a normal run's.  The launches must be idempotent.
template <class Set, class Launch>
cudaError_t tune_launch(int n, cudaStream_t s, Set&& set, Launch&& launch, double* ms_out,
                        int* best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_ms = 1e30;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (ms_out) ms_out[i] = 0.0;
    if (!set(i)) continue;                     // candidate not applicable
    double ms = 0.0;
    e = time_launch(s, e0, e1, launch, &ms);
    if (e == cudaSuccess) {
      if (ms_out) ms_out[i] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        *best = i;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) set(*best);
  if (e == cudaSuccess) e = launch();
  return e;
}

}  // extern "C++"

// Synthesis of one chunk while timing the candidate tilings (autotuner): each
// candidate reruns the same launch on the same beam rows (before the history
// shift).
cudaError_t tune_ippf(lp_plan* p, const lp::Chunk& c, cudaStream_t s, double* ms_out) {
  // runs of 64 .. 2048 frames per block, and the balanced tiling (0)
  static const int cand[7] = {64, 128, 256, 512, 1024, 2048, 0};
  int best = -1;
  for (int i = 0; i < 7; ++i)
    if (cand[i] == p->frames_per_cta) best = i;
  const int keep = p->frames_per_cta;
  auto set = [&](int i) {
    if (i < 0) {
      p->frames_per_cta = keep;
      return true;
    }
    if (cand[i] > c.nf) return false;
    p->frames_per_cta = cand[i];
    return true;
  };
  auto launch = [&]() {
    cudaError_t e = cudaMemsetAsync(p->buf.trig_count, 0, sizeof(unsigned long long), s);
    return e == cudaSuccess ? lp::launch_ippf(*p, c, s) : e;
  };
  return tune_launch(7, s, set, launch, ms_out, &best);
}

// Beamformer launch over chunk c while timing the configurations (GEMM
// autotuner): each reruns the same launch on the same input; it rewrites the
// chunk's beam rows and noise partials.
cudaError_t tune_gemm(lp_plan* p, const void* x, long long stride, const lp::Chunk& c,
                      cudaStream_t s, double* ms_out) {
  int desc[2 * LP_MAX_GEMM_CONFIGS];
  const int n = lp::beamform_gemm_configs(*p, desc, LP_MAX_GEMM_CONFIGS);
  if (ms_out)
    for (int i = n; i < LP_MAX_GEMM_CONFIGS; ++i) ms_out[i] = 0.0;
  int best = -1;
  auto set = [&](int i) {
    p->gemm_cfg = i;
    return true;
  };
  auto launch = [&]() {
    return p->cfg.precision == LP_PREC_FP16 ? lp::launch_beamform_tc(*p, x, stride, c, s)
                                            : lp::launch_beamform_f32(*p, x, stride, s);
  };
  return tune_launch(n, s, set, launch, ms_out, &best);
}

lp_status process(lp_plan* p, const void* x, int64_t pol_stride, void* stream, Tune tune,
                  double* tune_ms);

}  // namespace

lp_status lp_process_block(lp_plan* p, const void* x, void* stream) {
  if (!p) return LP_ERR_ARG;
  const auto& sh = p->shape;
  return process(p, x, (int64_t)sh.K * sh.F * sh.S, stream, kTuneNone, nullptr);
}

lp_status lp_process_block_strided(lp_plan* p, const void* x, int64_t pol_stride, void* stream) {
  return process(p, x, pol_stride, stream, kTuneNone, nullptr);
}

lp_status lp_plan_autotune(lp_plan* p, const void* x, void* stream, int32_t* best,
                           double* ms_out) {
  if (!p || !best) return LP_ERR_ARG;
  const auto& sh = p->shape;
  const lp_status st = process(p, x, (int64_t)sh.K * sh.F * sh.S, stream, kTuneSynth, ms_out);
  if (st == LP_OK) *best = p->frames_per_cta;
  return st;
}

int lp_plan_gemm_configs(const lp_plan* p, int32_t* desc, int max) {
  if (!p || !p->bound || max < 0 || (max > 0 && !desc)) return -1;
  int all[2 * LP_MAX_GEMM_CONFIGS];
  const int n = lp::beamform_gemm_configs(*p, all, LP_MAX_GEMM_CONFIGS);
  for (int i = 0; i < 2 * std::min(n, max); ++i) desc[i] = all[i];
  return n;
}

lp_status lp_plan_set_gemm_config(lp_plan* p, int index) {
  if (lp_status st = need_bound(p)) return st;
  int all[2 * LP_MAX_GEMM_CONFIGS];
  const int n = lp::beamform_gemm_configs(*p, all, LP_MAX_GEMM_CONFIGS);
  if (index < -1 || index >= n)
    return fail(p, LP_ERR_ARG, "gemm configuration %d not in [-1, %d)", index, n);
  if (p->graph_exec) {
    if (set_device(p) != LP_OK) return LP_ERR_CUDA;
    if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  p->gemm_cfg = index;
  return LP_OK;
}

lp_status lp_plan_autotune_gemm(lp_plan* p, const void* x, void* stream, int32_t* best,
                                double* ms_out) {
  if (!p || !best) return LP_ERR_ARG;
  const auto& sh = p->shape;
  const lp_status st = process(p, x, (int64_t)sh.K * sh.F * sh.S, stream, kTuneGemm, ms_out);
  if (st == LP_OK) *best = p->gemm_cfg;
  return st;
}

namespace {

// Host input, whole block, two polarisations: each polarisation's slab is
// copied on the plan's copy stream and its streams are beamformed,
// noise-levelled, synthesised and shifted as soon as it has landed, so the copy
// of polarisation 1 overlaps the work on polarisation 0 (every stream's noise
// level needs only its own polarisation).  The copy stream first waits for the
// caller's stream, so earlier work on the input and on the staging buffer is
// done.
lp_status process_host_pipelined(lp_plan* p, const void* x, int64_t pol_stride, cudaStream_t s) {
  const auto& sh = p->shape;
  const long long slab = (long long)sh.K * sh.F * sh.S;
  const size_t bpc = p->cfg.input_dtype == LP_INPUT_INT8 ? 2 : 4;
  const bool fp16 = p->cfg.precision == LP_PREC_FP16;
  if (fp16 && ((long long)sh.F * sh.S * bpc) % 16)
    return fail(p, LP_ERR_ARG, "input and pol stride must be 16-byte aligned");
  if (!p->copy_stream) {
    LP_CUDA(p, cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    LP_CUDA(p, cudaEventCreateWithFlags(&p->ev_entry, cudaEventDisableTiming));
    for (auto& ev : p->ev_pol) LP_CUDA(p, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  char* staging = static_cast<char*>(p->buf.staging);
  const int par = (int)(p->block_index & 1);
  if (p->cfg.stream_blocks) {
    // streaming: this staging buffer was last read by the beamformer of the
    // block two calls back; the copy waits for that, not for all earlier work
    if (p->free_recorded[par]) LP_CUDA(p, cudaStreamWaitEvent(p->copy_stream, p->ev_free[par], 0));
  } else {
    LP_CUDA(p, cudaEventRecord(p->ev_entry, s));
    LP_CUDA(p, cudaStreamWaitEvent(p->copy_stream, p->ev_entry, 0));
  }
  for (int pol = 0; pol < 2; ++pol) {
    prof_mark(p, LP_STAGE_H2D, 0, p->copy_stream, pol);
    LP_CUDA(p, cudaMemcpyAsync(staging + pol * slab * bpc,
                               static_cast<const char*>(x) + pol * pol_stride * bpc, slab * bpc,
                               cudaMemcpyHostToDevice, p->copy_stream));
    prof_mark(p, LP_STAGE_H2D, 1, p->copy_stream, pol);
    LP_CUDA(p, cudaEventRecord(p->ev_pol[pol], p->copy_stream));
  }
  cudaError_t e = cudaMemsetAsync(p->buf.trig_count, 0, sizeof(unsigned long long), s);
  lp::Chunk c;
  c.nf = sh.F;
  for (int pol = 0; pol < 2 && e == cudaSuccess; ++pol) {
    const lp::PolSel ps{pol, 1};
    e = cudaStreamWaitEvent(s, p->ev_pol[pol], 0);
    prof_mark(p, LP_STAGE_BEAMFORM, 0, s, pol);
    if (e == cudaSuccess)
      e = fp16 ? lp::launch_beamform_tc(*p, staging, slab, c, s, ps)
               : lp::launch_beamform_f32(*p, staging, slab, s, ps);
    if (e == cudaSuccess && pol == 1 && p->cfg.stream_blocks) {
      e = cudaEventRecord(p->ev_free[par], s);      // staging buffer read for the last time
      p->free_recorded[par] = e == cudaSuccess;
    }
    prof_mark(p, LP_STAGE_BEAMFORM, 1, s, pol);
    prof_mark(p, LP_STAGE_SIGMA, 0, s, pol);
    if (e == cudaSuccess) e = lp::launch_sigma(*p, s, ps);
    prof_mark(p, LP_STAGE_SIGMA, 1, s, pol);
    if (p->cfg.fine_dedisp) {
      prof_mark(p, LP_STAGE_FINE, 0, s, pol);
      if (e == cudaSuccess) e = lp::launch_fine(*p, s, ps);
      prof_mark(p, LP_STAGE_FINE, 1, s, pol);
    }
    prof_mark(p, LP_STAGE_SYNTH, 0, s, pol);
    if (e == cudaSuccess) e = lp::launch_ippf(*p, c, s, ps);
    prof_mark(p, LP_STAGE_SYNTH, 1, s, pol);
    prof_mark(p, LP_STAGE_SHIFT, 0, s, pol);
    if (e == cudaSuccess) e = lp::launch_history_shift(*p, c, s, ps);
    prof_mark(p, LP_STAGE_SHIFT, 1, s, pol);
  }
  LP_CUDA(p, e);
  if (p->profiling && p->prof_n < lp_plan::kProfSlots) p->prof_n += 1;
  p->last_stream = s;
  p->block_index += 1;
  return LP_OK;
}

lp_status process_inner(lp_plan* p, const void* x, int64_t pol_stride, void* stream, Tune tune,
                        double* tune_ms) {
  if (lp_status st = need_bound(p)) return st;
  if (!p->weights_set || !p->tec_set)
    return fail(p, LP_ERR_STATE, "lp_set_weights and lp_set_tec must precede lp_process_block");
  if (!x) return fail(p, LP_ERR_ARG, "null input");
  const auto& sh = p->shape;
  const long long slab = (long long)sh.K * sh.F * sh.S;
  if (pol_stride < slab && sh.P > 1)
    return fail(p, LP_ERR_ARG, "pol_stride %lld is smaller than one pol slab (%lld)",
                (long long)pol_stride, slab);
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaPointerAttributes attr;
  LP_CUDA(p, cudaPointerGetAttributes(&attr, x));
  const void* xd = x;
  long long stride = pol_stride;
  const size_t bpc = p->cfg.input_dtype == LP_INPUT_INT8 ? 2 : 4;   // bytes per complex sample
  const bool host = attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged;
  const bool graph_mode = p->cfg.use_graph && !p->profiling && !tune;
  if (host && p->buf.staging && sh.P == 2 && p->fc == sh.F && !tune && !graph_mode &&
      p->cfg.inversion == LP_INV_FIR && !p->cfg.fullrate_dedisp)
    return process_host_pipelined(p, x, pol_stride, s);
  if (host) {
    if (!p->buf.staging)
      return fail(p, LP_ERR_ARG, "host input needs host_input = 1 in the configuration");
    prof_mark(p, LP_STAGE_H2D, 0, s);
    for (int pol = 0; pol < sh.P; ++pol)
      LP_CUDA(p, cudaMemcpyAsync(static_cast<char*>(p->buf.staging) + pol * slab * bpc,
                                 static_cast<const char*>(x) + pol * pol_stride * bpc, slab * bpc,
                                 cudaMemcpyHostToDevice, s));
    prof_mark(p, LP_STAGE_H2D, 1, s);
    xd = p->buf.staging;
    stride = slab;
  } else if (attr.device != p->device) {
    return fail(p, LP_ERR_ARG, "input lives on device %d, plan on %d", attr.device, p->device);
  }
  const size_t align = p->cfg.precision == LP_PREC_FP16 ? 16 : bpc;   // bulk copies
  if (reinterpret_cast<uintptr_t>(xd) % align || (stride * bpc) % align ||
      (p->cfg.precision == LP_PREC_FP16 && ((long long)sh.F * sh.S * bpc) % align))
    return fail(p, LP_ERR_ARG, "input and pol stride must be %zu-byte aligned", align);

  const bool graph = graph_mode;
  if (tune && p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);     // the tiling changes
    p->graph_exec = nullptr;
  }
  if (graph && !s) return fail(p, LP_ERR_ARG, "graph mode needs a non-default stream");
  if (graph && p->graph_exec && p->graph_x == xd && p->graph_stride == stride) {
    LP_CUDA(p, cudaGraphLaunch(p->graph_exec, s));
  } else {
    if (graph) LP_CUDA(p, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(p->buf.trig_count, 0, sizeof(unsigned long long), s);
    const bool fp16 = p->cfg.precision == LP_PREC_FP16;
    if (p->fc == sh.F) {
      lp::Chunk c;
      c.nf = sh.F;
      prof_mark(p, LP_STAGE_BEAMFORM, 0, s);
      if (e == cudaSuccess)
        e = tune == kTuneGemm ? tune_gemm(p, xd, stride, c, s, tune_ms)
            : fp16            ? lp::launch_beamform_tc(*p, xd, stride, c, s)
                              : lp::launch_beamform_f32(*p, xd, stride, s);
      prof_mark(p, LP_STAGE_BEAMFORM, 1, s);
      prof_mark(p, LP_STAGE_SIGMA, 0, s);
      if (e == cudaSuccess && p->cfg.inversion == LP_INV_FIR) e = lp::launch_sigma(*p, s);
      prof_mark(p, LP_STAGE_SIGMA, 1, s);
      if (p->cfg.fine_dedisp) {
        prof_mark(p, LP_STAGE_FINE, 0, s);
        if (e == cudaSuccess) e = lp::launch_fine(*p, s);
        prof_mark(p, LP_STAGE_FINE, 1, s);
      }
      prof_mark(p, LP_STAGE_SYNTH, 0, s);
      const bool lsmr = p->cfg.inversion == LP_INV_LSMR;
      if (e == cudaSuccess && lsmr) {
        e = lp::launch_lsmr(*p, s);
        // the paper's order: the inversion, then the full-rate filter of the
        // recovered series, then the per-phase noise level and the trigger
        if (e == cudaSuccess && !p->cfg.fullrate_dedisp) e = lp::launch_lsmr_trigger(*p, s);
      } else if (e == cudaSuccess) {
        e = tune == kTuneSynth ? tune_ippf(p, c, s, tune_ms) : lp::launch_ippf(*p, c, s);
      }
      prof_mark(p, LP_STAGE_SYNTH, 1, s);
      if (p->cfg.fullrate_dedisp) {
        prof_mark(p, LP_STAGE_FULLRATE, 0, s);
        if (e == cudaSuccess) e = lp::launch_fullrate(*p, s);
        if (e == cudaSuccess && lsmr) e = lp::launch_lsmr_trigger(*p, s);
        prof_mark(p, LP_STAGE_FULLRATE, 1, s);
      }
      prof_mark(p, LP_STAGE_SHIFT, 0, s);
      if (e == cudaSuccess) e = lp::launch_history_shift(*p, c, s);
      if (e == cudaSuccess && p->cfg.fullrate_dedisp) e = lp::launch_fullrate_shift(*p, s);
      prof_mark(p, LP_STAGE_SHIFT, 1, s);
    } else {
      // chunked block: the noise level needs the whole block, so a first
      // beamformer pass only sums |beam|^2; then each chunk is beamformed into
      // the beam rows, synthesised and shifted.  Stage times cover all chunks.
      lp::Chunk all;
      all.nf = sh.F;
      all.write_beams = false;
      prof_mark(p, LP_STAGE_BEAMFORM, 0, s);
      if (e == cudaSuccess) e = lp::launch_beamform_tc(*p, xd, stride, all, s);
      prof_mark(p, LP_STAGE_SIGMA, 0, s);
      if (e == cudaSuccess) e = lp::launch_sigma(*p, s);
      prof_mark(p, LP_STAGE_SIGMA, 1, s);
      for (long long f0 = 0; f0 < sh.F && e == cudaSuccess; f0 += p->fc) {
        lp::Chunk c;
        c.f_base = f0;
        c.nf = p->fc;
        c.write_power = false;
        c.last = f0 + p->fc >= sh.F;
        e = tune == kTuneGemm && f0 == 0 ? tune_gemm(p, xd, stride, c, s, tune_ms)
                                         : lp::launch_beamform_tc(*p, xd, stride, c, s);
        if (e == cudaSuccess)
          e = tune == kTuneSynth && f0 == 0 ? tune_ippf(p, c, s, tune_ms)
                                            : lp::launch_ippf(*p, c, s);
        if (e == cudaSuccess) e = lp::launch_history_shift(*p, c, s);
      }
      prof_mark(p, LP_STAGE_BEAMFORM, 1, s);
    }
    if (graph) {
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(s, &g);
      if (e == cudaSuccess) e = ec;
      if (e == cudaSuccess) {
        if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
        e = cudaGraphInstantiate(&p->graph_exec, g, 0);
      }
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) {
        p->graph_x = xd;
        p->graph_stride = stride;
        e = cudaGraphLaunch(p->graph_exec, s);
      }
    }
    LP_CUDA(p, e);
  }
  if (p->profiling && p->prof_n < lp_plan::kProfSlots) p->prof_n += 1;
  p->last_stream = s;
  p->block_index += 1;
  return LP_OK;
}

// One block: with stream_blocks, block b uses staging buffer and trigger list
// b mod 2 and the end of its work is recorded for lp_get_triggers_block.
lp_status process(lp_plan* p, const void* x, int64_t pol_stride, void* stream, Tune tune,
                  double* tune_ms) {
  if (lp_status st = need_bound(p)) return st;
  if (!p->cfg.stream_blocks) return process_inner(p, x, pol_stride, stream, tune, tune_ms);
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  for (int i = 0; i < 2; ++i) {
    if (!p->ev_free[i]) LP_CUDA(p, cudaEventCreateWithFlags(&p->ev_free[i], cudaEventDisableTiming));
    if (!p->ev_done[i]) LP_CUDA(p, cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming));
  }
  if (!p->read_stream)
    LP_CUDA(p, cudaStreamCreateWithFlags(&p->read_stream, cudaStreamNonBlocking));
  const long long blk = p->block_index;
  const int par = (int)(blk & 1);
  p->buf.trig = p->trig_buf[par];
  p->buf.trig_count = p->count_buf[par];
  if (p->staging_buf[par]) p->buf.staging = p->staging_buf[par];
  const lp_status st = process_inner(p, x, pol_stride, stream, tune, tune_ms);
  if (st != LP_OK) return st;
  LP_CUDA(p, cudaEventRecord(p->ev_done[par], static_cast<cudaStream_t>(stream)));
  p->block_in[par] = blk;
  return LP_OK;
}

// Sorted copy of n records of a trigger list (device) to the caller.
lp_status read_triggers(lp_plan* p, const lp::TriggerRec* trig, unsigned long long cnt,
                        cudaStream_t rs, lp_trigger* out, int64_t cap, int64_t* n_total) {
  *n_total = (int64_t)cnt;
  const long long kept = std::min<long long>((long long)cnt, p->cfg.trigger_cap);
  std::vector<lp_trigger> all((size_t)kept);
  if (kept > 0) {
    LP_CUDA(p, cudaMemcpyAsync(all.data(), trig, sizeof(lp_trigger) * (size_t)kept,
                               cudaMemcpyDeviceToHost, rs));
    LP_CUDA(p, cudaStreamSynchronize(rs));
  }
  std::sort(all.begin(), all.end(), [](const lp_trigger& a, const lp_trigger& b) {
    if (a.beam != b.beam) return a.beam < b.beam;
    if (a.tec != b.tec) return a.tec < b.tec;
    if (a.pol != b.pol) return a.pol < b.pol;
    return a.n < b.n;
  });
  const long long ncopy = std::min<long long>(kept, cap);
  if (ncopy > 0) std::memcpy(out, all.data(), sizeof(lp_trigger) * (size_t)ncopy);
  if ((long long)cnt > cap || (long long)cnt > p->cfg.trigger_cap)
    return fail(p, LP_ERR_OVERFLOW, "%llu triggers, %lld copied", cnt, ncopy);
  return LP_OK;
}

}  // namespace

lp_status lp_get_triggers_block(lp_plan* p, int64_t block, lp_trigger* out, int64_t cap,
                                int64_t* n_total) {
  if (lp_status st = need_bound(p)) return st;
  if (!n_total || cap < 0 || (cap > 0 && !out)) return fail(p, LP_ERR_ARG, "bad output buffer");
  if (!p->cfg.stream_blocks) {
    if (block != p->block_index - 1)
      return fail(p, LP_ERR_STATE, "block %lld is not the last processed block",
                  (long long)block);
    return lp_get_triggers(p, out, cap, n_total);
  }
  const int par = (int)(block & 1);
  if (block < 0 || p->block_in[par] != block)
    return fail(p, LP_ERR_STATE, "block %lld is not one of the last two processed blocks",
                (long long)block);
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  // wait for that block only; reads on a stream of their own, so that neither
  // the next block's kernels nor its host copy are waited for
  LP_CUDA(p, cudaEventSynchronize(p->ev_done[par]));
  cudaStream_t rs = p->read_stream;
  int err = 0;
  unsigned long long cnt = 0;
  LP_CUDA(p, cudaMemcpyAsync(&err, p->buf.err, sizeof err, cudaMemcpyDeviceToHost, rs));
  LP_CUDA(p, cudaMemcpyAsync(&cnt, p->count_buf[par], sizeof cnt, cudaMemcpyDeviceToHost, rs));
  LP_CUDA(p, cudaStreamSynchronize(rs));
  if (err) return fail(p, LP_ERR_TIMEOUT, "a bounded device wait gave up (tensor-core beamformer)");
  return read_triggers(p, p->trig_buf[par], cnt, rs, out, cap, n_total);
}

lp_status lp_get_triggers(lp_plan* p, lp_trigger* out, int64_t cap, int64_t* n_total) {
  if (lp_status st = need_bound(p)) return st;
  if (!n_total || cap < 0 || (cap > 0 && !out)) return fail(p, LP_ERR_ARG, "bad output buffer");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
  unsigned long long cnt = 0;
  LP_CUDA(p, cudaMemcpy(&cnt, p->buf.trig_count, sizeof cnt, cudaMemcpyDeviceToHost));
  *n_total = (int64_t)cnt;
  const long long kept = std::min<long long>((long long)cnt, p->cfg.trigger_cap);
  std::vector<lp_trigger> all((size_t)kept);
  if (kept > 0)
    LP_CUDA(p, cudaMemcpy(all.data(), p->buf.trig, sizeof(lp_trigger) * (size_t)kept,
                          cudaMemcpyDeviceToHost));
  std::sort(all.begin(), all.end(), [](const lp_trigger& a, const lp_trigger& b) {
    if (a.beam != b.beam) return a.beam < b.beam;
    if (a.tec != b.tec) return a.tec < b.tec;
    if (a.pol != b.pol) return a.pol < b.pol;
    return a.n < b.n;
  });
  const long long ncopy = std::min<long long>(kept, cap);
  if (ncopy > 0) std::memcpy(out, all.data(), sizeof(lp_trigger) * (size_t)ncopy);
  if ((long long)cnt > cap || (long long)cnt > p->cfg.trigger_cap)
    return fail(p, LP_ERR_OVERFLOW, "%llu triggers, %lld copied", cnt, ncopy);
  return LP_OK;
}

lp_status lp_get_timeseries(lp_plan* p, int beam, int tec, int pol, float* out) {
  if (lp_status st = need_bound(p)) return st;
  const int j = stream_of(p, beam, tec, pol);
  if (j < 0 || !out) return fail(p, LP_ERR_ARG, "bad stream or buffer");
  if (p->buf.xhat) {
    // LSMR inversion: the real part of the recovered series, stored phase-major
    if (set_device(p) != LP_OK) return LP_ERR_CUDA;
    if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
    const size_t F = (size_t)p->shape.F;
    std::vector<float2> xs(F * kM);
    LP_CUDA(p, cudaMemcpy(xs.data(), p->buf.xhat + (size_t)j * kM * F, sizeof(float2) * F * kM,
                          cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < (size_t)kM; ++q)
      for (size_t i = 0; i < F; ++i) out[i * kM + q] = xs[q * F + i].x;
    return LP_OK;
  }
  if (!p->buf.y) return fail(p, LP_ERR_STATE, "store_timeseries is off");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
  const size_t n = (size_t)p->shape.F * kM;
  LP_CUDA(p, cudaMemcpy(out, p->buf.y + (size_t)j * n, n * sizeof(float), cudaMemcpyDeviceToHost));
  return LP_OK;
}

lp_status lp_get_beams(lp_plan* p, int beam, int tec, int pol, float* out) {
  if (lp_status st = need_bound(p)) return st;
  if (p->fc != p->shape.F)
    return fail(p, LP_ERR_STATE, "a chunked plan keeps only one chunk of beam rows");
  const int j = stream_of(p, beam, tec, pol);
  if (j < 0 || !out) return fail(p, LP_ERR_ARG, "bad stream or buffer");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
  const auto& sh = p->shape;
  // After a block the row holds [prefix = last 16 frames][F frames]; the
  // block's frames sit at positions 16 .. F+15.
  LP_CUDA(p, cudaMemcpy2D(out, sizeof(float2) * sh.F,
                          p->buf.beams + (size_t)j * sh.K * p->row() + lp::kPrefix,
                          sizeof(float2) * p->row(), sizeof(float2) * sh.F, sh.K,
                          cudaMemcpyDeviceToHost));
  return LP_OK;
}

lp_status lp_get_sigma(lp_plan* p, double* out) {
  if (lp_status st = need_bound(p)) return st;
  if (!out) return fail(p, LP_ERR_ARG, "null output");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
  const int J = p->shape.J();
  if (p->buf.lsmr_sigma2) {
    // LSMR inversion: the RMS over phases of the per-phase levels
    std::vector<double> s2((size_t)J * kM);
    LP_CUDA(p, cudaMemcpy(s2.data(), p->buf.lsmr_sigma2, sizeof(double) * s2.size(),
                          cudaMemcpyDeviceToHost));
    for (int j = 0; j < J; ++j) {
      double acc = 0.0;
      for (int q = 0; q < kM; ++q) acc += s2[(size_t)j * kM + q];
      out[j] = std::sqrt(acc / kM);
    }
    return LP_OK;
  }
  std::vector<double> s2(J);
  LP_CUDA(p, cudaMemcpy(s2.data(), p->buf.sigma2, sizeof(double) * J, cudaMemcpyDeviceToHost));
  for (int j = 0; j < J; ++j) out[j] = std::sqrt(s2[j]);
  return LP_OK;
}

lp_status lp_get_lsmr_sigma(lp_plan* p, double* out) {
  if (lp_status st = need_bound(p)) return st;
  if (!out) return fail(p, LP_ERR_ARG, "null output");
  if (!p->buf.lsmr_sigma2) return fail(p, LP_ERR_STATE, "the plan does not use the LSMR inversion");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
  const size_t n = (size_t)p->shape.J() * kM;
  std::vector<double> s2(n);
  LP_CUDA(p, cudaMemcpy(s2.data(), p->buf.lsmr_sigma2, sizeof(double) * n, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < n; ++i) out[i] = std::sqrt(s2[i]);
  return LP_OK;
}

lp_status lp_reset_stream(lp_plan* p, void* stream) {
  if (lp_status st = need_bound(p)) return st;
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto& sh = p->shape;
  LP_CUDA(p, cudaMemsetAsync(p->buf.beams, 0,
                             sizeof(float2) * (size_t)sh.J() * sh.K * p->row(), s));
  if (p->buf.beams_fine)
    LP_CUDA(p, cudaMemsetAsync(p->buf.beams_fine, 0,
                               sizeof(float2) * (size_t)sh.J() * sh.K * p->row(), s));
  LP_CUDA(p, cudaMemsetAsync(p->buf.sigma2, 0, sizeof(double) * sh.J(), s));
  if (p->buf.ufull)                    // the series history of the full-rate filter
    LP_CUDA(p, cudaMemset2DAsync(p->buf.ufull, sizeof(float2) * lp::fullrate_row(*p), 0,
                                 sizeof(float2) * lp::kFrTaps, sh.J(), s));
  if (p->buf.lsmr_sigma2)
    LP_CUDA(p, cudaMemsetAsync(p->buf.lsmr_sigma2, 0, sizeof(double) * sh.J() * kM, s));
  LP_CUDA(p, cudaMemsetAsync(p->buf.trig_count, 0, sizeof(unsigned long long), s));
  if (p->count_buf[1])
    LP_CUDA(p, cudaMemsetAsync(p->count_buf[1], 0, sizeof(unsigned long long), s));
  p->block_in[0] = p->block_in[1] = -1;
  LP_CUDA(p, cudaMemsetAsync(p->buf.blk, 0, sizeof(long long), s));
  p->last_stream = s;
  p->block_index = 0;
  return LP_OK;
}

int lp_launches_per_block(const lp_plan* p) {
  // beamformer, sigma, (fine filter: one launch per 65535 rows,) synthesis,
  // history shift; chunked: power pass + sigma + 3 per chunk
  if (!p) return 4;
  const long long rows = (long long)p->shape.J() * p->shape.K;
  const int fine = p->cfg.fine_dedisp ? (int)((rows + 65534) / 65535) : 0;
  if (p->cfg.inversion == LP_INV_LSMR) {  // beamformer, inverse FFT, LSMR + trigger per
    const int nj = (int)((p->shape.J() + 65534) / 65535);   // 65535 streams, sigma, shift
    // full-rate filter: the filter (per 65535 streams) and its history shift
    return 4 + fine + 2 * nj + (p->cfg.fullrate_dedisp ? 1 + nj : 0);
  }
  // full-rate filter: one launch per 65535 streams, and its history shift
  const int nj = (int)((p->shape.J() + 65534) / 65535);
  if (p->fc == 0 || p->fc == p->shape.F) return 4 + fine + (p->cfg.fullrate_dedisp ? 1 + nj : 0);
  return 2 + 3 * (int)(p->shape.F / p->fc);
}

lp_status lp_profile_enable(lp_plan* p, int enable) {
  if (!p) return LP_ERR_ARG;
  if (enable && !p->prof) {
    lp_plan::ProfTable* t = new (std::nothrow) lp_plan::ProfTable();
    if (!t) return fail(p, LP_ERR_OOM, "no host memory for the profiling table");
    p->prof.reset(t);
  }
  p->profiling = enable != 0;
  return LP_OK;
}

lp_status lp_profile_read(lp_plan* p, double* total_ms, int64_t* blocks) {
  if (lp_status st = need_bound(p)) return st;
  if (!total_ms || !blocks) return fail(p, LP_ERR_ARG, "null output");
  if (set_device(p) != LP_OK) return LP_ERR_CUDA;
  if (sync_last(p) != LP_OK) return LP_ERR_CUDA;
  for (int st = 0; st < LP_NUM_STAGES; ++st) total_ms[st] = 0.0;
  for (int slot = 0; p->prof && slot < p->prof_n; ++slot) {
    for (int st = 0; st < LP_NUM_STAGES; ++st) {
      for (int part = 0; part < lp_plan::kProfParts; ++part) {
        if (!p->prof->used[slot][st][part]) continue;
        float ms = 0.f;
        LP_CUDA(p, cudaEventElapsedTime(&ms, p->prof->ev[slot][st][part][0],
                                        p->prof->ev[slot][st][part][1]));
        total_ms[st] += ms;
        p->prof->used[slot][st][part] = false;
      }
    }
  }
  *blocks = p->prof_n;
  p->prof_n = 0;
  return LP_OK;
}

void lp_plan_destroy(lp_plan* p) {
  if (!p) return;
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->prof)
    for (auto& slot : p->prof->ev)
      for (auto& st : slot)
        for (auto& part : st)
          for (auto& ev : part)
            if (ev) cudaEventDestroy(ev);
  if (p->copy_stream) {
    cudaStreamSynchronize(p->copy_stream);
    cudaStreamDestroy(p->copy_stream);
  }
  if (p->ev_entry) cudaEventDestroy(p->ev_entry);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_free[i]) cudaEventDestroy(p->ev_free[i]);
    if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
  }
  if (p->read_stream) cudaStreamDestroy(p->read_stream);
  for (auto& ev : p->ev_pol)
    if (ev) cudaEventDestroy(ev);
  delete p;
}

const char* lp_last_error(const lp_plan* p) { return p ? p->err.c_str() : "null plan"; }

const char* lp_status_string(lp_status s) {
  switch (s) {
    case LP_OK: return "ok";
    case LP_ERR_ARG: return "invalid argument";
    case LP_ERR_CUDA: return "CUDA error";
    case LP_ERR_OOM: return "workspace too small";
    case LP_ERR_STATE: return "call out of order";
    case LP_ERR_OVERFLOW: return "trigger buffer overflow";
    case LP_ERR_TIMEOUT: return "device wait timed out";
    case LP_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

}  // extern "C"
