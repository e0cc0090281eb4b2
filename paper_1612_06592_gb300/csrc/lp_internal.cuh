// Internal declarations shared by the kernels and the C ABI of the GB300
// lunar-pulse pipeline.  Not part of the public interface (see include/lp.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <memory>
#include <string>

#include "../../include/lp.h"

namespace lp {

constexpr int kM = 1024;              // filter-bank size: 1024 samples per frame
constexpr int kBins = kM / 2;         // 512 bins of a real 200 MHz input
constexpr int kTaps = 16;             // synthesis taps (frames)
constexpr int kHist = kTaps - 1;      // 15 history frames per stream
constexpr int kPrefix = 16;           // frames stored before a block's first frame
constexpr double kFs = 200e6;         // 5 ns sampling (Sec. 2)
constexpr double kNu0 = kFs / 2;      // sky frequency of bin 0 (second Nyquist zone)
constexpr double kC = 299792458.0;
constexpr double kKappa = 40.308;     // e^2 / (8 pi^2 eps0 m_e), m^3 s^-2
constexpr double kTecu = 1e16;

// Channel-domain fine de-dispersion (Sec. 3, third paragraph): taps along
// frames per (subband, STEC trial), common delay in frames, Kaiser beta of the
// taps' window, frequency points of the taps' inverse DTFT.
constexpr int kFineTaps = 17;
constexpr int kFineDelay = 8;
constexpr double kFineBeta = 4.0;
constexpr int kFineGrid = 1024;
static_assert(kFineTaps - 1 <= kPrefix, "the filter's history must fit the row prefix");

// Full-rate de-dispersion (Sec. 3, third paragraph, at full resolution): taps
// of the streaming filter of the synthesised series, their common delay, the
// flat part of their window and the transform size of the set-up and of the
// overlap-save filter.
constexpr int kFrTaps = 2048;
constexpr int kFrDelay = 1024;
constexpr int kFrFlat = 1536;
constexpr int kFrN = 8192;

// I0(x) = sum_k ((x/2)^k / k!)^2, summed until the terms vanish (Kaiser windows).
__device__ inline double bessel_i0_series(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 200; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

// Device trigger record; same layout as lp_trigger.
struct TriggerRec {
  long long n;
  int beam, tec, pol, stream;
  float env, sigma;
};
static_assert(sizeof(TriggerRec) == sizeof(lp_trigger), "trigger layout");

// Views into the bound workspace.
struct Buffers {
  double* station_enu;     // [S][3]
  double* beam_dir;        // [B][3]
  double* tec;             // [Tr]
  float2* w32;             // [K][B][S] FP32 weights (FP32 form)
  __half* wtc;             // tensor-core A operand (FP16 form), see k_beamform_tc.cu
  float2* dd;              // [K][Tr] de-dispersion phasors
  double* proto;           // [16384] unnormalised prototype (scratch for filter build)
  float* g;                // [16384] synthesis filter * 2/M
  float4* tw1024;          // [32 p1][32 l] exp(+2 pi i p1 l / 1024) as (c, c, s, s)
  double* filter_sums;     // [2]: sum h, sum h^2 of the unnormalised prototype
  float2* beams;           // [J][K][row], row = F + 16, frame m at m + 16
  float2* beams_fine;      // same layout, after the fine de-dispersion filter, or null
  float4* fine_taps;       // [K][Tr][kFineTaps] (r.re, r.re, -r.im, r.im), or null
  float2* zt;              // LSMR inversion: [J][M][F + 16] windowed sums, phase-major, or null
  float2* xhat;            // LSMR inversion: [J][M][F] recovered analytic series, or null
  double* lsmr_sigma2;     // LSMR inversion: [J][M] running noise variance per phase
  float* lsmr_theta2;      // LSMR inversion: [J][M] (k_sigma sigma)^2
  float* power_part;       // [J][K][n_ftiles] partial sums of |beam|^2
  double* sigma2;          // [J]
  float* theta;            // [J] k_sigma * sigma
  float* theta2;           // [J] theta^2 in FP32 (threshold on |u|^2)
  unsigned long long* trig_count;  // [1]
  TriggerRec* trig;        // [trigger_cap]
  float* y;                // [J][F*M] or null
  float2* ufull;           // full-rate mode: [J][kFrTaps + F*M] synthesised series, history first
  float2* fr_hd;           // full-rate mode: [Tr][16][512] taps' spectrum / kFrN (kernel order)
  float2* fr_tw;           // full-rate mode: FFT twiddles [16][512], then [16][32], as (c, s)
  double2* fr_h;           // full-rate set-up scratch: [kFrTaps] taps of one trial
  double2* fr_H;           // full-rate set-up scratch: [kFrN] response of one trial
  double2* fr_E;           // full-rate set-up scratch: [kFrN] exp(+2 pi i m / kFrN)
  void* staging;           // one block of input or null
  int* err;                // device error word: 1 = a bounded wait gave up
  long long* blk;          // device block counter (advanced by the history shift)
};

struct Shape {
  int S, P, K, B, Tr;
  long long F;
  int J() const { return B * Tr * P; }
  long long row() const { return F + kPrefix; }
};

}  // namespace lp

namespace lp {
// Plans whose per-block launches can be fused into one launch of each kernel
// (lp_group): their per-plan parameters travel in the kernel's parameter block.
constexpr int kMaxGroup = LP_MAX_GROUP;

// Per-plan parameters of the synthesis kernel.
struct IppfPlan {
  const float2* beams;     // rows the synthesis reads (the plan's synth_rows)
  const float* g;
  const float4* tw;
  const float* theta;
  const float* theta2;
  const long long* blk;
  float* y;
  float2* u;               // full-rate mode: series rows (the kernel then stores u and
                           // does not trigger); LSMR right-hand sides: the zt rows; or null
  long long u_row;
  TriggerRec* trig;
  unsigned long long* count;
  long long cap;
  float k_sigma;
  int K, first_bin, P, Tr;
  int stream_end;          // launch streams of plans 0 .. this one
};
template <int N>
struct IppfArgsN {
  long long F, row, F_total, f_base;   // frames of the launch, row length, block frames, offset
  int frames_per_cta;                  // > 0: runs of this many frames; 0: balanced tiling
  int nstreams;                        // launch streams (all plans)
  int pol0, npol, n;
  IppfPlan pl[N];
};
using IppfArgs = IppfArgsN<kMaxGroup>;

// Per-plan parameters of the noise-level kernel.
struct SigmaPlan {
  const float* part;             // noise partials [J][n_per_stream]
  const double* sums;            // sum h, sum h^2 of the prototype
  const long long* blk;
  double* sigma2;
  float* theta;
  float* theta2;
  unsigned long long* count;     // trigger counter zeroed here (group launches) or null
  double alpha, k_sigma;
  int n_per_stream, P;
  int stream_end;
};
struct SigmaArgs {
  long long F;
  int pol0, npol, n;
  SigmaPlan pl[kMaxGroup];
};

// Per-plan parameters of the history shift.
struct ShiftPlan {
  float2* beams;
  float2* fine;
  long long* blk;
  int K, P;
  long long elem_end;            // shifted elements (rows x 16) of plans 0 .. this one
};
struct ShiftArgs {
  long long F, row;
  int advance, pol0, npol, n;
  ShiftPlan pl[kMaxGroup];
};

// One launch range of a block: frames [f_base, f_base + nf) of the block.
struct Chunk {
  long long f_base = 0, nf = 0;
  bool write_beams = true;   // beamformer writes beam rows (false: noise partials only)
  bool write_power = true;   // beamformer writes noise partials
  bool last = true;          // last chunk of the block: the history shift advances the block
};
// The polarisations one launch covers: pols [pol0, pol0 + npol) (npol 0: all).
// Launch stream jj maps to j = (jj / npol) P + pol0 + jj mod npol, the plan's
// stream order, so npol = P is the identity.
struct PolSel {
  int pol0 = 0, npol = 0;
};
__host__ __device__ inline long long sel_stream(long long jj, int P, int pol0, int npol) {
  return (jj / npol) * P + pol0 + jj % npol;
}
}  // namespace lp

struct lp_plan {
  lp::Shape shape;
  long long fc = 0;          // frames per chunk held in the beam rows (F unless chunked)
  long long row() const { return fc + lp::kPrefix; }
  lp_config cfg;
  bool configured = false;
  bool bound = false;
  bool weights_set = false;
  bool tec_set = false;
  int device = -1;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  lp::Buffers buf{};
  long long block_index = 0;
  cudaStream_t last_stream = nullptr;
  int n_ftiles_bf = 0;     // frame tiles of the beamformer (power partials)
  int frames_per_cta = 0;  // synthesis tiling: frames per block, 0 = balanced (one block per SM)
  double nu_ref = 0;
  std::string err;
  // stage timing (lp_profile_enable): event pairs per recorded block, one per
  // part (the polarisations of a host block are processed as separate parts)
  bool profiling = false;
  static constexpr int kProfSlots = 256;
  static constexpr int kProfParts = 2;
  struct ProfTable {       // ~52 KB: on the heap, made by lp_profile_enable
    cudaEvent_t ev[kProfSlots][LP_NUM_STAGES][kProfParts][2] = {};
    bool used[kProfSlots][LP_NUM_STAGES][kProfParts] = {};
  };
  std::shared_ptr<ProfTable> prof;
  int prof_n = 0;
  // host input: copies of the next polarisation overlap the work on the
  // previous one (a copy stream of the plan, one event per polarisation)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_entry = nullptr;
  cudaEvent_t ev_pol[2] = {};
  // streaming host blocks (cfg.stream_blocks): block b uses staging buffer and
  // trigger list b mod 2; ev_free[i] marks the last beamformer read of staging
  // buffer i, ev_done[i] the end of the block in trigger list i
  void* staging_buf[2] = {};
  lp::TriggerRec* trig_buf[2] = {};
  unsigned long long* count_buf[2] = {};
  cudaEvent_t ev_free[2] = {};
  cudaEvent_t ev_done[2] = {};
  cudaStream_t read_stream = nullptr;    // trigger reads of lp_get_triggers_block
  bool free_recorded[2] = {};
  long long block_in[2] = {-1, -1};
  // graph mode (cfg.use_graph): the per-block launch sequence captured once
  cudaGraphExec_t graph_exec = nullptr;
  const void* graph_x = nullptr;
  long long graph_stride = -1;
  long long tune_blk = 0;    // host copy of the device block counter (autotuner)
  int gemm_cfg = -1;         // beamformer configuration (index into beamform_gemm_configs; -1: default)
  // TMA map of the beam rows (CUtensorMap, 128 bytes) for the FP16 form
  alignas(64) unsigned char beams_map[128] = {};
};

namespace lp {

// ---- kernel launchers (each returns the cudaError of the launch) ----------
cudaError_t launch_prototype(const lp_plan& p, cudaStream_t s);
cudaError_t launch_weights(const lp_plan& p, cudaStream_t s);
cudaError_t launch_weights_tc(const lp_plan& p, cudaStream_t s);
cudaError_t encode_beams_map(lp_plan& p);
cudaError_t launch_dedisp(const lp_plan& p, cudaStream_t s);
// x: station block, pol slab p at x + p * pol_stride complex samples, each
// slab [K][F][S] complex samples contiguous
cudaError_t launch_beamform_f32(const lp_plan& p, const void* x, long long pol_stride,
                                cudaStream_t s, PolSel ps = {});
cudaError_t launch_beamform_tc(const lp_plan& p, const void* x, long long pol_stride,
                               const Chunk& c, cudaStream_t s, PolSel ps = {});
cudaError_t launch_sigma(const lp_plan& p, cudaStream_t s, PolSel ps = {});
cudaError_t launch_ippf(const lp_plan& p, const Chunk& c, cudaStream_t s, PolSel ps = {});
cudaError_t launch_ippf_zt(const lp_plan& p, cudaStream_t s);
// One launch of a kernel for the plans of a group (see lp_group in lp.h):
// plan i reads its polarisation slabs at xs[i].  zero_counts: the noise-level
// launch also zeroes every plan's trigger counter.
cudaError_t launch_beamform_tc_plans(const lp_plan* const* plans, const void* const* xs,
                                     long long pol_stride, int n, const Chunk& c, cudaStream_t s,
                                     PolSel ps = {});
cudaError_t launch_sigma_plans(const lp_plan* const* plans, int n, bool zero_counts,
                               cudaStream_t s, PolSel ps = {});
cudaError_t launch_ippf_plans(const lp_plan* const* plans, int n, const Chunk& c, cudaStream_t s,
                              PolSel ps = {});
cudaError_t launch_history_shift_plans(const lp_plan* const* plans, int n, const Chunk& c,
                                       cudaStream_t s, PolSel ps = {});
// advances the device block counter when c.last and ps covers the last pol
cudaError_t launch_history_shift(const lp_plan& p, const Chunk& c, cudaStream_t s,
                                 PolSel ps = {});
// fine de-dispersion: the taps (from the STEC values) and the filter of the
// block's beam rows into the second row buffer
cudaError_t launch_fine_taps(const lp_plan& p, cudaStream_t s);
cudaError_t launch_fine(const lp_plan& p, cudaStream_t s, PolSel ps = {});
// full-rate de-dispersion: the taps' spectrum (from the STEC values), the
// filter of the synthesised series with the trigger, and the series history
cudaError_t launch_fullrate_taps(const lp_plan& p, cudaStream_t s);
cudaError_t launch_fullrate(const lp_plan& p, cudaStream_t s, PolSel ps = {});
cudaError_t launch_fullrate_shift(const lp_plan& p, cudaStream_t s, PolSel ps = {});
// LSMR chain: the recovered series into the full-rate filter's series rows
long long fullrate_row(const lp_plan& p);
size_t fullrate_table_bytes();
// PPF inversion by windowed LSMR (replaces the synthesis and the trigger)
cudaError_t launch_lsmr(const lp_plan& p, cudaStream_t s);
cudaError_t launch_lsmr_trigger(const lp_plan& p, cudaStream_t s);
int lsmr_window();
// the rows the synthesis reads: the filtered ones when fine de-dispersion is on
inline const float2* synth_rows(const lp_plan& p);

// Opt-in shared-memory limits of the kernels (per device; call with it current).
cudaError_t init_kernel_attributes(const Shape& sh);
// The opt-in limit is a property of the kernel on the current device, shared by
// every plan of the process: it is only ever raised (to the largest need seen),
// so a plan that needs less never lowers the limit another plan launches with.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

int beamform_f32_frame_tile();
// Beamformer configurations the GEMM autotuner may pick, two ints each: FP16 form
// (int8 stages, FP16 stages) that fit the shared memory; FP32 form (beams per
// accumulator pass, 0).  Returns the count (at most max).
int beamform_gemm_configs(const lp_plan& p, int* desc, int max);
int beamform_tc_frame_tile();
int beamform_tc_partials(long long F);
size_t beamform_tc_weight_bytes(const Shape& sh);

}  // namespace lp

inline const float2* lp::synth_rows(const lp_plan& p) {
  return p.buf.beams_fine ? p.buf.beams_fine : p.buf.beams;
}
