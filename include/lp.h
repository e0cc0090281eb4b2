/*
 * lp.h -- C ABI of the GB300 lunar nanosecond-pulse hot path.
 *
 * The pipeline follows arXiv:1612.06592 (Winchen et al., "Realtime processing
 * of LOFAR data for the detection of nano-second pulses from the Moon"):
 * station subband data are combined into tied-array beams (Sec. 3, first
 * paragraph), corrected for ionospheric dispersion by a STEC-dependent phase in
 * the frequency domain (Sec. 3, third paragraph), turned back into a 200 MHz
 * time series by inverting the polyphase filter bank (Sec. 2 last paragraph and
 * Sec. 3 second paragraph; here an inverse FFT followed by a 16-tap synthesis
 * FIR instead of the paper's sparse solve) and triggered on the envelope
 * amplitude (Sec. 2, Fig. 1).
 *
 * Conventions used by every entry point:
 *   S stations, P polarisations, K contiguous subbands starting at bin
 *   first_bin of a 1024-point filter bank (512 bins, bin b at sky frequency
 *   100 MHz + b * 195.3125 kHz), B beams, Tr STEC trials, F frames per block
 *   (one frame = 1024 samples at 200 MHz = 5.12 us).
 *   A stream is one (beam b, trial t, polarisation p), index j = (b*Tr + t)*P + p.
 *   Output sample n counts 200 MHz samples from the stream start; block i
 *   covers n in [(i*F - 15)*1024, ((i+1)*F - 15)*1024); samples n < 0 (the
 *   first 15 frames of block 0) are computed from zero history and never
 *   trigger.
 *
 * Memory: the library allocates no device memory.  The caller asks for the
 * workspace size, allocates it (cudaMalloc, a PyTorch tensor, ...) and binds
 * it; the plan keeps device pointers into it and all state (synthesis history,
 * running noise level, trigger buffer, phase tables) lives there.  The caller
 * keeps ownership and frees it after lp_plan_destroy.
 *
 * Errors: no entry point aborts.  Every call returns an lp_status; on failure
 * lp_last_error(plan) holds a message.  CUDA errors are caught and reported
 * as LP_ERR_CUDA.  Calls on one plan must not run concurrently from several
 * host threads.
 */
#ifndef LP_H
#define LP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_plan lp_plan;

typedef enum {
  LP_OK = 0,
  LP_ERR_ARG = 1,       /* invalid argument or shape                          */
  LP_ERR_CUDA = 2,      /* a CUDA call or kernel failed                       */
  LP_ERR_OOM = 3,       /* workspace too small                                */
  LP_ERR_STATE = 4,     /* call out of order (e.g. process before set_weights) */
  LP_ERR_OVERFLOW = 5,  /* more triggers than the buffer holds                */
  LP_ERR_TIMEOUT = 6,   /* a bounded device wait gave up                      */
  LP_ERR_BUSY = 7       /* resource in use                                    */
} lp_status;

enum { LP_INPUT_INT8 = 1, LP_INPUT_INT16 = 2 };

/* Beamformer arithmetic.  LP_PREC_FP32: plain FP32 FMA station sum.
 * LP_PREC_FP16: tensor-core CGEMM, weights split into an FP16 high and low
 * part, FP32 accumulation; int8 samples are exact in FP16, int16 samples v
 * enter as the two exact FP16 parts 256 (v >> 8) and v & 255 (four products
 * per sample instead of two).  Needs a multiple of 4 stations. */
enum { LP_PREC_FP32 = 0, LP_PREC_FP16 = 1 };

typedef struct {
  int32_t input_dtype;      /* LP_INPUT_INT8 or LP_INPUT_INT16                  */
  int32_t precision;        /* LP_PREC_FP32 or LP_PREC_FP16                     */
  int32_t first_bin;        /* first selected bin, 1 <= first_bin, first_bin+K <= 512 */
  int32_t taps;             /* synthesis taps; must be 16                       */
  double kaiser_beta;       /* Kaiser window beta of the prototype (9)          */
  double k_sigma;           /* trigger threshold in units of sigma_y (6)        */
  double sigma_alpha;       /* weight of the newest block in the running sigma  */
  double nu_ref_hz;         /* de-dispersion reference; <= 0: band centre       */
  int64_t trigger_cap;      /* device trigger buffer capacity (records)         */
  int32_t store_timeseries; /* 1: keep y = Re u of every stream for lp_get_timeseries */
  int32_t host_input;       /* 1: reserve a device copy of one block so that
                               lp_process_block accepts host pointers            */
  int32_t frames_per_cta;   /* synthesis frames per thread block (a positive multiple of 8);
                               0 = balanced: one block per SM, each walking an equal,
                               contiguous range of the streams' frames */
  int32_t use_graph;        /* 1: lp_process_block replays a captured CUDA graph of the
                               block's launches (needs a non-default stream; recaptured
                               when the input address or pol stride changes; not with
                               profiling) */
  int32_t chunk_frames;     /* 0: the beam rows hold the whole block.  > 0 (FP16 form,
                               multiple of 256 dividing block_len): the block is
                               processed in chunks of this many frames, so the beam
                               intermediate is sized for one chunk; a first beamformer
                               pass sums |beam|^2 over the whole block for the noise
                               level (the same sigma as unchunked) */
  int32_t fine_dedisp;      /* 1: after the per-subband STEC phase, filter each
                               (subband, trial) along frames with the rest of the
                               phase across the subband (Sec. 3, third paragraph,
                               at channel resolution: 17 taps, delay within 4
                               frames of centre, else lp_set_tec fails).  Pulses
                               appear 8 frames (8192 samples) later; needs a second
                               beam-row buffer; not with chunk_frames; lp_get_beams
                               returns the rows before the filter.  0: off */
  int32_t inversion;        /* LP_INV_FIR (0): inverse FFT + 16-tap synthesis FIR, with
                               the trigger.  LP_INV_LSMR (1): the paper's inverse FFT
                               + sparse solve (Sec. 3, second paragraph): per stream
                               and phase the PPF window's banded system, solved in
                               windows of 256 frames (16 of overlap) by lsmr_iters
                               LSMR iterations; block_len a multiple of 256; the
                               trigger runs on the recovered series against a noise
                               level per stream and phase (lp_get_lsmr_sigma); the
                               series lags the frames by 16 (sample (m - 16) M + p)
                               and lp_get_timeseries returns its real part; not with
                               chunk_frames or host blocks per polarisation (a host
                               block is copied whole first) */
  int32_t lsmr_iters;       /* LSMR iterations per window (25); 1 .. 1000 */
  int32_t stream_blocks;    /* 1: streaming host blocks (host_input = 1, whole blocks, no
                               graph, no group): two staging buffers and two trigger lists,
                               used by alternate blocks, so that the host-to-device copy of
                               the next block starts as soon as the block two calls back has
                               been beamformed (not after all earlier work on the stream) and
                               overlaps this block's synthesis; lp_get_triggers_block reads
                               a block's triggers while the next block runs.  0: off */
  int32_t fullrate_dedisp;  /* 1: de-disperse at full resolution after the inversion (Sec. 3,
                               third paragraph: the STEC phase on the spectrum of the
                               200 MHz series): the beamformer applies no per-subband
                               phase, the synthesis keeps each stream's analytic series
                               and a streaming filter of 2048 taps (the response sampled
                               on 8192 frequencies and inverted, a Tukey window flat over
                               the central 1536 taps, a delay of 1024 samples: pulses
                               appear one frame later) applies the whole phase; the trigger
                               and the stored time series are those of the filtered
                               series, the noise level that of the synthesis.  With
                               inversion = LP_INV_LSMR (the paper's order) the filter runs
                               on the recovered series and the LSMR path's per-phase noise
                               level and trigger then run on the filtered series.
                               lp_set_tec refuses STEC values whose group delays over
                               100-200 MHz leave 768 samples of the reference delay.  Not
                               with chunk_frames, fine_dedisp, stream_blocks or in a plan
                               group.  0: off */
} lp_config;

enum { LP_INV_FIR = 0, LP_INV_LSMR = 1 };

/* One trigger: envelope sample above k_sigma * sigma of its stream. */
typedef struct {
  int64_t n;        /* 200 MHz sample index from the stream start */
  int32_t beam;
  int32_t tec;      /* STEC trial index */
  int32_t pol;
  int32_t stream;   /* j = (beam*Tr + tec)*P + pol */
  float env;        /* envelope |u[n]| */
  float sigma;      /* sigma_y of the stream for this block */
} lp_trigger;

/* Fill *cfg with the defaults: int8, FP32, first_bin 12, 16 taps, beta 9,
 * k_sigma 6, alpha 0.25, band-centre reference, 1<<20 triggers, no time
 * series, device input, automatic tiling. */
void lp_config_default(lp_config* cfg);

/* Create a host-side plan for the given shape (Sec. 3: N_S stations, beams
 * toward the Moon, several STEC values).  No device work.  Limits:
 * 1 <= stations <= 64, pols in {1,2}, 1 <= subbands <= 511, 1 <= beams <= 1024,
 * 1 <= tec_trials <= 64, 16 <= block_len <= 2^22 and a multiple of 8. */
lp_status lp_plan_create(lp_plan** out, int stations, int pols, int subbands,
                         int beams, int tec_trials, int64_t block_len);

/* Validate and store a configuration (host only).  Must precede
 * lp_plan_workspace_bytes. */
lp_status lp_plan_configure(lp_plan* plan, const lp_config* cfg);

/* Device workspace the plan needs, in bytes. */
lp_status lp_plan_workspace_bytes(const lp_plan* plan, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned, >= workspace bytes) on
 * the current device.  Zeroes the stream state and builds the synthesis
 * filter on the device, asynchronously on `stream` (a cudaStream_t, NULL for
 * the legacy default stream). */
lp_status lp_plan_bind_workspace(lp_plan* plan, void* device_ptr, size_t bytes,
                                 void* stream);

/* Beam weights w[k,b,s] = exp(-2 pi i nu_k (r_s . s_b) / c) from station
 * positions and beam directions (Sec. 3, first paragraph: "a complex weight
 * given by the station position and the beam direction").
 * station_enu_m: host doubles [S][3] (east, north, up in metres);
 * beam_dir: host doubles [B][3] unit vectors in the same frame.
 * The phase is formed and range-reduced in FP64 on the device, then FP32
 * sincos.  Asynchronous on `stream`; the host arrays may be reused on return. */
lp_status lp_set_weights(lp_plan* plan, const double* station_enu_m,
                         const double* beam_dir, void* stream);

/* STEC trials in TEC units, host doubles [Tr] (Sec. 3, third paragraph:
 * multiply in the frequency domain by a complex weight depending on STEC;
 * several values are tried).  D[k,t] = exp(-2 pi i A_t (nu_k - nu_ref)^2 /
 * (nu_k nu_ref^2)), A_t = 40.308 * STEC_t * 1e16 / c, formed in FP64. */
lp_status lp_set_tec(lp_plan* plan, const double* tec_tecu, void* stream);

/* Process one block of station data, asynchronously on `stream`: the whole
 * realtime chain of Sec. 2 (last paragraph, Fig. 1) on one block -- station
 * signals summed into beams with complex weights (Sec. 3, first paragraph),
 * the STEC phase in the frequency domain (Sec. 3, third paragraph), the
 * inverse FFT of the PPF inversion (Sec. 3, second paragraph) followed here by
 * the 16-tap synthesis FIR, and the envelope trigger that would start the
 * read-out of the transient buffers (Sec. 2, fourth paragraph).
 * x: [P][K][F][S][2] (re, im) int8 or int16, C order, host or device
 * pointer (host pointers need host_input = 1; the copy is part of the call).
 * Runs: beamform + de-disperse, block noise power and running sigma, inverse
 * FFT + synthesis FIR + envelope threshold, history shift.  Triggers of the
 * previous block are discarded.  A host block with P = 2 (not chunked, no
 * graph) is copied one polarisation at a time on a stream of the plan, and
 * the work on polarisation 0 overlaps the copy of polarisation 1; the copy
 * starts once earlier work on `stream` is done, and `stream` finishes after
 * both copies. */
lp_status lp_process_block(lp_plan* plan, const void* x, void* stream);

/* As lp_process_block, for a view of a larger array: pol slab p starts
 * pol_stride complex samples after slab p-1 (each slab [K][F][S][2]
 * contiguous).  Used to hand several plans different subband ranges of one
 * resident station block.  pol_stride must be >= K*F*S (when P = 2) and keep
 * 16-byte alignment for the FP16 form. */
lp_status lp_process_block_strided(lp_plan* plan, const void* x, int64_t pol_stride,
                                   void* stream);

/* The trigger read-out (Sec. 2, fourth paragraph: the recovered nanosecond
 * signal is used only to trigger the read-out of the transient buffer boards;
 * Fig. 1, last step).  Synchronise and copy the triggers of the last processed
 * block to host memory `out` (capacity `cap`, may be NULL when cap == 0), sorted by
 * (beam, tec, pol, n).  *n_total receives the number found.  Returns
 * LP_ERR_OVERFLOW when *n_total exceeds cap or the device buffer (the first
 * min(cap, trigger_cap) records, in sorted order of those kept, are copied). */
lp_status lp_get_triggers(lp_plan* plan, lp_trigger* out, int64_t cap,
                          int64_t* n_total);

/* The trigger read-out of one of the last two processed blocks (block counts
 * lp_process_block calls from the plan's start or last lp_reset_stream, from
 * 0): waits only for that block's work, so with stream_blocks = 1 the next
 * block may already be in flight (its copy and kernels continue).  Otherwise
 * as lp_get_triggers.  LP_ERR_STATE for a block that is not one of the last
 * two (or, without stream_blocks, not the last). */
lp_status lp_get_triggers_block(lp_plan* plan, int64_t block, lp_trigger* out, int64_t cap,
                                int64_t* n_total);

/* The recovered nanosecond-resolution series of one beam (Sec. 3, second
 * paragraph: the inverse FFT of the filtered signal and the inversion of the
 * PPF window; Sec. 2, fourth paragraph: the 5 ns time resolution the PPF had
 * reduced to about 5 us).  Synchronise and copy y = Re u of one stream for the
 * last block, F*1024 floats to host memory, sample (m - 15) M + p of frame m at [m M + p]
 * (store_timeseries = 1 only).  With the LSMR inversion: the real part of the
 * recovered series, sample (m - 16) M + p at [m M + p] (always kept; the
 * stream's complex series, stored phase-major on the device, passes through a
 * temporary host buffer of F * 1024 * 8 bytes for the reordering).
 * LP_ERR_STATE when no series is kept. */
lp_status lp_get_timeseries(lp_plan* plan, int beam, int tec, int pol,
                            float* out_host);

/* Synchronise and copy the beamformed, de-dispersed subband data of one
 * stream for the last block, host floats [K][F][2]. */
lp_status lp_get_beams(lp_plan* plan, int beam, int tec, int pol, float* out_host);

/* Synchronise and copy the running sigma_y of every stream, host doubles [J]
 * (LSMR inversion: the RMS over phases of the per-phase levels). */
lp_status lp_get_sigma(lp_plan* plan, double* sigma_host);

/* LSMR inversion only: the running noise level of the recovered series per
 * stream and phase, host doubles [J][1024] (the solver's noise gain depends on
 * the phase, so the trigger compares |x| with k_sigma times this level).
 * LP_ERR_STATE on a plan without the LSMR inversion. */
lp_status lp_get_lsmr_sigma(lp_plan* plan, double* sigma_host);

/* Forget the stream: zero synthesis history and noise state, block counter 0. */
lp_status lp_reset_stream(lp_plan* plan, void* stream);

/* Autotuner (the paper has no counterpart; it tunes the synthesis kernel's
 * tiling): processes block x exactly as lp_process_block does, and inside that
 * block times the synthesis kernel for frames_per_cta in {64, 128, ..., 2048}
 * (<= the chunk length) and the balanced tiling (0) on the same beam rows,
 * keeps the fastest for later blocks and returns it in *best (ms per candidate
 * in ms_out[7] when not NULL, in that order, 0 for skipped candidates).  The outputs do not depend on the tiling, so the
 * block's results are those of lp_process_block.  Synchronises `stream`;
 * drops a captured graph.  Device input only (contiguous layout). */
lp_status lp_plan_autotune(lp_plan* plan, const void* x, void* stream, int32_t* best,
                           double* ms_out);

/* Beamformer configurations (the GEMM autotuner's candidates; no counterpart
 * in the paper).  Writes up to max pairs into desc[2 i], desc[2 i + 1] and
 * returns their number (at most LP_MAX_GEMM_CONFIGS), or -1 for an unbound
 * plan.  FP16 form: (input ring stages, FP16 ring stages) of the tensor-core
 * beamformer that fit the shared memory for this shape, deepest first; FP32
 * form: (beams per accumulator pass, 0), i.e. (8, 0), (16, 0) and (4, 0).  Every
 * configuration computes the same beams bit for bit. */
#define LP_MAX_GEMM_CONFIGS 8
int lp_plan_gemm_configs(const lp_plan* plan, int32_t* desc, int max);

/* Select beamformer configuration `index` (from lp_plan_gemm_configs) for later
 * blocks; -1 restores the default (the deepest FP16 rings, 8 FP32 beams).
 * LP_ERR_ARG for an index out of range.  Drops a captured graph. */
lp_status lp_plan_set_gemm_config(lp_plan* plan, int index);

/* GEMM autotuner: processes block x exactly as lp_process_block does, and
 * inside that block times the beamformer launch (the whole block, or the
 * block's first chunk for a chunked plan) in every configuration of
 * lp_plan_gemm_configs, mean of 3 timed runs after one warm-up run, on the
 * same input and beam rows; keeps the fastest for later blocks and returns its
 * index in *best (ms per configuration in ms_out[LP_MAX_GEMM_CONFIGS] when not
 * NULL).  The beams do not depend on the configuration, so the block's results
 * are those of lp_process_block.  Synchronises `stream`; drops a captured graph.
 * Device input only (contiguous layout). */
lp_status lp_plan_autotune_gemm(lp_plan* plan, const void* x, void* stream, int32_t* best,
                                double* ms_out);

/* Number of kernel launches lp_process_block makes for a device block (for
 * accounting): 4 (beamformer, noise level, synthesis, history shift), one more
 * with fine_dedisp, 6 with the LSMR inversion (beamformer, inverse FFT, LSMR,
 * noise level, trigger, history shift), two more with fullrate_dedisp (the
 * filter and its history shift); the fine filter adds a launch, and the LSMR
 * and trigger kernels, and the full-rate filter, one each per 65535 rows /
 * streams beyond the first.  A host block processed per polarisation makes
 * twice the FIR-path count. */
int lp_launches_per_block(const lp_plan* plan);

/* Stage timing.  When enabled, lp_process_block records a CUDA event pair
 * around each stage on the stream it launches on (the host-to-device copy,
 * the beamformer, the noise level, the synthesis, the history shift, the fine
 * de-dispersion filter), for up
 * to 256 blocks.  lp_profile_read synchronises, adds the durations of every
 * recorded block into total_ms[LP_NUM_STAGES] (milliseconds), stores their
 * number in *blocks and forgets them. */
enum { LP_STAGE_H2D = 0, LP_STAGE_BEAMFORM = 1, LP_STAGE_SIGMA = 2, LP_STAGE_SYNTH = 3,
       LP_STAGE_SHIFT = 4, LP_STAGE_FINE = 5, LP_STAGE_FULLRATE = 6, LP_NUM_STAGES = 7 };
lp_status lp_profile_enable(lp_plan* plan, int enable);
lp_status lp_profile_read(lp_plan* plan, double* total_ms, int64_t* blocks);

/* ---- Groups: several plans' blocks in shared launches ---------------------
 *
 * No counterpart in the paper; this is the serving loop's batching.  Requests
 * that subscribe to one station stream each own a plan (their beams, STEC
 * trials and contiguous subband range, with their own history, noise level
 * and trigger list).  A group fuses the per-block launches of up to
 * LP_MAX_GROUP such plans: one beamformer launch over every plan's work items,
 * one noise-level launch (which also clears every plan's trigger counter), one
 * synthesis launch over every plan's streams and one history shift -- four
 * launches per block however many plans (four per polarisation with
 * lp_group_process_block_pol).  Each plan computes exactly what its own
 * lp_process_block computes, bit for bit.
 *
 * Member plans: bound, lp_set_weights and lp_set_tec done, the FP16 form,
 * whole blocks (chunk_frames 0), the FIR synthesis without fine
 * de-dispersion, one device, equal stations, polarisations, block length and
 * input type.  The group uses the first plan's synthesis tiling and
 * beamformer configuration (results do not depend on either) and reports a
 * timed-out device wait through the first plan's lp_get_triggers. */
#define LP_MAX_GROUP 32
typedef struct lp_group lp_group;

/* Host only: a group of n distinct plans (1 <= n <= LP_MAX_GROUP).  The plans
 * stay owned by the caller and must outlive the group.  LP_ERR_ARG for a bad
 * list, LP_ERR_STATE when a plan does not qualify (see above). */
lp_status lp_group_create(lp_group** out, lp_plan* const* plans, int n);

/* One block for every plan of the group, asynchronously on `stream`.
 * x: device block [P][subbands][F][S][2] complex int8 or int16 (the plans'
 * type) holding the contiguous bins [first_bin, first_bin + subbands),
 * 16-byte aligned with 16-byte aligned subband rows (F * S * 2 or 4 bytes);
 * each plan reads its own bins.
 * Afterwards each plan's lp_get_triggers / lp_get_sigma / lp_get_timeseries
 * read its results as after lp_process_block. */
lp_status lp_group_process_block(lp_group* group, const void* x, int32_t subbands,
                                 int32_t first_bin, void* stream);

/* The same block one polarisation at a time (pol = 0, then 1, ... for every
 * block), four launches per call, with the layout and results of
 * lp_group_process_block: only x's slab of polarisation `pol` is read, so a
 * caller can launch a polarisation as soon as its slab has arrived.
 * LP_ERR_ARG for pol outside [0, P); LP_ERR_STATE for a polarisation out of
 * order, and for lp_group_process_block in the middle of a block.  A call that
 * fails leaves the group expecting the same polarisation again. */
lp_status lp_group_process_block_pol(lp_group* group, const void* x, int32_t subbands,
                                     int32_t first_bin, int32_t pol, void* stream);

/* Plans in the group; kernel launches per block (4). */
int lp_group_size(const lp_group* group);
int lp_group_launches_per_block(const lp_group* group);
const char* lp_group_last_error(const lp_group* group);
/* Frees the host object only (the plans are the caller's). */
void lp_group_destroy(lp_group* group);

/* Size of the static device scratch of lp_process_block_noalloc: 16 MiB,
 * held by every GPU that loads the library until the process exits. */
#define LP_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code running inside a host process that
 * forbids device allocation once it is running (a real-time loop with a fixed
 * memory budget) or that owns the device heap itself (a plug-in handed only
 * the buffers its framework planned) -- and so cannot bind a plan workspace.
 * It runs one block of the FP32 form (beam weights and de-dispersion tables,
 * beamforming, noise level, synthesis and trigger) as the first block of a
 * stream (zero history) and allocates nothing: its scratch is a static device
 * array of LP_NOALLOC_SCRATCH_BYTES.
 *   Shape arguments as lp_plan_create; cfg as lp_plan_configure (precision
 *   must be LP_PREC_FP32; store_timeseries, host_input and stream_blocks are ignored).
 *   station_enu_m [S][3], beam_dir [B][3], tec_tecu [Tr]: host doubles.
 *   x: device block [P][K][F][S][2], aligned to one complex sample (2 bytes
 *   int8, 4 bytes int16).
 *   y: device floats [J][F*1024], y = Re u of every stream (written).
 *   sigma2: device doubles [J] (written) or NULL: the block's sigma_y^2.
 *   triggers: device records, capacity trigger_cap (>= 0), unsorted;
 *   trigger_count: device counter (set to the number found) or NULL.
 *   Every device argument must be device or managed memory of the current
 *   device, aligned to its element type; otherwise LP_ERR_ARG before any
 *   GPU work.
 *   err/errlen: optional host buffer for a message.
 * Returns LP_ERR_ARG, without touching the device, for a shape whose scratch
 * would exceed LP_NOALLOC_SCRATCH_BYTES.  Asynchronous on `stream`; the host
 * geometry arrays are copied from pageable memory, so they may be reused on
 * return.  All calls on a device share the scratch (it keeps the last call's
 * contents; the call clears what must start at zero), so calls whose GPU work
 * overlaps race and must be serialised by the caller.  The first call on a
 * device looks up the scratch address and should come before any stream
 * capture. */
lp_status lp_process_block_noalloc(int stations, int pols, int subbands, int beams,
                                   int tec_trials, int64_t block_len, const lp_config* cfg,
                                   const double* station_enu_m, const double* beam_dir,
                                   const double* tec_tecu, const void* x, float* y,
                                   double* sigma2, lp_trigger* triggers, int64_t trigger_cap,
                                   unsigned long long* trigger_count, void* stream, char* err,
                                   size_t errlen);

void lp_plan_destroy(lp_plan* plan);
const char* lp_last_error(const lp_plan* plan);
const char* lp_status_string(lp_status s);

/* ---- Two-stage beamforming: preliminary beams of station groups --------
 *
 * Sec. 4 (network paragraph): only a few 16-bit station streams fit through
 * the link to the processing cluster, so the correlator first forms
 * preliminary beams from subsets of stations and the final beams are formed
 * from those.  lp_prebeam is that first stage on the GPU:
 *     pb[p][k][m][g] = sum over stations s of group g of w1[k][s] x[p][k][m][s],
 *     w1[k][s] = exp(-2 pi i nu_k ((r_s - r_g) . s_g) / c),
 * r_g the group's phase centre (mean position of its stations), s_g the
 * group's direction, nu_k the sky frequency of bin first_bin + k.  Each value
 * leaves as complex int16, round half to even of scale * pb, saturated to
 * [-32767, 32767], in the station-block layout [P][K][F][G][2] (re, im), so
 * that an lp_plan with stations = G, LP_INPUT_INT16 and the group centres as
 * station positions (lp_prebeam_group_centres) forms the final beams.
 * Groups are disjoint; a station in no group is unused.  FP32 products and
 * sums; the phase argument in FP64 cycles. */
typedef struct lp_prebeam lp_prebeam;

/* Shapes only (no device work): stations S, pols 1 or 2, subbands K, frames F,
 * groups 1 <= G <= S, bins [first_bin, first_bin + K) inside [1, 512),
 * LP_INPUT_INT8 or LP_INPUT_INT16.  LP_ERR_ARG for anything out of range. */
lp_status lp_prebeam_create(lp_prebeam** out, int stations, int pols, int subbands,
                            int64_t block_len, int groups, int first_bin, int input_dtype);

/* Device workspace of the preliminary-beam plan in bytes (weight table,
 * member lists, saturation counter; sized for every station in a group).  Like
 * the pipeline plan, lp_prebeam allocates no device memory: the caller
 * allocates the workspace and binds it. */
lp_status lp_prebeam_workspace_bytes(const lp_prebeam* pb, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned, >= the workspace bytes)
 * on the device it lives on; clears the saturation counter on `stream`.  Once
 * per plan (LP_ERR_STATE for a second bind); the caller frees the memory after
 * lp_prebeam_destroy. */
lp_status lp_prebeam_bind_workspace(lp_prebeam* pb, void* device_ptr, size_t bytes,
                                    void* stream);

/* group_of_station[S] in [-1, G) (-1: unused; every group needs a station),
 * station_enu[S][3] metres, group_dir[G][3] unit vectors (host arrays, read
 * before return).  Computes the phase centres and the weight table in the
 * bound workspace on `stream`.  LP_ERR_STATE before a workspace is bound,
 * LP_ERR_ARG for a bad table, LP_ERR_CUDA for a CUDA failure. */
lp_status lp_prebeam_set_groups(lp_prebeam* pb, const int32_t* group_of_station,
                                const double* station_enu, const double* group_dir,
                                void* stream);

/* The group phase centres, host doubles [G][3] (the final stage's station
 * positions).  LP_ERR_STATE before lp_prebeam_set_groups. */
lp_status lp_prebeam_group_centres(lp_prebeam* pb, double* centre_enu);

/* One block: x device [P][K][F][S][2] int8 or int16 (the plan's dtype, aligned
 * to its complex sample), y device [P][K][F][G][2] int16 (4-byte aligned, the
 * caller's), scale > 0.  Asynchronous on `stream`; y must not overlap x. */
lp_status lp_prebeam_run(lp_prebeam* pb, const void* x, void* y, float scale, void* stream);

/* Synchronises the last stream used and returns, in *n, how many int16 values
 * saturated since the previous call (then resets the count). */
lp_status lp_prebeam_saturated(lp_prebeam* pb, int64_t* n);

const char* lp_prebeam_last_error(const lp_prebeam* pb);
void lp_prebeam_destroy(lp_prebeam* pb);

#ifdef __cplusplus
}
#endif
#endif /* LP_H */
