// lp_group: the per-block launches of several plans fused into one launch of
// each kernel (continuous batching of the serving loop).
//
// A group holds bound plans that subscribe to one station stream: each plan
// covers its own contiguous subband range, beams and STEC trials, and keeps
// its own synthesis history, running noise level, block counter and trigger
// list in its own workspace.  lp_group_process_block runs, for all of them,
// one beamformer launch (the work items of every plan in one persistent
// grid), one noise-level launch (which also clears every plan's trigger
// counter), one synthesis launch over every plan's streams and one history
// shift: four launches per block whatever the number of plans (or four per
// polarisation with lp_group_process_block_pol, so that the second
// polarisation's copy can run under the first's kernels).  Each plan's
// arithmetic is the one its own lp_process_block performs, in the same order,
// so its results are bit for bit those it gives alone.
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "lp_internal.cuh"

struct lp_group {
  std::vector<lp_plan*> plans;
  int device = -1;
  long long blocks = 0;
  int next_pol = 0;        // per-polarisation calls: the polarisation the block needs next
  std::string err;
};

namespace {

lp_status gfail(lp_group* g, lp_status st, const char* fmt, ...) {
  if (g) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g->err = buf;
  }
  return st;
}

// Why plan q cannot join a group led by plan p0 (nullptr: it can).
const char* incompatible(const lp_plan& p0, const lp_plan& q) {
  if (!q.bound || !q.weights_set || !q.tec_set)
    return "a plan is not bound or lacks lp_set_weights / lp_set_tec";
  if (q.cfg.precision != LP_PREC_FP16) return "group launches take the FP16 tensor-core form";
  if (q.fc != q.shape.F) return "group launches take whole blocks (chunk_frames = 0)";
  if (q.cfg.stream_blocks) return "group launches do not take stream_blocks plans";
  if (q.cfg.fine_dedisp || q.cfg.fullrate_dedisp || q.cfg.inversion != LP_INV_FIR)
    return "group launches take the FIR synthesis without fine or full-rate de-dispersion";
  if (q.device != p0.device) return "the plans live on different devices";
  if (q.shape.S != p0.shape.S || q.shape.P != p0.shape.P || q.shape.F != p0.shape.F)
    return "the plans differ in stations, polarisations or block length";
  if (q.cfg.input_dtype != p0.cfg.input_dtype) return "the plans differ in input type";
  return nullptr;
}

// The block (ps: all polarisations) or one polarisation of it, for every plan:
// the noise-level launch of the first polarisation clears the trigger
// counters, and the history shift advances the block counters once ps reaches
// the last polarisation.
lp_status group_block(lp_group* g, const void* x, int32_t subbands, int32_t first_bin,
                      lp::PolSel ps, void* stream) {
  if (!x) return gfail(g, LP_ERR_ARG, "null input");
  const lp_plan& p0 = *g->plans[0];
  const auto& sh = p0.shape;
  if (subbands < 1 || first_bin < 1 || first_bin + subbands > lp::kBins)
    return gfail(g, LP_ERR_ARG, "bins [%d, %d) must lie inside [1, 512)", first_bin,
                 first_bin + subbands);
  for (lp_plan* p : g->plans) {
    if (const char* why = incompatible(p0, *p)) return gfail(g, LP_ERR_STATE, "%s", why);
    if (p->cfg.first_bin < first_bin || p->cfg.first_bin + p->shape.K > first_bin + subbands)
      return gfail(g, LP_ERR_ARG, "a plan's bins [%d, %d) lie outside the block's [%d, %d)",
                   p->cfg.first_bin, p->cfg.first_bin + p->shape.K, first_bin,
                   first_bin + subbands);
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != g->device) e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return gfail(g, LP_ERR_CUDA, "%s", cudaGetErrorString(e));
  cudaPointerAttributes attr;
  e = cudaPointerGetAttributes(&attr, x);
  if (e != cudaSuccess) return gfail(g, LP_ERR_CUDA, "%s", cudaGetErrorString(e));
  if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
      attr.device != g->device)
    return gfail(g, LP_ERR_ARG, "the block must be device memory of the plans' device");
  // every plan's slab offset keeps the 16-byte alignment of the beamformer's
  // bulk copies
  const long long slab = (long long)sh.F * sh.S *
                         (p0.cfg.input_dtype == LP_INPUT_INT8 ? 2 : 4);   // bytes of one subband row
  if (reinterpret_cast<uintptr_t>(x) % 16 || slab % 16)
    return gfail(g, LP_ERR_ARG, "block and subband rows must be 16-byte aligned");
  const int n = (int)g->plans.size();
  std::vector<const void*> xs(n);
  std::vector<const lp_plan*> cp(g->plans.begin(), g->plans.end());
  for (int i = 0; i < n; ++i)
    xs[i] = static_cast<const char*>(x) + (long long)(cp[i]->cfg.first_bin - first_bin) * slab;
  const long long pol_stride = (long long)subbands * sh.F * sh.S;   // complex samples
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lp::Chunk c;
  c.nf = sh.F;
  const bool first = ps.pol0 == 0;
  const bool last = ps.npol == 0 || ps.pol0 + ps.npol == sh.P;
  e = lp::launch_beamform_tc_plans(cp.data(), xs.data(), pol_stride, n, c, s, ps);
  if (e == cudaSuccess) e = lp::launch_sigma_plans(cp.data(), n, first, s, ps);
  if (e == cudaSuccess) e = lp::launch_ippf_plans(cp.data(), n, c, s, ps);
  if (e == cudaSuccess) e = lp::launch_history_shift_plans(cp.data(), n, c, s, ps);
  if (e != cudaSuccess) return gfail(g, LP_ERR_CUDA, "%s", cudaGetErrorString(e));
  for (lp_plan* p : g->plans) p->last_stream = s;
  if (last) {
    for (lp_plan* p : g->plans) p->block_index += 1;
    g->blocks += 1;
  }
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_group_create(lp_group** out, lp_plan* const* plans, int n) {
  if (!out) return LP_ERR_ARG;
  *out = nullptr;
  if (!plans || n < 1 || n > lp::kMaxGroup) return LP_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return LP_ERR_ARG;
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return LP_ERR_ARG;       // a plan appears once
    if (incompatible(*plans[0], *plans[i])) return LP_ERR_STATE;
  }
  lp_group* g = new (std::nothrow) lp_group;
  if (!g) return LP_ERR_OOM;
  g->plans.assign(plans, plans + n);
  g->device = plans[0]->device;
  *out = g;
  return LP_OK;
}

lp_status lp_group_process_block(lp_group* g, const void* x, int32_t subbands,
                                 int32_t first_bin, void* stream) {
  if (!g) return LP_ERR_ARG;
  if (g->next_pol != 0)
    return gfail(g, LP_ERR_STATE, "the block's polarisation %d has not been processed",
                 g->next_pol);
  return group_block(g, x, subbands, first_bin, lp::PolSel{}, stream);
}

lp_status lp_group_process_block_pol(lp_group* g, const void* x, int32_t subbands,
                                     int32_t first_bin, int32_t pol, void* stream) {
  if (!g) return LP_ERR_ARG;
  const int P = g->plans[0]->shape.P;
  if (pol < 0 || pol >= P) return gfail(g, LP_ERR_ARG, "polarisation %d outside [0, %d)", pol, P);
  if (pol != g->next_pol)
    return gfail(g, LP_ERR_STATE, "polarisation %d expected, %d given", g->next_pol, pol);
  const lp_status st = group_block(g, x, subbands, first_bin, lp::PolSel{pol, 1}, stream);
  if (st == LP_OK) g->next_pol = (pol + 1) % P;
  return st;
}

int lp_group_size(const lp_group* g) { return g ? (int)g->plans.size() : 0; }

int lp_group_launches_per_block(const lp_group* g) { return g ? 4 : 0; }

const char* lp_group_last_error(const lp_group* g) { return g ? g->err.c_str() : "null group"; }

void lp_group_destroy(lp_group* g) { delete g; }

}  // extern "C"
