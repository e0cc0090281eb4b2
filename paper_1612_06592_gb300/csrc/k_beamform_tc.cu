// Beamforming + de-dispersion on the tensor cores (FP16 form); filled in by
// the tcgen05 implementation.
#include "lp_internal.cuh"

namespace lp {

int beamform_tc_frame_tile() { return 128; }
size_t beamform_tc_weight_bytes(const Shape& sh) { return (size_t)sh.K * 256 * 4 * sizeof(__half); }
cudaError_t launch_beamform_tc(const lp_plan&, const void*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lp
