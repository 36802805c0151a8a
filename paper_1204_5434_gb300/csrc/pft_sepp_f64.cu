// The separable pencil march in FP64 (its own translation unit: compiled in parallel).
#include "pft_engine.h"
#include "pft_sepp.cuh"

namespace pft {
cudaError_t sepp_launch_f64(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm) {
  return sepp_launch_t<double>(g, ss, j, members, sm);
}
}  // namespace pft
