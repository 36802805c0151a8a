// The separable pencil march of an FP64 context in double-float arithmetic (its own
// translation unit: compiled in parallel).
#include "pft_engine.h"
#include "pft_sepp.cuh"

namespace pft {
cudaError_t sepp_launch_dd(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm) {
  return sepp_launch_t<dd>(g, ss, j, members, sm);
}
}  // namespace pft
