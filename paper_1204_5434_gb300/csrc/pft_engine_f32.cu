// FP32-mixed engine: propagators and FFTs in float, accumulation in double.
#include "pft_engine_t.cuh"

namespace pft {
Engine* make_engine_f32() { return new EngineT<float>(); }
}  // namespace pft
