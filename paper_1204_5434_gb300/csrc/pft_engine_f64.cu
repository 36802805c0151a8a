// FP64 engine: every step in double.  Also hosts the Philox test-hook launchers.
#include "pft_engine_t.cuh"

namespace pft {
Engine* make_engine_f64() { return new EngineT<double>(); }

cudaError_t launch_philox_normals(unsigned long long seed, unsigned long long instance, unsigned long long step,
                                  int field, long long M, double* out, cudaStream_t st) {
  const long long nblk = (M + 3) / 4;
  const int blocks = (int)((nblk + 255) / 256 < 4096 ? (nblk + 255) / 256 : 4096);
  k_philox_normals<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(seed, instance, step, field, M, out);
  return cudaGetLastError();
}

cudaError_t launch_philox_raw(const unsigned int ctr[4], const unsigned int key[2], long long count,
                              unsigned int* out, cudaStream_t st) {
  const int blocks = (int)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
  k_philox_raw<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]),
                                                       make_uint2(key[0], key[1]), count, out);
  return cudaGetLastError();
}
static __global__ void k_narrow_rn(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = narrow_rn(x[i]);
}

cudaError_t launch_narrow_rn(const double* x, float* y, long long n, cudaStream_t st) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_narrow_rn<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}
}  // namespace pft
