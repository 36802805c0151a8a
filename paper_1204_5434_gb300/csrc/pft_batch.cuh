// pft_batch.cuh -- batched pass kernels: one launch runs the same pass of one contour
// step for every active instance of a size class (blockIdx.y = instance).  Instances
// of different contour lengths stay in one launch sequence: at step s the active
// instances are those with Ns >= s, a prefix of the class's members sorted by Ns.
#pragma once
#include "pft_passes.cuh"

namespace pft {

// Everything one instance needs for one contour step of one march.
struct BatchStep {
  const void* in;       // q_{s-1} (or qd_{s-1})
  const void* B;        // Boltzmann factor of this split step
  void* out;            // q_s (or qd_s)
  const void* partner;  // forward slice paired with qd_s (conjugate march)
  double cA, cB;        // quadrature weights of that pair
  void* spec;           // spectrum scratch of the instance
  void* accA;
  void* accB;
  const void* tw[4];    // twiddles x, y, z, z/2
  const void* d[3];     // diffusion tables
};

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(Tile<T>::C * Plan<N>::TPC)
kb_strided(const BatchStep* __restrict__ st, long long ncols, long long cin, long long s_outer, long long s_k, int nzc,
           int axis) {
  const BatchStep& s = st[blockIdx.y];
  strided_body<T, N, MODE>((cpx<T>*)s.spec, ncols, cin, s_outer, s_k, (const cpx<T>*)s.tw[axis], (const T*)s.d[0],
                           (const T*)s.d[1], (const T*)s.d[2], nzc, (long long)blockIdx.x);
}

template <typename T, int N2>
__global__ void __launch_bounds__(PencilsPerCta<T, N2>::v * Plan<N2>::TPC)
kb_zf_r2c(const BatchStep* __restrict__ st, long long npen) {
  const BatchStep& s = st[blockIdx.y];
  zf_r2c_body<T, N2>((const T*)s.in, (const T*)s.B, (cpx<T>*)s.spec, npen, (const cpx<T>*)s.tw[3],
                     (const cpx<T>*)s.tw[2], (long long)blockIdx.x);
}

template <typename T, int N2, int EPI>
__global__ void __launch_bounds__(PencilsPerCta<T, N2>::v * Plan<N2>::TPC)
kb_zi_c2r(const BatchStep* __restrict__ st, long long npen) {
  const BatchStep& s = st[blockIdx.y];
  zi_c2r_body<T, N2, EPI>((const cpx<T>*)s.spec, (const T*)s.B, (T*)s.out, (const T*)s.partner, (double*)s.accA,
                          (double*)s.accB, s.cA, s.cB, npen, (const cpx<T>*)s.tw[3], (const cpx<T>*)s.tw[2],
                          (long long)blockIdx.x);
}

template <typename T, int N>
__global__ void __launch_bounds__(PencilsPerCta<T, N>::v * Plan<N>::TPC)
kb_zf_c2c(const BatchStep* __restrict__ st, long long npen) {
  const BatchStep& s = st[blockIdx.y];
  zf_c2c_body<T, N>((const cpx<T>*)s.in, (const cpx<T>*)s.B, (cpx<T>*)s.spec, npen, (const cpx<T>*)s.tw[2],
                    (long long)blockIdx.x);
}

template <typename T, int N, int EPI>
__global__ void __launch_bounds__(PencilsPerCta<T, N>::v * Plan<N>::TPC)
kb_zi_c2c(const BatchStep* __restrict__ st, long long npen) {
  const BatchStep& s = st[blockIdx.y];
  zi_c2c_body<T, N, EPI>((const cpx<T>*)s.spec, (const cpx<T>*)s.B, (cpx<T>*)s.out, (const cpx<T>*)s.partner,
                         (double2*)s.accA, (double2*)s.accB, s.cA, s.cB, npen, (const cpx<T>*)s.tw[2],
                         (long long)blockIdx.x);
}

}  // namespace pft
