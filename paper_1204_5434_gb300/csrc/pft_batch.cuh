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
  const void* Bnext;    // Boltzmann factor of the next split step (fused z passes), or null
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

// Fused z passes of consecutive contour steps on the same pencils: inverse z of step s
// (half spectrum -> nz reals), x B_s, store q_s; then x B_{s+1}, forward z of step s+1
// back into the spectrum.  The C2R output and the R2C input share one thread
// distribution, so q_s never leaves registers between the two transforms.
template <typename T, int N2>
__global__ void __launch_bounds__(PencilsPerCta<T, N2>::v * Plan<N2>::TPC)
kb_zz_r2c(const BatchStep* __restrict__ st, long long npen) {
  const BatchStep& s = st[blockIdx.y];
  using Z = cpx<T>;
  constexpr int P = PencilsPerCta<T, N2>::v;
  constexpr int E = Plan<N2>::E;
  constexpr int TPC = Plan<N2>::TPC;
  constexpr int LD = pencil_ld<T>(N2);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long pen = (long long)blockIdx.x * P + p;
  const bool valid = pen < npen;
  const long long pc = valid ? pen : 0;
  XchPencil<T> x{reinterpret_cast<Z*>(smraw) + p * LD};
  Z* sp = (Z*)s.spec + pc * (N2 + 1);
  const Z* twh = (const Z*)s.tw[3];
  const Z* twf = (const Z*)s.tw[2];
  const long long o = pc * N2;
  // FP32: B_s of the pencil first (its latency overlaps the inverse transform) and kept
  // for step s+1 inside a block; FP64 (FP64-pipe bound, registers short) loads it after
  constexpr bool kPre = sizeof(T) == 4;
  const Z* b2 = reinterpret_cast<const Z*>(s.B) + o;
  Z bb[E];
  if (kPre) {
#pragma unroll
    for (int i = 0; i < E; i++) bb[i] = b2[t + TPC * i];
  }
#pragma unroll
  for (int i = 0; i < E; i++) x.put(t + TPC * i, valid ? sp[t + TPC * i] : mk<T>(T(0), T(0)));
  if (t == 0) x.put(N2, valid ? sp[N2] : mk<T>(T(0), T(0)));
  __syncwarp();
  Z v[E];
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int k = t + TPC * i;
    const Z xk = x.get(k);
    const Z xc = cconj(x.get(N2 - k));
    const Z d = rot90<true>(cmulc(csub(xk, xc), twf[k]));
    v[i] = cadd(cadd(xk, xc), d);
  }
  __syncwarp();
  fft<T, true, N2>(v, t, twh, x);
  Z* q2 = reinterpret_cast<Z*>(s.out) + o;
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int m = t + TPC * i;
    const Z b = kPre ? bb[i] : b2[m];
    v[i].x *= b.x;
    v[i].y *= b.y;
    if (valid) q2[m] = v[i];
  }
  if (!s.Bnext) return;  // uniform per launch member
  const Z* bn = reinterpret_cast<const Z*>(s.Bnext) + o;
  if constexpr (kPre) {
    if (s.Bnext != s.B) {  // the block junction; inside a block the same factors apply again
#pragma unroll
      for (int i = 0; i < E; i++) bb[i] = bn[t + TPC * i];
    }
#pragma unroll
    for (int i = 0; i < E; i++) {
      v[i].x *= bb[i].x;
      v[i].y *= bb[i].y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; i++) {
      const Z b = bn[t + TPC * i];
      v[i].x *= b.x;
      v[i].y *= b.y;
    }
  }
  fft<T, false, N2>(v, t, twh, x);  // the inverse ended with a barrier after its last reads
#pragma unroll
  for (int i = 0; i < E; i++) x.put(t + TPC * i, v[i]);
  __syncwarp();
  const T h = T(0.5);
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int k = t + TPC * i;
    const Z zc = cconj(x.get(k == 0 ? 0 : N2 - k));
    const Z ev = cscale(cadd(v[i], zc), h);
    const Z od = cscale(rot90<false>(csub(v[i], zc)), h);
    if (valid) sp[k] = cadd(ev, cmul(twf[k], od));
  }
  if (valid && t == 0) sp[N2] = mk<T>(v[0].x - v[0].y, T(0));
}

// Complex fields: inverse z of step s, x B_s, store, x B_{s+1}, forward z of step s+1.
template <typename T, int N>
__global__ void __launch_bounds__(PencilsPerCta<T, N>::v * Plan<N>::TPC)
kb_zz_c2c(const BatchStep* __restrict__ st, long long npen) {
  const BatchStep& s = st[blockIdx.y];
  using Z = cpx<T>;
  constexpr int P = PencilsPerCta<T, N>::v;
  constexpr int E = Plan<N>::E;
  constexpr int TPC = Plan<N>::TPC;
  constexpr int LD = pencil_ld<T>(N);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long pen = (long long)blockIdx.x * P + p;
  const bool valid = pen < npen;
  const long long o = (valid ? pen : 0) * N;
  XchPencil<T> x{reinterpret_cast<Z*>(smraw) + p * LD};
  Z* sp = (Z*)s.spec;
  const Z* tw = (const Z*)s.tw[2];
  // FP32: B_s first (its latency overlaps the inverse transform) and kept for step s+1
  // inside a block; FP64 (FP64-pipe bound, registers short) loads it after
  constexpr bool kPre = sizeof(T) == 4;
  Z v[E], bb[E];
  const Z* B = (const Z*)s.B;
  if (kPre) {
#pragma unroll
    for (int i = 0; i < E; i++) bb[i] = B[o + t + TPC * i];
  }
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = valid ? sp[o + t + TPC * i] : mk<T>(T(0), T(0));
  fft<T, true, N>(v, t, tw, x);
  Z* q = (Z*)s.out;
#pragma unroll
  for (int i = 0; i < E; i++) {
    const long long m = o + t + TPC * i;
    v[i] = cmul(v[i], kPre ? bb[i] : B[m]);
    if (valid) q[m] = v[i];
  }
  if (!s.Bnext) return;
  const Z* Bn = (const Z*)s.Bnext;
  if constexpr (kPre) {
    if (s.Bnext != s.B) {  // the block junction; inside a block the same factors apply again
#pragma unroll
      for (int i = 0; i < E; i++) bb[i] = Bn[o + t + TPC * i];
    }
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cmul(v[i], bb[i]);
  } else {
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cmul(v[i], Bn[o + t + TPC * i]);
  }
  if (n_stages<Plan<N>>() > 1) __syncwarp();
  fft<T, false, N>(v, t, tw, x);
  if (valid) {
#pragma unroll
    for (int i = 0; i < E; i++) sp[o + t + TPC * i] = v[i];
  }
}

}  // namespace pft
