// pft_persist.cuh -- a whole march of a real-field (SCFT) system in ONE persistent
// cooperative launch over every SM (two CTAs per SM), FP32 propagators.
//
// Each contour step (the split step of Eq. 13) runs the same tiles as the pass kernels,
// spread over all CTAs, with a bounded grid barrier between phases instead of a kernel
// boundary:
//   y forward | x forward, x D(k)/M, x inverse | y inverse | z inverse of step s with
//   its epilogue (x B_s, store q_s or accumulate the quadrature of Eq. 8), x B_{s+1},
//   z forward of step s+1 -- the last two fused in registers on the same pencils.
#pragma once
#include "pft_passes.cuh"

namespace pft {

struct PersistArgs {
  const float* BA;
  const float* BB;
  float* hist;
  const float* qd0;
  float* qd_out;
  float2* spec;
  double* accA;
  double* accB;
  const float2* twx;
  const float2* twy;
  const float2* twz;
  const float2* twh;
  const float* dx;
  const float* dy;
  const float* dz;
  int Ns;
  int NsA;
  unsigned* bar;
  int* err;
  long long spin_limit;
};

__device__ __forceinline__ unsigned p_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void p_red_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void p_fence() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Bounded grid barrier on a counter that only grows within a launch: the k-th barrier
// waits for k * gridDim.x arrivals (reset to 0 by the host before each launch).  Returns
// false in every thread if a wait ran out or another CTA already failed.
__device__ __forceinline__ bool p_barrier(const PersistArgs& a, int* s_flag, unsigned& k) {
  k++;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    p_fence();
    p_red_release(a.bar, 1u);
    const unsigned target = k * gridDim.x;
    const long long t0 = clock64();
    while (p_ld_acquire(a.bar) < target) {
      if (*(volatile int*)a.err) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > a.spin_limit) {
        atomicExch(a.err, 1);
        ok = 0;
        break;
      }
    }
    p_fence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

template <int N> struct Persist {
  static constexpr int THREADS = 256;
  static constexpr int N2 = N / 2;
  static constexpr int NZH = N2 + 1;
  using XPL = Plan<N>;                        // x and y transforms
  using ZPL = Plan<N2>;                       // packed z transforms
  static constexpr int C = THREADS / XPL::TPC;  // columns per strided tile
  static constexpr int P = THREADS / ZPL::TPC;  // pencils per z tile
  static constexpr int LDZ = pencil_ld<float>(N2);
  static constexpr size_t SMEM_X = (size_t)N * C * sizeof(float2);
  static constexpr size_t SMEM_Z = (size_t)P * LDZ * sizeof(float2);
  static constexpr size_t SMEM = SMEM_X > SMEM_Z ? SMEM_X : SMEM_Z;
  static_assert(THREADS % XPL::TPC == 0 && THREADS % ZPL::TPC == 0, "thread split");
};

// z inverse of step s on P pencils (when zin), epilogue, then z forward of step s+1
// (when Bnext): the C2R output and the R2C input share the thread distribution.
template <int N>
__device__ __forceinline__ void zz_tile(const PersistArgs& a, long long tile, bool zin, const float* __restrict__ qin,
                                        const float* __restrict__ Bcur, float* __restrict__ qstore,
                                        const float* __restrict__ partner, double cA, double cB,
                                        const float* __restrict__ Bnext) {
  using R = Persist<N>;
  constexpr int N2 = R::N2, E = R::ZPL::E, TPC = R::ZPL::TPC, P = R::P;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int pi = threadIdx.x / TPC;
  const long long npen = (long long)N * N;
  const long long pen = tile * P + pi;
  const bool valid = pen < npen;
  const long long pc = valid ? pen : 0;
  XchPencil<float> x{reinterpret_cast<float2*>(smraw) + pi * R::LDZ};
  float2* sp = a.spec + pc * R::NZH;
  const long long o = pc * N2;  // float2 index of this pencil's first pair
  float2 v[E];
  if (!zin) {
    const float2* q2 = reinterpret_cast<const float2*>(qin) + o;
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = valid ? q2[t + TPC * i] : make_float2(0.f, 0.f);
  } else {
    float2 pv[E];
    const bool acc_on = partner != nullptr && valid;
    if (acc_on) {
      const float2* pp = reinterpret_cast<const float2*>(partner) + o;
#pragma unroll
      for (int i = 0; i < E; i++) pv[i] = __ldcs(pp + t + TPC * i);
    }
#pragma unroll
    for (int i = 0; i < E; i++) x.put(t + TPC * i, valid ? sp[t + TPC * i] : make_float2(0.f, 0.f));
    if (t == 0) x.put(N2, valid ? sp[N2] : make_float2(0.f, 0.f));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      const float2 xk = x.get(k);
      const float2 xc = cconj(x.get(N2 - k));
      const float2 d = rot90<true>(cmulc(csub(xk, xc), a.twz[k]));
      v[i] = cadd(cadd(xk, xc), d);
    }
    __syncthreads();
    fft<float, true, N2, typename R::ZPL>(v, t, a.twh, x);
    const float2* b2 = reinterpret_cast<const float2*>(Bcur) + o;
    float2* qs = qstore ? reinterpret_cast<float2*>(qstore) + o : nullptr;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int m = t + TPC * i;
      const float2 b = b2[m];
      v[i].x *= b.x;
      v[i].y *= b.y;
      if (qs && valid) __stcs(qs + m, v[i]);
    }
    if (acc_on) {
      for (int blk = 0; blk < 2; blk++) {
        const double c = blk ? cB : cA;
        if (c == 0.0) continue;
        double2* acc = reinterpret_cast<double2*>(blk ? a.accB : a.accA) + o;
        double2 av[E];
#pragma unroll
        for (int i = 0; i < E; i++) av[i] = acc[t + TPC * i];
#pragma unroll
        for (int i = 0; i < E; i++) {
          av[i].x += c * widen(v[i].x * pv[i].x);
          av[i].y += c * widen(v[i].y * pv[i].y);
          acc[t + TPC * i] = av[i];
        }
      }
    }
  }
  if (Bnext) {
    const float2* b2 = reinterpret_cast<const float2*>(Bnext) + o;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const float2 b = b2[t + TPC * i];
      v[i].x *= b.x;
      v[i].y *= b.y;
    }
    __syncthreads();
    fft<float, false, N2, typename R::ZPL>(v, t, a.twh, x);
#pragma unroll
    for (int i = 0; i < E; i++) x.put(t + TPC * i, v[i]);
    __syncthreads();
    float2 zc[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      zc[i] = cconj(x.get(k == 0 ? 0 : N2 - k));
    }
    const float h = 0.5f;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      const float2 ev = cscale(cadd(v[i], zc[i]), h);
      const float2 od = cscale(rot90<false>(csub(v[i], zc[i])), h);
      if (valid) sp[k] = cadd(ev, cmul(a.twz[k], od));
    }
    if (valid && t == 0) sp[N2] = make_float2(v[0].x - v[0].y, 0.f);
  }
  __syncthreads();  // this tile's shared-memory reads precede the next tile's writes
}

template <int N, bool BWD>
__global__ void __launch_bounds__(Persist<N>::THREADS, 2) k_persist_march(PersistArgs a) {
  using R = Persist<N>;
  __shared__ int s_flag;
  unsigned nbar = 0;
  const long long M = (long long)N * N * N;
  const long long ncols = (long long)N * R::NZH;
  const long long nxt = (ncols + R::C - 1) / R::C;               // strided tiles
  const long long nzt = ((long long)N * N + R::P - 1) / R::P;      // z tiles
  const int Ns = a.Ns, NsA = a.NsA;
  auto Bof = [&](int s) -> const float* {
    const int n = BWD ? Ns + 1 - s : s;
    return (n <= NsA) ? a.BA : a.BB;
  };
  // z forward of step 1 from the initial condition
  for (long long tile = blockIdx.x; tile < nzt; tile += gridDim.x)
    zz_tile<N>(a, tile, false, BWD ? a.qd0 : a.hist, nullptr, nullptr, nullptr, 0.0, 0.0, Bof(1));
  if (!p_barrier(a, &s_flag, nbar)) return;
#pragma unroll 1
  for (int s = 1; s <= Ns; s++) {
    for (long long tile = blockIdx.x; tile < nxt; tile += gridDim.x)
      strided_body<float, N, 0, typename R::XPL, R::C>(a.spec, ncols, R::NZH, (long long)N * R::NZH, R::NZH, a.twy,
                                                       a.dx, a.dy, a.dz, R::NZH, tile);
    if (!p_barrier(a, &s_flag, nbar)) return;
    for (long long tile = blockIdx.x; tile < nxt; tile += gridDim.x)
      strided_body<float, N, 2, typename R::XPL, R::C>(a.spec, ncols, ncols, 0, ncols, a.twx, a.dx, a.dy, a.dz,
                                                       R::NZH, tile);
    if (!p_barrier(a, &s_flag, nbar)) return;
    for (long long tile = blockIdx.x; tile < nxt; tile += gridDim.x)
      strided_body<float, N, 1, typename R::XPL, R::C>(a.spec, ncols, R::NZH, (long long)N * R::NZH, R::NZH, a.twy,
                                                       a.dx, a.dy, a.dz, R::NZH, tile);
    if (!p_barrier(a, &s_flag, nbar)) return;
    const float* Bn = Bof(s);
    const float* Bnext = (s < Ns) ? Bof(s + 1) : nullptr;
    float* qstore;
    const float* partner = nullptr;
    double cA = 0.0, cB = 0.0;
    if (!BWD) {
      qstore = a.hist + (long long)s * M;
    } else {
      const int pn = Ns - s;
      qstore = (s == Ns) ? a.qd_out : nullptr;
      partner = a.hist + (long long)pn * M;
      if (NsA > 0 && pn <= NsA) cA = (pn == 0 || pn == NsA) ? 0.5 : 1.0;
      if (NsA < Ns && pn >= NsA) cB = (pn == NsA || pn == Ns) ? 0.5 : 1.0;
    }
    for (long long tile = blockIdx.x; tile < nzt; tile += gridDim.x)
      zz_tile<N>(a, tile, true, nullptr, Bn, qstore, partner, cA, cB, Bnext);
    if (s < Ns && !p_barrier(a, &s_flag, nbar)) return;
  }
}

}  // namespace pft
