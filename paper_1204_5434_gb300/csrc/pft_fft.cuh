// pft_fft.cuh -- complex helpers and the register-distributed Stockham FFT used by
// every pass kernel of the contour step (the FFT / inverse-FFT pair of the
// pseudo-spectral operator splitting, Eq. 13).
//
// Distribution: a length-N transform is held by TPC = N/E threads, E elements each;
// thread t holds elements t + TPC*i (i = 0..E-1).  Each Stockham stage of radix R
// performs E/R butterflies per thread on registers b + r*(E/R), multiplies by the
// stage twiddles, and (between stages) exchanges through shared memory so that the
// thread again holds t + TPC*i.  The output of the last stage lands in natural order
// in the same distribution, so a forward transform, a pointwise multiply and an
// inverse transform chain with no shared-memory round trip in between.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pft {

// ----------------------------------------------------------------- complex types
template <typename T> struct cpx_t;
template <> struct cpx_t<float> { using type = float2; };
template <> struct cpx_t<double> { using type = double2; };
template <typename T> using cpx = typename cpx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T re, T im) { cpx<T> z; z.x = re; z.y = im; return z; }
template <typename Z> __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <typename Z> __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename Z> __device__ __forceinline__ Z cmul(Z a, Z b) {
  Z r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename Z> __device__ __forceinline__ Z cmulc(Z a, Z b) {
  Z r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename Z, typename S> __device__ __forceinline__ Z cscale(Z a, S s) { a.x *= s; a.y *= s; return a; }
template <typename Z> __device__ __forceinline__ Z cconj(Z a) { a.y = -a.y; return a; }
// multiply by -i (INV=false) or +i (INV=true)
template <bool INV, typename Z> __device__ __forceinline__ Z rot90(Z a) {
  Z r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// float -> double by bit manipulation on the integer pipe (exact for zero and normal
// floats; the propagator products are never subnormal, infinite or NaN in a sane solve,
// and a subnormal would only be flushed to zero): GB300 runs F2F.F64 on its 1/64-rate
// FP64 pipe, which the quadrature needs for its one DFMA per term.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return (u & 0x80000000u) ? -0.0 : 0.0;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lo = (u & 0x7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double d) { return d; }

// ------------------------------------------------------------ small DFT kernels
// Forward: y_k = sum_n a_n exp(-2 pi i n k / R); inverse: exp(+...), unnormalised.
template <int R, bool INV, typename Z> struct Dft;

template <bool INV, typename Z> struct Dft<2, INV, Z> {
  __device__ __forceinline__ static void run(Z* a) {
    Z t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  }
};

template <bool INV, typename Z> struct Dft<3, INV, Z> {
  __device__ __forceinline__ static void run(Z* a) {
    using S = decltype(a[0].x);
    const S h = S(0.5);
    const S s3 = S(0.86602540378443864676372317075294);  // sin(2 pi/3)
    Z t1 = cadd(a[1], a[2]);
    Z t2 = csub(a[1], a[2]);
    Z m = csub(a[0], cscale(t1, h));
    Z r = rot90<INV>(cscale(t2, s3));  // -i s3 t2 (forward)
    a[0] = cadd(a[0], t1);
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
  }
};

template <bool INV, typename Z> struct Dft<4, INV, Z> {
  __device__ __forceinline__ static void run(Z* a) {
    Z t0 = cadd(a[0], a[2]);
    Z t1 = csub(a[0], a[2]);
    Z t2 = cadd(a[1], a[3]);
    Z t3 = rot90<INV>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

template <bool INV, typename Z> struct Dft<8, INV, Z> {
  __device__ __forceinline__ static void run(Z* a) {
    using S = decltype(a[0].x);
    const S r2 = S(0.70710678118654752440084436210485);
    Z e[4] = {a[0], a[2], a[4], a[6]};
    Z o[4] = {a[1], a[3], a[5], a[7]};
    Dft<4, INV, Z>::run(e);
    Dft<4, INV, Z>::run(o);
    // twiddles w8^k, k = 0..3 (w8 = exp(-i pi/4) forward)
    Z o1, o2, o3;
    if (INV) {
      o1.x = r2 * (o[1].x - o[1].y); o1.y = r2 * (o[1].x + o[1].y);
      o3.x = -r2 * (o[3].x + o[3].y); o3.y = r2 * (o[3].x - o[3].y);
    } else {
      o1.x = r2 * (o[1].x + o[1].y); o1.y = r2 * (o[1].y - o[1].x);
      o3.x = r2 * (o[3].y - o[3].x); o3.y = -r2 * (o[3].x + o[3].y);
    }
    o2 = rot90<INV>(o[2]);
    a[0] = cadd(e[0], o[0]); a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], o1);   a[5] = csub(e[1], o1);
    a[2] = cadd(e[2], o2);   a[6] = csub(e[2], o2);
    a[3] = cadd(e[3], o3);   a[7] = csub(e[3], o3);
  }
};

// 16-point DFT as 4 x 4: DFT-4 over n1 for each n2 (n = 4 n1 + n2), twiddle by
// w16^(n2 k1), DFT-4 over n2 for each k1 (k = k1 + 4 k2).
template <bool INV, typename Z> struct Dft<16, INV, Z> {
  __device__ __forceinline__ static void run(Z* a) {
    using S = decltype(a[0].x);
    const S c1 = S(0.92387953251128675613), s1 = S(0.38268343236508977173);  // cos, sin(pi/8)
    const S r2 = S(0.70710678118654752440);
    Z b[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) {
      Z t[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
      Dft<4, INV, Z>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; k1++) b[n2][k1] = t[k1];
    }
    // twiddles w16^m, m = n2*k1 (forward: exp(-i pi m/8); inverse: conjugate)
    const S sg = INV ? S(1) : S(-1);
    auto tw = [&](Z z, S cr, S si) {  // z * (cr + i sg si)
      Z r;
      r.x = z.x * cr - z.y * sg * si;
      r.y = z.x * sg * si + z.y * cr;
      return r;
    };
    b[1][1] = tw(b[1][1], c1, s1);
    b[1][2] = tw(b[1][2], r2, r2);
    b[1][3] = tw(b[1][3], s1, c1);
    b[2][1] = tw(b[2][1], r2, r2);
    b[2][2] = rot90<INV>(b[2][2]);
    b[2][3] = tw(b[2][3], -r2, r2);
    b[3][1] = tw(b[3][1], s1, c1);
    b[3][2] = tw(b[3][2], -r2, r2);
    b[3][3] = tw(b[3][3], -c1, -s1);
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
      Z t[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
      Dft<4, INV, Z>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; k2++) a[k1 + 4 * k2] = t[k2];
    }
  }
};

// ------------------------------------------------------------------- FFT plans
// Plan<N>: radices (applied first to last), elements per thread E (a multiple of
// every radix), threads per column TPC = N/E.
template <int... Rs> struct Radices {};
// A plan: length N, E elements per thread, radices applied first to last.
template <int N_, int E_, int... Rs> struct PlanX {
  static constexpr int N = N_;
  static constexpr int E = E_;
  static constexpr int TPC = N_ / E_;
  using R = Radices<Rs...>;
};
template <int N> struct Plan;
#define PFT_PLAN(N_, E_, ...) \
  template <> struct Plan<N_> : PlanX<N_, E_, __VA_ARGS__> {};
PFT_PLAN(2, 2, 2)
PFT_PLAN(3, 3, 3)
PFT_PLAN(4, 4, 4)
PFT_PLAN(6, 6, 3, 2)
PFT_PLAN(8, 8, 8)
PFT_PLAN(12, 12, 3, 4)
PFT_PLAN(16, 4, 4, 4)
PFT_PLAN(24, 12, 3, 4, 2)
PFT_PLAN(32, 8, 8, 4)
PFT_PLAN(48, 12, 3, 4, 4)
PFT_PLAN(64, 8, 8, 8)
PFT_PLAN(96, 12, 3, 4, 4, 2)
PFT_PLAN(128, 16, 16, 8)
PFT_PLAN(192, 12, 3, 4, 4, 4)
PFT_PLAN(256, 16, 16, 16)
#undef PFT_PLAN

// ------------------------------------------------------------ Stockham stages
// Exchange object interface:  put(pos, z) stores element `pos` of this thread's
// column, get(pos) loads it, sync() is a CTA-wide barrier.
template <typename T, bool INV, int N, int E, int NS, class X, int R, int... REST>
__device__ __forceinline__ void fft_stages(cpx<T> (&v)[E], int t, const cpx<T>* __restrict__ tw, X& xch) {
  constexpr int TPC = N / E;
  constexpr int NB = E / R;
  static_assert(E % R == 0, "radix must divide elements per thread");
#pragma unroll
  for (int b = 0; b < NB; b++) {
    cpx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; r++) u[r] = v[b + r * NB];
    const int j = t + b * TPC;
    const int k = (NS == 1) ? 0 : (j % NS);
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; r++) {
        cpx<T> w = tw[r * k * (N / (NS * R))];
        u[r] = INV ? cmulc(u[r], w) : cmul(u[r], w);
      }
    }
    Dft<R, INV, cpx<T>>::run(u);
    if constexpr (sizeof...(REST) == 0) {
#pragma unroll
      for (int r = 0; r < R; r++) v[b + r * NB] = u[r];
    } else {
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) xch.put(base + r * NS, u[r]);
    }
  }
  if constexpr (sizeof...(REST) > 0) {
    xch.sync();
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = xch.get(t + TPC * i);
    xch.sync();
    fft_stages<T, INV, N, E, NS * R, X, REST...>(v, t, tw, xch);
  }
}

template <typename T, bool INV, int N, int E, class X, int... Rs>
__device__ __forceinline__ void fft_run(cpx<T> (&v)[E], int t, const cpx<T>* __restrict__ tw, X& xch,
                                        Radices<Rs...>) {
  fft_stages<T, INV, N, E, 1, X, Rs...>(v, t, tw, xch);
}

// In-register transform of length N with plan PL.  tw: exp(-2 pi i m / N).
template <typename T, bool INV, int N, class PL = Plan<N>, class X>
__device__ __forceinline__ void fft(cpx<T> (&v)[PL::E], int t, const cpx<T>* __restrict__ tw, X& xch) {
  static_assert(PL::N == N, "plan length");
  fft_run<T, INV, N, PL::E, X>(v, t, tw, xch, typename PL::R{});
}

// Does the plan need exchanges (more than one stage)?
template <int... Rs> __host__ __device__ constexpr int count_stages(Radices<Rs...>) { return sizeof...(Rs); }
template <class PL> __host__ __device__ constexpr int n_stages() { return count_stages(typename PL::R{}); }

}  // namespace pft
