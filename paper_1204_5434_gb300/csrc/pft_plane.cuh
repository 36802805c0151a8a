// pft_plane.cuh -- the y and z parts of a contour step as ONE batched kernel per step:
// one CTA per (member, x-plane) loads that plane of the spectrum into shared memory and
// does  y inverse | z inverse of step s (C2R), x B_s, store q_s, x B_{s+1}, z forward of
// step s+1 (R2C) | y forward,  then stores the plane back.  Together with the batched x
// pass (forward x, x D(k)/M, inverse x) a step of both propagators is two launches.
// Real fields (SCFT), FP32 propagators, grids whose y-z plane fits in shared memory.
#pragma once
#include "pft_batch.cuh"

namespace pft {

template <int NY, int NZ> struct PlaneCfg {
  static constexpr int N2 = NZ / 2;
  static constexpr int NZH = N2 + 1;
  using YPL = Plan<NY>;   // column (y) transforms
  using ZPL = Plan<N2>;   // row (z) transforms of the packed half length
  static constexpr int YT = YPL::TPC, YE = YPL::E;
  static constexpr int ZT = ZPL::TPC, ZE = ZPL::E;
  // enough column groups for the NZH columns in at most two rounds
  static constexpr int GROUPS = (NZH + 1) / 2;
  static constexpr int THREADS_Y = ((NZH <= 64) ? NZH : GROUPS) * YT;
  static constexpr int THREADS = ((THREADS_Y + 31) / 32) * 32;
  static constexpr int YCOLS = THREADS / YT;   // column groups per round
  static constexpr int ROWS = THREADS / ZT;    // rows per round
  static constexpr int LDP = N2 + (N2 >> 4) + 2;
  static constexpr int PLANE_E = NY * NZH;
  static constexpr int PLANE_K = (PLANE_E + THREADS - 1) / THREADS;
  static constexpr size_t SMEM = (size_t)NY * LDP * sizeof(float2);
  static_assert(THREADS % YT == 0 && THREADS % ZT == 0, "thread split");
};

struct PRow {
  float2* s;
  __device__ __forceinline__ static int idx(int pos) { return pos + (pos >> 4); }
  __device__ __forceinline__ void put(int pos, float2 z) { s[idx(pos)] = z; }
  __device__ __forceinline__ float2 get(int pos) const { return s[idx(pos)]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct PCol {
  float2* s;
  int ld;
  int off;
  __device__ __forceinline__ void put(int pos, float2 z) { s[pos * ld + off] = z; }
  __device__ __forceinline__ float2 get(int pos) const { return s[pos * ld + off]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

template <int NY, int NZ, bool INV>
__device__ __forceinline__ void plane_cols(float2* __restrict__ W, const float2* __restrict__ twy) {
  using R = PlaneCfg<NY, NZ>;
  constexpr int E = R::YE, TPC = R::YT;
  const int c = threadIdx.x % R::YCOLS;
  const int t = threadIdx.x / R::YCOLS;
#pragma unroll 1
  for (int c0 = 0; c0 < R::NZH; c0 += R::YCOLS) {
    int kz = c0 + c;
    if (kz >= R::NZH) kz = R::NZH - 1;  // idle groups repeat the last column (identical writes)
    PCol x{W, R::LDP, PRow::idx(kz)};
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = x.get(t + TPC * i);
    __syncthreads();
    fft<float, INV, NY, typename R::YPL>(v, t, twy, x);
#pragma unroll
    for (int i = 0; i < E; i++) x.put(t + TPC * i, v[i]);
    __syncthreads();
  }
}

// Rows of the plane.  zin: the rows hold a half spectrum to invert (else q comes from
// `qin`); the inverse is multiplied by B and stored to `qout`; if Bnext, the row is
// multiplied by Bnext and transformed forward back into the plane.
template <int NY, int NZ>
__device__ __forceinline__ void plane_rows(float2* __restrict__ W, long long rowbase, bool zin,
                                           const float* __restrict__ qin, const float* __restrict__ B,
                                           float* __restrict__ qout, const float* __restrict__ Bnext,
                                           const float2* __restrict__ twz, const float2* __restrict__ twh) {
  using R = PlaneCfg<NY, NZ>;
  constexpr int N2 = R::N2, E = R::ZE, TPC = R::ZT;
  const int t = threadIdx.x % TPC;
  const int rr = threadIdx.x / TPC;
#pragma unroll 1
  for (int r0 = 0; r0 < NY; r0 += R::ROWS) {
    const bool dup = (r0 + rr >= NY);  // past the last row: repeat it, no global stores
    const int y = dup ? NY - 1 : r0 + rr;
    PRow x{W + y * R::LDP};
    const long long off = (rowbase + y) * N2;  // float2 index of the row's first pair
    float2 v[E];
    if (!zin) {
      const float2* q2 = reinterpret_cast<const float2*>(qin) + off;
#pragma unroll
      for (int i = 0; i < E; i++) v[i] = q2[t + TPC * i];
    } else {
      float2 xk[E], xc[E];
#pragma unroll
      for (int i = 0; i < E; i++) {
        const int k = t + TPC * i;
        xk[i] = x.get(k);
        xc[i] = cconj(x.get(N2 - k));
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < E; i++) {
        const int k = t + TPC * i;
        const float2 d = rot90<true>(cmulc(csub(xk[i], xc[i]), twz[k]));
        v[i] = cadd(cadd(xk[i], xc[i]), d);
      }
      fft<float, true, N2, typename R::ZPL>(v, t, twh, x);
      const float2* b2 = reinterpret_cast<const float2*>(B) + off;
      float2* q2 = reinterpret_cast<float2*>(qout) + off;
#pragma unroll
      for (int i = 0; i < E; i++) {
        const int m = t + TPC * i;
        const float2 b = b2[m];
        v[i].x *= b.x;
        v[i].y *= b.y;
        if (!dup) q2[m] = v[i];
      }
    }
    if (Bnext) {
      const float2* b2 = reinterpret_cast<const float2*>(Bnext) + off;
#pragma unroll
      for (int i = 0; i < E; i++) {
        const float2 b = b2[t + TPC * i];
        v[i].x *= b.x;
        v[i].y *= b.y;
      }
      __syncthreads();  // the inverse's reads of this row are complete
      fft<float, false, N2, typename R::ZPL>(v, t, twh, x);
#pragma unroll
      for (int i = 0; i < E; i++) x.put(t + TPC * i, v[i]);
      __syncthreads();
      float2 zc[E];
#pragma unroll
      for (int i = 0; i < E; i++) {
        const int k = t + TPC * i;
        zc[i] = cconj(x.get(k == 0 ? 0 : N2 - k));
      }
      __syncthreads();
      const float h = 0.5f;
#pragma unroll
      for (int i = 0; i < E; i++) {
        const int k = t + TPC * i;
        const float2 ev = cscale(cadd(v[i], zc[i]), h);
        const float2 od = cscale(rot90<false>(csub(v[i], zc[i])), h);
        x.put(k, cadd(ev, cmul(twz[k], od)));
      }
      if (t == 0) x.put(N2, make_float2(v[0].x - v[0].y, 0.f));
    }
    __syncthreads();
  }
}

// MODE 0: first step (rows from q_0 = st.in, z forward, y forward, store plane).
// MODE 1: a full step (load plane, y inverse, z inverse / epilogue / z forward of the
//         next step when st.Bnext, y forward, store plane; last step: no forward part).
template <int NY, int NZ, int MODE>
__global__ void __launch_bounds__(PlaneCfg<NY, NZ>::THREADS)
kb_plane_r2c(const BatchStep* __restrict__ st, int nx) {
  using R = PlaneCfg<NY, NZ>;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* W = reinterpret_cast<float2*>(smraw);
  const int p = blockIdx.x;
  float2* g = reinterpret_cast<float2*>(s.spec) + (long long)p * R::PLANE_E;
  const float2* twy = (const float2*)s.tw[1];
  const float2* twz = (const float2*)s.tw[2];
  const float2* twh = (const float2*)s.tw[3];
  const long long rowbase = (long long)p * NY;
  (void)nx;
  const float* Bfwd = (MODE == 0) ? (const float*)s.B : (const float*)s.Bnext;
  if (MODE == 1) {
    float2 r[R::PLANE_K];
#pragma unroll
    for (int k = 0; k < R::PLANE_K; k++) {
      const int e = threadIdx.x + k * R::THREADS;
      if (e < R::PLANE_E) r[k] = g[e];
    }
#pragma unroll
    for (int k = 0; k < R::PLANE_K; k++) {
      const int e = threadIdx.x + k * R::THREADS;
      if (e < R::PLANE_E) {
        const int ky = e / R::NZH, kz = e - ky * R::NZH;
        W[ky * R::LDP + PRow::idx(kz)] = r[k];
      }
    }
    __syncthreads();
    plane_cols<NY, NZ, true>(W, twy);
    plane_rows<NY, NZ>(W, rowbase, true, nullptr, (const float*)s.B, (float*)s.out, Bfwd, twz, twh);
  } else {
    plane_rows<NY, NZ>(W, rowbase, false, (const float*)s.in, nullptr, nullptr, Bfwd, twz, twh);
  }
  if (!Bfwd) return;  // last step: q_Ns stored, nothing to transform forward
  plane_cols<NY, NZ, false>(W, twy);
#pragma unroll 4
  for (int e = threadIdx.x; e < R::PLANE_E; e += R::THREADS) {
    const int ky = e / R::NZH, kz = e - ky * R::NZH;
    g[e] = W[ky * R::LDP + PRow::idx(kz)];
  }
}

}  // namespace pft
