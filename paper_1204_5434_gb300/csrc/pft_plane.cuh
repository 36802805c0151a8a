// pft_plane.cuh -- the y and z parts of a contour step as one batched kernel per step
// (one CTA per (member, x-plane)), with the plane's spectrum moved between HBM and the
// column transforms in registers:
//   columns: load the column's half-spectrum values straight into the registers of the
//            y inverse transform (a warp reads 32 consecutive kz of one ky: 256 B),
//   rows:    z inverse of step s (C2R), x B_s, store q_s, x B_{s+1}, z forward of step
//            s+1 (R2C) on the rows of the plane in shared memory,
//   columns: y forward transform, results stored from registers to HBM.
// Shared memory holds kz < nz/2 of every ky under an XOR swizzle (conflict-free for the
// column accesses, a warp on 32 consecutive kz of one ky, and for the two access
// patterns of the 8-thread row transforms, two rows per half-warp); the Nyquist column
// kz = nz/2 sits in a separate array.  Real fields (SCFT), FP32 propagators.
#pragma once
#include "pft_batch.cuh"

namespace pft {

// Position p (0 <= p < N2) of row y in shared memory: the low four bits of p are XORed
// with 2 (p / 16) and, on odd rows, with 9.  A bijection within each aligned block of 16.
__device__ __forceinline__ int pswz(int y, int p) {
  return (p & ~15) | ((p & 15) ^ (((p >> 4) << 1) & 15) ^ ((y & 1) ? 9 : 0));
}

template <int NY, int NZ, int YC_ = (NZ / 2 < 64 ? NZ / 2 : 64), class YPL_ = Plan<NY>> struct PlaneCfg {
  static constexpr int N2 = NZ / 2;
  static constexpr int NZH = N2 + 1;
  using YPL = YPL_;
  using ZPL = Plan<N2>;
  static constexpr int YT = YPL::TPC, YE = YPL::E;
  static constexpr int ZT = ZPL::TPC, ZE = ZPL::E;
  static constexpr int YC = YC_;                    // regular columns per round
  static constexpr int CR = N2 / YC;                // column rounds
  static constexpr int THREADS = YC * YT + 32;      // plus one warp for the Nyquist column
  static constexpr int ROWS = THREADS / ZT;         // rows per round
  static constexpr size_t SMEM = ((size_t)NY * N2 + 2 * NY) * sizeof(float2);
  static_assert(N2 % YC == 0 && YC % 32 == 0, "column rounds");
  static_assert(YT <= 32 && THREADS % ZT == 0 && ROWS % 2 == 0, "thread split");
  static_assert(N2 >= 16, "swizzle blocks of 16");
  // rows are warp-local and the repeated rows past the last one fill whole warps, which
  // skip the row phase
  static_assert(32 % ZT == 0 && ((NY % ROWS) * ZT) % 32 == 0, "warp-local rows");
};

// One column of the plane for the Stockham exchanges: a regular column (kz < N2) under
// the swizzle, or a linear array (the Nyquist column, or scratch for idle threads).
struct PColS {
  float2* w;    // plane base, or the linear array
  int kz;       // column, or -1 for a linear array
  int n2;
  __device__ __forceinline__ int at(int pos) const { return kz < 0 ? pos : pos * n2 + pswz(pos, kz); }
  __device__ __forceinline__ void put(int pos, float2 z) { w[at(pos)] = z; }
  __device__ __forceinline__ float2 get(int pos) const { return w[at(pos)]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// A row and the threads that transform it lie in one warp (ZT threads per row, 32/ZT rows
// per warp), so the row exchanges need only the warp to synchronise.
struct PRowS {
  float2* w;  // row base W + y * N2
  int y;
  __device__ __forceinline__ void put(int pos, float2 z) { w[pswz(y, pos)] = z; }
  __device__ __forceinline__ float2 get(int pos) const { return w[pswz(y, pos)]; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// Column role of this thread in a round: regular column kz (or -1 for the Nyquist
// column, -2 for an idle thread) and its position index t within the column.
template <class R> __device__ __forceinline__ void col_role(int round, int& kz, int& t) {
  const int tid = threadIdx.x;
  if (tid < R::YC * R::YT) {
    kz = round * R::YC + tid % R::YC;
    t = tid / R::YC;
  } else {
    const int e = tid - R::YC * R::YT;
    t = e % R::YT;
    kz = (round == 0 && e < R::YT) ? -1 : -2;
  }
}

// MODE 0: first step (rows from q_0 = st.in, x B, z forward, y forward to HBM).
// MODE 1: a full step (y inverse from HBM, rows: z inverse, x B, store q, then if
//         st.Bnext: x Bnext, z forward; y forward to HBM).
template <int NY, int NZ, int MODE, int YC = PlaneCfg<NY, NZ>::YC, class YPL = Plan<NY>, int MINB = 1>
__global__ void __launch_bounds__(PlaneCfg<NY, NZ, YC, YPL>::THREADS, MINB)
kb_plane_r2c(const BatchStep* __restrict__ st) {
  using R = PlaneCfg<NY, NZ, YC, YPL>;
  constexpr int N2 = R::N2, NZH = R::NZH;
  constexpr int YE = R::YE, YT = R::YT, ZE = R::ZE, ZT = R::ZT;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* W = reinterpret_cast<float2*>(smraw);
  float2* Wn = W + NY * N2;      // Nyquist column
  float2* Wd = Wn + NY;          // scratch of idle threads
  const int p = blockIdx.x;
  float2* g = reinterpret_cast<float2*>(s.spec) + (long long)p * NY * NZH;
  const float2* twy = (const float2*)s.tw[1];
  const float2* twz = (const float2*)s.tw[2];
  const float2* twh = (const float2*)s.tw[3];
  const long long rowbase = (long long)p * NY;
  const float* Bfwd = (MODE == 0) ? (const float*)s.B : (const float*)s.Bnext;

  if (MODE == 1) {
    // ---- y inverse: HBM -> registers -> transform -> shared memory
#pragma unroll 1
    for (int round = 0; round < R::CR; round++) {
      int kz, t;
      col_role<R>(round, kz, t);
      const int gk = kz >= 0 ? kz : (kz == -1 ? N2 : 0);
      float2 v[YE];
#pragma unroll
      for (int i = 0; i < YE; i++) v[i] = g[(long long)(t + YT * i) * NZH + gk];
      PColS x{kz >= 0 ? W : (kz == -1 ? Wn : Wd), kz >= 0 ? kz : -1, N2};
      fft<float, true, NY, YPL>(v, t, twy, x);
#pragma unroll
      for (int i = 0; i < YE; i++) x.put(t + YT * i, v[i]);
    }
    __syncthreads();
  }

  // ---- rows
  {
    const int t = threadIdx.x % ZT;
    const int rr = threadIdx.x / ZT;
#pragma unroll 1
    for (int r0 = 0; r0 < NY; r0 += R::ROWS) {
      if (r0 + rr >= NY) continue;  // past the last row: whole warps, idle in this round
      const int y = r0 + rr;
      PRowS x{W + y * N2, y};
      const long long off = (rowbase + y) * N2;  // float2 index of the row's first pair
      float2 v[ZE];
      float2 bc[ZE];  // B of this row (MODE 1)
      if (MODE == 0) {
        const float2* q2 = reinterpret_cast<const float2*>(s.in) + off;
#pragma unroll
        for (int i = 0; i < ZE; i++) v[i] = q2[t + ZT * i];
      } else {
        // the factors of this row first: their latency overlaps the inverse transform
        const float2* b2 = reinterpret_cast<const float2*>(s.B) + off;
#pragma unroll
        for (int i = 0; i < ZE; i++) bc[i] = b2[t + ZT * i];
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int k = t + ZT * i;
          const float2 xk = x.get(k);
          const float2 xc = cconj(k == 0 ? Wn[y] : x.get(N2 - k));
          const float2 d = rot90<true>(cmulc(csub(xk, xc), twz[k]));
          v[i] = cadd(cadd(xk, xc), d);
        }
        __syncwarp();  // every read of the row precedes the transform's writes
        fft<float, true, N2, typename R::ZPL>(v, t, twh, x);
        float2* q2 = reinterpret_cast<float2*>(s.out) + off;
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          v[i].x *= bc[i].x;
          v[i].y *= bc[i].y;
          q2[t + ZT * i] = v[i];
        }
      }
      if (Bfwd) {
        if (MODE == 1 && Bfwd == (const float*)s.B) {
          // the next split step lies in the same block: same factor, already loaded
#pragma unroll
          for (int i = 0; i < ZE; i++) {
            v[i].x *= bc[i].x;
            v[i].y *= bc[i].y;
          }
        } else {
          const float2* b2 = reinterpret_cast<const float2*>(Bfwd) + off;
#pragma unroll
          for (int i = 0; i < ZE; i++) {
            const float2 b = b2[t + ZT * i];
            v[i].x *= b.x;
            v[i].y *= b.y;
          }
        }
        __syncwarp();  // the inverse's reads of this row are complete
        fft<float, false, N2, typename R::ZPL>(v, t, twh, x);
#pragma unroll
        for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
        __syncwarp();
        const float2 nyq = make_float2(v[0].x - v[0].y, 0.f);
        const float h = 0.5f;
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int k = t + ZT * i;
          const float2 zc = cconj(x.get(k == 0 ? 0 : N2 - k));
          const float2 ev = cscale(cadd(v[i], zc), h);
          const float2 od = cscale(rot90<false>(csub(v[i], zc)), h);
          v[i] = cadd(ev, cmul(twz[k], od));
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
        if (t == 0) Wn[y] = nyq;
      }
      __syncwarp();  // the row's shared-memory traffic is done before the warp moves on
    }
  }
  __syncthreads();  // the columns read every row
  if (!Bfwd) return;  // last step: q_Ns stored, nothing to transform forward

  // ---- y forward: shared memory -> transform -> HBM
#pragma unroll 1
  for (int round = 0; round < R::CR; round++) {
    int kz, t;
    col_role<R>(round, kz, t);
    PColS x{kz >= 0 ? W : (kz == -1 ? Wn : Wd), kz >= 0 ? kz : -1, N2};
    float2 v[YE];
#pragma unroll
    for (int i = 0; i < YE; i++) v[i] = x.get(t + YT * i);
    __syncthreads();
    fft<float, false, NY, YPL>(v, t, twy, x);
    if (kz != -2) {
      const int gk = kz >= 0 ? kz : N2;
#pragma unroll
      for (int i = 0; i < YE; i++) g[(long long)(t + YT * i) * NZH + gk] = v[i];
    }
  }
}

}  // namespace pft
