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
// patterns of the 8-thread row transforms, two rows per half-warp).
// The kz = 0 and kz = nz/2 columns of a real plane are real in y, so the two ride in one
// complex column, X0 + i XN: its y inverse gives x0 + i xN (the row's DC and Nyquist
// inputs, both real), the rows store DC + i Nyquist in slot kz = 0, and the y forward of
// that column is split by Hermitian symmetry, X0[k] = (Z[k] + conj Z[-k]) / 2 and
// XN[k] = -i (Z[k] - conj Z[-k]) / 2.  Every thread owns a regular column: 16 warps at
// 128^3, 8 at 64^3.  B_s of the plane is copied to shared memory asynchronously while the
// y inverse runs; the twiddle tables are copied to shared memory at the start.  Real
// fields (SCFT), FP32 propagators.
#pragma once
#include "pft_batch.cuh"

namespace pft {

// Position p (0 <= p < N2) of row y in shared memory: the low four bits of p are XORed
// with 2 (p / 16) and, on odd rows, with 9.  A bijection within each aligned block of 16.
__device__ __forceinline__ int pswz(int y, int p) {
  return (p & ~15) | ((p & 15) ^ (((p >> 4) << 1) & 15) ^ ((y & 1) ? 9 : 0));
}

// The two radices of a two-stage plan.
template <class RR> struct Radix2;
template <int A, int B> struct Radix2<Radices<A, B>> { static constexpr int r1 = A, r2 = B; };

template <int NY, int NZ, int YC_ = (NZ / 2 < 64 ? NZ / 2 : 64), class YPL_ = Plan<NY>> struct PlaneCfg {
  static constexpr int N2 = NZ / 2;
  static constexpr int NZH = N2 + 1;
  using YPL = YPL_;
  using ZPL = Plan<N2>;
  static constexpr int YT = YPL::TPC, YE = YPL::E;
  static constexpr int ZT = ZPL::TPC, ZE = ZPL::E;
  static constexpr int ZR1 = Radix2<typename ZPL::R>::r1, ZR2 = Radix2<typename ZPL::R>::r2;  // row radices
  static constexpr int YC = YC_;                    // regular columns per round
  static constexpr int CR = N2 / YC;                // column rounds
  static constexpr int THREADS = YC * YT;
  static constexpr int ROWS = THREADS / ZT;         // rows per round
  // the plane (kz < N2), the packed column's forward transform, B_s of the plane (fetched
  // while the y inverse runs) and the y, z, z/2 twiddles
  static constexpr size_t SMEM = ((size_t)NY * N2 + NY) * sizeof(float2) + (size_t)NY * NZ * sizeof(float) +
                                 (size_t)(NY + NZ + N2) * sizeof(float2);
  // B rows in 16-byte chunks: chunk c of row y sits at c ^ bsw(y), so that the warp's rows
  // (32 / ZT of them, ZT / 2 chunks each per access) spread over the 8 chunk slots of a
  // 128-byte bank line
  static constexpr int BROWS = 16 / ZT;
  __device__ static __forceinline__ int bsw(int y) { return (y % BROWS) * (ZT / 2); }
  static_assert(N2 % YC == 0 && YC % 32 == 0, "column rounds");
  static_assert(YT <= 32 && THREADS % ZT == 0 && ROWS % 2 == 0, "thread split");
  static_assert(N2 >= 16, "swizzle blocks of 16");
  // rows are warp-local and the repeated rows past the last one fill whole warps, which
  // skip the row phase
  static_assert(32 % ZT == 0 && ((NY % ROWS) * ZT) % 32 == 0, "warp-local rows");
  static_assert(ZT <= 16 && 16 % ZT == 0 && NZ / 4 >= 8, "B chunk swizzle");
};

// One column of the plane (kz < N2, under the swizzle) for the Stockham exchanges.
struct PColS {
  float2* w;  // plane base
  int kz;
  int n2;
  __device__ __forceinline__ int at(int pos) const { return pos * n2 + pswz(pos, kz); }
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

// Row transforms: two-stage plans (radix R1 then R2, N = R1 R2) whose second-stage
// twiddles w^(r k) depend only on the thread's position t in the row; they are loaded
// once per kernel into registers (NB2 (R2 - 1) of them) instead of once per transform.
template <class PL> struct TwoStage;
template <int N_, int E_, int R1_, int R2_> struct TwoStage<PlanX<N_, E_, R1_, R2_>> {
  static constexpr int N = N_, E = E_, R1 = R1_, R2 = R2_, TPC = N_ / E_;
  static constexpr int NB1 = E / R1, NB2 = E / R2;
  static constexpr int NW = NB2 * (R2 - 1);
  static_assert(R1 * R2 == N && E % R1 == 0 && E % R2 == 0, "two-stage plan");
  // wr[b (R2 - 1) + r - 1] = tw[r k], k = (t + b TPC) mod R1
  __device__ static __forceinline__ void load(float2 (&wr)[NW], int t, const float2* __restrict__ tw) {
#pragma unroll
    for (int b = 0; b < NB2; b++) {
      const int k = (t + b * TPC) % R1;
#pragma unroll
      for (int r = 1; r < R2; r++) wr[b * (R2 - 1) + r - 1] = tw[r * k];
    }
  }
  // the Stockham transform of fft() for this plan, twiddles from wr
  template <bool INV, class X>
  __device__ static __forceinline__ void run(float2 (&v)[E], int t, const float2 (&wr)[NW], X& xch) {
#pragma unroll
    for (int b = 0; b < NB1; b++) {
      float2 u[R1];
#pragma unroll
      for (int r = 0; r < R1; r++) u[r] = v[b + r * NB1];
      Dft<R1, INV, float2>::run(u);
      const int base = (t + b * TPC) * R1;
#pragma unroll
      for (int r = 0; r < R1; r++) xch.put(base + r, u[r]);
    }
    xch.sync();
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = xch.get(t + TPC * i);
    xch.sync();
#pragma unroll
    for (int b = 0; b < NB2; b++) {
      float2 u[R2];
#pragma unroll
      for (int r = 0; r < R2; r++) u[r] = v[b + r * NB2];
#pragma unroll
      for (int r = 1; r < R2; r++) {
        const float2 w = wr[b * (R2 - 1) + r - 1];
        u[r] = INV ? cmulc(u[r], w) : cmul(u[r], w);
      }
      Dft<R2, INV, float2>::run(u);
#pragma unroll
      for (int r = 0; r < R2; r++) v[b + r * NB2] = u[r];
    }
  }
};
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
  float2* Wd = W + NY * N2;                       // the packed column's forward transform
  float* Bs = reinterpret_cast<float*>(Wd + NY);  // B_s of this plane (MODE 1)
  float2* tws = Wd + NY + NY * NZ / 2;            // twiddles y, z, z/2
  const int p = blockIdx.x;
  float2* g = reinterpret_cast<float2*>(s.spec) + (long long)p * NY * NZH;
  const long long rowbase = (long long)p * NY;
  const float* Bfwd = (MODE == 0) ? (const float*)s.B : (const float*)s.Bnext;
  const int ct = threadIdx.x / YC;  // position index within a column
  const int cc = threadIdx.x % YC;  // column within a round
  if (MODE == 1) {
    // B_s of the plane into shared memory by asynchronous 16-byte copies, waited for
    // after the y inverse
    constexpr int CPR = NZ / 4;  // chunks per row
    const float* Bg = (const float*)s.B + rowbase * NZ;
    const unsigned sb = (unsigned)__cvta_generic_to_shared(Bs);
#pragma unroll
    for (int c = threadIdx.x; c < NY * CPR; c += R::THREADS) {
      const int y = c / CPR;
      const unsigned dst = sb + (unsigned)((y * CPR + ((c % CPR) ^ R::bsw(y))) * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(Bg + (long long)c * 4) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int i = threadIdx.x; i < NY + NZ + N2; i += R::THREADS) {
    const float2* src = i < NY ? (const float2*)s.tw[1] + i
                               : (i < NY + NZ ? (const float2*)s.tw[2] + (i - NY) : (const float2*)s.tw[3] + (i - NY - NZ));
    tws[i] = *src;
  }
  const float2* twy = tws;
  const float2* twz = tws + NY;
  const float2* twh = tws + NY + NZ;
  __syncthreads();

  if (MODE == 1) {
    // ---- y inverse.  Column kz = 0 carries X0 + i XN (X0, XN the kz = 0 and kz = N2
    // columns, each Hermitian in ky): its inverse is x0 + i xN with x0, xN real.
#pragma unroll 1
    for (int round = 0; round < R::CR; round++) {
      const int kz = round * YC + cc;
      float2 v[YE];
#pragma unroll
      for (int i = 0; i < YE; i++) v[i] = g[(long long)(ct + YT * i) * NZH + kz];
      if (kz == 0) {
#pragma unroll
        for (int i = 0; i < YE; i++) {
          const float2 xn = g[(long long)(ct + YT * i) * NZH + N2];
          v[i] = make_float2(v[i].x - xn.y, v[i].y + xn.x);
        }
      }
      PColS x{W, kz, N2};
      fft<float, true, NY, YPL>(v, ct, twy, x);
#pragma unroll
      for (int i = 0; i < YE; i++) x.put(ct + YT * i, v[i]);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }

  // ---- rows
  {
    const int t = threadIdx.x % ZT;
    const int rr = threadIdx.x / ZT;
    using RT = TwoStage<PlanX<N2, ZE, R::ZR1, R::ZR2>>;
    // this thread's twiddles of the rows: the real-transform split w_nz^k, k = t + ZT i,
    // and the second transform stage
    float2 tz[ZE], wr[RT::NW];
#pragma unroll
    for (int i = 0; i < ZE; i++) tz[i] = twz[t + ZT * i];
    RT::load(wr, t, twh);
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
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int k = t + ZT * i;
          float2 xk = x.get(k);
          float2 xc;
          if (k == 0) {  // packed x0 + i xN of this row: both real
            xc = make_float2(xk.y, 0.f);
            xk.y = 0.f;
          } else {
            xc = cconj(x.get(N2 - k));
          }
          const float2 d = rot90<true>(cmulc(csub(xk, xc), tz[i]));
          v[i] = cadd(cadd(xk, xc), d);
        }
        __syncwarp();  // every read of the row precedes the transform's writes
        RT::template run<true>(v, t, wr, x);
        float2* q2 = reinterpret_cast<float2*>(s.out) + off;
        const float2* b2s = reinterpret_cast<const float2*>(Bs) + y * N2;
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int m = t + ZT * i;  // float2 m of the row: chunk m / 2, half m % 2
          bc[i] = b2s[(((m >> 1) ^ R::bsw(y)) << 1) | (m & 1)];
        }
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
        RT::template run<false>(v, t, wr, x);
#pragma unroll
        for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
        __syncwarp();
        const float h = 0.5f;
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int k = t + ZT * i;
          const float2 zc = cconj(x.get(k == 0 ? 0 : N2 - k));
          const float2 ev = cscale(cadd(v[i], zc), h);
          const float2 od = cscale(rot90<false>(csub(v[i], zc)), h);
          float2 X = cadd(ev, cmul(tz[i], od));
          if (k == 0) X.y = v[i].x - v[i].y;  // DC (real) + i Nyquist (real)
          v[i] = X;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
      }
      __syncwarp();  // the row's shared-memory traffic is done before the warp moves on
    }
  }
  __syncthreads();  // the columns read every row
  if (!Bfwd) return;  // last step: q_Ns stored, nothing to transform forward

  // ---- y forward; the packed column's transform Z = X0 + i XN is split after a barrier:
  // X0[k] = (Z[k] + conj Z[-k]) / 2, XN[k] = -i (Z[k] - conj Z[-k]) / 2
#pragma unroll 1
  for (int round = 0; round < R::CR; round++) {
    const int kz = round * YC + cc;
    PColS x{W, kz, N2};
    float2 v[YE];
#pragma unroll
    for (int i = 0; i < YE; i++) v[i] = x.get(ct + YT * i);
    __syncthreads();
    fft<float, false, NY, YPL>(v, ct, twy, x);
    if (kz == 0) {
#pragma unroll
      for (int i = 0; i < YE; i++) Wd[ct + YT * i] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < YE; i++) g[(long long)(ct + YT * i) * NZH + kz] = v[i];
    }
  }
  __syncthreads();
  // the split, one ky per thread
  for (int k = threadIdx.x; k < NY; k += R::THREADS) {
    const float2 z = Wd[k];
    const float2 zm = cconj(Wd[(NY - k) & (NY - 1)]);
    g[(long long)k * NZH] = cscale(cadd(z, zm), 0.5f);
    g[(long long)k * NZH + N2] = cscale(rot90<false>(csub(z, zm)), 0.5f);
  }
}


}  // namespace pft
