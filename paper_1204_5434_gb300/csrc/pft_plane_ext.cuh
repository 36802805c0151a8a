// pft_plane_ext.cuh -- further kernels built on the plane kernel's layout (the y and z
// parts of a step in one CTA per x-plane): the fused step of the reverse-mode adjoint
// (real fields) and the plane kernel for complex Langevin fields.
#pragma once
#include "pft_plane.cuh"
#include "pft_narrow.cuh"

namespace pft {

// ------------------------------------------------ reverse-mode adjoint step (real)
// One step k of an adjoint chain (lambda of the q march or mu of the q-dagger march) on
// the plane kernel: the spectrum holds the z and y forward transforms of B_k lambda_k
// with the x pass (D) applied; the kernel runs y^-1 and z^-1 to z = F^-1 D F (B_k
// lambda_k), then per point
//   dw     += -(ds/2) [lambda_k q_k + B_k q_{k-1} z]                 (FP64)
//   lambda_{k-1} = B_k z + (ds/Q) (cA G_A + cB G_B) src               (FP64, rounded)
// and, unless k = 1, the z and y forward transforms of B_{k-1} lambda_{k-1} for the
// next step.  The same arithmetic as the pencil passes followed by k_adjoint_update.
struct AdjPlaneStep {
  const float* lam;       // lambda_k
  float* lam_next;        // lambda_{k-1}
  const float* B;         // B_k
  const float* Bnext;     // B_{k-1}, or null at k = 1
  const float* qk;        // q_k (or qd_k)
  const float* qk1;       // q_{k-1}
  const float* src;       // partner slice of the source at k-1
  double cA, cB;          // quadrature weights of that source
  double* dw;             // gradient accumulator of the block of step k
  void* spec;
  const void* tw[4];
};

template <int NY, int NZ>
__global__ void __launch_bounds__(PlaneCfg<NY, NZ>::THREADS, 1)
kb_plane_adj(const AdjPlaneStep* __restrict__ st, const double* __restrict__ GA, const double* __restrict__ GB,
             const double* __restrict__ Qp, double ds) {
  using R = PlaneCfg<NY, NZ>;
  constexpr int N2 = R::N2, NZH = R::NZH;
  constexpr int YE = R::YE, YT = R::YT, ZE = R::ZE, ZT = R::ZT, YC = R::YC;
  const AdjPlaneStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* W = reinterpret_cast<float2*>(smraw);
  float2* Wd = W + NY * N2;
  float* Bs = reinterpret_cast<float*>(Wd + NY);
  float2* tws = Wd + NY + NY * NZ / 2;
  const int p = blockIdx.x;
  float2* g = reinterpret_cast<float2*>(s.spec) + (long long)p * NY * NZH;
  const long long rowbase = (long long)p * NY;
  const int ct = threadIdx.x / YC;
  const int cc = threadIdx.x % YC;
  {
    constexpr int CPR = NZ / 4;
    const float* Bg = s.B + rowbase * NZ;
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

  // ---- y inverse (packed DC / Nyquist column as in kb_plane_r2c)
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
    fft<float, true, NY, typename R::YPL>(v, ct, twy, x);
#pragma unroll
    for (int i = 0; i < YE; i++) x.put(ct + YT * i, v[i]);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();

  // ---- rows: z^-1, the adjoint update, x B_{k-1}, z
  {
    const int t = threadIdx.x % ZT;
    const int rr = threadIdx.x / ZT;
    using RT = TwoStage<PlanX<N2, ZE, R::ZR1, R::ZR2>>;
    float2 tz[ZE], wr[RT::NW];
#pragma unroll
    for (int i = 0; i < ZE; i++) tz[i] = twz[t + ZT * i];
    RT::load(wr, t, twh);
    const double h = -0.5 * ds;
    const double f = ds / Qp[0];
    const double g0 = f * s.cA, g1 = f * s.cB;
#pragma unroll 1
    for (int r0 = 0; r0 < NY; r0 += R::ROWS) {
      if (r0 + rr >= NY) continue;
      const int y = r0 + rr;
      PRowS x{W + y * N2, y};
      const long long off = (rowbase + y) * N2;  // float2 index of the row's first pair
      float2 v[ZE];
#pragma unroll
      for (int i = 0; i < ZE; i++) {
        const int k = t + ZT * i;
        float2 xk = x.get(k);
        float2 xc;
        if (k == 0) {
          xc = make_float2(xk.y, 0.f);
          xk.y = 0.f;
        } else {
          xc = cconj(x.get(N2 - k));
        }
        const float2 d = rot90<true>(cmulc(csub(xk, xc), tz[i]));
        v[i] = cadd(cadd(xk, xc), d);
      }
      __syncwarp();
      RT::template run<true>(v, t, wr, x);
      const float2* b2s = reinterpret_cast<const float2*>(Bs) + y * N2;
#pragma unroll
      for (int i = 0; i < ZE; i++) {
        const int m = t + ZT * i;
        const long long o = off + m;
        const float2 b = b2s[(((m >> 1) ^ R::bsw(y)) << 1) | (m & 1)];
        const float2 z = v[i];
        const float2 lam = reinterpret_cast<const float2*>(s.lam)[o];
        const float2 qk = reinterpret_cast<const float2*>(s.qk)[o];
        const float2 qk1 = reinterpret_cast<const float2*>(s.qk1)[o];
        const float2 sr = reinterpret_cast<const float2*>(s.src)[o];
        double2 dw = reinterpret_cast<const double2*>(s.dw)[o];
        dw.x = fma(h, widen(lam.x * qk.x) + widen(b.x * qk1.x * z.x), dw.x);
        dw.y = fma(h, widen(lam.y * qk.y) + widen(b.y * qk1.y * z.y), dw.y);
        reinterpret_cast<double2*>(s.dw)[o] = dw;
        double gx = 0.0, gy = 0.0;
        if (g0 != 0.0) {
          const double2 a = reinterpret_cast<const double2*>(GA)[o];
          gx += g0 * a.x;
          gy += g0 * a.y;
        }
        if (g1 != 0.0) {
          const double2 a = reinterpret_cast<const double2*>(GB)[o];
          gx += g1 * a.x;
          gy += g1 * a.y;
        }
        const float2 ln = make_float2(narrow_rn(fma(gx, widen(sr.x), widen(b.x * z.x))),
                                      narrow_rn(fma(gy, widen(sr.y), widen(b.y * z.y))));
        reinterpret_cast<float2*>(s.lam_next)[o] = ln;
        v[i] = ln;
      }
      if (s.Bnext) {
        if (s.Bnext == s.B) {
#pragma unroll
          for (int i = 0; i < ZE; i++) {
            const int m = t + ZT * i;
            const float2 b = b2s[(((m >> 1) ^ R::bsw(y)) << 1) | (m & 1)];
            v[i].x *= b.x;
            v[i].y *= b.y;
          }
        } else {
          const float2* b2 = reinterpret_cast<const float2*>(s.Bnext) + off;
#pragma unroll
          for (int i = 0; i < ZE; i++) {
            const float2 b = b2[t + ZT * i];
            v[i].x *= b.x;
            v[i].y *= b.y;
          }
        }
        __syncwarp();
        RT::template run<false>(v, t, wr, x);
#pragma unroll
        for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
        __syncwarp();
        const float hh = 0.5f;
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int k = t + ZT * i;
          const float2 zc = cconj(x.get(k == 0 ? 0 : N2 - k));
          const float2 ev = cscale(cadd(v[i], zc), hh);
          const float2 od = cscale(rot90<false>(csub(v[i], zc)), hh);
          float2 X = cadd(ev, cmul(tz[i], od));
          if (k == 0) X.y = v[i].x - v[i].y;
          v[i] = X;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (!s.Bnext) return;

  // ---- y forward (split of the packed column as in kb_plane_r2c)
#pragma unroll 1
  for (int round = 0; round < R::CR; round++) {
    const int kz = round * YC + cc;
    PColS x{W, kz, N2};
    float2 v[YE];
#pragma unroll
    for (int i = 0; i < YE; i++) v[i] = x.get(ct + YT * i);
    __syncthreads();
    fft<float, false, NY, typename R::YPL>(v, ct, twy, x);
    if (kz == 0) {
#pragma unroll
      for (int i = 0; i < YE; i++) Wd[ct + YT * i] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < YE; i++) g[(long long)(ct + YT * i) * NZH + kz] = v[i];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NY; k += R::THREADS) {
    const float2 z = Wd[k];
    const float2 zm = cconj(Wd[(NY - k) & (NY - 1)]);
    g[(long long)k * NZH] = cscale(cadd(z, zm), 0.5f);
    g[(long long)k * NZH + N2] = cscale(rot90<false>(csub(z, zm)), 0.5f);
  }
}

// ----------------------------------------------------------- complex fields (CL)
// The same step for complex fields: the plane holds NY x NZ complex values (all kz), the
// rows are complex transforms of length NZ (no real split), B is complex.  One CTA per
// x-plane, NZ columns on YT threads each, NY rows on ZT threads each, one round of both
// (64^3: 512 threads).  B_s of the plane is copied to shared memory by cp.async during
// the y inverse as in the real kernel.
template <int NY, int NZ> struct PlaneCfgC {
  using YPL = Plan<NY>;
  using ZPL = Plan<NZ>;
  static constexpr int YT = YPL::TPC, YE = YPL::E;
  static constexpr int ZT = ZPL::TPC, ZE = ZPL::E;
  static constexpr int ZR1 = Radix2<typename ZPL::R>::r1, ZR2 = Radix2<typename ZPL::R>::r2;
  static constexpr int THREADS = NZ * YT;
  static constexpr int ROWS = THREADS / ZT;
  // plane, B_s of the plane, y and z twiddles
  static constexpr size_t SMEM = (size_t)NY * NZ * sizeof(float2) * 2 + (size_t)(NY + NZ) * sizeof(float2);
  static constexpr int BROWS = 16 / ZT;
  __device__ static __forceinline__ int bsw(int y) { return (y % BROWS) * (ZT / 2); }
  static_assert(NZ % 32 == 0 && THREADS <= 1024 && ROWS == NY, "one round of columns and rows");
  static_assert(32 % ZT == 0 && ZT <= 16 && 16 % ZT == 0 && NZ / 2 >= 8, "warp-local rows, B chunk swizzle");
};

// MODE 0: first step (rows from q_0, x B, z forward; y forward to HBM).
// MODE 1: a full step (y inverse from HBM; rows: z inverse, x B, store q, then if
//         st.Bnext: x Bnext, z forward; y forward to HBM).
template <int NY, int NZ, int MODE>
__global__ void __launch_bounds__(PlaneCfgC<NY, NZ>::THREADS, 1) kb_plane_c2c(const BatchStep* __restrict__ st) {
  using R = PlaneCfgC<NY, NZ>;
  constexpr int YE = R::YE, YT = R::YT, ZE = R::ZE, ZT = R::ZT;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* W = reinterpret_cast<float2*>(smraw);  // [NY][NZ] under the swizzle
  float2* Bs = W + NY * NZ;                       // B_s of this plane (MODE 1)
  float2* tws = Bs + NY * NZ;                     // twiddles y, z
  const int p = blockIdx.x;
  float2* g = reinterpret_cast<float2*>(s.spec) + (long long)p * NY * NZ;
  const long long rowbase = (long long)p * NY;
  const float2* Bfwd = (const float2*)((MODE == 0) ? s.B : s.Bnext);
  const int ct = threadIdx.x / NZ;  // position index within a column
  const int kz = threadIdx.x % NZ;  // column
  if (MODE == 1) {
    constexpr int CPR = NZ / 2;  // 16-byte chunks per row
    const float2* Bg = (const float2*)s.B + rowbase * NZ;
    const unsigned sb = (unsigned)__cvta_generic_to_shared(Bs);
#pragma unroll
    for (int c = threadIdx.x; c < NY * CPR; c += R::THREADS) {
      const int y = c / CPR;
      const unsigned dst = sb + (unsigned)((y * CPR + ((c % CPR) ^ R::bsw(y))) * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(Bg + (long long)c * 2) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int i = threadIdx.x; i < NY + NZ; i += R::THREADS)
    tws[i] = i < NY ? ((const float2*)s.tw[1])[i] : ((const float2*)s.tw[2])[i - NY];
  const float2* twy = tws;
  const float2* twz = tws + NY;
  __syncthreads();

  if (MODE == 1) {
    // ---- y inverse: HBM -> registers -> transform -> shared memory
    float2 v[YE];
#pragma unroll
    for (int i = 0; i < YE; i++) v[i] = g[(long long)(ct + YT * i) * NZ + kz];
    PColS x{W, kz, NZ};
    fft<float, true, NY, typename R::YPL>(v, ct, twy, x);
#pragma unroll
    for (int i = 0; i < YE; i++) x.put(ct + YT * i, v[i]);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }

  // ---- rows (one round: every row on ZT threads of one warp)
  {
    const int t = threadIdx.x % ZT;
    const int y = threadIdx.x / ZT;
    using RT = TwoStage<PlanX<NZ, ZE, R::ZR1, R::ZR2>>;
    float2 wr[RT::NW];
    RT::load(wr, t, twz);
    PRowS x{W + y * NZ, y};
    const long long off = (rowbase + y) * NZ;
    float2 v[ZE];
    if (MODE == 0) {
      const float2* q2 = reinterpret_cast<const float2*>(s.in) + off;
#pragma unroll
      for (int i = 0; i < ZE; i++) v[i] = q2[t + ZT * i];
    } else {
#pragma unroll
      for (int i = 0; i < ZE; i++) v[i] = x.get(t + ZT * i);
      __syncwarp();  // every read of the row precedes the transform's writes
      RT::template run<true>(v, t, wr, x);
      float2* q2 = reinterpret_cast<float2*>(s.out) + off;
      const float2* b2s = Bs + y * NZ;
#pragma unroll
      for (int i = 0; i < ZE; i++) {
        const int m = t + ZT * i;  // element m of the row: chunk m / 2, half m % 2
        v[i] = cmul(v[i], b2s[(((m >> 1) ^ R::bsw(y)) << 1) | (m & 1)]);
        q2[m] = v[i];
      }
    }
    if (Bfwd) {
      if (MODE == 1 && Bfwd == (const float2*)s.B) {
        // the next split step lies in the same block: same factor, in shared memory
        const float2* b2s = Bs + y * NZ;
#pragma unroll
        for (int i = 0; i < ZE; i++) {
          const int m = t + ZT * i;
          v[i] = cmul(v[i], b2s[(((m >> 1) ^ R::bsw(y)) << 1) | (m & 1)]);
        }
      } else {
        const float2* b2 = Bfwd + off;
#pragma unroll
        for (int i = 0; i < ZE; i++) v[i] = cmul(v[i], b2[t + ZT * i]);
      }
      __syncwarp();  // the inverse's reads of this row are complete
      RT::template run<false>(v, t, wr, x);
#pragma unroll
      for (int i = 0; i < ZE; i++) x.put(t + ZT * i, v[i]);
    }
    __syncwarp();
  }
  __syncthreads();  // the columns read every row
  if (!Bfwd) return;  // last step: q_Ns stored, nothing to transform forward

  // ---- y forward: shared memory -> transform -> HBM
  {
    PColS x{W, kz, NZ};
    float2 v[YE];
#pragma unroll
    for (int i = 0; i < YE; i++) v[i] = x.get(ct + YT * i);
    __syncthreads();
    fft<float, false, NY, typename R::YPL>(v, ct, twy, x);
#pragma unroll
    for (int i = 0; i < YE; i++) g[(long long)(ct + YT * i) * NZ + kz] = v[i];
  }
}


}  // namespace pft
