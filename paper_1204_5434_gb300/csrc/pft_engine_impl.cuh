// pft_engine_impl.cuh -- one system's solve in working precision T (float: the
// FP32-mixed path; double: the FP64 path).  Contour steps run through the pass
// kernels of pft_passes.cuh; everything that accumulates (quadrature, reductions,
// Hamiltonian, field update, Boltzmann exponentials) runs in double.
#pragma once
#include <math.h>

#include <string>
#include <vector>

#include "pft_engine.h"
#include "pft_passes.cuh"
#include "pft_narrow.cuh"
#include "pft_dd.cuh"

namespace pft {

constexpr int PW_THREADS = 256;  // pointwise / reduction block size

// ------------------------------------------------------------------ reductions
// Block sum of K per-thread values into out[0..K) (ADD: out[j] += sum).
template <int K, bool ADD = false>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], double* __restrict__ out) {
  __shared__ double red[K][PW_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; j++) {
    double s = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[j][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < PW_THREADS / 32; w++) s += red[threadIdx.x][w];
    if (ADD) {
      out[threadIdx.x] += s;
    } else {
      out[threadIdx.x] = s;
    }
  }
}

// Deterministic second stage: scal[off + j] = sum over blocks of partials[b*K + j].
template <int K>
__global__ void __launch_bounds__(PW_THREADS) k_reduce_final(const double* __restrict__ partials, int nblk,
                                                             double* __restrict__ dst) {
  double v[K];
#pragma unroll
  for (int j = 0; j < K; j++) v[j] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += PW_THREADS) {
#pragma unroll
    for (int j = 0; j < K; j++) v[j] += partials[(long long)b * K + j];
  }
  block_reduce_store<K>(v, dst);
}

// --------------------------------------------------------------- small helpers
__device__ __forceinline__ double2 cexp_d(double2 z) {
  double s, c;
  sincos(z.y, &s, &c);
  const double e = exp(z.x);
  return make_double2(e * c, e * s);
}
__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv_d(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

template <typename T> __device__ __forceinline__ void store_w(T* p, long long i, double v) { p[i] = (T)v; }
template <typename T> __device__ __forceinline__ void store_w(cpx<T>* p, long long i, double2 v) {
  p[i] = mk<T>((T)v.x, (T)v.y);
}

// Boltzmann factor exp(-w ds/2) in the propagators' precision: the exponent is formed in
// double from the FP64 field, the exponential evaluated in T (for T = float the result is
// stored as float anyway, and GB300's FP64 pipe is 1/64 of its FP32 rate).
template <typename T> __device__ __forceinline__ T boltz(double w, double ds) {
  return (T)exp(-w * ds * 0.5);
}
// FP32 factors: the FP64 argument narrowed by the integer-pipe round-to-nearest (the same
// float as a conversion, without GB300's 1/64-rate F2F), then expf
template <> __device__ __forceinline__ float boltz<float>(double w, double ds) {
  return expf(narrow_rn(-w * ds * 0.5));
}
template <typename T> __device__ __forceinline__ cpx<T> boltz_c(double2 w, double ds) {
  const double2 z = cexp_d(make_double2(-w.x * ds * 0.5, -w.y * ds * 0.5));
  return mk<T>((T)z.x, (T)z.y);
}
template <> __device__ __forceinline__ float2 boltz_c<float>(double2 w, double ds) {
  const float zr = (float)(-w.x * ds * 0.5), zi = (float)(-w.y * ds * 0.5);
  float s, c;
  sincosf(zi, &s, &c);
  const float e = expf(zr);
  return make_float2(e * c, e * s);
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies by
// fixed odd constants, high halves xored with the other words and the round key;
// the key advances by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const unsigned int M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const unsigned int W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const unsigned int lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const unsigned int lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// Four standard normals from one Philox block (Box-Muller on word pairs).
__device__ __forceinline__ void philox_normal4(unsigned long long seed, unsigned long long instance,
                                               unsigned long long step, int field, long long blk, double* z) {
  const uint4 ctr = make_uint4((unsigned int)blk, (unsigned int)field, (unsigned int)step, (unsigned int)instance);
  const uint2 key = make_uint2((unsigned int)(seed & 0xffffffffull), (unsigned int)(seed >> 32));
  const uint4 x = philox4x32_10(ctr, key);
  const double sc = 1.0 / 4294967296.0;
  const double u0 = ((double)x.x + 0.5) * sc, u1 = ((double)x.y + 0.5) * sc;
  const double u2 = ((double)x.z + 0.5) * sc, u3 = ((double)x.w + 0.5) * sc;
  const double r1 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
  double s1, c1, s2, c2;
  sincospi(2.0 * u1, &s1, &c1);
  sincospi(2.0 * u3, &s2, &c2);
  z[0] = r1 * c1;
  z[1] = r1 * s1;
  z[2] = r2 * c2;
  z[3] = r2 * s2;
}

static __global__ void k_philox_normals(unsigned long long seed, unsigned long long instance, unsigned long long step,
                                 int field, long long M, double* __restrict__ out) {
  const long long nblk = (M + 3) / 4;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nblk;
       b += (long long)gridDim.x * blockDim.x) {
    double z[4];
    philox_normal4(seed, instance, step, field, b, z);
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (4 * b + j < M) out[4 * b + j] = z[j];
  }
}

static __global__ void k_philox_raw(uint4 c0, uint2 key, long long count, unsigned int* __restrict__ out) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < count;
       b += (long long)gridDim.x * blockDim.x) {
    uint4 c = c0;
    c.x = c0.x + (unsigned int)b;
    const uint4 r = philox4x32_10(c, key);
    out[4 * b + 0] = r.x;
    out[4 * b + 1] = r.y;
    out[4 * b + 2] = r.z;
    out[4 * b + 3] = r.w;
  }
}

// ------------------------------------------------------------ pointwise kernels
template <typename W> __device__ __forceinline__ W one_val();
template <> __device__ __forceinline__ float one_val<float>() { return 1.f; }
template <> __device__ __forceinline__ double one_val<double>() { return 1.0; }
template <> __device__ __forceinline__ float2 one_val<float2>() { return make_float2(1.f, 0.f); }
template <> __device__ __forceinline__ double2 one_val<double2>() { return make_double2(1.0, 0.0); }

// The Richardson combination of Eq. 13, q = (4 A(ds/2)A(ds/2) q - A(ds) q) / 3, over n
// working-precision values (the same expression as the combining z-inverse epilogue).
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_rqm4_combine(const T* __restrict__ half2, const T* __restrict__ full,
                                                              T* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (T(4) * half2[i] - full[i]) / T(3);
}

// FP64 values split into double-float pairs (the Boltzmann factors of the double-float
// march, once per solve; n doubles, real and imaginary parts alike).
static __global__ void k_split_dd(const double* __restrict__ a, dd* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = dd_from_double(a[i]);
}

template <typename W> __global__ void k_fill_one(W* __restrict__ dst, long long M) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    dst[i] = one_val<W>();
}

// Boltzmann factors (Eq. 13) of real SCFT fields and the Eq. 3 field term.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_prepare_real(const double* __restrict__ wp, const double* __restrict__ wm,
                                                             T* __restrict__ BA, T* __restrict__ BB, double ds, double chiN,
                                                             long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double p = wp[i], m = wm[i];
    BA[i] = boltz<T>(p - m, ds);
    BB[i] = boltz<T>(p + m, ds);
    acc[0] += m * m * ichiN - p;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// Complex Langevin fields: wA = i w+ - w-, wB = i w+ + w-.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_prepare_cplx(const double2* __restrict__ wp, const double2* __restrict__ wm,
                                                             cpx<T>* __restrict__ BA, cpx<T>* __restrict__ BB, double ds,
                                                             double chiN, long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 p = wp[i], m = wm[i];
    const double2 ip = make_double2(-p.y, p.x);
    const double2 wA = make_double2(ip.x - m.x, ip.y - m.y);
    const double2 wB = make_double2(ip.x + m.x, ip.y + m.y);
    BA[i] = boltz_c<T>(wA, ds);
    BB[i] = boltz_c<T>(wB, ds);
    acc[0] += (m.x * m.x - m.y * m.y) * ichiN + p.y;
    acc[1] += 2.0 * m.x * m.y * ichiN - p.x;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// Half-step Boltzmann factors exp(-w ds/4) of the 4th-order scheme (the two A(ds/2)
// blocks of Eq. 13), real SCFT fields and complex Langevin fields.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_half_boltz_real(const double* __restrict__ wp,
                                                                const double* __restrict__ wm, T* __restrict__ BA,
                                                                T* __restrict__ BB, double hds, long long M) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double p = wp[i], m = wm[i];
    BA[i] = boltz<T>(p - m, hds);
    BB[i] = boltz<T>(p + m, hds);
  }
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_half_boltz_cplx(const double2* __restrict__ wp,
                                                                const double2* __restrict__ wm, cpx<T>* __restrict__ BA,
                                                                cpx<T>* __restrict__ BB, double hds, long long M) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 p = wp[i], m = wm[i];
    const double2 ip = make_double2(-p.y, p.x);
    BA[i] = boltz_c<T>(make_double2(ip.x - m.x, ip.y - m.y), hds);
    BB[i] = boltz_c<T>(make_double2(ip.x + m.x, ip.y + m.y), hds);
  }
}

// Sum of q_Ns for Q (Eq. 4) and the m = 0 term of the quadrature (qd_0 = 1).
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_qsum_real(const T* __restrict__ q, double* __restrict__ accA,
                                                          double* __restrict__ accB, double cA, double cB, long long M,
                                                          double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double v = widen(q[i]);
    acc[0] += v;
    if (accA) {  // the qd_0 = 1 term of the quadrature (none when a later kernel forms it)
      accA[i] = cA * v;
      accB[i] = cB * v;
    }
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_qsum_cplx(const cpx<T>* __restrict__ q, double2* __restrict__ accA,
                                                          double2* __restrict__ accB, double cA, double cB, long long M,
                                                          double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = make_double2((double)q[i].x, (double)q[i].y);
    acc[0] += v.x;
    acc[1] += v.y;
    accA[i] = make_double2(cA * v.x, cA * v.y);
    accB[i] = make_double2(cB * v.x, cB * v.y);
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// Contour quadrature of Eq. 8 over the stored histories of both propagators:
// accA = sum_n cA_n q_n qd_{Ns-n}, accB likewise (trapezoid weights on each block).  The
// integrand is the product in the propagators' precision, the running sums are FP64.
// Two grid points per thread (real) or one (complex).
__device__ __forceinline__ void trap_w(int n, int Ns, int NsA, double* cA, double* cB) {
  *cA = 0.0;
  *cB = 0.0;
  if (NsA > 0 && n <= NsA) *cA = (n == 0 || n == NsA) ? 0.5 : 1.0;
  if (NsA < Ns && n >= NsA) *cB = (n == NsA || n == Ns) ? 0.5 : 1.0;
}

// Compensated FP32 partial sum (Knuth's TwoSum): after add(x_1) ... add(x_k), hi + lo is
// the exact sum of the x_j except for the rounding of the small correction lo itself,
// i.e. within k 2^-48 of the sum relative to it.  Flushed into an FP64 running sum every
// kQuadChunk terms, it spares the FP64 pipe (1/64 of the FP32 rate on GB300) one DFMA per
// term while the result stays that of an FP64 summation of the same FP32 products to far
// below their own rounding (2^-24).
struct F2Sum {
  float hi = 0.f, lo = 0.f;
  // the _rn intrinsics keep the compiler from contracting any of these into an FMA
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
    hi = s;
  }
  __device__ __forceinline__ void flush(double* acc) {
    *acc += widen(hi);
    *acc += widen(lo);
    hi = 0.f;
    lo = 0.f;
  }
};
constexpr int kQuadChunk = 16;

// Sum over n in [n0, n1] of w_n * q_n * qd_{Ns-n} for a pair of points, weights 1/2 at
// both ends of the block (the block's trapezoid rule), FP64 running sums.  FP32
// propagators: the products are FP32 (as before), summed in compensated FP32 over chunks
// of kQuadChunk slices that are added to the FP64 sums (the weights 1/2 and 1 are exact).
template <typename T>
__device__ __forceinline__ void quad_block(const T* __restrict__ hist, const T* __restrict__ qdh,
                                           const T* __restrict__ qd0, long long M, int Ns, int n0, int n1,
                                           long long i, double* s0, double* s1) {
  double a0 = 0.0, a1 = 0.0;
  if (n1 > n0) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll 1
      for (int c0 = n0; c0 <= n1; c0 += kQuadChunk) {
        const int c1 = min(c0 + kQuadChunk - 1, n1);
        F2Sum f0, f1;
#pragma unroll 4
        for (int n = c0; n <= c1; n++) {
          const int m = Ns - n;
          const float2 q = reinterpret_cast<const float2*>(hist + (long long)n * M)[i];
          const float2 d = reinterpret_cast<const float2*>(m == 0 ? qd0 : qdh + (long long)m * M)[i];
          const float w = (n == n0 || n == n1) ? 0.5f : 1.0f;
          f0.add(__fmul_rn(__fmul_rn(q.x, d.x), w));
          f1.add(__fmul_rn(__fmul_rn(q.y, d.y), w));
        }
        f0.flush(&a0);
        f1.flush(&a1);
      }
    } else {
#pragma unroll 4
      for (int n = n0; n <= n1; n++) {
        const int m = Ns - n;
        const cpx<T> q = reinterpret_cast<const cpx<T>*>(hist + (long long)n * M)[i];
        const cpx<T> d = reinterpret_cast<const cpx<T>*>(m == 0 ? qd0 : qdh + (long long)m * M)[i];
        const double w = (n == n0 || n == n1) ? 0.5 : 1.0;
        a0 = fma(w, widen(q.x * d.x), a0);
        a1 = fma(w, widen(q.y * d.y), a1);
      }
    }
  }
  *s0 = a0;
  *s1 = a1;
}

// FP32 real fields, four points a thread (16-byte loads of both histories): the
// trapezoid sums of one block over n in [n0, n1], compensated FP32 over chunks of
// kQuadChunk slices flushed into FP64 (as quad_block).
__device__ __forceinline__ void quad_block4(const float* __restrict__ hist, const float* __restrict__ qdh,
                                            const float* __restrict__ qd0, long long M, int Ns, int n0, int n1,
                                            long long i4, double (&a)[4]) {
#pragma unroll
  for (int k = 0; k < 4; k++) a[k] = 0.0;
  if (n1 <= n0) return;
#pragma unroll 1
  for (int c0 = n0; c0 <= n1; c0 += kQuadChunk) {
    const int c1 = min(c0 + kQuadChunk - 1, n1);
    F2Sum f[4];
#pragma unroll 4
    for (int n = c0; n <= c1; n++) {
      const int m = Ns - n;
      const float4 q = reinterpret_cast<const float4*>(hist + (long long)n * M)[i4];
      const float4 d = reinterpret_cast<const float4*>(m == 0 ? qd0 : qdh + (long long)m * M)[i4];
      const float w = (n == n0 || n == n1) ? 0.5f : 1.0f;
      f[0].add(__fmul_rn(__fmul_rn(q.x, d.x), w));
      f[1].add(__fmul_rn(__fmul_rn(q.y, d.y), w));
      f[2].add(__fmul_rn(__fmul_rn(q.z, d.z), w));
      f[3].add(__fmul_rn(__fmul_rn(q.w, d.w), w));
    }
#pragma unroll
    for (int k = 0; k < 4; k++) f[k].flush(&a[k]);
  }
}

static __global__ void __launch_bounds__(PW_THREADS) k_quadrature_real4(const float* __restrict__ hist,
                                                                 const float* __restrict__ qdh,
                                                                 const float* __restrict__ qd0, long long M, int Ns,
                                                                 int NsA, double* __restrict__ accA,
                                                                 double* __restrict__ accB) {
  const long long M4 = M / 4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M4; i += (long long)gridDim.x * blockDim.x) {
    double a[4];
    quad_block4(hist, qdh, qd0, M, Ns, 0, NsA, i, a);
    reinterpret_cast<double2*>(accA)[2 * i] = make_double2(a[0], a[1]);
    reinterpret_cast<double2*>(accA)[2 * i + 1] = make_double2(a[2], a[3]);
    quad_block4(hist, qdh, qd0, M, Ns, NsA, Ns, i, a);
    reinterpret_cast<double2*>(accB)[2 * i] = make_double2(a[0], a[1]);
    reinterpret_cast<double2*>(accB)[2 * i + 1] = make_double2(a[2], a[3]);
  }
}

// The quadrature above fused with the densities and force sums of the solve's tail:
// phi = ds acc / Q (Q from s[S_Q]), and per block the sums of phiA, phiB, (phiA + phiB -
// 1)^2 and (2 W-/chiN + phiB - phiA)^2 into partials (6 a block, as k_finalize_real).
static __global__ void __launch_bounds__(PW_THREADS) k_quadrature_final_real4(const float* __restrict__ hist,
                                                                       const float* __restrict__ qdh,
                                                                       const float* __restrict__ qd0, long long M,
                                                                       int Ns, int NsA, double* __restrict__ accA,
                                                                       double* __restrict__ accB,
                                                                       const double* __restrict__ wm,
                                                                       const double* __restrict__ s, double ds,
                                                                       double chiN, double* __restrict__ partials) {
  const double f = ds / s[S_Q];
  const double ichiN = 1.0 / chiN;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const long long M4 = M / 4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M4; i += (long long)gridDim.x * blockDim.x) {
    double a[4], b[4];
    quad_block4(hist, qdh, qd0, M, Ns, 0, NsA, i, a);
    quad_block4(hist, qdh, qd0, M, Ns, NsA, Ns, i, b);
    const double2 m01 = reinterpret_cast<const double2*>(wm)[2 * i];
    const double2 m23 = reinterpret_cast<const double2*>(wm)[2 * i + 1];
    const double m[4] = {m01.x, m01.y, m23.x, m23.y};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      a[k] *= f;
      b[k] *= f;
      const double fp = a[k] + b[k] - 1.0, fm = 2.0 * m[k] * ichiN + b[k] - a[k];
      acc[0] += a[k];
      acc[2] += b[k];
      acc[4] += fp * fp;
      acc[5] += fm * fm;
    }
    reinterpret_cast<double2*>(accA)[2 * i] = make_double2(a[0], a[1]);
    reinterpret_cast<double2*>(accA)[2 * i + 1] = make_double2(a[2], a[3]);
    reinterpret_cast<double2*>(accB)[2 * i] = make_double2(b[0], b[1]);
    reinterpret_cast<double2*>(accB)[2 * i + 1] = make_double2(b[2], b[3]);
  }
  block_reduce_store<6>(acc, partials + 6 * blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_quadrature_real(const T* __restrict__ hist, const T* __restrict__ qdh,
                                                                const T* __restrict__ qd0, long long M, int Ns, int NsA,
                                                                double* __restrict__ accA, double* __restrict__ accB) {
  const long long M2 = M / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M2; i += (long long)gridDim.x * blockDim.x) {
    double a0, a1, b0, b1;
    quad_block<T>(hist, qdh, qd0, M, Ns, 0, NsA, i, &a0, &a1);
    quad_block<T>(hist, qdh, qd0, M, Ns, NsA, Ns, i, &b0, &b1);
    reinterpret_cast<double2*>(accA)[i] = make_double2(a0, a1);
    reinterpret_cast<double2*>(accB)[i] = make_double2(b0, b1);
  }
}

template <typename T>
__device__ __forceinline__ void quad_block_c(const cpx<T>* __restrict__ hist, const cpx<T>* __restrict__ qdh,
                                             const cpx<T>* __restrict__ qd0, long long M, int Ns, int n0, int n1,
                                             long long i, double* sr, double* si) {
  double ar = 0.0, ai = 0.0;
  if (n1 > n0) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll 1
      for (int c0 = n0; c0 <= n1; c0 += kQuadChunk) {
        const int c1 = min(c0 + kQuadChunk - 1, n1);
        F2Sum fr, fi;
#pragma unroll 4
        for (int n = c0; n <= c1; n++) {
          const int m = Ns - n;
          const float2 q = hist[(long long)n * M + i];
          const float2 d = (m == 0 ? qd0 : qdh + (long long)m * M)[i];
          const float2 pq = cmul(q, d);
          const float w = (n == n0 || n == n1) ? 0.5f : 1.0f;
          fr.add(__fmul_rn(pq.x, w));
          fi.add(__fmul_rn(pq.y, w));
        }
        fr.flush(&ar);
        fi.flush(&ai);
      }
    } else {
#pragma unroll 4
      for (int n = n0; n <= n1; n++) {
        const int m = Ns - n;
        const cpx<T> q = hist[(long long)n * M + i];
        const cpx<T> d = (m == 0 ? qd0 : qdh + (long long)m * M)[i];
        const cpx<T> pq = cmul(q, d);
        const double w = (n == n0 || n == n1) ? 0.5 : 1.0;
        ar = fma(w, widen(pq.x), ar);
        ai = fma(w, widen(pq.y), ai);
      }
    }
  }
  *sr = ar;
  *si = ai;
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_quadrature_cplx(const cpx<T>* __restrict__ hist,
                                                                const cpx<T>* __restrict__ qdh,
                                                                const cpx<T>* __restrict__ qd0, long long M, int Ns,
                                                                int NsA, double2* __restrict__ accA,
                                                                double2* __restrict__ accB) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    double ar, ai, br, bi;
    quad_block_c<T>(hist, qdh, qd0, M, Ns, 0, NsA, i, &ar, &ai);
    quad_block_c<T>(hist, qdh, qd0, M, Ns, NsA, Ns, i, &br, &bi);
    accA[i] = make_double2(ar, ai);
    accB[i] = make_double2(br, bi);
  }
}

// One chunk of the contour quadrature of Eq. 8 on the checkpointed separable march: for
// the np pairs (q_{Ns-m}, qd_m) of the chunk, accA += sum cA q qd and accB += sum cB q qd
// (trapezoid weights of the pair's forward slice; 0, 1/2 or 1).  FP32 propagators: the
// products and the weighted sum in compensated FP32 (TwoSum), flushed into the FP64
// accumulators once per chunk; FP64: one FMA per term.
struct QuadPair {
  const void* q;
  const void* qd;
  double cA, cB;
};
template <typename T, int KIND>
__global__ void __launch_bounds__(PW_THREADS) k_quad_pairs(const QuadPair* __restrict__ pr, int np, long long M,
                                                           double* __restrict__ accA, double* __restrict__ accB) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    if constexpr (KIND == 0) {
      double a = accA[i], b = accB[i];
      if constexpr (sizeof(T) == 4) {
        F2Sum fa, fb;
        for (int p = 0; p < np; p++) {
          const float v = __fmul_rn(reinterpret_cast<const float*>(pr[p].q)[i], reinterpret_cast<const float*>(pr[p].qd)[i]);
          fa.add(__fmul_rn(v, (float)pr[p].cA));
          fb.add(__fmul_rn(v, (float)pr[p].cB));
        }
        fa.flush(&a);
        fb.flush(&b);
      } else {
        for (int p = 0; p < np; p++) {
          const double v = reinterpret_cast<const double*>(pr[p].q)[i] * reinterpret_cast<const double*>(pr[p].qd)[i];
          a = fma(pr[p].cA, v, a);
          b = fma(pr[p].cB, v, b);
        }
      }
      accA[i] = a;
      accB[i] = b;
    } else {
      double2* A2 = reinterpret_cast<double2*>(accA);
      double2* B2 = reinterpret_cast<double2*>(accB);
      double2 a = A2[i], b = B2[i];
      if constexpr (sizeof(T) == 4) {
        F2Sum far, fai, fbr, fbi;
        for (int p = 0; p < np; p++) {
          const float2 v = cmul(reinterpret_cast<const float2*>(pr[p].q)[i], reinterpret_cast<const float2*>(pr[p].qd)[i]);
          const float wa = (float)pr[p].cA, wb = (float)pr[p].cB;
          far.add(__fmul_rn(v.x, wa));
          fai.add(__fmul_rn(v.y, wa));
          fbr.add(__fmul_rn(v.x, wb));
          fbi.add(__fmul_rn(v.y, wb));
        }
        far.flush(&a.x);
        fai.flush(&a.y);
        fbr.flush(&b.x);
        fbi.flush(&b.y);
      } else {
        for (int p = 0; p < np; p++) {
          const double2 v = cmul(reinterpret_cast<const double2*>(pr[p].q)[i], reinterpret_cast<const double2*>(pr[p].qd)[i]);
          a.x = fma(pr[p].cA, v.x, a.x);
          a.y = fma(pr[p].cA, v.y, a.y);
          b.x = fma(pr[p].cB, v.x, b.x);
          b.y = fma(pr[p].cB, v.y, b.y);
        }
      }
      A2[i] = a;
      B2[i] = b;
    }
  }
}

// Contour quadrature of Eq. 8 with a weight table: accA = sum_n w[n] q_n qd_{Ns-n},
// accB = sum_n w[Ns+1+n] q_n qd_{Ns-n} (composite Simpson weights of the 4th-order
// scheme).  Integrand in the propagators' precision, FP64 sums; two grid points per
// thread (real) or one (complex).
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_quadrature_w_real(const T* __restrict__ hist, const T* __restrict__ qdh,
                                                                  const T* __restrict__ qd0, long long M, int Ns,
                                                                  const double* __restrict__ w,
                                                                  double* __restrict__ accA, double* __restrict__ accB) {
  const long long M2 = M / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M2; i += (long long)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
#pragma unroll 2
    for (int n = 0; n <= Ns; n++) {
      const int m = Ns - n;
      const cpx<T> q = reinterpret_cast<const cpx<T>*>(hist + (long long)n * M)[i];
      const cpx<T> d = reinterpret_cast<const cpx<T>*>(m == 0 ? qd0 : qdh + (long long)m * M)[i];
      const double p0 = widen(q.x * d.x), p1 = widen(q.y * d.y);
      const double wa = w[n], wb = w[Ns + 1 + n];
      a0 = fma(wa, p0, a0);
      a1 = fma(wa, p1, a1);
      b0 = fma(wb, p0, b0);
      b1 = fma(wb, p1, b1);
    }
    reinterpret_cast<double2*>(accA)[i] = make_double2(a0, a1);
    reinterpret_cast<double2*>(accB)[i] = make_double2(b0, b1);
  }
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_quadrature_w_cplx(const cpx<T>* __restrict__ hist,
                                                                  const cpx<T>* __restrict__ qdh,
                                                                  const cpx<T>* __restrict__ qd0, long long M, int Ns,
                                                                  const double* __restrict__ w,
                                                                  double2* __restrict__ accA,
                                                                  double2* __restrict__ accB) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
#pragma unroll 2
    for (int n = 0; n <= Ns; n++) {
      const int m = Ns - n;
      const cpx<T> pq = cmul(hist[(long long)n * M + i], (m == 0 ? qd0 : qdh + (long long)m * M)[i]);
      const double pr = widen(pq.x), pi = widen(pq.y);
      const double wa = w[n], wb = w[Ns + 1 + n];
      ar = fma(wa, pr, ar);
      ai = fma(wa, pi, ai);
      br = fma(wb, pr, br);
      bi = fma(wb, pi, bi);
    }
    accA[i] = make_double2(ar, ai);
    accB[i] = make_double2(br, bi);
  }
}

// Q, lnQ (principal branch) and H = C dV field_sum - C V lnQ (Eqs. 3, 4).
static __global__ void k_observables(double* __restrict__ s, double M, double C) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double qr = s[S_QSUM] / M, qi = s[S_QSUM + 1] / M;
  s[S_Q] = qr;
  s[S_Q + 1] = qi;
  double lr, li;
  if (qi == 0.0) {
    lr = log(fabs(qr));
    li = (qr < 0.0) ? 3.14159265358979323846 : 0.0;
  } else {
    lr = 0.5 * log(qr * qr + qi * qi);
    li = atan2(qi, qr);
  }
  s[S_LNQ] = lr;
  s[S_LNQ + 1] = li;
  const double V = s[S_VOL];
  const double dV = V / M;
  s[S_H] = C * dV * s[S_FIELD] - C * V * lr;
  s[S_H + 1] = C * dV * s[S_FIELD + 1] - C * V * li;
}

// phi = ds * acc / Q (Eq. 8) in place, plus sums of phi and of the squared forces (Eq. 7).
static __global__ void __launch_bounds__(PW_THREADS) k_finalize_real(double* __restrict__ accA, double* __restrict__ accB,
                                                              const double* __restrict__ wm, const double* __restrict__ s,
                                                              double ds, double chiN, long long M,
                                                              double* __restrict__ partials) {
  const double f = ds / s[S_Q];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double a = accA[i] * f, b = accB[i] * f;
    accA[i] = a;
    accB[i] = b;
    const double fp = a + b - 1.0, fm = 2.0 * wm[i] * ichiN + b - a;
    acc[0] += a;
    acc[2] += b;
    acc[4] += fp * fp;
    acc[5] += fm * fm;
  }
  block_reduce_store<6>(acc, partials + 6 * blockIdx.x);
}

static __global__ void __launch_bounds__(PW_THREADS) k_finalize_cplx(double2* __restrict__ accA, double2* __restrict__ accB,
                                                              const double2* __restrict__ wm, const double* __restrict__ s,
                                                              double ds, double chiN, long long M,
                                                              double* __restrict__ partials) {
  const double2 f = cdiv_d(make_double2(ds, 0.0), make_double2(s[S_Q], s[S_Q + 1]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = cmul_d(accA[i], f), b = cmul_d(accB[i], f);
    accA[i] = a;
    accB[i] = b;
    const double2 fp = make_double2(a.x + b.x - 1.0, a.y + b.y);  // |i fp| = |fp|
    const double2 m = wm[i];
    const double2 fm = make_double2(2.0 * m.x * ichiN + b.x - a.x, 2.0 * m.y * ichiN + b.y - a.y);
    acc[0] += a.x;
    acc[1] += a.y;
    acc[2] += b.x;
    acc[3] += b.y;
    acc[4] += fp.x * fp.x + fp.y * fp.y;
    acc[5] += fm.x * fm.x + fm.y * fm.y;
  }
  block_reduce_store<6>(acc, partials + 6 * blockIdx.x);
}

// Explicit Euler SCFT relaxation (Eq. 9, no noise, Wick-rotated), then the new
// Boltzmann factors and field term.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_step_scft(double* __restrict__ wp, double* __restrict__ wm,
                                                          const double* __restrict__ phiA, const double* __restrict__ phiB,
                                                          T* __restrict__ BA, T* __restrict__ BB, double lam, double ds,
                                                          double chiN, long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double a = phiA[i], b = phiB[i];
    double p = wp[i], m = wm[i];
    const double fp = a + b - 1.0, fm = 2.0 * m * ichiN + b - a;
    p += lam * fp;
    m -= lam * fm;
    wp[i] = p;
    wm[i] = m;
    BA[i] = boltz<T>(p - m, ds);
    BB[i] = boltz<T>(p + m, ds);
    acc[0] += m * m * ichiN - p;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// The same step for FP32 factors, two grid points a thread (16-byte loads): the field
// update in FP64, the factors' arguments from the narrowed fields (integer-pipe rounding)
// times -ds/2 in FP32 -- within one FP32 rounding of the FP64 argument, far below the
// rounding of the stored factor -- so that the FP64 pipe (1/64 of FP32 on GB300) does
// only the update and the field-term sum.
static __global__ void __launch_bounds__(PW_THREADS) k_step_scft2(double* __restrict__ wp, double* __restrict__ wm,
                                                                  const double* __restrict__ phiA,
                                                                  const double* __restrict__ phiB,
                                                                  float* __restrict__ BA, float* __restrict__ BB,
                                                                  double lam, double ds, double chiN, long long M,
                                                                  double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const double ichiN = 1.0 / chiN;
  const double cm = 1.0 - 2.0 * lam * ichiN;  // W- <- cm W- - lam (phiB - phiA)
  const float hds = (float)(-0.5 * ds);
  const long long M2 = M / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M2; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = reinterpret_cast<const double2*>(phiA)[i], b = reinterpret_cast<const double2*>(phiB)[i];
    double2 p = reinterpret_cast<double2*>(wp)[i], m = reinterpret_cast<double2*>(wm)[i];
    p.x += lam * (a.x + b.x - 1.0);
    p.y += lam * (a.y + b.y - 1.0);
    m.x = cm * m.x - lam * (b.x - a.x);
    m.y = cm * m.y - lam * (b.y - a.y);
    reinterpret_cast<double2*>(wp)[i] = p;
    reinterpret_cast<double2*>(wm)[i] = m;
    reinterpret_cast<float2*>(BA)[i] = make_float2(expf(narrow_rn(p.x - m.x) * hds), expf(narrow_rn(p.y - m.y) * hds));
    reinterpret_cast<float2*>(BB)[i] = make_float2(expf(narrow_rn(p.x + m.x) * hds), expf(narrow_rn(p.y + m.y) * hds));
    acc[0] += (m.x * m.x + m.y * m.y) * ichiN - (p.x + p.y);
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// Euler-Maruyama complex Langevin step (Eq. 9 with the Eq. 7 forces per C and real
// noise of variance 2 dt/(C dV)), four grid points per thread so that one Philox
// block serves four consecutive points of each field.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_step_cl(double2* __restrict__ wp, double2* __restrict__ wm,
                                                        const double2* __restrict__ phiA, const double2* __restrict__ phiB,
                                                        cpx<T>* __restrict__ BA, cpx<T>* __restrict__ BB, double dt,
                                                        double noise_std, const double* __restrict__ eta_p,
                                                        const double* __restrict__ eta_m, unsigned long long seed,
                                                        unsigned long long instance, unsigned long long step_arg,
                                                        const unsigned long long* __restrict__ step_dev, double ds,
                                                        double chiN, long long M, double* __restrict__ partials) {
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  double acc[2] = {0.0, 0.0};
  const unsigned long long step = step_dev ? *step_dev : step_arg;
  const long long nblk = (M + 3) / 4;
  for (long long bk = blockIdx.x * (long long)blockDim.x + threadIdx.x; bk < nblk;
       bk += (long long)gridDim.x * blockDim.x) {
    double zp[4], zm[4];
    if (eta_p) {
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const long long i = 4 * bk + j;
        zp[j] = (i < M) ? eta_p[i] : 0.0;
        zm[j] = (i < M) ? eta_m[i] : 0.0;
      }
    } else {
      philox_normal4(seed, instance, step, 0, bk, zp);
      philox_normal4(seed, instance, step, 1, bk, zm);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        zp[j] *= noise_std;
        zm[j] *= noise_std;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long i = 4 * bk + j;
      if (i >= M) break;
      const double2 a = phiA[i], b = phiB[i];
      double2 p = wp[i], m = wm[i];
      // dH/dw+ per C = i (phiA + phiB - 1)
      const double2 s = make_double2(a.x + b.x - 1.0, a.y + b.y);
      const double2 fp = make_double2(-s.y, s.x);
      const double2 fm = make_double2(2.0 * m.x * ichiN + b.x - a.x, 2.0 * m.y * ichiN + b.y - a.y);
      p.x += -dt * fp.x + zp[j];
      p.y += -dt * fp.y;
      m.x += -dt * fm.x + zm[j];
      m.y += -dt * fm.y;
      wp[i] = p;
      wm[i] = m;
      const double2 ip = make_double2(-p.y, p.x);
      const double2 wA = make_double2(ip.x - m.x, ip.y - m.y);
      const double2 wB = make_double2(ip.x + m.x, ip.y + m.y);
      BA[i] = boltz_c<T>(wA, ds);
      BB[i] = boltz_c<T>(wB, ds);
      acc[0] += (m.x * m.x - m.y * m.y) * ichiN + p.y;
      acc[1] += 2.0 * m.x * m.y * ichiN - p.x;
    }
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// --------------------------------------------- reverse-mode adjoint of the march
// One step of both adjoint marches (real fields): with z = K(B lambda) from the batched
// transforms, each chain adds -(ds/2)(lambda q_k + B q_{k-1} z) to the gradient of the
// block of its split step and moves to lambda_{k-1} = B z + g (ds/Q)(cA GA + cB GB) src,
// src the partner history slice of the source term.  Chain 0 adjoins the q march, chain 1
// the qd march.
struct AdjChain {
  const void* lam;   // lambda_k
  void* lam_next;    // lambda_{k-1}
  const void* z;     // K(B_k lambda_k)
  const void* qk;    // q_k (or qd_k)
  const void* qk1;   // q_{k-1}
  const void* B;     // factor of the split step
  const void* src;   // partner slice of the source at k-1
  double cA, cB;     // quadrature weights of that source
  int blockA;        // the split step lies in the A block
};

// One chain per launch (the two chains run on two streams), each with its own gradient
// accumulators dwA, dwB.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_adjoint_update(AdjChain c, const double* __restrict__ GA,
                                                               const double* __restrict__ GB,
                                                               const double* __restrict__ s, double ds,
                                                               double* __restrict__ dwA, double* __restrict__ dwB,
                                                               long long M) {
  const double f = ds / s[S_Q];
  const double h = -0.5 * ds;
  double* __restrict__ dw = c.blockA ? dwA : dwB;
  const double g0 = f * c.cA, g1 = f * c.cB;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const T lam = ((const T*)c.lam)[i];
    const T z = ((const T*)c.z)[i];
    const T B = ((const T*)c.B)[i];
    dw[i] = fma(h, widen(lam * ((const T*)c.qk)[i]) + widen(B * ((const T*)c.qk1)[i] * z), dw[i]);
    double g = 0.0;
    if (g0 != 0.0) g += g0 * GA[i];
    if (g1 != 0.0) g += g1 * GB[i];
    ((T*)c.lam_next)[i] = narrow_rn_as(fma(g, widen(((const T*)c.src)[i]), widen(B * z)), T(0));
  }
}

// lambda_Ns = g_Ns qd_0 and mu_Ns = g_0 q_0 (both starting slices are the initial
// conditions), and the gradient accumulators cleared.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_adjoint_init(T* __restrict__ lam, T* __restrict__ mu,
                                                             const T* __restrict__ qd0, const T* __restrict__ q0,
                                                             const double* __restrict__ GA,
                                                             const double* __restrict__ GB,
                                                             const double* __restrict__ s, double ds, double cAl,
                                                             double cBl, double cAm, double cBm,
                                                             double* __restrict__ dw, long long M) {
  const double f = ds / s[S_Q];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double ga = GA[i], gb = GB[i];
    lam[i] = (T)(f * (cAl * ga + cBl * gb) * (double)qd0[i]);
    mu[i] = (T)(f * (cAm * ga + cBm * gb) * (double)q0[i]);
    for (int j = 0; j < 4; j++) dw[(long long)j * M + i] = 0.0;
  }
}

// ---- the adjoint on the separable march (FP32 real fields): both adjoint marches store
// their histories (lambda_k, mu_m) and one pass forms the gradient afterwards.
// Set-up: gA = (ds/Q) GA and gB = (ds/Q) GB in FP32 (the sources of the marches are
// (cA_k gA + cB_k gB) times a history slice), lambda_Ns = (cA_Ns gA + cB_Ns gB) qd_0 and
// mu_Ns = (cA_0 gA + cB_0 gB) q_0.
static __global__ void __launch_bounds__(PW_THREADS) k_adjsep_init(
    const double* __restrict__ GA, const double* __restrict__ GB, const double* __restrict__ s, double ds,
    float* __restrict__ gA, float* __restrict__ gB, float* __restrict__ lamNs, float* __restrict__ muNs,
    const float* __restrict__ qd0, const float* __restrict__ q0, float cAl, float cBl, float cAm, float cBm,
    long long M) {
  const double f = ds / s[S_Q];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const float a = narrow_rn(f * GA[i]), b = narrow_rn(f * GB[i]);
    gA[i] = a;
    gB[i] = b;
    lamNs[i] = (cAl * a + cBl * b) * qd0[i];
    muNs[i] = (cAm * a + cBm * b) * q0[i];
  }
}

// Trapezoid weights of slice n on each block (as trap_w), in FP32 (exact: 0, 1/2, 1).
__device__ __forceinline__ void trap_wf(int n, int Ns, int NsA, float* cA, float* cB) {
  *cA = 0.f;
  *cB = 0.f;
  if (NsA > 0 && n <= NsA) *cA = (n == 0 || n == NsA) ? 0.5f : 1.f;
  if (NsA < Ns && n >= NsA) *cB = (n == NsA || n == Ns) ? 0.5f : 1.f;
}

// The gradient of the loss from the stored histories, one pass, four points a thread.
// Step n of the lambda chain (split step n) adds -(ds/2) [lambda_n q_n + q_{n-1}
// (lambda_{n-1} - a_{n-1})] (B_n z_n = lambda_{n-1} - a_{n-1}, a_k = (cA_k gA + cB_k gB)
// qd_{Ns-k}); step m = Ns + 1 - n of the mu chain (split step n as well) adds -(ds/2)
// [mu_m qd_m + qd_{m-1} (mu_{m-1} - b_{m-1})], b_k = (cA_{Ns-k} gA + cB_{Ns-k} gB) q_{Ns-k}.
// Both go to the block of split step n; the sums are compensated FP32 over chunks of
// kQuadChunk steps flushed into FP64.  Then dL/dW+ = dwA + dwB + gamma (phiA + phiB)/M and
// dL/dW- = dwB - dwA + gamma (phiB - phiA)/M.
static __global__ void __launch_bounds__(PW_THREADS) k_adjsep_grad(
    const float* __restrict__ lam, const float* __restrict__ mu, const float* __restrict__ hist,
    const float* __restrict__ qdh, const float* __restrict__ qd0, const float* __restrict__ gA,
    const float* __restrict__ gB, const double* __restrict__ phiA, const double* __restrict__ phiB,
    const double* __restrict__ gamma, double invM, double ds, int Ns, int NsA, long long M, double* __restrict__ dwp,
    double* __restrict__ dwm) {
  const long long M4 = M / 4;
  const double gm = gamma[0] * invM;
  auto qd = [&](int m) { return m == 0 ? qd0 : qdh + (long long)m * M; };
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M4; i += (long long)gridDim.x * blockDim.x) {
    const float4 ga = reinterpret_cast<const float4*>(gA)[i], gb = reinterpret_cast<const float4*>(gB)[i];
    const float gaa[4] = {ga.x, ga.y, ga.z, ga.w}, gbb[4] = {gb.x, gb.y, gb.z, gb.w};
    // values of step n - 1: lambda_{n-1}, q_{n-1}, mu_{Ns+1-n}, qd_{Ns+1-n}
    float4 lp = reinterpret_cast<const float4*>(lam)[i];
    float4 qp = reinterpret_cast<const float4*>(hist)[i];
    float4 mp = reinterpret_cast<const float4*>(mu + (long long)Ns * M)[i];
    float4 dp = reinterpret_cast<const float4*>(qd(Ns))[i];
    double dA[4] = {0, 0, 0, 0}, dB[4] = {0, 0, 0, 0};
    F2Sum fA[4], fB[4];
    int cnt = 0;
#pragma unroll 1
    for (int n = 1; n <= Ns; n++) {
      const int m = Ns + 1 - n;
      const float4 ln = reinterpret_cast<const float4*>(lam + (long long)n * M)[i];
      const float4 qn = reinterpret_cast<const float4*>(hist + (long long)n * M)[i];
      const float4 mm1 = reinterpret_cast<const float4*>(mu + (long long)(m - 1) * M)[i];
      const float4 dm1 = reinterpret_cast<const float4*>(qd(m - 1))[i];
      float cAa, cBa, cAb, cBb;
      trap_wf(n - 1, Ns, NsA, &cAa, &cBa);  // weights of a_{n-1}
      trap_wf(Ns - m + 1, Ns, NsA, &cAb, &cBb);  // weights of b_{m-1}: index Ns - (m - 1) = n
      const float l1[4] = {lp.x, lp.y, lp.z, lp.w}, q1[4] = {qp.x, qp.y, qp.z, qp.w};
      const float l0[4] = {ln.x, ln.y, ln.z, ln.w}, q0v[4] = {qn.x, qn.y, qn.z, qn.w};
      const float mu0[4] = {mp.x, mp.y, mp.z, mp.w}, d0[4] = {dp.x, dp.y, dp.z, dp.w};
      const float mu1[4] = {mm1.x, mm1.y, mm1.z, mm1.w}, d1[4] = {dm1.x, dm1.y, dm1.z, dm1.w};
      const bool blkA = (n <= NsA);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        // lambda chain: a_{n-1} = (cA gA + cB gB) qd_{Ns-n+1}; qd_{Ns+1-n} = d0
        const float a = (cAa * gaa[k] + cBa * gbb[k]) * d0[k];
        const float tl = __fadd_rn(__fmul_rn(l0[k], q0v[k]), __fmul_rn(q1[k], __fsub_rn(l1[k], a)));
        // mu chain: b_{m-1} = (cA_n gA + cB_n gB) q_n
        const float b = (cAb * gaa[k] + cBb * gbb[k]) * q0v[k];
        const float tm = __fadd_rn(__fmul_rn(mu0[k], d0[k]), __fmul_rn(d1[k], __fsub_rn(mu1[k], b)));
        if (blkA) {
          fA[k].add(tl);
          fA[k].add(tm);
        } else {
          fB[k].add(tl);
          fB[k].add(tm);
        }
      }
      lp = ln;
      qp = qn;
      mp = mm1;
      dp = dm1;
      if (++cnt == kQuadChunk || n == Ns) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
          fA[k].flush(&dA[k]);
          fB[k].flush(&dB[k]);
        }
        cnt = 0;
      }
    }
    const double h = -0.5 * ds;
    const double2 pA0 = reinterpret_cast<const double2*>(phiA)[2 * i], pA1 = reinterpret_cast<const double2*>(phiA)[2 * i + 1];
    const double2 pB0 = reinterpret_cast<const double2*>(phiB)[2 * i], pB1 = reinterpret_cast<const double2*>(phiB)[2 * i + 1];
    const double pa[4] = {pA0.x, pA0.y, pA1.x, pA1.y}, pb[4] = {pB0.x, pB0.y, pB1.x, pB1.y};
    double op[4], om[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const double a = h * dA[k] + gm * pa[k], b = h * dB[k] + gm * pb[k];
      op[k] = a + b;
      om[k] = b - a;
    }
    reinterpret_cast<double2*>(dwp)[2 * i] = make_double2(op[0], op[1]);
    reinterpret_cast<double2*>(dwp)[2 * i + 1] = make_double2(op[2], op[3]);
    reinterpret_cast<double2*>(dwm)[2 * i] = make_double2(om[0], om[1]);
    reinterpret_cast<double2*>(dwm)[2 * i + 1] = make_double2(om[2], om[3]);
  }
}

// gamma = sum_x (GA phiA + GB phiB), partial sums per block.
static __global__ void __launch_bounds__(PW_THREADS) k_adjoint_gamma(const double* __restrict__ GA,
                                                                     const double* __restrict__ GB,
                                                                     const double* __restrict__ phiA,
                                                                     const double* __restrict__ phiB, long long M,
                                                                     double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    acc[0] += GA[i] * phiA[i] + GB[i] * phiB[i];
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// dL/dW+ = dwA + dwB + gamma (phiA + phiB)/M, dL/dW- = dwB - dwA + gamma (phiB - phiA)/M,
// dwA and dwB the sums of the two chains' accumulators (dw[0..1] chain 0, dw[2..3] chain 1).
static __global__ void __launch_bounds__(PW_THREADS) k_adjoint_finish(const double* __restrict__ dw,
                                                                      const double* __restrict__ phiA,
                                                                      const double* __restrict__ phiB,
                                                                      const double* __restrict__ gamma, double invM,
                                                                      double* __restrict__ dwp,
                                                                      double* __restrict__ dwm, long long M) {
  const double gm = gamma[0] * invM;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double a = dw[i] + dw[2 * M + i] + gm * phiA[i], b = dw[M + i] + dw[3 * M + i] + gm * phiB[i];
    dwp[i] = a + b;
    dwm[i] = b - a;
  }
}

// ------------------------------------------------ Edwards homopolymer model (Eq. 2)
// Boltzmann factor of the one field (W = i omega stored in SCFT mode, omega in CL mode)
// and the field term of H per C: -(b/2) W^2 (SCFT) or (b/2) omega^2 (CL), b = B/C.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_prepare_edw_real(const double* __restrict__ W, T* __restrict__ BA,
                                                                 double ds, double b, long long M,
                                                                 double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double w = W[i];
    BA[i] = boltz<T>(w, ds);
    acc[0] -= 0.5 * b * w * w;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_prepare_edw_cplx(const double2* __restrict__ w, cpx<T>* __restrict__ BA,
                                                                 double ds, double b, long long M,
                                                                 double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 o = w[i];
    BA[i] = boltz_c<T>(make_double2(-o.y, o.x), ds);  // the chain feels i omega
    acc[0] += 0.5 * b * (o.x * o.x - o.y * o.y);
    acc[1] += b * o.x * o.y;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// phi = ds acc / Q in place (accB cleared), plus the sum of phi and of |force per C|^2:
// phi - b W (SCFT) or b omega + i phi (CL).
static __global__ void __launch_bounds__(PW_THREADS) k_finalize_edw_real(double* __restrict__ accA,
                                                                         double* __restrict__ accB,
                                                                         const double* __restrict__ W,
                                                                         const double* __restrict__ s, double ds,
                                                                         double b, long long M,
                                                                         double* __restrict__ partials) {
  const double f = ds / s[S_Q];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double p = accA[i] * f;
    accA[i] = p;
    accB[i] = 0.0;
    const double F = p - b * W[i];
    acc[0] += p;
    acc[4] += F * F;
  }
  block_reduce_store<6>(acc, partials + 6 * blockIdx.x);
}

static __global__ void __launch_bounds__(PW_THREADS) k_finalize_edw_cplx(double2* __restrict__ accA,
                                                                         double2* __restrict__ accB,
                                                                         const double2* __restrict__ w,
                                                                         const double* __restrict__ s, double ds,
                                                                         double b, long long M,
                                                                         double* __restrict__ partials) {
  const double2 f = cdiv_d(make_double2(ds, 0.0), make_double2(s[S_Q], s[S_Q + 1]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 p = cmul_d(accA[i], f);
    accA[i] = p;
    accB[i] = make_double2(0.0, 0.0);
    const double2 o = w[i];
    const double2 F = make_double2(b * o.x - p.y, b * o.y + p.x);  // b omega + i phi
    acc[0] += p.x;
    acc[1] += p.y;
    acc[4] += F.x * F.x + F.y * F.y;
  }
  block_reduce_store<6>(acc, partials + 6 * blockIdx.x);
}

// SCFT relaxation of the Wick-rotated field, ascent with the force per C:
// W += lam (phi - b W); then its Boltzmann factor and field term.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_step_edw_scft(double* __restrict__ W, const double* __restrict__ phi,
                                                              T* __restrict__ BA, double lam, double ds, double b,
                                                              long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    double w = W[i];
    w += lam * (phi[i] - b * w);
    W[i] = w;
    BA[i] = boltz<T>(w, ds);
    acc[0] -= 0.5 * b * w * w;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// Euler-Maruyama complex Langevin step: omega += -dt (b omega + i phi) + eta, real eta of
// variance 2 dt/(C dV) from the Philox stream (field 0) or the caller.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_step_edw_cl(double2* __restrict__ w, const double2* __restrict__ phi,
                                                            cpx<T>* __restrict__ BA, double dt, double noise_std,
                                                            const double* __restrict__ eta,
                                                            unsigned long long seed, unsigned long long instance,
                                                            unsigned long long step_arg,
                                                            const unsigned long long* __restrict__ step_dev, double ds,
                                                            double b, long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const unsigned long long step = step_dev ? *step_dev : step_arg;
  const long long nblk = (M + 3) / 4;
  for (long long bk = blockIdx.x * (long long)blockDim.x + threadIdx.x; bk < nblk;
       bk += (long long)gridDim.x * blockDim.x) {
    double z[4];
    if (eta) {
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const long long i = 4 * bk + j;
        z[j] = (i < M) ? eta[i] : 0.0;
      }
    } else {
      philox_normal4(seed, instance, step, 0, bk, z);
#pragma unroll
      for (int j = 0; j < 4; j++) z[j] *= noise_std;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long i = 4 * bk + j;
      if (i >= M) break;
      double2 o = w[i];
      const double2 p = phi[i];
      o.x += -dt * (b * o.x - p.y) + z[j];
      o.y += -dt * (b * o.y + p.x);
      w[i] = o;
      BA[i] = boltz_c<T>(make_double2(-o.y, o.x), ds);
      acc[0] += 0.5 * b * (o.x * o.x - o.y * o.y);
      acc[1] += b * o.x * o.y;
    }
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// ------------------------------------------------- semi-implicit step (Eq. 11)
// Debye function of the whole chain, g_D(x) = 2 (e^{-x} + x - 1) / x^2 at x = k^2 (Rg = 1):
// the closed form from x = 0.1 up, below it the Taylor series 2 sum_{j>=0} (-x)^j / (j+2)!
// through x^9 (the closed form loses digits to cancellation there).
__device__ __forceinline__ double debye_chain(double x) {
  if (x >= 0.1) return 2.0 * (exp(-x) + x - 1.0) / (x * x);
  const double c[10] = {1.0,          -2.0 / 6.0,      2.0 / 24.0,      -2.0 / 120.0,      2.0 / 720.0,
                        -2.0 / 5040.0, 2.0 / 40320.0, -2.0 / 362880.0, 2.0 / 3628800.0, -2.0 / 39916800.0};
  double r = c[9];
#pragma unroll
  for (int j = 8; j >= 0; j--) r = fma(r, x, c[j]);
  return r;
}

// SCFT: G = lam (phiA + phiB - 1) as a complex array for the transform, and the
// exchange field with its linear term implicit: W- = (W- - lam (phiB - phiA)) / (1 + 2 lam/chiN).
static __global__ void __launch_bounds__(PW_THREADS) k_sis_force_real(const double* __restrict__ phiA,
                                                               const double* __restrict__ phiB,
                                                               double* __restrict__ wm, double2* __restrict__ G,
                                                               double lam, double chiN, long long M) {
  const double inv = 1.0 / (1.0 + 2.0 * lam / chiN);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double a = phiA[i], b = phiB[i];
    G[i] = make_double2(lam * (a + b - 1.0), 0.0);
    wm[i] = (wm[i] - lam * (b - a)) * inv;
  }
}

// CL: G = -dt i (phiA + phiB - 1) + eta+ and w- = (w- - dt (phiB - phiA) + eta-) / (1 + 2 dt/chiN),
// the noise from the Philox stream (same counters as the Euler-Maruyama step) or the caller.
static __global__ void __launch_bounds__(PW_THREADS) k_sis_force_cplx(const double2* __restrict__ phiA,
                                                               const double2* __restrict__ phiB,
                                                               double2* __restrict__ wm, double2* __restrict__ G,
                                                               double dt, double noise_std,
                                                               const double* __restrict__ eta_p,
                                                               const double* __restrict__ eta_m,
                                                               unsigned long long seed, unsigned long long instance,
                                                               unsigned long long step_arg,
                                                               const unsigned long long* __restrict__ step_dev,
                                                               double chiN, long long M) {
  const unsigned long long step = step_dev ? *step_dev : step_arg;
  const double inv = 1.0 / (1.0 + 2.0 * dt / chiN);
  const long long nblk = (M + 3) / 4;
  for (long long bk = blockIdx.x * (long long)blockDim.x + threadIdx.x; bk < nblk;
       bk += (long long)gridDim.x * blockDim.x) {
    double zp[4], zm[4];
    if (eta_p) {
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const long long i = 4 * bk + j;
        zp[j] = (i < M) ? eta_p[i] : 0.0;
        zm[j] = (i < M) ? eta_m[i] : 0.0;
      }
    } else {
      philox_normal4(seed, instance, step, 0, bk, zp);
      philox_normal4(seed, instance, step, 1, bk, zm);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        zp[j] *= noise_std;
        zm[j] *= noise_std;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long i = 4 * bk + j;
      if (i >= M) break;
      const double2 a = phiA[i], b = phiB[i];
      // -dt i (s - 1) with s = phiA + phiB
      const double sr = a.x + b.x - 1.0, si = a.y + b.y;
      G[i] = make_double2(dt * si + zp[j], -dt * sr);
      double2 m = wm[i];
      m.x = (m.x - dt * (b.x - a.x) + zm[j]) * inv;
      m.y = (m.y - dt * (b.y - a.y)) * inv;
      wm[i] = m;
    }
  }
}

// G^(k) /= 1 + a g_D(k^2) on the full (nx, ny, nz) complex grid; k^2 from the per-axis
// tables (the z table may hold only kz <= nz/2: k^2 is even in kz).
static __global__ void __launch_bounds__(PW_THREADS) k_sis_scale(double2* __restrict__ G, const double* __restrict__ gx,
                                                          const double* __restrict__ gy, const double* __restrict__ gz,
                                                          int ny, int nz, double a, long long M) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(i % nz);
    const long long r = i / nz;
    const int ky = (int)(r % ny);
    const int kx = (int)(r / ny);
    const int kzz = kz <= nz - kz ? kz : nz - kz;
    const double k2 = gx[kx] + gy[ky] + gz[kzz];
    const double f = 1.0 / (1.0 + a * debye_chain(k2));
    double2 g = G[i];
    g.x *= f;
    g.y *= f;
    G[i] = g;
  }
}

// W+ += Re(G)/M (the unnormalised inverse transform), then the Boltzmann factors of the
// new fields and the field term of Eq. 3.
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_sis_apply_real(double* __restrict__ wp, const double* __restrict__ wm,
                                                               const double2* __restrict__ G, T* __restrict__ BA,
                                                               T* __restrict__ BB, double invM, double ds, double chiN,
                                                               long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double p = wp[i] + G[i].x * invM, m = wm[i];
    wp[i] = p;
    BA[i] = boltz<T>(p - m, ds);
    BB[i] = boltz<T>(p + m, ds);
    acc[0] += m * m * ichiN - p;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_sis_apply_cplx(double2* __restrict__ wp, const double2* __restrict__ wm,
                                                               const double2* __restrict__ G, cpx<T>* __restrict__ BA,
                                                               cpx<T>* __restrict__ BB, double invM, double ds,
                                                               double chiN, long long M, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    double2 p = wp[i];
    const double2 g = G[i], m = wm[i];
    p.x += g.x * invM;
    p.y += g.y * invM;
    wp[i] = p;
    const double2 ip = make_double2(-p.y, p.x);
    BA[i] = boltz_c<T>(make_double2(ip.x - m.x, ip.y - m.y), ds);
    BB[i] = boltz_c<T>(make_double2(ip.x + m.x, ip.y + m.y), ds);
    acc[0] += (m.x * m.x - m.y * m.y) * ichiN + p.y;
    acc[1] += 2.0 * m.x * m.y * ichiN - p.x;
  }
  block_reduce_store<2>(acc, partials + 2 * blockIdx.x);
}

// Precision conversion of one slice (real or complex as 2 reals).
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ src, B* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (B)src[i];
}

// Exact gradients of the discrete H in the grid values of W+ and W- (Eq. 7 forces
// times C dV).  Either output may be null.
static __global__ void __launch_bounds__(PW_THREADS) k_grad_fields(const double* __restrict__ phiA,
                                                                   const double* __restrict__ phiB,
                                                                   const double* __restrict__ wm, double* __restrict__ gp,
                                                                   double* __restrict__ gm, double cdv, double chiN,
                                                                   long long M) {
  const double ichiN = 1.0 / chiN;  // one division per thread, not per point
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double a = phiA[i], b = phiB[i];
    if (gp) gp[i] = cdv * (a + b - 1.0);
    if (gm) gm[i] = cdv * (2.0 * wm[i] * ichiN + b - a);
  }
}

// Box derivative (stress) contraction for real fields: for one contour step,
// sum over the half spectrum of w(kz) Re[conj(u^) v^] k_a^2 exp(-k^2 ds), a = x, y, z,
// accumulated into per-block partials (same block -> same slots every step).
template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_stress_real(const cpx<T>* __restrict__ u, const cpx<T>* __restrict__ v,
                                                            const double* __restrict__ k2x, const double* __restrict__ k2y,
                                                            const double* __restrict__ k2z, const double* __restrict__ ex,
                                                            const double* __restrict__ ey, const double* __restrict__ ez,
                                                            int nx, int ny, int nzh, int nz, double* __restrict__ partials) {
  // exp(-k^2 ds) = ex[kx] ey[ky] ez[kz]; the float spectra are widened exactly
  double acc[3] = {0.0, 0.0, 0.0};
  const long long Ms = (long long)nx * ny * nzh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Ms; i += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(i % nzh);
    const long long r = i / nzh;
    const int ky = (int)(r % ny), kx = (int)(r / ny);
    const double wz = (kz == 0 || 2 * kz == nz) ? 1.0 : 2.0;
    const cpx<T> a = u[i], b = v[i];
    const double re = fma(widen(a.x), widen(b.x), widen(a.y) * widen(b.y));
    const double w = wz * re * (ex[kx] * ey[ky] * ez[kz]);
    acc[0] = fma(w, k2x[kx], acc[0]);
    acc[1] = fma(w, k2y[ky], acc[1]);
    acc[2] = fma(w, k2z[kz], acc[2]);
  }
  block_reduce_store<3, true>(acc, partials + 3 * blockIdx.x);
}

}  // namespace pft

namespace pft {
static __global__ void k_increment_u64(unsigned long long* __restrict__ c, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] += 1ull;
}
}  // namespace pft
