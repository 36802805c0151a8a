// pft_passes.cuh -- the FFT pass kernels of one contour step
//   q_n = B_n * F^-1[ D * F[ B_n * q_{n-1} ] ]        (operator splitting, Eq. 13)
// on an [nx][ny][nz] grid (z contiguous).  One step is five passes over the
// spectrum buffer, each a batch of 1D transforms held in registers:
//   zf : z transform of B*q   (real->half spectrum in SCFT mode, complex in CL mode)
//   yf : y transform
//   x  : x transform, multiply by D(k)/M, inverse x transform   (fused)
//   yi : inverse y transform
//   zi : inverse z transform, multiply by B, store q_n; in the conjugate march
//        also accumulate c_n q_n qd_{Ns-n} into the FP64 density sums (Eq. 8)
#pragma once
#include "pft_fft.cuh"

namespace pft {

// Shared-memory exchange for column-interleaved tiles [pos][LD] (strided passes:
// consecutive threads own consecutive columns, so every access is conflict-free).
template <typename T> struct XchCols {
  cpx<T>* s;
  int ld;
  int c;
  __device__ __forceinline__ void put(int pos, cpx<T> z) { s[pos * ld + c] = z; }
  __device__ __forceinline__ cpx<T> get(int pos) const { return s[pos * ld + c]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Shared-memory exchange for pencil tiles [p][padded pos] (z passes: consecutive
// threads own consecutive elements of one pencil).  One pad slot every 128 bytes
// breaks the power-of-two strides of the Stockham scatter.
template <typename T> struct XchPencil {
  static constexpr int SH = (sizeof(cpx<T>) == 8) ? 4 : 3;
  cpx<T>* s;  // start of this thread's pencil
  __device__ __forceinline__ static int idx(int pos) { return pos + (pos >> SH); }
  __device__ __forceinline__ void put(int pos, cpx<T> z) { s[idx(pos)] = z; }
  __device__ __forceinline__ cpx<T> get(int pos) const { return s[idx(pos)]; }
  // a pencil's threads lie in one warp and pencil kernels launch whole warps
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};
template <typename T> __host__ __device__ constexpr int pencil_ld(int n) {
  return n + (n >> ((sizeof(cpx<T>) == 8) ? 4 : 3)) + 2;
}

// Columns per CTA of the strided passes and pencils per CTA of the z passes.
template <typename T> struct Tile { static constexpr int C = (sizeof(T) == 4) ? 16 : 8; };
// Pencils per CTA: about 256 threads, with the pencil tile inside the 48 KB of
// dynamic shared memory a launch gets without an opt-in attribute.
// Whole warps per CTA (a multiple of 32 / TPC pencils), so that the pencil exchanges
// synchronise only their warp.
template <typename T, int N> struct PencilsPerCta {
  static_assert(Plan<N>::TPC <= 32 && 32 % Plan<N>::TPC == 0, "a pencil's threads lie in one warp");
  static constexpr int unit = 32 / Plan<N>::TPC;  // pencils per warp
  static constexpr int by_threads = 256 / Plan<N>::TPC;
  static constexpr int by_smem = (48 * 1024) / (pencil_ld<T>(N) * (int)sizeof(cpx<T>));
  static constexpr int raw = by_threads < by_smem ? by_threads : by_smem;
  static constexpr int v = raw >= unit ? raw - raw % unit : unit;
};

// ---------------------------------------------------------------- strided pass
// MODE 0: forward transform; 1: inverse transform; 2: forward, multiply by
// dk[k]*dy[ky]*dz[kz], inverse (the x pass of a contour step); 3: multiply by the
// same factor, inverse (completes a step whose forward x transform already ran).
// Column col in [0, ncols): element k at data[(col / cin) * s_outer + col % cin + k * s_k].
template <typename T, int N, int MODE, class PL = Plan<N>, int C = Tile<T>::C>
__device__ __forceinline__ void strided_body(cpx<T>* __restrict__ data, long long ncols, long long cin, long long s_outer, long long s_k,
          const cpx<T>* __restrict__ tw, const T* __restrict__ dk, const T* __restrict__ dy,
          const T* __restrict__ dz, int nzc, long long tile) {
  constexpr int E = PL::E;
  constexpr int TPC = PL::TPC;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
  const int c = threadIdx.x % C;
  const int t = threadIdx.x / C;
  const long long col = (long long)tile * C + c;
  const bool valid = col < ncols;
  const long long colc = valid ? col : 0;
  const long long base = (colc / cin) * s_outer + (colc % cin);
  cpx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; i++) {
    v[i] = valid ? data[base + (long long)(t + TPC * i) * s_k] : mk<T>(T(0), T(0));
  }
  XchCols<T> x{sm, C, c};
  if (MODE == 1) {
    fft<T, true, N, PL>(v, t, tw, x);
  } else if (MODE != 3) {
    fft<T, false, N, PL>(v, t, tw, x);
  }
  if (MODE == 2 || MODE == 3) {
    const long long ky = colc / nzc, kz = colc % nzc;
    const T dyz = dy[ky] * dz[kz];
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], dk[t + TPC * i] * dyz);
    // the forward transform ended with a barrier after its last shared-memory reads
    fft<T, true, N, PL>(v, t, tw, x);
  }
  if (valid) {
#pragma unroll
    for (int i = 0; i < E; i++) data[base + (long long)(t + TPC * i) * s_k] = v[i];
  }
}

template <typename T, int N, int MODE, class PL = Plan<N>, int C = Tile<T>::C>
__global__ void __launch_bounds__(C * PL::TPC)
k_strided(cpx<T>* __restrict__ data, long long ncols, long long cin, long long s_outer, long long s_k,
          const cpx<T>* __restrict__ tw, const T* __restrict__ dk, const T* __restrict__ dy,
          const T* __restrict__ dz, int nzc) {
  strided_body<T, N, MODE, PL, C>(data, ncols, cin, s_outer, s_k, tw, dk, dy, dz, nzc, (long long)blockIdx.x);
}

// ----------------------------------------------------------- z passes, real
// Forward: pencil of nz = 2*N2 reals (times B) packed as N2 complex pairs, complex
// transform of length N2, then the even/odd split into the nz/2+1 half spectrum.
// twh: exp(-2 pi i m/N2); twf: exp(-2 pi i m/nz).
template <typename T, int N2>
__device__ __forceinline__ void zf_r2c_body(const T* __restrict__ q, const T* __restrict__ B, cpx<T>* __restrict__ spec, long long npen,
         const cpx<T>* __restrict__ twh, const cpx<T>* __restrict__ twf, long long tile) {
  constexpr int P = PencilsPerCta<T, N2>::v;
  constexpr int E = Plan<N2>::E;
  constexpr int TPC = Plan<N2>::TPC;
  constexpr int LD = pencil_ld<T>(N2);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long pen = (long long)tile * P + p;
  const bool valid = pen < npen;
  const long long pc = valid ? pen : 0;
  XchPencil<T> x{reinterpret_cast<cpx<T>*>(smraw) + p * LD};
  const cpx<T>* q2 = reinterpret_cast<const cpx<T>*>(q) + pc * N2;
  const cpx<T>* b2 = B ? reinterpret_cast<const cpx<T>*>(B) + pc * N2 : nullptr;
  cpx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; i++) {
    cpx<T> z = valid ? q2[t + TPC * i] : mk<T>(T(0), T(0));
    if (b2 && valid) {
      const cpx<T> b = b2[t + TPC * i];
      z.x *= b.x;
      z.y *= b.y;
    }
    v[i] = z;
  }
  fft<T, false, N2>(v, t, twh, x);  // ends with a barrier after its last reads
#pragma unroll
  for (int i = 0; i < E; i++) x.put(t + TPC * i, v[i]);
  __syncwarp();
  const T h = T(0.5);
  cpx<T>* out = spec + pc * (N2 + 1);
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int k = t + TPC * i;
    const cpx<T> zk = v[i];
    const cpx<T> zc = cconj(x.get(k == 0 ? 0 : N2 - k));
    const cpx<T> ev = cscale(cadd(zk, zc), h);
    const cpx<T> od = cscale(rot90<false>(csub(zk, zc)), h);  // -i/2 (Zk - conj Z_{N2-k})
    const cpx<T> X = cadd(ev, cmul(twf[k], od));
    if (valid) out[k] = X;
  }
  if (valid && t == 0) {
    const cpx<T> z0 = v[0];
    out[N2] = mk<T>(z0.x - z0.y, T(0));
  }
}

template <typename T, int N2>
__global__ void __launch_bounds__(PencilsPerCta<T, N2>::v * Plan<N2>::TPC)
k_zf_r2c(const T* __restrict__ q, const T* __restrict__ B, cpx<T>* __restrict__ spec, long long npen,
         const cpx<T>* __restrict__ twh, const cpx<T>* __restrict__ twf) {
  zf_r2c_body<T, N2>(q, B, spec, npen, twh, twf, (long long)blockIdx.x);
}

// Inverse: half spectrum -> N2 complex (even/odd merge, unnormalised) -> inverse
// transform -> nz reals.  EPI 0: out = B*y; EPI 1: out = B*y and
// accA += cA*out*partner, accB += cB*out*partner (FP64); EPI 2: out = y;
// EPI 3: out = (4 B*y - partner) / 3, the Richardson combination of Eq. 13 (B*y the two
// half steps, partner the full step).
template <typename T, int N2, int EPI>
__device__ __forceinline__ void zi_c2r_body(const cpx<T>* __restrict__ spec, const T* __restrict__ B, T* __restrict__ qout,
         const T* __restrict__ partner, double* __restrict__ accA, double* __restrict__ accB, double cA,
         double cB, long long npen, const cpx<T>* __restrict__ twh, const cpx<T>* __restrict__ twf, long long tile) {
  constexpr int P = PencilsPerCta<T, N2>::v;
  constexpr int E = Plan<N2>::E;
  constexpr int TPC = Plan<N2>::TPC;
  constexpr int LD = pencil_ld<T>(N2);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long pen = (long long)tile * P + p;
  const bool valid = pen < npen;
  const long long pc = valid ? pen : 0;
  XchPencil<T> x{reinterpret_cast<cpx<T>*>(smraw) + p * LD};
  const cpx<T>* in = spec + pc * (N2 + 1);
  // FP32: the epilogue's factor and partner first, so that their latency overlaps the
  // transform (FP64 is FP64-pipe bound and short of registers: it loads them after)
  constexpr bool kPre = sizeof(T) == 4;
  const long long o = pc * N2;
  const cpx<T>* b2 = reinterpret_cast<const cpx<T>*>(B);
  const cpx<T>* f2 = reinterpret_cast<const cpx<T>*>(partner);
  cpx<T> bb[E], ff[E];
  if (kPre) {
#pragma unroll
    for (int i = 0; i < E; i++) {
      if (EPI != 2) bb[i] = b2[o + t + TPC * i];
      if (EPI == 3) ff[i] = f2[o + t + TPC * i];
    }
  }
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int k = t + TPC * i;
    x.put(k, valid ? in[k] : mk<T>(T(0), T(0)));
  }
  if (t == 0) x.put(N2, valid ? in[N2] : mk<T>(T(0), T(0)));
  __syncwarp();
  cpx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int k = t + TPC * i;
    const cpx<T> xk = x.get(k);
    const cpx<T> xc = cconj(x.get(N2 - k));
    // Z_k = (X_k + conj X_{N2-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{N2-k})
    const cpx<T> d = rot90<true>(cmulc(csub(xk, xc), twf[k]));
    v[i] = cadd(cadd(xk, xc), d);
  }
  __syncwarp();
  fft<T, true, N2>(v, t, twh, x);
  if (!valid) return;
  cpx<T>* q2 = reinterpret_cast<cpx<T>*>(qout);
#pragma unroll
  for (int i = 0; i < E; i++) {
    const long long m = o + t + TPC * i;
    cpx<T> y = v[i];
    if (EPI != 2) {
      const cpx<T> b = kPre ? bb[i] : b2[m];
      y.x *= b.x;
      y.y *= b.y;
    }
    if (EPI == 3) {
      const cpx<T> f = kPre ? ff[i] : f2[m];
      y.x = (T(4) * y.x - f.x) / T(3);
      y.y = (T(4) * y.y - f.y) / T(3);
    }
    q2[m] = y;
    if (EPI == 1) {
      // integrand q qd in the propagators' precision, sum in FP64 (one DFMA each)
      const cpx<T> pp = reinterpret_cast<const cpx<T>*>(partner)[m];
      const double p0 = widen(y.x * pp.x);
      const double p1 = widen(y.y * pp.y);
      if (cA != 0.0) {
        double2* a = reinterpret_cast<double2*>(accA) + m;
        double2 av = *a;
        av.x += cA * p0;
        av.y += cA * p1;
        *a = av;
      }
      if (cB != 0.0) {
        double2* a = reinterpret_cast<double2*>(accB) + m;
        double2 av = *a;
        av.x += cB * p0;
        av.y += cB * p1;
        *a = av;
      }
    }
  }
}

template <typename T, int N2, int EPI>
__global__ void __launch_bounds__(PencilsPerCta<T, N2>::v * Plan<N2>::TPC)
k_zi_c2r(const cpx<T>* __restrict__ spec, const T* __restrict__ B, T* __restrict__ qout,
         const T* __restrict__ partner, double* __restrict__ accA, double* __restrict__ accB, double cA,
         double cB, long long npen, const cpx<T>* __restrict__ twh, const cpx<T>* __restrict__ twf) {
  zi_c2r_body<T, N2, EPI>(spec, B, qout, partner, accA, accB, cA, cB, npen, twh, twf, (long long)blockIdx.x);
}

// -------------------------------------------------------- z passes, complex
// Forward: pencil of nz complex values times complex B, transform of length nz.
template <typename T, int N>
__device__ __forceinline__ void zf_c2c_body(const cpx<T>* __restrict__ q, const cpx<T>* __restrict__ B, cpx<T>* __restrict__ spec, long long npen,
         const cpx<T>* __restrict__ tw, long long tile) {
  constexpr int P = PencilsPerCta<T, N>::v;
  constexpr int E = Plan<N>::E;
  constexpr int TPC = Plan<N>::TPC;
  constexpr int LD = pencil_ld<T>(N);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long pen = (long long)tile * P + p;
  const bool valid = pen < npen;
  const long long o = (valid ? pen : 0) * N;
  XchPencil<T> x{reinterpret_cast<cpx<T>*>(smraw) + p * LD};
  cpx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; i++) {
    cpx<T> z = valid ? q[o + t + TPC * i] : mk<T>(T(0), T(0));
    if (B && valid) z = cmul(z, B[o + t + TPC * i]);
    v[i] = z;
  }
  fft<T, false, N>(v, t, tw, x);
  if (valid) {
#pragma unroll
    for (int i = 0; i < E; i++) spec[o + t + TPC * i] = v[i];
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(PencilsPerCta<T, N>::v * Plan<N>::TPC)
k_zf_c2c(const cpx<T>* __restrict__ q, const cpx<T>* __restrict__ B, cpx<T>* __restrict__ spec, long long npen,
         const cpx<T>* __restrict__ tw) {
  zf_c2c_body<T, N>(q, B, spec, npen, tw, (long long)blockIdx.x);
}

// Inverse: transform of length nz, then the epilogue (EPI as for k_zi_c2r, complex
// products, no conjugation: the density sums are bilinear in q and qd).
template <typename T, int N, int EPI>
__device__ __forceinline__ void zi_c2c_body(const cpx<T>* __restrict__ spec, const cpx<T>* __restrict__ B, cpx<T>* __restrict__ qout,
         const cpx<T>* __restrict__ partner, double2* __restrict__ accA, double2* __restrict__ accB, double cA,
         double cB, long long npen, const cpx<T>* __restrict__ tw, long long tile) {
  constexpr int P = PencilsPerCta<T, N>::v;
  constexpr int E = Plan<N>::E;
  constexpr int TPC = Plan<N>::TPC;
  constexpr int LD = pencil_ld<T>(N);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long pen = (long long)tile * P + p;
  const bool valid = pen < npen;
  const long long o = (valid ? pen : 0) * N;
  XchPencil<T> x{reinterpret_cast<cpx<T>*>(smraw) + p * LD};
  // FP32: the epilogue's factor and partner first (latency overlaps the transform)
  constexpr bool kPre = sizeof(T) == 4;
  cpx<T> bb[E], ff[E];
  if (kPre) {
#pragma unroll
    for (int i = 0; i < E; i++) {
      if (EPI != 2) bb[i] = B[o + t + TPC * i];
      if (EPI == 3) ff[i] = partner[o + t + TPC * i];
    }
  }
  cpx<T> v[E];
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = valid ? spec[o + t + TPC * i] : mk<T>(T(0), T(0));
  fft<T, true, N>(v, t, tw, x);
  if (!valid) return;
#pragma unroll
  for (int i = 0; i < E; i++) {
    const long long m = o + t + TPC * i;
    cpx<T> y = v[i];
    if (EPI != 2) y = cmul(y, kPre ? bb[i] : B[m]);
    if (EPI == 3) {
      const cpx<T> f = kPre ? ff[i] : partner[m];
      y.x = (T(4) * y.x - f.x) / T(3);
      y.y = (T(4) * y.y - f.y) / T(3);
    }
    qout[m] = y;
    if (EPI == 1) {
      // integrand q qd in the propagators' precision, sum in FP64
      const cpx<T> pq = cmul(y, partner[m]);
      double2 pr;
      pr.x = widen(pq.x);
      pr.y = widen(pq.y);
      if (cA != 0.0) {
        double2 a = accA[m];
        a.x += cA * pr.x;
        a.y += cA * pr.y;
        accA[m] = a;
      }
      if (cB != 0.0) {
        double2 a = accB[m];
        a.x += cB * pr.x;
        a.y += cB * pr.y;
        accB[m] = a;
      }
    }
  }
}

template <typename T, int N, int EPI>
__global__ void __launch_bounds__(PencilsPerCta<T, N>::v * Plan<N>::TPC)
k_zi_c2c(const cpx<T>* __restrict__ spec, const cpx<T>* __restrict__ B, cpx<T>* __restrict__ qout,
         const cpx<T>* __restrict__ partner, double2* __restrict__ accA, double2* __restrict__ accB, double cA,
         double cB, long long npen, const cpx<T>* __restrict__ tw) {
  zi_c2c_body<T, N, EPI>(spec, B, qout, partner, accA, accB, cA, cB, npen, tw, (long long)blockIdx.x);
}

}  // namespace pft
