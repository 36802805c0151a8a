// pft_sepp.cuh -- the separable march on pencils: any grid, real or complex fields,
// either precision, two launches per contour step.
//
// As in pft_sep.cuh the diffusion operator of Eq. 13 is applied as Kx Ky Kz, three 1D
// periodic Gaussian convolutions (d_a real and even, 1/n_a folded in), in alternating
// order so that consecutive steps' convolutions along x (and along z) meet in one kernel:
//   z kernel:  Kz, x B_s, store q_s, x B_{s+1}, Kz     (lines along z, contiguous)
//   y kernel:  Ky                                      (lines along y, strided)
//   x kernel:  Kx, x B_s, store q_s, x B_{s+1}, Kx     (lines along x, strided)
// The march is a first z launch (x B_1, Kz) and then, for s = 1..Ns, a y launch and the x
// (s odd) or z (s even) launch that stores q_s; an entry without Bnext stops after its store
// (so members of a batch with different Ns share the launches).
// Lines: complex fields (KIND 1) transform each line; real fields (KIND 0) carry two real
// lines as one complex line a + i b -- along x and y the pair (z, z+1) (a complex element
// of the field viewed as pairs), along z the rows (y, y+1) of one x-plane.
// Arithmetic: float, double, or double-float (dd, pft_dd.cuh: an FP64 context's march on
// the FP32 pipe).  The working field between launches, the Boltzmann factors and the
// tables are in the working type; q_0 and the stored q_s are in the history's type
// (SeppHist: the working type, or FP64 for double-float).
#pragma once
#include <type_traits>

#include "pft_batch.cuh"
#include "pft_dd.cuh"

namespace pft {

template <typename T> struct SeppHist { using S = T; };
template <> struct SeppHist<dd> { using S = double; };
template <typename T> __device__ __forceinline__ T hist_in(typename SeppHist<T>::S x) {
  if constexpr (std::is_same<T, dd>::value) return dd_from_double(x); else return x;
}
template <typename T> __device__ __forceinline__ typename SeppHist<T>::S hist_out(T x) {
  if constexpr (std::is_same<T, dd>::value) return dd_to_double(x); else return x;
}
template <typename T> __device__ __forceinline__ cpx<T> hist_in_c(cpx<typename SeppHist<T>::S> z) {
  return mk<T>(hist_in<T>(z.x), hist_in<T>(z.y));
}
template <typename T> __device__ __forceinline__ cpx<typename SeppHist<T>::S> hist_out_c(cpx<T> z) {
  return mk<typename SeppHist<T>::S>(hist_out<T>(z.x), hist_out<T>(z.y));
}

// x B for one element: componentwise for real pairs, complex product for complex fields.
template <int KIND, typename Z>
__device__ __forceinline__ Z sepp_mul(Z v, Z b) {
  if constexpr (KIND == 0) {
    v.x *= b.x;
    v.y *= b.y;
    return v;
  } else {
    return cmul(v, b);
  }
}

// Strided lines (x or y): line `col` (0 <= col < nlines) starts at (col / cin) s_outer +
// col % cin and its element pos sits s_k further per step (units: complex elements of the
// field, which for real fields are the (z, z+1) pairs).  PW 0: the convolution only; PW 2:
// conv, x B_s, store q_s, then (if st.Bnext) x B_{s+1}, conv.  AX: the axis (0 x, 1 y)
// whose twiddles st.tw[AX] and factors st.d[AX] apply.
// Registers: at most 128 a thread (2 CTAs of 256 threads, 4 of 128 per SM); double-float
// (twice the registers a value in flight) at most 255.
template <typename T> constexpr int sepp_occ() { return std::is_same<T, dd>::value ? 256 : 512; }
// Transform plan: Plan<N>, except that double-float lines of 128 and 256 points hold 8
// elements a thread (radices 8, 4, 4 and 8, 8, 4): half the registers of Plan<N>'s 16, at
// the cost of one more exchange.
template <typename T, int N> struct SeppPlan { using type = Plan<N>; };
// Fused kernels whose two convolutions run as two turns of a loop instead of two unrolled
// copies: double-float (a dozen FP32 operations an FP64 one), and lines of 128 points and
// more in any precision.
template <typename T, int N> __host__ __device__ constexpr bool sepp_rolled() { return std::is_same<T, dd>::value || N >= 128; }
template <> struct SeppPlan<dd, 128> { using type = PlanX<128, 8, 8, 4, 4>; };
template <> struct SeppPlan<dd, 256> { using type = PlanX<256, 8, 8, 8, 4>; };

// Register lines (line variant 1, FP32 lines of at most 48 points): one thread holds a whole
// line, so the exchanges between Stockham stages permute a thread's own elements through a
// local array whose indices are compile-time constants once the stages are unrolled --
// registers, no shared memory, no barriers.
template <int N> struct RegPlan { static constexpr bool ok = false; };
#define PFT_REGPLAN(N_, ...) \
  template <> struct RegPlan<N_> : PlanX<N_, N_, __VA_ARGS__> { static constexpr bool ok = true; };
PFT_REGPLAN(4, 4)
PFT_REGPLAN(6, 3, 2)
PFT_REGPLAN(8, 8)
PFT_REGPLAN(12, 3, 4)
PFT_REGPLAN(16, 16)
PFT_REGPLAN(24, 3, 8)
PFT_REGPLAN(32, 4, 8)
PFT_REGPLAN(48, 3, 16)
#undef PFT_REGPLAN
inline bool sepp_reg_ok(int n) {
  return n == 4 || n == 6 || n == 8 || n == 12 || n == 16 || n == 24 || n == 32 || n == 48;
}
template <typename T, int N> struct XchReg {
  cpx<T> b[N];
  __device__ __forceinline__ void put(int pos, cpx<T> z) { b[pos] = z; }
  __device__ __forceinline__ cpx<T> get(int pos) const { return b[pos]; }
  __device__ __forceinline__ void sync() const {}
};

// Wide lines (line variant 3, FP32 lines of 32, 48 and 64 points): twice the elements a
// thread of Plan<N>, in another radix order (16 2, 3 8 2, 16 4): fewer threads a line and
// fewer exchanges at 32 and 64 points, more registers.
template <int N> struct WidePlan { static constexpr bool ok = false; };
#define PFT_WIDEPLAN(N_, E_, ...) \
  template <> struct WidePlan<N_> : PlanX<N_, E_, __VA_ARGS__> { static constexpr bool ok = true; };
PFT_WIDEPLAN(32, 16, 16, 2)
PFT_WIDEPLAN(48, 24, 3, 8, 2)
PFT_WIDEPLAN(64, 16, 16, 4)
#undef PFT_WIDEPLAN
// Lengths of line variants 2 and 3.
inline bool sepp_wide_ok(int n) { return n == 32 || n == 48 || n == 64; }

// FP32 kernels that carry B_s (x lines and z lines with PW 2, not register lines) stage it in
// shared memory by cp.async at the start.
template <typename T, int PW, int AX, int V> __host__ __device__ constexpr bool sepp_pre_smem() {
  return std::is_same<T, float>::value && PW == 2 && AX != 1 && V != 1;
}

// Line kernel configuration of variant V: plan, lines per CTA, threads.  Variants 0 (Plan<N>,
// 16 FP32 lines a CTA), 1 (register lines), 2 (Plan<N>, 32 lines a CTA: twice the CTA, each
// row of a tile one 256-byte run), 3 (WidePlan<N>, 32 lines a CTA); the autotuners choose.
template <typename T, int N, int V> struct SeppLineCfg {
  using PL = typename SeppPlan<T, N>::type;
  static constexpr int C = Tile<T>::C;
  static constexpr int THREADS = C * PL::TPC;
  static constexpr int MINB = (sepp_occ<T>() / THREADS) > 0 ? sepp_occ<T>() / THREADS : 1;
};
template <typename T, int N> struct SeppLineCfg<T, N, 2> {
  using PL = typename SeppPlan<T, N>::type;
  static constexpr int C = 32;
  static constexpr int THREADS = C * PL::TPC;
  static constexpr int MINB = (sepp_occ<T>() / THREADS) > 0 ? sepp_occ<T>() / THREADS : 1;
};
template <typename T, int N> struct SeppLineCfg<T, N, 3> {
  using PL = WidePlan<N>;
  static constexpr int C = 32;
  static constexpr int THREADS = C * PL::TPC;
  static constexpr int MINB = (384 / THREADS) > 0 ? 384 / THREADS : 1;  // up to 170 registers
};
template <typename T, int N> struct SeppLineCfg<T, N, 1> {
  using PL = RegPlan<N>;
  static constexpr int C = 64;  // lines (threads) per CTA
  static constexpr int THREADS = 64;
  static constexpr int MINB = 4;  // up to 255 registers a thread (a 48-point complex line is 96)
};
// Offsets are 32-bit: a field holds fewer than 2^31 complex elements.
template <typename T, int N, int KIND, int PW, int AX, int V = 0>
__global__ void __launch_bounds__(SeppLineCfg<T, N, V>::THREADS, SeppLineCfg<T, N, V>::MINB)
kb_sepp_line(const BatchStep* __restrict__ st, int nlines, int cin, int s_outer, int s_k) {
  using Z = cpx<T>;
  using PL = typename SeppLineCfg<T, N, V>::PL;
  constexpr int E = PL::E, TPC = PL::TPC, C = SeppLineCfg<T, N, V>::C;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  Z* sm = reinterpret_cast<Z*>(smraw);
  const int c = threadIdx.x % C;
  const int t = (V == 1) ? 0 : threadIdx.x / C;  // register lines: one thread a line
  const int col = blockIdx.x * C + c;
  const bool valid = col < nlines;
  const int colc = valid ? col : 0;
  const int base = (colc / cin) * s_outer + (colc % cin) + t * s_k;  // element t of the line
  const int step = TPC * s_k;
  const Z* tw = reinterpret_cast<const Z*>(s.tw[AX]);
  const T* d = reinterpret_cast<const T*>(s.d[AX]);
  Z* F = reinterpret_cast<Z*>(s.spec);
  Z v[E];
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = F[base + i * step];
  // double-float lines of 128 and 256 points (registers to spare under the 255 cap): B_s of
  // the line first, so that its latency overlaps the transforms instead of stalling the
  // multiply after them (at 64 points the extra registers cost more occupancy than it saves)
  constexpr bool kPreB = std::is_same<T, dd>::value && PW == 2 && N >= 128;
  Z bpre[kPreB ? E : 1];
  if constexpr (kPreB) {
    const Z* B = reinterpret_cast<const Z*>(s.B);
#pragma unroll
    for (int i = 0; i < E; i++) bpre[i] = B[base + i * step];
  }
  // FP32 x lines: B_s of the tile (N rows of C consecutive lines, after the exchange area)
  // copied to shared memory by 16-byte cp.async now, so that its latency hides behind the
  // first convolution (the lines sit at the 128-register cap: no room to hold it in
  // registers); whole tiles with an even row pitch (16-byte chunks) only
  constexpr bool kPreS = sepp_pre_smem<T, PW, AX, V>();
  const bool pre = kPreS && (blockIdx.x + 1) * C <= nlines && (s_k % 2) == 0;
  Z* Bt = sm + N * C;
  if constexpr (kPreS) {
    if (pre) {
      constexpr int CH = C / 2;  // 16-byte chunks a tile row
      const unsigned sb = (unsigned)__cvta_generic_to_shared(Bt);
      const Z* Bg = reinterpret_cast<const Z*>(s.B) + blockIdx.x * C;
      for (int k = threadIdx.x; k < N * CH; k += SeppLineCfg<T, N, V>::THREADS) {
        const int xr = k / CH, ch = k % CH;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + (unsigned)((xr * C + 2 * ch) * 8)),
                     "l"(Bg + (long long)xr * s_k + 2 * ch)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  auto make_x = [&]() {
    if constexpr (V == 1) {
      return XchReg<T, N>{};
    } else {
      return XchCols<T>{sm, C, c};
    }
  };
  auto x = make_x();
  auto conv = [&]() {  // K_a: forward transform, x d_a, inverse transform
    fft<T, false, N, PL>(v, t, tw, x);
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], d[t + TPC * i]);
    fft<T, true, N, PL>(v, t, tw, x);
  };
  auto bsteps = [&]() -> bool {  // x B_s, store q_s, x B_{s+1}; false at the chain's end
    const Z* B = reinterpret_cast<const Z*>(s.B);
    const Z* Bn = reinterpret_cast<const Z*>(s.Bnext);
    cpx<typename SeppHist<T>::S>* q = reinterpret_cast<cpx<typename SeppHist<T>::S>*>(s.out);
    const bool more = (Bn != nullptr);
    const bool same = (Bn == B);
    if constexpr (kPreS) {
      if (pre) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();  // every thread's chunks of the tile have landed
      }
    }
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int o = base + i * step;
      Z b;
      if constexpr (kPreB) b = bpre[i];
      else if (kPreS && pre) b = Bt[(t + TPC * i) * C + c];
      else b = B[o];
      v[i] = sepp_mul<KIND>(v[i], b);
      if (valid) q[o] = hist_out_c<T>(v[i]);
      if (more) v[i] = sepp_mul<KIND>(v[i], same ? b : Bn[o]);
    }
    return more;
  };
  if constexpr (sepp_rolled<T, N>() && PW == 2) {
    // the two convolutions as two turns of one loop: one copy of the unrolled transforms,
    // which twice over overflow the instruction cache
#pragma unroll 1
    for (int r = 0; r < 2; r++) {
      conv();
      if (r == 0 && !bsteps()) return;
    }
  } else {
    conv();
    if (PW == 2) {
      if (!bsteps()) return;
      conv();
    }
  }
  if (valid) {
#pragma unroll
    for (int i = 0; i < E; i++) F[base + i * step] = v[i];
  }
}

// Lines along z (contiguous).  Complex fields: line l is the pencil at l N.  Real fields:
// line l carries the rows 2l and 2l+1 (floats at 2l N + pos and (2l+1) N + pos).
// PW 1: the first launch of a march (x B_1 on q_0 = st.in, then Kz); PW 2: Kz, x B_s,
// store q_s, then (if st.Bnext) x B_{s+1}, Kz.
template <typename T, int N> struct SeppZCfg {
  using PL = typename SeppPlan<T, N>::type;
  // pencils per CTA as PencilsPerCta, for this plan's threads per pencil
  static constexpr int unit = 32 / PL::TPC;
  // double-float at 128 and 256 points: 128-thread CTAs (150 to 200 registers a thread: two
  // or three CTAs an SM, not one)
  static constexpr int by_threads = ((std::is_same<T, dd>::value && N >= 128) ? 128 : 256) / PL::TPC;
  static constexpr int by_smem = (48 * 1024) / (pencil_ld<T>(N) * (int)sizeof(cpx<T>));
  static constexpr int raw = by_threads < by_smem ? by_threads : by_smem;
  static constexpr int P = raw >= unit ? raw - raw % unit : unit;
  static constexpr int THREADS = P * PL::TPC;
  static constexpr int MINB = (sepp_occ<T>() / THREADS) > 0 ? sepp_occ<T>() / THREADS : 1;
};
template <typename T, int N, int KIND, int PW>
__global__ void __launch_bounds__(SeppZCfg<T, N>::THREADS, SeppZCfg<T, N>::MINB)
kb_sepp_z(const BatchStep* __restrict__ st, long long nlines) {
  using Z = cpx<T>;
  using PL = typename SeppZCfg<T, N>::PL;
  constexpr int E = PL::E, TPC = PL::TPC, P = SeppZCfg<T, N>::P, LD = pencil_ld<T>(N);
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = threadIdx.x % TPC;
  const int p = threadIdx.x / TPC;
  const long long l = (long long)blockIdx.x * P + p;
  const bool valid = l < nlines;
  const long long lc = valid ? l : 0;
  XchPencil<T> x{reinterpret_cast<Z*>(smraw) + p * LD};
  const Z* tw = reinterpret_cast<const Z*>(s.tw[2]);
  const T* d = reinterpret_cast<const T*>(s.d[2]);
  // element pos of the line: complex index lc N + pos, or the floats ra + pos, rb + pos
  const long long ra = 2 * lc * N, rb = ra + N;
  auto ld = [&](const void* a, int pos) -> Z {
    if constexpr (KIND == 1) {
      return reinterpret_cast<const Z*>(a)[lc * N + pos];
    } else {
      const T* f = reinterpret_cast<const T*>(a);
      return mk<T>(f[ra + pos], f[rb + pos]);
    }
  };
  auto stz = [&](void* a, int pos, Z z) {
    if constexpr (KIND == 1) {
      reinterpret_cast<Z*>(a)[lc * N + pos] = z;
    } else {
      T* f = reinterpret_cast<T*>(a);
      f[ra + pos] = z.x;
      f[rb + pos] = z.y;
    }
  };
  // q_0 and q_s: the history's type
  using HS = typename SeppHist<T>::S;
  auto ldh = [&](const void* a, int pos) -> Z {
    if constexpr (KIND == 1) {
      return hist_in_c<T>(reinterpret_cast<const cpx<HS>*>(a)[lc * N + pos]);
    } else {
      const HS* f = reinterpret_cast<const HS*>(a);
      return mk<T>(hist_in<T>(f[ra + pos]), hist_in<T>(f[rb + pos]));
    }
  };
  auto sth = [&](void* a, int pos, Z z) {
    if constexpr (KIND == 1) {
      reinterpret_cast<cpx<HS>*>(a)[lc * N + pos] = hist_out_c<T>(z);
    } else {
      HS* f = reinterpret_cast<HS*>(a);
      f[ra + pos] = hist_out<T>(z.x);
      f[rb + pos] = hist_out<T>(z.y);
    }
  };
  Z v[E];
  // double-float at 128 and 256 points: B_s first, as in the line kernel
  constexpr bool kPreB = std::is_same<T, dd>::value && N >= 128 && PW == 2;
  Z bpre[kPreB ? E : 1];
  // FP32: B_s of the CTA's P lines -- one contiguous run of P N 8-byte elements, complex
  // (KIND 1) or the float row pairs (KIND 0) -- copied to shared memory after the exchange
  // area by 16-byte cp.async at the start (whole tiles only)
  constexpr bool kPreS = sepp_pre_smem<T, PW, 2, 0>();
  const long long l0 = (long long)blockIdx.x * P;
  const bool pre = kPreS && l0 + P <= nlines;
  Z* Bt = reinterpret_cast<Z*>(smraw) + P * LD;
  if constexpr (kPreS) {
    if (pre) {
      const unsigned sb = (unsigned)__cvta_generic_to_shared(Bt);
      const char* Bg = reinterpret_cast<const char*>(s.B) + l0 * N * 8;
      for (int k = threadIdx.x; k < P * N / 2; k += SeppZCfg<T, N>::THREADS)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + (unsigned)(k * 16)),
                     "l"(Bg + (long long)k * 16)
                     : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  // B_s at position pos of this thread's line from the staged tile
  auto ldbt = [&](int pos) -> Z {
    if constexpr (KIND == 1) {
      return Bt[p * N + pos];
    } else {
      const T* f = reinterpret_cast<const T*>(Bt) + 2 * p * N;
      return mk<T>(f[pos], f[N + pos]);
    }
  };
  auto conv = [&]() {  // Kz: forward transform, x d_z, inverse transform
    fft<T, false, N, PL>(v, t, tw, x);
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], d[t + TPC * i]);
    fft<T, true, N, PL>(v, t, tw, x);
  };
  auto bsteps = [&]() -> bool {  // x B_s, store q_s, x B_{s+1}; false at the chain's end
    const bool more = (s.Bnext != nullptr);
    const bool same = (s.Bnext == s.B);
    if constexpr (kPreS) {
      if (pre) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();  // every thread's chunks of the tile have landed
      }
    }
#pragma unroll
    for (int i = 0; i < E; i++) {
      Z b;
      if constexpr (kPreB) b = bpre[i];
      else if (kPreS && pre) b = ldbt(t + TPC * i);
      else b = ld(s.B, t + TPC * i);
      v[i] = sepp_mul<KIND>(v[i], b);
      if (valid) sth(s.out, t + TPC * i, v[i]);
      if (more) v[i] = sepp_mul<KIND>(v[i], same ? b : ld(s.Bnext, t + TPC * i));
    }
    if (!more) return false;
    if (n_stages<PL>() > 1) __syncwarp();
    return true;
  };
  if (PW == 1) {
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = sepp_mul<KIND>(ldh(s.in, t + TPC * i), ld(s.B, t + TPC * i));
    conv();
  } else {
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = ld(s.spec, t + TPC * i);
    if constexpr (kPreB) {
#pragma unroll
      for (int i = 0; i < E; i++) bpre[i] = ld(s.B, t + TPC * i);
    }
    if constexpr (sepp_rolled<T, N>()) {
      // the two convolutions as two turns of one loop (one copy of the code)
#pragma unroll 1
      for (int r = 0; r < 2; r++) {
        conv();
        if (r == 0 && !bsteps()) return;
      }
    } else {
      conv();
      if (!bsteps()) return;
      conv();
    }
  }
  if (valid) {
#pragma unroll
    for (int i = 0; i < E; i++) stz(s.spec, t + TPC * i, v[i]);
  }
}

}  // namespace pft

namespace pft {

// ------------------------------------------------------------------ launches
template <typename T, int N, int KIND, int PW, int AX, int V>
cudaError_t sepp_line_v(const BatchStep* st, long long nlines, long long cin, long long s_outer, long long s_k,
                        int members, cudaStream_t sm) {
  using CF = SeppLineCfg<T, N, V>;
  constexpr int C = CF::C;
  const dim3 grid((unsigned)((nlines + C - 1) / C), (unsigned)members);
  // the exchange area, and the staged B_s tile after it
  constexpr size_t smem = V == 1 ? 0 : (size_t)N * C * sizeof(cpx<T>) * (sepp_pre_smem<T, PW, AX, V>() ? 2 : 1);
  auto kern = kb_sepp_line<T, N, KIND, PW, AX, V>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, CF::THREADS, smem, sm>>>(st, (int)nlines, (int)cin, (int)s_outer, (int)s_k);
  return cudaGetLastError();
}
// lv 1: register lines where the length has a register plan; lv 2: 32-line tiles of Plan<N>;
// lv 3: 32-line tiles of WidePlan<N> at 32, 48 and 64 points; FP32 only; variant 0 otherwise
template <typename T, int N, int KIND, int PW, int AX>
cudaError_t sepp_line_n(const BatchStep* st, long long nlines, long long cin, long long s_outer, long long s_k,
                        int members, cudaStream_t sm, int lv) {
  if constexpr (std::is_same<T, float>::value && RegPlan<N>::ok) {
    if (lv == 1) return sepp_line_v<T, N, KIND, PW, AX, 1>(st, nlines, cin, s_outer, s_k, members, sm);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (lv == 2) return sepp_line_v<T, N, KIND, PW, AX, 2>(st, nlines, cin, s_outer, s_k, members, sm);
  }
  if constexpr (std::is_same<T, float>::value && WidePlan<N>::ok) {
    if (lv == 3) return sepp_line_v<T, N, KIND, PW, AX, 3>(st, nlines, cin, s_outer, s_k, members, sm);
  }
  return sepp_line_v<T, N, KIND, PW, AX, 0>(st, nlines, cin, s_outer, s_k, members, sm);
}

template <typename T, int N, int KIND, int PW>
cudaError_t sepp_z_n(const BatchStep* st, long long nlines, int members, cudaStream_t sm) {
  constexpr int P = SeppZCfg<T, N>::P;
  const dim3 grid((unsigned)((nlines + P - 1) / P), (unsigned)members);
  // the pencil exchange area, and the staged B_s tile after it
  constexpr size_t smem = (size_t)P * pencil_ld<T>(N) * sizeof(cpx<T>) +
                          (sepp_pre_smem<T, PW, 2, 0>() ? (size_t)P * N * sizeof(cpx<T>) : 0);
  auto kern = kb_sepp_z<T, N, KIND, PW>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, SeppZCfg<T, N>::THREADS, smem, sm>>>(st, nlines);
  return cudaGetLastError();
}

#define PFT_SEPP_CASE(NV, ...) \
  case NV: {                   \
    constexpr int N = NV;      \
    __VA_ARGS__;               \
  } break;
#define PFT_SEPP_AXIS(n, ...)                                                                                        \
  switch (n) {                                                                                                       \
    PFT_SEPP_CASE(4, __VA_ARGS__) PFT_SEPP_CASE(6, __VA_ARGS__) PFT_SEPP_CASE(8, __VA_ARGS__)                        \
    PFT_SEPP_CASE(12, __VA_ARGS__) PFT_SEPP_CASE(16, __VA_ARGS__) PFT_SEPP_CASE(24, __VA_ARGS__)                     \
    PFT_SEPP_CASE(32, __VA_ARGS__) PFT_SEPP_CASE(48, __VA_ARGS__) PFT_SEPP_CASE(64, __VA_ARGS__)                     \
    PFT_SEPP_CASE(96, __VA_ARGS__) PFT_SEPP_CASE(128, __VA_ARGS__) PFT_SEPP_CASE(192, __VA_ARGS__)                   \
    PFT_SEPP_CASE(256, __VA_ARGS__)                                                                                  \
    default: return cudaErrorInvalidValue;                                                                           \
  }

template <typename T, int KIND>
cudaError_t sepp_launch_k(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm) {
  const long long nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long nzz = KIND == 0 ? nz / 2 : nz;  // complex elements per row
  cudaError_t e = cudaSuccess;
  if (j == 0) {  // x B_1, Kz
    const long long nl = KIND == 0 ? nx * ny / 2 : nx * ny;
    PFT_SEPP_AXIS(g.n[2], e = (sepp_z_n<T, N, KIND, 1>(ss, nl, members, sm)));
    return e;
  }
  // Ky on the lines (x, z element) along y
  PFT_SEPP_AXIS(g.n[1], e = (sepp_line_n<T, N, KIND, 0, 1>(ss, nx * nzz, nzz, ny * nzz, nzz, members, sm, g.lv)));
  if (e != cudaSuccess) return e;
  if (j & 1) {  // Kx, x B_j, store q_j, x B_{j+1}, Kx
    PFT_SEPP_AXIS(g.n[0], e = (sepp_line_n<T, N, KIND, 2, 0>(ss, ny * nzz, ny * nzz, 0, ny * nzz, members, sm, g.lv)));
  } else {      // Kz, x B_j, store q_j, x B_{j+1}, Kz
    const long long nl = KIND == 0 ? nx * ny / 2 : nx * ny;
    PFT_SEPP_AXIS(g.n[2], e = (sepp_z_n<T, N, KIND, 2>(ss, nl, members, sm)));
  }
  return e;
}

template <typename T>
cudaError_t sepp_launch_t(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm) {
  return g.kind == 0 ? sepp_launch_k<T, 0>(g, ss, j, members, sm) : sepp_launch_k<T, 1>(g, ss, j, members, sm);
}

#undef PFT_SEPP_AXIS
#undef PFT_SEPP_CASE

}  // namespace pft
