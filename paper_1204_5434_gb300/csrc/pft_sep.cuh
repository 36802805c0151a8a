// pft_sep.cuh -- the contour step of real fields as three one-dimensional Gaussian
// convolutions, one launch per contour step.
//
// The diffusion factor of Eq. 13 is separable, exp(-k^2 ds) = dx(kx) dy(ky) dz(kz), and the
// 3D DFT is the product of the 1D DFTs along the three axes, so the diffusion operator
// F^-1 D F equals Kx Ky Kz with K_a = F_a^-1 d_a F_a the periodic Gaussian convolution
// along axis a (d_a real and even, 1/n_a folded in).  Each K_a maps real fields to real
// fields and the three commute.  Two real lines along an axis ride as one complex line
// (a + i b): K_a of it is K_a a + i K_a b, since d_a is real and even -- no Hermitian
// split, no half spectrum.
//
// Alternating the order of the three factors from one step to the next puts the two x
// convolutions of consecutive steps side by side, and likewise the y and z ones:
//   plane kernel (one CTA per x-plane): Ky, Kz, x B_s, store q_s, x B_{s+1}, Kz, Ky
//   x kernel (pencils along x):         Kx, x B_s, store q_s, x B_{s+1}, Kx
// so one launch advances one contour step (the two kinds alternate) and the field between
// launches is real (4 bytes a point), read and written in place.  The march of Ns steps
// is a first plane launch (x B_1, Kz, Ky) followed by Ns launches, the last of which
// stops after its store.  FP32 propagators, ny = nz = N in {64, 128}.
#pragma once
#include "pft_plane.cuh"
#include "pft_sepp.cuh"
#include "pft_tma.cuh"

namespace pft {

template <int N> struct SepCfg {
  using PL = Plan<N>;
  static constexpr int E = PL::E, TPC = PL::TPC;
  static constexpr int R1 = Radix2<typename PL::R>::r1;
  static constexpr int LINES = N / 2;           // complex lines per phase: row pairs / column pairs
  static constexpr int THREADS = LINES * TPC;    // 512 at N = 128, 256 at N = 64
  static constexpr int BPITCH = N + 8;           // floats per B row in shared memory (bank spread)
  static constexpr int RSH = (R1 == 16) ? 4 : 3; // row-exchange swizzle shift: log2(R1)
  // shared memory: Ucol [N][N/2] float2 (column exchanges and both transposes), Urow
  // [N/2][N] float2 (row exchanges), B_s [N][BPITCH] float, twiddles [N] float2, dy, dz
  // [N] float, one mbarrier
  static constexpr size_t UCOL = (size_t)N * (N / 2) * sizeof(float2);
  static constexpr size_t UROW = (size_t)(N / 2) * N * sizeof(float2);
  static constexpr size_t BS = (size_t)N * BPITCH * sizeof(float);
  static constexpr size_t SMEM = UCOL + UROW + BS + (size_t)N * sizeof(float2) + 2 * (size_t)N * sizeof(float) + 16;
  static_assert(TPC == 8 && 32 % TPC == 0, "eight threads per line, four lines per warp");
  static_assert(N / 2 >= 16 && LINES % 32 == 0, "swizzle blocks and whole-warp column rounds");
  // Ucol: float2 of row y, column pair cc, at y (N/2) + (cc ^ 4 (y mod 4)): the column
  // phase (a warp on 32 consecutive cc of one row) and the transposed row accesses (eight
  // threads on eight consecutive floats of each of four rows y = 0..3 mod 4) are both
  // conflict-free
  __device__ static __forceinline__ int ucol(int y, int cc) { return y * (N / 2) + (cc ^ ((y & 3) << 2)); }
  __device__ static __forceinline__ int ucol_f(int y, int k) { return y * N + (k ^ ((y & 3) << 3)); }
  // Urow: position p of line L at L N + (p ^ ((p >> RSH) & 7) ^ 8 (L & 1)): the radix-R1
  // stage puts (p = R1 t + r) and the second-stage gets (p = t + 8 i) of two lines per
  // half-warp touch 16 distinct bank pairs
  __device__ static __forceinline__ int urow(int L, int p) { return L * N + (p ^ ((p >> RSH) & 7) ^ ((L & 1) << 3)); }
};

// Column exchange: position pos of column pair cc in Ucol, CTA-wide barrier.
template <int N> struct XSepCol {
  float2* u;
  int cc;
  __device__ __forceinline__ void put(int pos, float2 z) { u[SepCfg<N>::ucol(pos, cc)] = z; }
  __device__ __forceinline__ float2 get(int pos) const { return u[SepCfg<N>::ucol(pos, cc)]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Row exchange: position pos of line L in Urow; a line's threads lie in one warp.
template <int N> struct XSepRow {
  float2* u;
  int L;
  __device__ __forceinline__ void put(int pos, float2 z) { u[SepCfg<N>::urow(L, pos)] = z; }
  __device__ __forceinline__ float2 get(int pos) const { return u[SepCfg<N>::urow(L, pos)]; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// MODE 0: first launch of a march (rows of q_0 = st.in, x B_1, Kz, Ky).
// MODE 1: Ky, Kz, x B_s, store q_s, x B_{s+1}, Kz, Ky.
// MODE 2: last launch (Ky, Kz, x B_Ns, store q_Ns).
// The field plane st.spec[p] is read and written in place.  Per-axis factors:
// st.d[1] = dy, st.d[2] = dz (full length, 1/n folded in); twiddles st.tw[1] (length N).
// ADJ 1: the adjoint march of Eq. 13's steps (reverse mode): after x B_s the source of the
// step, (cA gA + cB gB) * partner, is added before the store (st.accA, st.accB hold the
// FP32 arrays gA, gB; st.partner the paired history slice; no source where partner is null).
template <int N, int MODE, int ADJ = 0>
__global__ void __launch_bounds__(SepCfg<N>::THREADS, 1) kb_sep_plane(const BatchStep* __restrict__ st, int* err) {
  using R = SepCfg<N>;
  constexpr int E = R::E, TPC = R::TPC, LINES = R::LINES, H = N / 2;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Ucol = reinterpret_cast<float2*>(smraw);
  float* Ucf = reinterpret_cast<float*>(smraw);
  float2* Urow = reinterpret_cast<float2*>(smraw + R::UCOL);
  float* Bs = reinterpret_cast<float*>(smraw + R::UCOL + R::UROW);
  float2* tws = reinterpret_cast<float2*>(smraw + R::UCOL + R::UROW + R::BS);
  float* dys = reinterpret_cast<float*>(tws + N);
  float* dzs = dys + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(dzs + N);
  const int tid = threadIdx.x;
  const int p = blockIdx.x;
  const long long pbase = (long long)p * N * N;  // float offset of the plane
  float* F = reinterpret_cast<float*>(s.spec) + pbase;
  float2* F2 = reinterpret_cast<float2*>(F);
  const float* Bg = reinterpret_cast<const float*>(s.B) + pbase;

  const int cc = tid % LINES, ct = tid / LINES;  // column phase: column pair, position
  const int L = tid / TPC, t = tid % TPC;        // row phase: line (rows L, L + N/2), position
  float2 v[E];
  // the field's column pairs straight from global memory (in flight during the set-up)
  if (MODE != 0) {
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = F2[(long long)(ct + TPC * i) * H + cc];
  }
  // B_s of the plane into shared memory, one bulk copy per row (rows padded to BPITCH)
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) mbar_arrive_expect_tx(bar, (unsigned)(N * N * sizeof(float)));
  if (tid < N) bulk_g2s(Bs + tid * R::BPITCH, Bg + (long long)tid * N, (unsigned)(N * sizeof(float)), bar);
  for (int i = tid; i < N; i += R::THREADS) {
    tws[i] = reinterpret_cast<const float2*>(s.tw[1])[i];
    dys[i] = reinterpret_cast<const float*>(s.d[1])[i];
    dzs[i] = reinterpret_cast<const float*>(s.d[2])[i];
  }
  __syncthreads();

  XSepCol<N> xc{Ucol, cc};
  XSepRow<N> xr{Urow, L};
  using RT = TwoStage<PlanX<N, E, R::R1, Radix2<typename Plan<N>::R>::r2>>;
  float2 wr[RT::NW];
  RT::load(wr, t, tws);

  if (MODE != 0) {
    // ---- Ky
    fft<float, false, N>(v, ct, tws, xc);
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], dys[ct + TPC * i]);
    fft<float, true, N>(v, ct, tws, xc);
    // transpose to the rows
#pragma unroll
    for (int i = 0; i < E; i++) Ucol[R::ucol(ct + TPC * i, cc)] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      v[i] = make_float2(Ucf[R::ucol_f(L, k)], Ucf[R::ucol_f(L + H, k)]);
    }
    // ---- Kz on the row pairs
    RT::template run<false>(v, t, wr, xr);
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], dzs[t + TPC * i]);
    RT::template run<true>(v, t, wr, xr);
  } else {
    const float* q0 = reinterpret_cast<const float*>(s.in) + pbase;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      v[i] = make_float2(q0[(long long)L * N + k], q0[(long long)(L + H) * N + k]);
    }
  }
  if (!mbar_wait(bar, 0, err, 1)) return;  // B_s has arrived

  // ---- x B_s, store q_s, x B_{s+1} (an entry without Bnext ends its march here)
  const bool more = (MODE == 1) && (s.Bnext != nullptr);
  {
    const bool same = (s.Bnext == s.B);
    const float* Bn = reinterpret_cast<const float*>(s.Bnext) + pbase;
    float* q = reinterpret_cast<float*>(s.out) + pbase;
    const bool src = ADJ && MODE != 0 && s.partner;
    const float* sp = reinterpret_cast<const float*>(s.partner) + pbase;
    const float* gA = reinterpret_cast<const float*>(s.accA) + pbase;
    const float* gB = reinterpret_cast<const float*>(s.accB) + pbase;
    const float cA = (float)s.cA, cB = (float)s.cB;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      const float ba = Bs[L * R::BPITCH + k], bb = Bs[(L + H) * R::BPITCH + k];
      v[i].x *= ba;
      v[i].y *= bb;
      if (src) {
        const long long ra = (long long)L * N + k, rb = (long long)(L + H) * N + k;
        v[i].x += (cA * gA[ra] + cB * gB[ra]) * sp[ra];
        v[i].y += (cA * gA[rb] + cB * gB[rb]) * sp[rb];
      }
      if (MODE != 0) {
        q[(long long)L * N + k] = v[i].x;
        q[(long long)(L + H) * N + k] = v[i].y;
        if (more) {
          if (same) {
            v[i].x *= ba;
            v[i].y *= bb;
          } else {
            v[i].x *= Bn[(long long)L * N + k];
            v[i].y *= Bn[(long long)(L + H) * N + k];
          }
        }
      }
    }
  }
  if (MODE == 2 || (MODE == 1 && !more)) return;

  // ---- Kz of the next step
  __syncwarp();
  RT::template run<false>(v, t, wr, xr);
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = cscale(v[i], dzs[t + TPC * i]);
  RT::template run<true>(v, t, wr, xr);
  // transpose to the column pairs (each line writes only its own two rows)
#pragma unroll
  for (int i = 0; i < E; i++) {
    const int k = t + TPC * i;
    Ucf[R::ucol_f(L, k)] = v[i].x;
    Ucf[R::ucol_f(L + H, k)] = v[i].y;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = Ucol[R::ucol(ct + TPC * i, cc)];
  __syncthreads();  // every column read precedes the exchanges' writes
  // ---- Ky of the next step, then the field back to global memory
  fft<float, false, N>(v, ct, tws, xc);
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = cscale(v[i], dys[ct + TPC * i]);
  fft<float, true, N>(v, ct, tws, xc);
#pragma unroll
  for (int i = 0; i < E; i++) F2[(long long)(ct + TPC * i) * H + cc] = v[i];
}

// The x kernel: C pencils along x per CTA (consecutive column pairs (y, z/2) of every
// x-plane), each a complex line a + i b of two real lines.
// MODE 1: Kx, x B_s, store q_s, x B_{s+1}, Kx.  MODE 2: Kx, x B_Ns, store q_Ns.
// P = NYZ^2 / 2 column pairs per x-plane (ny = nz = NYZ); st.d[0] = dx (full length,
// 1/nx folded in); twiddles st.tw[0].  B_s of the tile is copied to shared memory by
// 16-byte cp.async chunks at the start, so its latency hides behind the first Kx.
// KIND 1: complex fields -- each x-line is one complex line (P = NYZ^2 of them) and B
// multiplies as a complex factor.  XPL: the transform plan of the x-lines (elements a
// thread and radices); the CTA has C * XPL::TPC threads.
template <int NX> struct SepXAlt;  // the alternative x plan: half the elements a thread
template <> struct SepXAlt<128> { using P = PlanX<128, 8, 8, 4, 4>; };
template <> struct SepXAlt<64> { using P = PlanX<64, 4, 4, 4, 4>; };
template <int NX, class XPL> struct SepXCfg {
  static constexpr int THREADS = 16 * XPL::TPC;
  static constexpr int MINB = THREADS <= 128 ? 4 : 3;
};
template <int NX, int NYZ, int MODE, int C = 16, int KIND = 0, class XPL = Plan<NX>, int ADJ = 0>
__global__ void __launch_bounds__(SepXCfg<NX, XPL>::THREADS, SepXCfg<NX, XPL>::MINB) kb_sep_x(const BatchStep* __restrict__ st) {
  static_assert(C == 16, "sixteen lines a CTA");
  // lines per x-plane: column pairs (real) or columns (complex) of the ny = nz = NYZ plane
  constexpr long long P = KIND ? (long long)NYZ * NYZ : (long long)NYZ * NYZ / 2;
  static_assert(P % C == 0, "whole tiles");
  using PL = XPL;
  constexpr int E = PL::E, TPC = PL::TPC;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  float2* Bt = sm + NX * C;            // B_s of the tile, [x][C]
  float2* tws = Bt + NX * C;
  float* dxs = reinterpret_cast<float*>(tws + NX);
  const int c = threadIdx.x % C;
  const int t = threadIdx.x / C;
  const long long col0 = (long long)blockIdx.x * C;
  const long long col = col0 + c;
  const long long colc = col;
  float2* F2 = reinterpret_cast<float2*>(s.spec);
  float2 v[E];
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = F2[(long long)(t + TPC * i) * P + colc];
  {
    constexpr int CH = C / 2;  // 16-byte chunks per row of the tile
    const unsigned sb = (unsigned)__cvta_generic_to_shared(Bt);
    const float2* Bg = reinterpret_cast<const float2*>(s.B) + col0;
    for (int k = threadIdx.x; k < NX * CH; k += C * TPC) {
      const int xr = k / CH, ch = k % CH;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + (unsigned)((xr * C + 2 * ch) * 8)),
                   "l"(Bg + (long long)xr * P + 2 * ch)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int i = threadIdx.x; i < NX; i += C * TPC) {
    tws[i] = reinterpret_cast<const float2*>(s.tw[0])[i];
    dxs[i] = reinterpret_cast<const float*>(s.d[0])[i];
  }
  __syncthreads();  // twiddles and factors in shared memory
  XchCols<float> x{sm, C, c};
  fft<float, false, NX, PL>(v, t, tws, x);
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = cscale(v[i], dxs[t + TPC * i]);
  fft<float, true, NX, PL>(v, t, tws, x);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();  // every thread's chunks of B_s have landed
  const bool more = (MODE == 1) && (s.Bnext != nullptr);  // no Bnext: the entry's last step
  {
    const bool same = (s.Bnext == s.B);
    const float2* Bn2 = reinterpret_cast<const float2*>(s.Bnext);
    float2* q2 = reinterpret_cast<float2*>(s.out);
    const bool src = ADJ && s.partner;  // the adjoint's source (real fields): (cA gA + cB gB) partner
    const float2* sp2 = reinterpret_cast<const float2*>(s.partner);
    const float2* gA2 = reinterpret_cast<const float2*>(s.accA);
    const float2* gB2 = reinterpret_cast<const float2*>(s.accB);
    const float cA = (float)s.cA, cB = (float)s.cB;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const long long o = (long long)(t + TPC * i) * P + colc;
      const float2 b = Bt[(t + TPC * i) * C + c];
      v[i] = sepp_mul<KIND>(v[i], b);
      if (src) {
        const float2 ga = gA2[o], gb = gB2[o], pp = sp2[o];
        v[i].x += (cA * ga.x + cB * gb.x) * pp.x;
        v[i].y += (cA * ga.y + cB * gb.y) * pp.y;
      }
      q2[o] = v[i];
      if (more) v[i] = sepp_mul<KIND>(v[i], same ? b : Bn2[o]);
    }
  }
  if (!more) return;
  fft<float, false, NX, PL>(v, t, tws, x);
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = cscale(v[i], dxs[t + TPC * i]);
  fft<float, true, NX, PL>(v, t, tws, x);
#pragma unroll
  for (int i = 0; i < E; i++) F2[(long long)(t + TPC * i) * P + col] = v[i];
}

template <int NX, int C = 16> constexpr size_t sep_x_smem() {
  return 2 * (size_t)NX * C * sizeof(float2) + (size_t)NX * sizeof(float2) + (size_t)NX * sizeof(float);
}

}  // namespace pft

namespace pft {

// ----------------------------------------------------------------- complex fields
// The same march for complex (CL) fields with ny = nz = N = 64: every line is complex (no
// pairing): N column lines along y and N row lines along z per plane, 8 threads a line.
template <int N> struct SepCfgC {
  using PL = Plan<N>;
  static constexpr int E = PL::E, TPC = PL::TPC;
  static constexpr int R1 = Radix2<typename PL::R>::r1;
  static constexpr int LINES = N;
  static constexpr int THREADS = LINES * TPC;  // 512 at N = 64
  static constexpr int BPITCH = N + 8;         // complex elements per B row in shared memory
  static constexpr int RSH = (R1 == 16) ? 4 : 3;
  static constexpr size_t UCOL = (size_t)N * N * sizeof(float2);
  static constexpr size_t UROW = (size_t)N * N * sizeof(float2);
  static constexpr size_t BS = (size_t)N * BPITCH * sizeof(float2);
  static constexpr size_t SMEM = UCOL + UROW + BS + (size_t)N * sizeof(float2) + 2 * (size_t)N * sizeof(float) + 16;
  static_assert(TPC == 8 && N % 32 == 0 && N >= 32, "eight threads a line, whole-warp column rounds");
  // Ucol: element (y, z) at y N + (z ^ 8 (y mod 2)): column accesses (32 consecutive z of
  // one row) and row accesses (two rows per half-warp, eight consecutive z each) are both
  // conflict-free
  __device__ static __forceinline__ int ucol(int y, int z) { return y * N + (z ^ ((y & 1) << 3)); }
  __device__ static __forceinline__ int urow(int L, int p) { return L * N + (p ^ ((p >> RSH) & 7) ^ ((L & 1) << 3)); }
};

template <int N> struct XSepColC {
  float2* u;
  int z;
  __device__ __forceinline__ void put(int pos, float2 v) { u[SepCfgC<N>::ucol(pos, z)] = v; }
  __device__ __forceinline__ float2 get(int pos) const { return u[SepCfgC<N>::ucol(pos, z)]; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
template <int N> struct XSepRowC {
  float2* u;
  int L;
  __device__ __forceinline__ void put(int pos, float2 v) { u[SepCfgC<N>::urow(L, pos)] = v; }
  __device__ __forceinline__ float2 get(int pos) const { return u[SepCfgC<N>::urow(L, pos)]; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// MODE as kb_sep_plane (0 first launch, 1 a step -- an entry without Bnext ends there --,
// 2 the last step); complex B and q, the products complex.
template <int N, int MODE>
__global__ void __launch_bounds__(SepCfgC<N>::THREADS, 1) kb_sep_plane_c(const BatchStep* __restrict__ st, int* err) {
  using R = SepCfgC<N>;
  constexpr int E = R::E, TPC = R::TPC, LINES = R::LINES;
  const BatchStep& s = st[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Ucol = reinterpret_cast<float2*>(smraw);
  float2* Urow = reinterpret_cast<float2*>(smraw + R::UCOL);
  float2* Bs = reinterpret_cast<float2*>(smraw + R::UCOL + R::UROW);
  float2* tws = reinterpret_cast<float2*>(smraw + R::UCOL + R::UROW + R::BS);
  float* dys = reinterpret_cast<float*>(tws + N);
  float* dzs = dys + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(dzs + N);
  const int tid = threadIdx.x;
  const long long pbase = (long long)blockIdx.x * N * N;  // complex offset of the plane
  float2* F = reinterpret_cast<float2*>(s.spec) + pbase;
  const float2* Bg = reinterpret_cast<const float2*>(s.B) + pbase;
  const int cz = tid % LINES, ct = tid / LINES;  // column phase: column z, position
  const int L = tid / TPC, t = tid % TPC;        // row phase: row y = L, position
  float2 v[E];
  if (MODE != 0) {
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = F[(long long)(ct + TPC * i) * N + cz];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) mbar_arrive_expect_tx(bar, (unsigned)(N * N * sizeof(float2)));
  if (tid < N) bulk_g2s(Bs + tid * R::BPITCH, Bg + (long long)tid * N, (unsigned)(N * sizeof(float2)), bar);
  for (int i = tid; i < N; i += R::THREADS) {
    tws[i] = reinterpret_cast<const float2*>(s.tw[1])[i];
    dys[i] = reinterpret_cast<const float*>(s.d[1])[i];
    dzs[i] = reinterpret_cast<const float*>(s.d[2])[i];
  }
  __syncthreads();
  XSepColC<N> xc{Ucol, cz};
  XSepRowC<N> xr{Urow, L};
  using RT = TwoStage<PlanX<N, E, R::R1, Radix2<typename Plan<N>::R>::r2>>;
  float2 wr[RT::NW];
  RT::load(wr, t, tws);

  if (MODE != 0) {
    // ---- Ky on the columns, transpose, Kz on the rows
    fft<float, false, N>(v, ct, tws, xc);
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], dys[ct + TPC * i]);
    fft<float, true, N>(v, ct, tws, xc);
#pragma unroll
    for (int i = 0; i < E; i++) Ucol[R::ucol(ct + TPC * i, cz)] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = Ucol[R::ucol(L, t + TPC * i)];
    RT::template run<false>(v, t, wr, xr);
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = cscale(v[i], dzs[t + TPC * i]);
    RT::template run<true>(v, t, wr, xr);
  } else {
    const float2* q0 = reinterpret_cast<const float2*>(s.in) + pbase;
#pragma unroll
    for (int i = 0; i < E; i++) v[i] = q0[(long long)L * N + t + TPC * i];
  }
  if (!mbar_wait(bar, 0, err, 1)) return;

  const bool more = (MODE == 1) && (s.Bnext != nullptr);
  {
    const bool same = (s.Bnext == s.B);
    const float2* Bn = reinterpret_cast<const float2*>(s.Bnext) + pbase;
    float2* q = reinterpret_cast<float2*>(s.out) + pbase;
#pragma unroll
    for (int i = 0; i < E; i++) {
      const int k = t + TPC * i;
      const float2 b = Bs[L * R::BPITCH + k];
      v[i] = cmul(v[i], b);
      if (MODE != 0) {
        q[(long long)L * N + k] = v[i];
        if (more) v[i] = cmul(v[i], same ? b : Bn[(long long)L * N + k]);
      }
    }
  }
  if (MODE == 2 || (MODE == 1 && !more)) return;

  // ---- Kz of the next step, transpose, Ky, the field back to global memory
  __syncwarp();
  RT::template run<false>(v, t, wr, xr);
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = cscale(v[i], dzs[t + TPC * i]);
  RT::template run<true>(v, t, wr, xr);
#pragma unroll
  for (int i = 0; i < E; i++) Ucol[R::ucol(L, t + TPC * i)] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = Ucol[R::ucol(ct + TPC * i, cz)];
  __syncthreads();
  fft<float, false, N>(v, ct, tws, xc);
#pragma unroll
  for (int i = 0; i < E; i++) v[i] = cscale(v[i], dys[ct + TPC * i]);
  fft<float, true, N>(v, ct, tws, xc);
#pragma unroll
  for (int i = 0; i < E; i++) F[(long long)(ct + TPC * i) * N + cz] = v[i];
}

}  // namespace pft
