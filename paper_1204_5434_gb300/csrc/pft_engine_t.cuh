// pft_engine_t.cuh -- EngineT<T>: launch sequences of one system in working
// precision T.  Included once per precision (pft_engine_f32.cu, pft_engine_f64.cu).
#pragma once
#include <math.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <type_traits>

#include "pft_engine_impl.cuh"
#include "pft_batch.cuh"
#include "pft_plane_ext.cuh"
#include "pft_sep.cuh"

namespace pft {

#define PFT_CASE(NV, ...) \
  case NV: {              \
    constexpr int N = NV; \
    __VA_ARGS__;          \
  } break;
// FFT lengths of a grid axis
#define PFT_DISPATCH_AXIS(n, ...)                                                                                  \
  switch (n) {                                                                                                     \
    PFT_CASE(4, __VA_ARGS__) PFT_CASE(6, __VA_ARGS__) PFT_CASE(8, __VA_ARGS__) PFT_CASE(12, __VA_ARGS__)           \
    PFT_CASE(16, __VA_ARGS__) PFT_CASE(24, __VA_ARGS__) PFT_CASE(32, __VA_ARGS__) PFT_CASE(48, __VA_ARGS__)        \
    PFT_CASE(64, __VA_ARGS__) PFT_CASE(96, __VA_ARGS__) PFT_CASE(128, __VA_ARGS__) PFT_CASE(192, __VA_ARGS__)      \
    PFT_CASE(256, __VA_ARGS__)                                                                                     \
    default: return cudaErrorInvalidValue;                                                                         \
  }
// half lengths nz/2 of the real-to-complex z transform
#define PFT_DISPATCH_HALF(n, ...)                                                                                  \
  switch (n) {                                                                                                     \
    PFT_CASE(2, __VA_ARGS__) PFT_CASE(3, __VA_ARGS__) PFT_CASE(4, __VA_ARGS__) PFT_CASE(6, __VA_ARGS__)            \
    PFT_CASE(8, __VA_ARGS__) PFT_CASE(12, __VA_ARGS__) PFT_CASE(16, __VA_ARGS__) PFT_CASE(24, __VA_ARGS__)         \
    PFT_CASE(32, __VA_ARGS__) PFT_CASE(48, __VA_ARGS__) PFT_CASE(64, __VA_ARGS__) PFT_CASE(96, __VA_ARGS__)        \
    PFT_CASE(128, __VA_ARGS__)                                                                                     \
    default: return cudaErrorInvalidValue;                                                                         \
  }

// Composite Simpson weights (in units of ds) of the slices n0..n1, added into w[n0..n1]:
// 1/3, 4/3, 1/3 on each pair of intervals; with an odd interval count of at least three
// the last three intervals take Simpson's 3/8 rule (3/8, 9/8, 9/8, 3/8); a block of one
// interval takes the trapezoid rule.  Exact for cubics, the order of the 4th-order
// scheme of Eq. 13.
inline void simpson_block(int n0, int n1, double* w) {
  const int len = n1 - n0;
  if (len <= 0) return;
  if (len == 1) {
    w[n0] += 0.5;
    w[n1] += 0.5;
    return;
  }
  const int pairs_end = (len % 2 == 0) ? n1 : n1 - 3;
  for (int a = n0; a < pairs_end; a += 2) {
    w[a] += 1.0 / 3.0;
    w[a + 1] += 4.0 / 3.0;
    w[a + 2] += 1.0 / 3.0;
  }
  if (len % 2 == 1) {
    const double e[4] = {3.0 / 8.0, 9.0 / 8.0, 9.0 / 8.0, 3.0 / 8.0};
    for (int j = 0; j < 4; j++) w[pairs_end + j] += e[j];
  }
}

// batched pass launches cover every compiled size
#define PFT_BATCH_AXIS PFT_DISPATCH_AXIS
#define PFT_BATCH_HALF PFT_DISPATCH_HALF

// Quadrature weights of the contour integrals (Eq. 8): trapezoid rule on each block.
inline void trapezoid_weight(int n, int Ns, int NsA, double* cA, double* cB) {
  *cA = 0.0;
  *cB = 0.0;
  if (NsA > 0 && n <= NsA) *cA = (n == 0 || n == NsA) ? 0.5 : 1.0;
  if (NsA < Ns && n >= NsA) *cB = (n == NsA || n == Ns) ? 0.5 : 1.0;
}

template <typename T>
class EngineT : public Engine {
 public:
  using Z = cpx<T>;

  size_t elem_bytes() const override { return sizeof(T); }
  bool plane_applies(const CtxData& c) const override { return plane_supported(c); }
  bool sep_applies(const CtxData& c) const override { return sep_supported(c); }
  bool sepp_applies(const CtxData& c) const override { return sepp_supported(c); }
  bool dd_applies(const CtxData& c) const override { return dd_supported(c); }
  bool sepp_reg_applies(const CtxData& c) const override { return sepp_reg_supported(c); }
  bool sepp_lv_applies(const CtxData& c, int lv) const override { return sepp_lv_supported(c, lv); }

  // ------------------------------------------------------------------ tables
  cudaError_t upload_tables(CtxData& c) override {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int nzc = (c.kind == PFT_SCFT_REAL) ? nz / 2 + 1 : nz;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t off = 0;
    const int twn[4] = {nx, ny, nz, nz / 2};
    for (int a = 0; a < 4; a++) {
      c.tw_off[a] = off;
      off = al(off + sizeof(Z) * (size_t)twn[a]);
    }
    const int dn[3] = {nx, ny, nzc};
    for (int a = 0; a < 3; a++) {
      c.d_off[a] = off;
      off = al(off + sizeof(T) * (size_t)dn[a]);
    }
    for (int a = 0; a < 3; a++) {
      c.g_off[a] = off;
      off = al(off + sizeof(double) * (size_t)dn[a]);
    }
    for (int a = 0; a < 3; a++) {
      c.e_off[a] = off;
      off = al(off + sizeof(double) * (size_t)dn[a]);
    }
    // half-step diffusion tables exp(-k^2 ds/2) of the 4th-order scheme
    for (int a = 0; a < 3; a++) {
      c.dh_off[a] = off;
      off = al(off + sizeof(T) * (size_t)dn[a]);
    }
    // per-axis Gaussian factors of the separable march, full axis, 1/n_a folded in
    for (int a = 0; a < 3; a++) {
      c.sd_off[a] = off;
      off = al(off + sizeof(T) * (size_t)c.n[a]);
    }
    // FP64 twiddles of the full x, y, z lengths (the transforms of the semi-implicit step)
    for (int a = 0; a < 3; a++) {
      c.t64_off[a] = off;
      off = al(off + sizeof(double2) * (size_t)twn[a]);
    }
    if (!c.tables) {
      cudaError_t e = cudaMalloc(&c.tables, off);
      if (e != cudaSuccess) return e;
      c.tables_bytes = off;
      c.bytes += off;
    }
    std::vector<unsigned char> h(off, 0);
    for (int a = 0; a < 4; a++) {
      Z* tw = reinterpret_cast<Z*>(h.data() + c.tw_off[a]);
      for (int m = 0; m < twn[a]; m++) {
        const double ang = -2.0 * M_PI * (double)m / (double)twn[a];
        tw[m] = mk<T>((T)cos(ang), (T)sin(ang));
      }
    }
    for (int a = 0; a < 3; a++) {
      double2* tw = reinterpret_cast<double2*>(h.data() + c.t64_off[a]);
      for (int m = 0; m < twn[a]; m++) {
        const double ang = -2.0 * M_PI * (double)m / (double)twn[a];
        tw[m] = make_double2(cos(ang), sin(ang));
      }
    }
    const double Md = (double)c.M;
    for (int a = 0; a < 3; a++) {
      const int na = c.n[a];
      T* d = reinterpret_cast<T*>(h.data() + c.d_off[a]);
      double* g = reinterpret_cast<double*>(h.data() + c.g_off[a]);
      for (int m = 0; m < dn[a]; m++) {
        const int mm = (m <= na / 2) ? m : m - na;
        const double k = 2.0 * M_PI * (double)mm / c.L[a];
        double dval = exp(-k * k * c.ds);
        double hval = exp(-k * k * c.ds * 0.5);
        if (a == 0) {  // inverse-transform normalisation 1/M folded into D
          dval /= Md;
          hval /= Md;
        }
        d[m] = (T)dval;
        reinterpret_cast<T*>(h.data() + c.dh_off[a])[m] = (T)hval;
        g[m] = k * k;
        reinterpret_cast<double*>(h.data() + c.e_off[a])[m] = exp(-k * k * c.ds);
      }
      T* sd = reinterpret_cast<T*>(h.data() + c.sd_off[a]);
      for (int m = 0; m < na; m++) {
        const int mm = (m <= na / 2) ? m : m - na;
        const double k = 2.0 * M_PI * (double)mm / c.L[a];
        sd[m] = (T)(exp(-k * k * c.ds) / (double)na);
      }
    }
    return cudaMemcpyAsync(c.tables, h.data(), off, cudaMemcpyHostToDevice, c.stream);
  }

  cudaError_t fill_ones(CtxData& c, void* dst) override {
    const int blocks = c.npart;
    if (c.kind == PFT_SCFT_REAL) {
      k_fill_one<T><<<blocks, PW_THREADS, 0, c.stream>>>(reinterpret_cast<T*>(dst), c.M);
    } else {
      k_fill_one<Z><<<blocks, PW_THREADS, 0, c.stream>>>(reinterpret_cast<Z*>(dst), c.M);
    }
    return cudaGetLastError();
  }

  // ---------------------------------------------------------------- a1: fields
  cudaError_t prepare_fields(CtxData& c) override {
    mark(c, KK_PREPARE);
    if (c.edw) {
      if (c.kind == PFT_SCFT_REAL) {
        k_prepare_edw_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)c.wp, (T*)c.BA, c.ds, c.bC, c.M,
                                                                    c.partials);
      } else {
        k_prepare_edw_cplx<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const double2*)c.wp, (Z*)c.BA, c.ds, c.bC, c.M,
                                                                    c.partials);
      }
    } else if (c.kind == PFT_SCFT_REAL) {
      k_prepare_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>(
          (const double*)c.wp, (const double*)c.wm, (T*)c.BA, (T*)c.BB, c.ds, c.chiN, c.M, c.partials);
    } else {
      k_prepare_cplx<T><<<c.npart, PW_THREADS, 0, c.stream>>>(
          (const double2*)c.wp, (const double2*)c.wm, (Z*)c.BA, (Z*)c.BB, c.ds, c.chiN, c.M, c.partials);
    }
    k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_FIELD);
    return half_boltz(c);
  }

  // quarter-step factors exp(-w ds/4) of the 4th-order scheme (nothing for SPLIT2)
  cudaError_t half_boltz(CtxData& c) {
    if (c.scheme != 1) return cudaGetLastError();
    if (c.kind == PFT_SCFT_REAL) {
      k_half_boltz_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)c.wp, (const double*)c.wm, (T*)c.BAh,
                                                                 (T*)c.BBh, 0.5 * c.ds, c.M);
    } else {
      k_half_boltz_cplx<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const double2*)c.wp, (const double2*)c.wm, (Z*)c.BAh,
                                                                 (Z*)c.BBh, 0.5 * c.ds, c.M);
    }
    return cudaGetLastError();
  }

  // ------------------------------------------------------- one contour step
  // out = B * F^-1[ D F[ B * in ] ]; epi 1 also accumulates the density sums.
  cudaError_t contour_step(CtxData& c, const void* in, const void* B, void* out, int epi, const void* partner,
                           double cA, double cB) {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const Z* twx = tab<Z>(c, c.tw_off[0]);
    const Z* twy = tab<Z>(c, c.tw_off[1]);
    const Z* twz = tab<Z>(c, c.tw_off[2]);
    const Z* twh = tab<Z>(c, c.tw_off[3]);
    const T* dx = tab<T>(c, c.d_off[0]);
    const T* dy = tab<T>(c, c.d_off[1]);
    const T* dz = tab<T>(c, c.d_off[2]);
    Z* spec = (Z*)c.spec;
    const long long npen = (long long)nx * ny;
    const long long nzc = c.nzh;
    cudaError_t e;
    mark(c, KK_Z_FWD);
    if (c.kind == PFT_SCFT_REAL) {
      PFT_DISPATCH_HALF(nz / 2, e = launch_zf_r2c<N>(c, (const T*)in, (const T*)B, spec, npen, twh, twz));
    } else {
      PFT_DISPATCH_AXIS(nz, e = launch_zf_c2c<N>(c, (const Z*)in, (const Z*)B, spec, npen, twz));
    }
    if (e != cudaSuccess) return e;
    mark(c, KK_Y_FWD);
    PFT_DISPATCH_AXIS(ny, e = launch_strided<N, 0>(c, spec, nx * nzc, nzc, ny * nzc, nzc, twy, dx, dy, dz, (int)nzc));
    if (e != cudaSuccess) return e;
    mark(c, KK_X_FUSED);
    PFT_DISPATCH_AXIS(nx, e = launch_strided<N, 2>(c, spec, ny * nzc, ny * nzc, 0, ny * nzc, twx, dx, dy, dz, (int)nzc));
    if (e != cudaSuccess) return e;
    mark(c, KK_Y_INV);
    PFT_DISPATCH_AXIS(ny, e = launch_strided<N, 1>(c, spec, nx * nzc, nzc, ny * nzc, nzc, twy, dx, dy, dz, (int)nzc));
    if (e != cudaSuccess) return e;
    mark(c, epi == 0 ? KK_Z_INV_FWD : KK_Z_INV_BWD);
    if (c.kind == PFT_SCFT_REAL) {
      if (epi == 0) {
        PFT_DISPATCH_HALF(nz / 2, e = launch_zi_c2r<N, 0>(c, spec, (const T*)B, (T*)out, nullptr, nullptr, nullptr,
                                                          0.0, 0.0, npen, twh, twz));
      } else {
        PFT_DISPATCH_HALF(nz / 2, e = launch_zi_c2r<N, 1>(c, spec, (const T*)B, (T*)out, (const T*)partner,
                                                          (double*)c.accA, (double*)c.accB, cA, cB, npen, twh, twz));
      }
    } else {
      if (epi == 0) {
        PFT_DISPATCH_AXIS(nz, e = launch_zi_c2c<N, 0>(c, spec, (const Z*)B, (Z*)out, nullptr, nullptr, nullptr, 0.0,
                                                      0.0, npen, twz));
      } else {
        PFT_DISPATCH_AXIS(nz, e = launch_zi_c2c<N, 1>(c, spec, (const Z*)B, (Z*)out, (const Z*)partner,
                                                      (double2*)c.accA, (double2*)c.accB, cA, cB, npen, twz));
      }
    }
    return e;
  }

  // ------------------------------------------------------------- a2 .. a6
  // q_n of the history (every slice, or checkpoint / segment slots)
  void* q_at(const CtxData& c, int n) const {
    return (char*)c.hist + (size_t)q_slot(c, n) * slice_bytes(c, sizeof(T));
  }

  // With a checkpointed history: before the conjugate step paired with q_n, recompute
  // the segment q_{cK+1} .. q_n (c = n / K) from its checkpoint when n is the top of
  // its segment (one forward split step per slice, Eq. 13).
  cudaError_t recompute_segment(CtxData& c, int n) {
    const int K = c.ckK;
    if (K <= 1 || n % K == 0) return cudaSuccess;
    if (n != c.Ns - 1 && (n + 1) % K != 0) return cudaSuccess;
    for (int j = n - n % K + 1; j <= n; j++) {
      const void* B = (j <= c.NsA) ? c.BA : c.BB;
      cudaError_t e = contour_step(c, q_at(c, j - 1), B, q_at(c, j), 0, nullptr, 0.0, 0.0);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // ------------------------------------------- checkpointed history, separable march
  // With every K-th slice kept (ckK >= 2) on a context whose plan is a separable march
  // (2 or 3; the pencil kernels serve both): the forward march stores the checkpoints (the
  // other slices go to the segment slots, overwritten later); then, from the top segment
  // down, each segment q_{gK+1} .. q_{gK+K-1} is recomputed from its checkpoint by a short
  // separable march, the conjugate march advances by the segment's chunk of steps (one
  // chain across the chunks, its field in spec2, the chunk's qd slices in K slots), and one
  // kernel adds the chunk's pairs to the accumulators of Eq. 8.
  static bool ck_sepp_applies(const CtxData& c) {
    return c.concurrent && c.ckK >= 2 && c.scheme == 0 && !c.edw && (c.plan_plane == 2 || c.plan_plane == 3) &&
           sepp_supported(c);
  }
  int ck_top(const CtxData& c) const { return (c.Ns - 1) / c.ckK; }
  cudaError_t prepare_ck_sepp(CtxData& c) {
    if (c.stepsCK) return cudaSuccess;
    const int K = c.ckK, Ns = c.Ns;
    const size_t slice = slice_bytes(c, sizeof(T));
    cudaError_t e = cudaSuccess;
    if (!c.qdk) {  // kept if a later allocation below fails, and reused by the next attempt
      if ((e = cudaMalloc(&c.qdk, (size_t)K * slice)) != cudaSuccess) return e;
      c.bytes += (size_t)K * slice;
    }
    const char* t = (const char*)c.tables;
    auto blk = [&](int s) -> const void* { return (s <= c.NsA) ? c.BA : c.BB; };
    auto entry = [&](const void* in, const void* B, void* out, void* spec, const void* Bn) {
      BatchStep x;
      memset(&x, 0, sizeof(x));
      x.in = in;
      x.B = B;
      x.out = out;
      x.spec = spec;
      x.Bnext = Bn;
      for (int a = 0; a < 4; a++) x.tw[a] = t + c.tw_off[a];
      for (int a = 0; a < 3; a++) x.d[a] = t + c.sd_off[a];
      return x;
    };
    std::vector<BatchStep> h;
    for (int s = 1; s <= Ns; s++)  // forward march: entry s-1 stores q_s
      h.push_back(entry(q_at(c, s - 1), blk(s), q_at(c, s), c.spec, s < Ns ? blk(s + 1) : nullptr));
    c.ckRoff.assign((size_t)ck_top(c) + 1, 0);
    for (int g = ck_top(c); g >= 0; g--) {  // segment recomputes (field in spec, free after the forward march)
      const int n0 = g * K, n1 = std::min(n0 + K - 1, Ns - 1);
      c.ckRoff[g] = (int)h.size();
      for (int s = n0 + 1; s <= n1; s++)
        h.push_back(entry(q_at(c, n0), blk(s), q_at(c, s), c.spec, s < n1 ? blk(s + 1) : nullptr));
    }
    const size_t coff = h.size();
    std::vector<QuadPair> pr((size_t)Ns);
    for (int g = ck_top(c); g >= 0; g--) {  // conjugate march in chunks: qd_m pairs with q_{Ns-m}
      const int n0 = g * K, n1 = std::min(n0 + K - 1, Ns - 1);
      const int m0 = Ns - n1, m1 = Ns - n0;
      for (int m = m0; m <= m1; m++) {
        const int nb = Ns + 1 - m;  // split step index of this conjugate step
        void* out = (m == Ns) ? c.qd[Ns & 1] : (void*)((char*)c.qdk + (size_t)(m - m0) * slice);
        h.push_back(entry(m == 1 ? c.qd0 : nullptr, blk(nb), out, c.spec2, m < Ns ? blk(nb - 1) : nullptr));
        QuadPair& p = pr[(size_t)m - 1];
        p.q = q_at(c, Ns - m);
        p.qd = out;
        trapezoid_weight(Ns - m, Ns, c.NsA, &p.cA, &p.cB);
      }
    }
    if (h.size() != coff + (size_t)Ns) return cudaErrorInvalidValue;
    c.ckRoff.push_back((int)coff);  // the conjugate entries start here
    // the pair table first: stepsCK marks the path as prepared, so it is set last
    void* dpr = nullptr;
    void* dst = nullptr;
    e = cudaMalloc(&dpr, pr.size() * sizeof(QuadPair));
    if (e == cudaSuccess) e = cudaMemcpy(dpr, pr.data(), pr.size() * sizeof(QuadPair), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&dst, h.size() * sizeof(BatchStep));
    if (e == cudaSuccess) e = cudaMemcpy(dst, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (dpr) cudaFree(dpr);
      if (dst) cudaFree(dst);
      return e;
    }
    c.pairsCK = dpr;
    c.stepsCK = dst;
    c.bytes += pr.size() * sizeof(QuadPair) + h.size() * sizeof(BatchStep);
    return cudaSuccess;
  }
  // Launches j0 .. j1 of a separable pencil march whose entries (one member) start at st.
  cudaError_t ck_run(CtxData& c, const SeppGeom& g, const BatchStep* st, int j0, int j1, cudaStream_t sm) {
    for (int j = j0; j <= j1; j++) {
      if (sm == c.stream) mark(c, KK_PAIR_STEP);
      cudaError_t e = std::is_same<T, float>::value ? sepp_launch_f32(g, st + (j == 0 ? 0 : j - 1), j, 1, sm)
                                                    : sepp_launch_f64(g, st + (j == 0 ? 0 : j - 1), j, 1, sm);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t record_solve_ck_sepp(CtxData& c) {
    const int K = c.ckK, Ns = c.Ns;
    SeppGeom g;
    for (int a = 0; a < 3; a++) g.n[a] = c.n[a];
    g.kind = (c.kind == PFT_SCFT_REAL) ? 0 : 1;
    g.lv = (c.plan_plane == 3) ? c.plan_xv : 0;
    const BatchStep* st = (const BatchStep*)c.stepsCK;
    const BatchStep* cst = st + c.ckRoff.back();
    const QuadPair* pr = (const QuadPair*)c.pairsCK;
    cudaError_t e = ck_run(c, g, st, 0, Ns, c.stream);  // forward march, checkpoints kept
    if (e != cudaSuccess) return e;
    if ((e = solve_mid(c)) != cudaSuccess) return e;  // Q and the (q_Ns, qd_0) term
    // the segment recomputes on the second stream (field in spec, free once the forward
    // march is done), each after the quadrature of the chunk before it has read the segment
    // slots, so that recompute g runs beside conjugate chunk g
    const bool two = !c.profiling && c.plan_streams;
    cudaStream_t rs = two ? c.stream2 : c.stream;
    if (two) {
      if ((e = cudaEventRecord(c.fork_ev, c.stream)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(rs, c.fork_ev, 0)) != cudaSuccess) return e;
    }
    for (int s = ck_top(c); s >= 0; s--) {
      const int n0 = s * K, n1 = std::min(n0 + K - 1, Ns - 1);
      if (n1 > n0 && (e = ck_run(c, g, st + c.ckRoff[s], 0, n1 - n0, rs)) != cudaSuccess) return e;
      if (two && (e = cudaEventRecord(c.join_ev, rs)) != cudaSuccess) return e;
      const int m0 = Ns - n1, m1 = Ns - n0;
      if ((e = ck_run(c, g, cst, m0 == 1 ? 0 : m0, m1, c.stream)) != cudaSuccess) return e;
      if (two && (e = cudaStreamWaitEvent(c.stream, c.join_ev, 0)) != cudaSuccess) return e;
      mark(c, KK_QUADRATURE);
      if (c.kind == PFT_SCFT_REAL)
        k_quad_pairs<T, 0><<<c.npart, PW_THREADS, 0, c.stream>>>(pr + (m0 - 1), m1 - m0 + 1, c.M, (double*)c.accA,
                                                                  (double*)c.accB);
      else
        k_quad_pairs<T, 1><<<c.npart, PW_THREADS, 0, c.stream>>>(pr + (m0 - 1), m1 - m0 + 1, c.M, (double*)c.accA,
                                                                  (double*)c.accB);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if (two && s > 0) {  // the next recompute overwrites the slots this quadrature read
        if ((e = cudaEventRecord(c.fork_ev, c.stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(rs, c.fork_ev, 0)) != cudaSuccess) return e;
      }
    }
    // the second stream's last work (the bottom segment's recompute) precedes the last
    // quadrature, which the context stream already waited for
    return solve_tail(c);  // densities and force norms
  }

  cudaError_t record_solve(CtxData& c) {
    cudaError_t e;
    if (c.scheme == 1) return record_solve_rqm4(c);
    if (c.concurrent && c.ckK == 1) return record_solve_concurrent(c);
    if (ck_sepp_applies(c) && c.stepsCK) return record_solve_ck_sepp(c);
    // forward march (Eqs. 5, 13); a checkpointed history keeps every K-th slice and q_Ns
    for (int n = 1; n <= c.Ns; n++) {
      const void* B = (n <= c.NsA) ? c.BA : c.BB;
      e = contour_step(c, q_at(c, n - 1), B, q_at(c, n), 0, nullptr, 0.0, 0.0);
      if (e != cudaSuccess) return e;
    }
    // Q (Eq. 4) and the qd_0 = 1 term of the quadrature
    if ((e = solve_mid(c)) != cudaSuccess) return e;
    double cA, cB;
    // conjugate march with fused quadrature (Eq. 8)
    for (int m = 1; m <= c.Ns; m++) {
      const int nb = c.Ns + 1 - m;  // split step index of this qd step
      const void* B = (nb <= c.NsA) ? c.BA : c.BB;
      const void* in = (m == 1) ? c.qd0 : c.qd[(m - 1) & 1];
      void* out = c.qd[m & 1];
      const int pn = c.Ns - m;  // forward slice paired with qd_m
      trapezoid_weight(pn, c.Ns, c.NsA, &cA, &cB);
      if ((e = recompute_segment(c, pn)) != cudaSuccess) return e;
      e = contour_step(c, in, B, out, 1, q_at(c, pn), cA, cB);
      if (e != cudaSuccess) return e;
    }
    // densities and force norms
    return solve_tail(c);
  }

  cudaError_t solve_mid(CtxData& c) override { return solve_mid_q(c, true); }

  // Q (Eq. 4) from q_Ns; with_acc: also the qd_0 = 1 terms of the quadrature into the
  // accumulators (the march-fused quadrature of the sequential path needs them; the
  // quadrature over both histories forms every term itself).
  cudaError_t solve_mid_q(CtxData& c, bool with_acc) {
    double cA, cB;
    trapezoid_weight(c.Ns, c.Ns, c.NsA, &cA, &cB);
    mark(c, KK_REDUCE);
    if (c.kind == PFT_SCFT_REAL) {
      k_qsum_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const T*)q_at(c, c.Ns),
                                                          with_acc ? (double*)c.accA : nullptr,
                                                          (double*)c.accB, cA, cB, c.M, c.partials);
    } else {
      k_qsum_cplx<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const Z*)q_at(c, c.Ns), (double2*)c.accA,
                                                          (double2*)c.accB, cA, cB, c.M, c.partials);
    }
    k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_QSUM);
    k_observables<<<1, 32, 0, c.stream>>>(c.scal, (double)c.M, c.C);
    return cudaGetLastError();
  }

  cudaError_t solve_tail(CtxData& c) override {
    mark(c, KK_REDUCE);
    if (c.edw) {
      if (c.kind == PFT_SCFT_REAL) {
        k_finalize_edw_real<<<c.npart, PW_THREADS, 0, c.stream>>>((double*)c.accA, (double*)c.accB, (const double*)c.wp,
                                                                  c.scal, c.ds, c.bC, c.M, c.partials);
      } else {
        k_finalize_edw_cplx<<<c.npart, PW_THREADS, 0, c.stream>>>((double2*)c.accA, (double2*)c.accB,
                                                                  (const double2*)c.wp, c.scal, c.ds, c.bC, c.M,
                                                                  c.partials);
      }
    } else if (c.kind == PFT_SCFT_REAL) {
      k_finalize_real<<<c.npart, PW_THREADS, 0, c.stream>>>((double*)c.accA, (double*)c.accB, (const double*)c.wm,
                                                            c.scal, c.ds, c.chiN, c.M, c.partials);
    } else {
      k_finalize_cplx<<<c.npart, PW_THREADS, 0, c.stream>>>((double2*)c.accA, (double2*)c.accB, (const double2*)c.wm,
                                                            c.scal, c.ds, c.chiN, c.M, c.partials);
    }
    k_reduce_final<6><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_PHIA);
    return cudaGetLastError();
  }

  // ------------------------------------------------------------- a9: batches
  cudaError_t batch_contour_step(const BatchGeom& g, const BatchStep* st, int nact, int epi,
                                 cudaStream_t stream) override {
    if (nact <= 0) return cudaSuccess;
    cudaError_t e = batch_zf(g, st, nact, stream);
    if (e != cudaSuccess) return e;
    if ((e = batch_mid(g, st, nact, stream)) != cudaSuccess) return e;
    return batch_zi(g, st, nact, epi, stream);
  }

  cudaError_t batch_zf(const BatchGeom& g, const BatchStep* st, int nact, cudaStream_t stream) {
    const long long npen = (long long)g.n[0] * g.n[1];
    const int nz = g.n[2];
    cudaError_t e = cudaSuccess;
    if (g.kind == PFT_SCFT_REAL) {
      PFT_BATCH_HALF(nz / 2, e = (bz_r2c<N>(st, npen, nact, stream)));
    } else {
      PFT_BATCH_AXIS(nz, e = (bz_c2c<N>(st, npen, nact, stream)));
    }
    return e;
  }

  cudaError_t batch_zz(const BatchGeom& g, const BatchStep* st, int nact, cudaStream_t stream) {
    const long long npen = (long long)g.n[0] * g.n[1];
    const int nz = g.n[2];
    cudaError_t e = cudaSuccess;
    if (g.kind == PFT_SCFT_REAL) {
      PFT_BATCH_HALF(nz / 2, e = (bzz_r2c<N>(st, npen, nact, stream)));
    } else {
      PFT_BATCH_AXIS(nz, e = (bzz_c2c<N>(st, npen, nact, stream)));
    }
    return e;
  }

  cudaError_t batch_mid(const BatchGeom& g, const BatchStep* st, int nact, cudaStream_t stream) {
    const int nx = g.n[0], ny = g.n[1];
    const long long nzc = g.nzh;
    cudaError_t e = cudaSuccess;
    PFT_BATCH_AXIS(ny, e = (bs<N, 0>(st, nx * nzc, nzc, ny * nzc, nzc, (int)nzc, 1, nact, stream)));
    if (e != cudaSuccess) return e;
    PFT_BATCH_AXIS(nx, e = (bs<N, 2>(st, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, nact, stream)));
    if (e != cudaSuccess) return e;
    PFT_BATCH_AXIS(ny, e = (bs<N, 1>(st, nx * nzc, nzc, ny * nzc, nzc, (int)nzc, 1, nact, stream)));
    return e;
  }

  cudaError_t batch_zi(const BatchGeom& g, const BatchStep* st, int nact, int epi, cudaStream_t stream) {
    const long long npen = (long long)g.n[0] * g.n[1];
    const int nz = g.n[2];
    cudaError_t e = cudaSuccess;
    if (g.kind == PFT_SCFT_REAL) {
      if (epi == 0) {
        PFT_BATCH_HALF(nz / 2, e = (bzi_c2r<N, 0>(st, npen, nact, stream)));
      } else if (epi == 1) {
        PFT_BATCH_HALF(nz / 2, e = (bzi_c2r<N, 1>(st, npen, nact, stream)));
      } else {
        PFT_BATCH_HALF(nz / 2, e = (bzi_c2r<N, 3>(st, npen, nact, stream)));
      }
    } else {
      if (epi == 0) {
        PFT_BATCH_AXIS(nz, e = (bzi_c2c<N, 0>(st, npen, nact, stream)));
      } else if (epi == 1) {
        PFT_BATCH_AXIS(nz, e = (bzi_c2c<N, 1>(st, npen, nact, stream)));
      } else {
        PFT_BATCH_AXIS(nz, e = (bzi_c2c<N, 3>(st, npen, nact, stream)));
      }
    }
    return e;
  }

  // Both marches at once (Eqs. 5, 13): step s of q and step s of qd in the same five
  // launches (two members), then Q (Eq. 4), the quadrature of Eq. 8 over the two stored
  // histories, densities and H.
  cudaError_t prepare_concurrent(CtxData& c) {
    const size_t we = (c.kind == PFT_SCFT_REAL ? sizeof(T) : sizeof(Z));
    const size_t slice = (size_t)c.M * we;
    cudaError_t e;
    if (!c.qdh && !c.edw) {  // the Edwards chain is reversible: qd = q, one history
      e = cudaMalloc(&c.qdh, (size_t)(c.Ns + 1) * slice);
      if (e != cudaSuccess) return e;
      c.bytes += (size_t)(c.Ns + 1) * slice;
    }
    if (!c.steps2) {
      std::vector<BatchStep> h((size_t)2 * c.Ns);
      const char* hist = (const char*)c.hist;
      char* qdh = (char*)c.qdh;
      const char* t = (const char*)c.tables;
      for (int s = 1; s <= c.Ns; s++) {
        BatchStep& f = h[(size_t)2 * (s - 1)];
        BatchStep& b = h[(size_t)2 * (s - 1) + 1];
        memset(&f, 0, sizeof(f));
        memset(&b, 0, sizeof(b));
        f.in = hist + (size_t)(s - 1) * slice;
        f.B = (s <= c.NsA) ? c.BA : c.BB;
        f.out = (void*)(hist + (size_t)s * slice);
        f.spec = c.spec;
        const int nb = c.Ns + 1 - s;
        if (s < c.Ns) f.Bnext = (s + 1 <= c.NsA) ? c.BA : c.BB;
        if (qdh) {
          b.in = (s == 1) ? c.qd0 : (const void*)(qdh + (size_t)(s - 1) * slice);
          b.B = (nb <= c.NsA) ? c.BA : c.BB;
          b.out = qdh + (size_t)s * slice;
          b.spec = c.spec2;
          if (s < c.Ns) b.Bnext = (nb - 1 <= c.NsA) ? c.BA : c.BB;
        }
        for (int a = 0; a < 4; a++) f.tw[a] = b.tw[a] = t + c.tw_off[a];
        for (int a = 0; a < 3; a++) f.d[a] = b.d[a] = t + c.d_off[a];
      }
      e = cudaMalloc(&c.steps2, h.size() * sizeof(BatchStep));
      if (e != cudaSuccess) return e;
      c.bytes += h.size() * sizeof(BatchStep);
      e = cudaMemcpy(c.steps2, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
      if (sep_supported(c) || sepp_supported(c)) {
        // the separable marches: the same steps with the full-axis factors and twiddles
        for (auto& b : h)
          for (int a = 0; a < 3; a++) b.d[a] = t + c.sd_off[a];
        e = cudaMalloc(&c.stepsS, h.size() * sizeof(BatchStep));
        if (e != cudaSuccess) return e;
        c.bytes += h.size() * sizeof(BatchStep);
        e = cudaMemcpy(c.stepsS, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        if (dd_supported(c) && (e = prepare_dd(c, h)) != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }

  // ---------------------------------------------------------------- double-float march
  // Plan 4 of an FP64 context: the separable pencil march with every transform, diffusion
  // and Boltzmann product in double-float arithmetic on the FP32 pipe; q_0 and the stored
  // q_s stay FP64, so everything after the march (quadrature, densities, H, gradients) is
  // the FP64 path's.
  static bool dd_supported(const CtxData& c) { return std::is_same<T, double>::value && sepp_supported(c); }

  // Tables (twiddles of the three axes, the per-axis factors exp(-k_a^2 ds)/n_a, split from
  // their FP64 values), the two split Boltzmann factors, and the step entries (from the
  // separable march's entries h, with B, twiddles and factors redirected).
  cudaError_t prepare_dd(CtxData& c, std::vector<BatchStep> h) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t be = (c.kind == PFT_SCFT_REAL ? sizeof(dd) : sizeof(dd2)) * (size_t)c.M;
    size_t off = 0;
    for (int a = 0; a < 3; a++) {
      c.ddtw_off[a] = off;
      off = al(off + sizeof(dd2) * (size_t)c.n[a]);
    }
    for (int a = 0; a < 3; a++) {
      c.ddsd_off[a] = off;
      off = al(off + sizeof(dd) * (size_t)c.n[a]);
    }
    const size_t tab = off;
    for (int b = 0; b < 2; b++) {
      c.ddB_off[b] = off;
      off = al(off + be);
    }
    cudaError_t e;
    if (!c.ddbuf) {
      if ((e = cudaMalloc(&c.ddbuf, off)) != cudaSuccess) return e;
      c.bytes += off;
    }
    std::vector<unsigned char> t(tab, 0);
    for (int a = 0; a < 3; a++) {
      const int na = c.n[a];
      dd2* tw = reinterpret_cast<dd2*>(t.data() + c.ddtw_off[a]);
      dd* sd = reinterpret_cast<dd*>(t.data() + c.ddsd_off[a]);
      for (int m = 0; m < na; m++) {
        const double ang = -2.0 * M_PI * (double)m / (double)na;
        tw[m].x = dd_split_host(cos(ang));
        tw[m].y = dd_split_host(sin(ang));
        const int mm = (m <= na / 2) ? m : m - na;
        const double k = 2.0 * M_PI * (double)mm / c.L[a];
        sd[m] = dd_split_host(exp(-k * k * c.ds) / (double)na);
      }
    }
    if ((e = cudaMemcpy(c.ddbuf, t.data(), tab, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    char* base = (char*)c.ddbuf;
    auto mapB = [&](const void* B) -> const void* {
      if (B == nullptr) return nullptr;
      return base + (B == c.BA ? c.ddB_off[0] : c.ddB_off[1]);
    };
    for (auto& b : h) {
      b.B = mapB(b.B);
      b.Bnext = mapB(b.Bnext);
      for (int a = 0; a < 3; a++) {
        b.tw[a] = base + c.ddtw_off[a];
        b.d[a] = base + c.ddsd_off[a];
      }
      b.tw[3] = nullptr;
    }
    if (!c.stepsD) {
      if ((e = cudaMalloc(&c.stepsD, h.size() * sizeof(BatchStep))) != cudaSuccess) return e;
      c.bytes += h.size() * sizeof(BatchStep);
    }
    return cudaMemcpy(c.stepsD, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
  }

  // The split Boltzmann factors of this solve (first launches of the solve's graph).
  cudaError_t split_dd(CtxData& c) {
    const long long n = (c.kind == PFT_SCFT_REAL ? 1 : 2) * c.M;
    char* base = (char*)c.ddbuf;
    k_split_dd<<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)c.BA, (dd*)(base + c.ddB_off[0]), n);
    if (c.BB && c.BB != c.BA)
      k_split_dd<<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)c.BB, (dd*)(base + c.ddB_off[1]), n);
    return cudaGetLastError();
  }

  // ---------------------------------------------------------------- separable march
  // On pencils (plan 3): complex fields of any supported size, real fields with ny and nz
  // even (rows and z pairs carried two at a time).
  static bool sepp_supported(const CtxData& c) {
    return c.kind != PFT_SCFT_REAL || (c.n[1] % 2 == 0 && c.n[2] % 2 == 0);
  }
  // Register lines (plan 3 with variant 1, code 19): FP32, and a register plan for the x
  // and the y length.
  static bool sepp_reg_supported(const CtxData& c) {
    return std::is_same<T, float>::value && sepp_supported(c) && sepp_reg_ok(c.n[0]) && sepp_reg_ok(c.n[1]);
  }
  // Line variant lv of plan 3 (code 3 + 16 lv): 0 Plan<N> in 16-line tiles, 1 register lines,
  // 2 Plan<N> in 32-line tiles (FP32), 3 twice the elements a thread in 32-line tiles (FP32, x
  // and y lengths of 32, 48 or 64).
  static bool sepp_lv_supported(const CtxData& c, int lv) {
    if (lv == 0) return sepp_supported(c);
    if (lv == 1) return sepp_reg_supported(c);
    if (lv == 2) return std::is_same<T, float>::value && sepp_supported(c);
    if (lv == 3)
      return std::is_same<T, float>::value && sepp_supported(c) && sepp_wide_ok(c.n[0]) && sepp_wide_ok(c.n[1]);
    return false;
  }
  cudaError_t sepp_march(CtxData& c, const BatchStep* st, int members, cudaStream_t sm) {
    SeppGeom g;
    for (int a = 0; a < 3; a++) g.n[a] = c.n[a];
    g.kind = (c.kind == PFT_SCFT_REAL) ? 0 : 1;
    g.lv = (c.plan_plane == 3) ? c.plan_xv : 0;
    for (int j = 0; j <= c.Ns; j++) {
      if (members == 2) mark(c, KK_PAIR_STEP);
      const BatchStep* ss = st + (size_t)2 * (j == 0 ? 0 : j - 1);
      cudaError_t e = c.plan_plane == 4 ? sepp_launch_dd(g, ss, j, members, sm)
                      : std::is_same<T, float>::value ? sepp_launch_f32(g, ss, j, members, sm)
                                                      : sepp_launch_f64(g, ss, j, members, sm);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // On the plane kernel (plane 2): FP32, nx in {64, 128}; real fields with ny = nz in
  // {64, 128}, complex fields with ny = nz = 64.
  static bool sep_supported(const CtxData& c) {
    if constexpr (!std::is_same<T, float>::value) {
      return false;
    } else {
      if (c.n[1] != c.n[2] || !(c.n[0] == 64 || c.n[0] == 128)) return false;
      if (c.kind != PFT_SCFT_REAL) return c.n[1] == 64;
      return c.n[1] == 64 || c.n[1] == 128;
    }
  }

  template <int N, int MODE>
  static cudaError_t launch_sep_plane_c(const BatchStep* st, int nx, int members, int* err, cudaStream_t sm) {
    using R = SepCfgC<N>;
    auto kern = kb_sep_plane_c<N, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)nx, (unsigned)members), R::THREADS, R::SMEM, sm>>>(st, err);
    return cudaGetLastError();
  }

  template <int N, int MODE, int ADJ = 0>
  static cudaError_t launch_sep_plane(const BatchStep* st, int nx, int members, int* err, cudaStream_t sm) {
    using R = SepCfg<N>;
    auto kern = kb_sep_plane<N, MODE, ADJ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)nx, (unsigned)members), R::THREADS, R::SMEM, sm>>>(st, err);
    return cudaGetLastError();
  }

  // XV 0: the x-lines on Plan<NX> (16 elements a thread at 128); XV 1: on SepXAlt (half
  // the elements a thread, twice the threads, one more exchange)
  template <int NX, int NYZ, int MODE, int KIND, int XV, int ADJ = 0>
  static cudaError_t launch_sep_x(const BatchStep* st, int members, cudaStream_t sm) {
    constexpr int C = 16;
    constexpr long long P = KIND ? (long long)NYZ * NYZ : (long long)NYZ * NYZ / 2;
    using XPL = typename std::conditional<XV == 1, typename SepXAlt<NX>::P, Plan<NX>>::type;
    auto kern = kb_sep_x<NX, NYZ, MODE, C, KIND, XPL, ADJ>;
    const unsigned grid = (unsigned)(P / C);
    kern<<<dim3(grid, (unsigned)members), C * XPL::TPC, sep_x_smem<NX, C>(), sm>>>(st);
    return cudaGetLastError();
  }
  template <int NX, int MODE, int XV>
  static cudaError_t launch_sep_x_v(const BatchStep* st, int nyz, int kind, int members, cudaStream_t sm) {
    if (kind != PFT_SCFT_REAL)
      return nyz == 64 ? launch_sep_x<NX, 64, MODE, 1, XV>(st, members, sm) : cudaErrorNotSupported;
    if (nyz == 128) return launch_sep_x<NX, 128, MODE, 0, XV>(st, members, sm);
    if (nyz == 64) return launch_sep_x<NX, 64, MODE, 0, XV>(st, members, sm);
    return cudaErrorNotSupported;
  }
  template <int NX, int MODE>
  static cudaError_t launch_sep_x_n(const BatchStep* st, int nyz, int kind, int xv, int members, cudaStream_t sm) {
    return xv ? launch_sep_x_v<NX, MODE, 1>(st, nyz, kind, members, sm)
              : launch_sep_x_v<NX, MODE, 0>(st, nyz, kind, members, sm);
  }

  // launch j of a separable march (j = 0: the first plane launch; j >= 1 stores q_j)
  cudaError_t sep_launch(CtxData& c, const BatchStep* ss, int j, int members, cudaStream_t sm) {
    return sep_launch_g(c.n, c.kind, (j == 0) ? 0 : (j == c.Ns ? 2 : 1), j, members, c.kerr, ss, sm, c.plan_xv);
  }
  // mode 0: first launch; 1: a step (entries without Bnext end there); 2: the last step;
  // xv: the x kernel's plan variant
  static cudaError_t sep_launch_g(const int n[3], int kind, int mode, int j, int members, int* err,
                                  const BatchStep* ss, cudaStream_t sm, int xv) {
    if constexpr (!std::is_same<T, float>::value) {
      return cudaErrorNotSupported;
    } else {
      const int nx = n[0], N = n[1];
      if (j >= 1 && (j & 1)) {  // x kernel
        if (nx == 128)
          return mode == 2 ? launch_sep_x_n<128, 2>(ss, N, kind, xv, members, sm)
                           : launch_sep_x_n<128, 1>(ss, N, kind, xv, members, sm);
        if (nx == 64)
          return mode == 2 ? launch_sep_x_n<64, 2>(ss, N, kind, xv, members, sm)
                           : launch_sep_x_n<64, 1>(ss, N, kind, xv, members, sm);
        return cudaErrorNotSupported;
      }
      if (kind != PFT_SCFT_REAL) {
        if (N != 64) return cudaErrorNotSupported;
        if (mode == 0) return launch_sep_plane_c<64, 0>(ss, nx, members, err, sm);
        return mode == 2 ? launch_sep_plane_c<64, 2>(ss, nx, members, err, sm) : launch_sep_plane_c<64, 1>(ss, nx, members, err, sm);
      }
      if (N == 128) {
        if (mode == 0) return launch_sep_plane<128, 0>(ss, nx, members, err, sm);
        return mode == 2 ? launch_sep_plane<128, 2>(ss, nx, members, err, sm)
                         : launch_sep_plane<128, 1>(ss, nx, members, err, sm);
      }
      if (N == 64) {
        if (mode == 0) return launch_sep_plane<64, 0>(ss, nx, members, err, sm);
        return mode == 2 ? launch_sep_plane<64, 2>(ss, nx, members, err, sm) : launch_sep_plane<64, 1>(ss, nx, members, err, sm);
      }
      return cudaErrorNotSupported;
    }
  }

  // Launch j of an adjoint separable march (real fields, ny = nz = N, the source added
  // before each store; the march's last entry has no Bnext).
  template <int N>
  static cudaError_t sep_adj_launch_n(const BatchStep* ss, int nx, int j, int* err, cudaStream_t sm) {
    if (j >= 1 && (j & 1)) {
      if (nx == 128) return launch_sep_x<128, N, 1, 0, 0, 1>(ss, 1, sm);
      if (nx == 64) return launch_sep_x<64, N, 1, 0, 0, 1>(ss, 1, sm);
      return cudaErrorNotSupported;
    }
    return j == 0 ? launch_sep_plane<N, 0, 1>(ss, nx, 1, err, sm) : launch_sep_plane<N, 1, 1>(ss, nx, 1, err, sm);
  }
  cudaError_t sep_adj_launch(CtxData& c, const BatchStep* ss, int j, cudaStream_t sm) {
    if constexpr (!std::is_same<T, float>::value) {
      return cudaErrorNotSupported;
    } else {
      if (c.n[1] == 128) return sep_adj_launch_n<128>(ss, c.n[0], j, c.kerr, sm);
      if (c.n[1] == 64) return sep_adj_launch_n<64>(ss, c.n[0], j, c.kerr, sm);
      return cudaErrorNotSupported;
    }
  }

  // Reverse-mode adjoint on the separable march (FP32 real fields where plan 2 applies):
  // the lambda march (adjoint of the q march) and the mu march (of the qd march) are the
  // separable march run backwards with a source added at every step -- lambda_{k-1} =
  // B_k K(B_k lambda_k) + a_{k-1} -- on two streams, each storing its history; one pass
  // over the four histories then forms the gradient (k_adjsep_grad).
  cudaError_t adjoint_sep(CtxData& c, const double* GA, const double* GB, double* dwp, double* dwm) {
    const size_t slice = (size_t)c.M * sizeof(float);
    const int Ns = c.Ns;
    cudaError_t e;
    if (!c.adjS) {  // lambda and mu histories (Ns + 1 slices each), gA, gB
      const size_t bytes = (size_t)(2 * Ns + 4) * slice;
      if ((e = cudaMalloc(&c.adjS, bytes)) != cudaSuccess) return e;
      c.bytes += bytes;
    }
    float* lam = (float*)c.adjS;
    float* mu = lam + (size_t)(Ns + 1) * c.M;
    float* gA = mu + (size_t)(Ns + 1) * c.M;
    float* gB = gA + c.M;
    const float* hist = (const float*)c.hist;
    auto qd = [&](int m) { return m == 0 ? (const float*)c.qd0 : (const float*)c.qdh + (size_t)m * c.M; };
    auto Bof = [&](int split) { return (const float*)((split <= c.NsA) ? c.BA : c.BB); };
    if (!c.stepsAS) {  // entries 2(j-1): lambda step j (k = Ns + 1 - j); 2(j-1) + 1: mu step j
      std::vector<BatchStep> h((size_t)2 * Ns);
      const char* t = (const char*)c.tables;
      for (int j = 1; j <= Ns; j++) {
        BatchStep& f = h[(size_t)2 * (j - 1)];
        BatchStep& b = h[(size_t)2 * (j - 1) + 1];
        memset(&f, 0, sizeof(f));
        memset(&b, 0, sizeof(b));
        const int k = Ns + 1 - j, m = Ns + 1 - j;
        double cA, cB;
        f.spec = c.spec;
        f.in = lam + (size_t)Ns * c.M;
        f.B = Bof(k);
        f.out = lam + (size_t)(k - 1) * c.M;
        if (k - 1 >= 1) f.Bnext = Bof(k - 1);
        f.partner = qd(Ns - k + 1);
        trapezoid_weight(k - 1, Ns, c.NsA, &cA, &cB);
        f.cA = cA;
        f.cB = cB;
        b.spec = c.spec2;
        b.in = mu + (size_t)Ns * c.M;
        b.B = Bof(Ns + 1 - m);
        b.out = mu + (size_t)(m - 1) * c.M;
        if (m - 1 >= 1) b.Bnext = Bof(Ns + 2 - m);
        b.partner = hist + (size_t)(Ns - m + 1) * c.M;
        trapezoid_weight(Ns - m + 1, Ns, c.NsA, &cA, &cB);
        b.cA = cA;
        b.cB = cB;
        f.accA = b.accA = gA;
        f.accB = b.accB = gB;
        for (int x = 0; x < 4; x++) f.tw[x] = b.tw[x] = t + c.tw_off[x];
        for (int x = 0; x < 3; x++) f.d[x] = b.d[x] = t + c.sd_off[x];
      }
      if ((e = cudaMalloc(&c.stepsAS, h.size() * sizeof(BatchStep))) != cudaSuccess) return e;
      c.bytes += h.size() * sizeof(BatchStep);
      if ((e = cudaMemcpy(c.stepsAS, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    }
    double cAl, cBl, cAm, cBm;
    trapezoid_weight(Ns, Ns, c.NsA, &cAl, &cBl);
    trapezoid_weight(0, Ns, c.NsA, &cAm, &cBm);
    k_adjsep_init<<<c.npart, PW_THREADS, 0, c.stream>>>(GA, GB, c.scal, c.ds, gA, gB, lam + (size_t)Ns * c.M,
                                                        mu + (size_t)Ns * c.M, qd(0), hist, (float)cAl, (float)cBl,
                                                        (float)cAm, (float)cBm, c.M);
    k_adjoint_gamma<<<c.npart, PW_THREADS, 0, c.stream>>>(GA, GB, (const double*)c.accA, (const double*)c.accB, c.M,
                                                          c.partials);
    k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_GAMMA);
    if ((e = cudaEventRecord(c.fork_ev, c.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream2, c.fork_ev, 0)) != cudaSuccess) return e;
    for (int ch = 0; ch < 2; ch++) {
      cudaStream_t sm = ch ? c.stream2 : c.stream;
      for (int j = 0; j <= Ns; j++) {
        const BatchStep* ss = (const BatchStep*)c.stepsAS + (size_t)2 * (j == 0 ? 0 : j - 1) + ch;
        if ((e = sep_adj_launch(c, ss, j, sm)) != cudaSuccess) return e;
      }
    }
    if ((e = cudaEventRecord(c.join_ev, c.stream2)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream, c.join_ev, 0)) != cudaSuccess) return e;
    k_adjsep_grad<<<c.npart, PW_THREADS, 0, c.stream>>>(lam, mu, hist, (const float*)c.qdh, (const float*)c.qd0, gA, gB,
                                                        (const double*)c.accA, (const double*)c.accB,
                                                        c.scal + S_GAMMA, 1.0 / (double)c.M, c.ds, Ns, c.NsA, c.M,
                                                        dwp, dwm);
    return cudaGetLastError();
  }

  // A whole separable march of `members` chains whose step-1 entry is st (entries of
  // consecutive steps two apart).
  cudaError_t sep_march(CtxData& c, const BatchStep* st, int members, cudaStream_t sm) {
    for (int j = 0; j <= c.Ns; j++) {
      const BatchStep* ss = st + (size_t)2 * (j == 0 ? 0 : j - 1);
      cudaError_t e = sep_launch(c, ss, j, members, sm);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  cudaError_t record_solve_concurrent(CtxData& c) {
    BatchGeom g;
    for (int a = 0; a < 3; a++) g.n[a] = c.n[a];
    g.kind = c.kind;
    g.nzh = c.nzh;
    const BatchStep* st = (const BatchStep*)c.steps2;
    cudaError_t e;
    if (c.plan_plane == 4 && c.stepsD && (e = split_dd(c)) != cudaSuccess) return e;
    if (c.edw) {  // one reversible chain: the forward march is the whole solve
      if ((e = march_chain(c, g, st, c.stream)) != cudaSuccess) return e;
      return finish_concurrent(c);
    }
    if (!c.profiling && c.plan_streams) {
      // one chain per propagator on two streams: the two marches are independent until
      // the quadrature, and their kernels fill each other's idle SMs
      if ((e = cudaEventRecord(c.fork_ev, c.stream)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c.stream2, c.fork_ev, 0)) != cudaSuccess) return e;
      for (int m = 0; m < 2; m++) {
        cudaStream_t sm = m ? c.stream2 : c.stream;
        if ((e = march_chain(c, g, st + m, sm)) != cudaSuccess) return e;
      }
      if ((e = cudaEventRecord(c.join_ev, c.stream2)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c.stream, c.join_ev, 0)) != cudaSuccess) return e;
      return finish_concurrent(c);
    }
    if (c.plan_plane == 3 && c.stepsS) {  // separable pencil march, both propagators per launch
      if ((e = sepp_march(c, (const BatchStep*)c.stepsS, 2, c.stream)) != cudaSuccess) return e;
      return finish_concurrent(c);
    }
    if (c.plan_plane == 4 && c.stepsD) {  // the same in double-float arithmetic
      if ((e = sepp_march(c, (const BatchStep*)c.stepsD, 2, c.stream)) != cudaSuccess) return e;
      return finish_concurrent(c);
    }
    if (c.plan_plane == 2 && c.stepsS) {  // separable march, both propagators per launch
      for (int j = 0; j <= c.Ns; j++) {
        mark(c, KK_PAIR_STEP);
        const BatchStep* ss = (const BatchStep*)c.stepsS + (size_t)2 * (j == 0 ? 0 : j - 1);
        if ((e = sep_launch(c, ss, j, 2, c.stream)) != cudaSuccess) return e;
      }
      return finish_concurrent(c);
    }
    if (plane_supported(c) && c.plan_plane) {
      // plane kernel (z and y of step 1), then per step: x pass, plane kernel
      // (y^-1, z^-1 of step s fused with z of step s+1, y)
      mark(c, KK_PAIR_STEP);
      if ((e = batch_plane(c, st, 0, 2, c.stream)) != cudaSuccess) return e;
      const int nx = c.n[0], ny = c.n[1];
      const long long nzc = c.nzh;
      for (int s = 1; s <= c.Ns; s++) {
        mark(c, KK_PAIR_STEP);
        const BatchStep* ss = st + (size_t)2 * (s - 1);
        PFT_BATCH_AXIS(nx, e = (bs<N, 2>(ss, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, 2, c.stream)));
        if (e != cudaSuccess) return e;
        if ((e = batch_plane(c, ss, 1, 2, c.stream)) != cudaSuccess) return e;
      }
      return finish_concurrent(c);
    }
    // z forward of step 1, then per step: y, x (D), y^-1, and the z inverse of step s
    // fused with the z forward of step s+1
    mark(c, KK_PAIR_STEP);
    if ((e = batch_zf(g, st, 2, c.stream)) != cudaSuccess) return e;
    for (int s = 1; s <= c.Ns; s++) {
      mark(c, KK_PAIR_STEP);
      const BatchStep* ss = st + (size_t)2 * (s - 1);
      if ((e = batch_mid(g, ss, 2, c.stream)) != cudaSuccess) return e;
      if ((e = batch_zz(g, ss, 2, c.stream)) != cudaSuccess) return e;
    }
    return finish_concurrent(c);
  }

  // All Ns steps of one propagator on `sm`: st points at the member's entry of step 1
  // (entries of consecutive steps are two apart).
  cudaError_t march_chain(CtxData& c, const BatchGeom& g, const BatchStep* st, cudaStream_t sm) {
    cudaError_t e;
    if (c.plan_plane == 2 && c.stepsS) {  // separable march: one launch per contour step
      const BatchStep* ss = (const BatchStep*)c.stepsS + (st - (const BatchStep*)c.steps2);
      return sep_march(c, ss, 1, sm);
    }
    if (c.plan_plane == 3 && c.stepsS) {  // separable pencil march: two launches per step
      const BatchStep* ss = (const BatchStep*)c.stepsS + (st - (const BatchStep*)c.steps2);
      return sepp_march(c, ss, 1, sm);
    }
    if (c.plan_plane == 4 && c.stepsD) {  // the same in double-float arithmetic
      const BatchStep* ss = (const BatchStep*)c.stepsD + (st - (const BatchStep*)c.steps2);
      return sepp_march(c, ss, 1, sm);
    }
    if (plane_supported(c) && c.plan_plane) {
      if ((e = batch_plane(c, st, 0, 1, sm)) != cudaSuccess) return e;
      const int nx = c.n[0], ny = c.n[1];
      const long long nzc = c.nzh;
      for (int s = 1; s <= c.Ns; s++) {
        const BatchStep* ss = st + (size_t)2 * (s - 1);
        PFT_BATCH_AXIS(nx, e = (bs<N, 2>(ss, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, 1, sm)));
        if (e != cudaSuccess) return e;
        if ((e = batch_plane(c, ss, 1, 1, sm)) != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    if ((e = batch_zf(g, st, 1, sm)) != cudaSuccess) return e;
    for (int s = 1; s <= c.Ns; s++) {
      const BatchStep* ss = st + (size_t)2 * (s - 1);
      if ((e = batch_mid(g, ss, 1, sm)) != cudaSuccess) return e;
      if ((e = batch_zz(g, ss, 1, sm)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // Autotuner of the pass march: one timed eager solve (after a warm-up solve) for each
  // plan -- plane kernel or pencil passes where the plane kernel applies, two chains on
  // two streams or two-member launches -- on the context's own fields; the fastest is
  // kept and cached per (grid, field kind, precision, Ns).
  cudaError_t tune_plan(CtxData& c) {
    c.tuned = true;
    char key[160];
    snprintf(key, sizeof(key), "%dx%dx%d/%s/%s/Ns%d", c.n[0], c.n[1], c.n[2],
             c.kind == PFT_SCFT_REAL ? "real" : "complex", sizeof(T) == 4 ? "fp32" : "fp64", c.Ns);
    int pl = 0, sm = 0;
    if (plan_cache_lookup(key, &pl, &sm)) {
      const int fam = pl & 15;
      c.plan_xv = (fam == 2) ? (pl >> 4) & 1 : (fam == 3 && sepp_lv_supported(c, pl >> 4)) ? (pl >> 4) : 0;
      if (fam == 3 && sepp_supported(c) && c.stepsS) c.plan_plane = 3;
      else c.plan_plane = (fam == 2 && sep_supported(c) && c.stepsS) ? 2 : ((fam == 1 && plane_supported(c)) ? 1 : 0);
      c.plan_streams = sm ? 1 : 0;
      return cudaSuccess;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = -1.f;
    int bpl = c.plan_plane, bsm = c.plan_streams, bxv = c.plan_xv;
    // candidates: separable pencil march (four line variants), separable plane march (two
    // x-kernel plans), plane kernel, pencil passes; two chains or two-member launches
    for (int cand = 0; cand < 16 && e == cudaSuccess; cand++) {
      static const int fam_of[8] = {3, 3, 3, 3, 2, 2, 1, 0}, xv_of[8] = {0, 1, 2, 3, 0, 1, 0, 0};
      const int cpl = fam_of[cand / 2], cxv = xv_of[cand / 2], csm = (cand & 1) ? 0 : 1;
      if (cpl == 3 && !(sepp_supported(c) && c.stepsS)) continue;
      if (cpl == 3 && !sepp_lv_supported(c, cxv)) continue;
      if (cpl == 2 && !(sep_supported(c) && c.stepsS)) continue;
      if (cpl == 1 && !plane_supported(c)) continue;
      c.plan_plane = cpl;
      c.plan_xv = cxv;
      c.plan_streams = csm;
      if ((e = record_solve(c)) != cudaSuccess) break;  // warm-up
      if ((e = cudaEventRecord(e0, c.stream)) != cudaSuccess) break;
      if ((e = record_solve(c)) != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, c.stream)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (best < 0.f || ms < best) {
        best = ms;
        bpl = cpl;
        bsm = csm;
        bxv = cxv;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c.plan_plane = bpl;
    c.plan_streams = bsm;
    c.plan_xv = bxv;
    if (e != cudaSuccess) return e;
    plan_cache_store(key, bpl + 16 * bxv, bsm, (double)best);
    return cudaSuccess;
  }

  cudaError_t batch_pair_step(const BatchGeom& g, const BatchStep* st, int nact, bool first,
                              cudaStream_t stream) override {
    if (nact <= 0) return cudaSuccess;
    cudaError_t e;
    if (plane_geom(g)) {
      // plane kernel (z and y of step 1), then per step: x pass, plane kernel
      CtxData cg;
      for (int a = 0; a < 3; a++) cg.n[a] = g.n[a];
      cg.kind = g.kind;
      if (first && (e = batch_plane(cg, st, 0, nact, stream)) != cudaSuccess) return e;
      const long long nzc = g.nzh;
      PFT_BATCH_AXIS(g.n[0], e = (bs<N, 2>(st, g.n[1] * nzc, g.n[1] * nzc, 0, g.n[1] * nzc, (int)nzc, 0, nact, stream)));
      if (e != cudaSuccess) return e;
      return batch_plane(cg, st, 1, nact, stream);
    }
    if (first && (e = batch_zf(g, st, nact, stream)) != cudaSuccess) return e;
    if ((e = batch_mid(g, st, nact, stream)) != cudaSuccess) return e;
    return batch_zz(g, st, nact, stream);
  }

  bool batch_plan_ok(const BatchGeom& g, int plan) const override {
    if (plan == 0 || plan == 1) return true;
    CtxData cg;
    for (int a = 0; a < 3; a++) cg.n[a] = g.n[a];
    cg.kind = g.kind;
    if (plan == 2) return sep_supported(cg);
    if (plan == 3) return sepp_supported(cg);
    if ((plan & 15) == 3) return sepp_lv_supported(cg, plan >> 4);  // 19, 35, 51
    return false;
  }

  // Launch j of a separable march of a batch class (plan 2: plane and x kernels; plan 3:
  // pencils) over nact entries; an entry without Bnext ends its member's march there.
  cudaError_t batch_sep_launch(const BatchGeom& g, const BatchStep* ss, int j, int nact, int plan, int* err,
                               cudaStream_t sm) override {
    if (nact <= 0) return cudaSuccess;
    if (plan == 2) return sep_launch_g(g.n, g.kind, j == 0 ? 0 : 1, j, nact, err, ss, sm, 0);
    SeppGeom sg;
    for (int a = 0; a < 3; a++) sg.n[a] = g.n[a];
    sg.kind = (g.kind == PFT_SCFT_REAL) ? 0 : 1;
    sg.lv = ((plan & 15) == 3) ? plan >> 4 : 0;
    return std::is_same<T, float>::value ? sepp_launch_f32(sg, ss, j, nact, sm) : sepp_launch_f64(sg, ss, j, nact, sm);
  }

  cudaError_t finish_both(CtxData& c) override { return finish_concurrent(c); }

  int batch_pair_launches(const BatchGeom& g, bool first) const override {
    return plane_geom(g) ? (first ? 3 : 2) : (first ? 5 : 4);
  }

  // the plane kernel applies to a batch class of this geometry
  static bool plane_geom(const BatchGeom& g) {
    CtxData cg;
    for (int a = 0; a < 3; a++) cg.n[a] = g.n[a];
    cg.kind = g.kind;
    return plane_supported(cg);
  }

  cudaError_t quadrature(CtxData& c) override {
    mark(c, KK_QUADRATURE);
    const int blocks = c.sms * 8;
    const void* qdh = c.edw ? c.hist : c.qdh;
    const void* qd0 = c.edw ? c.hist : c.qd0;
    if (c.kind == PFT_SCFT_REAL) {
      if (std::is_same<T, float>::value && c.M % 4 == 0) {  // 16-byte loads, four points a thread
        k_quadrature_real4<<<blocks, PW_THREADS, 0, c.stream>>>((const float*)c.hist, (const float*)qdh,
                                                                (const float*)qd0, c.M, c.Ns, c.NsA,
                                                                (double*)c.accA, (double*)c.accB);
      } else {
        k_quadrature_real<T><<<blocks, PW_THREADS, 0, c.stream>>>((const T*)c.hist, (const T*)qdh, (const T*)qd0,
                                                                 c.M, c.Ns, c.NsA, (double*)c.accA, (double*)c.accB);
      }
    } else {
      k_quadrature_cplx<T><<<blocks, PW_THREADS, 0, c.stream>>>((const Z*)c.hist, (const Z*)qdh, (const Z*)qd0, c.M,
                                                               c.Ns, c.NsA, (double2*)c.accA, (double2*)c.accB);
    }
    return cudaGetLastError();
  }

  // ------------------------------------------- reverse-mode adjoint (f3)
  // Adjoint marches of q (chain 0) and qd (chain 1) for a loss on the densities, both in
  // the same batched transforms: per step k = Ns .. 1, z = K(B lambda_k) by the z forward,
  // y, x (D), y inverse and z inverse passes (no final factor), then k_adjoint_update.
  cudaError_t adjoint(CtxData& c, const double* GA, const double* GB, double* dwp, double* dwm) override {
    if (c.kind != PFT_SCFT_REAL || !c.qdh) return cudaErrorNotSupported;
    if (c.plan_plane == 2 && sep_supported(c) && c.M % 4 == 0) return adjoint_sep(c, GA, GB, dwp, dwm);
    const size_t slice = (size_t)c.M * sizeof(T);
    cudaError_t e;
    if (!c.adj) {  // lambda and mu ping-pong, the two z slices, four FP64 accumulators
      const size_t bytes = 6 * slice + 4 * (size_t)c.M * sizeof(double);
      if ((e = cudaMalloc(&c.adj, bytes)) != cudaSuccess) return e;
      c.bytes += bytes;
    }
    char* a = (char*)c.adj;
    T* lam[2] = {(T*)a, (T*)(a + slice)};
    T* mu[2] = {(T*)(a + 2 * slice), (T*)(a + 3 * slice)};
    T* z0 = (T*)(a + 4 * slice);
    T* z1 = (T*)(a + 5 * slice);
    double* dw = (double*)(a + 6 * slice);  // [4][M]: dwA, dwB of chain 0, then of chain 1
    const char* hist = (const char*)c.hist;
    const char* qdh = (const char*)c.qdh;
    auto qs = [&](int j) { return (const T*)(hist + (size_t)j * slice); };
    auto qds = [&](int j) { return j == 0 ? (const T*)c.qd0 : (const T*)(qdh + (size_t)j * slice); };
    auto Bof = [&](int split) { return (const T*)((split <= c.NsA) ? c.BA : c.BB); };
    if (!c.stepsa) {  // entries 2(k-1) and 2(k-1)+1: the transforms of step k of both chains
      std::vector<BatchStep> h((size_t)2 * c.Ns);
      const char* t = (const char*)c.tables;
      for (int k = 1; k <= c.Ns; k++) {
        BatchStep& f = h[(size_t)2 * (k - 1)];
        BatchStep& b = h[(size_t)2 * (k - 1) + 1];
        memset(&f, 0, sizeof(f));
        memset(&b, 0, sizeof(b));
        f.in = lam[(c.Ns - k) & 1];
        f.B = Bof(k);
        f.out = z0;
        f.spec = c.spec;
        b.in = mu[(c.Ns - k) & 1];
        b.B = Bof(c.Ns + 1 - k);
        b.out = z1;
        b.spec = c.spec2;
        for (int x = 0; x < 4; x++) f.tw[x] = b.tw[x] = t + c.tw_off[x];
        for (int x = 0; x < 3; x++) f.d[x] = b.d[x] = t + c.d_off[x];
      }
      if ((e = cudaMalloc(&c.stepsa, h.size() * sizeof(BatchStep))) != cudaSuccess) return e;
      c.bytes += h.size() * sizeof(BatchStep);
      e = cudaMemcpy(c.stepsa, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
    }
    BatchGeom g;
    for (int x = 0; x < 3; x++) g.n[x] = c.n[x];
    g.kind = c.kind;
    g.nzh = c.nzh;
    double cA, cB, cAm, cBm;
    trapezoid_weight(c.Ns, c.Ns, c.NsA, &cA, &cB);
    trapezoid_weight(0, c.Ns, c.NsA, &cAm, &cBm);
    k_adjoint_init<T><<<c.npart, PW_THREADS, 0, c.stream>>>(lam[0], mu[0], qds(0), qs(0), GA, GB, c.scal, c.ds, cA, cB,
                                                            cAm, cBm, dw, c.M);
    const BatchStep* st = (const BatchStep*)c.stepsa;
    // the two adjoint chains on two streams
    if ((e = cudaEventRecord(c.fork_ev, c.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream2, c.fork_ev, 0)) != cudaSuccess) return e;
    if constexpr (std::is_same<T, float>::value) {
      if (plane_supported(c) && c.plan_plane) {
        if (!c.stepsap) {  // entries 2(k-1) + ch: step k of chain ch
          std::vector<AdjPlaneStep> h((size_t)2 * c.Ns);
          const char* t = (const char*)c.tables;
          for (int k = 1; k <= c.Ns; k++) {
            const int cur = (c.Ns - k) & 1;
            for (int ch = 0; ch < 2; ch++) {
              AdjPlaneStep& a = h[(size_t)2 * (k - 1) + ch];
              memset(&a, 0, sizeof(a));
              const int split = ch ? c.Ns + 1 - k : k;         // split step of this chain at k
              a.lam = (ch ? mu : lam)[cur];
              a.lam_next = (ch ? mu : lam)[cur ^ 1];
              a.B = Bof(split);
              a.Bnext = (k > 1) ? Bof(ch ? split + 1 : split - 1) : nullptr;
              a.qk = ch ? qds(k) : qs(k);
              a.qk1 = ch ? qds(k - 1) : qs(k - 1);
              a.src = ch ? qs(c.Ns - k + 1) : qds(c.Ns - k + 1);
              trapezoid_weight(ch ? c.Ns - k + 1 : k - 1, c.Ns, c.NsA, &a.cA, &a.cB);
              a.dw = dw + (size_t)(2 * ch + (split <= c.NsA ? 0 : 1)) * c.M;
              a.spec = ch ? c.spec2 : c.spec;
              for (int x = 0; x < 4; x++) a.tw[x] = t + c.tw_off[x];
            }
          }
          if ((e = cudaMalloc(&c.stepsap, h.size() * sizeof(AdjPlaneStep))) != cudaSuccess) return e;
          c.bytes += h.size() * sizeof(AdjPlaneStep);
          e = cudaMemcpy(c.stepsap, h.data(), h.size() * sizeof(AdjPlaneStep), cudaMemcpyHostToDevice);
          if (e != cudaSuccess) return e;
        }
        const AdjPlaneStep* ap = (const AdjPlaneStep*)c.stepsap;
        const int nx = c.n[0], ny = c.n[1];
        const long long nzc = c.nzh;
        for (int ch = 0; ch < 2; ch++) {
          cudaStream_t sm = ch ? c.stream2 : c.stream;
          // z and y forward of B_Ns lambda_Ns (the plane kernel's first step), then per
          // step: x pass (D), the fused adjoint step
          if ((e = batch_plane(c, st + (size_t)2 * (c.Ns - 1) + ch, 0, 1, sm)) != cudaSuccess) return e;
          for (int k = c.Ns; k >= 1; k--) {
            const BatchStep* sc = st + (size_t)2 * (k - 1) + ch;
            PFT_BATCH_AXIS(nx, e = (bs<N, 2>(sc, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, 1, sm)));
            if (e != cudaSuccess) return e;
            if ((e = launch_plane_adj(c, ap + (size_t)2 * (k - 1) + ch, GA, GB, sm)) != cudaSuccess) return e;
          }
        }
        goto joined;
      }
    }
    for (int k = c.Ns; k >= 1; k--) {
      const BatchStep* ss = st + (size_t)2 * (k - 1);
      const int cur = (c.Ns - k) & 1;
      AdjChain c0, c1;
      c0.lam = lam[cur];
      c0.lam_next = lam[cur ^ 1];
      c0.z = z0;
      c0.qk = qs(k);
      c0.qk1 = qs(k - 1);
      c0.B = Bof(k);
      c0.src = qds(c.Ns - k + 1);
      trapezoid_weight(k - 1, c.Ns, c.NsA, &c0.cA, &c0.cB);
      c0.blockA = (k <= c.NsA) ? 1 : 0;
      c1.lam = mu[cur];
      c1.lam_next = mu[cur ^ 1];
      c1.z = z1;
      c1.qk = qds(k);
      c1.qk1 = qds(k - 1);
      c1.B = Bof(c.Ns + 1 - k);
      c1.src = qs(c.Ns - k + 1);
      trapezoid_weight(c.Ns - k + 1, c.Ns, c.NsA, &c1.cA, &c1.cB);
      c1.blockA = (c.Ns + 1 - k <= c.NsA) ? 1 : 0;
      const long long npen = (long long)c.n[0] * c.n[1];
      for (int ch = 0; ch < 2; ch++) {
        cudaStream_t sm = ch ? c.stream2 : c.stream;
        const BatchStep* sc = ss + ch;
        if ((e = batch_zf(g, sc, 1, sm)) != cudaSuccess) return e;
        if ((e = batch_mid(g, sc, 1, sm)) != cudaSuccess) return e;
        PFT_BATCH_HALF(c.n[2] / 2, e = (bzi_c2r<N, 2>(sc, npen, 1, sm)));
        if (e != cudaSuccess) return e;
        k_adjoint_update<T><<<c.npart, PW_THREADS, 0, sm>>>(ch ? c1 : c0, GA, GB, c.scal, c.ds, dw + 2 * ch * c.M,
                                                           dw + (2 * ch + 1) * c.M, c.M);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
    }
  joined:
    if ((e = cudaEventRecord(c.join_ev, c.stream2)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream, c.join_ev, 0)) != cudaSuccess) return e;
    k_adjoint_gamma<<<c.npart, PW_THREADS, 0, c.stream>>>(GA, GB, (const double*)c.accA, (const double*)c.accB, c.M,
                                                         c.partials);
    k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_GAMMA);
    k_adjoint_finish<<<c.npart, PW_THREADS, 0, c.stream>>>(dw, (const double*)c.accA, (const double*)c.accB,
                                                          c.scal + S_GAMMA, 1.0 / (double)c.M, dwp, dwm, c.M);
    return cudaGetLastError();
  }

  // Q, the quadrature over both histories, densities and H
  cudaError_t finish_concurrent(CtxData& c) {
    cudaError_t e;
    const bool real = (c.kind == PFT_SCFT_REAL);
    if ((e = solve_mid_q(c, !real)) != cudaSuccess) return e;
    if (std::is_same<T, float>::value && real && !c.edw && c.M % 4 == 0) {
      // the quadrature with the densities and force sums of the tail in one pass
      mark(c, KK_QUADRATURE);
      const int nb = c.npart;
      k_quadrature_final_real4<<<nb, PW_THREADS, 0, c.stream>>>(
          (const float*)c.hist, (const float*)c.qdh, (const float*)c.qd0, c.M, c.Ns, c.NsA, (double*)c.accA,
          (double*)c.accB, (const double*)c.wm, c.scal, c.ds, c.chiN, c.partials);
      mark(c, KK_REDUCE);
      k_reduce_final<6><<<1, PW_THREADS, 0, c.stream>>>(c.partials, nb, c.scal + S_PHIA);
      return cudaGetLastError();
    }
    if ((e = quadrature(c)) != cudaSuccess) return e;
    return solve_tail(c);
  }

  // ------------------------------------------------------ 4th-order scheme
  // One contour step of Eq. 13 for both propagators, three members per propagator
  // (entries 3p .. 3p+2 of a step, p = 0 for q and 1 for qd):
  //   3p      A(ds) of the previous slice                          -> rq[p]
  //   3p + 1  first A(ds/2) (z inverse fused with the z forward of the second)
  //   3p + 2  second A(ds/2), stored as (4 A(ds/2)A(ds/2) q - A(ds) q) / 3 -> q_s, qd_s
  // Per step and propagator (one chain per stream): z forward, y, x (D), y inverse of the
  // first two members; z inverse of the full step; fused z inverse / z forward of the
  // first half step; y, x (D/2), y inverse and combining z inverse of the second.
  cudaError_t prepare_rqm4(CtxData& c) {
    const size_t we = (c.kind == PFT_SCFT_REAL ? sizeof(T) : sizeof(Z));
    const size_t slice = (size_t)c.M * we;
    const size_t spec_b = (size_t)c.M * sizeof(Z);
    cudaError_t e;
    if (!c.qdh) {
      if ((e = cudaMalloc(&c.qdh, (size_t)(c.Ns + 1) * slice)) != cudaSuccess) return e;
      c.bytes += (size_t)(c.Ns + 1) * slice;
    }
    if (!c.rq) {
      // four propagator slices, then two spectra
      const size_t b = 4 * slice + 2 * spec_b;
      if ((e = cudaMalloc(&c.rq, b)) != cudaSuccess) return e;
      c.bytes += b;
    }
    if (!c.qw) {
      std::vector<double> w((size_t)2 * (c.Ns + 1), 0.0);
      simpson_block(0, c.NsA, w.data());
      simpson_block(c.NsA, c.Ns, w.data() + (c.Ns + 1));
      if ((e = cudaMalloc(&c.qw, w.size() * sizeof(double))) != cudaSuccess) return e;
      c.bytes += w.size() * sizeof(double);
      if ((e = cudaMemcpy(c.qw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    }
    if (!c.steps2) {
      // on the plane kernels the second half step stores B y into the scratch slice of the
      // first (free by then) and a separate kernel forms the combination
      c.rq_plane = plane_supported(c) && c.plan_plane;
      char* rq = (char*)c.rq;
      void* rqs[4] = {rq, rq + slice, rq + 2 * slice, rq + 3 * slice};
      void* spec3 = rq + 4 * slice;
      void* spec4 = rq + 4 * slice + spec_b;
      std::vector<BatchStep> h((size_t)6 * c.Ns);
      const char* hist = (const char*)c.hist;
      char* qdh = (char*)c.qdh;
      const char* t = (const char*)c.tables;
      for (int s = 1; s <= c.Ns; s++) {
        BatchStep* e6 = &h[(size_t)6 * (s - 1)];
        memset(e6, 0, 6 * sizeof(BatchStep));
        const int nb = c.Ns + 1 - s;  // block index of the conjugate march's step
        const void* in[2] = {hist + (size_t)(s - 1) * slice,
                             (s == 1) ? c.qd0 : (const void*)(qdh + (size_t)(s - 1) * slice)};
        void* out[2] = {(void*)(hist + (size_t)s * slice), qdh + (size_t)s * slice};
        const bool inA[2] = {s <= c.NsA, nb <= c.NsA};
        void* full_spec[2] = {c.spec, c.spec2};
        void* half_spec[2] = {spec3, spec4};
        for (int p = 0; p < 2; p++) {
          const void* Bf = inA[p] ? c.BA : c.BB;
          const void* Bh = inA[p] ? c.BAh : c.BBh;
          BatchStep& f = e6[3 * p];       // entries of one propagator are contiguous:
          BatchStep& h1 = e6[3 * p + 1];  // full step, first and second half step
          BatchStep& h2 = e6[3 * p + 2];
          f.in = in[p];
          f.B = Bf;
          f.out = rqs[p];
          f.spec = full_spec[p];
          h1.in = in[p];
          h1.B = Bh;
          h1.out = rqs[2 + p];
          h1.spec = half_spec[p];
          h1.Bnext = Bh;
          h2.B = Bh;
          h2.out = c.rq_plane ? rqs[2 + p] : out[p];
          h2.partner = rqs[p];
          h2.spec = half_spec[p];
          for (BatchStep* b : {&f, &h1, &h2})
            for (int a = 0; a < 4; a++) b->tw[a] = t + c.tw_off[a];
          for (int a = 0; a < 3; a++) {
            f.d[a] = t + c.d_off[a];
            h1.d[a] = h2.d[a] = t + c.dh_off[a];
          }
        }
      }
      if ((e = cudaMalloc(&c.steps2, h.size() * sizeof(BatchStep))) != cudaSuccess) return e;
      c.bytes += h.size() * sizeof(BatchStep);
      e = cudaMemcpy(c.steps2, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  cudaError_t record_solve_rqm4(CtxData& c) {
    BatchGeom g;
    for (int a = 0; a < 3; a++) g.n[a] = c.n[a];
    g.kind = c.kind;
    g.nzh = c.nzh;
    const BatchStep* st = (const BatchStep*)c.steps2;
    cudaError_t e;
    // one chain per propagator on two streams, three members per step (full step, first
    // and second half step)
    if ((e = cudaEventRecord(c.fork_ev, c.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream2, c.fork_ev, 0)) != cudaSuccess) return e;
    for (int s = 1; s <= c.Ns; s++) {
      mark(c, KK_PAIR_STEP);
      for (int p = 0; p < 2; p++) {
        cudaStream_t sm = p ? c.stream2 : c.stream;
        const BatchStep* e3 = st + (size_t)6 * (s - 1) + 3 * p;
        if (c.rq_plane) {
          // full and first half step: rows x B, z and y forward; x pass (D, D/2); y^-1,
          // z^-1, x B, store (the half step then x B_h, z and y forward of the second);
          // second half: x pass (D/2), y^-1, z^-1, x B_h; the combination
          const int nx = c.n[0], ny = c.n[1];
          const long long nzc = c.nzh;
          if ((e = batch_plane(c, e3, 0, 2, sm)) != cudaSuccess) return e;
          PFT_BATCH_AXIS(nx, e = (bs<N, 2>(e3, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, 2, sm)));
          if (e != cudaSuccess) return e;
          if ((e = batch_plane(c, e3, 1, 2, sm)) != cudaSuccess) return e;
          PFT_BATCH_AXIS(nx, e = (bs<N, 2>(e3 + 2, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, 1, sm)));
          if (e != cudaSuccess) return e;
          if ((e = batch_plane(c, e3 + 2, 1, 1, sm)) != cudaSuccess) return e;
          const size_t slice = (size_t)c.M * sizeof(T);  // real working-precision slice
          const char* rq = (const char*)c.rq;
          const size_t sl = (c.kind == PFT_SCFT_REAL) ? slice : 2 * slice;
          T* outp = (T*)((char*)(p ? c.qdh : c.hist) + (size_t)s * sl);
          const long long nval = (c.kind == PFT_SCFT_REAL) ? c.M : 2 * c.M;
          k_rqm4_combine<T><<<c.npart, PW_THREADS, 0, sm>>>((const T*)(rq + (size_t)(2 + p) * sl),
                                                            (const T*)(rq + (size_t)p * sl), outp, nval);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
          continue;
        }
        if ((e = batch_zf(g, e3, 2, sm)) != cudaSuccess) return e;
        if ((e = batch_mid(g, e3, 2, sm)) != cudaSuccess) return e;
        if ((e = batch_zi(g, e3, 1, 0, sm)) != cudaSuccess) return e;
        if ((e = batch_zz(g, e3 + 1, 1, sm)) != cudaSuccess) return e;
        if ((e = batch_mid(g, e3 + 2, 1, sm)) != cudaSuccess) return e;
        if ((e = batch_zi(g, e3 + 2, 1, 3, sm)) != cudaSuccess) return e;
      }
    }
    if ((e = cudaEventRecord(c.join_ev, c.stream2)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream, c.join_ev, 0)) != cudaSuccess) return e;
    if ((e = solve_mid(c)) != cudaSuccess) return e;
    mark(c, KK_QUADRATURE);
    const int blocks = c.sms * 8;
    if (c.kind == PFT_SCFT_REAL) {
      k_quadrature_w_real<T><<<blocks, PW_THREADS, 0, c.stream>>>((const T*)c.hist, (const T*)c.qdh, (const T*)c.qd0,
                                                                 c.M, c.Ns, c.qw, (double*)c.accA, (double*)c.accB);
    } else {
      k_quadrature_w_cplx<T><<<blocks, PW_THREADS, 0, c.stream>>>((const Z*)c.hist, (const Z*)c.qdh, (const Z*)c.qd0,
                                                                 c.M, c.Ns, c.qw, (double2*)c.accA, (double2*)c.accB);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return solve_tail(c);
  }

  // The plane kernel (y and z of a step in shared memory): FP32 real fields on 64^3 or
  // 128^3 style grids (ny = nz in {64, 128}).
  static bool plane_supported(const CtxData& c) {
    if constexpr (!std::is_same<T, float>::value) {
      return false;
    } else {
      if (c.kind == PFT_SCFT_REAL) return c.n[1] == c.n[2] && (c.n[1] == 64 || c.n[1] == 128);
      return c.n[1] == 64 && c.n[2] == 64;  // complex: the 64 x 64 plane kernel
    }
  }

  template <int NY, int MODE>
  static cudaError_t launch_plane(const BatchStep* st, int nx, int members, cudaStream_t stream) {
    using R = PlaneCfg<NY, NY>;
    auto kern = kb_plane_r2c<NY, NY, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)nx, (unsigned)members), R::THREADS, R::SMEM, stream>>>(st);
    return cudaGetLastError();
  }

  template <int NY, int MODE>
  static cudaError_t launch_plane_c(const BatchStep* st, int nx, int members, cudaStream_t stream) {
    using R = PlaneCfgC<NY, NY>;
    auto kern = kb_plane_c2c<NY, NY, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)nx, (unsigned)members), R::THREADS, R::SMEM, stream>>>(st);
    return cudaGetLastError();
  }

  // one fused adjoint step (real fields, FP32) of one chain
  static cudaError_t launch_plane_adj(CtxData& c, const AdjPlaneStep* ap, const double* GA, const double* GB,
                                      cudaStream_t sm) {
    cudaError_t e = cudaErrorNotSupported;
    auto go = [&](auto kern, size_t smem, int threads) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return;
      kern<<<dim3((unsigned)c.n[0], 1), threads, smem, sm>>>(ap, GA, GB, c.scal + S_Q, c.ds);
      e = cudaGetLastError();
    };
    if (c.n[1] == 64) go(kb_plane_adj<64, 64>, PlaneCfg<64, 64>::SMEM, PlaneCfg<64, 64>::THREADS);
    if (c.n[1] == 128) go(kb_plane_adj<128, 128>, PlaneCfg<128, 128>::SMEM, PlaneCfg<128, 128>::THREADS);
    return e;
  }

  // the plane kernel over `members` consecutive entries of st
  cudaError_t batch_plane(CtxData& c, const BatchStep* st, int mode, int members, cudaStream_t sm) {
    if constexpr (!std::is_same<T, float>::value) {
      return cudaErrorNotSupported;
    } else {
      const int nx = c.n[0];
      if (c.kind != PFT_SCFT_REAL) {
        if (c.n[1] == 64 && c.n[2] == 64)
          return mode ? launch_plane_c<64, 1>(st, nx, members, sm) : launch_plane_c<64, 0>(st, nx, members, sm);
        return cudaErrorNotSupported;
      }
      if (c.n[1] == 64)
        return mode ? launch_plane<64, 1>(st, nx, members, sm) : launch_plane<64, 0>(st, nx, members, sm);
      if (c.n[1] == 128)
        return mode ? launch_plane<128, 1>(st, nx, members, sm) : launch_plane<128, 0>(st, nx, members, sm);
      return cudaErrorNotSupported;
    }
  }

  cudaError_t enqueue_solve(CtxData& c) override {
    if ((c.plan_plane == 1 || c.plan_plane == 2) && !plane_supported(c)) c.plan_plane = sepp_supported(c) ? 3 : 0;
    if (c.plan_plane == 3 && !sepp_supported(c)) c.plan_plane = 0;
    if (c.plan_plane == 4 && !dd_supported(c)) c.plan_plane = sepp_supported(c) ? 3 : 0;
    if (c.scheme == 1) {
      cudaError_t e = prepare_rqm4(c);
      if (e != cudaSuccess) return e;
    } else if (c.concurrent && c.ckK == 1) {
      cudaError_t e = prepare_concurrent(c);
      if (e != cudaSuccess) return e;
      if (c.autotune && !c.tuned && !c.edw && !c.profiling) {
        if ((e = tune_plan(c)) != cudaSuccess) return e;
      }
    } else if (ck_sepp_applies(c)) {
      cudaError_t e = prepare_ck_sepp(c);
      if (e != cudaSuccess) return e;
    }
    if (!c.use_graph || c.profiling) return record_solve(c);
    if (!c.graph_valid) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      e = record_solve(c);
      cudaError_t e2 = cudaStreamEndCapture(c.stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
      }
      if (e2 != cudaSuccess) return e2;
      size_t nn = 0;
      if ((e = cudaGraphGetNodes(g, nullptr, &nn)) == cudaSuccess) {
        std::vector<cudaGraphNode_t> nodes(nn);
        e = cudaGraphGetNodes(g, nodes.data(), &nn);
        long long k = 0;
        for (size_t i = 0; i < nn && e == cudaSuccess; i++) {
          cudaGraphNodeType ty;
          e = cudaGraphNodeGetType(nodes[i], &ty);
          if (ty == cudaGraphNodeTypeKernel) k++;
        }
        c.graph_kernels = k;
      }
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
      }
      e = cudaGraphInstantiate(&c.graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
      c.graph_valid = true;
    }
    return cudaGraphLaunch(c.graph, c.stream);
  }

  // -------------------------------------------------------------- a7: step
  cudaError_t field_step(CtxData& c, int step_kind, double lam, const double* eta_p, const double* eta_m) override {
    mark(c, KK_FIELD_STEP);
    if (step_kind == PFT_STEP_SCFT_SIS || step_kind == PFT_STEP_CL_SIS) return sis_step(c, step_kind, lam, eta_p, eta_m);
    if (c.edw) {
      if (step_kind == PFT_STEP_SCFT_EULER) {
        k_step_edw_scft<T><<<c.npart, PW_THREADS, 0, c.stream>>>((double*)c.wp, (const double*)c.accA, (T*)c.BA, lam,
                                                                 c.ds, c.bC, c.M, c.partials);
      } else {
        const double dV = c.L[0] * c.L[1] * c.L[2] / (double)c.M;
        const double std = sqrt(2.0 * lam / (c.C * dV));
        k_step_edw_cl<T><<<c.npart, PW_THREADS, 0, c.stream>>>((double2*)c.wp, (const double2*)c.accA, (Z*)c.BA, lam, std,
                                                               eta_p, c.seed, c.instance, (unsigned long long)c.step,
                                                               c.step_dev, c.ds, c.bC, c.M, c.partials);
      }
      k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_FIELD);
      return cudaGetLastError();
    }
    if (step_kind == PFT_STEP_SCFT_EULER) {
      if (std::is_same<T, float>::value && c.M % 2 == 0) {
        k_step_scft2<<<c.npart, PW_THREADS, 0, c.stream>>>((double*)c.wp, (double*)c.wm, (const double*)c.accA,
                                                           (const double*)c.accB, (float*)c.BA, (float*)c.BB, lam, c.ds,
                                                           c.chiN, c.M, c.partials);
      } else {
        k_step_scft<T><<<c.npart, PW_THREADS, 0, c.stream>>>((double*)c.wp, (double*)c.wm, (const double*)c.accA,
                                                             (const double*)c.accB, (T*)c.BA, (T*)c.BB, lam, c.ds,
                                                             c.chiN, c.M, c.partials);
      }
    } else {
      const double dV = c.L[0] * c.L[1] * c.L[2] / (double)c.M;
      const double std = sqrt(2.0 * lam / (c.C * dV));
      k_step_cl<T><<<c.npart, PW_THREADS, 0, c.stream>>>((double2*)c.wp, (double2*)c.wm, (const double2*)c.accA,
                                                         (const double2*)c.accB, (Z*)c.BA, (Z*)c.BB, lam, std, eta_p,
                                                         eta_m, c.seed, c.instance, (unsigned long long)c.step,
                                                         c.step_dev, c.ds, c.chiN, c.M, c.partials);
    }
    k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_FIELD);
    return half_boltz(c);
  }

  // ------------------------------------------- semi-implicit step (Eq. 11)
  // Force and exchange-field update, FP64 transform of the W+ increment, division by
  // 1 + a g_D(k), inverse transform, W+ update with the new Boltzmann factors.
  cudaError_t sis_step(CtxData& c, int step_kind, double a, const double* eta_p, const double* eta_m) {
    cudaError_t e;
    if (!c.sis) {
      if ((e = cudaMalloc(&c.sis, (size_t)c.M * sizeof(double2))) != cudaSuccess) return e;
      c.bytes += (size_t)c.M * sizeof(double2);
    }
    double2* G = (double2*)c.sis;
    if (step_kind == PFT_STEP_SCFT_SIS) {
      k_sis_force_real<<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)c.accA, (const double*)c.accB,
                                                             (double*)c.wm, G, a, c.chiN, c.M);
    } else {
      const double dV = c.L[0] * c.L[1] * c.L[2] / (double)c.M;
      const double std = sqrt(2.0 * a / (c.C * dV));
      k_sis_force_cplx<<<c.npart, PW_THREADS, 0, c.stream>>>((const double2*)c.accA, (const double2*)c.accB,
                                                             (double2*)c.wm, G, a, std, eta_p, eta_m, c.seed,
                                                             c.instance, (unsigned long long)c.step, c.step_dev,
                                                             c.chiN, c.M);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = fft3d_f64(c, G, false)) != cudaSuccess) return e;
    k_sis_scale<<<c.npart, PW_THREADS, 0, c.stream>>>(G, tab<double>(c, c.g_off[0]), tab<double>(c, c.g_off[1]),
                                                      tab<double>(c, c.g_off[2]), c.n[1], c.n[2], a, c.M);
    if ((e = fft3d_f64(c, G, true)) != cudaSuccess) return e;
    if (c.kind == PFT_SCFT_REAL) {
      k_sis_apply_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>((double*)c.wp, (const double*)c.wm, G, (T*)c.BA,
                                                                (T*)c.BB, 1.0 / (double)c.M, c.ds, c.chiN, c.M,
                                                                c.partials);
    } else {
      k_sis_apply_cplx<T><<<c.npart, PW_THREADS, 0, c.stream>>>((double2*)c.wp, (const double2*)c.wm, G, (Z*)c.BA,
                                                                (Z*)c.BB, 1.0 / (double)c.M, c.ds, c.chiN, c.M,
                                                                c.partials);
    }
    k_reduce_final<2><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_FIELD);
    return half_boltz(c);
  }

  // Complex FP64 3D transform in place (unnormalised both ways) with the FP64 twiddles.
  cudaError_t fft3d_f64(CtxData& c, double2* d, bool inverse) {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const double2* twx = tab<double2>(c, c.t64_off[0]);
    const double2* twy = tab<double2>(c, c.t64_off[1]);
    const double2* twz = tab<double2>(c, c.t64_off[2]);
    const long long npen = (long long)nx * ny;
    cudaError_t e;
    if (!inverse) {
      PFT_DISPATCH_AXIS(nz, e = (d_zf_c2c<N>(c, d, npen, twz)));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(ny, e = (d_strided<N, 0>(c, d, (long long)nx * nz, nz, (long long)ny * nz, nz, twy)));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(nx, e = (d_strided<N, 0>(c, d, (long long)ny * nz, (long long)ny * nz, 0, (long long)ny * nz, twx)));
    } else {
      PFT_DISPATCH_AXIS(nx, e = (d_strided<N, 1>(c, d, (long long)ny * nz, (long long)ny * nz, 0, (long long)ny * nz, twx)));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(ny, e = (d_strided<N, 1>(c, d, (long long)nx * nz, nz, (long long)ny * nz, nz, twy)));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(nz, e = (d_zi_c2c<N>(c, d, npen, twz)));
    }
    return e;
  }

  // ---------------------------------------------------------- test hook: FFT
  cudaError_t fft3d(CtxData& c, void* data, int inverse) override {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const Z* twx = tab<Z>(c, c.tw_off[0]);
    const Z* twy = tab<Z>(c, c.tw_off[1]);
    const Z* twz = tab<Z>(c, c.tw_off[2]);
    Z* d = (Z*)data;
    const long long npen = (long long)nx * ny;
    cudaError_t e;
    if (!inverse) {
      PFT_DISPATCH_AXIS(nz, e = launch_zf_c2c<N>(c, d, nullptr, d, npen, twz));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(ny, e = launch_strided<N, 0>(c, d, (long long)nx * nz, nz, (long long)ny * nz, nz, twy, nullptr,
                                                     nullptr, nullptr, nz));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(nx, e = launch_strided<N, 0>(c, d, (long long)ny * nz, (long long)ny * nz, 0, (long long)ny * nz,
                                                     twx, nullptr, nullptr, nullptr, nz));
    } else {
      PFT_DISPATCH_AXIS(nx, e = launch_strided<N, 1>(c, d, (long long)ny * nz, (long long)ny * nz, 0, (long long)ny * nz,
                                                     twx, nullptr, nullptr, nullptr, nz));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(ny, e = launch_strided<N, 1>(c, d, (long long)nx * nz, nz, (long long)ny * nz, nz, twy, nullptr,
                                                     nullptr, nullptr, nz));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(nz, e = launch_zi_c2c<N, 2>(c, d, nullptr, d, nullptr, nullptr, nullptr, 0.0, 0.0, npen, twz));
    }
    return e;
  }

  // ------------------------------------------------------- a8: gradients
  // Field gradients from the densities of the last solve, and the box derivative of
  // lnQ: the conjugate march is run again and, at every step, the forward spectra
  // u^ = F[B_n qd_{Ns-n}] and v^ = F[B_n q_{n-1}] are contracted with
  // k_a^2 exp(-k^2 ds) over the half spectrum (S_STRESS; the host applies
  // 2 ds / (L_a Q M^2)).  Real SCFT fields only.
  cudaError_t gradients(CtxData& c, double* dwp, double* dwm) override {
    if (c.kind != PFT_SCFT_REAL || c.scheme != 0) return cudaErrorNotSupported;
    const double dV = c.L[0] * c.L[1] * c.L[2] / (double)c.M;
    if (dwp || dwm) {
      k_grad_fields<<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)c.accA, (const double*)c.accB,
                                                          (const double*)c.wm, dwp, dwm, c.C * dV, c.chiN, c.M);
    }
    cudaError_t e = cudaMemsetAsync(c.partials, 0, (size_t)c.npart * 3 * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    if (c.concurrent && c.qdh && c.ckK == 1) return gradients_from_histories(c);
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const Z* twx = tab<Z>(c, c.tw_off[0]);
    const Z* twy = tab<Z>(c, c.tw_off[1]);
    const Z* twz = tab<Z>(c, c.tw_off[2]);
    const Z* twh = tab<Z>(c, c.tw_off[3]);
    const T* dx = tab<T>(c, c.d_off[0]);
    const T* dy = tab<T>(c, c.d_off[1]);
    const T* dz = tab<T>(c, c.d_off[2]);
    const double* gx = tab<double>(c, c.g_off[0]);
    const double* gy = tab<double>(c, c.g_off[1]);
    const double* gz = tab<double>(c, c.g_off[2]);
    Z* u = (Z*)c.spec;
    Z* v = (Z*)c.spec2;
    const long long npen = (long long)nx * ny;
    const long long nzc = c.nzh;
    for (int m = 1; m <= c.Ns; m++) {
      const int nb = c.Ns + 1 - m;
      const T* B = (const T*)((nb <= c.NsA) ? c.BA : c.BB);
      const T* in = (const T*)((m == 1) ? c.qd0 : c.qd[(m - 1) & 1]);
      T* out = (T*)c.qd[m & 1];
      if ((e = recompute_segment(c, nb - 1)) != cudaSuccess) return e;
      const T* qprev = (const T*)q_at(c, nb - 1);
      for (int w = 0; w < 2; w++) {
        Z* sp = w ? v : u;
        PFT_DISPATCH_HALF(nz / 2, e = launch_zf_r2c<N>(c, w ? qprev : in, B, sp, npen, twh, twz));
        if (e != cudaSuccess) return e;
        PFT_DISPATCH_AXIS(ny, e = launch_strided<N, 0>(c, sp, nx * nzc, nzc, ny * nzc, nzc, twy, dx, dy, dz, (int)nzc));
        if (e != cudaSuccess) return e;
        PFT_DISPATCH_AXIS(nx, e = launch_strided<N, 0>(c, sp, ny * nzc, ny * nzc, 0, ny * nzc, twx, dx, dy, dz, (int)nzc));
        if (e != cudaSuccess) return e;
      }
      k_stress_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>(u, v, gx, gy, gz, tab<double>(c, c.e_off[0]),
                                                            tab<double>(c, c.e_off[1]), tab<double>(c, c.e_off[2]), nx,
                                                            ny, (int)nzc, nz, c.partials);
      PFT_DISPATCH_AXIS(nx, e = launch_strided<N, 3>(c, u, ny * nzc, ny * nzc, 0, ny * nzc, twx, dx, dy, dz, (int)nzc));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_AXIS(ny, e = launch_strided<N, 1>(c, u, nx * nzc, nzc, ny * nzc, nzc, twy, dx, dy, dz, (int)nzc));
      if (e != cudaSuccess) return e;
      PFT_DISPATCH_HALF(nz / 2, e = launch_zi_c2r<N, 0>(c, u, B, out, nullptr, nullptr, nullptr, 0.0, 0.0, npen, twh,
                                                        twz));
      if (e != cudaSuccess) return e;
    }
    k_reduce_final<3><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_STRESS);
    return cudaGetLastError();
  }

  // Box derivative from the two stored histories of the last (concurrent) solve: for each
  // split step n the forward spectra of B_n qd_{Ns-n} and B_n q_{n-1} (two members of
  // batched z and y forward passes, or of the plane kernel's first step, then the x
  // forward pass), then the contraction.
  cudaError_t gradients_from_histories(CtxData& c) {
    const size_t slice = (size_t)c.M * sizeof(T);
    cudaError_t e;
    if (!c.stepsg) {
      std::vector<BatchStep> h((size_t)2 * c.Ns);
      const char* hist = (const char*)c.hist;
      const char* qdh = (const char*)c.qdh;
      const char* t = (const char*)c.tables;
      for (int n = 1; n <= c.Ns; n++) {
        BatchStep& u = h[(size_t)2 * (n - 1)];
        BatchStep& v = h[(size_t)2 * (n - 1) + 1];
        memset(&u, 0, sizeof(u));
        memset(&v, 0, sizeof(v));
        const int m = c.Ns - n;
        u.in = (m == 0) ? c.qd0 : (const void*)(qdh + (size_t)m * slice);
        v.in = hist + (size_t)(n - 1) * slice;
        u.B = v.B = (n <= c.NsA) ? c.BA : c.BB;
        u.spec = c.spec;
        v.spec = c.spec2;
        for (int a = 0; a < 4; a++) u.tw[a] = v.tw[a] = t + c.tw_off[a];
        for (int a = 0; a < 3; a++) u.d[a] = v.d[a] = t + c.d_off[a];
      }
      e = cudaMalloc(&c.stepsg, h.size() * sizeof(BatchStep));
      if (e != cudaSuccess) return e;
      c.bytes += h.size() * sizeof(BatchStep);
      e = cudaMemcpy(c.stepsg, h.data(), h.size() * sizeof(BatchStep), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
    }
    BatchGeom g;
    for (int a = 0; a < 3; a++) g.n[a] = c.n[a];
    g.kind = c.kind;
    g.nzh = c.nzh;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const long long nzc = c.nzh;
    const double* gx = tab<double>(c, c.g_off[0]);
    const double* gy = tab<double>(c, c.g_off[1]);
    const double* gz = tab<double>(c, c.g_off[2]);
    const BatchStep* st = (const BatchStep*)c.stepsg;
    const bool plane = plane_supported(c) && c.plan_plane;
    for (int n = 1; n <= c.Ns; n++) {
      const BatchStep* ss = st + (size_t)2 * (n - 1);
      if (plane) {  // rows x B, z and y forward in one kernel (the plane kernel's first step)
        if ((e = batch_plane(c, ss, 0, 2, c.stream)) != cudaSuccess) return e;
      } else {
        if ((e = batch_zf(g, ss, 2, c.stream)) != cudaSuccess) return e;
        PFT_BATCH_AXIS(ny, e = (bs<N, 0>(ss, nx * nzc, nzc, ny * nzc, nzc, (int)nzc, 1, 2, c.stream)));
        if (e != cudaSuccess) return e;
      }
      PFT_BATCH_AXIS(nx, e = (bs<N, 0>(ss, ny * nzc, ny * nzc, 0, ny * nzc, (int)nzc, 0, 2, c.stream)));
      if (e != cudaSuccess) return e;
      k_stress_real<T><<<c.npart, PW_THREADS, 0, c.stream>>>((const Z*)c.spec, (const Z*)c.spec2, gx, gy, gz,
                                                            tab<double>(c, c.e_off[0]), tab<double>(c, c.e_off[1]),
                                                            tab<double>(c, c.e_off[2]), nx, ny, (int)nzc, nz,
                                                            c.partials);
    }
    k_reduce_final<3><<<1, PW_THREADS, 0, c.stream>>>(c.partials, c.npart, c.scal + S_STRESS);
    return cudaGetLastError();
  }

  cudaError_t to_f64(CtxData& c, const void* src, void* dst, long long cnt) override {
    k_convert<T, double><<<c.npart, PW_THREADS, 0, c.stream>>>((const T*)src, (double*)dst, cnt);
    return cudaGetLastError();
  }
  cudaError_t from_f64(CtxData& c, const void* src, void* dst, long long cnt) override {
    k_convert<double, T><<<c.npart, PW_THREADS, 0, c.stream>>>((const double*)src, (T*)dst, cnt);
    return cudaGetLastError();
  }

 private:
  // FP64 complex transform launches (independent of the working precision T)
  template <int N, int MODE>
  static cudaError_t d_strided(CtxData& c, double2* data, long long ncols, long long cin, long long s_outer,
                               long long s_k, const double2* tw) {
    constexpr int C = Tile<double>::C;
    const long long blocks = (ncols + C - 1) / C;
    k_strided<double, N, MODE><<<(unsigned)blocks, C * Plan<N>::TPC, (size_t)N * C * sizeof(double2), c.stream>>>(
        data, ncols, cin, s_outer, s_k, tw, nullptr, nullptr, nullptr, 1);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t d_zf_c2c(CtxData& c, double2* d, long long npen, const double2* tw) {
    constexpr int P = PencilsPerCta<double, N>::v;
    k_zf_c2c<double, N><<<(unsigned)((npen + P - 1) / P), P * Plan<N>::TPC, (size_t)P * pencil_ld<double>(N) * sizeof(double2),
                          c.stream>>>(d, nullptr, d, npen, tw);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t d_zi_c2c(CtxData& c, double2* d, long long npen, const double2* tw) {
    constexpr int P = PencilsPerCta<double, N>::v;
    k_zi_c2c<double, N, 2><<<(unsigned)((npen + P - 1) / P), P * Plan<N>::TPC,
                             (size_t)P * pencil_ld<double>(N) * sizeof(double2), c.stream>>>(
        d, nullptr, d, nullptr, nullptr, nullptr, 0.0, 0.0, npen, tw);
    return cudaGetLastError();
  }

  template <int N, int MODE>
  static cudaError_t bs(const BatchStep* st, long long ncols, long long cin, long long s_outer, long long s_k, int nzc,
                        int axis, int nact, cudaStream_t stream) {
    constexpr int C = Tile<T>::C;
    const dim3 grid((unsigned)((ncols + C - 1) / C), (unsigned)nact);
    kb_strided<T, N, MODE><<<grid, C * Plan<N>::TPC, (size_t)N * C * sizeof(Z), stream>>>(st, ncols, cin, s_outer, s_k,
                                                                                          nzc, axis);
    return cudaGetLastError();
  }
  template <int N2>
  static cudaError_t bz_r2c(const BatchStep* st, long long npen, int nact, cudaStream_t stream) {
    constexpr int P = PencilsPerCta<T, N2>::v;
    const dim3 grid((unsigned)((npen + P - 1) / P), (unsigned)nact);
    kb_zf_r2c<T, N2><<<grid, P * Plan<N2>::TPC, (size_t)P * pencil_ld<T>(N2) * sizeof(Z), stream>>>(st, npen);
    return cudaGetLastError();
  }
  template <int N2, int EPI>
  static cudaError_t bzi_c2r(const BatchStep* st, long long npen, int nact, cudaStream_t stream) {
    constexpr int P = PencilsPerCta<T, N2>::v;
    const dim3 grid((unsigned)((npen + P - 1) / P), (unsigned)nact);
    kb_zi_c2r<T, N2, EPI><<<grid, P * Plan<N2>::TPC, (size_t)P * pencil_ld<T>(N2) * sizeof(Z), stream>>>(st, npen);
    return cudaGetLastError();
  }
  template <int N2>
  static cudaError_t bzz_r2c(const BatchStep* st, long long npen, int nact, cudaStream_t stream) {
    constexpr int P = PencilsPerCta<T, N2>::v;
    const dim3 grid((unsigned)((npen + P - 1) / P), (unsigned)nact);
    kb_zz_r2c<T, N2><<<grid, P * Plan<N2>::TPC, (size_t)P * pencil_ld<T>(N2) * sizeof(Z), stream>>>(st, npen);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t bzz_c2c(const BatchStep* st, long long npen, int nact, cudaStream_t stream) {
    constexpr int P = PencilsPerCta<T, N>::v;
    const dim3 grid((unsigned)((npen + P - 1) / P), (unsigned)nact);
    kb_zz_c2c<T, N><<<grid, P * Plan<N>::TPC, (size_t)P * pencil_ld<T>(N) * sizeof(Z), stream>>>(st, npen);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t bz_c2c(const BatchStep* st, long long npen, int nact, cudaStream_t stream) {
    constexpr int P = PencilsPerCta<T, N>::v;
    const dim3 grid((unsigned)((npen + P - 1) / P), (unsigned)nact);
    kb_zf_c2c<T, N><<<grid, P * Plan<N>::TPC, (size_t)P * pencil_ld<T>(N) * sizeof(Z), stream>>>(st, npen);
    return cudaGetLastError();
  }
  template <int N, int EPI>
  static cudaError_t bzi_c2c(const BatchStep* st, long long npen, int nact, cudaStream_t stream) {
    constexpr int P = PencilsPerCta<T, N>::v;
    const dim3 grid((unsigned)((npen + P - 1) / P), (unsigned)nact);
    kb_zi_c2c<T, N, EPI><<<grid, P * Plan<N>::TPC, (size_t)P * pencil_ld<T>(N) * sizeof(Z), stream>>>(st, npen);
    return cudaGetLastError();
  }

  template <typename P> static const P* tab(const CtxData& c, size_t off) {
    return reinterpret_cast<const P*>(reinterpret_cast<const char*>(c.tables) + off);
  }

  template <int N, int MODE>
  cudaError_t launch_strided(CtxData& c, Z* data, long long ncols, long long cin, long long s_outer, long long s_k,
                             const Z* tw, const T* dk, const T* dy, const T* dz, int nzc) {
    constexpr int C = Tile<T>::C;
    const int threads = C * Plan<N>::TPC;
    const size_t smem = (size_t)N * C * sizeof(Z);
    const long long blocks = (ncols + C - 1) / C;
    k_strided<T, N, MODE><<<(unsigned)blocks, threads, smem, c.stream>>>(data, ncols, cin, s_outer, s_k, tw, dk, dy, dz,
                                                                         nzc);
    return cudaGetLastError();
  }

  template <int N2>
  cudaError_t launch_zf_r2c(CtxData& c, const T* q, const T* B, Z* spec, long long npen, const Z* twh, const Z* twf) {
    constexpr int P = PencilsPerCta<T, N2>::v;
    const int threads = P * Plan<N2>::TPC;
    const size_t smem = (size_t)P * pencil_ld<T>(N2) * sizeof(Z);
    const long long blocks = (npen + P - 1) / P;
    k_zf_r2c<T, N2><<<(unsigned)blocks, threads, smem, c.stream>>>(q, B, spec, npen, twh, twf);
    return cudaGetLastError();
  }

  template <int N2, int EPI>
  cudaError_t launch_zi_c2r(CtxData& c, const Z* spec, const T* B, T* out, const T* partner, double* accA, double* accB,
                            double cA, double cB, long long npen, const Z* twh, const Z* twf) {
    constexpr int P = PencilsPerCta<T, N2>::v;
    const int threads = P * Plan<N2>::TPC;
    const size_t smem = (size_t)P * pencil_ld<T>(N2) * sizeof(Z);
    const long long blocks = (npen + P - 1) / P;
    k_zi_c2r<T, N2, EPI><<<(unsigned)blocks, threads, smem, c.stream>>>(spec, B, out, partner, accA, accB, cA, cB, npen,
                                                                         twh, twf);
    return cudaGetLastError();
  }

  template <int N>
  cudaError_t launch_zf_c2c(CtxData& c, const Z* q, const Z* B, Z* spec, long long npen, const Z* tw) {
    constexpr int P = PencilsPerCta<T, N>::v;
    const int threads = P * Plan<N>::TPC;
    const size_t smem = (size_t)P * pencil_ld<T>(N) * sizeof(Z);
    const long long blocks = (npen + P - 1) / P;
    k_zf_c2c<T, N><<<(unsigned)blocks, threads, smem, c.stream>>>(q, B, spec, npen, tw);
    return cudaGetLastError();
  }

  template <int N, int EPI>
  cudaError_t launch_zi_c2c(CtxData& c, const Z* spec, const Z* B, Z* out, const Z* partner, double2* accA,
                            double2* accB, double cA, double cB, long long npen, const Z* tw) {
    constexpr int P = PencilsPerCta<T, N>::v;
    const int threads = P * Plan<N>::TPC;
    const size_t smem = (size_t)P * pencil_ld<T>(N) * sizeof(Z);
    const long long blocks = (npen + P - 1) / P;
    k_zi_c2c<T, N, EPI><<<(unsigned)blocks, threads, smem, c.stream>>>(spec, B, out, partner, accA, accB, cA, cB, npen,
                                                                        tw);
    return cudaGetLastError();
  }
};

}  // namespace pft
