// pft_static.cu -- a contour step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another framework owns
// the device allocator, plug-ins that may only touch memory they are handed, or
// steps enqueued after a process has fixed its memory budget.  This entry point takes
// the same split step as the library's contexts (FP64, real fields) but keeps its
// scratch -- the Boltzmann factor, the half spectrum and the twiddle/diffusion
// tables -- in one file-scope static device array of fixed size.  Every GPU that
// loads the library holds that array until the process exits.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "pft_engine.h"
#include "pft_passes.cuh"

namespace pft {
namespace {
constexpr long long kStaticMaxPointsDecl = 64LL * 64 * 64;
constexpr size_t kStaticBytesDecl =
    (size_t)kStaticMaxPointsDecl * (sizeof(double) + sizeof(double2)) + 64 * 1024;
}  // namespace
}  // namespace pft

// The scratch: Boltzmann factor | half spectrum | tables.  Host code must not pass this
// symbol to a kernel -- on the host it is a stand-in, not a device address; its device
// address is looked up per device (scratch_address below).
static __device__ __align__(256) unsigned char g_static_scratch[pft::kStaticBytesDecl];

namespace pft {
namespace {

constexpr long long kStaticMaxPoints = 64LL * 64 * 64;        // largest grid the scratch holds
constexpr size_t kTableBytes = 64 * 1024;                        // twiddles + diffusion tables
constexpr size_t kBBytes = (size_t)kStaticMaxPoints * sizeof(double);
constexpr size_t kSpecBytes = (size_t)kStaticMaxPoints * sizeof(double2);
constexpr size_t kStaticBytes = kBBytes + kSpecBytes + kTableBytes;
constexpr int kMaxDevices = 64;

static_assert(kStaticBytes == kStaticBytesDecl, "scratch layout");

std::mutex g_mu;
unsigned char* g_dev_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_dev_addr[dev] = (unsigned char*)p;
  }
  *out = g_dev_addr[dev];
  return cudaSuccess;
}

// Twiddles exp(-2 pi i m/len) of the four transform lengths and the per-axis
// diffusion factors exp(-k^2 ds) (1/M folded into the x factor), computed on device.
struct TableLayout {
  int len[4];      // nx, ny, nz, nz/2
  size_t tw[4];    // element offsets (double2) of the twiddle tables
  size_t d[3];     // element offsets (double) of the diffusion tables
  int dn[3];       // nx, ny, nz/2+1
};

__global__ void k_static_tables(double2* __restrict__ tw, double* __restrict__ dtab, TableLayout t, double Lx,
                                double Ly, double Lz, double ds, double invM) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int a = 0; a < 4; a++) {
    if (i < t.len[a]) {
      double s, c;
      sincospi(-2.0 * (double)i / (double)t.len[a], &s, &c);
      tw[t.tw[a] + i] = make_double2(c, s);
    }
  }
  const double L[3] = {Lx, Ly, Lz};
  const int n[3] = {t.len[0], t.len[1], t.len[2]};
  for (int a = 0; a < 3; a++) {
    if (i < t.dn[a]) {
      const int mm = (i <= n[a] / 2) ? i : i - n[a];
      const double k = 2.0 * 3.14159265358979323846 * (double)mm / L[a];
      double v = exp(-k * k * ds);
      if (a == 0) v *= invM;
      dtab[t.d[a] + i] = v;
    }
  }
}

__global__ void k_static_boltzmann(const double* __restrict__ w, double* __restrict__ B, double ds, long long M) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    B[i] = exp(-w[i] * ds * 0.5);
}

#define PFT_S_CASE(NV, ...) \
  case NV: {                \
    constexpr int N = NV;   \
    __VA_ARGS__;            \
  } break;
#define PFT_S_AXIS(n, ...)                                                                                       \
  switch (n) {                                                                                                   \
    PFT_S_CASE(4, __VA_ARGS__) PFT_S_CASE(6, __VA_ARGS__) PFT_S_CASE(8, __VA_ARGS__) PFT_S_CASE(12, __VA_ARGS__) \
    PFT_S_CASE(16, __VA_ARGS__) PFT_S_CASE(24, __VA_ARGS__) PFT_S_CASE(32, __VA_ARGS__)                           \
    PFT_S_CASE(48, __VA_ARGS__) PFT_S_CASE(64, __VA_ARGS__)                                                      \
    default: return cudaErrorInvalidValue;                                                                       \
  }
#define PFT_S_HALF(n, ...)                                                                                       \
  switch (n) {                                                                                                   \
    PFT_S_CASE(2, __VA_ARGS__) PFT_S_CASE(3, __VA_ARGS__) PFT_S_CASE(4, __VA_ARGS__) PFT_S_CASE(6, __VA_ARGS__)  \
    PFT_S_CASE(8, __VA_ARGS__) PFT_S_CASE(12, __VA_ARGS__) PFT_S_CASE(16, __VA_ARGS__)                           \
    PFT_S_CASE(24, __VA_ARGS__) PFT_S_CASE(32, __VA_ARGS__)                                                      \
    default: return cudaErrorInvalidValue;                                                                       \
  }

template <int N, int MODE>
cudaError_t strided(double2* data, long long ncols, long long cin, long long s_outer, long long s_k, const double2* tw,
                    const double* dk, const double* dy, const double* dz, int nzc, cudaStream_t st) {
  constexpr int C = Tile<double>::C;
  const long long blocks = (ncols + C - 1) / C;
  k_strided<double, N, MODE><<<(unsigned)blocks, C * Plan<N>::TPC, (size_t)N * C * sizeof(double2), st>>>(
      data, ncols, cin, s_outer, s_k, tw, dk, dy, dz, nzc);
  return cudaGetLastError();
}

template <int N2>
cudaError_t zf(const double* q, const double* B, double2* spec, long long npen, const double2* twh, const double2* twf,
               cudaStream_t st) {
  constexpr int P = PencilsPerCta<double, N2>::v;
  k_zf_r2c<double, N2><<<(unsigned)((npen + P - 1) / P), P * Plan<N2>::TPC,
                         (size_t)P * pencil_ld<double>(N2) * sizeof(double2), st>>>(q, B, spec, npen, twh, twf);
  return cudaGetLastError();
}

template <int N2>
cudaError_t zi(const double2* spec, const double* B, double* out, long long npen, const double2* twh,
               const double2* twf, cudaStream_t st) {
  constexpr int P = PencilsPerCta<double, N2>::v;
  k_zi_c2r<double, N2, 0><<<(unsigned)((npen + P - 1) / P), P * Plan<N2>::TPC,
                            (size_t)P * pencil_ld<double>(N2) * sizeof(double2), st>>>(
      spec, B, out, nullptr, nullptr, nullptr, 0.0, 0.0, npen, twh, twf);
  return cudaGetLastError();
}

cudaError_t static_step(const int n[3], const double L[3], double ds, const double* w, const double* qin, double* qout,
                        cudaStream_t st) {
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return e;
  const int nx = n[0], ny = n[1], nz = n[2];
  const long long M = (long long)nx * ny * nz;
  const int nzc = nz / 2 + 1;
  double* B = (double*)base;
  double2* spec = (double2*)(base + kBBytes);
  unsigned char* tabs = base + kBBytes + kSpecBytes;
  TableLayout t;
  t.len[0] = nx;
  t.len[1] = ny;
  t.len[2] = nz;
  t.len[3] = nz / 2;
  size_t off = 0;
  for (int a = 0; a < 4; a++) {
    t.tw[a] = off;
    off += (size_t)t.len[a];
  }
  double2* tw = (double2*)tabs;
  double* dtab = (double*)(tabs + off * sizeof(double2));
  t.dn[0] = nx;
  t.dn[1] = ny;
  t.dn[2] = nzc;
  size_t doff = 0;
  for (int a = 0; a < 3; a++) {
    t.d[a] = doff;
    doff += (size_t)t.dn[a];
  }
  k_static_tables<<<1, 256, 0, st>>>(tw, dtab, t, L[0], L[1], L[2], ds, 1.0 / (double)M);
  k_static_boltzmann<<<256, 256, 0, st>>>(w, B, ds, M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const double2* twx = tw + t.tw[0];
  const double2* twy = tw + t.tw[1];
  const double2* twz = tw + t.tw[2];
  const double2* twh = tw + t.tw[3];
  const double* dx = dtab + t.d[0];
  const double* dy = dtab + t.d[1];
  const double* dz = dtab + t.d[2];
  const long long npen = (long long)nx * ny;
  PFT_S_HALF(nz / 2, e = zf<N>(qin, B, spec, npen, twh, twz, st));
  if (e != cudaSuccess) return e;
  PFT_S_AXIS(ny, e = (strided<N, 0>(spec, (long long)nx * nzc, nzc, (long long)ny * nzc, nzc, twy, dx, dy, dz, nzc, st)));
  if (e != cudaSuccess) return e;
  PFT_S_AXIS(nx, e = (strided<N, 2>(spec, (long long)ny * nzc, (long long)ny * nzc, 0, (long long)ny * nzc, twx, dx, dy,
                                    dz, nzc, st)));
  if (e != cudaSuccess) return e;
  PFT_S_AXIS(ny, e = (strided<N, 1>(spec, (long long)nx * nzc, nzc, (long long)ny * nzc, nzc, twy, dx, dy, dz, nzc, st)));
  if (e != cudaSuccess) return e;
  PFT_S_HALF(nz / 2, e = zi<N>(spec, B, qout, npen, twh, twz, st));
  return e;
}

}  // namespace
}  // namespace pft

extern "C" pft_status pft_contour_step_static(const int n[3], const double L[3], int Ns, const double* w,
                                              const double* q_in, double* q_out, void* stream) {
  if (!n || !L || !w || !q_in || !q_out) {
    pft::set_error("pft_contour_step_static: NULL argument");
    return PFT_ERR_ARG;
  }
  if (Ns < 1) {
    pft::set_error("pft_contour_step_static: Ns must be >= 1");
    return PFT_ERR_ARG;
  }
  for (int a = 0; a < 3; a++) {
    if (!pft::axis_supported(n[a])) {
      pft::set_error("pft_contour_step_static: grid size " + std::to_string(n[a]) + " has no FFT plan");
      return PFT_ERR_SHAPE;
    }
    if (n[a] > 64) {
      pft::set_error("pft_contour_step_static: n[" + std::to_string(a) + "]=" + std::to_string(n[a]) +
                     " exceeds the static scratch limit of 64 points per axis (64^3 points in all)");
      return PFT_ERR_ARG;
    }
    if (!(L[a] > 0.0) || !isfinite(L[a])) {
      pft::set_error("pft_contour_step_static: box lengths must be positive");
      return PFT_ERR_ARG;
    }
  }
  const long long M = (long long)n[0] * n[1] * n[2];
  if (M > pft::kStaticMaxPoints) {
    pft::set_error("pft_contour_step_static: grid of " + std::to_string(M) + " points exceeds the static scratch (" +
                   std::to_string(pft::kStaticMaxPoints) + " points)");
    return PFT_ERR_ARG;
  }
  cudaError_t e = pft::static_step(n, L, 1.0 / Ns, w, q_in, q_out, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    pft::set_error(std::string("pft_contour_step_static: ") + cudaGetErrorString(e));
    (void)cudaGetLastError();
    return PFT_ERR_CUDA;
  }
  return PFT_OK;
}
