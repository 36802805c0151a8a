// pft_engine.h -- host-side state of one system and the precision-specific engine
// interface (the kernels live in pft_engine_impl.cuh, instantiated per precision).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <string>
#include <vector>

#include "../../include/pft.h"

namespace pft {

// Offsets into the device scalar block (doubles).
enum ScalarSlot {
  S_QSUM = 0,       // sum_x q_Ns (re, im)
  S_FIELD = 2,      // sum_x [W-^2/chiN - i w+]   (re, im) of the fields the solve used
  S_PHIA = 4,       // sum_x phiA (re, im)
  S_PHIB = 6,       // sum_x phiB (re, im)
  S_FP2 = 8,        // sum_x |force+|^2
  S_FM2 = 9,        // sum_x |force-|^2
  S_Q = 10,         // Q (re, im)
  S_LNQ = 12,       // lnQ (re, im)
  S_H = 14,         // H (re, im)
  S_STRESS = 16,    // sum over steps/modes of the box-derivative contraction (3)
  S_DLNQ = 20,      // dlnQ/dL_a (3)
  S_VOL = 24,       // box volume V (written by the host)
  S_GAMMA = 26,     // adjoint: sum_x (GA phiA + GB phiB) (2 slots of the reduction)
  S_COUNT = 32
};

struct CtxData {
  // system
  int n[3];
  double L[3];
  int Ns, NsA;
  double fA, ds;
  double chiN, C;
  pft_kind kind;
  pft_precision prec;
  long long M;     // grid points
  int nzh;         // nz/2+1 (real mode) or nz (complex mode): last spectrum extent
  long long Ms;    // spectrum elements nx*ny*nzh
  // runtime
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the concurrent marches run one chain per propagator: member 0 on `stream`, member 1
  // on `stream2`, forked from and joined back into `stream` (graph branches when captured)
  cudaStream_t stream2 = nullptr;
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev = nullptr;
  int device = 0;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  long long graph_kernels = -1;  // kernel nodes of the captured solve graph
  unsigned long long seed = 0, instance = 0;
  long long step = 0;
  bool fields_set = false, solved = false;
  int sms = 152;
  // device buffers (elements in brackets)
  void* wp = nullptr;     // [M] f64 or c128
  void* wm = nullptr;
  void* BA = nullptr;     // [M] working precision, real or complex
  void* BB = nullptr;
  void* hist = nullptr;   // [(Ns+1) * M] q_0..q_Ns
  void* qd[2] = {nullptr, nullptr};  // conjugate propagator ping-pong
  void* qd0 = nullptr;    // [M] initial condition of qd
  void* spec = nullptr;   // [M] complex working precision (>= Ms)
  void* spec2 = nullptr;  // [M] second spectrum (box derivative)
  void* accA = nullptr;   // [M] f64 or c128: quadrature sums, then phiA
  void* accB = nullptr;
  double* partials = nullptr;  // [npart * 16]: per-block partial sums of the reductions
  double* scal = nullptr;      // [S_COUNT]
  double* scal_host = nullptr; // pinned mirror
  void* tables = nullptr;      // twiddles + diffusion factors
  size_t tw_off[4] = {0, 0, 0, 0};  // x, y, z (full nz), z half (nz/2): byte offsets
  size_t d_off[3] = {0, 0, 0};      // dx (with 1/M), dy, dz
  size_t sd_off[3] = {0, 0, 0};     // per-axis factors exp(-k_a^2 ds)/n_a over the full axis (separable march)
  size_t g_off[3] = {0, 0, 0};      // k_a^2 per axis (FP64): box derivative, SIS Debye factor
  size_t e_off[3] = {0, 0, 0};      // exp(-k_a^2 ds) per axis (FP64): box derivative
  size_t t64_off[3] = {0, 0, 0};    // FP64 twiddles x, y, z (full nz) for the SIS transforms
  void* sis = nullptr;              // [M] complex FP64 scratch of the semi-implicit step
  void* adj = nullptr;              // adjoint scratch: 6 working-precision slices + 2 M FP64
  void* stepsa = nullptr;           // [2 Ns] BatchStep of the adjoint transforms
  void* stepsap = nullptr;          // [2 Ns] AdjPlaneStep of the adjoint on the plane kernel
  void* adjS = nullptr;             // adjoint on the separable march: lambda and mu histories, gA, gB
  void* stepsAS = nullptr;          // [2 Ns] its step entries
  size_t tables_bytes = 0;
  int npart = 0;
  int* kerr = nullptr;  // kernel error word: a bounded wait that ran out (read by pft_get_observables)
  size_t bytes = 0;
  // optional device counter read by the CL field step instead of `step` (batches)
  const unsigned long long* step_dev = nullptr;
  // concurrent marches (pass kernels): q and qd advance together, two members per
  // launch; the qd history is kept and the quadrature runs once over both histories
  bool concurrent = true;
  void* qdh = nullptr;      // [(Ns+1) * M] qd_0..qd_Ns (slice 0 unused: qd0 holds it)
  void* steps2 = nullptr;   // [2 * Ns] BatchStep: forward and conjugate step s
  void* stepsS = nullptr;   // [2 * Ns] the same steps with the separable march's tables
  // double-float separable march (plan 4, FP64 contexts): dd twiddles and per-axis factors,
  // the Boltzmann factors split into dd, and the step entries pointing at them
  void* ddbuf = nullptr;
  size_t ddtw_off[3] = {0, 0, 0};
  size_t ddsd_off[3] = {0, 0, 0};
  size_t ddB_off[2] = {0, 0};
  void* stepsD = nullptr;   // [2 * Ns]
  void* stepsg = nullptr;   // [2 * Ns] BatchStep: the two spectra of the box derivative
  // checkpointed history (ckK >= 2) on the separable pencil march: the step entries of the
  // forward march [Ns], of every segment recompute [<= Ns] and of the conjugate march [Ns];
  // the quadrature pairs (q_{Ns-m}, qd_m) [Ns]; K conjugate slices of the current chunk
  void* stepsCK = nullptr;
  void* pairsCK = nullptr;
  void* qdk = nullptr;
  std::vector<int> ckRoff;  // first recompute entry of segment g
  // RQM4 (scheme 1): quarter-step Boltzmann factors, half-step diffusion tables, three
  // scratch slices for the full and the two half steps, quadrature weight tables
  // plan of the concurrent pass march: plane kernel (1) or pencil passes (0) where the
  // plane kernel applies, two propagator chains on two streams (1) or two-member launches
  // on one stream (0); chosen by timing at the first solve when `autotune` is set
  int plan_plane = 1;
  int plan_streams = 1;
  int plan_xv = 0;  // plan variant: plan 2, the x kernel (0: Plan<nx>, 1: half the elements a thread); plan 3, the line variant (0-3)
  bool autotune = false;
  bool tuned = false;
  bool edw = false;   // Edwards homopolymer model: one field, q-dagger = q
  double bC = 0.0;    // its B / C
  int scheme = 0;
  // q history: ckK = 1 keeps every slice in hist; ckK = K >= 2 keeps q_{cK} in slots
  // 0..nck-1 (nck = Ns/K + 1), q_Ns in slot nck when K does not divide Ns, and the
  // segment q_{cK+j} (j = 1..K-1) being recomputed in slots nck+j
  bool rq_plane = false;  // RQM4 steps on the plane kernels (decided when the step table is built)
  int ckK = 1;
  int nck = 0;
  void* BAh = nullptr;
  void* BBh = nullptr;
  size_t dh_off[3] = {0, 0, 0};
  void* rq = nullptr;       // [3 * M]
  double* qw = nullptr;     // [2 * (Ns+1)] weights of the A and B blocks
  // profiling: an event recorded before every launch (eager solves only)
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  int ev_used = 0;
};

// Kernel classes reported by pft_profile_step.
enum KernelKind {
  KK_Z_FWD = 0, KK_Y_FWD, KK_X_FUSED, KK_Y_INV, KK_Z_INV_FWD, KK_Z_INV_BWD, KK_REDUCE, KK_FIELD_STEP,
  KK_PREPARE, KK_PAIR_STEP, KK_QUADRATURE, KK_COUNT
};
extern const char* const kKernelKindNames[KK_COUNT];

// Record the event that opens the next launch (no-op unless profiling).
inline void mark(CtxData& c, int kind) {
  if (!c.profiling || c.ev_used >= (int)c.ev.size()) return;
  cudaEventRecord(c.ev[c.ev_used], c.stream);
  c.ev_kind[c.ev_used] = kind;
  c.ev_used++;
}

// Bytes of one propagator slice in the working precision.
inline size_t slice_bytes(const CtxData& c, size_t elem) {
  return (size_t)c.M * (c.kind == PFT_SCFT_REAL ? elem : 2 * elem);
}
// History slot holding q_n (see CtxData::ckK).
inline int q_slot(const CtxData& c, int n) {
  if (c.ckK <= 1) return n;
  if (n % c.ckK == 0) return n / c.ckK;
  if (n == c.Ns) return c.nck;
  return c.nck + n % c.ckK;
}
// Slots the history needs.
inline int q_slots(const CtxData& c) { return c.ckK <= 1 ? c.Ns + 1 : c.nck + c.ckK; }
// Is q_n kept after a solve (a checkpoint, q_Ns, or every slice)?
inline bool q_kept(const CtxData& c, int n) { return c.ckK <= 1 || n % c.ckK == 0 || n == c.Ns; }

struct BatchStep;

// Geometry shared by the members of one batch class.
struct BatchGeom {
  int n[3];
  pft_kind kind;
  int nzh;
};

// The separable pencil march (pft_sepp.cuh): grid and field kind (0 real, 1 complex).
struct SeppGeom {
  int n[3];
  int kind;
  int lv = 0;  // line variant: 1 = register lines (FP32, x and y lengths with a register plan)
};
// Launch j (0..Ns) of a separable pencil march for `members` entries starting at ss (for
// j >= 1 the entries of contour step j; j = 0 uses those of step 1).  Real fields need
// ny and nz even.  Returns cudaErrorInvalidValue for a length without an FFT plan.
cudaError_t sepp_launch_f32(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm);
cudaError_t sepp_launch_f64(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm);
// the same march in double-float arithmetic (FP64 history, dd tables and factors)
cudaError_t sepp_launch_dd(const SeppGeom& g, const BatchStep* ss, int j, int members, cudaStream_t sm);

class Engine {
 public:
  virtual ~Engine() {}
  virtual size_t elem_bytes() const = 0;      // working-precision real element
  virtual bool plane_applies(const CtxData& c) const = 0;  // can the y/z plane kernel run this grid?
  virtual bool sep_applies(const CtxData& c) const = 0;    // can the separable march run it?
  virtual bool sepp_applies(const CtxData& c) const = 0;
  virtual bool dd_applies(const CtxData& c) const = 0;     // the double-float separable march (plan 4)?
  virtual bool sepp_reg_applies(const CtxData& c) const = 0;  // plan 3 with register lines (code 19)?
  virtual bool sepp_lv_applies(const CtxData& c, int lv) const = 0;  // plan 3 with line variant lv (code 3 + 16 lv)?
  virtual cudaError_t upload_tables(CtxData& c) = 0;
  virtual cudaError_t fill_ones(CtxData& c, void* dst) = 0;
  virtual cudaError_t prepare_fields(CtxData& c) = 0;   // Boltzmann factors + field term
  virtual cudaError_t enqueue_solve(CtxData& c) = 0;    // marches, Q, densities, H
  virtual cudaError_t solve_mid(CtxData& c) = 0;        // Q and the qd_0 quadrature term (after the forward march)
  virtual cudaError_t solve_tail(CtxData& c) = 0;       // densities and force norms (after the conjugate march)
  // One contour step of every active instance of a batch class (epi 0: forward, 1: conjugate).
  virtual cudaError_t batch_contour_step(const BatchGeom& g, const BatchStep* d_steps, int nactive, int epi,
                                         cudaStream_t st) = 0;
  // one step of both marches for `nactive` entries (pairs of forward / conjugate members):
  // z forward when `first`, then y, x (D), y inverse, and the fused z inverse / forward
  virtual cudaError_t batch_pair_step(const BatchGeom& g, const BatchStep* d_steps, int nactive, bool first,
                                      cudaStream_t stream) = 0;
  // kernels one batch_pair_step launches for this geometry
  // plans 0..3 of a batch class: may this class geometry run plan `plan`?
  virtual bool batch_plan_ok(const BatchGeom& g, int plan) const = 0;
  // launch j of a separable march (plan 2 or 3) of a batch class over nact entries
  virtual cudaError_t batch_sep_launch(const BatchGeom& g, const BatchStep* ss, int j, int nact, int plan, int* err,
                                       cudaStream_t sm) = 0;
  // Q, the quadrature over both stored histories, densities and sums (after both marches)
  virtual cudaError_t finish_both(CtxData& c) = 0;
  virtual int batch_pair_launches(const BatchGeom& g, bool first) const = 0;
  // contour quadrature of Eq. 8 over the stored q and qd histories (after solve_mid)
  virtual cudaError_t quadrature(CtxData& c) = 0;
  // reverse-mode adjoint of the last solve for a loss with dL/dphiA = GA, dL/dphiB = GB
  // (device FP64 arrays), into dL/dW+ and dL/dW- (device FP64 arrays)
  virtual cudaError_t adjoint(CtxData& c, const double* GA, const double* GB, double* dwp, double* dwm) = 0;
  virtual cudaError_t field_step(CtxData& c, int step_kind, double lam, const double* eta_p,
                                 const double* eta_m) = 0;
  virtual cudaError_t fft3d(CtxData& c, void* data, int inverse) = 0;   // complex, in place
  virtual cudaError_t gradients(CtxData& c, double* dwp, double* dwm) = 0;  // + stress into scal
  // precision conversion of `count` reals (a complex value counts as two)
  virtual cudaError_t to_f64(CtxData& c, const void* src, void* dst_f64, long long count) = 0;
  virtual cudaError_t from_f64(CtxData& c, const void* src_f64, void* dst, long long count) = 0;
};

Engine* make_engine_f32();
Engine* make_engine_f64();

cudaError_t launch_philox_normals(unsigned long long seed, unsigned long long instance, unsigned long long step,
                                  int field, long long M, double* out, cudaStream_t st);
cudaError_t launch_narrow_rn(const double* x, float* y, long long n, cudaStream_t st);
cudaError_t launch_philox_raw(const unsigned int ctr[4], const unsigned int key[2], long long count,
                              unsigned int* out, cudaStream_t st);

bool axis_supported(int n);
bool batch_axis_supported(int n);
void set_error(const std::string& s);

// Plan cache of the autotuner: in memory, and in the text file named by the environment
// variable PFT_AUTOTUNE_CACHE (one line per entry: key plane streams ms) when it is set.
bool plan_cache_lookup(const std::string& key, int* plane, int* streams);
void plan_cache_store(const std::string& key, int plane, int streams, double ms);

}  // namespace pft

// The context object behind the opaque pft_ctx handle.
struct pft_ctx {
  pft::CtxData d;
  pft::Engine* eng = nullptr;
  void* io = nullptr;   // [M] complex128 staging for conversions and host noise
  bool have_obs = false;
};
