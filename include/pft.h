/*
 * pft.h -- C ABI of the GB300 (sm_103a) pseudo-spectral propagator library for an
 * incompressible AB diblock melt (Delaney & Fredrickson, "Polymer Field-Theory
 * Simulations on Graphics Processing Units", arXiv:1204.5434).
 *
 * What the library computes (the paper's method, Sec. "Model" and "Algorithms"):
 *   - Boltzmann factors  B_A,B = exp(-w_A,B ds/2) from the fields           (Eq. 13)
 *   - forward march      q_n  = B_n F^-1[ D F[ B_n q_{n-1} ] ],  q_0 = 1     (Eqs. 5, 13)
 *   - backward march     qd_m = same step with the B block first, qd_0 = 1   (Eq. 5)
 *     fused with the contour quadrature of q(s) qd(1-s) into phi_A, phi_B    (Eq. 8)
 *   - Q = (1/V) int q(x, 1) and lnQ                                         (Eq. 4)
 *   - H = C int [w-^2/chiN - i w+] - C V lnQ                                 (Eq. 3)
 *   - field update by explicit Euler (SCFT) or Euler-Maruyama complex
 *     Langevin with real Gaussian noise                              (Eqs. 7, 9, 10)
 *   - exact gradients of the discrete H in the fields and box lengths (stress)
 *
 * Conventions (all entry points):
 *   - grid n[3] = (nx, ny, nz), arrays row-major [x][y][z] (z contiguous),
 *     M = nx*ny*nz.  Every n[a] must be one of 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128,
 *     192, 256 (products of 2 and 3 with a compiled FFT plan); nz must be even.
 *   - lengths in units of Rg; ds = 1/Ns; NsA = floor(fA*Ns + 1/2) contour steps on A.
 *   - PFT_SCFT_REAL: fields are real float64 arrays W+ (= i*omega+) and W- (= omega-);
 *     PFT_CL_COMPLEX: fields are complex128 arrays omega+ and omega- (interleaved
 *     re, im).  All API-facing arrays are float64 / complex128 in either precision.
 *   - PFT_FP64 runs every step in double.  PFT_FP32_MIXED runs the propagators, FFTs
 *     and Boltzmann factors in float (the integrand q*qd of the contour quadrature is
 *     the float product of the two float propagators) and keeps the field update, the
 *     contour quadrature sums, every spatial reduction, Q, lnQ and H in double.
 *   - Pointers marked "host or device" are read/written according to the pft_mem
 *     argument.  Device pointers must be readable on the context's stream when the
 *     call is made.  The library copies inputs; the caller keeps ownership of every
 *     pointer it passes and of every output buffer.
 *   - Calls are asynchronous on the context's stream except those that write host
 *     memory, which synchronise that stream before returning.
 *   - Every entry point returns pft_status; nothing throws or aborts.  A context is
 *     thread-compatible, not thread-safe.
 */
#ifndef PFT_H
#define PFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PFT_OK = 0,
  PFT_ERR_ARG = 1,        /* null pointer, out-of-range parameter */
  PFT_ERR_SHAPE = 2,      /* a grid size without a compiled FFT plan, odd nz */
  PFT_ERR_OOM = 3,        /* device allocation failed */
  PFT_ERR_CUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  PFT_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
  PFT_ERR_NONFINITE = 6,  /* Q or H is not finite (e.g. CL blow-up) */
  PFT_ERR_STATE = 7,      /* call out of order, e.g. solve before set_fields */
  PFT_ERR_IO = 8,         /* checkpoint file could not be read or written */
  PFT_ERR_UNSUPPORTED = 9 /* valid request this build does not implement */
} pft_status;

typedef enum { PFT_SCFT_REAL = 0, PFT_CL_COMPLEX = 1 } pft_kind;
typedef enum { PFT_FP64 = 0, PFT_FP32_MIXED = 1 } pft_precision;
typedef enum { PFT_HOST = 0, PFT_DEVICE = 1 } pft_mem;
typedef enum {
  PFT_STEP_SCFT_EULER = 0,
  PFT_STEP_CL_EULER_MARUYAMA = 1,
  PFT_STEP_SCFT_SIS = 2,
  PFT_STEP_CL_SIS = 3
} pft_step_kind;
/* How the marches run.  PASSES (and AUTO, the same): the pass kernels of each contour
 * step -- a plane kernel for the y and z transforms plus an x pass where the grid has
 * one (FP32 real fields with ny = nz = 64 or 128, complex with ny = nz = 64), pencil
 * passes elsewhere -- replayed as one CUDA graph per solve.  Other values: PFT_ERR_ARG. */
typedef enum { PFT_MARCH_AUTO = 0, PFT_MARCH_PASSES = 1 } pft_march;

/* Contour scheme.  SPLIT2: the 2nd-order split step A(ds) of Eq. 13 with the trapezoid
 * rule per block for Eq. 8.  RQM4: the 4th-order Richardson combination of Eq. 13,
 * q(s+ds) = -(1/3)[A(ds) - 4 A(ds/2) A(ds/2)] q, with composite Simpson weights per
 * block (Simpson 3/8 on the last three intervals of an odd block, the trapezoid rule
 * for a one-interval block); PASSES march only, no gradients. */
typedef enum { PFT_SCHEME_SPLIT2 = 0, PFT_SCHEME_RQM4 = 1 } pft_scheme;

typedef struct { int n[3]; double L[3]; } pft_grid;          /* grid points and box (Rg) */
typedef struct { int Ns; double fA; } pft_chain;              /* contour steps, A fraction */
/* Chain model.  DIBLOCK: incompressible AB diblock melt (Eq. 3), fields W+/W- (SCFT) or
 * omega+/omega- (CL).  EDWARDS: homopolymers in implicit solvent (Eq. 2),
 * H = (B/2) int omega^2 - C V lnQ[i omega]: one field (the first field argument; the
 * second is ignored and may be NULL), stored Wick-rotated as W = i omega in SCFT mode and
 * as omega in CL mode; the chain is reversible, so q-dagger = q and one march is run;
 * phi = (1/Q) int ds q(s) q(1-s) is returned as phiA (phiB = 0); chiN and fA are unused.
 * EDWARDS runs the SPLIT2 scheme on the pass march with the full history, Euler or
 * Euler-Maruyama steps; other options give PFT_ERR_UNSUPPORTED. */
typedef enum { PFT_ARCH_DIBLOCK = 0, PFT_ARCH_EDWARDS = 1 } pft_arch;

typedef struct {
  double chiN;     /* chi_AB N (diblock) */
  double C;        /* chains per Rg^3 (both models) */
  pft_kind kind;   /* real SCFT or complex Langevin fields */
  pft_arch arch;   /* 0 (memset) = DIBLOCK */
  double B;        /* excluded-volume parameter of the Edwards model (>= 0) */
} pft_model;

typedef struct {
  pft_precision precision;
  int use_graph;            /* 1: replay each solve as one captured CUDA graph */
  void* stream;             /* cudaStream_t to run on; NULL: the library creates one */
  unsigned long long seed;  /* Philox key of the CL noise */
  unsigned long long instance; /* Philox counter word: independent replica streams */
  pft_march march;          /* PFT_MARCH_AUTO or PFT_MARCH_PASSES */
  pft_scheme scheme;        /* PFT_SCHEME_SPLIT2 (0) or PFT_SCHEME_RQM4 */
  int checkpoint;           /* q history: 0 = AUTO (every slice when the two histories fit in
                               60% of the free device memory, else every ceil(sqrt(Ns))-th),
                               1 = every slice, K >= 2 = every K-th slice (clamped to Ns): the
                               conjugate march recomputes each segment of K-1 slices from its
                               checkpoint (one extra forward march).  Under a separable plan (2
                               or 3) the marches run on the separable pencil kernels and the
                               conjugate march's slices of a segment's chunk occupy K extra
                               slots; otherwise the pencil passes march one propagator after the
                               other.  K >= 2 needs the SPLIT2 scheme (else PFT_ERR_UNSUPPORTED). */
  int autotune;             /* 1: at the first solve, time the plans of the march that apply
                               (separable march on pencils with its line variants, separable
                               march on the plane kernel with its x variants, plane kernel,
                               pencil passes; two propagator chains on two streams or
                               two-member launches) on the context's own data and keep the
                               fastest; cached per (grid, field kind, precision, Ns) in memory and,
                               if the environment variable PFT_AUTOTUNE_CACHE names a file, in
                               that file (read at the first lookup, appended after tuning).
                               0: the fixed plan (plane kernel where it applies, two chains). */
} pft_opts;

/* Observables of the last solve.  Complex quantities are {re, im}; in SCFT mode the
 * imaginary parts are zero. */
typedef struct {
  double Q[2];          /* single-chain partition function, Eq. 4 */
  double lnQ[2];        /* principal logarithm of Q */
  double H[2];          /* Hamiltonian, Eq. 3 */
  double h[2];          /* intensive H/(C V) */
  double phiA_mean[2];  /* volume average of phi_A (= NsA/Ns up to round-off) */
  double phiB_mean[2];
  double force_p_rms;   /* rms of the W+ (omega+) force of Eq. 7, per C */
  double force_m_rms;   /* rms of the W- (omega-) force */
  double fA_eff;        /* NsA/Ns */
  int NsA;
  long long step;       /* field steps taken since set_fields */
} pft_obs;

typedef struct pft_ctx pft_ctx;

/* Human-readable name of a status code (static storage). */
const char* pft_status_string(pft_status s);

/* Text of the last error raised on this thread (CUDA error string or argument
 * diagnostic); empty if none.  Static thread-local storage. */
const char* pft_last_error(void);

/* Create a context for one system: validates sizes, builds the FFT plans and the
 * per-axis twiddle and diffusion tables, and allocates every device buffer it will
 * use (fields, Boltzmann factors, the q history of Ns+1 slices, two qd slices, the
 * spectrum, FP64 density accumulators, reduction scratch).  On failure *out is NULL.
 * Errors: PFT_ERR_ARG, PFT_ERR_SHAPE, PFT_ERR_OOM, PFT_ERR_CUDA. */
pft_status pft_create(pft_ctx** out, const pft_grid* grid, const pft_chain* chain,
                      const pft_model* model, const pft_opts* opts);

/* Free every device buffer, graph and (if the library created it) stream. NULL is a no-op. */
pft_status pft_destroy(pft_ctx* ctx);

/* Device memory held by the context, in bytes. */
pft_status pft_memory_bytes(const pft_ctx* ctx, size_t* bytes);

/* The context's stream (cudaStream_t) as an opaque pointer. */
pft_status pft_get_stream(const pft_ctx* ctx, void** stream);

/* Block the host until all work queued on the context's stream has finished. */
pft_status pft_synchronize(pft_ctx* ctx);

/* Copy the two fields in (M elements each; float64 in SCFT, complex128 in CL mode),
 * recompute the Boltzmann factors (Eq. 13) and reset the step counter.
 * wp, wm: host or device per `where`. */
pft_status pft_set_fields(pft_ctx* ctx, const void* wp, const void* wm, pft_mem where);

/* Copy the current fields out (same layout as pft_set_fields). */
pft_status pft_get_fields(pft_ctx* ctx, void* wp, void* wm, pft_mem where);

/* Change the box lengths L[3] (Rg); the fields stay fixed on the grid. */
pft_status pft_set_box(pft_ctx* ctx, const double L[3]);
pft_status pft_get_box(const pft_ctx* ctx, double L[3]);

/* One full solve for the current fields: forward march (Eqs. 5, 13), Q (Eq. 4),
 * backward march with fused contour quadrature (Eq. 8), densities and H (Eq. 3).
 * Error: PFT_ERR_STATE before the first pft_set_fields. */
pft_status pft_solve(pft_ctx* ctx);

/* Observables of the last solve (synchronises the stream).
 * Error: PFT_ERR_STATE before a solve; PFT_ERR_NONFINITE if Q or H is not finite
 * (the struct is still filled). */
pft_status pft_get_observables(pft_ctx* ctx, pft_obs* obs);

/* Segment densities phi_A, phi_B of the last solve (Eq. 8, phi = rho/rho0), M
 * elements each, float64 (SCFT) or complex128 (CL).  Host or device per `where`. */
pft_status pft_get_densities(pft_ctx* ctx, void* phiA, void* phiB, pft_mem where);

/* One field update from the densities of the last solve (Eq. 9 with the Eq. 7 forces
 * taken per C):
 *   PFT_STEP_SCFT_EULER (SCFT mode):  W+ += lam (phiA+phiB-1);
 *                                     W- -= lam (2 W-/chiN + phiB - phiA)
 *   PFT_STEP_CL_EULER_MARUYAMA (CL):  w+ += -dt i (phiA+phiB-1) + eta+;
 *                                     w- += -dt (2 w-/chiN + phiB - phiA) + eta-
 * Edwards model (force per C, b = B/C): SCFT W += lam (phi - b W); CL
 * omega += -dt (b omega + i phi) + eta (eta_m unused; Philox field 0);
 * and the semi-implicit steps (diblock only) of Eq. 11 (the linear part of the force at the new time):
 *   PFT_STEP_SCFT_SIS (SCFT mode):    W+^(k) += lam F+^(k) / (1 + lam g_D(k));
 *                                     W- = (W- - lam (phiB - phiA)) / (1 + 2 lam/chiN)
 *   PFT_STEP_CL_SIS (CL):             w+^(k) += (-dt i F^(k) + eta+^(k)) / (1 + dt g_D(k)),
 *                                     F = phiA+phiB-1;
 *                                     w- = (w- - dt (phiB - phiA) + eta-) / (1 + 2 dt/chiN)
 * with g_D(k) = 2 (e^{-x} + x - 1)/x^2, x = k^2 (the whole chain's Debye function, Rg = 1)
 * and ^ the discrete Fourier transform (one forward and one inverse FP64 transform of the
 * w+ increment per step).
 * eta+/- are real Gaussian with variance 2 dt/(C dV) (below Eq. 10).  If eta_p and
 * eta_m are NULL the library draws them from its Philox4x32-10 stream (key = seed,
 * counter = (point/4, field, step, instance)); otherwise they are caller arrays of M
 * float64 values, already scaled, host or device per `where`.  The Boltzmann factors
 * for the next solve are recomputed in the same kernel.
 * Errors: PFT_ERR_STATE without a prior solve; PFT_ERR_ARG for a step kind that does
 * not match the model kind. */
pft_status pft_field_step(pft_ctx* ctx, pft_step_kind kind, double lam_or_dt,
                          const void* eta_p, const void* eta_m, pft_mem where);

/* Reverse-mode adjoint of the last solve for a loss L(phiA, phiB) given on the grid as
 * dL_dphiA and dL_dphiB (M float64 each): writes dL/dW+ and dL/dW- (M float64 each), the
 * exact gradient of L through the discrete march (2nd-order steps, trapezoid quadrature,
 * the normalisation by Q).  Method: the q and qd marches are adjoined backwards with the
 * source terms of the quadrature (Eq. 8), the two adjoint chains on two streams; every
 * step adds -(ds/2) [lambda_k q_k + B_k q_{k-1} F^-1 D F (B_k lambda_k)] to the gradient
 * of its block (FP64 accumulation in both precisions).  Arrays on host or device per
 * `where`.
 * Errors: PFT_ERR_UNSUPPORTED unless real SCFT diblock fields, SPLIT2, the pass march and
 * both histories kept (checkpoint 1); PFT_ERR_STATE without a solve at the current fields. */
pft_status pft_adjoint(pft_ctx* ctx, const void* dL_dphiA, const void* dL_dphiB, void* dL_dwp, void* dL_dwm,
                       pft_mem where);

/* Exact gradients of the discrete H of the last solve:
 *   dH_dwp, dH_dwm (M float64 each, host or device per `where`, either may be NULL):
 *     C dV (phiA+phiB-1) and C dV (2 W-/chiN + phiB - phiA)          (Eq. 7 x C dV)
 *   dH_dL[3] (host, may be NULL): dH/dL_a = H/L_a - C V dlnQ/dL_a, the box derivative
 *     at fixed grid values, from the bilinear contraction of the forward and
 *     conjugate spectra with d(exp(-k^2 ds))/dL_a over every contour step.
 *   dlnQ_dL[3] (host, may be NULL).
 * SCFT mode only (PFT_ERR_UNSUPPORTED in CL mode).  Runs one extra march. */
pft_status pft_gradients(pft_ctx* ctx, void* dH_dwp, void* dH_dwm, double dH_dL[3],
                         double dlnQ_dL[3], pft_mem where);

/* Checkpoint and resume of a run (no counterpart in the paper).  pft_save writes the
 * state a field-update loop needs to continue bit for bit: the box L, the fields W+ and
 * W- (float64 or complex128 as stored; W- omitted for the Edwards model), the complex
 * Langevin noise key and counter (seed, instance, steps taken since the fields were
 * set) and the system's parameters for validation.  File layout (little-endian): the
 * 8 bytes "PFTCKPT1", uint32 version (1), uint32 header bytes (112), the header (n[3],
 * Ns, kind, arch, precision as int32, 4 zero bytes; L[3], fA, chiN, C, B as float64;
 * seed, instance as uint64; step as int64), the fields, then a 64-bit FNV-1a hash of
 * every byte before it.
 * The file is written to `path` through a temporary file in the same directory and
 * renamed, so an interrupted save leaves the previous checkpoint intact.
 * pft_load reads such a file into a context of the same system (grid, Ns, kind, arch,
 * fA, chiN, C, B must match; the precision may differ), sets the box, the fields and
 * the noise key and counter; a solve is needed before observables.
 * Errors: PFT_ERR_ARG for NULL arguments or a checkpoint of another system;
 * PFT_ERR_STATE (save) before fields are set; PFT_ERR_IO when the file cannot be
 * written or read, is not a checkpoint, is truncated or fails its hash. */
pft_status pft_save(pft_ctx* ctx, const char* path);
pft_status pft_load(pft_ctx* ctx, const char* path);

/* Batches of independent systems ------------------------------------------ */

/* One member of a batch: its grid, chain and model, and the Philox key of its complex
 * Langevin noise (the counter's instance word is the member index). */
typedef struct {
  pft_grid grid;
  pft_chain chain;
  pft_model model;
  unsigned long long seed;
} pft_instance_desc;

typedef enum {
  PFT_BATCH_GRAPHED = 0,      /* batched pass launches, one CUDA graph per field update */
  PFT_BATCH_PER_INSTANCE = 1  /* one launch sequence per instance, instance after instance */
} pft_batch_mode;

typedef struct pft_batch pft_batch;

/* Create `count` independent systems (SCFT and CL mixed; grid sizes up to 64 per axis
 * from 4,6,8,12,16,24,32,48,64; any Ns and fA) in one precision.  Members with equal
 * field kind and grid form a class; one field update of the whole batch runs each
 * contour step of each class as five batched launches over the members still
 * marching (members of a class sorted by Ns), then every member's reductions and
 * field update.  stream: cudaStream_t or NULL (the batch creates one).
 * Errors: PFT_ERR_ARG, PFT_ERR_SHAPE, PFT_ERR_OOM, PFT_ERR_CUDA. */
pft_status pft_batch_create(pft_batch** out, int count, const pft_instance_desc* descs,
                            pft_precision precision, void* stream);
pft_status pft_batch_destroy(pft_batch* b);

/* Fields of member i (layout as pft_set_fields); resets its step counter. */
pft_status pft_batch_set_fields(pft_batch* b, int i, const void* wp, const void* wm, pft_mem where);
pft_status pft_batch_get_fields(pft_batch* b, int i, void* wp, void* wm, pft_mem where);

/* `updates` field updates of every member: solve (Eqs. 3-5, 8, 13) then the field
 * step of Eq. 9 -- explicit Euler with `lam` for SCFT members, Euler-Maruyama with
 * `dt` and the library's Philox noise for CL members.  GRAPHED captures one update of
 * the whole batch as a CUDA graph (recaptured when lam or dt change) and replays it.
 * Asynchronous on the batch stream.  Error: PFT_ERR_STATE if a member has no fields. */
pft_status pft_batch_run(pft_batch* b, int updates, double lam, double dt, pft_batch_mode mode);

/* Per-class plan autotuner of a batch (uses the instances' current fields): for every class
 * of equal field kind and grid, time the class's two marches and densities under each plan
 * that applies to it and keep the fastest; the next graphed run captures the chosen plans.
 * Plans: 0 -- one march after the other, the quadrature fused into the conjugate march;
 * 1 -- both marches in the same launches (the 3D transform pair of each step: plane kernel
 * and x pass for FP32 classes with ny = nz = 64 or 128, else the pencil passes with the z
 * passes of consecutive steps fused), the quadrature after the marches over both
 * histories (one extra q-dagger history per instance); 2 -- the separable march of
 * pft_get_plan's plan 2 (FP32 real classes with nx = ny = nz in {64, 128}); 3 -- the
 * separable march on pencils (plan 3 of pft_get_plan); 19 -- plan 3 with register lines
 * (FP32 classes whose x and y lengths are in {4, 6, 8, 12, 16, 24, 32, 48}: one thread
 * transforms a whole x or y line in registers, no shared-memory exchange); 35 -- plan 3
 * with the x and y lines in tiles of 32 lines a CTA instead of 16 (FP32 classes); 51 --
 * plan 3 with twice the elements a thread on the x and y lines, in another radix order
 * (16 2 at 32 points, 3 8 2 at 48, 16 4 at 64), in tiles of 32 lines (FP32 classes whose x
 * and y lengths are 32, 48 or 64).  Plans 2, 3, 19, 35 and 51 run both marches in the same
 * launches and the quadrature after them, as plan 1.  The default is plan 2 where it
 * applies, else plan 3.
 * Errors: PFT_ERR_STATE if an instance has no fields; PFT_ERR_OOM. */
pft_status pft_batch_autotune(pft_batch* batch);

/* Set the plan (0, 1, 2, 3, 19, 35 or 51, as for pft_batch_autotune) of class `cls`, or of every class it
 * applies to for cls = -1.  Errors: PFT_ERR_ARG for a bad index or plan,
 * PFT_ERR_UNSUPPORTED for a plan that does not apply to class `cls`. */
pft_status pft_batch_set_plan(pft_batch* batch, int cls, int plan);

/* Number of batch plans the autotuner times, in the order of pft_batch_class_info's
 * tuned_ms: 0, 1, 2, 3, 19, 35, 51. */
#define PFT_BATCH_PLANS 7

/* Class `cls` (0 .. classes-1 of pft_batch_info): grid n[3], field kind, member count, plan
 * in use and the autotuner's timings of plans 0, 1, 2, 3, 19, 35 and 51 in ms
 * (tuned_ms[0..PFT_BATCH_PLANS-1]; -1 if not tuned or not applicable).  Any output pointer
 * may be NULL.  Errors: PFT_ERR_ARG for a bad index. */
pft_status pft_batch_class_info(const pft_batch* batch, int cls, int n[3], int* kind, int* members, int* plan,
                                float tuned_ms[PFT_BATCH_PLANS]);

/* Observables and densities of member i's last solve (synchronises). */
pft_status pft_batch_get_observables(pft_batch* b, int i, pft_obs* obs);
pft_status pft_batch_get_densities(pft_batch* b, int i, void* phiA, void* phiB, pft_mem where);
/* Wait for the batch stream.  Errors: PFT_ERR_TIMEOUT if a bounded wait in a kernel of
 * the updates since the last call ran out (their results are invalid), PFT_ERR_CUDA. */
pft_status pft_batch_synchronize(pft_batch* b);

/* Grid-point contour steps per field update (sum of 2 M Ns), number of classes, and
 * kernel launches per captured update (0 before the first GRAPHED run). */
pft_status pft_batch_info(const pft_batch* b, double* units_per_update, int* nclasses, long long* launches);
pft_status pft_batch_get_stream(const pft_batch* b, void** stream);

/* Per-kernel-class device times of one solve, for roofline reporting. */
#define PFT_PROFILE_KINDS 16
typedef struct {
  int nkinds;
  char name[PFT_PROFILE_KINDS][24];
  long long launches[PFT_PROFILE_KINDS];
  double ms[PFT_PROFILE_KINDS];                /* summed device time of the class */
  double bytes_per_launch[PFT_PROFILE_KINDS];  /* arrays one launch must read + write */
  double step_fwd_ms;  /* mean device time of one forward contour step (its 5 launches) */
  double step_bwd_ms;  /* mean device time of one conjugate contour step with quadrature */
  double total_ms;     /* first to last event */
} pft_profile;

/* Run one solve launch by launch (not graph-replayed) with a CUDA event recorded on
 * the context's stream before every kernel, then, if step_kind >= 0, one field step
 * of that kind with lam_or_dt and the library's own noise; fill *out with the device
 * time per kernel class.  Same effect on the context as pft_solve (+ pft_field_step).
 * Synchronises.  Errors: as pft_solve / pft_field_step. */
pft_status pft_profile_step(pft_ctx* ctx, int step_kind, double lam_or_dt, pft_profile* out);

/* One contour step that allocates no device memory, for callers that cannot call
 * cudaMalloc (code running while another framework owns the device allocator, or a
 * plug-in that may only use the memory it is handed).  The paper has no counterpart:
 * it is this library's own addition.
 *   q_out = B * F^-1[ D * F[ B * q_in ] ],  B = exp(-w/(2 Ns)),  D = exp(-k^2/Ns)
 * in FP64 on real fields, with the library's context conventions (grid n[3], box
 * L[3] in Rg, row-major [x][y][z]).  w, q_in, q_out: device float64 arrays of
 * M = n[0]*n[1]*n[2] values owned by the caller; q_out may alias q_in; the call is
 * asynchronous on `stream` (cudaStream_t or NULL for the legacy default stream).
 * Scratch (Boltzmann factor, half spectrum, twiddle and diffusion tables) lives in
 * one static device array of about 6.3 MB that every GPU loading the library keeps
 * until the process exits; the limit is 64 points per axis (64^3 points).  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  The address is kept for the rest of the
 * process: a caller that destroys the device's primary context (cudaDeviceReset) must
 * not call this entry point on that device again in the same process.  All calls share
 * the array and each call overwrites every part of it that it reads, so nothing needs
 * clearing between calls -- but calls whose work overlaps on the GPU (different
 * streams or devices sharing a context without ordering) race on it.  Allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 * Errors: PFT_ERR_ARG (NULL pointer, Ns < 1, non-positive L, any n[a] > 64),
 * PFT_ERR_SHAPE (a size without an FFT plan), PFT_ERR_CUDA. */
pft_status pft_contour_step_static(const int n[3], const double L[3], int Ns, const double* w,
                                   const double* q_in, double* q_out, void* stream);

/* Test hooks -------------------------------------------------------------- */

/* 3D DFT of M complex128 values through the library's own FFT passes in the
 * context's precision (forward: exp(-i k.x), unnormalised; inverse: exp(+i k.x),
 * also unnormalised).  in/out host or device per `where`, may alias. */
pft_status pft_fft3d(pft_ctx* ctx, const void* in, void* out, int inverse, pft_mem where);

/* Copy slice `s` (0..Ns) of the forward propagator history (which = 0), the last
 * conjugate propagator slice qd_Ns (which = 1, s ignored), or slice s of the conjugate
 * history (which = 2; contexts that keep it: the concurrent SPLIT2 march with the full
 * history, else PFT_ERR_UNSUPPORTED) out as float64/complex128. */
pft_status pft_get_propagator(pft_ctx* ctx, int which, int s, void* out, pft_mem where);

/* Replace the initial condition q_0 = qd_0 = 1 by a caller array (M values, float64
 * or complex128 by kind; NULL restores 1).  Used by the diffusion-only test. */
pft_status pft_debug_set_q0(pft_ctx* ctx, const void* q0, pft_mem where);

/* Plan of the pass march in use.  *plane: 0 = pencil passes (a 3D transform pair per
 * contour step); 1 = the y/z plane kernel plus an x pass per step (FP32 real fields with
 * ny = nz = 64 or 128, complex fields with ny = nz = 64); 2 = the separable march (FP32 real
 * fields, ny = nz and nx in {64, 128}): the diffusion factor exp(-k^2 ds) of Eq. 13 is the
 * product of three per-axis factors, so F^-1 D F is the product of three 1D periodic
 * Gaussian convolutions, applied in alternating axis order so that one launch -- a y/z
 * plane kernel or an x kernel in turn -- advances one contour step; 3 = the separable
 * march on pencils (complex fields, real fields with ny and nz even; either precision):
 * per contour step one launch of the y convolution and one of the x or z kernel, which
 * carries the two convolutions of consecutive steps along its axis; 4 = plan 3 of an FP64
 * context in double-float arithmetic (each value an unevaluated sum of two floats, about
 * 48 significant bits, computed on the FP32 pipe; the history, the quadrature and
 * everything after the march stay FP64); 19 = plan 3 with register lines (FP32, x and y
 * lengths in {4, 6, 8, 12, 16, 24, 32, 48}: one thread transforms a whole x or y line in
 * registers, no shared-memory exchange); 35 = plan 3 with the x and y lines in tiles of 32
 * lines a CTA instead of 16 (FP32); 51 = plan 3 with twice the elements a thread on the x
 * and y lines, in another radix order, in tiles of 32 lines (FP32, x and y lengths of 32,
 * 48 or 64); 18 = plan 2 with the x
 * kernel on half the elements a thread (twice the threads, one more exchange: at nx = 128
 * eight elements and radices 8, 4, 4 instead of 16 and 16, 8).  *streams = 1 if the
 * two propagators run as two chains on two streams.  Either pointer may be NULL.
 * Errors: PFT_ERR_ARG for a NULL ctx. */
pft_status pft_get_plan(const pft_ctx* ctx, int* plane, int* streams);

/* Fix the plan of the pass march (codes as pft_get_plan reports them); the context
 * keeps it (no autotuning) and recaptures its solve graph at the next pft_solve.  The RQM4
 * scheme, the adjoint and the box derivative run the plane kernel wherever plane >= 1.
 * Errors: PFT_ERR_ARG (NULL ctx, values out of range), PFT_ERR_UNSUPPORTED (a plan the
 * context's grid, field kind or precision does not allow). */
pft_status pft_set_plan(pft_ctx* ctx, int plane, int streams);

/* History interval in use: 1 = every slice of q is kept, K >= 2 = every K-th slice (see
 * pft_opts.checkpoint).  Errors: PFT_ERR_ARG for NULL arguments. */
pft_status pft_get_checkpoint(const pft_ctx* ctx, int* K);

/* Kernel launches of this library per call, for accounting (no counterpart in the
 * paper).  *solve: the kernel nodes of the CUDA graph one pft_solve replays, counted
 * when the graph was captured; -1 before the first graphed solve and for contexts that
 * solve without a graph (use_graph = 0).  *field_step:
 * the kernels one pft_field_step launches.  Either pointer may be NULL.
 * Errors: PFT_ERR_ARG for a NULL ctx. */
pft_status pft_launch_counts(const pft_ctx* ctx, long long* solve, long long* field_step);

/* Fused multiply-add throughput of the current device, in TFLOP/s (2 flops per FMA):
 * independent FMA chains on every SM for about 20 ms, timed with CUDA events on `stream`
 * (cudaStream_t, NULL for the legacy default stream) after one warm-up launch.  No
 * counterpart in the paper: the FP64 contour step is bound by the FP64 pipe, and this is
 * the denominator of its roofline (precision PFT_FP64: DFMA; PFT_FP32_MIXED: FFMA).
 * Allocates and frees a small output buffer (stream-ordered); synchronises the stream.
 * Errors: PFT_ERR_ARG (NULL tflops, unknown precision), PFT_ERR_CUDA. */
pft_status pft_fma_throughput(int precision, double* tflops, void* stream);

/* Standard normals of the device Philox stream (same layout as the CL noise) for
 * points 0..M-1 into a device float64 array, on `stream` (cudaStream_t or NULL). */
pft_status pft_philox_normals(unsigned long long seed, unsigned long long instance,
                              unsigned long long step, int field, long long M,
                              double* out_device, void* stream);

/* Raw Philox4x32-10 blocks: out_device receives 4*count uint32 words, block i from
 * counter (i + ctr0, ctr1, ctr2, ctr3) and key (k0, k1). */
pft_status pft_philox_raw(const unsigned int ctr[4], const unsigned int key[2], long long count,
                          unsigned int* out_device, void* stream);

/* The library's double -> float narrowing on the integer pipe (used where an FP64 result
 * is stored in a float propagator array): y[i] = x[i] rounded to nearest, ties to even,
 * for results in the normal float range; below the smallest normal float a signed zero,
 * overflow gives infinity, NaN stays NaN.  x (n float64) and y (n float32) are device
 * pointers, on `stream` (NULL: the default stream).  Errors: PFT_ERR_ARG, PFT_ERR_CUDA. */
pft_status pft_debug_narrow_rn(const double* x_device, float* y_device, long long n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PFT_H */
