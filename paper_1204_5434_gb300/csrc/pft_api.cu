// pft_api.cu -- the extern "C" entry points declared in include/pft.h.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pft_engine.h"

using pft::CtxData;
using pft::Engine;


namespace pft {
const char* const kKernelKindNames[KK_COUNT] = {"z_fwd",      "y_fwd",     "x_fused",   "y_inv",
                                                "z_inv_fwd",  "z_inv_bwd", "reduce",    "field_step",
                                                "prepare",    "pair_step",
                                                "quadrature"};
static thread_local std::string g_err;
void set_error(const std::string& s) { g_err = s; }

bool batch_axis_supported(int n) {
  switch (n) {
    case 4: case 6: case 8: case 12: case 16: case 24: case 32: case 48: case 64:
      return true;
    default:
      return false;
  }
}

namespace {
std::mutex g_plan_mu;
std::map<std::string, std::pair<int, int>> g_plans;
bool g_plans_loaded = false;

void load_plan_file() {
  g_plans_loaded = true;
  const char* path = getenv("PFT_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[256];
  int plane = 0, streams = 0;
  double ms = 0.0;
  while (fscanf(f, "%255s %d %d %lf", key, &plane, &streams, &ms) == 4) g_plans[key] = {plane, streams};
  fclose(f);
}
}  // namespace

bool plan_cache_lookup(const std::string& key, int* plane, int* streams) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (!g_plans_loaded) load_plan_file();
  auto it = g_plans.find(key);
  if (it == g_plans.end()) return false;
  *plane = it->second.first;
  *streams = it->second.second;
  return true;
}

void plan_cache_store(const std::string& key, int plane, int streams, double ms) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (!g_plans_loaded) load_plan_file();
  g_plans[key] = {plane, streams};
  const char* path = getenv("PFT_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %.6f\n", key.c_str(), plane, streams, ms);
  fclose(f);
}

bool axis_supported(int n) {
  switch (n) {
    case 4: case 6: case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192:
    case 256:
      return true;
    default:
      return false;
  }
}
}  // namespace pft

namespace {

pft_status fail(pft_status s, const std::string& msg) {
  pft::set_error(msg);
  return s;
}

pft_status cuda_fail(cudaError_t e, const char* what) {
  pft::set_error(std::string(what) + ": " + cudaGetErrorString(e));
  (void)cudaGetLastError();  // clear a sticky launch error so later calls can proceed
  if (e == cudaErrorMemoryAllocation) return PFT_ERR_OOM;
  if (e == cudaErrorNotSupported) return PFT_ERR_UNSUPPORTED;
  return PFT_ERR_CUDA;
}

#define PFT_CK(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

size_t welem(const CtxData& d) {  // bytes of one working-precision propagator element
  const size_t r = (d.prec == PFT_FP64) ? 8 : 4;
  return d.kind == PFT_SCFT_REAL ? r : 2 * r;
}
size_t felem(const CtxData& d) { return d.kind == PFT_SCFT_REAL ? 8 : 16; }  // API element

cudaError_t dalloc(CtxData& d, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) d.bytes += bytes;
  return e;
}

void free_all(pft_ctx* c) {
  CtxData& d = c->d;
  if (d.graph) cudaGraphExecDestroy(d.graph);
  for (cudaEvent_t ev : d.ev) cudaEventDestroy(ev);
  void* bufs[] = {d.wp, d.wm, d.BA, d.BB, d.hist, d.qd[0], d.qd[1], d.qd0, d.spec, d.spec2,
                  d.accA, d.accB, d.partials, d.scal, d.tables, c->io, d.kerr, d.qdh, d.steps2, d.stepsS, d.stepsg,
                  d.BAh, d.BBh, d.rq, d.qw, d.sis, d.adj, d.stepsa, d.stepsap, d.adjS, d.stepsAS, d.ddbuf, d.stepsD,
                  d.stepsCK, d.pairsCK, d.qdk};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (d.scal_host) cudaFreeHost(d.scal_host);
  if (d.own_stream && d.stream) cudaStreamDestroy(d.stream);
  if (d.stream2) cudaStreamDestroy(d.stream2);
  if (d.fork_ev) cudaEventDestroy(d.fork_ev);
  if (d.join_ev) cudaEventDestroy(d.join_ev);
  delete c->eng;
  delete c;
}

cudaMemcpyKind kind_in(pft_mem w) { return w == PFT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind kind_out(pft_mem w) { return w == PFT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

pft_status write_volume(CtxData& d) {
  const double V = d.L[0] * d.L[1] * d.L[2];
  d.scal_host[pft::S_VOL] = V;
  PFT_CK(cudaMemcpyAsync(d.scal + pft::S_VOL, d.scal_host + pft::S_VOL, sizeof(double), cudaMemcpyHostToDevice,
                         d.stream));
  PFT_CK(cudaStreamSynchronize(d.stream));
  return PFT_OK;
}

}  // namespace

extern "C" {

const char* pft_status_string(pft_status s) {
  switch (s) {
    case PFT_OK: return "PFT_OK";
    case PFT_ERR_ARG: return "PFT_ERR_ARG: invalid argument";
    case PFT_ERR_SHAPE: return "PFT_ERR_SHAPE: unsupported grid size";
    case PFT_ERR_OOM: return "PFT_ERR_OOM: device memory exhausted";
    case PFT_ERR_CUDA: return "PFT_ERR_CUDA: CUDA runtime error";
    case PFT_ERR_TIMEOUT: return "PFT_ERR_TIMEOUT: bounded device wait expired";
    case PFT_ERR_NONFINITE: return "PFT_ERR_NONFINITE: non-finite Q or H";
    case PFT_ERR_STATE: return "PFT_ERR_STATE: call out of order";
    case PFT_ERR_IO: return "PFT_ERR_IO: file error";
    case PFT_ERR_UNSUPPORTED: return "PFT_ERR_UNSUPPORTED: not implemented for this configuration";
  }
  return "unknown pft_status";
}

const char* pft_last_error(void) { return pft::g_err.c_str(); }

pft_status pft_create(pft_ctx** out, const pft_grid* grid, const pft_chain* chain, const pft_model* model,
                      const pft_opts* opts) {
  if (!out) return fail(PFT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !chain || !model || !opts) return fail(PFT_ERR_ARG, "grid, chain, model and opts are required");
  for (int a = 0; a < 3; a++) {
    if (!pft::axis_supported(grid->n[a]))
      return fail(PFT_ERR_SHAPE, "grid size n[" + std::to_string(a) + "]=" + std::to_string(grid->n[a]) +
                                     " has no FFT plan (4,6,8,12,16,24,32,48,64,96,128,192,256)");
    if (!(grid->L[a] > 0.0) || !isfinite(grid->L[a])) return fail(PFT_ERR_ARG, "box lengths must be positive");
  }
  if (chain->Ns < 1 || chain->Ns > 100000) return fail(PFT_ERR_ARG, "Ns out of range [1, 100000]");
  if (!(chain->fA >= 0.0 && chain->fA <= 1.0)) return fail(PFT_ERR_ARG, "fA out of [0, 1]");
  if (model->arch != PFT_ARCH_DIBLOCK && model->arch != PFT_ARCH_EDWARDS) return fail(PFT_ERR_ARG, "unknown chain model");
  const bool edw = (model->arch == PFT_ARCH_EDWARDS);
  if (!(model->C > 0.0) || !isfinite(model->C)) return fail(PFT_ERR_ARG, "C must be positive");
  if (!edw && !(model->chiN > 0.0)) return fail(PFT_ERR_ARG, "chiN must be positive");
  if (edw && !(model->B >= 0.0 && isfinite(model->B))) return fail(PFT_ERR_ARG, "B must be finite and >= 0");
  if (edw && (opts->scheme != PFT_SCHEME_SPLIT2 || opts->checkpoint >= 2))
    return fail(PFT_ERR_UNSUPPORTED, "the Edwards model runs SPLIT2 with the full history");
  if (model->kind != PFT_SCFT_REAL && model->kind != PFT_CL_COMPLEX) return fail(PFT_ERR_ARG, "unknown model kind");
  if (opts->precision != PFT_FP64 && opts->precision != PFT_FP32_MIXED) return fail(PFT_ERR_ARG, "unknown precision");
  if (opts->scheme != PFT_SCHEME_SPLIT2 && opts->scheme != PFT_SCHEME_RQM4) return fail(PFT_ERR_ARG, "unknown scheme");
  if (opts->march != PFT_MARCH_AUTO && opts->march != PFT_MARCH_PASSES) return fail(PFT_ERR_ARG, "unknown march");
  if (opts->checkpoint < 0) return fail(PFT_ERR_ARG, "checkpoint interval must be >= 0");
  if (opts->checkpoint >= 2 && opts->scheme != PFT_SCHEME_SPLIT2)
    return fail(PFT_ERR_UNSUPPORTED, "a checkpointed history needs the SPLIT2 scheme");

  pft_ctx* c = new pft_ctx();
  CtxData& d = c->d;
  for (int a = 0; a < 3; a++) {
    d.n[a] = grid->n[a];
    d.L[a] = grid->L[a];
  }
  d.Ns = chain->Ns;
  d.fA = chain->fA;
  d.NsA = (int)floor(chain->fA * chain->Ns + 0.5);
  d.ds = 1.0 / chain->Ns;
  d.chiN = edw ? 1.0 : model->chiN;
  d.edw = edw;
  d.bC = edw ? model->B / model->C : 0.0;
  if (edw) {  // one block: the whole chain feels the one field
    d.fA = 1.0;
    d.NsA = d.Ns;
  }
  d.C = model->C;
  d.kind = model->kind;
  d.prec = opts->precision;
  d.use_graph = opts->use_graph != 0;
  d.seed = opts->seed;
  d.instance = opts->instance;
  d.M = (long long)d.n[0] * d.n[1] * d.n[2];
  d.nzh = (d.kind == PFT_SCFT_REAL) ? d.n[2] / 2 + 1 : d.n[2];
  d.Ms = (long long)d.n[0] * d.n[1] * d.nzh;

  cudaError_t e = cudaGetDevice(&d.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, d.device);
  if (e != cudaSuccess) {
    pft_status s = cuda_fail(e, "cudaGetDevice");
    free_all(c);
    return s;
  }
  d.npart = d.sms * 4;
  if (opts->stream) {
    d.stream = (cudaStream_t)opts->stream;
  } else {
    e = cudaStreamCreateWithFlags(&d.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      pft_status s = cuda_fail(e, "cudaStreamCreate");
      free_all(c);
      return s;
    }
    d.own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&d.stream2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.join_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    pft_status s = cuda_fail(e, "second stream");
    free_all(c);
    return s;
  }
  c->eng = (d.prec == PFT_FP64) ? pft::make_engine_f64() : pft::make_engine_f32();
  d.scheme = (opts->scheme == PFT_SCHEME_RQM4) ? 1 : 0;
  d.autotune = opts->autotune != 0;
  // the default plan (measured on GB300): the separable march on the plane kernel where it
  // applies (FP32), else the plane kernel, else the separable march on pencils (FP64: fewer
  // passes of the FP64-pipe-bound transforms; FP32: two field round trips a contour step
  // against the pencil passes' four), else the pencil passes
  if (c->eng->sep_applies(d)) d.plan_plane = 2;
  else if (c->eng->plane_applies(d)) d.plan_plane = 1;
  else if (c->eng->sepp_applies(d)) d.plan_plane = 3;
  else d.plan_plane = 0;

  const size_t M = (size_t)d.M;
  const size_t we = welem(d), fe = felem(d);
  const size_t ze = 2 * c->eng->elem_bytes();  // working-precision complex
  {
    // history interval: every slice, or every K-th with segment recomputation
    int K = opts->checkpoint;
    if (K == 0) {
      size_t free_b = 0, total_b = 0;
      K = 1;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const double need = 2.0 * (double)(d.Ns + 1) * (double)(M * we);  // q and qd histories
        if (need > 0.6 * (double)free_b) K = (int)ceil(sqrt((double)d.Ns));
      }
    }
    if (K > d.Ns) K = d.Ns;
    if (K < 2 || d.scheme != 0 || d.edw) K = 1;
    d.ckK = K;
    d.nck = (K > 1) ? d.Ns / K + 1 : 0;
  }
  struct {
    void** p;
    size_t b;
  } plan[] = {
      {&d.wp, M * fe},   {&d.wm, M * fe},    {&d.BA, M * we},     {&d.BB, M * we},
      {&d.hist, (size_t)pft::q_slots(d) * M * we}, {&d.qd[0], M * we}, {&d.qd[1], M * we}, {&d.qd0, M * we},
      {&d.spec, M * ze}, {&d.spec2, M * ze}, {&d.accA, M * fe},  {&d.accB, M * fe},
      {(void**)&d.partials, (size_t)d.npart * 16 * sizeof(double)}, {(void**)&d.scal, pft::S_COUNT * sizeof(double)},
      {&c->io, M * 16}, {(void**)&d.kerr, 16},
      // quarter-step Boltzmann factors of the 4th-order scheme
      {d.scheme ? &d.BAh : nullptr, M * we}, {d.scheme ? &d.BBh : nullptr, M * we},
  };
  for (auto& a : plan) {
    if (!a.p) continue;
    e = dalloc(d, a.p, a.b);
    if (e != cudaSuccess) {
      pft_status s = cuda_fail(e, "device allocation");
      free_all(c);
      return s;
    }
  }
  e = cudaMallocHost(&d.scal_host, pft::S_COUNT * sizeof(double));
  if (e == cudaSuccess) {
    memset(d.scal_host, 0, pft::S_COUNT * sizeof(double));
    e = cudaMemsetAsync(d.scal, 0, pft::S_COUNT * sizeof(double), d.stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d.partials, 0, (size_t)d.npart * 16 * sizeof(double), d.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.kerr, 0, 16, d.stream);
  if (e == cudaSuccess) e = c->eng->upload_tables(d);
  if (e == cudaSuccess) e = c->eng->fill_ones(d, d.hist);
  if (e == cudaSuccess) e = c->eng->fill_ones(d, d.qd0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
  if (e != cudaSuccess) {
    pft_status s = cuda_fail(e, "pft_create initialisation");
    free_all(c);
    return s;
  }
  pft_status s = write_volume(d);
  if (s != PFT_OK) {
    free_all(c);
    return s;
  }
  *out = c;
  return PFT_OK;
}

pft_status pft_destroy(pft_ctx* ctx) {
  if (!ctx) return PFT_OK;
  if (ctx->d.stream) cudaStreamSynchronize(ctx->d.stream);
  free_all(ctx);
  return PFT_OK;
}

pft_status pft_memory_bytes(const pft_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return fail(PFT_ERR_ARG, "NULL argument");
  *bytes = ctx->d.bytes;
  return PFT_OK;
}

pft_status pft_get_stream(const pft_ctx* ctx, void** stream) {
  if (!ctx || !stream) return fail(PFT_ERR_ARG, "NULL argument");
  *stream = (void*)ctx->d.stream;
  return PFT_OK;
}

pft_status pft_synchronize(pft_ctx* ctx) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  PFT_CK(cudaStreamSynchronize(ctx->d.stream));
  return PFT_OK;
}

pft_status pft_set_fields(pft_ctx* ctx, const void* wp, const void* wm, pft_mem where) {
  if (!ctx || !wp || (!wm && !ctx->d.edw)) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  const size_t b = (size_t)d.M * felem(d);
  PFT_CK(cudaMemcpyAsync(d.wp, wp, b, kind_in(where), d.stream));
  if (d.edw) {
    PFT_CK(cudaMemsetAsync(d.wm, 0, b, d.stream));  // the one-field model keeps the second field at 0
  } else {
    PFT_CK(cudaMemcpyAsync(d.wm, wm, b, kind_in(where), d.stream));
  }
  PFT_CK(ctx->eng->prepare_fields(d));
  if (where == PFT_HOST) PFT_CK(cudaStreamSynchronize(d.stream));
  d.fields_set = true;
  d.solved = false;
  ctx->have_obs = false;
  d.step = 0;
  return PFT_OK;
}

pft_status pft_get_fields(pft_ctx* ctx, void* wp, void* wm, pft_mem where) {
  if (!ctx || !wp || (!wm && !ctx->d.edw)) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (!d.fields_set) return fail(PFT_ERR_STATE, "fields not set");
  const size_t b = (size_t)d.M * felem(d);
  PFT_CK(cudaMemcpyAsync(wp, d.wp, b, kind_out(where), d.stream));
  if (wm) PFT_CK(cudaMemcpyAsync(wm, d.wm, b, kind_out(where), d.stream));
  if (where == PFT_HOST) PFT_CK(cudaStreamSynchronize(d.stream));
  return PFT_OK;
}

pft_status pft_set_box(pft_ctx* ctx, const double L[3]) {
  if (!ctx || !L) return fail(PFT_ERR_ARG, "NULL argument");
  for (int a = 0; a < 3; a++)
    if (!(L[a] > 0.0) || !isfinite(L[a])) return fail(PFT_ERR_ARG, "box lengths must be positive");
  CtxData& d = ctx->d;
  for (int a = 0; a < 3; a++) d.L[a] = L[a];
  PFT_CK(ctx->eng->upload_tables(d));
  return write_volume(d);
}

// ------------------------------------------------------------------ checkpoints
namespace {
struct CkptHeader {
  int32_t n[3];
  int32_t Ns, kind, arch, prec;
  double L[3];
  double fA, chiN, C, B;
  uint64_t seed, instance;
  int64_t step;
};
static_assert(sizeof(CkptHeader) == 7 * 4 + 4 + 7 * 8 + 3 * 8, "checkpoint header layout");
const char kCkptMagic[8] = {'P', 'F', 'T', 'C', 'K', 'P', 'T', '1'};
const uint32_t kCkptVersion = 1;

// 64-bit FNV-1a, continued over successive buffers
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}
const uint64_t kFnvBasis = 14695981039346656037ull;

void fill_header(const CtxData& d, CkptHeader* h) {
  memset(h, 0, sizeof(*h));
  for (int a = 0; a < 3; a++) {
    h->n[a] = d.n[a];
    h->L[a] = d.L[a];
  }
  h->Ns = d.Ns;
  h->kind = (int32_t)d.kind;
  h->arch = d.edw ? (int32_t)PFT_ARCH_EDWARDS : (int32_t)PFT_ARCH_DIBLOCK;
  h->prec = (int32_t)d.prec;
  h->fA = d.fA;
  h->chiN = d.chiN;
  h->C = d.C;
  h->B = d.edw ? d.bC * d.C : 0.0;
  h->seed = d.seed;
  h->instance = d.instance;
  h->step = d.step;
}
}  // namespace

pft_status pft_save(pft_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (!d.fields_set) return fail(PFT_ERR_STATE, "pft_save before pft_set_fields");
  const size_t b = (size_t)d.M * felem(d);
  const int nf = d.edw ? 1 : 2;
  std::vector<unsigned char> f((size_t)nf * b);
  PFT_CK(cudaMemcpyAsync(f.data(), d.wp, b, cudaMemcpyDeviceToHost, d.stream));
  if (nf == 2) PFT_CK(cudaMemcpyAsync(f.data() + b, d.wm, b, cudaMemcpyDeviceToHost, d.stream));
  PFT_CK(cudaStreamSynchronize(d.stream));
  CkptHeader h;
  fill_header(d, &h);
  const uint32_t ver = kCkptVersion, hb = (uint32_t)sizeof(CkptHeader);
  uint64_t hash = kFnvBasis;
  hash = fnv1a(hash, kCkptMagic, 8);
  hash = fnv1a(hash, &ver, 4);
  hash = fnv1a(hash, &hb, 4);
  hash = fnv1a(hash, &h, sizeof(h));
  hash = fnv1a(hash, f.data(), f.size());
  const std::string tmp = std::string(path) + ".tmp";
  FILE* fp = fopen(tmp.c_str(), "wb");
  if (!fp) return fail(PFT_ERR_IO, std::string("cannot write ") + tmp);
  bool ok = fwrite(kCkptMagic, 1, 8, fp) == 8 && fwrite(&ver, 4, 1, fp) == 1 && fwrite(&hb, 4, 1, fp) == 1 &&
            fwrite(&h, sizeof(h), 1, fp) == 1 && fwrite(f.data(), 1, f.size(), fp) == f.size() &&
            fwrite(&hash, 8, 1, fp) == 1;
  ok = (fclose(fp) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return fail(PFT_ERR_IO, std::string("cannot write ") + path);
  }
  return PFT_OK;
}

pft_status pft_load(pft_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(PFT_ERR_IO, std::string("cannot open ") + path);
  char magic[8];
  uint32_t ver = 0, hb = 0;
  CkptHeader h;
  bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, kCkptMagic, 8) == 0 && fread(&ver, 4, 1, fp) == 1 &&
            ver == kCkptVersion && fread(&hb, 4, 1, fp) == 1 && hb == sizeof(CkptHeader) &&
            fread(&h, sizeof(h), 1, fp) == 1;
  if (!ok) {
    fclose(fp);
    return fail(PFT_ERR_IO, std::string(path) + " is not a checkpoint of this format");
  }
  CkptHeader mine;
  fill_header(d, &mine);
  const bool same = h.n[0] == mine.n[0] && h.n[1] == mine.n[1] && h.n[2] == mine.n[2] && h.Ns == mine.Ns &&
                    h.kind == mine.kind && h.arch == mine.arch && h.fA == mine.fA && h.chiN == mine.chiN &&
                    h.C == mine.C && h.B == mine.B;
  if (!same) {
    fclose(fp);
    return fail(PFT_ERR_ARG, std::string(path) + " holds the state of another system");
  }
  for (int a = 0; a < 3; a++) {
    if (!(h.L[a] > 0.0) || !isfinite(h.L[a])) {
      fclose(fp);
      return fail(PFT_ERR_IO, std::string(path) + ": invalid box");
    }
  }
  const size_t b = (size_t)d.M * felem(d);
  const int nf = d.edw ? 1 : 2;
  std::vector<unsigned char> f((size_t)nf * b);
  uint64_t stored = 0;
  ok = fread(f.data(), 1, f.size(), fp) == f.size() && fread(&stored, 8, 1, fp) == 1;
  char extra;
  ok = ok && fread(&extra, 1, 1, fp) == 0;
  fclose(fp);
  if (!ok) return fail(PFT_ERR_IO, std::string(path) + " is truncated or too long");
  uint64_t hash = kFnvBasis;
  hash = fnv1a(hash, kCkptMagic, 8);
  hash = fnv1a(hash, &ver, 4);
  hash = fnv1a(hash, &hb, 4);
  hash = fnv1a(hash, &h, sizeof(h));
  hash = fnv1a(hash, f.data(), f.size());
  if (hash != stored) return fail(PFT_ERR_IO, std::string(path) + " fails its hash");
  pft_status st = pft_set_box(ctx, h.L);
  if (st != PFT_OK) return st;
  st = pft_set_fields(ctx, f.data(), nf == 2 ? f.data() + b : nullptr, PFT_HOST);
  if (st != PFT_OK) return st;
  d.seed = h.seed;
  d.instance = h.instance;
  d.step = h.step;
  return PFT_OK;
}

pft_status pft_get_box(const pft_ctx* ctx, double L[3]) {
  if (!ctx || !L) return fail(PFT_ERR_ARG, "NULL argument");
  for (int a = 0; a < 3; a++) L[a] = ctx->d.L[a];
  return PFT_OK;
}

pft_status pft_solve(pft_ctx* ctx) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  CtxData& d = ctx->d;
  if (!d.fields_set) return fail(PFT_ERR_STATE, "pft_solve before pft_set_fields");
  PFT_CK(ctx->eng->enqueue_solve(d));
  d.solved = true;
  ctx->have_obs = true;
  return PFT_OK;
}

pft_status pft_get_observables(pft_ctx* ctx, pft_obs* obs) {
  if (!ctx || !obs) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (!ctx->have_obs) return fail(PFT_ERR_STATE, "no solve since the fields were set");
  PFT_CK(cudaMemcpyAsync(d.scal_host, d.scal, pft::S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
  int kerr = 0;
  PFT_CK(cudaMemcpyAsync(&kerr, d.kerr, sizeof(int), cudaMemcpyDeviceToHost, d.stream));
  PFT_CK(cudaStreamSynchronize(d.stream));
  if (kerr != 0) {
    PFT_CK(cudaMemsetAsync(d.kerr, 0, sizeof(int), d.stream));
    PFT_CK(cudaStreamSynchronize(d.stream));
    return fail(PFT_ERR_TIMEOUT, "a bounded wait in a kernel of the last solve ran out (its results are invalid)");
  }
  const double* s = d.scal_host;
  const double V = d.L[0] * d.L[1] * d.L[2];
  const double Md = (double)d.M;
  memset(obs, 0, sizeof(*obs));
  for (int j = 0; j < 2; j++) {
    obs->Q[j] = s[pft::S_Q + j];
    obs->lnQ[j] = s[pft::S_LNQ + j];
    obs->H[j] = s[pft::S_H + j];
    obs->h[j] = s[pft::S_H + j] / (d.C * V);
    obs->phiA_mean[j] = s[pft::S_PHIA + j] / Md;
    obs->phiB_mean[j] = s[pft::S_PHIB + j] / Md;
  }
  obs->force_p_rms = sqrt(s[pft::S_FP2] / Md);
  obs->force_m_rms = sqrt(s[pft::S_FM2] / Md);
  obs->fA_eff = (double)d.NsA / d.Ns;
  obs->NsA = d.NsA;
  obs->step = d.step;
  if (!isfinite(obs->Q[0]) || !isfinite(obs->Q[1]) || !isfinite(obs->H[0]) || !isfinite(obs->H[1]))
    return fail(PFT_ERR_NONFINITE, "Q or H is not finite");
  return PFT_OK;
}

pft_status pft_get_densities(pft_ctx* ctx, void* phiA, void* phiB, pft_mem where) {
  if (!ctx || !phiA || !phiB) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (!ctx->have_obs) return fail(PFT_ERR_STATE, "no solve since the fields were set");
  const size_t b = (size_t)d.M * felem(d);
  PFT_CK(cudaMemcpyAsync(phiA, d.accA, b, kind_out(where), d.stream));
  PFT_CK(cudaMemcpyAsync(phiB, d.accB, b, kind_out(where), d.stream));
  if (where == PFT_HOST) PFT_CK(cudaStreamSynchronize(d.stream));
  return PFT_OK;
}

pft_status pft_field_step(pft_ctx* ctx, pft_step_kind kind, double lam_or_dt, const void* eta_p, const void* eta_m,
                          pft_mem where) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  CtxData& d = ctx->d;
  if (!d.solved) return fail(PFT_ERR_STATE, "pft_field_step needs a solve at the current fields");
  if (kind != PFT_STEP_SCFT_EULER && kind != PFT_STEP_CL_EULER_MARUYAMA && kind != PFT_STEP_SCFT_SIS &&
      kind != PFT_STEP_CL_SIS)
    return fail(PFT_ERR_ARG, "unknown step kind");
  const bool scft_step = (kind == PFT_STEP_SCFT_EULER || kind == PFT_STEP_SCFT_SIS);
  if (scft_step && d.kind != PFT_SCFT_REAL) return fail(PFT_ERR_ARG, "SCFT step needs real SCFT fields");
  if (!scft_step && d.kind != PFT_CL_COMPLEX) return fail(PFT_ERR_ARG, "complex Langevin step needs complex fields");
  if (d.edw && (kind == PFT_STEP_SCFT_SIS || kind == PFT_STEP_CL_SIS))
    return fail(PFT_ERR_UNSUPPORTED, "semi-implicit steps are implemented for the diblock model");
  if (!isfinite(lam_or_dt) || !(lam_or_dt > 0.0)) return fail(PFT_ERR_ARG, "step size must be positive");
  if ((eta_p == nullptr) != (eta_m == nullptr)) return fail(PFT_ERR_ARG, "give both noise arrays or neither");
  const double* ep = nullptr;
  const double* em = nullptr;
  if (eta_p && !scft_step) {
    if (where == PFT_HOST) {
      double* io = (double*)ctx->io;
      PFT_CK(cudaMemcpyAsync(io, eta_p, (size_t)d.M * 8, cudaMemcpyHostToDevice, d.stream));
      PFT_CK(cudaMemcpyAsync(io + d.M, eta_m, (size_t)d.M * 8, cudaMemcpyHostToDevice, d.stream));
      ep = io;
      em = io + d.M;
    } else {
      ep = (const double*)eta_p;
      em = (const double*)eta_m;
    }
  }
  PFT_CK(ctx->eng->field_step(d, kind, lam_or_dt, ep, em));
  if (eta_p && where == PFT_HOST) PFT_CK(cudaStreamSynchronize(d.stream));
  d.step++;
  d.solved = false;
  return PFT_OK;
}

pft_status pft_gradients(pft_ctx* ctx, void* dH_dwp, void* dH_dwm, double dH_dL[3], double dlnQ_dL[3],
                         pft_mem where) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  CtxData& d = ctx->d;
  if (d.kind != PFT_SCFT_REAL) return fail(PFT_ERR_UNSUPPORTED, "gradients need real SCFT fields");
  if (d.edw) return fail(PFT_ERR_UNSUPPORTED, "gradients are implemented for the diblock model");
  if (d.scheme != 0)
    return fail(PFT_ERR_UNSUPPORTED, "gradients are the exact derivatives of the 2nd-order scheme only");
  if (!d.solved) return fail(PFT_ERR_STATE, "pft_gradients needs a solve at the current fields");
  double* gp = nullptr;
  double* gm = nullptr;
  if (where == PFT_HOST) {
    gp = dH_dwp ? (double*)ctx->io : nullptr;
    gm = dH_dwm ? (double*)ctx->io + d.M : nullptr;
  } else {
    gp = (double*)dH_dwp;
    gm = (double*)dH_dwm;
  }
  PFT_CK(ctx->eng->gradients(d, gp, gm));
  if (where == PFT_HOST) {
    if (dH_dwp) PFT_CK(cudaMemcpyAsync(dH_dwp, gp, (size_t)d.M * 8, cudaMemcpyDeviceToHost, d.stream));
    if (dH_dwm) PFT_CK(cudaMemcpyAsync(dH_dwm, gm, (size_t)d.M * 8, cudaMemcpyDeviceToHost, d.stream));
  }
  PFT_CK(cudaMemcpyAsync(d.scal_host, d.scal, pft::S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
  PFT_CK(cudaStreamSynchronize(d.stream));
  const double* s = d.scal_host;
  const double Q = s[pft::S_Q], H = s[pft::S_H];
  const double Md = (double)d.M;
  const double V = d.L[0] * d.L[1] * d.L[2];
  for (int a = 0; a < 3; a++) {
    const double g = 2.0 * d.ds / (d.L[a] * Q * Md * Md) * s[pft::S_STRESS + a];
    if (dlnQ_dL) dlnQ_dL[a] = g;
    if (dH_dL) dH_dL[a] = H / d.L[a] - d.C * V * g;
  }
  return PFT_OK;
}

pft_status pft_adjoint(pft_ctx* ctx, const void* dL_dphiA, const void* dL_dphiB, void* dL_dwp, void* dL_dwm,
                       pft_mem where) {
  if (!ctx || !dL_dphiA || !dL_dphiB || !dL_dwp || !dL_dwm) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (d.kind != PFT_SCFT_REAL || d.edw || d.scheme != 0)
    return fail(PFT_ERR_UNSUPPORTED, "the adjoint is implemented for real SCFT diblock fields and SPLIT2");
  if (!(d.concurrent && d.ckK == 1))
    return fail(PFT_ERR_UNSUPPORTED, "the adjoint needs both histories kept");
  if (!d.solved || !d.qdh) return fail(PFT_ERR_STATE, "pft_adjoint needs a solve at the current fields");
  const size_t b = (size_t)d.M * 8;
  double* io = (double*)ctx->io;  // 2 M doubles of staging: the two loss gradients
  const double *GA, *GB;
  double *gp, *gm;
  double* out_stage = nullptr;
  if (where == PFT_HOST) {
    PFT_CK(cudaMemcpyAsync(io, dL_dphiA, b, cudaMemcpyHostToDevice, d.stream));
    PFT_CK(cudaMemcpyAsync(io + d.M, dL_dphiB, b, cudaMemcpyHostToDevice, d.stream));
    GA = io;
    GB = io + d.M;
    PFT_CK(cudaMalloc(&out_stage, 2 * b));
    gp = out_stage;
    gm = out_stage + d.M;
  } else {
    GA = (const double*)dL_dphiA;
    GB = (const double*)dL_dphiB;
    gp = (double*)dL_dwp;
    gm = (double*)dL_dwm;
  }
  cudaError_t e = ctx->eng->adjoint(d, GA, GB, gp, gm);
  if (e == cudaSuccess && where == PFT_HOST) {
    e = cudaMemcpyAsync(dL_dwp, gp, b, cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dL_dwm, gm, b, cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
  }
  if (out_stage) cudaFree(out_stage);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint");
  return PFT_OK;
}

pft_status pft_profile_step(pft_ctx* ctx, int step_kind, double lam_or_dt, pft_profile* out) {
  if (!ctx || !out) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (!d.fields_set) return fail(PFT_ERR_STATE, "pft_profile_step before pft_set_fields");
  if (step_kind >= 0) {
    const bool scft_step = (step_kind == PFT_STEP_SCFT_EULER || step_kind == PFT_STEP_SCFT_SIS);
    if (step_kind > PFT_STEP_CL_SIS || scft_step != (d.kind == PFT_SCFT_REAL))
      return fail(PFT_ERR_ARG, "step kind does not match the model kind");
    if (!isfinite(lam_or_dt) || !(lam_or_dt > 0.0)) return fail(PFT_ERR_ARG, "step size must be positive");
  }
  const size_t need = (size_t)10 * d.Ns + 64;
  while (d.ev.size() < need) {
    cudaEvent_t ev;
    PFT_CK(cudaEventCreate(&ev));
    d.ev.push_back(ev);
  }
  d.ev_kind.assign(d.ev.size(), -1);
  PFT_CK(cudaStreamSynchronize(d.stream));
  d.profiling = true;
  d.ev_used = 0;
  cudaError_t e = ctx->eng->enqueue_solve(d);
  if (e == cudaSuccess && step_kind >= 0) e = ctx->eng->field_step(d, step_kind, lam_or_dt, nullptr, nullptr);
  pft::mark(d, -1);
  d.profiling = false;
  if (e != cudaSuccess) return cuda_fail(e, "profiled solve");
  PFT_CK(cudaStreamSynchronize(d.stream));
  d.solved = true;
  ctx->have_obs = true;
  if (step_kind >= 0) {
    d.step++;
    d.solved = false;
  }
  memset(out, 0, sizeof(*out));
  out->nkinds = pft::KK_COUNT;
  for (int k = 0; k < pft::KK_COUNT; k++) strncpy(out->name[k], pft::kKernelKindNames[k], 23);
  for (int i = 0; i + 1 < d.ev_used; i++) {
    float ms = 0.f;
    PFT_CK(cudaEventElapsedTime(&ms, d.ev[i], d.ev[i + 1]));
    const int k = d.ev_kind[i];
    if (k >= 0 && k < pft::KK_COUNT) {
      out->ms[k] += ms;
      out->launches[k]++;
    }
  }
  float tot = 0.f;
  if (d.ev_used > 1) PFT_CK(cudaEventElapsedTime(&tot, d.ev[0], d.ev[d.ev_used - 1]));
  out->total_ms = tot;
  // forward march: from its first launch to the first reduction; conjugate march:
  // from the first z pass after that reduction to the next reduction.
  int iF = -1, iR1 = -1, iB = -1, iR2 = -1;
  for (int i = 0; i < d.ev_used; i++) {
    const int k = d.ev_kind[i];
    const bool march_start = (k == pft::KK_Z_FWD);
    if (iF < 0 && march_start) iF = i;
    else if (iF >= 0 && iR1 < 0 && k == pft::KK_REDUCE) iR1 = i;
    else if (iR1 >= 0 && iB < 0 && march_start) iB = i;
    else if (iB >= 0 && iR2 < 0 && k == pft::KK_REDUCE) iR2 = i;
  }
  {
    // concurrent marches: each pair step advances both propagators by one contour step
    double pair_ms = out->ms[pft::KK_PAIR_STEP];
    if (out->launches[pft::KK_PAIR_STEP] > 0) {
      out->step_fwd_ms = out->step_bwd_ms = pair_ms / (2.0 * out->launches[pft::KK_PAIR_STEP]);
      iF = -1;
      iB = -1;
    }
  }
  if (iF >= 0 && iR1 > iF) {
    float ms;
    PFT_CK(cudaEventElapsedTime(&ms, d.ev[iF], d.ev[iR1]));
    out->step_fwd_ms = ms / d.Ns;
  }
  if (iB >= 0 && iR2 > iB) {
    float ms;
    PFT_CK(cudaEventElapsedTime(&ms, d.ev[iB], d.ev[iR2]));
    out->step_bwd_ms = ms / d.Ns;
  }
  // compulsory bytes of one launch of each class
  const double M = (double)d.M, Ms = (double)d.Ms;
  const double we = (double)welem(d), ze = 2.0 * ctx->eng->elem_bytes(), fe = (double)felem(d);
  out->bytes_per_launch[pft::KK_Z_FWD] = 2 * M * we + Ms * ze;
  out->bytes_per_launch[pft::KK_Y_FWD] = 2 * Ms * ze;
  out->bytes_per_launch[pft::KK_X_FUSED] = 2 * Ms * ze;
  out->bytes_per_launch[pft::KK_Y_INV] = 2 * Ms * ze;
  out->bytes_per_launch[pft::KK_Z_INV_FWD] = Ms * ze + 2 * M * we;
  out->bytes_per_launch[pft::KK_Z_INV_BWD] = Ms * ze + 3 * M * we + 2 * M * fe;
  out->bytes_per_launch[pft::KK_FIELD_STEP] = 6 * M * fe + 2 * M * we;
  out->bytes_per_launch[pft::KK_PREPARE] = 2 * M * fe + 2 * M * we;
  out->bytes_per_launch[pft::KK_PAIR_STEP] = 2 * (2 * M * we + Ms * ze) + 6 * (2 * Ms * ze) + 2 * (Ms * ze + 2 * M * we);
  if (d.scheme == 1) {
    // 4th-order step of both propagators: four z forwards, 18 strided passes, two z
    // inverses, two fused z passes (B, out, Bnext), two combining z inverses (B, full, out)
    out->bytes_per_launch[pft::KK_PAIR_STEP] = 4 * (2 * M * we + Ms * ze) + 18 * (2 * Ms * ze) +
                                                2 * (Ms * ze + 2 * M * we) + 2 * (2 * Ms * ze + 3 * M * we) +
                                                2 * (Ms * ze + 3 * M * we);
  }
  out->bytes_per_launch[pft::KK_QUADRATURE] = 2.0 * (d.Ns + 1) * M * we + 2 * M * fe;
  return PFT_OK;
}

pft_status pft_fft3d(pft_ctx* ctx, const void* in, void* out, int inverse, pft_mem where) {
  if (!ctx || !in || !out) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  const size_t b = (size_t)d.M * 16;
  PFT_CK(cudaMemcpyAsync(ctx->io, in, b, kind_in(where), d.stream));
  PFT_CK(ctx->eng->from_f64(d, ctx->io, d.spec2, 2 * d.M));
  PFT_CK(ctx->eng->fft3d(d, d.spec2, inverse));
  PFT_CK(ctx->eng->to_f64(d, d.spec2, ctx->io, 2 * d.M));
  PFT_CK(cudaMemcpyAsync(out, ctx->io, b, kind_out(where), d.stream));
  PFT_CK(cudaStreamSynchronize(d.stream));
  return PFT_OK;
}

pft_status pft_get_propagator(pft_ctx* ctx, int which, int s, void* out, pft_mem where) {
  if (!ctx || !out) return fail(PFT_ERR_ARG, "NULL argument");
  CtxData& d = ctx->d;
  if (which < 0 || which > 2) return fail(PFT_ERR_ARG, "which must be 0 (q), 1 (last qd) or 2 (qd slice)");
  if (which != 1 && (s < 0 || s > d.Ns)) return fail(PFT_ERR_ARG, "slice out of range");
  const size_t we = welem(d);
  if (which == 2) {  // slice s of the conjugate history, where the context keeps one
    if (!(d.concurrent && d.qdh && d.ckK == 1 && !d.edw && d.scheme == 0))
      return fail(PFT_ERR_UNSUPPORTED, "this context keeps no conjugate history");
    const void* src2 = (s == 0) ? (const void*)d.qd0 : (const void*)((const char*)d.qdh + (size_t)s * d.M * we);
    const long long cnt2 = d.M * (d.kind == PFT_SCFT_REAL ? 1 : 2);
    PFT_CK(ctx->eng->to_f64(d, src2, ctx->io, cnt2));
    PFT_CK(cudaMemcpyAsync(out, ctx->io, (size_t)cnt2 * 8, kind_out(where), d.stream));
    PFT_CK(cudaStreamSynchronize(d.stream));
    return PFT_OK;
  }
  const void* qd_last = d.edw ? (const void*)((const char*)d.hist + (size_t)d.Ns * d.M * we) :  // qd = q
                        (d.concurrent && d.qdh && d.ckK == 1) ? (const void*)((const char*)d.qdh + (size_t)d.Ns * d.M * we)
                                                                  : d.qd[d.Ns & 1];
  if (which == 0 && !pft::q_kept(d, s))
    return fail(PFT_ERR_UNSUPPORTED, "slice " + std::to_string(s) + " is not kept by the checkpointed history");
  const void* src = (which == 0) ? (const void*)((const char*)d.hist + (size_t)pft::q_slot(d, s) * d.M * we) : qd_last;
  const long long cnt = d.M * (d.kind == PFT_SCFT_REAL ? 1 : 2);
  PFT_CK(ctx->eng->to_f64(d, src, ctx->io, cnt));
  PFT_CK(cudaMemcpyAsync(out, ctx->io, (size_t)cnt * 8, kind_out(where), d.stream));
  PFT_CK(cudaStreamSynchronize(d.stream));
  return PFT_OK;
}

pft_status pft_debug_set_q0(pft_ctx* ctx, const void* q0, pft_mem where) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  CtxData& d = ctx->d;
  if (!q0) {
    PFT_CK(ctx->eng->fill_ones(d, d.hist));
    PFT_CK(ctx->eng->fill_ones(d, d.qd0));
  } else {
    const long long cnt = d.M * (d.kind == PFT_SCFT_REAL ? 1 : 2);
    PFT_CK(cudaMemcpyAsync(ctx->io, q0, (size_t)cnt * 8, kind_in(where), d.stream));
    PFT_CK(ctx->eng->from_f64(d, ctx->io, d.hist, cnt));
    PFT_CK(ctx->eng->from_f64(d, ctx->io, d.qd0, cnt));
  }
  PFT_CK(cudaStreamSynchronize(d.stream));
  return PFT_OK;
}

pft_status pft_launch_counts(const pft_ctx* ctx, long long* solve, long long* field_step) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  const CtxData& d = ctx->d;
  if (solve) *solve = (d.use_graph && d.graph_valid) ? d.graph_kernels : -1;
  // the update kernel and its final reduction, plus the quarter-step factors of RQM4
  if (field_step) *field_step = 2 + (d.scheme == 1 ? 1 : 0);
  return PFT_OK;
}

pft_status pft_set_plan(pft_ctx* ctx, int code, int streams) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  CtxData& d = ctx->d;
  const int plane = code & 15, xv = code >> 4;
  if (code < 0 || plane > 4 || xv > 3 || (xv && plane != 2 && plane != 3) || (xv > 1 && plane != 3) || streams < 0 ||
      streams > 1)
    return fail(PFT_ERR_ARG, "plan code in {0, 1, 2, 3, 4, 18, 19, 35, 51}, streams in {0, 1}");
  if (plane == 1 && !ctx->eng->plane_applies(d))
    return fail(PFT_ERR_UNSUPPORTED, "the plane kernel needs FP32 with ny = nz = 64 or 128 (real) or 64 (complex)");
  if (plane == 2 && !ctx->eng->sep_applies(d))
    return fail(PFT_ERR_UNSUPPORTED, "the separable march needs FP32 real fields, ny = nz and nx in {64, 128}");
  if (plane == 3 && !ctx->eng->sepp_applies(d))
    return fail(PFT_ERR_UNSUPPORTED, "the separable pencil march needs ny and nz even for real fields");
  if (plane == 3 && xv == 1 && !ctx->eng->sepp_reg_applies(d))
    return fail(PFT_ERR_UNSUPPORTED, "register lines need FP32 and x, y lengths in {4, 6, 8, 12, 16, 24, 32, 48}");
  if (plane == 3 && xv > 1 && !ctx->eng->sepp_lv_applies(d, xv))
    return fail(PFT_ERR_UNSUPPORTED, "line variant 35 needs FP32, 51 FP32 and x, y lengths in {32, 48, 64}");
  if (plane == 4 && !ctx->eng->dd_applies(d))
    return fail(PFT_ERR_UNSUPPORTED, "the double-float march needs an FP64 context and ny, nz even for real fields");
  d.plan_plane = plane;
  d.plan_xv = xv;
  d.plan_streams = streams;
  d.tuned = true;  // an explicit plan is not re-tuned
  d.graph_valid = false;
  if (d.graph) {
    cudaGraphExecDestroy(d.graph);
    d.graph = nullptr;
  }
  return PFT_OK;
}

pft_status pft_get_plan(const pft_ctx* ctx, int* plane, int* streams) {
  if (!ctx) return fail(PFT_ERR_ARG, "NULL ctx");
  if (plane) *plane = ctx->d.plan_plane + 16 * ctx->d.plan_xv;
  if (streams) *streams = ctx->d.plan_streams;
  return PFT_OK;
}

pft_status pft_get_checkpoint(const pft_ctx* ctx, int* K) {
  if (!ctx || !K) return fail(PFT_ERR_ARG, "NULL argument");
  *K = ctx->d.ckK;
  return PFT_OK;
}


pft_status pft_philox_normals(unsigned long long seed, unsigned long long instance, unsigned long long step, int field,
                              long long M, double* out_device, void* stream) {
  if (!out_device || M < 0) return fail(PFT_ERR_ARG, "bad argument");
  if (M == 0) return PFT_OK;
  PFT_CK(pft::launch_philox_normals(seed, instance, step, field, M, out_device, (cudaStream_t)stream));
  return PFT_OK;
}

pft_status pft_philox_raw(const unsigned int ctr[4], const unsigned int key[2], long long count,
                          unsigned int* out_device, void* stream) {
  if (!ctr || !key || !out_device || count < 0) return fail(PFT_ERR_ARG, "bad argument");
  if (count == 0) return PFT_OK;
  PFT_CK(pft::launch_philox_raw(ctr, key, count, out_device, (cudaStream_t)stream));
  return PFT_OK;
}

pft_status pft_debug_narrow_rn(const double* x_device, float* y_device, long long n, void* stream) {
  if (!x_device || !y_device || n < 0) return fail(PFT_ERR_ARG, "bad argument");
  if (n == 0) return PFT_OK;
  PFT_CK(pft::launch_narrow_rn(x_device, y_device, n, (cudaStream_t)stream));
  return PFT_OK;
}

}  // extern "C"
