// pft_batch.cu -- many independent systems of uneven grid and contour sizes advanced
// together.  Instances are grouped into classes of equal field kind and grid; within a
// class the members are sorted by contour length, so at contour step s the instances
// still marching are a prefix of the class and one launch per pass covers all of them
// (blockIdx.y = instance).  One field update of every instance -- both marches of all
// classes, each instance's reductions and its field step -- is captured once as a CUDA
// graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "pft_batch.cuh"
#include "pft_engine.h"

namespace {

// The plans the batch autotuner times, in the order of BatchClass::tuned_ms.
const int kBatchPlans[PFT_BATCH_PLANS] = {0, 1, 2, 3, 19, 35, 51};
int batch_plan_index(int plan) {
  for (int k = 0; k < PFT_BATCH_PLANS; k++)
    if (kBatchPlans[k] == plan) return k;
  return -1;
}

struct BatchClass {
  pft::BatchGeom g;
  pft_kind kind;
  std::vector<int> members;   // instance indices, Ns descending
  int maxNs = 0;
  std::vector<int> active;    // active[s-1]: members with Ns >= s
  pft::BatchStep* d_fwd = nullptr;  // [maxNs][K]
  pft::BatchStep* d_bwd = nullptr;
  // plan 0: one march after the other, the quadrature fused into the conjugate march;
  // plan 1: both marches in the same launches (entries 2k / 2k+1 of a step), the z passes
  // of consecutive steps fused, the quadrature after the marches over both histories;
  // plan 2: the separable march on the plane and x kernels (FP32 real, ny = nz = nx in
  // {64, 128}); plan 3: the separable march on pencils -- both marches per launch, the
  // quadrature after them, as plan 1; plans 19, 35, 51: plan 3 with line variant 1, 2, 3
  // (register lines; 32-line tiles; twice the elements a thread in 32-line tiles)
  int plan = 3;
  pft::BatchStep* d_conc = nullptr;  // [maxNs][2K]
  pft::BatchStep* d_sep = nullptr;   // the same entries with the per-axis factors of plans 2, 3
  float tuned_ms[PFT_BATCH_PLANS] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f};  // autotuner timings of kBatchPlans
  // the class's branch of the captured update: its marches, reductions and field steps
  // run on their own stream, forked from and joined back into the batch stream, so that
  // the classes overlap on the GPU
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

__global__ void k_batch_increment(unsigned long long* __restrict__ c, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] += 1ull;
}

pft_status bfail(pft_status s, const std::string& m) {
  pft::set_error(m);
  return s;
}

pft_status bcuda(cudaError_t e, const char* what) {
  pft::set_error(std::string(what) + ": " + cudaGetErrorString(e));
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PFT_ERR_OOM : PFT_ERR_CUDA;
}

}  // namespace

struct pft_batch {
  std::vector<pft_ctx*> inst;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<BatchClass> classes;
  unsigned long long* d_steps = nullptr;
  int* d_err = nullptr;  // error word of the bounded waits in the separable plane kernel
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  double g_lam = -1.0, g_dt = -1.0;
  long long launches = 0;
  double units = 0.0;
};

namespace {

void batch_free(pft_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& c : b->classes) {
    if (c.d_fwd) cudaFree(c.d_fwd);
    if (c.d_bwd) cudaFree(c.d_bwd);
    if (c.d_conc) cudaFree(c.d_conc);
    if (c.d_sep) cudaFree(c.d_sep);
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.done) cudaEventDestroy(c.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_steps) cudaFree(b->d_steps);
  if (b->d_err) cudaFree(b->d_err);
  for (pft_ctx* c : b->inst)
    if (c) pft_destroy(c);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Per-instance step arguments of both marches.
void fill_steps(const pft_ctx* c, int s, bool bwd, pft::BatchStep* st) {
  const pft::CtxData& d = c->d;
  const size_t we = (d.prec == PFT_FP64 ? 8 : 4) * (d.kind == PFT_SCFT_REAL ? 1 : 2);
  const size_t slice = (size_t)d.M * we;
  const char* hist = (const char*)d.hist;
  memset(st, 0, sizeof(*st));
  if (!bwd) {
    st->in = hist + (size_t)(s - 1) * slice;
    st->B = (s <= d.NsA) ? d.BA : d.BB;
    st->out = (void*)(hist + (size_t)s * slice);
  } else {
    const int nb = d.Ns + 1 - s;
    st->B = (nb <= d.NsA) ? d.BA : d.BB;
    st->in = (s == 1) ? d.qd0 : d.qd[(s - 1) & 1];
    st->out = d.qd[s & 1];
    const int pn = d.Ns - s;
    st->partner = hist + (size_t)pn * slice;
    double cA = 0.0, cB = 0.0;
    if (d.NsA > 0 && pn <= d.NsA) cA = (pn == 0 || pn == d.NsA) ? 0.5 : 1.0;
    if (d.NsA < d.Ns && pn >= d.NsA) cB = (pn == d.NsA || pn == d.Ns) ? 0.5 : 1.0;
    st->cA = cA;
    st->cB = cB;
    st->accA = d.accA;
    st->accB = d.accB;
  }
  st->spec = d.spec;
  const char* t = (const char*)d.tables;
  for (int a = 0; a < 4; a++) st->tw[a] = t + d.tw_off[a];
  for (int a = 0; a < 3; a++) st->d[a] = t + d.d_off[a];
}

// Entries of step s of both marches of one instance (plan 1): forward into the q history,
// conjugate into the qd history, each with the factor of its next step for the fused z
// passes (none at the instance's last step).
void fill_pair(const pft_ctx* c, int s, pft::BatchStep* f, pft::BatchStep* b) {
  const pft::CtxData& d = c->d;
  const size_t we = (d.prec == PFT_FP64 ? 8 : 4) * (d.kind == PFT_SCFT_REAL ? 1 : 2);
  const size_t slice = (size_t)d.M * we;
  const char* hist = (const char*)d.hist;
  char* qdh = (char*)d.qdh;
  memset(f, 0, sizeof(*f));
  memset(b, 0, sizeof(*b));
  const int nb = d.Ns + 1 - s;
  f->in = hist + (size_t)(s - 1) * slice;
  f->B = (s <= d.NsA) ? d.BA : d.BB;
  f->out = (void*)(hist + (size_t)s * slice);
  f->spec = d.spec;
  b->in = (s == 1) ? d.qd0 : (const void*)(qdh + (size_t)(s - 1) * slice);
  b->B = (nb <= d.NsA) ? d.BA : d.BB;
  b->out = qdh + (size_t)s * slice;
  b->spec = d.spec2;
  if (s < d.Ns) {
    f->Bnext = (s + 1 <= d.NsA) ? d.BA : d.BB;
    b->Bnext = (nb - 1 <= d.NsA) ? d.BA : d.BB;
  }
  const char* t = (const char*)d.tables;
  for (int a = 0; a < 4; a++) f->tw[a] = b->tw[a] = t + d.tw_off[a];
  for (int a = 0; a < 3; a++) f->d[a] = b->d[a] = t + d.d_off[a];
}

// qd histories and the pair-step table of a class (plan 1), once.
pft_status prepare_pairs(pft_batch* b, BatchClass& c) {
  if (c.d_conc) return PFT_OK;
  for (int i : c.members) {
    pft::CtxData& d = b->inst[i]->d;
    if (d.qdh) continue;
    const size_t we = (d.prec == PFT_FP64 ? 8 : 4) * (d.kind == PFT_SCFT_REAL ? 1 : 2);
    const size_t bytes = (size_t)(d.Ns + 1) * d.M * we;
    cudaError_t e = cudaMalloc(&d.qdh, bytes);
    if (e != cudaSuccess) return bcuda(e, "batch qd history");
    d.bytes += bytes;
  }
  const int K = (int)c.members.size();
  std::vector<pft::BatchStep> h((size_t)c.maxNs * 2 * K);
  for (int s = 1; s <= c.maxNs; s++)
    for (int k = 0; k < c.active[s - 1]; k++)
      fill_pair(b->inst[c.members[k]], s, &h[((size_t)(s - 1) * K + k) * 2], &h[((size_t)(s - 1) * K + k) * 2 + 1]);
  const size_t bytes = h.size() * sizeof(pft::BatchStep);
  cudaError_t e = cudaMalloc(&c.d_conc, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(c.d_conc, h.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(e, "batch pair-step table");
  // the separable plans: the same entries with each member's full-axis factors
  for (int s = 1; s <= c.maxNs; s++)
    for (int k = 0; k < c.active[s - 1]; k++) {
      const pft::CtxData& d = b->inst[c.members[k]]->d;
      const char* t = (const char*)d.tables;
      for (int m = 0; m < 2; m++) {
        pft::BatchStep& x = h[((size_t)(s - 1) * K + k) * 2 + m];
        for (int a = 0; a < 3; a++) x.d[a] = t + d.sd_off[a];
      }
    }
  e = cudaMalloc(&c.d_sep, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(c.d_sep, h.data(), bytes, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? PFT_OK : bcuda(e, "batch separable step table");
}

// Both marches and the densities of one class under its plan, on `sm` (the members'
// context streams must be `sm` too).
pft_status record_class_solve(pft_batch* b, BatchClass& c, long long* launches, cudaStream_t sm) {
  const int K = (int)c.members.size();
  pft::Engine* eng = b->inst[c.members[0]]->eng;
  if (c.plan == 2 || (c.plan & 15) == 3) {
    for (int j = 0; j <= c.maxNs; j++) {
      const pft::BatchStep* st = c.d_sep + (size_t)(j == 0 ? 0 : j - 1) * 2 * K;
      const int nact = 2 * c.active[j == 0 ? 0 : j - 1];
      cudaError_t e = eng->batch_sep_launch(c.g, st, j, nact, c.plan, b->d_err, sm);
      if (e != cudaSuccess) return bcuda(e, "batched separable step");
      *launches += (c.plan != 2 && j > 0) ? 2 : 1;
    }
    for (int i : c.members) {
      pft_ctx* x = b->inst[i];
      cudaError_t e = x->eng->finish_both(x->d);
      if (e != cudaSuccess) return bcuda(e, "batched quadrature");
      *launches += 4;
    }
    return PFT_OK;
  }
  if (c.plan == 1) {
    for (int s = 1; s <= c.maxNs; s++) {
      const pft::BatchStep* st = c.d_conc + (size_t)(s - 1) * 2 * K;
      cudaError_t e = eng->batch_pair_step(c.g, st, 2 * c.active[s - 1], s == 1, sm);
      if (e != cudaSuccess) return bcuda(e, "batched pair step");
      *launches += eng->batch_pair_launches(c.g, s == 1);
    }
    for (int i : c.members) {
      pft_ctx* x = b->inst[i];
      cudaError_t e = x->eng->solve_mid(x->d);
      if (e == cudaSuccess) e = x->eng->quadrature(x->d);
      if (e == cudaSuccess) e = x->eng->solve_tail(x->d);
      if (e != cudaSuccess) return bcuda(e, "batched quadrature");
      *launches += 6;
    }
    return PFT_OK;
  }
  for (int march = 0; march < 2; march++) {
    for (int s = 1; s <= c.maxNs; s++) {
      const pft::BatchStep* st = (march ? c.d_bwd : c.d_fwd) + (size_t)(s - 1) * K;
      cudaError_t e = eng->batch_contour_step(c.g, st, c.active[s - 1], march, sm);
      if (e != cudaSuccess) return bcuda(e, "batched contour step");
      *launches += 5;
    }
    for (int i : c.members) {
      pft_ctx* x = b->inst[i];
      cudaError_t e = march ? x->eng->solve_tail(x->d) : x->eng->solve_mid(x->d);
      if (e != cudaSuccess) return bcuda(e, "batched reductions");
      *launches += march ? 2 : 3;
    }
  }
  return PFT_OK;
}

// One field update of every instance: each class on its own stream (forked from and
// joined back into b->stream), then the step counters on b->stream.
pft_status record_update(pft_batch* b, double lam, double dt) {
  long long launches = 0;
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch fork");
  for (auto& c : b->classes) {  // plan-1 tables are prepared before any capture
    if ((e = cudaStreamWaitEvent(c.stream, b->fork, 0)) != cudaSuccess) return bcuda(e, "class fork");
    for (int i : c.members) b->inst[i]->d.stream = c.stream;
    pft_status s = record_class_solve(b, c, &launches, c.stream);
    for (int i : c.members) {
      if (s != PFT_OK) break;
      pft_ctx* x = b->inst[i];
      const bool scft = (x->d.kind == PFT_SCFT_REAL);
      e = x->eng->field_step(x->d, scft ? PFT_STEP_SCFT_EULER : PFT_STEP_CL_EULER_MARUYAMA, scft ? lam : dt, nullptr,
                             nullptr);
      if (e != cudaSuccess) s = bcuda(e, "batched field step");
      launches += 2;
    }
    for (int i : c.members) b->inst[i]->d.stream = b->stream;
    if (s != PFT_OK) return s;
    if ((e = cudaEventRecord(c.done, c.stream)) != cudaSuccess) return bcuda(e, "class join");
    if ((e = cudaStreamWaitEvent(b->stream, c.done, 0)) != cudaSuccess) return bcuda(e, "class join");
  }
  const int n = (int)b->inst.size();
  k_batch_increment<<<(n + 255) / 256, 256, 0, b->stream>>>(b->d_steps, n);
  launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(e, "batched step counter");
  b->launches = launches;
  return PFT_OK;
}

}  // namespace

extern "C" {

pft_status pft_batch_create(pft_batch** out, int count, const pft_instance_desc* descs, pft_precision precision,
                            void* stream) {
  if (!out) return bfail(PFT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !descs) return bfail(PFT_ERR_ARG, "need at least one instance description");
  for (int i = 0; i < count; i++)
    if (descs[i].model.arch != PFT_ARCH_DIBLOCK)
      return bfail(PFT_ERR_UNSUPPORTED, "batch instance " + std::to_string(i) + ": batches hold diblock systems");
  for (int i = 0; i < count; i++)
    for (int a = 0; a < 3; a++)
      if (!pft::batch_axis_supported(descs[i].grid.n[a]))
        return bfail(PFT_ERR_SHAPE, "batch instance " + std::to_string(i) + ": grid sizes must be one of " +
                                        "4,6,8,12,16,24,32,48,64");
  pft_batch* b = new pft_batch();
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return bcuda(e, "cudaStreamCreate");
    }
    b->own_stream = true;
  }
  b->inst.assign(count, nullptr);
  for (int i = 0; i < count; i++) {
    pft_opts o;
    memset(&o, 0, sizeof(o));
    o.precision = precision;
    o.use_graph = 1;
    o.stream = b->stream;
    o.seed = descs[i].seed;
    o.instance = (unsigned long long)i;
    o.march = PFT_MARCH_PASSES;
    o.checkpoint = 1;
    pft_status s = pft_create(&b->inst[i], &descs[i].grid, &descs[i].chain, &descs[i].model, &o);
    if (s != PFT_OK) {
      std::string msg = pft_last_error();
      batch_free(b);
      return bfail(s, "batch instance " + std::to_string(i) + ": " + msg);
    }
    b->units += 2.0 * (double)b->inst[i]->d.M * b->inst[i]->d.Ns;
    // members march one propagator at a time with the quadrature inside the conjugate
    // march (the batched launches already fill the GPU), in both batch modes
    b->inst[i]->d.concurrent = false;
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    batch_free(b);
    return bcuda(e, "batch fork event");
  }
  e = cudaMalloc(&b->d_err, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 4 * sizeof(int), b->stream);
  if (e != cudaSuccess) {
    batch_free(b);
    return bcuda(e, "batch error word");
  }
  e = cudaMalloc(&b->d_steps, sizeof(unsigned long long) * count);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_steps, 0, sizeof(unsigned long long) * count, b->stream);
  if (e != cudaSuccess) {
    batch_free(b);
    return bcuda(e, "batch step counters");
  }
  for (int i = 0; i < count; i++) b->inst[i]->d.step_dev = b->d_steps + i;
  // classes of equal kind and grid, members by descending contour length
  std::map<std::tuple<int, int, int, int>, int> index;
  for (int i = 0; i < count; i++) {
    const pft::CtxData& d = b->inst[i]->d;
    auto key = std::make_tuple((int)d.kind, d.n[0], d.n[1], d.n[2]);
    auto it = index.find(key);
    if (it == index.end()) {
      BatchClass c;
      for (int a = 0; a < 3; a++) c.g.n[a] = d.n[a];
      c.g.kind = d.kind;
      c.g.nzh = d.nzh;
      c.kind = d.kind;
      // the default plan (measured on GB300 with the 256-instance batch): the separable
      // march on the plane kernel where it applies, else on pencils
      pft::Engine* eng = b->inst[i]->eng;
      c.plan = eng->batch_plan_ok(c.g, 2) ? 2 : (eng->batch_plan_ok(c.g, 3) ? 3 : 1);
      index[key] = (int)b->classes.size();
      b->classes.push_back(c);
      it = index.find(key);
    }
    b->classes[it->second].members.push_back(i);
  }
  for (auto& c : b->classes) {
    std::stable_sort(c.members.begin(), c.members.end(),
                     [&](int x, int y) { return b->inst[x]->d.Ns > b->inst[y]->d.Ns; });
    const int K = (int)c.members.size();
    c.maxNs = b->inst[c.members[0]]->d.Ns;
    c.active.assign(c.maxNs, 0);
    for (int s = 1; s <= c.maxNs; s++)
      for (int k = 0; k < K; k++)
        if (b->inst[c.members[k]]->d.Ns >= s) c.active[s - 1] = k + 1;
    std::vector<pft::BatchStep> hf((size_t)c.maxNs * K), hb((size_t)c.maxNs * K);
    for (int s = 1; s <= c.maxNs; s++)
      for (int k = 0; k < c.active[s - 1]; k++) {
        fill_steps(b->inst[c.members[k]], s, false, &hf[(size_t)(s - 1) * K + k]);
        fill_steps(b->inst[c.members[k]], s, true, &hb[(size_t)(s - 1) * K + k]);
      }
    const size_t bytes = hf.size() * sizeof(pft::BatchStep);
    e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_fwd, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_bwd, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_fwd, hf.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_bwd, hb.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      batch_free(b);
      return bcuda(e, "batch step tables");
    }
  }
  *out = b;
  return PFT_OK;
}

pft_status pft_batch_destroy(pft_batch* b) {
  if (!b) return PFT_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_free(b);
  return PFT_OK;
}

pft_status pft_batch_set_fields(pft_batch* b, int i, const void* wp, const void* wm, pft_mem where) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return bfail(PFT_ERR_ARG, "bad batch or instance index");
  pft_status s = pft_set_fields(b->inst[i], wp, wm, where);
  if (s != PFT_OK) return s;
  cudaError_t e = cudaMemsetAsync(b->d_steps + i, 0, sizeof(unsigned long long), b->stream);
  return e == cudaSuccess ? PFT_OK : bcuda(e, "reset step counter");
}

pft_status pft_batch_get_fields(pft_batch* b, int i, void* wp, void* wm, pft_mem where) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return bfail(PFT_ERR_ARG, "bad batch or instance index");
  return pft_get_fields(b->inst[i], wp, wm, where);
}

pft_status pft_batch_get_densities(pft_batch* b, int i, void* phiA, void* phiB, pft_mem where) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return bfail(PFT_ERR_ARG, "bad batch or instance index");
  return pft_get_densities(b->inst[i], phiA, phiB, where);
}

pft_status pft_batch_get_observables(pft_batch* b, int i, pft_obs* obs) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return bfail(PFT_ERR_ARG, "bad batch or instance index");
  return pft_get_observables(b->inst[i], obs);
}

pft_status pft_batch_run(pft_batch* b, int updates, double lam, double dt, pft_batch_mode mode) {
  if (!b || updates < 0) return bfail(PFT_ERR_ARG, "bad argument");
  if (!(lam > 0.0) || !(dt > 0.0) || !isfinite(lam) || !isfinite(dt))
    return bfail(PFT_ERR_ARG, "lam and dt must be positive");
  for (pft_ctx* x : b->inst)
    if (!x->d.fields_set) return bfail(PFT_ERR_STATE, "every batch instance needs pft_batch_set_fields first");
  for (auto& c : b->classes) {  // allocations and table uploads happen outside any capture
    if (c.plan == 0) continue;
    pft_status s = prepare_pairs(b, c);
    if (s != PFT_OK) return s;
  }
  if (mode == PFT_BATCH_GRAPHED) {
    if (!b->graph || lam != b->g_lam || dt != b->g_dt) {
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bcuda(e, "batch capture");
      pft_status s = record_update(b, lam, dt);
      e = cudaStreamEndCapture(b->stream, &g);
      if (s != PFT_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return bcuda(e, "batch capture end");
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bcuda(e, "batch graph instantiate");
      b->g_lam = lam;
      b->g_dt = dt;
    }
    for (int u = 0; u < updates; u++) {
      cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
      if (e != cudaSuccess) return bcuda(e, "batch graph launch");
    }
  } else if (mode == PFT_BATCH_PER_INSTANCE) {
    const int n = (int)b->inst.size();
    for (int u = 0; u < updates; u++) {
      for (pft_ctx* x : b->inst) {
        const bool scft = (x->d.kind == PFT_SCFT_REAL);
        cudaError_t e = x->eng->enqueue_solve(x->d);
        if (e == cudaSuccess)
          e = x->eng->field_step(x->d, scft ? PFT_STEP_SCFT_EULER : PFT_STEP_CL_EULER_MARUYAMA, scft ? lam : dt,
                                 nullptr, nullptr);
        if (e != cudaSuccess) return bcuda(e, "per-instance update");
      }
      k_batch_increment<<<(n + 255) / 256, 256, 0, b->stream>>>(b->d_steps, n);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return bcuda(e, "step counter");
    }
  } else {
    return bfail(PFT_ERR_ARG, "unknown batch mode");
  }
  for (pft_ctx* x : b->inst) {
    x->d.step += updates;
    x->d.solved = false;
    if (updates > 0) x->have_obs = true;
  }
  return PFT_OK;
}

pft_status pft_batch_autotune(pft_batch* b) {
  if (!b) return bfail(PFT_ERR_ARG, "NULL batch");
  for (pft_ctx* x : b->inst)
    if (!x->d.fields_set) return bfail(PFT_ERR_STATE, "every batch instance needs pft_batch_set_fields first");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return bcuda(e, "autotune events");
  pft_status st = PFT_OK;
  for (auto& c : b->classes) {
    float best = -1.f;
    int bplan = c.plan;
    pft::Engine* eng = b->inst[c.members[0]]->eng;
    for (int pi = 0; pi < PFT_BATCH_PLANS && st == PFT_OK; pi++) {
      const int plan = kBatchPlans[pi];
      if (!eng->batch_plan_ok(c.g, plan)) continue;
      c.plan = plan;
      if (plan >= 1 && (st = prepare_pairs(b, c)) != PFT_OK) break;
      long long n = 0;
      if ((st = record_class_solve(b, c, &n, b->stream)) != PFT_OK) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      if ((st = record_class_solve(b, c, &n, b->stream)) != PFT_OK) break;
      cudaEventRecord(e1, b->stream);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        st = bcuda(e, "autotune timing");
        break;
      }
      c.tuned_ms[pi] = ms;
      if (best < 0.f || ms < best) {
        best = ms;
        bplan = plan;
      }
    }
    c.plan = bplan;
    if (st != PFT_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (b->graph) {  // the next graphed run captures the chosen plans
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return st;
}

pft_status pft_batch_set_plan(pft_batch* b, int cls, int plan) {
  if (!b || cls < -1 || cls >= (int)b->classes.size()) return bfail(PFT_ERR_ARG, "bad batch or class index");
  if (batch_plan_index(plan) < 0) return bfail(PFT_ERR_ARG, "plan must be 0, 1, 2, 3, 19, 35 or 51");
  if (cls >= 0 && !b->inst[b->classes[cls].members[0]]->eng->batch_plan_ok(b->classes[cls].g, plan))
    return bfail(PFT_ERR_UNSUPPORTED, "plan " + std::to_string(plan) + " does not apply to class " + std::to_string(cls));
  for (int k = 0; k < (int)b->classes.size(); k++) {
    BatchClass& c = b->classes[k];
    // all classes (cls = -1): the classes the plan applies to
    if ((cls < 0 || k == cls) && b->inst[c.members[0]]->eng->batch_plan_ok(c.g, plan)) c.plan = plan;
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return PFT_OK;
}

pft_status pft_batch_class_info(const pft_batch* b, int cls, int n[3], int* kind, int* members, int* plan,
                                float tuned_ms[PFT_BATCH_PLANS]) {
  if (!b || cls < 0 || cls >= (int)b->classes.size()) return bfail(PFT_ERR_ARG, "bad batch or class index");
  const BatchClass& c = b->classes[cls];
  if (n)
    for (int a = 0; a < 3; a++) n[a] = c.g.n[a];
  if (kind) *kind = (int)c.kind;
  if (members) *members = (int)c.members.size();
  if (plan) *plan = c.plan;
  if (tuned_ms)
    for (int k = 0; k < PFT_BATCH_PLANS; k++) tuned_ms[k] = c.tuned_ms[k];
  return PFT_OK;
}

pft_status pft_batch_synchronize(pft_batch* b) {
  if (!b) return bfail(PFT_ERR_ARG, "NULL batch");
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch synchronize");
  if (err != 0) {
    cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    return bfail(PFT_ERR_TIMEOUT, "a bounded wait in a separable plane kernel ran out (the last updates are invalid)");
  }
  return PFT_OK;
}

pft_status pft_batch_info(const pft_batch* b, double* units_per_update, int* nclasses, long long* launches) {
  if (!b) return bfail(PFT_ERR_ARG, "NULL batch");
  if (units_per_update) *units_per_update = b->units;
  if (nclasses) *nclasses = (int)b->classes.size();
  if (launches) *launches = b->launches;
  return PFT_OK;
}

pft_status pft_batch_get_stream(const pft_batch* b, void** stream) {
  if (!b || !stream) return bfail(PFT_ERR_ARG, "NULL argument");
  *stream = (void*)b->stream;
  return PFT_OK;
}

}  // extern "C"
