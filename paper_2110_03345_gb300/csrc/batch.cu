// Uneven batches of independent 2D problems (forward modelling or gradients):
// one multi-problem stencil launch per time step, the whole run captured
// once into a CUDA graph (fwi_batch_*).
#include "fwi_plan.cuh"

using namespace fwi;

#define FWI_TRY_B(call)              \
  do {                               \
    fwi_status s_ = (call);          \
    if (s_ != FWI_OK) return bail(s_); \
  } while (0)

#define CUDA_TRY_B(call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bail(fail(FWI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)));   \
  } while (0)

// ---------------------------------------------------------------------------
// Uneven batches of independent 2D problems (forward modelling).
// ---------------------------------------------------------------------------
namespace {

struct BatchProblem {
  fwi_plan* P = nullptr;
  Call c;
  Carve tabC{nullptr};
  DevTable src;
  fwi_problem prob{};
  std::vector<double> srcxyz, recxyz;
};

}  // namespace

struct fwi_batch {
  std::vector<BatchProblem*> items;   // sorted by nt, longest first
  cudaStream_t st = nullptr;          // the caller's stream
  cudaStream_t ws = nullptr;          // internal non-blocking stream the runs (and the capture) use
  cudaEvent_t ready = nullptr;
  int device = 0;
  int R = 4;
  bool vd = false;
  bool tma = true;      // TMA-staged multi-problem kernel (else shared-memory staged)
  int shape = 0;        // tile shape of the batch's kernels
  bool uniform_w = false;   // every problem has the same stencil weights
  AxisW w[2] = {};          // {x, y} weights when uniform_w
  MultiDesc* d_desc = nullptr;
  MultiUnit* d_units = nullptr;
  bool grad = false;                  // a gradient batch
  // gradient batches: one stream per problem, forked from ws and joined back
  // (independent branches of the graph that the GPU runs concurrently)
  std::vector<cudaStream_t> bst;
  std::vector<cudaEvent_t> bjoin;
  cudaEvent_t fork = nullptr;
  std::vector<int> active_units;      // units of the problems still running at step n
  int max_steps = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  fwi_batch_stats stats{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~fwi_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(d_desc);
    cudaFree(d_units);
    for (BatchProblem* b : items) {
      if (b->P) b->P->st = st;   // (a gradient batch moved it to its branch stream)
      fwi_plan_destroy(b->P);
      delete b;
    }
    for (cudaEvent_t e : bjoin) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (cudaStream_t s : bst) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ready) cudaEventDestroy(ready);
    if (ws) cudaStreamDestroy(ws);
  }
};

namespace {

// Every step of every problem (and the final sampling / trace transposition)
// enqueued on b->st; captured into a graph when b->use_graph.
// Gradient batches: each problem's whole gradient (the forward with its
// history, misfit, adjoint with the imaging condition, finalisation; the
// single-problem kernels of fwi_gradient) on its own stream, forked from ws
// and joined back, so that a graph holds one independent branch per problem.
fwi_status batch_enqueue_grad(fwi_batch* b) {
  int64_t launches = 0, updates = 0;
  CUDA_TRY(cudaEventRecord(b->fork, b->ws));
  for (size_t i = 0; i < b->items.size(); ++i) {
    BatchProblem* it = b->items[i];
    Call& c = it->c;
    fwi_plan* P = it->P;
    const int ns = it->prob.geom.nshots;
    const size_t fs = (size_t)P->L.fstride;
    P->st = b->bst[i];
    CUDA_TRY(cudaStreamWaitEvent(P->st, b->fork, 0));
    CUDA_TRY(cudaMemsetAsync(P->d_flags, 0, sizeof(int) * 4, P->st));
    CUDA_TRY(cudaMemsetAsync(c.W.G, 0, fs * ns * sizeof(float), P->st));
    c.launches = 0;
    FWI_TRY(gradient_forward_batch(c, 0, 0, ns, it->src, it->prob.observed, it->prob.traces));
    FWI_TRY(gradient_adjoint_batch(c, 0, 0, ns, it->src));
    cudaError_t e = launch_grad_finalize(P->L, c.W.G, (ns + c.pl.S - 1) / c.pl.S, 1.0 / (P->dt * P->dt),
                                         it->prob.grad_m, P->d_flags, P->st);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    launches += c.launches + 1;
    updates += 2 * (int64_t)ns * P->L.nx * P->L.ny * (it->prob.nt - 1);
    CUDA_TRY(cudaEventRecord(b->bjoin[i], P->st));
    CUDA_TRY(cudaStreamWaitEvent(b->ws, b->bjoin[i], 0));
  }
  b->stats.launches = launches;
  b->stats.updates = updates;
  return FWI_OK;
}

fwi_status batch_enqueue(fwi_batch* b) {
  if (b->grad) return batch_enqueue_grad(b);
  int64_t launches = 0, updates = 0;
  for (int n = 0; n < b->max_steps; ++n) {
    cudaError_t e = b->tma ? launch_step2d_tma_multi(b->d_desc, b->d_units, b->active_units[n], n,
                                                     b->R, b->vd, b->shape,
                                                     b->uniform_w ? b->w : nullptr, b->ws)
                           : launch_step2d_multi(b->d_desc, b->d_units, b->active_units[n], n,
                                                 b->R, b->vd, b->ws);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("multi-problem step: ") + cudaGetErrorString(e));
    ++launches;
  }
  for (BatchProblem* it : b->items) {
    Call& c = it->c;
    const int nt = it->prob.nt;
    const int ns = it->prob.geom.nshots;
    const int nrec = it->prob.geom.nrec;
    float* last = ((nt - 1) & 1) ? c.W.U1 : c.W.U0;   // u^{nt-1}
    StepParams p = base_params(c);
    p.B = ns;
    p.u = last;
    p.smp_node = c.smp_node;
    p.smp_w = c.smp_w;
    p.smp_out = c.W.D;
    p.nrec = nrec;
    p.smp_off = (long long)(nt - 1) * c.pl.B * nrec;
    cudaError_t e = launch_sample(p, b->ws);
    if (e == cudaSuccess)
      e = launch_traces_out(c.W.D, it->prob.traces, c.pl.B, 0, ns, nrec, nt, it->P->d_flags, b->ws);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
    launches += 2;
    updates += (int64_t)ns * it->P->L.nx * it->P->L.ny * (nt - 1);
  }
  b->stats.launches = launches;
  b->stats.updates = updates;
  return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_batch_create(fwi_batch** out, int nprob, const fwi_problem* probs,
                            const fwi_options* opt, size_t hbm_budget_bytes, void* stream,
                            int use_graph) {
  if (!out || !probs || nprob < 1) return fail(FWI_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  fwi_batch* b = new fwi_batch();
  b->st = reinterpret_cast<cudaStream_t>(stream);
  b->use_graph = use_graph != 0;
  auto bail = [&](fwi_status s) { delete b; return s; };
  if (cudaGetDevice(&b->device) != cudaSuccess) return bail(fail(FWI_ERR_CUDA, "no CUDA device"));
  size_t used = 0;
  for (int i = 0; i < nprob; ++i) {
    const fwi_problem& pr = probs[i];
    if (pr.grid.ndim != 2) return bail(fail(FWI_ERR_UNSUPPORTED, "batches hold 2D problems"));
    if (i == 0) {
      b->R = pr.grid.order / 2;
      b->vd = pr.model.rho != nullptr;
    } else if (pr.grid.order / 2 != b->R || (pr.model.rho != nullptr) != b->vd) {
      return bail(fail(FWI_ERR_UNSUPPORTED, "a batch shares one stencil order and density mode"));
    }
    const bool g = pr.observed != nullptr;
    if (i == 0) b->grad = g;
    else if (g != b->grad)
      return bail(fail(FWI_ERR_INVALID_ARG, "a batch holds only forward or only gradient problems"));
    if (!pr.wavelet || (!g && !pr.traces) || (g && (!pr.grad_m || !pr.misfit)))
      return bail(fail(FWI_ERR_INVALID_ARG, "problem arrays are NULL"));
    if (pr.model.alpha0 ||
        (opt && (opt->time_order == 4 || opt->interp != FWI_INTERP_LINEAR || opt->boundary != 0)))
      return bail(fail(FWI_ERR_UNSUPPORTED,
                       "batches run the leapfrog with the sponge, without attenuation and with bi-/tri-linear points"));
    BatchProblem* it = new BatchProblem();
    b->items.push_back(it);
    it->prob = pr;
    if (!pr.geom.src_xyz || !pr.geom.rec_xyz) return bail(fail(FWI_ERR_INVALID_ARG, "coordinates are NULL"));
    it->srcxyz.assign(pr.geom.src_xyz, pr.geom.src_xyz + (size_t)pr.geom.nshots * pr.geom.nsrc * 2);
    it->recxyz.assign(pr.geom.rec_xyz, pr.geom.rec_xyz + (size_t)pr.geom.nrec * 2);
    it->prob.geom.src_xyz = it->srcxyz.data();
    it->prob.geom.rec_xyz = it->recxyz.data();
    const size_t left = hbm_budget_bytes ? (hbm_budget_bytes > used ? hbm_budget_bytes - used : 1) : 0;
    FWI_TRY_B(fwi_plan_create(&it->P, &pr.grid, pr.nt, pr.dt, left, stream));
    fwi_options o{};
    o.batch = pr.geom.nshots;   // every shot of the problem in one batch
    o.tile = opt ? opt->tile : 0;                  // 0: the default (TMA-staged) variant
    o.shots_per_cta = opt ? opt->shots_per_cta : 0;
    it->P->opt = o;   // (gradients: the full history if it fits the budget left, else checkpoints)
    FWI_TRY_B(begin_call(it->P, &it->prob.model, &it->prob.geom, pr.wavelet, g, it->c, it->tabC));
    if (it->c.pl.B != pr.geom.nshots)
      return bail(fail(FWI_ERR_BUDGET, "problem " + std::to_string(i) + " does not fit the budget with all its shots"));
    if (i == 0) {
      b->tma = it->c.pl.tma;
      b->shape = it->c.pl.shape;
      if (!b->tma && b->shape != 0)
        return bail(fail(FWI_ERR_UNSUPPORTED, "batches run the TMA variants or shared-memory variant 1"));
    }
    Carve srcC = it->tabC;
    FWI_TRY_B(build_source_table(it->c, 0, pr.geom.nshots, srcC, it->src));
    const size_t fs = (size_t)it->P->L.fstride;
    CUDA_TRY_B(cudaMemsetAsync(it->c.W.U0, 0, fs * pr.geom.nshots * sizeof(float), b->st));
    CUDA_TRY_B(cudaMemsetAsync(it->c.W.U1, 0, fs * pr.geom.nshots * sizeof(float), b->st));
    used += it->c.pl.bytes;
  }
  std::stable_sort(b->items.begin(), b->items.end(),
                   [](const BatchProblem* a, const BatchProblem* c) { return a->prob.nt > c->prob.nt; });
  if (b->grad && b->tma && !(opt && opt->shots_per_cta > 0) && !b->items.empty()) {
    // the problems' branches run concurrently, so the shot groups are sized
    // for the batch as a whole: the largest S <= 6 whose CTAs over all the
    // problems still make four waves of two per SM (each plan alone lowers S
    // until its own problem does)
    const int nsm = b->items[0]->P->nsm;
    int S = 6;
    for (; S > 1; --S) {
      long long ctas = 0;
      for (const BatchProblem* it : b->items)
        ctas += it->c.T.ntiles() * (long long)((it->prob.geom.nshots + S - 1) / S);
      if (ctas >= 8LL * nsm) break;
    }
    for (BatchProblem* it : b->items) it->c.pl.S = std::min(S, it->c.pl.B);
  }
  for (const BatchProblem* it : b->items) {
    b->stats.shots_per_cta = std::max(b->stats.shots_per_cta, it->c.pl.S);
    if (it->c.pl.K > 0) b->stats.checkpointed++;
  }
  if (!b->items.empty()) {
    b->w[0] = b->items[0]->P->wx;
    b->w[1] = b->items[0]->P->wy;
    b->uniform_w = true;
    for (const BatchProblem* it : b->items)
      if (std::memcmp(&it->P->wx, &b->w[0], sizeof(AxisW)) != 0 ||
          std::memcmp(&it->P->wy, &b->w[1], sizeof(AxisW)) != 0)
        b->uniform_w = false;
  }
  // descriptors and units (problems longest first: the running ones are a prefix)
  std::vector<MultiDesc> desc(b->items.size());
  std::vector<MultiUnit> units;
  std::vector<int> prefix;
  for (size_t k = 0; k < b->items.size(); ++k) {
    BatchProblem* it = b->items[k];
    Call& c = it->c;
    StepParams p = base_params(c);
    p.B = it->prob.geom.nshots;
    p.inj_off = it->src.off;
    p.inj_loc = it->src.loc;
    p.inj_vidx = it->src.vidx;
    p.inj_row = it->src.row;
    p.inj_w = it->src.w;
    p.vals = it->prob.wavelet;
    p.smp_node = c.smp_node;
    p.smp_w = c.smp_w;
    p.smp_out = c.W.D;
    p.nrec = it->prob.geom.nrec;
    p.S = 1;
    p.flags = it->P->d_flags + 1;
    p.S = c.pl.S;
    desc[k].p = p;
    desc[k].U0 = c.W.U0;
    desc[k].U1 = c.W.U1;
    desc[k].gx = c.T.gx;
    desc[k].nt = it->prob.nt;
    if (b->tma) {
      const CUtensorMap* m0 = find_map(c, c.W.U0);
      const CUtensorMap* m1 = find_map(c, c.W.U1);
      const CUtensorMap* i0 = find_map(c, c.W.U0, 1);
      const CUtensorMap* i1 = find_map(c, c.W.U1, 1);
      if (!m0 || !m1 || !i0 || !i1)
        return bail(fail(FWI_ERR_INVALID_ARG, "internal: missing tensor maps"));
      desc[k].map0 = *m0;
      desc[k].map1 = *m1;
      desc[k].imap0 = *i0;
      desc[k].imap1 = *i1;
    }
    // units: one per tile and shot group (TMA kernels loop S shots in a CTA)
    const int groups = b->tma ? (p.B + p.S - 1) / p.S : p.B;
    long long rank = 0;
    for (int gr = 0; gr < groups; ++gr)
      for (int ty = 0; ty < c.T.gy; ++ty)
        for (int tx = 0; tx < c.T.gx; ++tx) units.push_back({(int)k, tx, ty, gr, rank++});
    prefix.push_back((int)units.size());
  }
  b->max_steps = b->items.empty() ? 0 : b->items[0]->prob.nt - 1;
  b->active_units.assign(std::max(b->max_steps, 0), 0);
  for (int n = 0; n < b->max_steps; ++n) {
    int cnt = 0;
    for (size_t k = 0; k < b->items.size(); ++k)
      if (n < b->items[k]->prob.nt - 1) cnt = prefix[k];
    b->active_units[n] = cnt;
  }
  CUDA_TRY_B(cudaMalloc(&b->d_desc, desc.size() * sizeof(MultiDesc)));
  CUDA_TRY_B(cudaMalloc(&b->d_units, std::max<size_t>(units.size(), 1) * sizeof(MultiUnit)));
  CUDA_TRY_B(cudaMemcpy(b->d_desc, desc.data(), desc.size() * sizeof(MultiDesc), cudaMemcpyHostToDevice));
  if (!units.empty())
    CUDA_TRY_B(cudaMemcpy(b->d_units, units.data(), units.size() * sizeof(MultiUnit), cudaMemcpyHostToDevice));
  CUDA_TRY_B(cudaEventCreate(&b->e0));
  CUDA_TRY_B(cudaEventCreate(&b->e1));
  CUDA_TRY_B(cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming));
  CUDA_TRY_B(cudaStreamCreateWithFlags(&b->ws, cudaStreamNonBlocking));
  if (b->grad) {
    CUDA_TRY_B(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (size_t i = 0; i < b->items.size(); ++i) {
      cudaStream_t s = nullptr;
      cudaEvent_t e = nullptr;
      CUDA_TRY_B(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      b->bst.push_back(s);
      CUDA_TRY_B(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      b->bjoin.push_back(e);
    }
  }
  CUDA_TRY_B(cudaStreamSynchronize(b->st));
  if (b->use_graph) {
    // set the kernels' attributes outside the capture (zero-unit launch), then
    // capture every launch of a run
    {
      cudaError_t e = b->tma ? launch_step2d_tma_multi(b->d_desc, b->d_units, 0, 0, b->R, b->vd,
                                                       b->shape,
                                                       b->uniform_w ? b->w : nullptr, b->ws)
                             : launch_step2d_multi(b->d_desc, b->d_units, 0, 0, b->R, b->vd, b->ws);
      if (e != cudaSuccess) return bail(fail(FWI_ERR_CUDA, cudaGetErrorString(e)));
    }
    CUDA_TRY_B(cudaStreamBeginCapture(b->ws, cudaStreamCaptureModeThreadLocal));
    fwi_status s = batch_enqueue(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->ws, &g);
    if (s != FWI_OK) {
      if (g) cudaGraphDestroy(g);
      return bail(s);
    }
    if (e != cudaSuccess) return bail(fail(FWI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e)));
    b->graph = g;
    CUDA_TRY_B(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  b->stats.problems = (int)b->items.size();
  b->stats.units = (int64_t)units.size();
  *out = b;
  return FWI_OK;
}

fwi_status fwi_batch_run(fwi_batch* b) {
  if (!b) return fail(FWI_ERR_INVALID_ARG, "batch is NULL");
  CUDA_TRY(cudaSetDevice(b->device));
  // the run follows whatever the caller enqueued on its stream (inputs)
  CUDA_TRY(cudaEventRecord(b->ready, b->st));
  CUDA_TRY(cudaStreamWaitEvent(b->ws, b->ready, 0));
  for (BatchProblem* it : b->items) {
    const size_t fs = (size_t)it->P->L.fstride;
    const int ns = it->prob.geom.nshots;
    CUDA_TRY(cudaMemsetAsync(it->c.W.U0, 0, fs * ns * sizeof(float), b->ws));
    CUDA_TRY(cudaMemsetAsync(it->c.W.U1, 0, fs * ns * sizeof(float), b->ws));
    CUDA_TRY(cudaMemsetAsync(it->P->d_flags, 0, sizeof(int) * 4, b->ws));
  }
  CUDA_TRY(cudaEventRecord(b->e0, b->ws));
  if (b->use_graph) {
    CUDA_TRY(cudaGraphLaunch(b->exec, b->ws));
  } else {
    FWI_TRY(batch_enqueue(b));
  }
  CUDA_TRY(cudaEventRecord(b->e1, b->ws));
  CUDA_TRY(cudaStreamSynchronize(b->ws));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, b->e0, b->e1));
  b->stats.run_ms = ms;
  for (BatchProblem* it : b->items) {
    int flags[4];
    CUDA_TRY(cudaMemcpy(flags, it->P->d_flags, sizeof(flags), cudaMemcpyDeviceToHost));
    if (flags[0]) return fail(FWI_ERR_NONFINITE, "non-finite values in a batched problem");
    if (flags[1] & 2) return fail(FWI_ERR_TIMEOUT, "a bounded wait on a TMA copy timed out");
    if (b->grad) CUDA_TRY(cudaMemcpy(it->prob.misfit, it->P->d_J, sizeof(double), cudaMemcpyDeviceToHost));
  }
  return FWI_OK;
}

fwi_status fwi_batch_stats_get(const fwi_batch* b, fwi_batch_stats* out) {
  if (!b || !out) return fail(FWI_ERR_INVALID_ARG, "NULL argument");
  *out = b->stats;
  return FWI_OK;
}

void fwi_batch_destroy(fwi_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->st);
  delete b;
}

}  // extern "C"
