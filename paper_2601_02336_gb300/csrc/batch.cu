// Batched SMC over many events (Sec. 3 applied to each event independently).
//
// All particles of all events live in one set of device arrays. A stage round
// advances every event that is still tempering: the stage kernels (one
// reweight cluster per event, covariance, resampling, gather) and ONE
// persistent NUTS launch over every particle of every event, whose CTAs are
// ordered by event cost so the longest segments start first. Events that have
// finished return at once from every kernel (device-side flags), so the round
// is the same launch sequence every time: it is captured once as a CUDA graph
// and replayed, and the host looks at the events' flags only every few rounds.
//
// The NUTS slot count (particles per CTA) is picked by the autotuner
// (tune.cuh) on the batch's own first stage; the results do not depend on it.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "nuts_kernel.cuh"
#include "stage.cuh"
#include "tune.cuh"

using namespace sharpy;

namespace sharpy {

int ensure_fisher_tables(sharpy_ctx* c);
int enqueue_local_metric(sharpy_ctx* c, int64_t n, const double* theta, const double* beta_ptr, double beta,
                         double* mass, double* minv, double* chol, cudaStream_t s);

constexpr int kBatchRec = 10;  // beta, ess, dlnz, eps, accept, depth, leapfrogs, divergent, active bins, ln Z
constexpr int kRoundsPerCheck = 4;
constexpr int kTuneRound = 3;  // the first run tunes the slot count on this round (full mutations on copies)

// Start of a run: beta = 0, active, no stages, ln Z = 0, nothing done.
__global__ void batch_init_kernel(int ne, double* beta, int* active, int* stage, double* lnz, double* tot,
                                  int* done) {
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    beta[e] = 0.0;
    active[e] = 1;
    stage[e] = 0;
    lnz[2 * e] = lnz[2 * e + 1] = 0.0;
    tot[2 * e] = tot[2 * e + 1] = 0.0;
    done[e] = 0;
  }
}

// Per-event stage record after the round's mutation (one CTA per event).
__global__ void __launch_bounds__(256) batch_record_kernel(const StageArgs* sa, const NutsArgs* na, int metric,
                                                           double eps_scale, int max_stages, double* rec,
                                                           double* tot, int* done) {
  __shared__ double red[5][8];
  const int e = blockIdx.x;
  const StageArgs A = sa[e];
  if (*A.active == 0) return;
  const sharpy_nuts_stats* st = na[e].stats;
  double a[5] = {0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < A.n; i += blockDim.x) {
    a[0] += st[i].accept_sum;
    a[1] += st[i].depth_sum;
    a[2] += st[i].n_leapfrog;
    a[3] += st[i].n_divergent;
    a[4] += st[i].active_bins;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 5; ++k) {
    const double v = warp_sum(a[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = *A.stage;
    double* r = rec + ((int64_t)e * max_stages + (t - 1)) * kBatchRec;
    for (int k = 0; k < 5; ++k) {
      double s = red[k][0];
      for (int w = 1; w < 8; ++w) s += red[k][w];
      r[4 + k] = s;
    }
    r[0] = *A.beta_next;
    r[1] = *A.ess;
    r[2] = *A.dlnz;
    double eps = eps_scale;
    if (metric == 0) {
      double smin = INFINITY;
      for (int j = 0; j < A.D; ++j) smin = fmin(smin, sqrt(A.cov[j * A.D + j]));
      eps = eps_scale * smin;
    }
    r[3] = eps;
    r[9] = A.lnz_acc[0];
    tot[2 * e] += r[6];
    tot[2 * e + 1] += r[8];
    done[e] = (*A.beta_next >= 1.0 || t >= max_stages) ? 1 : 0;
  }
}

}  // namespace sharpy

struct sharpy_batch {
  int device = 0;
  int ne = 0;
  std::vector<sharpy_ctx*> ctx;
  std::vector<int64_t> n, off, doff;
  std::vector<int> D;
  sharpy_smc_options opt{};
  int ndet = 1;
  int64_t n_total = 0, max_n = 0, nd_total = 0;
  int max_d = 0;
  char* d_buf = nullptr;
  double *th = nullptr, *gr = nullptr, *ll = nullptr, *th0 = nullptr, *g0 = nullptr, *l0 = nullptr;
  double *w = nullptr, *beta = nullptr, *bnext = nullptr, *dlnz = nullptr, *ess = nullptr, *sumw = nullptr;
  double *lnz = nullptr, *cov = nullptr, *rec = nullptr, *tot = nullptr;
  double *pminv = nullptr, *pchol = nullptr;  // per-particle metric (option 2): [N_e][D_e][D_e] per event
  std::vector<int64_t> moff;                   // offset of event e in pminv / pchol
  unsigned long long* csum = nullptr;
  int32_t* anc = nullptr;
  sharpy_nuts_stats* st = nullptr;
  int *flags = nullptr, *active = nullptr, *stage = nullptr, *done = nullptr;
  StageArgs* d_stage = nullptr;
  NutsArgs* d_nuts = nullptr;
  NutsArgs* d_trial = nullptr;
  int2* d_map[kNumSlotChoices] = {};
  unsigned n_cta[kNumSlotChoices] = {};
  std::vector<StageArgs> h_stage;
  std::vector<NutsArgs> h_nuts, h_trial;
  int* h_flags = nullptr;  // pinned: active[ne], done[ne]
  int slots = 0;           // 0 until tuned
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_slots = 0;
  int64_t graph_kernels = 0;  // kernel nodes of the captured round
  int64_t launches = 0;       // kernels launched by the last run (graph replays count their nodes)
};

static void batch_free(sharpy_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_buf);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  delete b;
}

namespace {
template <class T>
T* carve(char*& p, size_t count) {
  T* r = reinterpret_cast<T*>(p);
  p += ((count * sizeof(T) + 255) / 256) * 256;
  return r;
}

int slot_index(int slots) {
  for (int i = 0; i < kNumSlotChoices; ++i)
    if (kSlotChoices[i] == slots) return i;
  return 0;
}

int enqueue_round_stage(sharpy_batch* b, cudaStream_t s) {
  StageArgs none{};
  int rc = enqueue_stage_kernels(none, b->d_stage, b->ne, b->max_n, b->max_d, true, true, 0ull, s);
  if (rc || b->opt.metric != 2) return rc;
  // local metric of every event's resampled particles at its new beta
  for (int e = 0; e < b->ne && !rc; ++e)
    rc = enqueue_local_metric(b->ctx[e], b->n[e], b->th + b->doff[e], b->beta + e, 0.0, nullptr,
                              b->pminv + b->moff[e], b->pchol + b->moff[e], s);
  return rc;
}

int enqueue_round_nuts(sharpy_batch* b, const NutsArgs* args, int slots, cudaStream_t s) {
  const int i = slot_index(slots);
  NutsArgs P{};
  P.batch = args;
  P.cta_map = b->d_map[i];
  P.local_metric = b->opt.metric == 2 ? 1 : 0;
  return launch_nuts(b->opt.precision, b->ndet, slots, P, b->n_cta[i], s);
}

int enqueue_round_record(sharpy_batch* b, cudaStream_t s) {
  batch_record_kernel<<<b->ne, 256, 0, s>>>(b->d_stage, b->d_nuts, b->opt.metric, b->opt.eps_scale,
                                            b->opt.max_stages, b->rec, b->tot, b->done);
  SHARPY_CUDA_TRY(cudaGetLastError());
  return SHARPY_OK;
}

// Capture one round (stage kernels, NUTS, record) as a graph for `slots`.
int capture_round(sharpy_batch* b, int slots) {
  if (b->exec && b->graph_slots == slots) return SHARPY_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  SHARPY_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  int rc = enqueue_round_stage(b, b->cap);
  if (!rc) rc = enqueue_round_nuts(b, b->d_nuts, slots, b->cap);
  if (!rc) rc = enqueue_round_record(b, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess || !g) return SHARPY_ECUDA;
  b->graph = g;
  SHARPY_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  b->graph_slots = slots;
  size_t nn = 0;
  SHARPY_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) SHARPY_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
  b->graph_kernels = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType ty;
    SHARPY_CUDA_TRY(cudaGraphNodeGetType(nodes[i], &ty));
    if (ty == cudaGraphNodeTypeKernel) ++b->graph_kernels;
  }
  return SHARPY_OK;
}
}  // namespace

extern "C" {

int sharpy_batch_create(sharpy_batch** out, sharpy_ctx* const* events, int n_events, const int64_t* n_particles,
                        const sharpy_smc_options* o) {
  if (!out || !events || !n_particles || !o || n_events < 1 || n_events > (1 << 16)) return SHARPY_EINVAL;
  *out = nullptr;
  if (!(o->alpha > 0.0 && o->alpha <= 1.0) || o->n_mut < 0 || o->max_depth < 0 || o->max_depth > SHARPY_MAX_DEPTH ||
      o->max_stages < 1 || !(o->eps_scale > 0.0) || (o->metric != 0 && o->metric != 1 && o->metric != 2) ||
      (o->precision != SHARPY_FP64 && o->precision != SHARPY_MIXED && o->precision != SHARPY_MIXED_SPLIT))
    return SHARPY_EINVAL;
  sharpy_batch* b = new sharpy_batch();
  b->ne = n_events;
  b->opt = *o;
  b->ctx.assign(events, events + n_events);
  const int kind = events[0] ? events[0]->model.model : -1;
  for (int e = 0; e < n_events; ++e) {
    sharpy_ctx* c = events[e];
    const int64_t ne = n_particles[e];
    int rc = check_ctx(c, true);
    if (rc || c->device != events[0]->device || c->model.model != kind || ne < 1 || ne > kMaxParticles ||
        c->first_id != 0) {
      delete b;
      return rc ? rc : SHARPY_EINVAL;
    }
    const int nd = c->model.model == SHARPY_MODEL_TAYLORF2 ? c->ev.n_det : 1;
    if (e == 0) b->ndet = nd;
    if (nd != b->ndet) {
      delete b;
      return SHARPY_EINVAL;
    }
    b->n.push_back(ne);
    b->off.push_back(b->n_total);
    b->doff.push_back(b->nd_total);
    b->D.push_back(c->model.n_dim);
    b->n_total += ne;
    b->nd_total += ne * c->model.n_dim;
    b->max_n = std::max(b->max_n, ne);
    b->max_d = std::max(b->max_d, c->model.n_dim);
  }
  b->device = events[0]->device;
  const int E = n_events;
  int64_t nm = 0;  // per-particle metric entries
  for (int e = 0; e < E; ++e) {
    b->moff.push_back(nm);
    nm += b->n[e] * b->D[e] * b->D[e];
    if (o->metric == 2 && events[e]->model.model == SHARPY_MODEL_TAYLORF2) {
      const int rc = ensure_fisher_tables(events[e]);
      if (rc) {
        delete b;
        return rc;
      }
    }
  }
  if (o->metric != 2) nm = 0;
  const int64_t N = b->n_total, ND = b->nd_total, S = o->max_stages;
  const int DD = b->max_d * b->max_d;
  // CTA maps: events by decreasing cost (bins x detectors), each event's CTAs in order
  std::vector<int> order(E);
  for (int e = 0; e < E; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return events[x]->ev.n_bins * events[x]->ev.n_det > events[y]->ev.n_bins * events[y]->ev.n_det;
  });
  std::vector<std::vector<int2>> maps(kNumSlotChoices);
  for (int i = 0; i < kNumSlotChoices; ++i) {
    for (int e : order) {
      const int64_t blocks = (b->n[e] + kSlotChoices[i] - 1) / kSlotChoices[i];
      for (int64_t j = 0; j < blocks; ++j) maps[i].push_back(make_int2(e, (int)j));
    }
    b->n_cta[i] = (unsigned)maps[i].size();
  }
  size_t bytes = 0;
  auto add = [&](size_t count, size_t elem) { bytes += ((count * elem + 255) / 256) * 256; };
  add(ND, 8); add(ND, 8); add(N, 8);        // th, gr, ll
  add(ND, 8); add(ND, 8); add(N, 8);        // th0, g0, l0
  add(N, 8); add(N, 8); add(N, 4);          // w, csum, anc
  add(N, sizeof(sharpy_nuts_stats));
  add(5 * (size_t)E, 8); add(2 * (size_t)E, 8); add((size_t)E * DD, 8); add((size_t)E * S * kBatchRec, 8);
  add(2 * (size_t)E, 8);                    // tot
  add(3 * (size_t)E, 4);                    // active, done, stage
  add(nm, 8); add(nm, 8);                   // per-particle metric
  add(E, sizeof(StageArgs)); add(E, sizeof(NutsArgs)); add(E, sizeof(NutsArgs));
  for (int i = 0; i < kNumSlotChoices; ++i) add(maps[i].size(), sizeof(int2));
  if (cudaSetDevice(b->device) != cudaSuccess || cudaMalloc((void**)&b->d_buf, bytes) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_flags, 2 * E * sizeof(int)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    batch_free(b);
    return SHARPY_ENOMEM;
  }
  char* p = b->d_buf;
  b->th = carve<double>(p, ND);
  b->gr = carve<double>(p, ND);
  b->ll = carve<double>(p, N);
  b->th0 = carve<double>(p, ND);
  b->g0 = carve<double>(p, ND);
  b->l0 = carve<double>(p, N);
  b->w = carve<double>(p, N);
  b->csum = carve<unsigned long long>(p, N);
  b->anc = carve<int32_t>(p, N);
  b->st = carve<sharpy_nuts_stats>(p, N);
  double* sc = carve<double>(p, 5 * (size_t)E);
  b->beta = sc;
  b->bnext = sc + E;
  b->dlnz = sc + 2 * E;
  b->ess = sc + 3 * E;
  b->sumw = sc + 4 * E;
  b->lnz = carve<double>(p, 2 * (size_t)E);
  b->cov = carve<double>(p, (size_t)E * DD);
  b->rec = carve<double>(p, (size_t)E * S * kBatchRec);
  b->tot = carve<double>(p, 2 * (size_t)E);
  b->flags = carve<int>(p, 3 * (size_t)E);
  b->pminv = carve<double>(p, nm);
  b->pchol = carve<double>(p, nm);
  b->active = b->flags;
  b->done = b->flags + E;
  b->stage = b->flags + 2 * E;
  b->d_stage = carve<StageArgs>(p, E);
  b->d_nuts = carve<NutsArgs>(p, E);
  b->d_trial = carve<NutsArgs>(p, E);
  for (int i = 0; i < kNumSlotChoices; ++i) b->d_map[i] = carve<int2>(p, maps[i].size());
  // per-event descriptors (keys are filled in by each run)
  b->h_stage.resize(E);
  b->h_nuts.resize(E);
  b->h_trial.resize(E);
  for (int e = 0; e < E; ++e) {
    sharpy_ctx* c = events[e];
    const int64_t o1 = b->off[e], od = b->doff[e];
    StageArgs& A = b->h_stage[e];
    A = StageArgs{};
    A.n = b->n[e];
    A.D = b->D[e];
    A.theta = b->th + od;
    A.lnl = b->ll + o1;
    A.grad = b->gr + od;
    A.beta_prev_ptr = b->beta + e;
    A.alpha = o->alpha;
    A.w = b->w + o1;
    A.csum = b->csum + o1;
    A.anc = b->anc + o1;
    A.th0 = b->th0 + od;
    A.g0 = b->g0 + od;
    A.l0 = b->l0 + o1;
    A.beta_next = b->bnext + e;
    A.dlnz = b->dlnz + e;
    A.ess = b->ess + e;
    A.sum_w = b->sumw + e;
    A.cov = b->cov + (size_t)e * DD;
    A.lnz_acc = b->lnz + 2 * e;
    A.beta_state = b->beta + e;
    A.status = c->d_status;
    A.active = b->active + e;
    A.stage = b->stage + e;
    A.max_stages = o->max_stages;
    NutsArgs& U = b->h_nuts[e];
    U = NutsArgs{};
    U.m = c->model;
    U.ev = c->ev;
    U.n = b->n[e];
    U.theta = A.theta;
    U.lnl = A.lnl;
    U.grad = A.grad;
    U.beta_ptr = b->beta + e;
    U.minv = o->metric == 1 ? A.cov : nullptr;
    U.cov_step = o->metric == 0 ? A.cov : nullptr;
    U.pminv = o->metric == 2 ? b->pminv + b->moff[e] : nullptr;
    U.pchol = o->metric == 2 ? b->pchol + b->moff[e] : nullptr;
    U.local_metric = o->metric == 2 ? 1 : 0;
    U.step = o->eps_scale;
    U.max_depth = o->max_depth;
    U.n_steps = o->n_mut;
    U.stats = b->st + o1;
    U.status = c->d_status;
    U.active = A.active;
    U.stage = A.stage;
    // the tuner's trial: one transition on the gather sources (free between stages)
    NutsArgs& T = b->h_trial[e];
    T = U;
    T.theta = A.th0;
    T.lnl = A.l0;
    T.grad = A.g0;
    T.n_steps = o->n_mut;
  }
  for (int i = 0; i < kNumSlotChoices; ++i)
    if (cudaMemcpy(b->d_map[i], maps[i].data(), maps[i].size() * sizeof(int2), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      batch_free(b);
      return SHARPY_ECUDA;
    }
  *out = b;
  return SHARPY_OK;
}

void sharpy_batch_destroy(sharpy_batch* b) { batch_free(b); }

int sharpy_batch_slots(sharpy_batch* b) { return b ? b->slots : 0; }

int64_t sharpy_batch_launches(sharpy_batch* b) { return b ? b->launches : -1; }

int sharpy_batch_set_slots(sharpy_batch* b, int slots) {
  if (!b || (slots != 0 && slots != 4 && slots != 8 && slots != 16 && slots != 32)) return SHARPY_EINVAL;
  b->slots = slots;
  return SHARPY_OK;
}

int sharpy_batch_run(sharpy_batch* b, const uint64_t* keys, sharpy_batch_result* results, int* rounds,
                     sharpy_stream stream) {
  if (!b || !keys || !results) return SHARPY_EINVAL;
  SHARPY_CUDA_TRY(cudaSetDevice(b->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int E = b->ne;
  nvtxRangePushA("sharpy_batch_run");
  struct RangeEnd {
    ~RangeEnd() { nvtxRangePop(); }
  } range_end;
  for (int e = 0; e < E; ++e) {
    b->h_stage[e].key = keys[e];
    b->h_nuts[e].key = keys[e];
    b->h_trial[e].key = keys[e];
  }
  // pageable sources: the copies have left the host buffers when the calls return
  SHARPY_CUDA_TRY(cudaMemcpyAsync(b->d_stage, b->h_stage.data(), E * sizeof(StageArgs), cudaMemcpyHostToDevice, s));
  SHARPY_CUDA_TRY(cudaMemcpyAsync(b->d_nuts, b->h_nuts.data(), E * sizeof(NutsArgs), cudaMemcpyHostToDevice, s));
  SHARPY_CUDA_TRY(cudaMemcpyAsync(b->d_trial, b->h_trial.data(), E * sizeof(NutsArgs), cudaMemcpyHostToDevice, s));
  batch_init_kernel<<<1, 256, 0, s>>>(E, b->beta, b->active, b->stage, b->lnz, b->tot, b->done);
  SHARPY_CUDA_TRY(cudaGetLastError());
  // kernels of one round: reweight, covariance, systematic, save, gather, the
  // local metric of every event (metric 2), NUTS, record
  const int64_t round_kernels = 7 + (b->opt.metric == 2 ? E : 0);
  b->launches = 1 + 2 * (int64_t)E;  // init, then prior draw and ln L of every event
  int rc = SHARPY_OK;
  for (int e = 0; e < E && !rc; ++e) {
    sharpy_ctx* c = b->ctx[e];
    double* th = b->th + b->doff[e];
    rc = sharpy_prior_sample(c, b->n[e], th, keys[e], 0, stream);
    if (!rc) rc = sharpy_loglike_grad(c, b->n[e], th, b->ll + b->off[e], b->gr + b->doff[e], b->opt.precision, stream);
  }
  if (rc) return rc;
  // The first rounds run eagerly. Until the batch is tuned, the slot count
  // comes from the CTA count (about two 32-slot CTAs per SM, else 16, else 8)
  // and round kTuneRound times each candidate on full mutations of copies of
  // the particles (the state of a mid-run stage, not the first one, whose
  // trees all reach the depth limit).
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int guess = b->n_cta[slot_index(32)] >= 2u * (unsigned)sms ? 32
                    : b->n_cta[slot_index(16)] >= 2u * (unsigned)sms ? 16 : 8;
  const int eager = b->slots ? 1 : kTuneRound;
  int nr = 0;
  for (int r = 1; r <= eager; ++r) {
    if ((rc = enqueue_round_stage(b, s))) return rc;
    if (r == kTuneRound && !b->slots) {
      SHARPY_CUDA_TRY(cudaMemcpyAsync(b->h_flags, b->flags, 2 * E * sizeof(int), cudaMemcpyDeviceToHost, s));
      SHARPY_CUDA_TRY(cudaStreamSynchronize(s));
      bool running = false;
      for (int e = 0; e < E; ++e) running = running || (b->h_flags[e] && !b->h_flags[E + e]);
      if (running) {
        TuneCandidate cands[kNumSlotChoices];
        auto trial = [&](int slots, cudaStream_t ts) -> int {
          SHARPY_CUDA_TRY(cudaMemcpyAsync(b->th0, b->th, b->nd_total * sizeof(double), cudaMemcpyDeviceToDevice, ts));
          SHARPY_CUDA_TRY(cudaMemcpyAsync(b->g0, b->gr, b->nd_total * sizeof(double), cudaMemcpyDeviceToDevice, ts));
          SHARPY_CUDA_TRY(cudaMemcpyAsync(b->l0, b->ll, b->n_total * sizeof(double), cudaMemcpyDeviceToDevice, ts));
          return enqueue_round_nuts(b, b->d_trial, slots, ts);
        };
        for (int i = 0; i < kNumSlotChoices; ++i) cands[i].slots = kSlotChoices[i];
        if ((rc = tune_slots(cands, kNumSlotChoices, trial, s, &b->slots))) return rc;
        b->launches += 2 * kNumSlotChoices;  // one untimed and one timed trial per candidate
      }
    }
    if ((rc = enqueue_round_nuts(b, b->d_nuts, b->slots ? b->slots : guess, s))) return rc;
    if ((rc = enqueue_round_record(b, s))) return rc;
    b->launches += round_kernels;
    ++nr;
  }
  if ((rc = capture_round(b, b->slots ? b->slots : guess))) return rc;
  for (;;) {
    SHARPY_CUDA_TRY(cudaMemcpyAsync(b->h_flags, b->flags, 2 * E * sizeof(int), cudaMemcpyDeviceToHost, s));
    SHARPY_CUDA_TRY(cudaStreamSynchronize(s));
    bool running = false;
    for (int e = 0; e < E; ++e) running = running || (b->h_flags[e] && !b->h_flags[E + e]);
    if (!running || nr >= b->opt.max_stages) break;
    const int k = std::min(kRoundsPerCheck, b->opt.max_stages - nr);
    for (int i = 0; i < k; ++i) SHARPY_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    b->launches += k * b->graph_kernels;
    nr += k;
  }
  // results
  std::vector<double> lz(2 * E), bt(E), tt(2 * E);
  std::vector<int> sg(E);
  SHARPY_CUDA_TRY(cudaMemcpyAsync(lz.data(), b->lnz, 2 * E * sizeof(double), cudaMemcpyDeviceToHost, s));
  SHARPY_CUDA_TRY(cudaMemcpyAsync(bt.data(), b->beta, E * sizeof(double), cudaMemcpyDeviceToHost, s));
  SHARPY_CUDA_TRY(cudaMemcpyAsync(tt.data(), b->tot, 2 * E * sizeof(double), cudaMemcpyDeviceToHost, s));
  SHARPY_CUDA_TRY(cudaMemcpyAsync(sg.data(), b->stage, E * sizeof(int), cudaMemcpyDeviceToHost, s));
  SHARPY_CUDA_TRY(cudaStreamSynchronize(s));
  int out = SHARPY_OK;
  for (int e = 0; e < E; ++e) {
    results[e].lnz = lz[2 * e];
    results[e].beta = bt[e];
    results[e].n_leapfrog = tt[2 * e];
    results[e].active_bins = tt[2 * e + 1];
    results[e].n_stages = sg[e];
    results[e].pad = 0;
    if (!std::isfinite(bt[e])) out = SHARPY_ENONFINITE;
    if (bt[e] < 1.0 && out == SHARPY_OK) out = SHARPY_ETIMEOUT;
  }
  if (rounds) *rounds = nr;
  return out;
}

int sharpy_batch_particles(sharpy_batch* b, int e, double* theta, double* lnl, sharpy_stream stream) {
  if (!b || e < 0 || e >= b->ne) return SHARPY_EINVAL;
  SHARPY_CUDA_TRY(cudaSetDevice(b->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (theta)
    SHARPY_CUDA_TRY(cudaMemcpyAsync(theta, b->th + b->doff[e], b->n[e] * b->D[e] * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
  if (lnl)
    SHARPY_CUDA_TRY(cudaMemcpyAsync(lnl, b->ll + b->off[e], b->n[e] * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return SHARPY_OK;
}

int sharpy_batch_stages(sharpy_batch* b, int e, sharpy_stage* stages, int cap, int* n) {
  if (!b || e < 0 || e >= b->ne || !stages || cap < 0 || !n) return SHARPY_EINVAL;
  SHARPY_CUDA_TRY(cudaSetDevice(b->device));
  const int S = b->opt.max_stages;
  std::vector<double> r((size_t)S * kBatchRec);
  int t = 0;
  SHARPY_CUDA_TRY(cudaMemcpy(&t, b->stage + e, sizeof(int), cudaMemcpyDeviceToHost));
  SHARPY_CUDA_TRY(cudaMemcpy(r.data(), b->rec + (size_t)e * S * kBatchRec, r.size() * sizeof(double),
                             cudaMemcpyDeviceToHost));
  const int m = std::min(std::min(t, S), cap);
  const double per = (double)b->n[e] * (b->opt.n_mut > 0 ? b->opt.n_mut : 1);
  double prev = 0.0;
  for (int i = 0; i < m; ++i) {
    const double* q = &r[(size_t)i * kBatchRec];
    sharpy_stage& g = stages[i];
    g.beta = q[0];
    g.dbeta = q[0] - prev;
    prev = q[0];
    g.ess = q[1];
    g.dlnz = q[2];
    g.eps = q[3];
    g.accept_mean = q[4] / per;
    g.depth_mean = q[5] / per;
    g.n_leapfrog = (int64_t)q[6];
    g.n_divergent = (int)q[7];
    g.pad = 0;
    g.active_bins = q[8];
    g.nuts_ms = 0.0;
    g.reweight_ms = 0.0;
    g.lnz = q[9];
  }
  *n = m;
  return SHARPY_OK;
}

}  // extern "C"
