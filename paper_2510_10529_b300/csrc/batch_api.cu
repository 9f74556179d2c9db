// Batched multi-problem execution, host side.
//
// invdft_batch_step steps every problem of a batch at once.  Each problem runs
// its own L-BFGS step (line search, forward solves, adjoint, gradient) on its
// own host thread and CUDA stream, so the independent problems overlap on the
// GPU.  Their Chebyshev filters -- the bulk of a forward solve -- meet in a
// filter service: a problem that reaches its filter posts it and waits; when
// every problem still running has posted (or finished), the last one to
// arrive launches a single cooperative persistent kernel (batch.cu) over the
// work queue of all posted problems, replaying a captured CUDA graph of that
// launch sequence when one exists for the same set of problems.  The column
// chunk of each problem's items is chosen per (order, width) class by a small
// autotuner on the first step.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "solvers.h"

struct invdft_batch_ctx;

namespace invdft {

invdft_status lbfgs_step(Ctx *c, const double *rd, const double *w, double *vxc,
                         invdft_stats *stats, cudaStream_t s);

struct BatchState {
  std::vector<Ctx *> probs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_ready, ev_end;
  cudaStream_t bstream = nullptr;
  cudaEvent_t ev_done = nullptr, ev_start = nullptr, t0 = nullptr, t1 = nullptr;
  BatchProb *h_probs = nullptr;      // pinned staging of the launch's descriptors
  int *h_err = nullptr;              // pinned copy of the device error word
  BatchProb *d_probs = nullptr;
  unsigned *d_done = nullptr;        // [kMaxBatch][kMaxBatchDeg + 1] phase counters
  int *d_queue = nullptr, *d_err = nullptr;
  int grid = 0, degree = 0;
  std::vector<int> tileC;            // column chunk of each problem's items
  bool tuned = false;
  std::vector<double> tune_ms;       // per problem: time of the chosen chunk in the tuning runs
  // filter service
  std::mutex mu;
  std::condition_variable cv;
  int active = 0, arrived = 0;
  unsigned long long gen = 0;
  std::vector<char> posted;
  std::vector<BatchProb> req;
  invdft_status last_launch = INVDFT_OK;
  std::string err;
  // graphs of the launch sequence, per (set of problems)
  bool graphs_ok = true;
  std::map<unsigned long long, cudaGraphExec_t> graphs;
  long long launches = 0, graph_launches = 0;
};

namespace {

// Default polls of a phase counter before a wait of the persistent kernel
// gives up (each poll backs off 256 ns, so well over a second)
constexpr int kBatchWaitLimit = 1 << 24;

// How long a posted filter waits for the other problems of the batch
constexpr long long kFilterWindowUs = 500;
constexpr size_t kMaxGraphs = 64;   // cached launch graphs (sets of problems)

int chunk_candidates(int ncol, int out[3]) {
  int n = 0;
  for (int C : {8, 16, 32})
    if (C == 8 || C / 2 < ncol) out[n++] = C;
  return n;
}

// even/odd blocks of the (symmetrised) centrosymmetric 1D matrices, as floats
void eo_tables(const Geom &g, float *tab) {
  const int P = g.p, Q = P + 1, H = P / 2;
  const int NE = (H + 1) * (H + 1), NO = H * H;
  for (int m = 0; m < 2; ++m) {
    const double *M = m == 0 ? g.A : g.B;
    float *e = tab + m * (NE + NO), *o = e + NE;
    auto sym = [&](int i, int j) { return 0.5 * (M[i * Q + j] + M[(P - i) * Q + (P - j)]); };
    for (int i = 0; i <= H; ++i)
      for (int k = 0; k <= H; ++k)
        e[i * (H + 1) + k] = (float)(k < H ? 0.5 * (sym(i, k) + sym(i, P - k)) : sym(i, H));
    for (int i = 0; i < H; ++i)
      for (int k = 0; k < H; ++k) o[i * H + k] = (float)(0.5 * (sym(i, k) - sym(i, P - k)));
  }
}

void set_chunk(const Ctx *c, int C, BatchProb *bp) {
  const int cells = c->g.ncell * c->g.ncell * c->g.ncell;
  bp->C = C;
  bp->nchunk = (c->nv + C - 1) / C;
  bp->items = cells * bp->nchunk;
}

// Queue the launch sequence for the posted problems (descriptors compacted
// in h_probs).  The caller holds the service lock.
invdft_status launch_locked(BatchState *B) {
  std::vector<int> part;
  for (int b = 0; b < (int)B->probs.size(); ++b)
    if (B->posted[b]) part.push_back(b);
  const int np = (int)part.size();
  if (np == 0) return INVDFT_OK;
  // the previous launch has consumed the staging buffer (every participant
  // synchronised on it before posting again; this wait is then immediate)
  if (cudaEventSynchronize(B->ev_done) != cudaSuccess) return INVDFT_ECUDA;
  unsigned long long mask = 0;
  int per_phase = 0;
  for (int i = 0; i < np; ++i) {
    B->h_probs[i] = B->req[part[i]];
    B->h_probs[i].item0 = per_phase;
    per_phase += B->h_probs[i].items;
    mask |= 1ull << part[i];
  }
  for (int b : part)
    if (cudaStreamWaitEvent(B->bstream, B->ev_ready[b], 0) != cudaSuccess) return INVDFT_ECUDA;
  const int m = B->degree;
  auto enqueue = [&](cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(B->d_probs, B->h_probs, np * sizeof(BatchProb),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(B->d_done, 0, (size_t)kMaxBatch * (kMaxBatchDeg + 1) * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_queue, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess)
      e = launch_batch_filter(B->d_probs, np, m, per_phase, B->d_queue, B->d_done, B->d_err,
                              B->grid, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B->h_err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    return e;
  };
  cudaError_t e = cudaSuccess;
  bool done = false;
  if (B->graphs_ok) {
    auto it = B->graphs.find(mask);
    if (it == B->graphs.end() && B->graphs.size() < kMaxGraphs) {
      // capture the sequence once for this set of problems
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      if (cudaStreamBeginCapture(B->bstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const cudaError_t ce = enqueue(B->bstream);
        const cudaError_t ee = cudaStreamEndCapture(B->bstream, &g);
        if (ce == cudaSuccess && ee == cudaSuccess &&
            cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
          it = B->graphs.emplace(mask, ge).first;
          count_graph(0);
        } else {
          B->graphs_ok = false;
          count_graph(2);
        }
        if (g) cudaGraphDestroy(g);
      } else {
        B->graphs_ok = false;
      }
      cudaGetLastError();   // a refused capture leaves no sticky error behind
    }
    if (B->graphs_ok && it != B->graphs.end()) {
      e = cudaGraphLaunch(it->second, B->bstream);
      ++B->graph_launches;
      count_graph(1);
      done = true;
    }
  }
  if (!done) e = enqueue(B->bstream);
  if (e == cudaSuccess) e = cudaEventRecord(B->ev_done, B->bstream);
  ++B->launches;
  if (e != cudaSuccess) {
    B->err = std::string("batched filter: ") + cudaGetErrorString(e);
    return INVDFT_ECUDA;
  }
  return INVDFT_OK;
}

// Release the waiting problems after a launch (lock held).
void release_locked(BatchState *B, invdft_status st) {
  B->last_launch = st;
  std::fill(B->posted.begin(), B->posted.end(), 0);
  B->arrived = 0;
  ++B->gen;
  B->cv.notify_all();
}

// Time one filter launch over every problem with the given chunks (tuning).
double time_launch(BatchState *B, const std::vector<int> &chunks) {
  const int n = (int)B->probs.size();
  int per_phase = 0;
  for (int b = 0; b < n; ++b) {
    BatchProb &bp = B->h_probs[b];
    batch_prob_static(B->probs[b], &bp);
    set_chunk(B->probs[b], chunks[b], &bp);
    bp.pk = B->probs[b]->scal + kScPk;
    bp.shift = 0.f;
    for (int k = 0; k <= kMaxBatchDeg; ++k) bp.alpha[k] = bp.beta[k] = 0.f;
    bp.item0 = per_phase;
    per_phase += bp.items;
  }
  const int m = std::min(B->degree, 6);
  cudaMemcpyAsync(B->d_probs, B->h_probs, n * sizeof(BatchProb), cudaMemcpyHostToDevice, B->bstream);
  cudaMemsetAsync(B->d_done, 0, (size_t)kMaxBatch * (kMaxBatchDeg + 1) * sizeof(unsigned), B->bstream);
  cudaMemsetAsync(B->d_queue, 0, sizeof(int), B->bstream);
  cudaMemsetAsync(B->d_err, 0, sizeof(int), B->bstream);
  cudaEventRecord(B->t0, B->bstream);
  cudaError_t e = launch_batch_filter(B->d_probs, n, m, per_phase, B->d_queue, B->d_done, B->d_err,
                                      B->grid, B->bstream);
  cudaEventRecord(B->t1, B->bstream);
  if (e != cudaSuccess || cudaEventSynchronize(B->t1) != cudaSuccess) return -1.0;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, B->t0, B->t1);
  int herr = 0;
  cudaMemcpy(&herr, B->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  return herr ? -1.0 : (double)ms;
}

// Column chunk per (order, width) class: each class in turn tries its
// candidates with the other classes fixed; the fastest whole launch wins.
void autotune(BatchState *B) {
  const int n = (int)B->probs.size();
  std::map<std::pair<int, int>, std::vector<int>> classes;
  for (int b = 0; b < n; ++b) {
    const Ctx *c = B->probs[b];
    classes[{c->g.p, (c->nv + 7) / 8}].push_back(b);
  }
  std::vector<int> chunks(n, 8);
  for (int b = 0; b < n; ++b) {
    int cand[3];
    const int nc = chunk_candidates(B->probs[b]->nv, cand);
    chunks[b] = cand[nc - 1];
  }
  B->tune_ms.assign(n, 0.0);
  for (auto &kv : classes) {
    int cand[3];
    const int nc = chunk_candidates(B->probs[kv.second[0]]->nv, cand);
    double best = -1.0;
    int bestC = chunks[kv.second[0]];
    for (int i = 0; i < nc; ++i) {
      for (int b : kv.second) chunks[b] = cand[i];
      time_launch(B, chunks);                    // warm-up
      const double ms = time_launch(B, chunks);
      if (ms >= 0.0 && (best < 0.0 || ms < best)) {
        best = ms;
        bestC = cand[i];
      }
    }
    for (int b : kv.second) {
      chunks[b] = bestC;
      B->tune_ms[b] = best;
    }
  }
  B->tileC = chunks;
  B->tuned = true;
}

}  // namespace

void batch_prob_static(const Ctx *c, BatchProb *bp) {
  std::memset(bp, 0, sizeof(*bp));
  bp->ncell = c->g.ncell;
  bp->Ni = c->g.Ni;
  bp->p = c->g.p;
  bp->ncol = c->nv;
  bp->buf[0] = (float *)c->C0;
  bp->buf[1] = (float *)c->C1;
  bp->buf[2] = (float *)c->C2;
  bp->E = c->E32;
  bp->v = c->vf;
  bp->dm1f = c->g.dm1f;
  bp->perm = c->g.p == 4 ? c->cell_perm : nullptr;
  bp->kc = (float)c->g.kc;
  eo_tables(c->g, bp->tab);
}

int batch_degree(const Ctx *c) { return c->batch ? c->batch->degree : 0; }

invdft_status batch_filter_submit(Ctx *c, int m, const double *alpha, const double *beta,
                                  double shift, cudaStream_t s) {
  BatchState *B = c->batch;
  const int b = c->batch_index;
  if (m != B->degree) {
    c->err = "batched filter: every problem of a batch needs the same Chebyshev degree";
    return INVDFT_EINVAL;
  }
  BatchProb bp;
  batch_prob_static(c, &bp);
  set_chunk(c, B->tileC[b], &bp);
  bp.pk = c->scal + kScPk;
  bp.shift = (float)shift;
  for (int k = 0; k <= m; ++k) {
    bp.alpha[k] = (float)alpha[k];
    bp.beta[k] = (float)beta[k];
  }
  if (cudaEventRecord(B->ev_ready[b], s) != cudaSuccess) return INVDFT_ECUDA;
  invdft_status st;
  {
    std::unique_lock<std::mutex> lk(B->mu);
    B->req[b] = bp;
    B->posted[b] = 1;
    ++B->arrived;
    const unsigned long long my = B->gen;
    if (B->arrived == B->active) {
      release_locked(B, launch_locked(B));
    } else if (!B->cv.wait_for(lk, std::chrono::microseconds(kFilterWindowUs),
                               [&] { return B->gen != my; })) {
      // the other problems are busy elsewhere (Rayleigh-Ritz, adjoint):
      // launch for those that have posted; the rest join a later launch
      release_locked(B, launch_locked(B));
    }
    st = B->last_launch;
    if (st != INVDFT_OK) c->err = B->err;
  }
  if (st != INVDFT_OK) return st;
  if (cudaStreamWaitEvent(s, B->ev_done, 0) != cudaSuccess) return INVDFT_ECUDA;
  // the error word of the launch (a phase wait that gave up)
  if (cudaEventSynchronize(B->ev_done) != cudaSuccess) return INVDFT_ECUDA;
  if (*B->h_err != 0) {
    c->err = "batched filter: a phase wait timed out";
    return INVDFT_ETIMEOUT;
  }
  return INVDFT_OK;
}

}  // namespace invdft

using namespace invdft;

struct invdft_batch_ctx : public BatchState {};

extern "C" {

invdft_status invdft_batch_create(const invdft_handle *handles, int n, invdft_batch *out) {
  if (!handles || !out || n < 1 || n > kMaxBatch) return INVDFT_EINVAL;
  *out = nullptr;
  for (int b = 0; b < n; ++b) {
    const Ctx *c = handles[b];
    // the persistent filter kernel covers uniform cubic meshes of order 2 or 4
    if (!c || !c->bound || c->o.prec == INVDFT_FP64 || c->o.cheb_degree != handles[0]->o.cheb_degree ||
        c->o.cheb_degree < 2 || c->o.cheb_degree > kMaxBatchDeg || c->nv > 256 || !c->g.cube ||
        !(c->g.p == 2 || c->g.p == 4))
      return INVDFT_EINVAL;
    for (int j = 0; j < b; ++j)
      if (handles[j] == handles[b]) return INVDFT_EINVAL;
  }
  invdft_batch_ctx *B = new (std::nothrow) invdft_batch_ctx();
  if (!B) return INVDFT_ENOMEM;
  B->degree = handles[0]->o.cheb_degree;
  bool ok = true;
  for (int b = 0; b < n; ++b) {
    B->probs.push_back(handles[b]);
    cudaStream_t s = nullptr;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    ok &= cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) == cudaSuccess;
    B->streams.push_back(s);
    B->ev_ready.push_back(e1);
    B->ev_end.push_back(e2);
  }
  ok &= cudaStreamCreateWithFlags(&B->bstream, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&B->ev_done, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&B->ev_start, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreate(&B->t0) == cudaSuccess && cudaEventCreate(&B->t1) == cudaSuccess;
  ok &= cudaHostAlloc((void **)&B->h_probs, kMaxBatch * sizeof(BatchProb), 0) == cudaSuccess;
  ok &= cudaHostAlloc((void **)&B->h_err, sizeof(int), 0) == cudaSuccess;
  ok &= cudaMalloc((void **)&B->d_probs, kMaxBatch * sizeof(BatchProb)) == cudaSuccess;
  ok &= cudaMalloc((void **)&B->d_done,
                   (size_t)kMaxBatch * (kMaxBatchDeg + 1) * sizeof(unsigned)) == cudaSuccess;
  ok &= cudaMalloc((void **)&B->d_queue, sizeof(int)) == cudaSuccess;
  // d_err[0]: error word of the persistent kernel; d_err[1]: its wait limit
  ok &= cudaMalloc((void **)&B->d_err, 2 * sizeof(int)) == cudaSuccess;
  if (ok) {
    const int limit[2] = {0, kBatchWaitLimit};
    ok &= cudaMemcpy(B->d_err, limit, sizeof(limit), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  int per_sm = 0, nsm = 0;
  ok &= batch_filter_occupancy(&per_sm) == cudaSuccess;
  ok &= cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) == cudaSuccess;
  B->grid = per_sm * nsm;
  if (ok) ok = cudaEventRecord(B->ev_done, B->bstream) == cudaSuccess;
  B->posted.assign(n, 0);
  B->req.resize(n);
  B->tileC.assign(n, 16);
  if (!ok || B->grid < 1) {
    invdft_batch_destroy(B);
    cudaGetLastError();
    return INVDFT_ECUDA;
  }
  *out = B;
  return INVDFT_OK;
}

invdft_status invdft_batch_destroy(invdft_batch B) {
  if (!B) return INVDFT_EINVAL;
  if (B->bstream) cudaStreamSynchronize(B->bstream);
  for (cudaStream_t s : B->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->ev_ready)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : B->ev_end)
    if (e) cudaEventDestroy(e);
  for (auto &kv : B->graphs) cudaGraphExecDestroy(kv.second);
  if (B->bstream) cudaStreamDestroy(B->bstream);
  for (cudaEvent_t e : {B->ev_done, B->ev_start, B->t0, B->t1})
    if (e) cudaEventDestroy(e);
  if (B->h_probs) cudaFreeHost(B->h_probs);
  if (B->h_err) cudaFreeHost(B->h_err);
  cudaFree(B->d_probs);
  cudaFree(B->d_done);
  cudaFree(B->d_queue);
  cudaFree(B->d_err);
  delete B;
  return INVDFT_OK;
}

invdft_status invdft_batch_step(invdft_batch B, const double *const *rho_data,
                                const double *const *w, double *const *v_xc,
                                invdft_stats *stats, invdft_status *status, void *stream) {
  if (!B || !rho_data || !w || !v_xc) return INVDFT_EINVAL;
  const int n = (int)B->probs.size();
  for (int b = 0; b < n; ++b)
    if (!rho_data[b] || !w[b] || !v_xc[b] || !B->probs[b]->have_potential) return INVDFT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!B->tuned) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return INVDFT_ECUDA;
    autotune(B);
  }
  if (cudaEventRecord(B->ev_start, s) != cudaSuccess) return INVDFT_ECUDA;
  for (int b = 0; b < n; ++b)
    if (cudaStreamWaitEvent(B->streams[b], B->ev_start, 0) != cudaSuccess) return INVDFT_ECUDA;
  std::vector<invdft_status> st(n, INVDFT_OK);
  std::vector<invdft_stats> local(n);
  {
    std::lock_guard<std::mutex> lk(B->mu);
    B->active = n;
    B->arrived = 0;
    std::fill(B->posted.begin(), B->posted.end(), 0);
  }
  std::vector<std::thread> threads;
  threads.reserve(n);
  for (int b = 0; b < n; ++b) {
    threads.emplace_back([&, b] {
      Ctx *c = B->probs[b];
      std::memset(&local[b], 0, sizeof(invdft_stats));
      c->batch = B;
      c->batch_index = b;
      st[b] = lbfgs_step(c, rho_data[b], w[b], v_xc[b], &local[b], B->streams[b]);
      c->batch = nullptr;
      c->batch_index = -1;
      cudaEventRecord(B->ev_end[b], B->streams[b]);
      std::unique_lock<std::mutex> lk(B->mu);
      --B->active;
      if (B->arrived > 0 && B->arrived == B->active) release_locked(B, launch_locked(B));
    });
  }
  for (auto &t : threads) t.join();
  invdft_status worst = INVDFT_OK;
  for (int b = 0; b < n; ++b) {
    if (cudaStreamWaitEvent(s, B->ev_end[b], 0) != cudaSuccess) return INVDFT_ECUDA;
    if (stats) stats[b] = local[b];
    if (status) status[b] = st[b];
    if (st[b] != INVDFT_OK && (worst == INVDFT_OK || worst == INVDFT_ENOCONV)) worst = st[b];
  }
  return worst;
}

invdft_status invdft_batch_set_wait_limit(invdft_batch B, int polls) {
  if (!B) return INVDFT_EINVAL;
  const int limit = polls >= 0 ? polls : kBatchWaitLimit;
  // the previous step has finished (batch steps are synchronous on the host)
  if (cudaMemcpy(B->d_err + 1, &limit, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    B->err = "batch_set_wait_limit: copy failed";
    return INVDFT_ECUDA;
  }
  return INVDFT_OK;
}

invdft_status invdft_batch_info(invdft_batch B, int *chunk_cols, double *info4) {
  if (!B) return INVDFT_EINVAL;
  if (chunk_cols)
    for (size_t b = 0; b < B->probs.size(); ++b) chunk_cols[b] = B->tileC[b];
  if (info4) {
    info4[0] = (double)B->launches;
    info4[1] = (double)B->graph_launches;
    info4[2] = (double)B->grid;
    info4[3] = B->tuned ? 1.0 : 0.0;
  }
  return INVDFT_OK;
}

}  // extern "C"
