// Batched mock realisations: many independent COLA runs (§2.2, §2.3; the paper runs thousands of
// them for covariance estimates, §3) enqueued as one launch sequence over several streams and
// captured once into a CUDA graph, so a replay costs one graph launch for all realisations.
// Host code only: every kernel is the single-realisation path's.
#include "cola_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <numeric>

namespace {

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return COLA_OK;
  std::fprintf(stderr, "cola batch: %s: %s\n", what, cudaGetErrorString(e));
  return COLA_ERR_CUDA;
}

#define BATCH_TRY(x)                \
  do {                              \
    const int st_ = (x);            \
    if (st_ != COLA_OK) return st_; \
  } while (0)

// Relative cost of one realisation: particle work plus N^3 log N mesh work per step.
double realisation_cost(const cola_params& p) {
  const double n = (double)p.np * p.np * p.np;
  const double m = (double)p.nmesh * p.nmesh * p.nmesh;
  return p.nstep * (84.0 * n + 104.0 * m * (1.0 + std::log2((double)p.nmesh) / 16.0));
}

}  // namespace

struct cola_batch {
  int count = 0;
  int nbins = 0;
  cudaStream_t main = nullptr;          // the caller's stream (may be the legacy default stream)
  cudaStream_t origin = nullptr;        // owned: capture origin and graph launch stream
  cudaEvent_t start = nullptr, done = nullptr;
  std::vector<cudaStream_t> streams;    // owned
  std::vector<int> lane;                // member -> stream index
  std::vector<cola_ctx*> ctx;           // owned
  std::vector<cola_batch_io> io;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool warmed = false;
};

namespace {

// Enqueue every member on its lane, the lanes forked from and joined back into `on`.
int enqueue(cola_batch* b, cudaStream_t on) {
  BATCH_TRY(cuda_status(cudaEventRecord(b->fork, on), "fork"));
  for (cudaStream_t s : b->streams) BATCH_TRY(cuda_status(cudaStreamWaitEvent(s, b->fork, 0), "fork wait"));
  for (int i = 0; i < b->count; ++i) {
    const cola_batch_io& o = b->io[i];
    BATCH_TRY(cola_run(b->ctx[i], o.white_noise, o.s, o.v, o.psi1, o.psi2, o.pk, b->nbins));
  }
  for (size_t l = 0; l < b->streams.size(); ++l) {
    BATCH_TRY(cuda_status(cudaEventRecord(b->join[l], b->streams[l]), "join"));
    BATCH_TRY(cuda_status(cudaStreamWaitEvent(on, b->join[l], 0), "join wait"));
  }
  return COLA_OK;
}

void drop_graph(cola_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

}  // namespace

extern "C" void cola_batch_destroy(cola_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  if (b->origin) cudaStreamSynchronize(b->origin);
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  drop_graph(b);
  for (cola_ctx* c : b->ctx) cola_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->start) cudaEventDestroy(b->start);
  if (b->done) cudaEventDestroy(b->done);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

extern "C" int cola_batch_create(const cola_params* params, const cola_batch_io* io, int count, int nbins,
                                 int nstreams, void* stream, cola_batch** out) {
  if (!out || !params || !io || count < 1 || nbins < 1 || nbins > 128 || nstreams < 1 || nstreams > 64)
    return COLA_ERR_INVALID;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    const cola_batch_io& o = io[i];
    if ((uintptr_t)o.white_noise % 16) return COLA_ERR_INVALID;   // NULL: drawn from params[i].seed
    for (const void* p : {(const void*)o.s, (const void*)o.v, (const void*)o.psi1, (const void*)o.psi2,
                          (const void*)o.pk})
      if (!p || (uintptr_t)p % 16) return COLA_ERR_INVALID;
  }
  cola_batch* b = new (std::nothrow) cola_batch;
  if (!b) return COLA_ERR_OOM;
  b->count = count;
  b->nbins = nbins;
  b->main = static_cast<cudaStream_t>(stream);
  b->io.assign(io, io + count);
  const int lanes = std::min(nstreams, count);
  auto fail = [&](int st) {
    cola_batch_destroy(b);
    return st;
  };
  int st = COLA_OK;
  b->streams.resize(lanes, nullptr);
  b->join.resize(lanes, nullptr);
  for (int l = 0; l < lanes && st == COLA_OK; ++l) {
    st = cuda_status(cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking), "stream");
    if (st == COLA_OK) st = cuda_status(cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming), "event");
  }
  if (st == COLA_OK) st = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  if (st == COLA_OK) st = cuda_status(cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming), "event");
  if (st == COLA_OK) st = cuda_status(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "event");
  if (st == COLA_OK) st = cuda_status(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking), "stream");
  if (st != COLA_OK) return fail(st);
  // longest-processing-time-first: the costliest realisation goes to the least loaded lane
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return realisation_cost(params[a]) > realisation_cost(params[c]); });
  std::vector<double> load(lanes, 0.0);
  b->lane.assign(count, 0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane[i] = l;
    load[l] += realisation_cost(params[i]);
  }
  b->ctx.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    if ((st = cola_create(&params[i], b->streams[b->lane[i]], &b->ctx[i])) != COLA_OK) return fail(st);
  }
  *out = b;
  return COLA_OK;
}

extern "C" int cola_batch_run(cola_batch* b, int use_graph) {
  if (!b) return COLA_ERR_INVALID;
  if (!use_graph || !b->warmed) {
    // eager: also the warm-up before a capture (first-use kernel attributes, P(k) bin edges)
    BATCH_TRY(enqueue(b, b->main));
    if (use_graph) {
      BATCH_TRY(cuda_status(cudaStreamSynchronize(b->main), "warm-up"));
      b->warmed = true;
    }
    if (!use_graph) return COLA_OK;
  }
  if (!b->exec) {
    // capture on the batch's own stream (the caller's may be the uncapturable legacy stream)
    BATCH_TRY(cuda_status(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed), "begin capture"));
    const int st = enqueue(b, b->origin);
    cudaGraph_t g = nullptr;
    const int st2 = cuda_status(cudaStreamEndCapture(b->origin, &g), "end capture");
    if (st != COLA_OK || st2 != COLA_OK) {
      if (g) cudaGraphDestroy(g);
      return st != COLA_OK ? st : st2;
    }
    b->graph = g;
    if (cuda_status(cudaGraphInstantiate(&b->exec, g, 0), "instantiate") != COLA_OK) {
      drop_graph(b);
      return COLA_ERR_CUDA;
    }
  }
  // order the replay after the caller's stream and the caller's stream after the replay
  BATCH_TRY(cuda_status(cudaEventRecord(b->start, b->main), "start"));
  BATCH_TRY(cuda_status(cudaStreamWaitEvent(b->origin, b->start, 0), "start wait"));
  BATCH_TRY(cuda_status(cudaGraphLaunch(b->exec, b->origin), "graph launch"));
  BATCH_TRY(cuda_status(cudaEventRecord(b->done, b->origin), "done"));
  return cuda_status(cudaStreamWaitEvent(b->main, b->done, 0), "done wait");
}

extern "C" int cola_batch_sync(cola_batch* b) {
  if (!b) return COLA_ERR_INVALID;
  BATCH_TRY(cuda_status(cudaStreamSynchronize(b->main), "batch sync"));
  int first = COLA_OK;
  for (cola_ctx* c : b->ctx) {
    const int st = cola_sync(c);
    if (first == COLA_OK) first = st;
  }
  return first;
}

extern "C" int cola_batch_tune(cola_batch* b, int reps) {
  if (!b || reps < 1) return COLA_ERR_INVALID;
  BATCH_TRY(cola_batch_sync(b));
  // one autotune per distinct (np, nmesh), on the first such member's current positions
  std::vector<std::pair<long long, int>> tuned;   // key -> schedule
  for (int i = 0; i < b->count; ++i) {
    cola_ctx* c = b->ctx[i];
    const long long key = ((long long)c->p.np << 32) | (unsigned)c->p.nmesh;
    int sc = -1;
    for (auto& t : tuned)
      if (t.first == key) sc = t.second;
    if (sc < 0) {
      const int r = cola_autotune(c, b->io[i].s, reps, &sc, nullptr, nullptr, 0);
      if (r < 0) return -r;
      tuned.push_back({key, sc});
    } else {
      BATCH_TRY(cola_set_schedule(c, sc));
    }
  }
  drop_graph(b);   // the captured launches used the old schedules
  return cuda_status(cudaDeviceSynchronize(), "tune");
}

extern "C" int cola_batch_info(cola_batch* b, int i, int* lane, int* schedule, size_t* graph_nodes) {
  if (!b || i < 0 || i >= b->count) return COLA_ERR_INVALID;
  if (lane) *lane = b->lane[i];
  if (schedule) BATCH_TRY(cola_get_schedule(b->ctx[i], schedule));
  if (graph_nodes) {
    *graph_nodes = 0;
    if (b->graph) BATCH_TRY(cuda_status(cudaGraphGetNodes(b->graph, nullptr, graph_nodes), "graph nodes"));
  }
  return COLA_OK;
}
