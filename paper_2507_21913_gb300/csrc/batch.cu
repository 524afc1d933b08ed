// Batched evaluation of many independent problems (one plan each) as one
// CUDA graph.
//
// The paper evaluates one problem at a time (Algorithm 2); independent
// problems share nothing, so a batch is a set of plans whose evaluations are
// issued on parallel branches of one graph.  Small problems do not fill the
// GPU on their own; on parallel branches their kernels overlap.  The graph is
// captured once for a set of (plan, q, pot, grad) pointers and replayed while
// those pointers and the plans' bounding squares (which enter the captured
// launch arguments) stay the same; otherwise it is captured again.
#include <algorithm>
#include <vector>

#include "common.cuh"

struct hpfmm_batch {
  std::vector<hpfmm_plan *> plans;
  std::vector<int> branch;                 // branch of each problem
  std::vector<cudaStream_t> streams;       // one per branch
  std::vector<cudaEvent_t> join;           // one per branch
  cudaEvent_t cfork = nullptr;             // fork inside the graph
  cudaEvent_t pre = nullptr, post = nullptr;  // caller stream <-> capture stream
  cudaStream_t origin = nullptr;           // capture stream
  cudaGraphExec_t exec = nullptr;
  std::vector<const double *> q;           // pointers of the captured graph
  std::vector<double *> pot, grad;
  std::vector<double> geom;                // x0, side of each plan at capture
  int64_t captures = 0;
};

namespace {

void batch_release(hpfmm_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->cfork, b->pre, b->post})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

hpfmm_status capture(hpfmm_batch *b, const double *const *q, double *const *pot,
                     double *const *grad) {
  const int np = (int)b->plans.size();
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaStream_t o = b->origin;
  HP_CUDA(cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal));
  hpfmm_status s = HPFMM_OK;
  cudaError_t e = cudaEventRecord(b->cfork, o);
  for (size_t k = 0; e == cudaSuccess && k < b->streams.size(); ++k)
    e = cudaStreamWaitEvent(b->streams[k], b->cfork, 0);
  if (e != cudaSuccess) {
    set_last_error("hpfmm_eval_batched: fork: %s", cudaGetErrorString(e));
    s = HPFMM_ECUDA;
  }
  for (int i = 0; s == HPFMM_OK && i < np; ++i)
    s = fmm_eval(b->plans[i], q[i], pot[i], grad ? grad[i] : nullptr, b->streams[b->branch[i]]);
  for (size_t k = 0; k < b->streams.size(); ++k) {
    cudaError_t e1 = cudaEventRecord(b->join[k], b->streams[k]);
    cudaError_t e2 = cudaStreamWaitEvent(o, b->join[k], 0);
    if (s == HPFMM_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) {
      set_last_error("hpfmm_eval_batched: join: %s",
                     cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
      s = HPFMM_ECUDA;
    }
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(o, &g);
  if (s == HPFMM_OK && e != cudaSuccess) {
    set_last_error("hpfmm_eval_batched: capture: %s", cudaGetErrorString(e));
    s = HPFMM_ECUDA;
  }
  if (s == HPFMM_OK) {
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      set_last_error("hpfmm_eval_batched: instantiate: %s", cudaGetErrorString(e));
      b->exec = nullptr;
      s = HPFMM_ECUDA;
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (s != HPFMM_OK) return s;
  b->q.assign(q, q + np);
  b->pot.assign(pot, pot + np);
  b->grad.assign(np, nullptr);
  if (grad) b->grad.assign(grad, grad + np);
  b->geom.resize(2 * np);
  for (int i = 0; i < np; ++i) {
    b->geom[2 * i] = b->plans[i]->x0;
    b->geom[2 * i + 1] = b->plans[i]->side;
  }
  ++b->captures;
  return HPFMM_OK;
}

}  // namespace

extern "C" hpfmm_status hpfmm_batch_create(hpfmm_plan *const *plans, int nprob, int nbranch,
                                           hpfmm_batch **out) {
  if (!plans || nprob < 1 || !out || nbranch < 0 || nbranch > 64) {
    set_last_error("hpfmm_batch_create: need plans, nprob >= 1, 0 <= nbranch <= 64, out");
    return HPFMM_EINVAL;
  }
  *out = nullptr;
  std::vector<hpfmm_plan *> v(plans, plans + nprob);
  for (hpfmm_plan *p : v)
    if (!p) {
      set_last_error("hpfmm_batch_create: null plan");
      return HPFMM_EINVAL;
    }
  std::vector<hpfmm_plan *> sorted = v;
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    set_last_error("hpfmm_batch_create: a plan appears twice (its workspace would race)");
    return HPFMM_EINVAL;
  }
  if (nbranch == 0) nbranch = std::min(nprob, 8);
  nbranch = std::min(nbranch, nprob);
  hpfmm_batch *b = new hpfmm_batch();
  b->plans = v;
  // longest-processing-time assignment of problems to branches (cost ~ n)
  std::vector<int> idx(nprob);
  for (int i = 0; i < nprob; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return v[a]->n > v[c]->n; });
  std::vector<int64_t> load(nbranch, 0);
  b->branch.assign(nprob, 0);
  for (int i : idx) {
    int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->branch[i] = k;
    load[k] += v[i]->n;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (cudaEvent_t *ev : {&b->cfork, &b->pre, &b->post})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  b->streams.assign(nbranch, nullptr);
  b->join.assign(nbranch, nullptr);
  for (int k = 0; e == cudaSuccess && k < nbranch; ++k) {
    e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    set_last_error("hpfmm_batch_create: %s", cudaGetErrorString(e));
    batch_release(b);
    return HPFMM_ECUDA;
  }
  *out = b;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_eval_batched(hpfmm_batch *b, const double *const *q,
                                           double *const *pot, double *const *grad,
                                           void *stream) {
  if (!b || !q || !pot) {
    set_last_error("hpfmm_eval_batched: need batch, q and pot");
    return HPFMM_EINVAL;
  }
  const int np = (int)b->plans.size();
  for (int i = 0; i < np; ++i) {
    const void *ptrs[] = {q[i], pot[i], grad ? grad[i] : nullptr};
    if (!q[i] || !pot[i]) {
      set_last_error("hpfmm_eval_batched: null q or pot for problem %d", i);
      return HPFMM_EINVAL;
    }
    for (const void *p : ptrs)
      if (p && !is_device_pointer(p)) {
        set_last_error("hpfmm_eval_batched: problem %d: arrays must be device memory", i);
        return HPFMM_EINVAL;
      }
    if (b->plans[i]->timing) {
      set_last_error("hpfmm_eval_batched: problem %d has pass timing on", i);
      return HPFMM_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the graph replays kernels only: the reaction tables of the plans' last
  // rebuilds are joined here, outside the capture, and the root squares the
  // capture used are compared with the current ones
  for (int i = 0; i < np; ++i) {
    HP_TRY(plan_join_tables(b->plans[i], st));
    HP_TRY(plan_host_geometry(b->plans[i]));
  }
  bool same = b->exec != nullptr;
  for (int i = 0; same && i < np; ++i)
    same = b->q[i] == q[i] && b->pot[i] == pot[i] && b->grad[i] == (grad ? grad[i] : nullptr) &&
           b->geom[2 * i] == b->plans[i]->x0 && b->geom[2 * i + 1] == b->plans[i]->side;
  // the graph reads the plans' trees: order the capture stream after the caller's work
  HP_CUDA(cudaEventRecord(b->pre, st));
  HP_CUDA(cudaStreamWaitEvent(b->origin, b->pre, 0));
  if (!same) HP_TRY(capture(b, q, pot, grad));
  HP_CUDA(cudaGraphLaunch(b->exec, b->origin));
  HP_CUDA(cudaEventRecord(b->post, b->origin));
  HP_CUDA(cudaStreamWaitEvent(st, b->post, 0));
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_batch_captures(const hpfmm_batch *b, int64_t *captures) {
  if (!b || !captures) {
    set_last_error("hpfmm_batch_captures: null argument");
    return HPFMM_EINVAL;
  }
  *captures = b->captures;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_batch_destroy(hpfmm_batch *b) {
  if (!b) return HPFMM_OK;
  if (b->origin) cudaStreamSynchronize(b->origin);
  batch_release(b);
  return HPFMM_OK;
}
