// api.cu -- the C ABI of include/hpfmm.h: argument checks, host/device
// staging, plan allocation, and the order of the passes.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "tc.cuh"

hpfmm_status fmm_set_smem_limits(int p);

static thread_local char g_err[512] = "";

void set_last_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

bool is_device_pointer(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" const char *hpfmm_status_string(hpfmm_status s) {
  switch (s) {
    case HPFMM_OK: return "ok";
    case HPFMM_EINVAL: return "invalid argument";
    case HPFMM_ENOMEM: return "device out of memory";
    case HPFMM_ECUDA: return "CUDA runtime error";
    case HPFMM_ETIMEOUT: return "bounded device wait gave up";
    case HPFMM_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

extern "C" const char *hpfmm_last_error(void) { return g_err; }

extern "C" const char *hpfmm_version(void) { return "hpfmm 0.1 sm_103a"; }

extern "C" void hpfmm_default_options(hpfmm_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof *opt);
  opt->prec = HPFMM_FP64;
  opt->tau_fp64 = 0.05;
}

#include <vector>

struct TimingState {
  std::vector<cudaEvent_t> pool;   // events, reused
  size_t used = 0;
  struct Rec { size_t a, b; int pass; };
  std::vector<Rec> recs;
  std::vector<int> open_pass;      // start event index per pass (one open at a time)
};

static cudaEvent_t next_event(TimingState *ts) {
  if (ts->used == ts->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ts->pool.push_back(e);
  }
  return ts->pool[ts->used++];
}

void pass_begin(hpfmm_plan *pl, cudaStream_t st, int pass) {
  if (!pl->timing || !pl->tstate) return;
  TimingState *ts = (TimingState *)pl->tstate;
  if (ts->open_pass.empty()) ts->open_pass.assign(HPFMM_NPASS, -1);
  cudaEvent_t e = next_event(ts);
  if (!e) return;
  cudaEventRecord(e, st);
  ts->open_pass[pass] = (int)(ts->used - 1);
}

void pass_end(hpfmm_plan *pl, cudaStream_t st, int pass, int nlaunch) {
  pl->launches[pass] += nlaunch;
  if (!pl->timing || !pl->tstate) return;
  TimingState *ts = (TimingState *)pl->tstate;
  if (ts->open_pass.empty() || ts->open_pass[pass] < 0) return;
  cudaEvent_t e = next_event(ts);
  if (!e) return;
  cudaEventRecord(e, st);
  ts->recs.push_back({(size_t)ts->open_pass[pass], ts->used - 1, pass});
  ts->open_pass[pass] = -1;
}

extern "C" hpfmm_status hpfmm_set_timing(hpfmm_plan *pl, int enable) {
  if (!pl) {
    set_last_error("hpfmm_set_timing: null plan");
    return HPFMM_EINVAL;
  }
  if (!pl->tstate) pl->tstate = new TimingState();
  pl->timing = enable != 0;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_read_timing(hpfmm_plan *pl, double ms[10], int64_t launches[10]) {
  if (!pl) {
    set_last_error("hpfmm_read_timing: null plan");
    return HPFMM_EINVAL;
  }
  if (ms)
    for (int i = 0; i < HPFMM_NPASS; ++i) ms[i] = 0.0;
  TimingState *ts = (TimingState *)pl->tstate;
  if (ts && !ts->recs.empty()) {
    HP_CUDA(cudaEventSynchronize(ts->pool[ts->recs.back().b]));
    for (auto &r : ts->recs) {
      float t = 0.f;
      HP_CUDA(cudaEventElapsedTime(&t, ts->pool[r.a], ts->pool[r.b]));
      if (ms) ms[r.pass] += t;
    }
    ts->recs.clear();
    ts->used = 0;
  }
  if (launches)
    for (int i = 0; i < HPFMM_NPASS; ++i) launches[i] = pl->launches[i];
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_read_timeline(hpfmm_plan *pl, int cap, int *pass, double *begin_ms,
                                            double *end_ms, int *count) {
  if (!pl || !count || cap < 0 || (cap > 0 && (!pass || !begin_ms || !end_ms))) {
    set_last_error("hpfmm_read_timeline: null plan, count or output arrays");
    return HPFMM_EINVAL;
  }
  *count = 0;
  TimingState *ts = (TimingState *)pl->tstate;
  if (!ts || ts->recs.empty()) return HPFMM_OK;
  // the events sit on several streams: wait for each before reading offsets
  for (auto &r : ts->recs) {
    HP_CUDA(cudaEventSynchronize(ts->pool[r.a]));
    HP_CUDA(cudaEventSynchronize(ts->pool[r.b]));
  }
  // the origin: the earliest begin event
  size_t o = ts->recs.front().a;
  for (auto &r : ts->recs) {
    float t = 0.f;
    HP_CUDA(cudaEventElapsedTime(&t, ts->pool[o], ts->pool[r.a]));
    if (t < 0.f) o = r.a;
  }
  int k = 0;
  for (auto &r : ts->recs) {
    if (k >= cap) break;
    float ta = 0.f, tb = 0.f;
    HP_CUDA(cudaEventElapsedTime(&ta, ts->pool[o], ts->pool[r.a]));
    HP_CUDA(cudaEventElapsedTime(&tb, ts->pool[o], ts->pool[r.b]));
    pass[k] = r.pass;
    begin_ms[k] = ta;
    end_ms[k] = tb;
    ++k;
  }
  *count = k;
  ts->recs.clear();
  ts->used = 0;
  return HPFMM_OK;
}

static void free_plan(hpfmm_plan *pl) {
  if (!pl) return;
  if (pl->side_stream) {
    cudaStreamSynchronize(pl->side_stream);
    cudaStreamDestroy(pl->side_stream);
  }
  if (pl->table_stream) {
    cudaStreamSynchronize(pl->table_stream);
    cudaStreamDestroy(pl->table_stream);
  }
  if (pl->m2l_stream) {
    cudaStreamSynchronize(pl->m2l_stream);
    cudaStreamDestroy(pl->m2l_stream);
  }
  if (pl->ev_s2m) cudaEventDestroy(pl->ev_s2m);
  if (pl->ev_up) cudaEventDestroy(pl->ev_up);
  if (pl->ev_m2lh) cudaEventDestroy(pl->ev_m2lh);
  if (pl->ev_tree) cudaEventDestroy(pl->ev_tree);
  if (pl->ev_geo) cudaEventDestroy(pl->ev_geo);
  if (pl->copy_stream) {
    cudaStreamSynchronize(pl->copy_stream);
    cudaStreamDestroy(pl->copy_stream);
  }
  for (cudaEvent_t ev : {pl->ev_qcopy, pl->ev_qfree, pl->ev_xcopy, pl->ev_xyfree, pl->ev_done})
    if (ev) cudaEventDestroy(ev);
  if (pl->ev_tables) cudaEventDestroy(pl->ev_tables);
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_join) cudaEventDestroy(pl->ev_join);
  if (pl->ev_gather) cudaEventDestroy(pl->ev_gather);
  if (pl->hgeo) cudaFreeHost(pl->hgeo);
  if (pl->tstate) {
    TimingState *ts = (TimingState *)pl->tstate;
    for (cudaEvent_t e : ts->pool) cudaEventDestroy(e);
    delete ts;
    pl->tstate = nullptr;
  }
  void *bufs[] = {pl->xs, pl->ys, pl->perm, pl->keys, pl->leaf_start, pl->loc32, pl->yabs, pl->t_m2m,
                  pl->t_l2l, pl->t_m2l, pl->t_refl, pl->t_rlog, pl->t_rlog0, pl->qs, pl->M,
                  pl->A, pl->B, pl->out_pot, pl->out_grad, pl->in_q, pl->status,
                  pl->t_binom, pl->geo, pl->t_m2l_pad, pl->adj, pl->mq, pl->mqsm,
                  pl->mM, pl->mA, pl->mB, pl->tflag, pl->tlist, pl->t_m2l_tc,
                  pl->ab_key, pl->ab_lo, pl->ab_hi, pl->ab_parent, pl->ab_lvl, pl->ab_child,
                  pl->ab_cut, pl->ab_off, pl->ab_idx, pl->ab_lev, pl->ab_btot, pl->ab_lrank,
                  pl->ab_leaf, pl->near, pl->loclo, pl->dgeom, pl->tree_ctr, pl->ctr, pl->mir_A, pl->mir_B,
                  pl->tree_tmp, pl->in_xy};
  for (void *b : bufs)
    if (b) cudaFree(b);
  delete pl;
}

hpfmm_status plan_dalloc(hpfmm_plan *pl, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HPFMM_ENOMEM : HPFMM_ECUDA;
  }
  pl->workspace_bytes += (int64_t)bytes;
  return HPFMM_OK;
}

static int choose_levels(int64_t n, int leaf) {
  double r = (double)n / (double)leaf;
  int H = r > 1.0 ? (int)floor(log(r) / log(4.0) + 0.5) : 1;
  if (H < 1) H = 1;
  if (H > 12) H = 12;
  return H;
}

// tree + tables for the points (x, y) of a plan whose buffers exist.  With
// wait, the host waits once, after the tree build, for the root square
// (validity, host copies of the geometry); otherwise nothing waits and the
// device reports invalid input through the status word.
// last-block counters of the fused upward pass: one per right-hand side of a
// multi-RHS pass set (at most 64)
constexpr int kCtrSlots = 64;

static hpfmm_status rebuild(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st,
                            bool wait) {
  const int64_t n = pl->n;
  const double *dx = x, *dy = y;
  cudaError_t e = cudaSuccess;
  // host coordinates: staged in a buffer of the plan, x on the copy stream
  // and y on the caller's, concurrently
  const bool staged = !is_device_pointer(x) || !is_device_pointer(y);
  cudaStream_t cs = pl->copy_stream ? pl->copy_stream : st;
  if (staged) {
    if (!pl->in_xy) HP_TRY(plan_dalloc(pl, (void **)&pl->in_xy, 2 * sizeof(double) * n));
    if (cs != st) e = cudaStreamWaitEvent(cs, pl->ev_xyfree, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pl->in_xy, x, sizeof(double) * n, cudaMemcpyDefault, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pl->in_xy + n, y, sizeof(double) * n, cudaMemcpyDefault, st);
    if (e == cudaSuccess && cs != st) e = cudaEventRecord(pl->ev_xcopy, cs);
    if (e == cudaSuccess && cs != st) e = cudaStreamWaitEvent(st, pl->ev_xcopy, 0);
    if (e != cudaSuccess) {
      set_last_error("staging the coordinates: %s", cudaGetErrorString(e));
      return HPFMM_ECUDA;
    }
    dx = pl->in_xy;
    dy = pl->in_xy + n;
  }
  hpfmm_status s = tree_build(pl, dx, dy, st);
  if (s == HPFMM_OK) {
    // the geometry to the host and the reaction tables (they depend on the
    // root square only) on the table stream, concurrent with what follows
    // (ev_tree: recorded by tree_build after its last kernel)
    e = cudaStreamWaitEvent(pl->table_stream, pl->ev_tree, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pl->hgeo, pl->geo, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                          pl->table_stream);
    if (e == cudaSuccess) e = cudaEventRecord(pl->ev_geo, pl->table_stream);
    if (e == cudaSuccess) s = tables_build(pl, pl->table_stream);
    if (e == cudaSuccess) e = cudaEventRecord(pl->ev_tables, pl->table_stream);
    if (e != cudaSuccess) {
      set_last_error("rebuild: table stream: %s", cudaGetErrorString(e));
      s = HPFMM_ECUDA;
    }
    pl->tables_pending = true;
  }
  const bool sync = wait || pl->adaptive;
  double hgeo[5] = {0, 0, 1, 0, 0};
  if (s == HPFMM_OK && sync) {
    e = cudaEventSynchronize(pl->ev_geo);
    if (e != cudaSuccess) {
      set_last_error("rebuild: %s", cudaGetErrorString(e));
      s = HPFMM_ECUDA;
    } else {
      memcpy(hgeo, pl->hgeo, sizeof hgeo);
    }
  }
  pl->geo_pending = s == HPFMM_OK && !sync;
  hpfmm_status s2 = tree_finish(pl, sync ? hgeo : nullptr, st);
  if (s == HPFMM_OK) s = s2;
  // the adaptive tree over the sorted points (it reads the coordinates for
  // its leaf frames, so before the staging buffer goes)
  if (s == HPFMM_OK && pl->adaptive) s = adaptive_build(pl, dx, dy, st);
  // the next staging copy waits for this rebuild's reads of the coordinates
  if (staged && cs != st) cudaEventRecord(pl->ev_xyfree, st);
  if (s != HPFMM_OK || !sync) return s;
  double kabs = sqrt(pl->kre * pl->kre + pl->kim * pl->kim);
  if (kabs * sqrt(5.0) * pl->side > 60.0) {
    set_last_error("|kappa| * sqrt(5) * side = %g exceeds 60, the range of the device I_n "
                   "evaluation", kabs * sqrt(5.0) * pl->side);
    return HPFMM_EUNSUPPORTED;
  }
  return HPFMM_OK;
}

hpfmm_status plan_host_geometry(hpfmm_plan *pl) {
  if (!pl->geo_pending) return HPFMM_OK;
  HP_CUDA(cudaEventSynchronize(pl->ev_geo));
  pl->geo_pending = false;
  if (pl->hgeo[2] == 0.0) {
    pl->x0 = pl->hgeo[0];
    pl->side = pl->hgeo[1];
    pl->qscale = pl->hgeo[3];
  }
  return HPFMM_OK;
}

hpfmm_status plan_join_tables(hpfmm_plan *pl, cudaStream_t st) {
  if (!pl->tables_pending) return HPFMM_OK;
  HP_CUDA(cudaStreamWaitEvent(st, pl->ev_tables, 0));
  pl->tables_pending = false;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_update_points(hpfmm_plan *pl, const double *x, const double *y,
                                            void *stream) {
  if (!pl || !x || !y) {
    set_last_error("hpfmm_update_points: null argument");
    return HPFMM_EINVAL;
  }
  return rebuild(pl, x, y, (cudaStream_t)stream, !pl->async_update);
}

extern "C" hpfmm_status hpfmm_create(const double *x, const double *y, int64_t n,
                                     double kappa_re, double kappa_im, int p, int leaf_size,
                                     const hpfmm_options *opt, void *stream, hpfmm_plan **out) {
  if (!out) {
    set_last_error("hpfmm_create: out is NULL");
    return HPFMM_EINVAL;
  }
  *out = nullptr;
  if (!x || !y || n < 1 || n > INT32_MAX) {
    set_last_error("hpfmm_create: need x, y and 1 <= n < 2^31");
    return HPFMM_EINVAL;
  }
  if (!(kappa_re > 0) || !(kappa_im >= 0) || !isfinite(kappa_re) || !isfinite(kappa_im)) {
    set_last_error("hpfmm_create: kappa must satisfy Re > 0, Im >= 0 (Z > 0, eps >= 0)");
    return HPFMM_EINVAL;
  }
  if (p < 1 || p > HPFMM_MAX_P || leaf_size < 1) {
    set_last_error("hpfmm_create: need 1 <= p <= %d and leaf_size >= 1", HPFMM_MAX_P);
    return HPFMM_EINVAL;
  }
  hpfmm_options o;
  hpfmm_default_options(&o);
  if (opt) o = *opt;
  for (int r : o.reserved)
    if (r != 0) {
      set_last_error("hpfmm_create: reserved option fields must be zero");
      return HPFMM_EINVAL;
    }
  if (o.prec != HPFMM_FP64 && o.prec != HPFMM_FP32 && o.prec != HPFMM_MIXED) {
    set_last_error("hpfmm_create: unknown precision %d", (int)o.prec);
    return HPFMM_EINVAL;
  }
  if (o.adaptive != 0 && o.adaptive != 1) {
    set_last_error("hpfmm_create: adaptive must be 0 or 1");
    return HPFMM_EINVAL;
  }
  if (o.adaptive && o.prec == HPFMM_FP64) {
    set_last_error("hpfmm_create: the adaptive tree is implemented in single and mixed precision");
    return HPFMM_EUNSUPPORTED;
  }
  if (o.adaptive && p > 31) {  // the adaptive M2L kernels map output orders to lanes
    set_last_error("hpfmm_create: the adaptive tree supports p <= 31");
    return HPFMM_EUNSUPPORTED;
  }
  if (o.adaptive && o.levels > kAdaptiveMaxLevel) {
    set_last_error("hpfmm_create: an adaptive tree has at most %d levels", kAdaptiveMaxLevel);
    return HPFMM_EINVAL;
  }
  if (o.async_update != 0 && o.async_update != 1) {
    set_last_error("hpfmm_create: async_update must be 0 or 1");
    return HPFMM_EINVAL;
  }
  if (o.levels < 0 || o.levels > 15 || !(o.tau_fp64 >= 0) || o.subtree_levels < 0 ||
      o.subtree_levels > 4 || o.m2l_mode < 0 || o.m2l_mode > 1 || !(o.root_side >= 0) ||
      !isfinite(o.root_x0) || !isfinite(o.root_side)) {
    set_last_error("hpfmm_create: levels must be in 0..15, subtree_levels in 0..4, m2l_mode in "
                   "0..1, tau_fp64 >= 0");
    return HPFMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("hpfmm_create: no usable CUDA device");
    return HPFMM_ECUDA;
  }
  hpfmm_plan *pl = new hpfmm_plan();
  pl->sms = sms;
  pl->n = n;
  pl->p = p;
  pl->prec = o.prec;
  pl->tau_fp64 = o.tau_fp64;
  pl->subtree = o.subtree_levels;
  pl->m2l_mode = o.m2l_mode;
  pl->root_x0 = o.root_x0;
  pl->root_side = o.root_side;
  pl->kre = kappa_re;
  pl->kim = kappa_im;
  pl->adaptive = o.adaptive;
  pl->async_update = o.adaptive ? 0 : o.async_update;
  pl->leaf_cap = leaf_size;
  if (pl->adaptive) {
    // depth cap: the uniform depth for this leaf size plus five levels of
    // refinement, at most kAdaptiveMaxLevel.  The sort buckets lie two levels
    // below the uniform depth, so that clustered points still fall into
    // buckets small enough for the warp and shared-memory sorts.
    const int hu = choose_levels(n, leaf_size);
    pl->H = o.levels > 0 ? o.levels : (hu + 5 < kAdaptiveMaxLevel ? hu + 5 : kAdaptiveMaxLevel);
    pl->Hsort = hu + 2 < pl->H ? hu + 2 : pl->H;
    pl->nbox = 0;  // expansion arrays follow the tree (adaptive_build)
  } else {
    pl->H = o.levels > 0 ? o.levels : choose_levels(n, leaf_size);
    pl->Hsort = pl->H;
    pl->nbox = level_offset(pl->H + 1);
  }
  pl->nleaf = 1 << (2 * pl->Hsort);
  const int P1 = p + 1;
  const size_t m2 = (size_t)P1 * P1;
  const bool f32 = pl->prec != HPFMM_FP64;
  const size_t csz = f32 ? sizeof(cf) : sizeof(cd);
  const size_t tf = f32 ? (sizeof(cd) + sizeof(cf)) : sizeof(cd);  // bytes per table entry
  hpfmm_status s = HPFMM_OK;
#define ALLOC(ptr, bytes)                                       \
  do {                                                          \
    s = plan_dalloc(pl, (void **)&(ptr), (bytes));                   \
    if (s != HPFMM_OK) { free_plan(pl); return s; }             \
  } while (0)
  if (!f32) {  // sorted coordinates: used by the double-precision passes only
    ALLOC(pl->xs, sizeof(double) * n);
    ALLOC(pl->ys, sizeof(double) * n);
  }
  ALLOC(pl->perm, sizeof(int64_t) * n);
  ALLOC(pl->keys, sizeof(uint64_t) * n);
  ALLOC(pl->leaf_start, sizeof(int) * (pl->nleaf + 1));
  if (f32) ALLOC(pl->loc32, sizeof(float2) * n);
  if (f32) ALLOC(pl->yabs, sizeof(float) * n);
  if (f32) ALLOC(pl->loclo, sizeof(float2) * n);
  if (f32 && !pl->adaptive) ALLOC(pl->near, sizeof(float4) * n);
  if (f32 && !pl->adaptive) {  // mirror M2L results: rows 0 and 1 of levels 1..H
    ALLOC(pl->mir_A, sizeof(cf) * 4 * (((size_t)1 << pl->H) - 1) * P1);
    ALLOC(pl->mir_B, sizeof(cf) * 4 * (((size_t)1 << pl->H) - 1) * P1);
  }
  ALLOC(pl->t_m2m, tf * 4 * m2);
  ALLOC(pl->t_l2l, tf * 4 * m2);
  ALLOC(pl->t_m2l, tf * 49 * m2);
  if (!pl->adaptive || f32) ALLOC(pl->t_m2l_pad, csz * 40 * 2 * 2 * (size_t)P1);
  if (f32 && pl->m2l_mode == 1)
    ALLOC(pl->t_m2l_tc, sizeof(float) * 40 * 2 * (size_t)tc_np(P1) * tc_kp(P1));
  ALLOC(pl->t_rlog, tf * 21 * m2);
  ALLOC(pl->t_refl, tf * (size_t)pl->H * 42 * m2);
  ALLOC(pl->t_rlog0, sizeof(cd) * 70);
  ALLOC(pl->t_binom, sizeof(double) * (2 * p + 2) * (2 * p + 2));
  ALLOC(pl->qs, (f32 ? sizeof(float) : sizeof(double)) * n);
  if (!pl->adaptive) {
    ALLOC(pl->M, csz * (size_t)pl->nbox * P1);
    ALLOC(pl->A, csz * (size_t)pl->nbox * P1);
    ALLOC(pl->B, csz * (size_t)pl->nbox * P1);
  }
  ALLOC(pl->status, sizeof(int));
  ALLOC(pl->geo, 8 * sizeof(double));
  ALLOC(pl->dgeom, sizeof(DevGeom));
  ALLOC(pl->tree_ctr, sizeof(unsigned));
  ALLOC(pl->ctr, kCtrSlots * sizeof(int));
#undef ALLOC
  if (pl->adaptive) {
    s = adaptive_alloc(pl);
    if (s != HPFMM_OK) { free_plan(pl); return s; }
  }
  s = fmm_set_smem_limits(p);
  if (s == HPFMM_OK) s = fmm_prepare();
  if (s == HPFMM_OK) s = adaptive_prepare();
  if (s != HPFMM_OK) { free_plan(pl); return s; }
  {
    // the far-field streams of a split evaluation -- side (S2M, M2M, coarse
    // M2L) and m2l (leaf-level M2L, bottom-row image/reaction pairs, mirror
    // M2L) -- take the greatest priority: their short dependent kernels then
    // take SMs before the blocks of the near field on the caller's stream,
    // which fills the rest.  The table stream (reaction tables of a rebuild,
    // started once the tree is built) takes it too: the mirror M2L waits for
    // the tables, and at the default priority their blocks queued behind the
    // near field's until it was almost done.
    int prio_lo = 0, prio_hi = 0;
    cudaError_t ce = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (ce == cudaSuccess)
      ce = cudaStreamCreateWithPriority(&pl->side_stream, cudaStreamNonBlocking, prio_hi);
    if (ce == cudaSuccess)
      ce = cudaStreamCreateWithPriority(&pl->table_stream, cudaStreamNonBlocking, prio_hi);
    if (ce == cudaSuccess)
      ce = cudaStreamCreateWithPriority(&pl->m2l_stream, cudaStreamNonBlocking, prio_hi);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&pl->ev_qcopy, &pl->ev_qfree, &pl->ev_xcopy, &pl->ev_xyfree, &pl->ev_done})
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_s2m, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_m2lh, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_up, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_tree, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_geo, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_tables, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pl->ev_gather, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaMallocHost((void **)&pl->hgeo, 8 * sizeof(double));
    if (ce != cudaSuccess) {
      set_last_error("hpfmm_create: %s", cudaGetErrorString(ce));
      free_plan(pl);
      return HPFMM_ECUDA;
    }
  }
  cudaError_t e = cudaMemsetAsync(pl->status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->tree_ctr, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->ctr, 0, kCtrSlots * sizeof(int), st);
  if (e != cudaSuccess) {
    set_last_error("hpfmm_create: %s", cudaGetErrorString(e));
    free_plan(pl);
    return HPFMM_ECUDA;
  }
  s = tables_static(pl, st);
  if (s == HPFMM_OK) s = rebuild(pl, x, y, st, true);  // creation always validates
  if (s != HPFMM_OK) {
    cudaStreamSynchronize(st);
    free_plan(pl);
    return s;
  }
  *out = pl;
  return HPFMM_OK;
}

static hpfmm_status ensure_stage(hpfmm_plan *pl, int nrhs) {
  if (pl->stage_rhs >= nrhs) return HPFMM_OK;
  if (pl->in_q) cudaFree(pl->in_q);
  if (pl->out_pot) cudaFree(pl->out_pot);
  if (pl->out_grad) cudaFree(pl->out_grad);
  pl->in_q = nullptr;
  pl->out_pot = pl->out_grad = nullptr;
  pl->stage_rhs = 0;
  HP_TRY(plan_dalloc(pl, (void **)&pl->in_q, sizeof(double) * pl->n * nrhs));
  HP_TRY(plan_dalloc(pl, &pl->out_pot, 2 * sizeof(double) * pl->n * nrhs));
  HP_TRY(plan_dalloc(pl, &pl->out_grad, 4 * sizeof(double) * pl->n * nrhs));
  pl->stage_rhs = nrhs;
  return HPFMM_OK;
}

// charge vectors per multi-RHS pass set
constexpr int kMultiMax = 64;

static hpfmm_status ensure_multi(hpfmm_plan *pl, int nr) {
  if (pl->mcap >= nr) return HPFMM_OK;
  void **bufs[] = {&pl->mq, &pl->mqsm, &pl->mM, &pl->mA, &pl->mB};
  for (void **b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  pl->mcap = 0;
  const size_t n = (size_t)pl->n, ncoef = (size_t)pl->nbox * (pl->p + 1);
  HP_TRY(plan_dalloc(pl, &pl->mq, sizeof(float) * n * nr));
  HP_TRY(plan_dalloc(pl, &pl->mqsm, sizeof(float) * n * fmm_multi_rp(nr)));
  HP_TRY(plan_dalloc(pl, &pl->mM, 2 * sizeof(float) * ncoef * nr));
  HP_TRY(plan_dalloc(pl, &pl->mA, 2 * sizeof(float) * ncoef * nr));
  HP_TRY(plan_dalloc(pl, &pl->mB, 2 * sizeof(float) * ncoef * nr));
  pl->mcap = nr;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_eval(hpfmm_plan *pl, const double *q, int nrhs, double *pot,
                                   double *grad, void *stream) {
  if (!pl || !q || !pot || nrhs < 1) {
    set_last_error("hpfmm_eval: need plan, q, pot and nrhs >= 1");
    return HPFMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = pl->n;
  bool qd = is_device_pointer(q), pd = is_device_pointer(pot);
  bool gd = !grad || is_device_pointer(grad);
  const double *dq = q;
  double *dpot = pot, *dgrad = grad;
  if (!qd || !pd || !gd) HP_TRY(ensure_stage(pl, nrhs));
  // host charges: copied on the copy stream, so that the copy overlaps the
  // tree build still running on the caller's stream; the caller's stream
  // waits for it before the passes
  cudaStream_t cs = pl->copy_stream ? pl->copy_stream : st;
  if (!qd) {
    if (cs != st) HP_CUDA(cudaStreamWaitEvent(cs, pl->ev_qfree, 0));
    HP_CUDA(cudaMemcpyAsync(pl->in_q, q, sizeof(double) * n * nrhs, cudaMemcpyDefault, cs));
    if (cs != st) {
      HP_CUDA(cudaEventRecord(pl->ev_qcopy, cs));
      HP_CUDA(cudaStreamWaitEvent(st, pl->ev_qcopy, 0));
    }
    dq = pl->in_q;
  }
  if (!pd) dpot = (double *)pl->out_pot;
  if (!gd) dgrad = (double *)pl->out_grad;
  if (nrhs > 1 && fmm_multi_supported(pl)) {
    // single precision: the charge vectors share one set of passes, kMultiMax at a time
    const int chunk = nrhs < kMultiMax ? nrhs : kMultiMax;
    HP_TRY(ensure_multi(pl, chunk));
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
      const int nr = nrhs - r0 < chunk ? nrhs - r0 : chunk;
      HP_TRY(fmm_eval_multi(pl, dq + (size_t)r0 * n, nr, dpot + (size_t)2 * r0 * n,
                            dgrad ? dgrad + (size_t)4 * r0 * n : nullptr, pl->mq, pl->mqsm,
                            pl->mM, pl->mA, pl->mB, st));
    }
  } else {
    for (int r = 0; r < nrhs; ++r) {
      HP_TRY(fmm_eval(pl, dq + (size_t)r * n, dpot + (size_t)2 * r * n,
                      dgrad ? dgrad + (size_t)4 * r * n : nullptr, st));
    }
  }
  // the next call's charge copy may start once this call's passes are done
  if (!qd && cs != st) HP_CUDA(cudaEventRecord(pl->ev_qfree, st));
  // host outputs: potential on the caller's stream, gradient on the copy
  // stream, concurrently
  cudaStream_t gs = st;
  if (!gd && cs != st) {
    HP_CUDA(cudaEventRecord(pl->ev_done, st));
    HP_CUDA(cudaStreamWaitEvent(cs, pl->ev_done, 0));
    gs = cs;
  }
  if (!pd)
    HP_CUDA(cudaMemcpyAsync(pot, dpot, 2 * sizeof(double) * n * nrhs, cudaMemcpyDefault, st));
  if (!gd)
    HP_CUDA(cudaMemcpyAsync(grad, dgrad, 4 * sizeof(double) * n * nrhs, cudaMemcpyDefault, gs));
  if (!pd || !gd) HP_CUDA(cudaStreamSynchronize(st));
  if (gs != st) HP_CUDA(cudaStreamSynchronize(gs));
  return HPFMM_OK;
}

// targets must be finite, on y >= 0 and inside the plan's root square; the
// valid targets in the bottom leaf row (by the sources' quantisation) are
// appended to list, when there is one, for the image/reaction kernel
__global__ void k_check_targets(const double *__restrict__ xt, const double *__restrict__ yt,
                                int64_t nt, double x0, double side, double qscale, int H,
                                int *__restrict__ flag, int64_t *__restrict__ list) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const double x = xt[i], y = yt[i];
  const bool ok = isfinite(x) && isfinite(y) && y >= 0.0 && x >= x0 && x <= x0 + side &&
                  y <= side;
  if (!ok) {
    atomicOr(flag, 1);
    return;
  }
  if (list && (quantise(y, side, qscale) >> (30 - H)) == 0) list[atomicAdd(flag + 1, 1)] = i;
}

extern "C" hpfmm_status hpfmm_eval_targets(hpfmm_plan *pl, const double *q, const double *xt,
                                           const double *yt, int64_t nt, double *pot,
                                           double *grad, void *stream) {
  if (!pl || !q || nt < 0 || (nt > 0 && (!xt || !yt || !pot))) {
    set_last_error("hpfmm_eval_targets: need plan, q, nt >= 0 and, for nt > 0, xt, yt, pot");
    return HPFMM_EINVAL;
  }
  if (nt == 0) return HPFMM_OK;
  const void *ptrs[] = {q, xt, yt, pot, grad};
  for (const void *p : ptrs)
    if (p && !is_device_pointer(p)) {
      set_last_error("hpfmm_eval_targets: arrays must be device memory");
      return HPFMM_EINVAL;
    }
  if (pl->adaptive) {
    set_last_error("hpfmm_eval_targets: not implemented for adaptive plans");
    return HPFMM_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HP_TRY(plan_host_geometry(pl));
  const bool single = pl->prec != HPFMM_FP64;
  if (!pl->tflag) HP_TRY(plan_dalloc(pl, (void **)&pl->tflag, 2 * sizeof(int)));
  if (single && nt > pl->tlist_cap) {
    HP_CUDA(cudaStreamSynchronize(st));
    if (pl->tlist) {
      cudaFree(pl->tlist);
      pl->workspace_bytes -= (int64_t)sizeof(int64_t) * pl->tlist_cap;
      pl->tlist = nullptr;
      pl->tlist_cap = 0;
    }
    HP_TRY(plan_dalloc(pl, (void **)&pl->tlist, sizeof(int64_t) * (size_t)nt));
    pl->tlist_cap = nt;
  }
  int hflag[2] = {0, 0};
  HP_CUDA(cudaMemsetAsync(pl->tflag, 0, 2 * sizeof(int), st));
  k_check_targets<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(
      xt, yt, nt, pl->x0, pl->side, pl->qscale, pl->H, pl->tflag, single ? pl->tlist : nullptr);
  HP_LAUNCH_CHECK();
  HP_CUDA(cudaMemcpyAsync(hflag, pl->tflag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  if (hflag[0]) {
    set_last_error("hpfmm_eval_targets: targets must be finite, with y >= 0, inside the root "
                   "square [%g, %g] x [0, %g]",
                   pl->x0, pl->x0 + pl->side, pl->side);
    return HPFMM_EINVAL;
  }
  return fmm_eval_targets(pl, q, xt, yt, nt, single ? pl->tlist : nullptr, hflag[1], pot, grad,
                          st);
}

extern "C" hpfmm_status hpfmm_destroy(hpfmm_plan *pl) {
  if (!pl) return HPFMM_OK;
  cudaDeviceSynchronize();
  free_plan(pl);
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_get_info(const hpfmm_plan *pl, hpfmm_plan_info *info) {
  if (!pl || !info) {
    set_last_error("hpfmm_get_info: null argument");
    return HPFMM_EINVAL;
  }
  HP_TRY(plan_host_geometry(const_cast<hpfmm_plan *>(pl)));
  info->n = pl->n;
  info->levels = pl->H;
  info->p = pl->p;
  info->prec = pl->prec;
  info->x0 = pl->x0;
  info->side = pl->side;
  info->workspace_bytes = pl->workspace_bytes;
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_get_order(const hpfmm_plan *pl, uint64_t *keys, int64_t *perm,
                                        void *stream) {
  if (!pl) {
    set_last_error("hpfmm_get_order: null plan");
    return HPFMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (keys)
    HP_CUDA(cudaMemcpyAsync(keys, pl->keys, sizeof(uint64_t) * pl->n, cudaMemcpyDefault, st));
  if (perm)
    HP_CUDA(cudaMemcpyAsync(perm, pl->perm, sizeof(int64_t) * pl->n, cudaMemcpyDefault, st));
  HP_CUDA(cudaStreamSynchronize(st));
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_sync(hpfmm_plan *pl, void *stream) {
  if (!pl) {
    set_last_error("hpfmm_sync: null plan");
    return HPFMM_EINVAL;
  }
  int hs = 0;
  cudaStream_t st = (cudaStream_t)stream;
  HP_CUDA(cudaMemcpyAsync(&hs, pl->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  HP_TRY(plan_host_geometry(pl));
  if (hs == 0) return HPFMM_OK;
  // reported once: the word is cleared (and, after a timeout, the fused
  // upward pass's counters reset) so that the plan can be used again
  HP_CUDA(cudaMemsetAsync(pl->status, 0, sizeof(int), st));
  if (hs & HPFMM_DEV_TIMEOUT) HP_CUDA(cudaMemsetAsync(pl->ctr, 0, kCtrSlots * sizeof(int), st));
  HP_CUDA(cudaStreamSynchronize(st));
  if (hs & HPFMM_DEV_TIMEOUT) {
    set_last_error("device status word = %d: a bounded device wait gave up", hs);
    return HPFMM_ETIMEOUT;
  }
  if (hs & HPFMM_DEV_EINVAL) {
    set_last_error("asynchronous rebuild: points must be finite with y > 0 (or the root square "
                   "does not contain them)");
    return HPFMM_EINVAL;
  }
  set_last_error("asynchronous rebuild: |kappa| * sqrt(5) * side exceeds 60, the range of the "
                 "device I_n evaluation");
  return HPFMM_EUNSUPPORTED;
}
