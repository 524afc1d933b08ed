// common.cuh -- shared definitions of the GB300 half-plane Robin FMM library:
// complex arithmetic, the plan object, error plumbing, tree geometry helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hpfmm.h"

#ifndef HPFMM_MAX_P
#define HPFMM_MAX_P 40
#endif
#define HPFMM_NPASS 10

// ---------------------------------------------------------------------------
// complex numbers (interleaved re, im)
template <typename R>
struct alignas(sizeof(R) * 2) cpx {
  R x, y;
};
using cd = cpx<double>;
using cf = cpx<float>;

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  cpx<R> z;
  z.x = a;
  z.y = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x + b.x, a.y + b.y);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x - b.x, a.y - b.y);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a) {
  return mk<R>(-a.x, -a.y);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) {
  return mk<R>(s * a.x, s * a.y);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> conj(cpx<R> a) {
  return mk<R>(a.x, -a.y);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> mul_i(cpx<R> a) {  // i * a
  return mk<R>(-a.y, a.x);
}
template <typename R>
__host__ __device__ __forceinline__ R abs2(cpx<R> a) {
  return a.x * a.x + a.y * a.y;
}
// a += b * c
template <typename R>
__host__ __device__ __forceinline__ void cfma(cpx<R> &a, cpx<R> b, cpx<R> c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cinv(cpx<R> b) {
  // 1/b = conj(b')/|b'|^2 * (1/s) with b' = b/s, s = |re| + |im| (no overflow);
  // two real divisions
  const R s = fabs(b.x) + fabs(b.y);
  const R is = R(1) / s;
  const R bx = b.x * is, by = b.y * is;
  const R id = is / (bx * bx + by * by);
  return mk<R>(bx * id, -by * id);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cdiv(cpx<R> a, cpx<R> b) {
  return a * cinv(b);
}
__device__ __forceinline__ cd cexp_d(cd z) {
  double s, c;
  sincos(z.y, &s, &c);
  double e = exp(z.x);
  return mk<double>(e * c, e * s);
}
__device__ __forceinline__ cd clog_d(cd z) {
  return mk<double>(0.5 * log(z.x * z.x + z.y * z.y), atan2(z.y, z.x));
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> to(cd z) {
  return mk<R>(R(z.x), R(z.y));
}

// ---------------------------------------------------------------------------
// Bulk (TMA) copies into shared memory tracked by an mbarrier.  Waits are
// bounded: after kMbarSpin unsuccessful polls the caller records a timeout in
// the plan's status word instead of spinning for ever.
constexpr int kMbarSpin = 1 << 20;
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared bulk copy: both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on phase `parity`; false when it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
  for (int it = 0; it < kMbarSpin; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}
// device status bits (the plan's status word): a bounded wait gave up;
// (asynchronous rebuilds) the points were invalid; |kappa| sqrt(5) side was
// beyond the range of the device I_n evaluation
enum { HPFMM_DEV_TIMEOUT = 1, HPFMM_DEV_EINVAL = 2, HPFMM_DEV_RANGE = 4 };

// Geometry of a uniform tree as the evaluation kernels read it: written on
// the device by the tree build, so that nothing between a rebuild and an
// evaluation waits for the host to learn the root square.  Level l has box
// side d_l = side 2^-l; d[l] is d_l rounded to single precision and dlo[l]
// the rest (d_l = d[l] + dlo[l] to about 2^-48 relative), so that offsets
// between single-precision leaf frames stay exact.
struct DevGeom {
  double x0, side, qscale;
  double logd[16];
  float d[16], invd[16], dlo[16];
};

// ---------------------------------------------------------------------------
// Morton geometry.  Key bit 2b holds bit b of ix, bit 2b+1 bit b of iy; the
// level-l box of a point is key >> (60 - 2l), its Morton index within level l.
__host__ __device__ __forceinline__ uint32_t compact1(uint64_t m) {
  // gather the even bits of m into the low 32 bits
  m &= 0x5555555555555555ull;
  m = (m | (m >> 1)) & 0x3333333333333333ull;
  m = (m | (m >> 2)) & 0x0f0f0f0f0f0f0f0full;
  m = (m | (m >> 4)) & 0x00ff00ff00ff00ffull;
  m = (m | (m >> 8)) & 0x0000ffff0000ffffull;
  m = (m | (m >> 16)) & 0x00000000ffffffffull;
  return (uint32_t)m;
}
__host__ __device__ __forceinline__ uint64_t spread1(uint32_t v) {
  uint64_t m = v;
  m = (m | (m << 16)) & 0x0000ffff0000ffffull;
  m = (m | (m << 8)) & 0x00ff00ff00ff00ffull;
  m = (m | (m << 4)) & 0x0f0f0f0f0f0f0f0full;
  m = (m | (m << 2)) & 0x3333333333333333ull;
  m = (m | (m << 1)) & 0x5555555555555555ull;
  return m;
}
__host__ __device__ __forceinline__ int box_ix(uint64_t m) { return (int)compact1(m); }
__host__ __device__ __forceinline__ int box_iy(uint64_t m) { return (int)compact1(m >> 1); }
__host__ __device__ __forceinline__ uint64_t box_morton(int ix, int iy) {
  return spread1((uint32_t)ix) | (spread1((uint32_t)iy) << 1);
}
// ix = min(floor((x - x0) / L * 2^30), 2^30 - 1) with the quotient correctly
// rounded, so that the key matches a plain IEEE host computation bit for bit.
// Fast path: s' = v * RN(2^30 / L) is within 2 ulp of the exact scaled
// quotient, and the correctly rounded RN(v / L) * 2^30 is within 1/2 ulp of
// it; when no integer lies within 4 ulp of s', both floors agree.  Otherwise
// (a fraction ~1e-7 of the points) the exact division decides.
__device__ __forceinline__ uint64_t quantise(double v, double L, double scale) {
  const double s = __dmul_rn(v, scale);
  // floor(s) and the distance of s to the nearest integers, in ulps of s,
  // from the bit pattern (s >= 0, s < 2^31)
  const long long b = __double_as_longlong(s);
  const int E = (int)((b >> 52) & 0x7ff) - 1023;
  bool safe;
  uint64_t f;
  if (E < 0) {  // s < 1
    f = 0;
    safe = s < 0.999999;
  } else {
    const uint64_t m = (uint64_t)(b & 0xfffffffffffffull) | (1ull << 52);
    const int fb = 52 - E;  // fraction bits (>= 21 here)
    f = m >> fb;
    const uint64_t frac = m & ((1ull << fb) - 1);
    safe = frac >= 4 && frac <= (1ull << fb) - 5;
  }
  if (!safe) {
    const double q = __ddiv_rn(v, L);
    double fl = floor(__dmul_rn(q, 1073741824.0));
    fl = fmax(fl, 0.0);
    f = (uint64_t)fl;
  }
  return f > 1073741823ull ? 1073741823ull : f;
}

// Two single-precision values in one 64-bit register and the paired FP32
// instructions of this architecture (add/sub/fma .f32x2: one issue slot for
// two results, each rounded to nearest as the scalar instruction rounds it).
// The near-field pair loops apply them to the (x, y) differences and field
// sums, the patch M2L to the real and imaginary halves of its complex
// multiply-adds.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2_pack(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2p v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2p f2_sub(f2p a, f2p b) {
  f2p d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p f2_add(f2p a, f2p b) {
  f2p d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p f2_fma(f2p a, f2p b, f2p c) {
  f2p d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Programmatic dependent launch (chains of short dependent kernels on one
// stream): a kernel launched by launch_dependent may be scheduled before its
// predecessor on the stream has finished; it calls pdl_wait() before its
// first access to memory the predecessor writes (the wait returns once the
// predecessor has completed and its writes are visible), and each kernel of
// the chain calls pdl_trigger() to let its successor be scheduled as its own
// blocks finish.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// centre of leaf (ix, iy) of side d in the root square starting at x0, with
// explicit roundings: the single-precision leaf frames of the sources and of
// separate targets must use bit-identical centres
__device__ __forceinline__ double2 leaf_centre_at(double x0, double d, int ix, int iy) {
  return make_double2(__fma_rn(ix + 0.5, d, x0), __dmul_rn(iy + 0.5, d));
}

// The single-precision Hankel form of the free-space M2L (the patch kernels
// of the uniform tree and the adaptive tree's kernel) scales its factors by
// powers of R = 2^kHankelLog2R -- the class vector entries g_j by R^-j (in
// the table), the moment and output factors 1/k! and 1/l! by R^k and R^l --
// which leaves every product, and so every result, unchanged bit for bit
// (powers of two scale exactly) but keeps the factors within the single-
// precision range up to p = 40: (2p - 1)! alone overflows past p = 21 and
// 1/p! underflows past p = 33.
constexpr int kHankelLog2R = 4;

// deepest level of an adaptive tree (its dense per-level box index has
// (4^(L+1) - 1) / 3 entries)
constexpr int kAdaptiveMaxLevel = 13;

// first box of level l in the level-concatenated box arrays: (4^l - 1) / 3
__host__ __device__ __forceinline__ int64_t level_offset(int l) {
  return ((int64_t(1) << (2 * l)) - 1) / 3;
}

// ---------------------------------------------------------------------------
// the plan
struct hpfmm_plan {
  int64_t n = 0;
  int H = 0;  // leaf level
  int p = 0;
  int prec = HPFMM_FP64;
  double tau_fp64 = 0.05;
  int subtree = 0;   // fused upward/downward subtree depth (0: automatic)
  int m2l_mode = 0;  // multi-RHS free M2L (16+ RHS): 0 FP32 FMA kernel, 1 tensor cores
  double root_x0 = 0, root_side = 0;  // root square override (root_side > 0)
  double kre = 1, kim = 0;
  double x0 = 0, side = 1;
  double qscale = 1073741824.0;  // 2^30 / side rounded: the key quantisation scale
  int Hsort = 0;     // level of the sort buckets (the leaf level H of a uniform tree)
  // adaptive tree (hpfmm_options.adaptive): boxes level by level, Morton order
  // within a level; see adaptive.cu
  int adaptive = 0;
  int leaf_cap = 32;       // split while a box holds more points than this
  int64_t acap = 0;        // box capacity (a bound on the number of boxes)
  int64_t ad_maxlev = 0;   // bound on the boxes of one level
  int64_t ad_nbox = 0;     // boxes of the current tree
  int64_t ad_mcap = 0;     // boxes the expansion arrays M, A, B hold
  int ad_depth = 0;        // deepest level with a box
  int ad_nleaf = 0;        // leaves of the current tree
  int ad_lev[32] = {};     // host copy: first box of each level, levels 0..H+1
  uint64_t *ab_key = nullptr;  // Morton key of a box at its level
  int *ab_lo = nullptr, *ab_hi = nullptr;  // point range (tree order)
  int *ab_parent = nullptr, *ab_lvl = nullptr;
  int4 *ab_child = nullptr;    // children by type (ix & 1) | (iy & 1) << 1, -1: none
  int4 *ab_cut = nullptr;      // split points of a box's range between its four children
  int *ab_off = nullptr;       // build scratch: children offsets, leaf flags
  int *ab_idx = nullptr;       // dense index per level: Morton key -> box (validated on use)
  int *ab_lev = nullptr;       // device: first box of each level
  int *ab_btot = nullptr;      // scan block totals
  int *ab_lrank = nullptr;     // per point: rank of its leaf in tree order
  int *ab_leaf = nullptr;      // leaves by rank
  int64_t nbox = 0;  // boxes over levels 0..H
  int nleaf = 0;     // 4^H

  // tree (device)
  double *xs = nullptr, *ys = nullptr;  // sorted coordinates
  int64_t *perm = nullptr;              // sorted position -> caller index
  uint64_t *keys = nullptr;             // sorted keys
  int *leaf_start = nullptr;            // nleaf + 1 offsets into the sorted order
  float2 *loc32 = nullptr;              // FP32 path: (x, y) relative to the leaf centre
  float2 *loclo = nullptr;              // FP32 path: the rest, (x, y) - centre - loc32
  float *yabs = nullptr;                // FP32 path: y itself (bottom-row image/reaction pairs)

  // tables (device, double); FP32 copies when prec != FP64
  void *t_m2m = nullptr;   // 4 x (p+1)^2 complex: child c -> parent
  void *t_l2l = nullptr;   // 4 x (p+1)^2 complex: parent -> child c (analytic part)
  void *t_m2l = nullptr;   // 49 offset classes x (p+1)^2 complex: free-space log M2L
  void *t_m2l_pad = nullptr;  // FP32 path: Hankel form of the 40 far classes (2 x 2(p+1) each)
  void *t_m2l_tc = nullptr;   // tensor-core M2L: the 40 far classes as tf32 hi/lo operands
  void *t_refl = nullptr;  // per level: 7 x 3 classes x (2p+1) complex: scaled I_k tables
  void *t_rlog = nullptr;  // per level: 7 x 3 classes x (p+1)^2 complex: image-log M2L
  void *t_rlog0 = nullptr;    // logs of the 49 free and 21 image class displacements
  double *t_binom = nullptr;  // binomial coefficients C(a, b), a, b < 2p + 2

  // workspace (device)
  void *qs = nullptr;  // sorted charges (R)
  void *M = nullptr;   // multipole moments, nbox x (p+1) complex (R)
  void *A = nullptr;   // analytic local expansion, nbox x (p+1) complex
  void *B = nullptr;   // anti-analytic local expansion
  void *out_pot = nullptr, *out_grad = nullptr;  // staging for host outputs
  double *in_q = nullptr;                         // staging for host charges
  int64_t stage_rhs = 0;
  double *adj = nullptr;  // adjoint workspace (20 n doubles), allocated on first use
  // multi-RHS workspace (single precision), for up to mcap charge vectors at once
  void *mq = nullptr, *mqsm = nullptr, *mM = nullptr, *mA = nullptr, *mB = nullptr;
  int mcap = 0;
  // hpfmm_eval_targets: validation flag and bottom-row target count (int[2]);
  // the list of targets in the bottom leaf row (single-precision plans)
  int *tflag = nullptr;
  int64_t *tlist = nullptr;
  int64_t tlist_cap = 0;
  // the far-field chain of a split single-precision evaluation
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_geo = nullptr, ev_tables = nullptr;
  // the geometry copy to the host and the reaction tables of a rebuild run on
  // table_stream once the root square is known (ev_tree, recorded inside the
  // tree build); the tables are joined into the evaluation's stream before
  // the mirror M2L that reads them
  cudaStream_t table_stream = nullptr;
  cudaEvent_t ev_tree = nullptr;
  // host-buffer calls: their copies on copy_stream, overlapping the tree
  // build (the charges) or each other (x and y; potential and gradient).
  // ev_qfree / ev_xyfree: the previous call's readers of the staging buffers
  // are done; ev_qcopy / ev_xcopy: the copies are done; ev_done: the
  // evaluation's outputs are written
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_qcopy = nullptr, ev_qfree = nullptr, ev_xcopy = nullptr, ev_xyfree = nullptr,
              ev_done = nullptr;
  double *in_xy = nullptr;  // staged coordinates of a host-buffer rebuild (x, then y)
  bool tables_pending = false;
  // fork / join of the far-field chain on the side stream (single
  // precision); ev_gather: the charges in tree order are written (the
  // bottom-row pairs wait for it)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_gather = nullptr;
  // the leaf level's M2L on its own stream, after the S2M (ev_s2m), joined
  // into the far-field chain (ev_m2lh)
  cudaStream_t m2l_stream = nullptr;
  cudaEvent_t ev_s2m = nullptr, ev_m2lh = nullptr;
  // the mirror M2L on the m2l stream after the upward pass (ev_up), into
  // mir_A / mir_B (rows 0 and 1 of every level), joined with the leaf-level
  // M2L (ev_m2lh) before the downward pass; single-precision uniform plans
  cudaEvent_t ev_up = nullptr;
  void *mir_A = nullptr, *mir_B = nullptr;
  float4 *near = nullptr;  // near-field sums per point (sorted order)
  double *hgeo = nullptr;  // pinned host copy of geo, written by the tree build
  int *status = nullptr;  // device status word
  double *geo = nullptr;  // device: x0, side, invalid flag, 2^30/side, largest leaf (int)
  DevGeom *dgeom = nullptr;  // device: level geometry of the current tree
  unsigned *tree_ctr = nullptr;  // device: last-block counter of the tree build
  int *ctr = nullptr;     // device: last-block counters of the fused upward pass, one per RHS
  int async_update = 0;   // hpfmm_options.async_update
  bool geo_pending = false;  // host copies x0 / side / qscale wait for ev_geo
  void *tree_tmp = nullptr;  // tree-build temporaries, kept for the rebuilds of the plan
  int64_t tree_tmp_bytes = 0;
  int sms = 0;               // streaming multiprocessors of the plan's device
  int64_t workspace_bytes = 0;

  // pass timing (events on the caller's stream) and launch counts
  bool timing = false;
  int64_t launches[HPFMM_NPASS] = {};
  void *tstate = nullptr;  // TimingState, see api.cu
};

// pass ids of hpfmm_read_timing
enum { PASS_TREE = 0, PASS_TABLES, PASS_GATHER, PASS_P2M, PASS_M2M, PASS_M2L_FREE,
       PASS_M2L_MIRROR, PASS_L2L, PASS_EVAL, PASS_NEAR_MIRROR };
// record the start / end of a pass on stream st (no-ops unless timing is on);
// pass_end also adds nlaunch to the pass's launch count
void pass_begin(hpfmm_plan *pl, cudaStream_t st, int pass);
void pass_end(hpfmm_plan *pl, cudaStream_t st, int pass, int nlaunch);

// ---------------------------------------------------------------------------
// error plumbing (host)
void set_last_error(const char *fmt, ...);
#define HP_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_last_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return HPFMM_ECUDA;                                                               \
    }                                                                                   \
  } while (0)
#define HP_LAUNCH_CHECK()                                                               \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) {                                                            \
      set_last_error("%s:%d kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return HPFMM_ECUDA;                                                               \
    }                                                                                   \
  } while (0)
#define HP_TRY(call)                       \
  do {                                     \
    hpfmm_status s_ = (call);              \
    if (s_ != HPFMM_OK) return s_;         \
  } while (0)

// internal entry points shared between translation units
hpfmm_status tree_build(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st);
hpfmm_status tree_finish(hpfmm_plan *pl, const double *hgeo, cudaStream_t st);
hpfmm_status tables_static(hpfmm_plan *pl, cudaStream_t st);
hpfmm_status tables_build(hpfmm_plan *pl, cudaStream_t st);
hpfmm_status fmm_eval(hpfmm_plan *pl, const double *q, double *pot, double *grad, cudaStream_t st);
// multi-RHS evaluation of nr charge vectors in one set of passes (single
// precision); qs: nr n floats, qsm: n fmm_multi_rp(nr) floats, M/A/B: nr nbox
// (p+1) complex floats each
bool fmm_multi_supported(const hpfmm_plan *pl);
// evaluation at nt separate targets (device arrays inside the root square)
hpfmm_status adaptive_build(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st);
hpfmm_status adaptive_eval(hpfmm_plan *pl, const double *q, double *pot, double *grad,
                           cudaStream_t st);
hpfmm_status adaptive_alloc(hpfmm_plan *pl);
// constant-memory set-up of the translation units that evaluate I_n on the
// device (a synchronous copy, so done at plan creation and never inside a
// stream capture such as the batched graph)
hpfmm_status fmm_prepare();
hpfmm_status adaptive_prepare();
hpfmm_status fmm_eval_targets(hpfmm_plan *pl, const double *q, const double *xt,
                              const double *yt, int64_t nt, const int64_t *blist,
                              int64_t nbottom, double *pot, double *grad, cudaStream_t st);
int fmm_multi_rp(int nr);
hpfmm_status fmm_eval_multi(hpfmm_plan *pl, const double *q, int nr, double *pot, double *grad,
                            void *qs, void *qsm, void *M, void *A, void *B, cudaStream_t st);
bool is_device_pointer(const void *p);
hpfmm_status plan_dalloc(hpfmm_plan *pl, void **p, size_t bytes);
// host copies of the root square (x0, side, qscale) of the current tree: waits
// for the geometry of an asynchronous rebuild when it has not arrived yet
hpfmm_status plan_host_geometry(hpfmm_plan *pl);
// order `st` after the reaction tables of the last rebuild (once per rebuild)
hpfmm_status plan_join_tables(hpfmm_plan *pl, cudaStream_t st);
