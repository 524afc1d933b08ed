// fmm.cu -- the FMM passes of Algorithms 1 and 2 on a uniform quadtree.
//
// One quadtree over the points (levels 0..H, box side d_l = L / 2^l) serves
// all four components of Algorithm 2: its boxes are the source and target
// boxes of the free-space FMM, and their mirrors (x, y) -> (x, -y) are the
// image-source boxes of Algorithm 1 (the tree "over targets and image
// sources"), for both Phi_2^+ and the x-mirrored Phi_2^-.
//
// Lists (uniform grid, level l):
//   free V-list of box t: children of the neighbours of parent(t) that are not
//     neighbours of t (levels l >= 2, the classic 2-D FMM);
//   mirror list of box t: boxes s with parent(s) a mirror-neighbour of
//     parent(t) and s not a mirror-neighbour of t, where boxes a, b are
//     mirror-neighbours when both lie in the bottom row (iy = 0) and
//     |ix_a - ix_b| <= 1, i.e. when a touches the mirror of b.  Only boxes in
//     rows 0 and 1 have a mirror list (levels l >= 1): the reaction and image
//     parts are far field everywhere else, which is why the paper finds the
//     reaction components much cheaper than the free-space ones (Section 4,
//     Example 2);
//   near field at the leaves: the 3x3 neighbourhood (free part, j != i) and,
//     for bottom-row leaves, the bottom-row neighbours (image and reaction).
// The admissibility of both lists is |r_c - r_c'| >= 2d, which satisfies the
// M2L condition |r_c - r_c'| > sqrt(2)(d_s + d_t)/2 of Theorem 3.7.
//
// Per box: one multipole vector M (power moments of the charges, scaled by d;
// the image and reaction moments are conj(M_n) and (-+i)^n conj/M_n, see
// tables.cu) and two local vectors A (analytic) and B (anti-analytic): the
// log parts, which are real parts of analytic functions, contribute L/2 to A
// and conj(L)/2 to B; Phi_2^+ contributes to A and Phi_2^- to B.
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "pairs.cuh"
#include "special.cuh"
#include "near32.cuh"
#include "tc.cuh"
#include "m2l_patch.cuh"
#include "fsplit.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;

// Box side, its reciprocal and log per level come from the plan's DevGeom
// record, written on the device by the tree build (no kernel repeats
// double-precision set-up arithmetic per thread: GB300's FP64 pipe is narrow).

// --------------------------------------------------------------------------
// gather the charges into tree order
// (blockIdx.y = RHS; qsm, when given, also receives the charges point-major:
// qsm[k * rp + r], for the multi-RHS near field)
template <typename R>
__global__ void k_gather_q(const double *__restrict__ q, const int64_t *__restrict__ perm,
                           int64_t n, R *__restrict__ qs, R *__restrict__ qsm, int rp) {
  pdl_wait();  // launched as a dependent of the tree build's last kernel
  pdl_trigger();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int r = blockIdx.y;
  const double qd = q[(size_t)r * n + perm[k]];
  R v;
  if constexpr (sizeof(R) == 4)
    v = fs_round(qd);  // the rounding by integer operations (no FP64 conversion)
  else
    v = qd;
  qs[(size_t)r * n + k] = v;
  if (qsm) qsm[(size_t)k * rp + r] = v;
}

// point position relative to its leaf centre, in units of the leaf side
template <typename R>
struct LeafPoints;

template <>
struct LeafPoints<double> {
  const double *xs, *ys;
  double x0;
  __device__ __forceinline__ void rel(int64_t k, double cx, double cy, double &rx,
                                      double &ry) const {
    rx = xs[k] - cx;
    ry = ys[k] - cy;
  }
};
template <>
struct LeafPoints<float> {
  const float2 *loc;
  __device__ __forceinline__ void rel(int64_t k, double, double, float &rx, float &ry) const {
    float2 v = loc[k];
    rx = v.x;
    ry = v.y;
  }
};

// --------------------------------------------------------------------------
// P2M (S2M, Eq. MEcoefficients up to the phase and conjugation, see tables.cu):
// M_n = sum_{j in leaf} Q_j ((z_j - z_c)/d)^n.  One warp per leaf; lanes take
// 32 points at a time, write q w^n into a shared buffer, then lanes sum the
// buffer column by column.
template <typename R>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_p2m(LeafPoints<R> pts, const R *__restrict__ qs, const int *__restrict__ leaf_start, int H,
      const DevGeom *__restrict__ dg, int p, cpx<R> *__restrict__ M) {
  const double x0 = dg->x0, side = dg->side;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int P1 = p + 1;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cpx<R> *buf = reinterpret_cast<cpx<R> *>(smem_raw) + (size_t)warp * P1 * 33;
  int leaf = blockIdx.x * kWarpsPerBlock + warp;
  int nleaf = 1 << (2 * H);
  if (leaf >= nleaf) return;
  double d = side / (double)(1 << H);
  double cx = x0 + (box_ix(leaf) + 0.5) * d, cy = (box_iy(leaf) + 0.5) * d;
  R invd = (R)(1.0 / d);
  int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
  cpx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
  for (int base = b0; base < b1; base += 32) {
    int k = base + lane;
    int cnt = min(32, b1 - base);
    if (k < b1) {
      R rx, ry;
      pts.rel(k, cx, cy, rx, ry);
      cpx<R> w = mk<R>(rx * invd, ry * invd);
      cpx<R> t = mk<R>(qs[k], 0);
      for (int n = 0; n < P1; ++n) {
        buf[n * 33 + lane] = t;
        t = t * w;
      }
    }
    __syncwarp();
    for (int n = lane; n < P1; n += 32) {
      cpx<R> s = mk<R>(0, 0);
      for (int j = 0; j < cnt; ++j) s = s + buf[n * 33 + j];
      if (n == lane) acc0 = acc0 + s;
      else acc1 = acc1 + s;
    }
    __syncwarp();
  }
  cpx<R> *out = M + (size_t)(level_offset(H) + leaf) * P1;
  if (lane < P1) out[lane] = acc0;
  if (lane + 32 < P1) out[lane + 32] = acc1;
}

// --------------------------------------------------------------------------
// Single-precision S2M, M_n = sum_j Q_j w_j^n with w_j = (z_j - z_c)/d: one
// thread per (leaf, n) or (leaf, group of orders), with no cross-thread
// reduction, so the short leaves of a deep tree keep every lane busy.  w^n by
// repeated squaring.
template <typename R>
__device__ __forceinline__ cpx<R> cpow_int(cpx<R> w, int n) {
  cpx<R> r = mk<R>(1, 0);
  while (n) {
    if (n & 1) r = r * w;
    w = w * w;
    n >>= 1;
  }
  return r;
}

constexpr int kS2mGroup = 8;  // orders per thread of the single-precision S2M (a power of 2)

// Single-precision S2M over a tile of kS2mLeaves consecutive leaves per block.
// The tile's points are contiguous in tree order, so the block first copies
// their leaf-frame positions and charges into shared memory with coalesced
// loads (a per-thread loop over global memory would wait on one load per
// point); a tile of more than kS2mCap points reads them from global memory
// instead.  Each thread then takes items (leaf, group of kS2mGroup = G
// consecutive orders n0 .. n0+G-1): w^n0 = (w^G)^(n0/G) from log2 G
// squarings, then one product per further n.  The sums are compensated (Kahan): the moments of a
// leaf are sums of up to hundreds of terms of both signs, and their rounding
// error is inherited by every far-field coefficient built from them.
constexpr int kS2mLeaves = 64, kS2mCap = 2048, kS2mThreads = 128;

__global__ void __launch_bounds__(kS2mThreads)
k_s2m_tile(const float2 *__restrict__ loc, const float *__restrict__ qs,
           const int *__restrict__ leaf_start, int H, const DevGeom *__restrict__ dg, int p,
           cf *__restrict__ M, RhsStride rs) {
  constexpr int G = kS2mGroup;
  __shared__ float2 sp[kS2mCap];
  __shared__ float sq[kS2mCap];
  pdl_trigger();  // the upward pass may be scheduled behind it
  const int P1 = p + 1, NB = (P1 + G - 1) / G;
  qs += blockIdx.y * rs.q;
  M += blockIdx.y * rs.m;
  const int nleaf = 1 << (2 * H);
  const int L0 = blockIdx.x * kS2mLeaves, L1 = min(L0 + kS2mLeaves, nleaf);
  const int t0 = leaf_start[L0], t1 = leaf_start[L1];
  const bool staged = t1 - t0 <= kS2mCap;
  if (staged) {
    for (int i = threadIdx.x; i < t1 - t0; i += blockDim.x) {
      sp[i] = loc[t0 + i];
      sq[i] = qs[t0 + i];
    }
  }
  __syncthreads();
  const float invd = dg->invd[H];
  for (int it = threadIdx.x; it < (L1 - L0) * NB; it += blockDim.x) {
    const int leaf = L0 + it / NB, nb = it % NB, n0 = G * nb;
    const int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
    // the compensated sums of the real and imaginary parts as paired FP32
    // additions (the same roundings as the scalar form)
    f2p acc[G], cmp[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = cmp[g] = f2_pack(0.f, 0.f);
    for (int j = b0; j < b1; ++j) {
      const float2 v = staged ? sp[j - t0] : loc[j];
      const float qj = staged ? sq[j - t0] : qs[j];
      const cf w = mk(v.x * invd, v.y * invd);
      cf wg = w;  // w^G by squarings
#pragma unroll
      for (int g = 1; g < G; g <<= 1) wg = wg * wg;
      cf wn = mk(qj, 0.f);
      for (int i = 0; i < nb; ++i) wn = wn * wg;  // q w^n0
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const f2p yv = f2_sub(f2_pack(wn.x, wn.y), cmp[g]);
        const f2p tv = f2_add(acc[g], yv);
        cmp[g] = f2_sub(f2_sub(tv, acc[g]), yv);
        acc[g] = tv;
        wn = wn * w;
      }
    }
    const size_t e0 = ((size_t)level_offset(H) + leaf) * P1;
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (n0 + g < P1) {
        float ax, ay;
        f2_unpack(acc[g], ax, ay);
        M[e0 + n0 + g] = mk(ax, ay);
      }
  }
}

// Multi-RHS S2M (single precision): the powers ((z_j - z_c)/d)^n of a point
// are formed once and applied to RC charge vectors (blockIdx.y selects RHS
// r0 .. r0 + RC - 1; charges point-major, qsm[k * rp + r]), with the same
// compensated summation per RHS as k_s2m_tile.
template <int RC>
__global__ void __launch_bounds__(256)
k_s2m_multi(const float2 *__restrict__ loc, const float *__restrict__ qsm, int rp, int nr,
            const int *__restrict__ leaf_start, int H, const DevGeom *__restrict__ dg, int p,
            cf *__restrict__ M, RhsStride rs) {
  const int P1 = p + 1;
  const float invd = dg->invd[H];
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nleaf = 1u << (2 * H);
  if (t >= nleaf * (unsigned)P1) return;
  const unsigned leaf = t / (unsigned)P1;
  const int n = (int)(t - leaf * (unsigned)P1);
  const int r0 = blockIdx.y * RC;
  const int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
  cf acc[RC], cmp[RC];
#pragma unroll
  for (int c = 0; c < RC; ++c) acc[c] = cmp[c] = mk(0.f, 0.f);
  for (int j = b0; j < b1; ++j) {
    const float2 v = loc[j];
    const cf wn = cpow_int(mk(v.x * invd, v.y * invd), n);
    const float4 *qv = reinterpret_cast<const float4 *>(qsm + (size_t)j * rp + r0);
#pragma unroll
    for (int c4 = 0; c4 < RC / 4; ++c4) {
      const float4 qq = __ldg(qv + c4);
      const float qa[4] = {qq.x, qq.y, qq.z, qq.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * c4 + u;
        const cf yv = qa[u] * wn - cmp[c];
        const cf tv = acc[c] + yv;
        cmp[c] = (tv - acc[c]) - yv;
        acc[c] = tv;
      }
    }
  }
  const size_t e = (size_t)level_offset(H) * P1 + t;
#pragma unroll
  for (int c = 0; c < RC; ++c)
    if (r0 + c < nr) M[(r0 + c) * rs.m + e] = acc[c];
}

// --------------------------------------------------------------------------
// Fused upward pass.  The tree below level l0 = H - k is split into subtrees
// of 4^k leaves; one block per subtree takes the leaf moments (S2M kernel) and
// merges them level by level up to l0 with the M2M shift (Eq. metome) in
// shared memory.  When the levels above l0 are small (l0 <= kCoarseBig), the
// block that finishes last (a counter in global memory) also runs them, l0 - 1
// down to 1, so the upward pass needs no further launch; deeper trees run
// them as separate launches.
constexpr int kCoarseBig = 5;  // coarse levels with at least 4^5 boxes get a multi-block launch

// a complex number read past L1 (written by another block of the same launch)
__device__ __forceinline__ cf ldcg_c(const cf *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ cd ldcg_c(const cd *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return mk(v.x, v.y);
}

// M2M of output (box b, order n) of level l from its four children (Eq.
// metome); children read past L1 (they may come from other blocks)
template <typename R>
__device__ __forceinline__ void m2m_item(int l, int e, int P1, const cpx<R> *__restrict__ Tm2m,
                                         cpx<R> *__restrict__ M) {
  const int b = e / P1, n = e % P1;
  const cpx<R> *child = M + (size_t)(level_offset(l + 1) + 4 * (int64_t)b) * P1;
  cpx<R> acc = mk<R>(0, 0);
  for (int c = 0; c < 4; ++c) {
    const cpx<R> *Tc = Tm2m + (size_t)c * P1 * P1 + (size_t)n * P1;
    for (int m = 0; m <= n; ++m) {
      const cpx<R> v = ldcg_c(&child[(size_t)c * P1 + m]);
      cfma(acc, Tc[m], v);
    }
  }
  M[(size_t)(level_offset(l) + b) * P1 + n] = acc;
}

// Shared-memory layout of a level's moments in the fused upward pass: boxes
// grouped by parent, [b / 4][b % 4][m], with a padded group stride GS = 4 P1
// + pad chosen so that the groups of consecutive parents start in different
// shared-memory banks (GS = 1 mod 16 complex floats, 1 mod 8 complex
// doubles): the lanes of a warp, one parent each, then read their children
// without bank conflicts.
template <typename R>
__host__ __device__ __forceinline__ int m2m_group_stride(int P1) {
  const int mod = sizeof(R) == 4 ? 16 : 8;
  const int g = 4 * P1;
  return g + ((1 - g) % mod + mod) % mod;
}
template <typename R>
__host__ __device__ __forceinline__ size_t m2m_slot(int b, int m, int P1) {
  return (size_t)(b >> 2) * m2m_group_stride<R>(P1) + (size_t)(b & 3) * P1 + m;
}

// M2M in shared memory from nchild boxes of level lc (child, grouped layout,
// Morton order from box `first` << 2) up to level lto: each level's boxes
// written after the previous ones in smem (grouped layout) and to M.  Item
// (order n, parent b) with the lanes over parents, so that the lanes of a
// warp share n and the length of the sum over m; then a coalesced copy of
// the level to M.
template <typename R>
__device__ __forceinline__ void m2m_levels_smem(cpx<R> *child, int nchild, int lc, int lto,
                                                int64_t first_child, int P1,
                                                const cpx<R> *__restrict__ T,
                                                cpx<R> *__restrict__ M) {
  const int GS = m2m_group_stride<R>(P1);
  for (int l = lc - 1; l >= lto; --l) {
    cpx<R> *par = child + (size_t)((nchild + 3) >> 2) * GS;
    const int npar = nchild >> 2;
    const int64_t first = first_child >> (2 * (lc - l));
    for (int e = threadIdx.x; e < npar * P1; e += blockDim.x) {
      const int n = e / npar, b = e - n * npar;
      cpx<R> acc = mk<R>(0, 0);
      const cpx<R> *mg = child + (size_t)b * GS;  // the four children of parent b
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const cpx<R> *Tc = T + (size_t)c * P1 * P1 + (size_t)n * P1;
        const cpx<R> *mc = mg + c * P1;
        for (int m = 0; m <= n; ++m) cfma(acc, Tc[m], mc[m]);
      }
      par[m2m_slot<R>(b, n, P1)] = acc;
    }
    __syncthreads();
    const size_t o = (size_t)(level_offset(l) + first) * P1;
    for (int e = threadIdx.x; e < npar * P1; e += blockDim.x) {
      const int b = e / P1, n = e - b * P1;
      M[o + e] = par[m2m_slot<R>(b, n, P1)];
    }
    child = par;
    nchild = npar;
  }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_upward(int H, int k, int p, const cpx<R> *__restrict__ Tm2m, cpx<R> *__restrict__ M,
         RhsStride rs, int *__restrict__ ctr) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_last;
  pdl_wait();  // launched as a dependent of the S2M
  const int P1 = p + 1;
  M += blockIdx.y * rs.m;
  cpx<R> *T = reinterpret_cast<cpx<R> *>(smem_raw);  // [4][P1][P1]
  cpx<R> *Ms = T + 4 * P1 * P1;                       // subtree boxes, level by level
  for (int e = threadIdx.x; e < 4 * P1 * P1; e += blockDim.x) T[e] = Tm2m[e];
  const int nl = 1 << (2 * k);                 // leaves per subtree
  const int64_t first_leaf = (int64_t)blockIdx.x * nl;  // Morton order: subtree = contiguous
  // leaf moments (computed by the S2M kernel) into shared memory
  for (int e = threadIdx.x; e < nl * P1; e += blockDim.x) {
    const int b = e / P1, m = e - b * P1;
    Ms[m2m_slot<R>(b, m, P1)] = M[(size_t)(level_offset(H) + first_leaf) * P1 + e];
  }
  __syncthreads();
  // M2M inside the subtree: level H-1 .. H-k
  m2m_levels_smem<R>(Ms, nl, H, H - k, first_leaf, P1, T, M);
  // the coarse levels l0 - 1 .. 1, by the last block to finish, from the
  // 4^l0 moments of level l0 staged in shared memory (l0 <= k: they fit where
  // the subtree was)
  const int l0 = H - k;
  if (!ctr || l0 <= 1) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr + blockIdx.y, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nb0 = 1 << (2 * l0);
  for (int e = threadIdx.x; e < nb0 * P1; e += blockDim.x) {
    const int b = e / P1, m = e - b * P1;
    Ms[m2m_slot<R>(b, m, P1)] = ldcg_c(M + (size_t)level_offset(l0) * P1 + e);
  }
  __syncthreads();
  m2m_levels_smem<R>(Ms, nb0, l0, 1, 0, P1, T, M);
  if (threadIdx.x == 0) ctr[blockIdx.y] = 0;  // ready for the next launch
}

// M2M for the small coarse levels lhi .. 1, one block, level by level
template <typename R>
__global__ void __launch_bounds__(1024)
k_m2m_coarse(int lhi, int p, const cpx<R> *__restrict__ Tm2m, cpx<R> *__restrict__ M,
             RhsStride rs) {
  const int P1 = p + 1;
  M += blockIdx.y * rs.m;
  for (int l = lhi; l >= 1; --l) {
    const int nb = 1 << (2 * l);
    for (int e = threadIdx.x; e < nb * P1; e += blockDim.x) m2m_item<R>(l, e, P1, Tm2m, M);
    __syncthreads();
  }
}

// the same for one level with many boxes, one thread per (box, n) over many blocks
template <typename R>
__global__ void __launch_bounds__(256)
k_m2m_level(int l, int p, const cpx<R> *__restrict__ Tm2m, cpx<R> *__restrict__ M, RhsStride rs) {
  const int P1 = p + 1;
  M += blockIdx.y * rs.m;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ((int64_t)1 << (2 * l)) * P1) m2m_item<R>(l, (int)e, P1, Tm2m, M);
}

// Fused downward pass.  One block per box of level l0 = H - k (the root of a
// subtree of 4^k leaves).  The block first forms the final local expansion of
// its root from the chain of its ancestors: the level-1 expansion (mirror
// M2L only) shifted down by L2L (Eq. letole1) and added to each ancestor's own
// M2L result, level by level -- a few small matrix-vector products per block,
// instead of launches for the coarse levels.  It then pushes the expansions
// down the subtree in shared memory (child = L2L(parent) + the child's own M2L
// result).  Without EVAL the leaf expansions are written to global memory;
// with EVAL (single-precision split evaluation) they stay in shared memory and
// the block evaluates them at its points (L2P, Eq. truncatedLE), adds the
// near-field sums of k_near32 and writes the outputs.
struct DownEval {
  const float2 *loc;
  const float4 *near;
  const int64_t *perm;
  const uint64_t *keys;  // sorted Morton keys: the leaf of each point
  const DevGeom *dg;
  double *pot, *grad;
};

// the per-point inputs of the fused L2P
struct PointIn {
  uint64_t key;
  float2 loc;
  float4 near;
  int64_t perm;
};
__device__ __forceinline__ PointIn load_point(const DownEval &ev, int i) {
  PointIn r;
  r.key = __ldg(ev.keys + i);
  r.loc = __ldg(ev.loc + i);
  r.near = __ldcs(ev.near + i);  // read once
  r.perm = __ldg(ev.perm + i);
  return r;
}

// slot of box (ix, iy <= 1) of level l >= 1 in the mirror M2L's separate
// outputs: the launch's block index, levels in order, rows 0 and 1 of 2^l
// boxes each
__host__ __device__ __forceinline__ int64_t mirror_slot(int l, int ix, int iy) {
  return ((int64_t(2) << l) - 4) + ((int64_t)iy << l) + ix;
}

template <typename R, bool EVAL>
__global__ void __launch_bounds__(256)
k_downward(int H, int k, int p, const cpx<R> *__restrict__ Tl2l, cpx<R> *__restrict__ A,
           cpx<R> *__restrict__ B, RhsStride rs, const int *__restrict__ leaf_start,
           int skip_empty, DownEval ev, const cpx<R> *__restrict__ Amir,
           const cpx<R> *__restrict__ Bmir) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int P1 = p + 1;
  const int64_t root = blockIdx.x;
  const int l0 = H - k;
  const int64_t lf0 = root << (2 * k);
  const int nl = 1 << (2 * k);
  const int i0 = leaf_start[lf0], i1 = leaf_start[lf0 + nl];
  if (skip_empty && i1 == i0) return;  // a subtree without points needs no leaf expansions
  // with EVAL: the first point's data, loaded now, used after the L2L levels
  PointIn pf{};
  if constexpr (EVAL) {
    if (i0 + (int)threadIdx.x < i1) pf = load_point(ev, i0 + (int)threadIdx.x);
  }
  A += blockIdx.y * rs.m;
  B += blockIdx.y * rs.m;
  cpx<R> *T = reinterpret_cast<cpx<R> *>(smem_raw);  // [4][P1][P1]
  // two ping-pong regions of nbuf boxes x (A, B), BS = 2 P1 + 1 coefficients
  // a box (an odd number of 8-byte words for single precision, so that the
  // lanes of a warp, one box each, read different banks): the leaf level
  // stays in shared memory with EVAL, else goes straight to global memory
  const int nbuf = EVAL ? nl : (1 << (2 * (k > 0 ? k - 1 : 0)));
  const int BS = 2 * P1 + 1;
  cpx<R> *cur = T + 4 * P1 * P1, *nxt = cur + (size_t)nbuf * BS;
  for (int e = threadIdx.x; e < 4 * P1 * P1; e += blockDim.x) T[e] = Tl2l[e];
  // ancestor chain: levels 1 .. l0 (level 0 has no expansion; level 1 has
  // the mirror M2L's result only)
  const int64_t a1 = root >> (2 * (l0 - 1));
  for (int e = threadIdx.x; e < P1; e += blockDim.x) {
    if (Amir) {
      const int64_t ms = mirror_slot(1, box_ix((uint64_t)a1), box_iy((uint64_t)a1)) * P1 + e;
      cur[e] = Amir[ms];
      cur[P1 + e] = Bmir[ms];
    } else {
      cur[e] = A[(size_t)(level_offset(1) + a1) * P1 + e];
      cur[P1 + e] = B[(size_t)(level_offset(1) + a1) * P1 + e];
    }
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, part = threadIdx.x & 7;
    const unsigned gmask = 0xffu << (lane & 24);
    for (int l = 2; l <= l0; ++l) {
      const int64_t bl = root >> (2 * (l0 - l));
      const int c = (int)(bl & 3);
      const size_t ce = (size_t)(level_offset(l) + bl) * P1;
      const int iyb = box_iy((uint64_t)bl);
      const int64_t msb = (Amir && iyb <= 1) ? mirror_slot(l, box_ix((uint64_t)bl), iyb) * P1 : -1;
      // output o (A then B) by a group of 8 threads, each a strided part of
      // the sum over n, combined by shuffles within the group
      for (int o0 = 0; o0 < 2 * P1; o0 += (int)blockDim.x >> 3) {
        const int o = o0 + ((int)threadIdx.x >> 3);
        const bool act = o < 2 * P1;
        const bool isb = o >= P1;
        const int m = isb ? o - P1 : o;
        cpx<R> acc = mk<R>(0, 0);
        if (act) {
          const cpx<R> *Tc = T + (size_t)c * P1 * P1 + (size_t)m * P1;
          const cpx<R> *src = cur + (isb ? P1 : 0);
          for (int n = m + part; n < P1; n += 8) cfma(acc, isb ? conj(Tc[n]) : Tc[n], src[n]);
        }
#pragma unroll
        for (int w = 1; w < 8; w <<= 1) {
          acc.x += __shfl_xor_sync(gmask, acc.x, w);
          acc.y += __shfl_xor_sync(gmask, acc.y, w);
        }
        if (act && part == 0) {
          cpx<R> own = isb ? B[ce + m] : A[ce + m];
          if (msb >= 0) own = own + (isb ? Bmir[msb + m] : Amir[msb + m]);
          nxt[o] = acc + own;
        }
      }
      __syncthreads();
      cpx<R> *t = cur; cur = nxt; nxt = t;
    }
  }
  // the subtree, level l0 + 1 .. H
  int np = 1;
  for (int l = l0 + 1; l <= H; ++l) {
    const int nc = np * 4;
    const int64_t first = root << (2 * (l - l0));
    if (EVAL || l < H) {
      // the level's own (M2L) coefficients into nxt, read coalesced, then
      // the L2L with lanes over boxes: the lanes of a warp share the output
      // order m (and the length of the sum over n) once a level has 32 boxes
      for (int e = threadIdx.x; e < nc * P1; e += blockDim.x) {
        const int b = e / P1, m = e % P1;
        const size_t ce = (size_t)(level_offset(l) + first) * P1 + e;
        cpx<R> sa = A[ce], sb = B[ce];
        if (Amir) {
          const uint64_t bx = (uint64_t)(first + b);
          const int iyb = box_iy(bx);
          if (iyb <= 1) {
            const int64_t ms = mirror_slot(l, box_ix(bx), iyb) * P1 + m;
            sa = sa + Amir[ms];
            sb = sb + Bmir[ms];
          }
        }
        nxt[(size_t)b * BS + m] = sa;
        nxt[(size_t)b * BS + P1 + m] = sb;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nc * P1; e += blockDim.x) {
        const int m = e / nc, b = e - m * nc, c = b & 3;
        const cpx<R> *pa = cur + (size_t)(b >> 2) * BS;
        const cpx<R> *pb = pa + P1;
        const cpx<R> *Tc = T + (size_t)c * P1 * P1 + (size_t)m * P1;
        cpx<R> sa = nxt[(size_t)b * BS + m], sb = nxt[(size_t)b * BS + P1 + m];
        for (int n = m; n < P1; ++n) {
          cfma(sa, Tc[n], pa[n]);
          cfma(sb, conj(Tc[n]), pb[n]);
        }
        nxt[(size_t)b * BS + m] = sa;
        nxt[(size_t)b * BS + P1 + m] = sb;
      }
      __syncthreads();
      cpx<R> *t = cur; cur = nxt; nxt = t;
      np = nc;
      continue;
    }
    if constexpr (!EVAL) {  // the leaf level without the L2P: into A, B
      for (int e = threadIdx.x; e < nc * P1; e += blockDim.x) {
        const int b = e / P1, m = e % P1, c = b & 3;
        const cpx<R> *pa = cur + (size_t)(b >> 2) * BS;
        const cpx<R> *pb = pa + P1;
        const cpx<R> *Tc = T + (size_t)c * P1 * P1 + (size_t)m * P1;
        const size_t ce = (size_t)(level_offset(l) + first + b) * P1 + m;
        cpx<R> sa = A[ce], sb = B[ce];
        if (Amir) {
          const uint64_t bx = (uint64_t)(first + b);
          const int iyb = box_iy(bx);
          if (iyb <= 1) {
            const int64_t ms = mirror_slot(l, box_ix(bx), iyb) * P1 + m;
            sa = sa + Amir[ms];
            sb = sb + Bmir[ms];
          }
        }
        for (int n = m; n < P1; ++n) {
          cfma(sa, Tc[n], pa[n]);
          cfma(sb, conj(Tc[n]), pb[n]);
        }
        A[ce] = sa;
        B[ce] = sb;
      }
      __syncthreads();
      cpx<R> *t = cur; cur = nxt; nxt = t;
      np = nc;
    }
  }
  if constexpr (EVAL) {
    // L2P at the subtree's points (contiguous in tree order), plus the near
    // sums; cur holds the leaf expansions (when k = 0, the root's)
    const float invd = ev.dg->invd[H];
    const float c4 = (float)(0.69314718055994530942 / (4.0 * HP_PI));
    const float i2pi = (float)(1.0 / HP_TWO_PI);
    const int ksh = 60 - 2 * H;
    // the point data of iteration i + blockDim.x is loaded while iteration i
    // computes (the first iteration's since the kernel's start)
    PointIn nx = pf;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const PointIn cu = nx;
      if (i + (int)blockDim.x < i1) nx = load_point(ev, i + (int)blockDim.x);
      const int lo = (int)((int64_t)(cu.key >> ksh) - lf0);  // the point's leaf in the subtree
      const cf *Al = reinterpret_cast<const cf *>(cur) + (size_t)lo * BS;
      const cf *Bl = Al + P1;
      const float2 me = cu.loc;
      const float4 nv = cu.near;
      const cf w = mk(me.x * invd, me.y * invd), wb = conj(w);
      cf va = Al[p], da = mk(0.f, 0.f), vb = Bl[p], db = mk(0.f, 0.f);
      for (int n = p - 1; n >= 0; --n) {
        da = da * w + va;
        va = va * w + Al[n];
        db = db * wb + vb;
        vb = vb * wb + Bl[n];
      }
      const float ur_ = va.x + vb.x - nv.x * c4;
      const float ui_ = va.y + vb.y;
      const cf gxo = invd * (da + db) + mk(-nv.y * i2pi, 0.f);
      const cf gyo = invd * (mul_i(da) - mul_i(db)) + mk(-nv.z * i2pi, 0.f);
      const int64_t o = cu.perm;
      double2 pv = make_double2(f2d(ur_), f2d(ui_));
      double4_16a gv;
      gv.x = f2d(gxo.x); gv.y = f2d(gxo.y); gv.z = f2d(gyo.x); gv.w = f2d(gyo.y);
      if (box_iy((uint64_t)(lf0 + lo)) == 0) {  // bottom row: image/reaction sums already there
        const double2 pm = reinterpret_cast<const double2 *>(ev.pot)[o];
        pv.x += pm.x;
        pv.y += pm.y;
        if (ev.grad) {
          const double4_16a gm = reinterpret_cast<const double4_16a *>(ev.grad)[o];
          gv.x += gm.x; gv.y += gm.y; gv.z += gm.z; gv.w += gm.w;
        }
      }
      reinterpret_cast<double2 *>(ev.pot)[o] = pv;
      if (ev.grad) reinterpret_cast<double4_16a *>(ev.grad)[o] = gv;
    }
  }
}

constexpr size_t kFusedSmem = 200 * 1024;

template <typename R>
size_t upward_smem(int p, int k) {
  const int P1 = p + 1;
  size_t ng = 0;  // parent groups of the levels (a single root box: one group)
  for (int j = 0; j <= k; ++j) ng += (size_t(1) << (2 * j) >> 2) > 0 ? (size_t(1) << (2 * j)) >> 2 : 1;
  return sizeof(cpx<R>) * (4 * (size_t)P1 * P1 + ng * m2m_group_stride<R>(P1));
}
template <typename R>
size_t downward_smem(int p, int k, bool eval) {
  const size_t P1 = p + 1;
  const size_t nbuf = eval ? (size_t(1) << (2 * k)) : (size_t(1) << (2 * (k > 0 ? k - 1 : 0)));
  return sizeof(cpx<R>) * (4 * P1 * P1 + 2 * nbuf * (2 * P1 + 1));
}

// --------------------------------------------------------------------------
// free-space M2L over the V-list.  Block = 32 target boxes of one child type
// (ix & 1, iy & 1), so that all of them share the same 27 source offsets;
// for each offset the (p+1)^2 translation matrix is staged in shared memory
// and applied to the 32 gathered source vectors (a small complex GEMM).
// Warp g accumulates the coefficients l = g, g + 4, g + 8, ... of its lane's
// target.
constexpr int kM2LMaxRows = (HPFMM_MAX_P + 1 + 3) / 4;

template <typename R>
__global__ void __launch_bounds__(128)
k_m2l_free(int l, int p, const DevGeom *__restrict__ dg, const cpx<R> *__restrict__ Tfree,
           const cd *__restrict__ logt, const cpx<R> *__restrict__ M, cpx<R> *__restrict__ A,
           cpx<R> *__restrict__ B) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int P1 = p + 1;
  cpx<R> *Ts = reinterpret_cast<cpx<R> *>(smem_raw);
  cpx<R> *Ms = Ts + P1 * P1;  // [k][33]
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int type = blockIdx.y;
  int a = type & 1, b = type >> 1;
  int64_t nparent = int64_t(1) << (2 * (l - 1));
  int64_t j = (int64_t)blockIdx.x * 32 + lane;
  bool valid = j < nparent;
  int64_t m = 4 * j + type;
  int ix = valid ? box_ix(m) : 0, iy = valid ? box_iy(m) : 0;
  int side_n = 1 << l;
  cpx<R> acc[kM2LMaxRows];
#pragma unroll
  for (int r = 0; r < kM2LMaxRows; ++r) acc[r] = mk<R>(0, 0);
  const int64_t off = level_offset(l);

  for (int dy = -2 - b; dy <= 3 - b; ++dy) {
    for (int dx = -2 - a; dx <= 3 - a; ++dx) {
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
      int cls = (dy + 3) * 7 + (dx + 3);
      __syncthreads();
      const cpx<R> *Tc = Tfree + (size_t)cls * P1 * P1;
      for (int e = threadIdx.x; e < P1 * P1; e += blockDim.x) Ts[e] = Tc[e];
      for (int e = threadIdx.x; e < 32 * P1; e += blockDim.x) {
        int t = e / P1, k = e % P1;
        int64_t jt = (int64_t)blockIdx.x * 32 + t;
        cpx<R> v = mk<R>(0, 0);
        if (jt < nparent) {
          int64_t mt = 4 * jt + type;
          int sx = box_ix(mt) + dx, sy = box_iy(mt) + dy;
          if (sx >= 0 && sy >= 0 && sx < side_n && sy < side_n)
            v = M[(size_t)(off + box_morton(sx, sy)) * P1 + k];
        }
        Ms[k * 33 + t] = v;
      }
      __syncthreads();
      for (int k = 0; k < P1; ++k) {
        cpx<R> mv = Ms[k * 33 + lane];
#pragma unroll
        for (int r = 0; r < kM2LMaxRows; ++r) {
          int row = warp + 4 * r;
          if (row < P1) cfma(acc[r], Ts[row * P1 + k], mv);
        }
      }
      if (warp == 0) {  // M_0 log(t d) term of L_0; only Re L_0 reaches the
                        // potential, so the arg part (large at coarse levels,
                        // cancelling between A and B) is left out
        cd lt = logt[cls];
        R m0 = Ms[lane].x;  // M_0 is real for real charges
        acc[0].x += m0 * (R)(lt.x + dg->logd[l]);
      }
    }
  }
  if (!valid) return;
  // L = -(1/2pi) sum ...; A = L/2, B = conj(L)/2
  const R s = (R)(-0.5 / HP_TWO_PI);
  cpx<R> *Ao = A + (size_t)(off + m) * P1;
  cpx<R> *Bo = B + (size_t)(off + m) * P1;
#pragma unroll
  for (int r = 0; r < kM2LMaxRows; ++r) {
    int row = warp + 4 * r;
    if (row < P1) {
      cpx<R> v = s * acc[r];
      Ao[row] = v;
      Bo[row] = conj(v);
    }
  }
  (void)iy;
  (void)ix;
}

// --------------------------------------------------------------------------
// The patch form of the free-space M2L (m2l_patch.cuh) is instantiated for
// every order in two translation units; this dispatches on p.
template <typename R>
bool launch_m2l_patch(int p, int H, int lmin, int lmax, const DevGeom *dg, const cpx<R> *Tpad,
                      const cd *logt, const cpx<R> *M, cpx<R> *A, cpx<R> *B, int *status,
                      cudaStream_t st, int nr, RhsStride rs, const int *leaf_start,
                      int skip_empty) {
  if constexpr (sizeof(R) == 8) {
    return m2l_patch_launch_64(p, H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st, nr, rs,
                               leaf_start, skip_empty);
  } else {
    if (p <= kPatchSplitP)
      return m2l_patch_launch_lo(p, H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st, nr, rs,
                                 leaf_start, skip_empty);
    return m2l_patch_launch_hi(p, H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st, nr, rs,
                               leaf_start, skip_empty);
  }
}

// --------------------------------------------------------------------------
// Free-space M2L for many charge vectors on the tensor cores (single
// precision path).  With R charge vectors the translations of one level are
// a batch of small dense products that share their matrices: for a V-list
// offset class delta, L_t[r] += T_delta M_{t + delta}[r] for every target t of
// one child type and every RHS r.  In real form (K = 2(p+1) inputs Re M, Im M;
// 2(p+1) outputs Re L, Im L) one CTA computes a tile of 128 rows -- G target
// boxes of one child type x 128/G RHS -- as D = sum_delta A_delta B_delta^T
// with tcgen05 kind::tf32 MMAs accumulating in tensor memory, where A_delta
// holds the source moments of the tile's rows and B_delta the real form of
// T_delta (plus the level's M_0 ln|t d| term on Re L_0).  Operands are split
// into tf32 hi + lo parts and multiplied as hi*hi + hi*lo + lo*hi, which keeps
// about 21 bits -- the accuracy of the FP32 FMA kernel.  The 27 classes of the
// child type are taken one after the other: stage A and B in shared memory
// (all threads), one thread issues the MMAs and commits them to an mbarrier,
// every thread waits (bounded) before the buffers are reused.
template <int P1>
__global__ void __launch_bounds__(128)
k_m2l_free_tc(int l, int rct, int nr, const DevGeom *__restrict__ dg,
              const float *__restrict__ Btab,
              const cd *__restrict__ logt, const cf *__restrict__ M, cf *__restrict__ A,
              cf *__restrict__ B, RhsStride rs, int *__restrict__ status) {
  constexpr int KP = tc_kp(P1), NP = tc_np(P1);
  constexpr unsigned NCOL = NP <= 32 ? 32u : (NP <= 64 ? 64u : 128u);
  constexpr int ASZ = 128 * KP, BSZ = NP * KP;  // floats per operand half
  constexpr unsigned BBYTES = 2u * BSZ * sizeof(float);
  extern __shared__ __align__(1024) float tsm[];
  // [2 buffers] x (A hi, A lo), then [2 buffers] x (B hi, B lo)
  float *abuf = tsm, *bbuf = tsm + 4 * ASZ;
  __shared__ __align__(8) uint64_t mbar[2], tbar[2];
  __shared__ unsigned tslot;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5;
  const float logd = (float)dg->logd[l];
  const int G = 128 / rct;
  const int type = blockIdx.x & 3, grp = blockIdx.x >> 2;
  const int a = type & 1, bb = type >> 1;
  const int r0 = blockIdx.y * rct;
  const int nside = 1 << l, npar = 1 << (2 * (l - 1));
  const int64_t off = level_offset(l);
  const int g = tid / rct, rr = tid % rct;
  const int pm = grp * G + g;
  const bool rvalid = pm < npar && r0 + rr < nr;
  const int tx = pm < npar ? 2 * box_ix(pm) + a : 0, ty = pm < npar ? 2 * box_iy(pm) + bb : 0;
  const cf *Mr = M + (size_t)(r0 + rr) * rs.m;
  __shared__ int cls[27];  // the 27 classes of this child type, in a fixed order
  if (warp == 0) tc_alloc(&tslot, NCOL);
  if (tid == 0) {
    int ncls = 0;
    for (int dy = -2 - bb; dy <= 3 - bb; ++dy)
      for (int dx = -2 - a; dx <= 3 - a; ++dx)
        if (!(dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1)) cls[ncls++] = (dy + 3) * 7 + (dx + 3);
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&tbar[0], 1);
    mbar_init(&tbar[1], 1);
    failed = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = tslot;
  const uint32_t idesc = tc_idesc_tf32(128, NP);
  const unsigned sbo = (unsigned)(KP / 4) * 128u;
  float lgacc = 0.f;  // sum over classes of Re M_0 ln|t d| (added to Re L_0)
  // operand staging of class index it into buffer it & 1: B by one bulk copy,
  // A by every thread (its row: the source moments in real form, split)
  auto stage = [&](int it) {
    const int buf = it & 1, c = cls[it];
    if (tid == 0) {
      mbar_expect_tx(&tbar[buf], BBYTES);
      bulk_g2s(bbuf + buf * 2 * BSZ, Btab + (size_t)c_slot[c] * 2 * BSZ, BBYTES, &tbar[buf]);
    }
    const int dx = c % 7 - 3, dy = c / 7 - 3;
    const int sx = tx + dx, sy = ty + dy;
    const bool ok = rvalid && sx >= 0 && sy >= 0 && sx < nside && sy < nside;
    float v[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) v[k] = 0.f;
    if (ok) {
      const cf *src = Mr + (size_t)(off + box_morton(sx, sy)) * P1;
#pragma unroll
      for (int m = 0; m < P1; ++m) {
        const cf z = src[m];
        v[m] = z.x;
        v[P1 + m] = z.y;
      }
      lgacc = fmaf(v[0], (float)logt[c].x + logd, lgacc);
    }
    float *ah = abuf + buf * 2 * ASZ, *al = ah + ASZ;
#pragma unroll
    for (int kg = 0; kg < KP / 4; ++kg) {
      float4 h, lo;
      tc_split(v[4 * kg], h.x, lo.x);
      tc_split(v[4 * kg + 1], h.y, lo.y);
      tc_split(v[4 * kg + 2], h.z, lo.z);
      tc_split(v[4 * kg + 3], h.w, lo.w);
      const int o = tc_off(tid, 4 * kg, KP);
      *reinterpret_cast<float4 *>(ah + o) = h;
      *reinterpret_cast<float4 *>(al + o) = lo;
    }
  };
  stage(0);
  for (int it = 0; it < 27; ++it) {
    const int buf = it & 1;
    tc_fence_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      if (!mbar_wait_bounded(&tbar[buf], (unsigned)((it >> 1) & 1))) {
        failed = 1;
      } else {
        const float *ah = abuf + buf * 2 * ASZ, *al = ah + ASZ;
        const float *bh = bbuf + buf * 2 * BSZ, *bl = bh + BSZ;
#pragma unroll 1
        for (int s = 0; s < KP / 8; ++s) {
          const unsigned o = (unsigned)s * 256u;
          const uint64_t dah = tc_sdesc(smem_u32(ah) + o, 128u, sbo);
          const uint64_t dal = tc_sdesc(smem_u32(al) + o, 128u, sbo);
          const uint64_t dbh = tc_sdesc(smem_u32(bh) + o, 128u, sbo);
          const uint64_t dbl = tc_sdesc(smem_u32(bl) + o, 128u, sbo);
          tc_mma_tf32(tbase, dah, dbh, idesc, it > 0 || s > 0);
          tc_mma_tf32(tbase, dah, dbl, idesc, true);
          tc_mma_tf32(tbase, dal, dbh, idesc, true);
        }
        tc_commit(&mbar[buf]);
      }
    }
    __syncthreads();
    if (failed) break;
    if (it + 1 < 27) {
      // the other buffer was read by the MMAs of class it - 1: wait for them
      if (it >= 1 && !mbar_wait_bounded(&mbar[buf ^ 1], (unsigned)(((it - 1) >> 1) & 1)))
        failed = 1;
      __syncthreads();
      if (failed) break;
      stage(it + 1);
    }
  }
  // completion of the last class's MMAs (class 26 used buffer 0)
  bool done = !failed && mbar_wait_bounded(&mbar[0], (unsigned)((26 >> 1) & 1));
  if (!done && tid == 0) atomicOr(status, HPFMM_DEV_TIMEOUT);
  tc_fence_after();
  if (done) {
    // epilogue: row tid of D -> L_n = D[n] + i D[P1 + n] (+ the log term on
    // Re L_0); A = s L, B = conj(s L)
    float d[NP];
#pragma unroll
    for (int cc = 0; cc < NP; cc += 8)
      tc_ld8(tbase + ((unsigned)(32 * warp) << 16) + (unsigned)cc, d + cc);
    if (rvalid) {
      const float sc = (float)(-0.5 / HP_TWO_PI);
      const size_t e0 = (size_t)(r0 + rr) * rs.m + (size_t)(off + box_morton(tx, ty)) * P1;
      d[0] += lgacc;
#pragma unroll
      for (int n = 0; n < P1; ++n) {
        const cf v = mk(sc * d[n], sc * d[P1 + n]);
        A[e0 + n] = v;
        B[e0 + n] = conj(v);
      }
    }
  } else {
    // make sure nothing is still writing TMEM or reading the buffers
    mbar_wait_bounded(&mbar[0], (unsigned)((26 >> 1) & 1));
    mbar_wait_bounded(&mbar[1], (unsigned)((25 >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tbase, NCOL);
}

template <int P1>
size_t m2l_tc_smem() {
  return sizeof(float) * 4 * (size_t)(128 + tc_np(P1)) * tc_kp(P1);
}

// RHS per tile row group: 16, 32 or 64
int m2l_tc_rct(int nr) { return nr > 32 ? 64 : (nr > 16 ? 32 : 16); }

// launches the tensor-core M2L for levels 2..H; false if p has no instance
bool launch_m2l_tc(int p, int H, const DevGeom *dg, const float *Btab, const cd *logt,
                   const cf *M, cf *A, cf *B, int *status, cudaStream_t st, int nr,
                   RhsStride rs) {
  if (!Btab) return false;
  static std::mutex mu;
  static signed char attr[64][41];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || p < 0 || p > 40) return false;
  const int rct = m2l_tc_rct(nr);
  const int G = 128 / rct;
  const unsigned ny = (unsigned)((nr + rct - 1) / rct);
#define HP_TC_CASE(PP)                                                                      \
  case PP: {                                                                                \
    const size_t sm = m2l_tc_smem<PP + 1>();                                                \
    {                                                                                       \
      std::lock_guard<std::mutex> lock(mu);                                                 \
      if (attr[dev][p] == 0) {                                                              \
        bool ok = cudaFuncSetAttribute(k_m2l_free_tc<PP + 1>,                               \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                       (int)sm) == cudaSuccess;                             \
        if (!ok) cudaGetLastError();                                                        \
        attr[dev][p] = ok ? 1 : -1;                                                         \
      }                                                                                     \
      if (attr[dev][p] < 0) return false;                                                   \
    }                                                                                       \
    for (int l = 2; l <= H; ++l) {                                                          \
      const int npar = 1 << (2 * (l - 1));                                                  \
      const unsigned nx = (unsigned)(4 * ((npar + G - 1) / G));                             \
      k_m2l_free_tc<PP + 1><<<dim3(nx, ny), 128, sm, st>>>(l, rct, nr, dg,                  \
                                                           Btab, logt, M, A, B, rs, status); \
    }                                                                                       \
    return true;                                                                            \
  }
  switch (p) {
    HP_TC_CASE(4) HP_TC_CASE(6) HP_TC_CASE(8) HP_TC_CASE(10) HP_TC_CASE(12)
    HP_TC_CASE(14) HP_TC_CASE(16) HP_TC_CASE(18) HP_TC_CASE(20)
    default: return false;
  }
#undef HP_TC_CASE
}

// All-levels form of the mirror M2L: one block of 4 warps per target box of
// rows 0 and 1 of every level 1..H; the warps split the (at most 12) sources
// of the mirror list, lanes run over the output index, and the four partial
// sums are reduced in shared memory.  Without Amir / Bmir, level 1
// initialises A and B and deeper levels add to the free-space result; with
// them, the results go there instead (box t of the launch at t (p+1), see
// mirror_slot), so that this kernel need not wait for the free-space M2L.
template <typename R>
__global__ void __launch_bounds__(128)
k_m2l_mirror_all(int H, int p, const DevGeom *__restrict__ dg, const cpx<R> *__restrict__ Timg,
                 const cd *__restrict__ logimg, const cpx<R> *__restrict__ Treact,
                 const cpx<R> *__restrict__ M, cpx<R> *__restrict__ A, cpx<R> *__restrict__ B,
                 RhsStride rs, cpx<R> *__restrict__ Amir, cpx<R> *__restrict__ Bmir) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int P1 = p + 1;
  M += blockIdx.y * rs.m;
  A += blockIdx.y * rs.m;
  B += blockIdx.y * rs.m;
  cpx<R> *red = reinterpret_cast<cpx<R> *>(smem_raw);  // [4 warps][3][P1]
  cpx<R> *msh = red + 4 * 3 * P1;                      // [4 warps][P1]
  int t = blockIdx.x, l = 1;
  for (; l <= H; ++l) {
    if (t < (2 << l)) break;
    t -= 2 << l;
  }
  const int nx = 1 << l;
  const int ixt = t % nx, iyt = t / nx, px = ixt >> 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t off = level_offset(l);
  const R logd = (R)dg->logd[l];
  cpx<R> *ms = msh + warp * P1;
  cpx<R> aL[2], aC[2], aD[2];
  for (int r = 0; r < 2; ++r) aL[r] = aC[r] = aD[r] = mk<R>(0, 0);
  // enumerate the mirror list; source number j goes to warp j % 4
  int j = 0;
  for (int iys = 0; iys <= 1; ++iys) {
    for (int ixs = 2 * (px - 1); ixs <= 2 * (px + 1) + 1; ++ixs) {
      if (ixs < 0 || ixs >= nx) continue;
      if (iyt == 0 && iys == 0 && abs(ixs - ixt) <= 1) continue;
      if ((j++ & 3) != warp) continue;
      const int dx = ixs - ixt, ysum = iyt + iys + 1;
      const int cls = (ysum - 1) * 7 + (dx + 3);
      const cpx<R> *src = M + (size_t)(off + box_morton(ixs, iys)) * P1;
      __syncwarp();
      for (int k = lane; k < P1; k += 32) ms[k] = src[k];
      __syncwarp();
      const cpx<R> *Ti = Timg + (size_t)cls * P1 * P1;
      const cpx<R> *Tp = Treact + ((size_t)((l - 1) * 21 + cls) * 2 + 0) * P1 * P1;
      const cpx<R> *Tm = Tp + (size_t)P1 * P1;
      int r = 0;
      for (int n = lane; n < P1; n += 32, ++r) {
        cpx<R> sL = mk<R>(0, 0), sC = mk<R>(0, 0), sD = mk<R>(0, 0);
        for (int k = 0; k < P1; ++k) {
          cpx<R> mv = ms[k], mc = conj(mv);
          cfma(sL, Ti[n * P1 + k], mc);
          cfma(sC, Tp[n * P1 + k], mc);
          cfma(sD, Tm[n * P1 + k], mv);
        }
        if (n == 0) sL.x += ms[0].x * ((R)logimg[cls].x + logd);  // M_0 ln|t d|
        aL[r] = aL[r] + sL;
        aC[r] = aC[r] + sC;
        aD[r] = aD[r] + sD;
      }
    }
  }
  int r = 0;
  for (int n = lane; n < P1; n += 32, ++r) {
    red[(warp * 3 + 0) * P1 + n] = aL[r];
    red[(warp * 3 + 1) * P1 + n] = aC[r];
    red[(warp * 3 + 2) * P1 + n] = aD[r];
  }
  __syncthreads();
  const R sc = (R)(0.5 / HP_TWO_PI);
  const int64_t m = off + box_morton(ixt, iyt);
  for (int n = threadIdx.x; n < P1; n += blockDim.x) {
    cpx<R> L = mk<R>(0, 0), C = mk<R>(0, 0), D = mk<R>(0, 0);
    for (int w = 0; w < 4; ++w) {
      L = L + red[(w * 3 + 0) * P1 + n];
      C = C + red[(w * 3 + 1) * P1 + n];
      D = D + red[(w * 3 + 2) * P1 + n];
    }
    L = sc * L;
    const cpx<R> va = L + C, vb = conj(L) + D;
    if (Amir) {
      Amir[(size_t)blockIdx.x * P1 + n] = va;
      Bmir[(size_t)blockIdx.x * P1 + n] = vb;
      continue;
    }
    const size_t e = (size_t)m * P1 + n;
    if (l >= 2) {
      A[e] = A[e] + va;
      B[e] = B[e] + vb;
    } else {
      A[e] = va;
      B[e] = vb;
    }
  }
}

// --------------------------------------------------------------------------
// Leaf evaluation: L2P of A and B (Eq. truncatedLE) plus the near field
// (free part over the 3x3 neighbourhood, image and reaction parts over the
// bottom-row neighbours), written in the caller's order.
// One warp per leaf, lanes over 32 targets at a time; source points staged
// per warp in shared memory.
struct SrcPt64 { double x, y, q; };

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_eval64(const double *__restrict__ xs, const double *__restrict__ ys,
         const double *__restrict__ qs, const int64_t *__restrict__ perm,
         const int *__restrict__ leaf_start, int H, const DevGeom *__restrict__ dg, int p,
         cd kappa, const cd *__restrict__ A, const cd *__restrict__ B, double *__restrict__ pot,
         double *__restrict__ grad) {
  __shared__ SrcPt64 sp[kWarpsPerBlock][32];
  const double x0 = dg->x0, side = dg->side;
  int P1 = p + 1;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int leaf = blockIdx.x * kWarpsPerBlock + warp;
  int nx = 1 << H;
  if (leaf >= nx * nx) return;
  int ix = box_ix(leaf), iy = box_iy(leaf);
  double d = side / (double)nx;
  double cx = x0 + (ix + 0.5) * d, cy = (iy + 0.5) * d;
  const cd *Al = A + (size_t)(level_offset(H) + leaf) * P1;
  const cd *Bl = B + (size_t)(level_offset(H) + leaf) * P1;
  int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
  for (int tb = b0; tb < b1; tb += 32) {
    int i = tb + lane;
    bool act = i < b1;
    double x = act ? xs[i] : cx, y = act ? ys[i] : cy;
    // L2P: Horner for the value and the derivative in w and conj(w)
    cd w = mk((x - cx) / d, (y - cy) / d), wb = conj(w);
    cd va = Al[p], da = mk(0.0, 0.0), vb = Bl[p], db = mk(0.0, 0.0);
    for (int n = p - 1; n >= 0; --n) {
      da = da * w + va;
      va = va * w + Al[n];
      db = db * wb + vb;
      vb = vb * wb + Bl[n];
    }
    cd u = va + vb;
    cd gx = (1.0 / d) * (da + db);
    cd gy = (1.0 / d) * (mul_i(da) - mul_i(db));
    PairAcc<double> acc;
    for (int ny = iy - 1; ny <= iy + 1; ++ny) {
      if (ny < 0 || ny >= nx) continue;
      for (int mxx = ix - 1; mxx <= ix + 1; ++mxx) {
        if (mxx < 0 || mxx >= nx) continue;
        uint64_t sl = box_morton(mxx, ny);
        int s0 = leaf_start[sl], s1 = leaf_start[sl + 1];
        bool mirror = (iy == 0 && ny == 0);
        for (int sb = s0; sb < s1; sb += 32) {
          __syncwarp();
          int js = sb + lane;
          if (js < s1) sp[warp][lane] = SrcPt64{xs[js], ys[js], qs[js]};
          __syncwarp();
          int cnt = min(32, s1 - sb);
          if (!act) continue;
          for (int k = 0; k < cnt; ++k) {
            SrcPt64 s = sp[warp][k];
            double dx = x - s.x;
            if (sb + k != i) pair_free(acc, dx, y - s.y, s.q);
            if (mirror) {
              double Y = y + s.y;
              pair_image(acc, dx, Y, s.q);
              pair_reaction_d(acc, dx, Y, s.q, kappa);
            }
          }
        }
      }
    }
    if (!act) continue;
    cd un, gxn, gyn;
    acc.finish(un, gxn, gyn);
    u = u + un;
    gx = gx + gxn;
    gy = gy + gyn;
    int64_t o = perm[i];
    pot[2 * o] = u.x;
    pot[2 * o + 1] = u.y;
    if (grad) {
      grad[4 * o + 0] = gx.x;
      grad[4 * o + 1] = gx.y;
      grad[4 * o + 2] = gy.x;
      grad[4 * o + 3] = gy.y;
    }
  }
}

// Single-precision leaf evaluation.  Coordinates are relative to the leaf
// centre (exact leaf offsets are added per source leaf), so that the pair
// differences keep full relative precision.  log via the SFU log2, the
// reaction pairs by the single-precision series when |P| <= 1 and the double
// routine otherwise (and always below tau_fp64 in MIXED mode).
struct SrcPt32 { float x, y, q, pad; };

// Single-precision leaf evaluation, lane-grouped.  A warp owns one target
// leaf.  Its targets are spread over groups of gs = 32, 16, 8 or 4 lanes
// (the smallest power of two >= the leaf size, at least 4): each group holds
// all the targets of the current chunk, the 32/gs groups take interleaved
// source subsets, and the partial sums are combined by shuffles.  Sources of
// the 3x3 neighbourhood are staged in per-warp shared memory in batches,
// with coordinates already shifted to the target leaf's frame.  The free part
// skips coincident positions (r^2 = 0), i.e. the j = i pair.
constexpr int kEvWarps = 8;

__device__ __forceinline__ void mirror_batch(const float4 *buf, int cnt, int g, int ng, float mx,
                                             float my, cf kap, const KappaLog &K, float tau,
                                             NearAcc &a) {
  for (int k = g; k < cnt; k += ng) mirror_pair(buf[k], mx, my, kap, K, tau, a);
}

__device__ __forceinline__ float xsum(float v, int from) {
#pragma unroll 1
  for (int o = from; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// tile geometry of the single-precision leaf kernel
constexpr int kTl = 4;             // target leaves per tile side
constexpr int kTlP = kTl + 2;      // patch leaves per side
constexpr int kTlCap = 2560;       // staged points per block
constexpr int kLsBytes = 80;       // tile leaf starts (kTl^2 + 1 ints), 16-byte padded

// Single-precision free-space near field (the j != i sum of Eq. 1.2 over the
// 3 x 3 leaf neighbourhood of each target), one target per lane.  A block
// takes a 4 x 4 tile of leaves -- 16 consecutive Morton leaves, so its
// targets are one contiguous range of the sorted points -- and stages the
// 6 x 6 leaves around it in shared memory, row by row: each point's position
// in the frame of the tile's first leaf as a float pair (hi, lo), converted
// once from its leaf frame by an exact two-sum with the leaf's offset (a
// multiple of the leaf side, itself split into hi + lo), and its charge.  A
// row of a target's neighbourhood is then one contiguous range of the staged
// points, and a pair difference (x_i - x_j) = (hi_i - hi_j) + (lo_i - lo_j)
// is exact up to its one rounding: without the lo parts the float frames
// would cost close pairs their relative precision (an absolute error of
// about 2^-25 d in every difference).  The target's own point is skipped by
// index.  Lanes of one warp may belong to two or three leaves: they run the
// same loops with their own bounds.  Patches larger than the buffer read
// from global memory, leaf by leaf in leaf frames.
// the free-space pairs of one target (tile-frame position mh + ml, as (x, y)
// pairs) with the staged sources lo .. hi - 1: lf += q log2 r^2 and
// g += q (dx, dy) / r^2, the differences formed as (hi - hi) + (lo - lo)
__device__ __forceinline__ void pair_loop(const float4 *__restrict__ src,
                                          const float *__restrict__ srcq, int lo, int hi,
                                          f2p mh, f2p ml, float &lf, f2p &g) {
#pragma unroll 4
  for (int k = lo; k < hi; ++k) {
    const float4 s = src[k];
    const float q = srcq[k];
    const f2p d = f2_add(f2_sub(mh, f2_pack(s.x, s.y)), f2_sub(ml, f2_pack(s.z, s.w)));
    float dx, dy;
    f2_unpack(d, dx, dy);
    const float r2 = fmaf(dx, dx, dy * dy);
    const float qi = q * fast_rcp(r2);
    lf = fmaf(q, fast_lg2(r2), lf);
    g = f2_fma(f2_pack(qi, qi), d, g);
  }
}

// the same over a range holding the target itself: the pair with r^2 = 0
// (the target, or a distinct point at the same position) contributes nothing
// (the free part excludes j = i and coincident points), one loop instead of
// two around the target's own index, so that the lanes of a warp -- whose
// targets sit at different positions in the range -- run one trip count
__device__ __forceinline__ void pair_loop_self(const float4 *__restrict__ src,
                                               const float *__restrict__ srcq, int lo, int hi,
                                               f2p mh, f2p ml, float &lf, f2p &g) {
#pragma unroll 4
  for (int k = lo; k < hi; ++k) {
    const float4 s = src[k];
    const f2p d = f2_add(f2_sub(mh, f2_pack(s.x, s.y)), f2_sub(ml, f2_pack(s.z, s.w)));
    float dx, dy;
    f2_unpack(d, dx, dy);
    const float r2 = fmaf(dx, dx, dy * dy);
    const bool ok = r2 > 0.f;
    const float q = ok ? srcq[k] : 0.f;
    const float rr = ok ? r2 : 1.f;
    const float qi = q * fast_rcp(rr);
    lf = fmaf(q, fast_lg2(rr), lf);
    g = f2_fma(f2_pack(qi, qi), d, g);
  }
}

// the target (hi, lo) shifted by -c leaf sides, as hi + lo: |c d| >= |hi|
// for c != 0, so the fast two-sum is exact (c = 0 leaves it unchanged)
__device__ __forceinline__ void frame_shift(float hi, float lo, int c, float d, float dlo,
                                            float &sh, float &sl) {
  const float b = -(float)c * d;
  sh = b + hi;
  sl = (hi - (sh - b)) + (lo - (float)c * dlo);
}

// (h, l) + (oh, ol) as hi + lo: the two-sum of h and oh (exact for any
// magnitudes), the low parts added
__device__ __forceinline__ void add_hilo(float h, float l, float oh, float ol, float &sh,
                                         float &sl) {
  sh = h + oh;
  const float bv = sh - h;
  const float e = (h - (sh - bv)) + (oh - bv);
  sl = (l + ol) + e;
}

__global__ void __launch_bounds__(kEvWarps * 32, 4)
k_near32(const float2 *__restrict__ loc, const float2 *__restrict__ loclo,
         const double *__restrict__ q, const int64_t *__restrict__ perm,
         const int *__restrict__ leaf_start, int H, const DevGeom *__restrict__ dg,
         float4 *__restrict__ near) {
  // launched as a dependent of the tree build's last kernel; the charges are
  // read in the caller's order through perm and rounded as the charge gather
  // rounds them (bit-identical to the gathered copy), so that the gather runs
  // beside this kernel instead of before it
  pdl_wait();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int *ls = reinterpret_cast<int *>(smem_raw);         // [kTl^2 + 1] tile leaf starts
  float4 *src = reinterpret_cast<float4 *>(smem_raw + kLsBytes);  // [kTlCap] (hi, lo)
  float *srcq = reinterpret_cast<float *>(src + kTlCap);          // [kTlCap] charges
  int *pst = reinterpret_cast<int *>(srcq + kTlCap);   // [kTlP^2 + 1]
  int *pbeg = pst + kTlP * kTlP + 1;                   // [kTlP^2]
  __shared__ float offh[kTlP], offl[kTlP];             // (c - 1) d as hi + lo, c = 0..5
  const float d = dg->d[H], dlo = dg->dlo[H];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = 1 << H;
  const int tps = nx >= kTl ? nx / kTl : 1;
  const int tx0 = (blockIdx.x % tps) * kTl, ty0 = (blockIdx.x / tps) * kTl;
  const int side = nx < kTl ? nx : kTl, nlt = side * side;
  const uint64_t L0 = box_morton(tx0, ty0);
  if (warp == 0) {
    int c0 = 0, c1 = 0;
    for (int h = 0; h < 2; ++h) {
      const int pi = lane + 32 * h;
      if (pi < kTlP * kTlP) {
        const int lx = tx0 - 1 + pi % kTlP, ly = ty0 - 1 + pi / kTlP;
        int b0 = 0, cnt = 0;
        if (lx >= 0 && ly >= 0 && lx < nx && ly < nx) {
          const uint64_t lf = box_morton(lx, ly);
          b0 = leaf_start[lf];
          cnt = leaf_start[lf + 1] - b0;
        }
        pbeg[pi] = b0;
        if (h == 0) c0 = cnt; else c1 = cnt;
      }
    }
    int i0 = c0, i1 = c1;
    for (int o = 1; o < 32; o <<= 1) {
      const int a0 = __shfl_up_sync(0xffffffffu, i0, o), a1 = __shfl_up_sync(0xffffffffu, i1, o);
      if (lane >= o) { i0 += a0; i1 += a1; }
    }
    const int tot0 = __shfl_sync(0xffffffffu, i0, 31);
    pst[lane] = i0 - c0;
    if (lane + 32 < kTlP * kTlP) pst[lane + 32] = tot0 + i1 - c1;
    if (lane == kTlP * kTlP - 32 - 1) pst[kTlP * kTlP] = tot0 + i1;
  } else if (warp == 1 && lane <= nlt) {
    ls[lane] = leaf_start[L0 + lane];
  } else if (warp == 2 && lane < kTlP) {
    // the offsets of the patch columns / rows from the tile's first leaf
    const double o = (double)(lane - 1) * ((double)d + (double)dlo);
    const float oh = (float)o;
    offh[lane] = oh;
    offl[lane] = (float)(o - (double)oh);
  }
  __syncthreads();
  const bool staged = pst[kTlP * kTlP] <= kTlCap;
  if (staged) {
    for (int pi = warp; pi < kTlP * kTlP; pi += kEvWarps) {
      const int b0 = pbeg[pi], cnt = pst[pi + 1] - pst[pi], o = pst[pi];
      const float ohx = offh[pi % kTlP], olx = offl[pi % kTlP];
      const float ohy = offh[pi / kTlP], oly = offl[pi / kTlP];
      for (int j = lane; j < cnt; j += 32) {
        const float2 v = loc[b0 + j], w = loclo[b0 + j];
        float hx, lx, hy, ly;
        add_hilo(v.x, w.x, ohx, olx, hx, lx);
        add_hilo(v.y, w.y, ohy, oly, hy, ly);
        src[o + j] = make_float4(hx, hy, lx, ly);
        srcq[o + j] = fs_round(q[perm[b0 + j]]);
      }
    }
  }
  __syncthreads();
  const int t0 = ls[0], t1 = ls[nlt];
  for (int tb = t0 + 32 * warp; tb < t1; tb += 32 * kEvWarps) {
    const int i = tb + lane;
    const bool act = i < t1;
    // the target's leaf: the last tile leaf whose start is <= i
    int li = 0;
    for (int step = 8; step > 0; step >>= 1)
      if (li + step < nlt && ls[li + step] <= i) li += step;
    const uint64_t leaf = L0 + li;
    const int ix = box_ix(leaf), iy = box_iy(leaf);
    const int px = ix - tx0 + 1, py = iy - ty0 + 1;
    float lf = 0.f, gx = 0.f, gy = 0.f;
    if (staged) {
      const int kself = pst[py * kTlP + px] + (i - ls[li]);
      float4 me = make_float4(0.f, 0.f, 0.f, 0.f);
      if (act) me = src[kself];
      const f2p mh = f2_pack(me.x, me.y), ml = f2_pack(me.z, me.w);
      f2p g = f2_pack(0.f, 0.f);
#pragma unroll 1
      for (int r = -1; r <= 1; ++r) {
        const int pi = (py + r) * kTlP + px;
        const int lo = pst[pi - 1];
        const int hi = act ? pst[pi + 2] : lo;
        if (r == 0) {
          pair_loop_self(src, srcq, lo, hi, mh, ml, lf, g);
        } else {
          pair_loop(src, srcq, lo, hi, mh, ml, lf, g);
        }
      }
      f2_unpack(g, gx, gy);
    } else if (act) {
      const float2 me = loc[i], ml = loclo[i];
      for (int r = -1; r <= 1; ++r) {
        float syh, syl;
        frame_shift(me.y, ml.y, r, d, dlo, syh, syl);
        for (int c = -1; c <= 1; ++c) {
          const int mx = ix + c, my = iy + r;
          if (mx < 0 || my < 0 || mx >= nx || my >= nx) continue;
          const uint64_t sl = box_morton(mx, my);
          const int s0 = leaf_start[sl], s1 = leaf_start[sl + 1];
          float sxh, sxl;
          frame_shift(me.x, ml.x, c, d, dlo, sxh, sxl);
          for (int k = s0; k < s1; ++k) {
            const float2 v = loc[k], w = loclo[k];
            const float dx = (sxh - v.x) + (sxl - w.x), dy = (syh - v.y) + (syl - w.y);
            const float r2 = fmaf(dx, dx, dy * dy);
            if (!(r2 > 0.f)) continue;  // j = i, or a coincident point
            const float qk = fs_round(q[perm[k]]);
            const float qi = qk * fast_rcp(r2);
            lf = fmaf(qk, fast_lg2(r2), lf);
            gx = fmaf(qi, dx, gx);
            gy = fmaf(qi, dy, gy);
          }
        }
      }
    }
    if (act) near[i] = make_float4(lf, gx, gy, 0.f);
  }
}
constexpr size_t kTpSmem = kLsBytes + (sizeof(float4) + sizeof(float)) * kTlCap +
                           sizeof(int) * (2 * kTlP * kTlP + 1);

// Multi-RHS leaf evaluation (single precision).  The free-space near-field
// pair kernel -- log2 r^2 and (dx, dy) / r^2 -- is formed once per pair and
// applied to RC charge vectors (blockIdx.y selects RHS r0 .. r0 + RC - 1),
// then the local expansions of each RHS are evaluated (L2P).  A block takes
// eight Morton-consecutive leaves (a 4 x 2 tile, one warp per leaf) and stages
// the 6 x 4 leaves around it in shared memory: positions (leaf frame) and the
// RC charges of each point (point-major rows of qsm, qsm[k * rp + r], so one
// 16-byte load carries four RHS).  Patches larger than the buffer read the
// same data from global memory.  Padded RHS r >= nr carry arbitrary charges
// and are not written.
constexpr int kMpW = 6, kMpH = 4, kMpCap = 1024;

template <int RC>
struct MultiAcc {
  float lf[RC], gx[RC], gy[RC];
};

template <int RC, bool CHECK>
__device__ __forceinline__ void multi_range(const float2 *pos, const float4 *qv, int lo, int hi,
                                            int g, int ng, float sx, float sy, MultiAcc<RC> &a) {
#pragma unroll 2
  for (int k = lo + g; k < hi; k += ng) {
    const float2 v = pos[k];
    const float dx = sx - v.x, dy = sy - v.y;
    float r2 = fmaf(dx, dx, dy * dy);
    float lg, ir;
    if (CHECK) {
      const bool ok = r2 > 0.f;
      r2 = ok ? r2 : 1.f;
      lg = ok ? fast_lg2(r2) : 0.f;
      ir = ok ? fast_rcp(r2) : 0.f;
    } else {
      lg = fast_lg2(r2);
      ir = fast_rcp(r2);
    }
    const float ex = dx * ir, ey = dy * ir;
#pragma unroll
    for (int c = 0; c < RC / 4; ++c) {
      const float4 qq = qv[(size_t)k * (RC / 4) + c];
      a.lf[4 * c] = fmaf(qq.x, lg, a.lf[4 * c]);
      a.lf[4 * c + 1] = fmaf(qq.y, lg, a.lf[4 * c + 1]);
      a.lf[4 * c + 2] = fmaf(qq.z, lg, a.lf[4 * c + 2]);
      a.lf[4 * c + 3] = fmaf(qq.w, lg, a.lf[4 * c + 3]);
      a.gx[4 * c] = fmaf(qq.x, ex, a.gx[4 * c]);
      a.gx[4 * c + 1] = fmaf(qq.y, ex, a.gx[4 * c + 1]);
      a.gx[4 * c + 2] = fmaf(qq.z, ex, a.gx[4 * c + 2]);
      a.gx[4 * c + 3] = fmaf(qq.w, ex, a.gx[4 * c + 3]);
      a.gy[4 * c] = fmaf(qq.x, ey, a.gy[4 * c]);
      a.gy[4 * c + 1] = fmaf(qq.y, ey, a.gy[4 * c + 1]);
      a.gy[4 * c + 2] = fmaf(qq.z, ey, a.gy[4 * c + 2]);
      a.gy[4 * c + 3] = fmaf(qq.w, ey, a.gy[4 * c + 3]);
    }
  }
}

template <int RC>
__global__ void __launch_bounds__(kEvWarps * 32, 2)
k_eval32m(const float2 *__restrict__ loc, const float *__restrict__ qsm, int rp, int nr,
          const int64_t *__restrict__ perm, const int *__restrict__ leaf_start, int H,
          const DevGeom *__restrict__ dg, int p, const cf *__restrict__ A,
          const cf *__restrict__ B, RhsStride rs, double *__restrict__ pot,
          double *__restrict__ grad) {
  constexpr int NP = kMpW * kMpH;
  const float d = dg->d[H], invd = dg->invd[H];
  __shared__ float2 spos[kMpCap];
  __shared__ float4 sq[kMpCap * (RC / 4)];
  __shared__ int pst[NP + 1], pbeg[NP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = 1 << H;
  const int r0 = blockIdx.y * RC;
  const int leaf0 = blockIdx.x * kEvWarps;
  const int tx0 = box_ix(leaf0), ty0 = box_iy(leaf0);  // the tile is x0..x0+3, y0..y0+1
  if (warp == 0) {
    int cnt = 0, b0 = 0;
    if (lane < NP) {
      const int lx = tx0 - 1 + lane % kMpW, ly = ty0 - 1 + lane / kMpW;
      if (lx >= 0 && ly >= 0 && lx < nx && ly < nx) {
        const uint64_t lf = box_morton(lx, ly);
        b0 = leaf_start[lf];
        cnt = leaf_start[lf + 1] - b0;
      }
    }
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane < NP) {
      pst[lane] = inc - cnt;
      pbeg[lane] = b0;
    }
    if (lane == NP - 1) pst[NP] = inc;
  }
  __syncthreads();
  const bool staged = pst[NP] <= kMpCap;
  if (staged) {
    for (int pi = warp; pi < NP; pi += kEvWarps) {
      const int b0 = pbeg[pi], cnt = pst[pi + 1] - pst[pi], o = pst[pi];
      for (int j = lane; j < cnt; j += 32) spos[o + j] = loc[b0 + j];
      for (int e = lane; e < cnt * (RC / 4); e += 32) {
        const int j = e / (RC / 4), c = e % (RC / 4);
        sq[(size_t)(o + j) * (RC / 4) + c] =
            __ldg(reinterpret_cast<const float4 *>(qsm + (size_t)(b0 + j) * rp + r0) + c);
      }
    }
  }
  __syncthreads();
  const int leaf = leaf0 + warp;
  if (leaf >= nx * nx) return;
  const int P1 = p + 1;
  const int ix = box_ix(leaf), iy = box_iy(leaf);
  const int px = ix - tx0 + 1, py = iy - ty0 + 1;  // patch coordinates of the leaf
  const int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
  const int T = b1 - b0;
  const int gs = T > 16 ? 32 : (T > 8 ? 16 : (T > 4 ? 8 : 4));
  const int ng = 32 / gs, g = lane / gs, tli = lane % gs;
  const float c4 = (float)(0.69314718055994530942 / (4.0 * HP_PI));
  const float i2pi = (float)(1.0 / HP_TWO_PI);
  for (int tb = b0; tb < b1; tb += gs) {
    const int i = tb + tli;
    const bool act = i < b1;
    const float2 me = act ? loc[i] : make_float2(0.f, 0.f);
    MultiAcc<RC> a;
#pragma unroll
    for (int c = 0; c < RC; ++c) a.lf[c] = a.gx[c] = a.gy[c] = 0.f;
#pragma unroll 1
    for (int rr = -1; rr <= 1; ++rr) {
      const int ny = iy + rr;
      if (ny < 0 || ny >= nx) continue;
#pragma unroll 1
      for (int cc = -1; cc <= 1; ++cc) {
        const int nxx = ix + cc;
        if (nxx < 0 || nxx >= nx) continue;
        const float sx = me.x - (float)cc * d, sy = me.y - (float)rr * d;
        if (staged) {
          const int pi = (py + rr) * kMpW + (px + cc);
          if (rr == 0 && cc == 0)
            multi_range<RC, true>(spos, sq, pst[pi], pst[pi + 1], g, ng, sx, sy, a);
          else
            multi_range<RC, false>(spos, sq, pst[pi], pst[pi + 1], g, ng, sx, sy, a);
        } else {
          const uint64_t sl = box_morton(nxx, ny);
          const int s0 = leaf_start[sl], s1 = leaf_start[sl + 1];
          // global rows are rp wide: view them as float4 rows of rp / 4 from r0
          for (int k = s0 + g; k < s1; k += ng) {
            const float2 v = loc[k];
            const float dx = sx - v.x, dy = sy - v.y;
            float r2 = fmaf(dx, dx, dy * dy);
            const bool ok = !(rr == 0 && cc == 0) || r2 > 0.f;
            r2 = ok ? r2 : 1.f;
            const float lg = ok ? fast_lg2(r2) : 0.f;
            const float ir = ok ? fast_rcp(r2) : 0.f;
            const float ex = dx * ir, ey = dy * ir;
            const float4 *qv = reinterpret_cast<const float4 *>(qsm + (size_t)k * rp + r0);
#pragma unroll
            for (int c = 0; c < RC / 4; ++c) {
              const float4 qq = __ldg(qv + c);
              const float qa[4] = {qq.x, qq.y, qq.z, qq.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                a.lf[4 * c + u] = fmaf(qa[u], lg, a.lf[4 * c + u]);
                a.gx[4 * c + u] = fmaf(qa[u], ex, a.gx[4 * c + u]);
                a.gy[4 * c + u] = fmaf(qa[u], ey, a.gy[4 * c + u]);
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      a.lf[c] = xsum(a.lf[c], gs);
      a.gx[c] = xsum(a.gx[c], gs);
      a.gy[c] = xsum(a.gy[c], gs);
    }
    if (!act || g != 0) continue;
    const cf w = mk(me.x * invd, me.y * invd), wb = conj(w);
    const int64_t o = perm[i];
    const size_t le = (size_t)(level_offset(H) + leaf) * P1;
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      const int r = r0 + c;
      if (r >= nr) break;
      const cf *Al = A + r * rs.m + le, *Bl = B + r * rs.m + le;
      cf va = Al[p], da = mk(0.f, 0.f), vb = Bl[p], db = mk(0.f, 0.f);
      for (int n = p - 1; n >= 0; --n) {
        da = da * w + va;
        va = va * w + Al[n];
        db = db * wb + vb;
        vb = vb * wb + Bl[n];
      }
      const float ur_ = va.x + vb.x - a.lf[c] * c4;
      const float ui_ = va.y + vb.y;
      const cf gxo = invd * (da + db) + mk(-a.gx[c] * i2pi, 0.f);
      const cf gyo = invd * (mul_i(da) - mul_i(db)) + mk(-a.gy[c] * i2pi, 0.f);
      reinterpret_cast<double2 *>(pot + r * rs.out)[o] = make_double2(f2d(ur_), f2d(ui_));
      if (grad) {
        double4_16a gv;
        gv.x = f2d(gxo.x); gv.y = f2d(gxo.y); gv.z = f2d(gyo.x); gv.w = f2d(gyo.y);
        reinterpret_cast<double4_16a *>(grad + 2 * r * rs.out)[o] = gv;
      }
    }
  }
}

// Evaluation at separate targets (Example 2: field points that are not
// sources, on y >= 0).  Targets stay in the caller's order and a warp takes
// 32 of them.  Each lane finds its target's leaf by the sources' own
// quantisation, so that a target placed on a source gets that source's leaf
// and leaf frame, and evaluates the leaf's local expansions (L2P, in the
// plan's precision).  The near field is then summed by the whole warp, one
// target at a time: lanes stride over the sources of the target's 3 x 3
// neighbour leaves and a butterfly reduction hands the sums to the target's
// lane.  Only targets whose neighbourhood holds sources take part, so the
// few field points next to dense leaves do not hold up the other lanes of
// their warp.  The free part is summed in the plan's precision (single
// precision in the leaf frames, as for the sources, with each neighbour
// leaf's exact offset).  The image and reaction parts of bottom-row pairs
// are summed here in double for double-precision plans, and by
// k_mirror_targets for single-precision ones.  A pair at zero distance skips
// its free term (log singularity).
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__global__ void __launch_bounds__(256)
k_eval_targets(const double *__restrict__ xt, const double *__restrict__ yt, int64_t nt,
               const double *__restrict__ xs, const double *__restrict__ ys,
               const float2 *__restrict__ loc, const R *__restrict__ qs,
               const int *__restrict__ leaf_start, int H, double x0, double side,
               double qscale, int p, cd kappa, const cpx<R> *__restrict__ A,
               const cpx<R> *__restrict__ B, double *__restrict__ pot,
               double *__restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = t < nt;
  const int P1 = p + 1, nx = 1 << H;
  const double d = ldexp(side, -H);
  const double x = act ? xt[t] : x0, y = act ? yt[t] : 0.0;
  const int ix = (int)(quantise(__dsub_rn(x, x0), side, qscale) >> (30 - H));
  const int iy = (int)(quantise(y, side, qscale) >> (30 - H));
  const double2 c = leaf_centre_at(x0, d, ix, iy);
  const double lx = x - c.x, ly = y - c.y;  // target in its leaf frame
  const R rd = (R)d, rinvd = (R)(1.0 / d);
  // far field: L2P with the leaf's expansions (Horner in w and conj(w))
  cd u = mk(0.0, 0.0), gx = u, gy = u;
  int cnt = 0;
  if (act) {
    const uint64_t leaf = box_morton(ix, iy);
    const cpx<R> *Al = A + (size_t)(level_offset(H) + leaf) * P1;
    const cpx<R> *Bl = B + (size_t)(level_offset(H) + leaf) * P1;
    const cpx<R> w = mk((R)lx * rinvd, (R)ly * rinvd), wb = conj(w);
    cpx<R> va = Al[p], da = mk<R>(0, 0), vb = Bl[p], db = mk<R>(0, 0);
    for (int n = p - 1; n >= 0; --n) {
      da = da * w + va;
      va = va * w + Al[n];
      db = db * wb + vb;
      vb = vb * wb + Bl[n];
    }
    auto c64 = [](cpx<R> z) { return mk((double)z.x, (double)z.y); };
    u = c64(va + vb);
    gx = (1.0 / d) * c64(da + db);
    gy = (1.0 / d) * c64(mul_i(da) - mul_i(db));
    for (int r = -1; r <= 1; ++r)
      for (int cc = -1; cc <= 1; ++cc) {
        const int mx = ix + cc, my = iy + r;
        if (mx < 0 || my < 0 || mx >= nx || my >= nx) continue;
        const uint64_t sl = box_morton(mx, my);
        cnt += leaf_start[sl + 1] - leaf_start[sl];
      }
  }
  // near field, one target of the warp at a time
  constexpr bool kSingle = sizeof(R) == 4;
  PairAcc<double> mine;  // the sums of this lane's own target
  unsigned hot = __ballot_sync(0xffffffffu, act && cnt > 0);
  while (hot) {
    const int h = __ffs(hot) - 1;
    hot &= hot - 1;
    const int hix = __shfl_sync(0xffffffffu, ix, h), hiy = __shfl_sync(0xffffffffu, iy, h);
    const double hx = __shfl_sync(0xffffffffu, x, h), hy = __shfl_sync(0xffffffffu, y, h);
    const R hlx = (R)__shfl_sync(0xffffffffu, lx, h), hly = (R)__shfl_sync(0xffffffffu, ly, h);
    R lf = 0, fx = 0, fy = 0;
    PairAcc<double> ma;
#pragma unroll 1
    for (int r = -1; r <= 1; ++r) {
      const int my = hiy + r;
      if (my < 0 || my >= nx) continue;
#pragma unroll 1
      for (int cc = -1; cc <= 1; ++cc) {
        const int mx = hix + cc;
        if (mx < 0 || mx >= nx) continue;
        const uint64_t sl = box_morton(mx, my);
        const int s0 = leaf_start[sl], s1 = leaf_start[sl + 1];
        const bool mirror = hiy == 0 && my == 0;
        // the target in the frame of this source leaf (exact leaf offset)
        const R ox = hlx - (R)cc * rd, oy = hly - (R)r * rd;
        for (int k = s0 + lane; k < s1; k += 32) {
          const R q = qs[k];
          R dx, dy;
          double sxa = 0.0, sya = 0.0;
          if constexpr (kSingle) {
            const float2 v = loc[k];
            dx = ox - v.x;
            dy = oy - v.y;
          } else {
            sxa = xs[k];
            sya = ys[k];
            dx = hx - sxa;
            dy = hy - sya;
          }
          const R r2 = dx * dx + dy * dy;
          if (r2 > R(0)) {
            if constexpr (kSingle) {
              const float qi = q * fast_rcp(r2);
              lf = fmaf(q, fast_lg2(r2), lf);
              fx = fmaf(qi, dx, fx);
              fy = fmaf(qi, dy, fy);
            } else {
              const double qi = q / r2;
              lf += q * log(r2);
              fx += qi * dx;
              fy += qi * dy;
            }
          }
          if (!kSingle && mirror) {
            const double ddx = hx - sxa, Y = hy + sya;
            pair_image(ma, ddx, Y, (double)q);
            pair_reaction_d(ma, ddx, Y, (double)q, kappa);
          }
        }
      }
    }
    lf = warp_sum(lf);
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    if (!kSingle && hiy == 0) {
      ma.li = warp_sum(ma.li);
      ma.gix = warp_sum(ma.gix);
      ma.giy = warp_sum(ma.giy);
      ma.ur.x = warp_sum(ma.ur.x);
      ma.ur.y = warp_sum(ma.ur.y);
      ma.grx.x = warp_sum(ma.grx.x);
      ma.grx.y = warp_sum(ma.grx.y);
      ma.gry.x = warp_sum(ma.gry.x);
      ma.gry.y = warp_sum(ma.gry.y);
    }
    if (lane == h) {
      mine = ma;
      // single precision sums q log2 r^2: the accumulator holds q ln r^2
      mine.lf = kSingle ? (double)lf * 0.69314718055994530942 : (double)lf;
      mine.gfx = (double)fx;
      mine.gfy = (double)fy;
    }
  }
  if (!act) return;
  cd un, gxn, gyn;
  mine.finish(un, gxn, gyn);
  u = u + un;
  gx = gx + gxn;
  gy = gy + gyn;
  pot[2 * t] = u.x;
  pot[2 * t + 1] = u.y;
  if (grad) {
    grad[4 * t + 0] = gx.x;
    grad[4 * t + 1] = gx.y;
    grad[4 * t + 2] = gy.x;
    grad[4 * t + 3] = gy.y;
  }
}

// Image and reaction near field of the bottom-row leaves (single precision
// with the double routine for |P| > 1 and, in MIXED mode, below tau), added
// to the outputs written by the leaf kernel.  One block per bottom-row leaf: the
// sources of the three bottom-row neighbours are staged in shared memory,
// lanes take 32 targets at a time and the 8 warps split the sources; the
// partial sums are reduced in shared memory.
constexpr int kMirSrc = 512;
constexpr int kMirSplit = 8;  // blocks per bottom-row leaf
__global__ void __launch_bounds__(kEvWarps * 32)
k_mirror32(const float2 *__restrict__ loc, const float *__restrict__ yabs,
           const float *__restrict__ qs,
           const int64_t *__restrict__ perm, const int *__restrict__ leaf_start, int H,
           const DevGeom *__restrict__ dg, KappaLog K, float tau, double *__restrict__ pot,
           double *__restrict__ grad, RhsStride rs, int assign) {
  const float d = dg->d[H];
  qs += blockIdx.y * rs.q;
  pot += blockIdx.y * rs.out;
  if (grad) grad += blockIdx.y * 2 * rs.out;
  __shared__ float4 src[kMirSrc];
  __shared__ float red[kEvWarps][9][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = 1 << H;
  const int ix = blockIdx.x;  // leaf (ix, 0)
  const cf kap = mk((float)K.kappa.x, (float)K.kappa.y);
  const uint64_t leaf = box_morton(ix, 0);
  const int b0 = leaf_start[leaf], b1 = leaf_start[leaf + 1];
  // source ranges of the bottom-row neighbours
  int s0[3], s1[3];
  float ox[3];
  int ns = 0;
  for (int k = 0; k < 3; ++k) {
    int mxx = ix - 1 + k;
    s0[k] = s1[k] = 0;
    ox[k] = (float)(mxx - ix) * d;
    if (mxx >= 0 && mxx < nx) {
      uint64_t sl = box_morton(mxx, 0);
      s0[k] = leaf_start[sl];
      s1[k] = leaf_start[sl + 1];
    }
    ns += s1[k] - s0[k];
  }
  const float c4 = (float)(0.69314718055994530942 / (4.0 * HP_PI));
  const float i2pi = (float)(1.0 / HP_TWO_PI);
  // target tiles of 32 are spread over gridDim.z blocks (leaves next to a
  // cluster hold many points)
  for (int tb = b0 + 32 * (int)blockIdx.z; tb < b1; tb += 32 * (int)gridDim.z) {
    const int i = tb + lane;
    const bool act = i < b1;
    const float2 me = act ? make_float2(loc[i].x, yabs[i]) : make_float2(0.f, 0.f);
    NearAcc acc;
    acc.lf = acc.gx = acc.gy = acc.li = acc.gix = acc.giy = 0.f;
    acc.ur = acc.grx = acc.gry = mk(0.f, 0.f);
    for (int base = 0; base < ns; base += kMirSrc) {
      __syncthreads();
      for (int e = threadIdx.x; e < kMirSrc && base + e < ns; e += blockDim.x) {
        int r = base + e, k = 0;
        while (r >= s1[k] - s0[k]) { r -= s1[k] - s0[k]; ++k; }
        const int js = s0[k] + r;
        const float2 v = loc[js];
        src[e] = make_float4(v.x + ox[k], yabs[js], qs[js], 0.f);
      }
      __syncthreads();
      const int cnt = min(kMirSrc, ns - base);
      mirror_batch(src, cnt, warp, kEvWarps, me.x, me.y, kap, K, tau, acc);
    }
    red[warp][0][lane] = acc.li;
    red[warp][1][lane] = acc.gix;
    red[warp][2][lane] = acc.giy;
    red[warp][3][lane] = acc.ur.x;
    red[warp][4][lane] = acc.ur.y;
    red[warp][5][lane] = acc.grx.x;
    red[warp][6][lane] = acc.grx.y;
    red[warp][7][lane] = acc.gry.x;
    red[warp][8][lane] = acc.gry.y;
    __syncthreads();
    if (warp == 0 && act) {
      float v[9];
      for (int c = 0; c < 9; ++c) {
        v[c] = 0.f;
        for (int w = 0; w < kEvWarps; ++w) v[c] += red[w][c][lane];
      }
      const int64_t o = perm[i];
      // assign: written before the leaf outputs, which then add it (split
      // evaluation); otherwise added to the leaf outputs
      const double w0 = (double)(v[0] * c4 + v[3] * i2pi), w1 = (double)(v[4] * i2pi);
      pot[2 * o] = assign ? w0 : pot[2 * o] + w0;
      pot[2 * o + 1] = assign ? w1 : pot[2 * o + 1] + w1;
      if (grad) {
        const double g0 = (double)((v[1] + v[5]) * i2pi), g1 = (double)(v[6] * i2pi);
        const double g2 = (double)((v[2] + v[7]) * i2pi), g3 = (double)(v[8] * i2pi);
        grad[4 * o + 0] = assign ? g0 : grad[4 * o + 0] + g0;
        grad[4 * o + 1] = assign ? g1 : grad[4 * o + 1] + g1;
        grad[4 * o + 2] = assign ? g2 : grad[4 * o + 2] + g2;
        grad[4 * o + 3] = assign ? g3 : grad[4 * o + 3] + g3;
      }
    }
    __syncthreads();
  }
}

// Image and reaction near field of separate targets in the bottom leaf row
// (single-precision plans), added to the outputs of k_eval_targets.  The
// targets come listed by the validation pass; one block per target, whose
// threads stride over the sources of the three bottom-row neighbour leaves
// (single precision where the series is accurate, else double, as in
// k_mirror32), then a block reduction.  A few field points next to a dense
// bottom-row leaf thus spread over many warps instead of serialising.
__global__ void __launch_bounds__(kEvWarps * 32)
k_mirror_targets(const int64_t *__restrict__ list, const double *__restrict__ xt,
                 const double *__restrict__ yt, const float2 *__restrict__ loc,
                 const float *__restrict__ yabs, const float *__restrict__ qs,
                 const int *__restrict__ leaf_start, int H,
                 double x0, double side, double qscale, KappaLog K, float tau,
                 double *__restrict__ pot, double *__restrict__ grad) {
  __shared__ float red[kEvWarps][9];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = list[blockIdx.x];
  const int nx = 1 << H;
  const double dd = ldexp(side, -H);
  const float d = (float)dd;
  const double x = xt[t], y = yt[t];
  const int ix = (int)(quantise(__dsub_rn(x, x0), side, qscale) >> (30 - H));
  const double2 c = leaf_centre_at(x0, dd, ix, 0);
  const float mx = (float)(x - c.x), my = (float)y;
  const cf kap = mk((float)K.kappa.x, (float)K.kappa.y);
  NearAcc acc;
  acc.lf = acc.gx = acc.gy = acc.li = acc.gix = acc.giy = 0.f;
  acc.ur = acc.grx = acc.gry = mk(0.f, 0.f);
  for (int k = 0; k < 3; ++k) {
    const int sx = ix - 1 + k;
    if (sx < 0 || sx >= nx) continue;
    const uint64_t sl = box_morton(sx, 0);
    const int s0 = leaf_start[sl], s1 = leaf_start[sl + 1];
    const float ox = (float)(k - 1) * d;
    for (int j = s0 + (int)threadIdx.x; j < s1; j += blockDim.x) {
      const float2 v = loc[j];
      mirror_pair(make_float4(v.x + ox, yabs[j], qs[j], 0.f), mx, my, kap, K, tau, acc);
    }
  }
  float v[9] = {acc.li,    acc.gix,   acc.giy,   acc.ur.x, acc.ur.y,
                acc.grx.x, acc.grx.y, acc.gry.x, acc.gry.y};
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    v[e] = warp_sum(v[e]);
    if (lane == 0) red[warp][e] = v[e];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    v[e] = 0.f;
    for (int w = 0; w < kEvWarps; ++w) v[e] += red[w][e];
  }
  const float c4 = (float)(0.69314718055994530942 / (4.0 * HP_PI));
  const float i2pi = (float)(1.0 / HP_TWO_PI);
  pot[2 * t] += (double)(v[0] * c4 + v[3] * i2pi);
  pot[2 * t + 1] += (double)(v[4] * i2pi);
  if (grad) {
    grad[4 * t + 0] += (double)((v[1] + v[5]) * i2pi);
    grad[4 * t + 1] += (double)(v[6] * i2pi);
    grad[4 * t + 2] += (double)((v[2] + v[7]) * i2pi);
    grad[4 * t + 3] += (double)(v[8] * i2pi);
  }
}

inline unsigned cdiv_u(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// workspace of a multi-RHS evaluation: nr right-hand sides, rp = nr rounded
// up to the leaf kernel's RHS chunk; arrays of the evaluation's real type
struct MultiWork {
  int nr, rp;
  void *qs, *qsm, *M, *A, *B;
};
constexpr int kRhsChunk = 8;

// separate targets: evaluate at (xt, yt) instead of at the sources
struct TargetWork {
  const double *xt, *yt;
  int64_t nt;
  const int64_t *blist;  // targets in the bottom leaf row (single precision)
  int64_t nbottom;
};

template <typename R>
hpfmm_status run_passes(hpfmm_plan *pl, const double *q, double *pot, double *grad,
                        cudaStream_t st, const MultiWork *mw, const TargetWork *tw = nullptr) {
  const int p = pl->p, P1 = p + 1, H = pl->H;
  const int64_t n = pl->n;
  const size_t m2 = (size_t)P1 * P1;
  // table pointers (FP32 copies follow the double block)
  auto tab = [&](void *base, size_t count) -> const cpx<R> * {
    if (sizeof(R) == 8) return (const cpx<R> *)base;
    return (const cpx<R> *)((cd *)base + count);
  };
  const cpx<R> *Tm2m = tab(pl->t_m2m, 4 * m2);
  const cpx<R> *Tl2l = tab(pl->t_l2l, 4 * m2);
  const cpx<R> *Tfree = tab(pl->t_m2l, 49 * m2);
  const cpx<R> *Timg = tab(pl->t_rlog, 21 * m2);
  const cpx<R> *Treact = tab(pl->t_refl, (size_t)H * 42 * m2);
  const cd *logs = (const cd *)pl->t_rlog0;
  const int nr = mw ? mw->nr : 1;
  R *qs = (R *)(mw ? mw->qs : pl->qs);
  cpx<R> *M = (cpx<R> *)(mw ? mw->M : pl->M), *A = (cpx<R> *)(mw ? mw->A : pl->A);
  cpx<R> *B = (cpx<R> *)(mw ? mw->B : pl->B);
  const RhsStride rs{n, pl->nbox * (int64_t)P1, 2 * n};
  if (mw && (sizeof(R) == 8 || H < 2)) {
    set_last_error("multi-RHS passes need the single-precision path and >= 2 levels");
    return HPFMM_EUNSUPPORTED;
  }
  const DevGeom *dg = pl->dgeom;

  // single precision, one RHS, the sources as targets: the free-space near
  // field needs only the sorted points and charges, so it runs on this
  // stream while the plan's side stream runs the far-field passes; L2P joins
  // them
  const int nxl = 1 << H, tps = nxl >= kTl ? nxl / kTl : 1;
  const bool split = sizeof(R) == 4 && !mw && !tw;
  if (split && !(pl->near && pl->side_stream && pl->ev_fork && pl->ev_join && pl->ev_gather)) {
    set_last_error("single-precision plan without its near-field buffer or side stream");
    return HPFMM_ECUDA;
  }
  // far-field chain: on the plan's high-priority side stream when split, so
  // that its short dependent kernels take SMs first and the near field fills
  // the rest
  cudaStream_t fs = st;
  // split single precision: the leaf level's M2L, the bottom-row
  // image/reaction pairs and the mirror M2L (into separate arrays that the
  // downward pass adds) on the plan's high-priority m2l stream, joined into
  // the far-field chain (ev_m2lh) before the downward pass
  const bool leaf_m2l_apart = split && H >= 3 && pl->m2l_stream && pl->ev_s2m && pl->ev_m2lh;
  const bool mirror_apart = leaf_m2l_apart && pl->mir_A && pl->ev_up;
  if (split) {
    HP_CUDA(cudaEventRecord(pl->ev_fork, st));
    HP_CUDA(cudaStreamWaitEvent(pl->side_stream, pl->ev_fork, 0));
    fs = pl->side_stream;
  }
  // the charges in tree order: first on the far-field chain when split (the
  // near field reads them through perm itself)
  pass_begin(pl, fs, PASS_GATHER);
  if (split)
    k_gather_q<R><<<dim3(cdiv_u(n, 256), nr), 256, 0, fs>>>(q, pl->perm, n, qs, (R *)nullptr, 0);
  else
    HP_CUDA(launch_dependent(k_gather_q<R>, dim3(cdiv_u(n, 256), nr), dim3(256), 0, st, q,
                             pl->perm, n, qs, mw ? (R *)mw->qsm : (R *)nullptr, mw ? mw->rp : 0));
  pass_end(pl, fs, PASS_GATHER, 1);
  if (split) {
    HP_CUDA(cudaEventRecord(pl->ev_gather, fs));
    pass_begin(pl, st, PASS_EVAL);
    HP_CUDA(launch_dependent(k_near32, dim3((unsigned)(tps * tps)), dim3(32 * kEvWarps), kTpSmem,
                             st, pl->loc32, pl->loclo, q, pl->perm,
                             pl->leaf_start, H, dg, pl->near));
    pass_end(pl, st, PASS_EVAL, 1);
    // the bottom-row image/reaction sums need only the sources too: written
    // now, added by the L2P kernel.  On the m2l stream (idle until the S2M is
    // done), off the near field's stream, after the gather.
    cudaStream_t ms = mirror_apart ? pl->m2l_stream : st;
    HP_CUDA(cudaStreamWaitEvent(ms, pl->ev_gather, 0));
    pass_begin(pl, ms, PASS_NEAR_MIRROR);
    k_mirror32<<<dim3((unsigned)(1 << H), 1, kMirSplit), 32 * kEvWarps, 0, ms>>>(
        pl->loc32, pl->yabs, (const float *)qs, pl->perm, pl->leaf_start, H, dg,
        kappa_log(pl->kre, pl->kim), pl->prec == HPFMM_MIXED ? (float)pl->tau_fp64 : 0.f, pot,
        grad, rs, 1);
    pass_end(pl, ms, PASS_NEAR_MIRROR, 1);
  }
  pass_begin(pl, fs, PASS_P2M);
  // upward pass (Algorithm 1): S2M at the leaves, M2M up to level 1
  int ksub = H - 4;  // subtrees of 4^ksub leaves, at least 256 of them
  if (ksub > 4) ksub = 4;
  if (ksub < 1) ksub = H - 1 < 1 ? H - 1 : 1;
  if (pl->subtree > 0) ksub = pl->subtree < H - 1 ? pl->subtree : H - 1;
  while (ksub > 1 &&
         (upward_smem<R>(p, ksub) > kFusedSmem || downward_smem<R>(p, ksub, false) > kFusedSmem))
    --ksub;
  const int l0 = H - ksub;
  if (sizeof(R) == 8) {
    LeafPoints<double> lp{pl->xs, pl->ys, 0.0};
    size_t shp2m = sizeof(cd) * P1 * 33 * kWarpsPerBlock;
    k_p2m<double><<<cdiv_u(pl->nleaf, kWarpsPerBlock), 32 * kWarpsPerBlock, shp2m, fs>>>(
        lp, (const double *)qs, pl->leaf_start, H, dg, p, (cd *)M);
  } else {
    if (mw)
      k_s2m_multi<kRhsChunk><<<dim3(cdiv_u((int64_t)pl->nleaf * P1, 256), mw->rp / kRhsChunk),
                               256, 0, fs>>>(pl->loc32, (const float *)mw->qsm, mw->rp, nr,
                                             pl->leaf_start, H, dg, p, (cf *)M, rs);
    else
      k_s2m_tile<<<cdiv_u(pl->nleaf, kS2mLeaves), kS2mThreads, 0, fs>>>(
          pl->loc32, (const float *)qs, pl->leaf_start, H, dg, p, (cf *)M, rs);
  }
  pass_end(pl, fs, PASS_P2M, 1);
  // split single precision: the M2L of the leaf level needs only the leaf
  // moments, so it runs on its own stream concurrently with the upward pass
  // and the coarser levels' M2L (it holds about three quarters of the
  // translations)
  bool leaf_m2l_done = false;
  if (leaf_m2l_apart) {
    HP_CUDA(cudaEventRecord(pl->ev_s2m, fs));
    HP_CUDA(cudaStreamWaitEvent(pl->m2l_stream, pl->ev_s2m, 0));
    pass_begin(pl, pl->m2l_stream, PASS_M2L_FREE);
    leaf_m2l_done = launch_m2l_patch<R>(p, H, H, H, dg, (const cpx<R> *)pl->t_m2l_pad, logs, M,
                                        A, B, pl->status, pl->m2l_stream, 1, rs, pl->leaf_start,
                                        1);
    pass_end(pl, pl->m2l_stream, PASS_M2L_FREE, leaf_m2l_done ? 1 : 0);
    if (!mirror_apart) HP_CUDA(cudaEventRecord(pl->ev_m2lh, pl->m2l_stream));
  }
  pass_begin(pl, fs, PASS_M2M);
  // the subtree blocks; when every level above them is small, the last of
  // them also runs those (levels l0 - 1 .. 1), otherwise the levels of 1024
  // boxes and more get one launch each and the small top levels one block
  const bool coarse_in_upward = ksub > 0 && l0 <= ksub;
  if (ksub > 0) {
    size_t sm = upward_smem<R>(p, ksub);
    unsigned nb = (unsigned)(int64_t(1) << (2 * l0));
    HP_CUDA(launch_dependent(k_upward<R>, dim3(nb, nr), dim3(256), sm, fs, H, ksub, p, Tm2m, M, rs,
                             coarse_in_upward ? pl->ctr : (int *)nullptr));
  }
  int nm2m = ksub > 0 ? 1 : 0;
  if (!coarse_in_upward) {
    for (int l = l0 - 1; l >= kCoarseBig; --l, ++nm2m)
      k_m2m_level<R><<<dim3(cdiv_u((int64_t(1) << (2 * l)) * P1, 256), nr), 256, 0, fs>>>(
          l, p, Tm2m, M, rs);
    const int lsmall = l0 - 1 < kCoarseBig - 1 ? l0 - 1 : kCoarseBig - 1;
    if (lsmall >= 1) {
      k_m2m_coarse<R><<<dim3(1, nr), 1024, 0, fs>>>(lsmall, p, Tm2m, M, rs);
      ++nm2m;
    }
  }
  pass_end(pl, fs, PASS_M2M, nm2m);
  // split single precision: the mirror M2L needs only the moments and the
  // reaction tables; it runs on the m2l stream after the leaf level's M2L,
  // concurrently with the coarser levels' free-space M2L, into its own small
  // arrays, which the downward pass adds
  if (mirror_apart) {
    HP_CUDA(cudaEventRecord(pl->ev_up, fs));
    HP_CUDA(cudaStreamWaitEvent(pl->m2l_stream, pl->ev_up, 0));
    HP_TRY(plan_join_tables(pl, pl->m2l_stream));
    pass_begin(pl, pl->m2l_stream, PASS_M2L_MIRROR);
    unsigned nb = (unsigned)(4 * ((1 << H) - 1));  // sum over l of 2 * 2^l boxes
    size_t sm = sizeof(cpx<R>) * (4 * 3 * P1 + 4 * P1);
    k_m2l_mirror_all<R><<<dim3(nb, 1), 128, sm, pl->m2l_stream>>>(
        H, p, dg, Timg, logs + 49, Treact, M, A, B, rs, (cpx<R> *)pl->mir_A, (cpx<R> *)pl->mir_B);
    pass_end(pl, pl->m2l_stream, PASS_M2L_MIRROR, 1);
    HP_CUDA(cudaEventRecord(pl->ev_m2lh, pl->m2l_stream));
  }
  // downward pass: M2L at every level (free V-list from level 2, mirror list
  // from level 1), then L2L from level 1 down to the leaves
  size_t shfree = sizeof(cpx<R>) * (m2 + (size_t)P1 * 33);
  bool patched = false, tc_m2l = false;
  if (H >= 2) {
    pass_begin(pl, fs, PASS_M2L_FREE);
    if (mw && nr >= 16 && pl->m2l_mode == 1)
      tc_m2l = patched = launch_m2l_tc(p, H, dg, (const float *)pl->t_m2l_tc, logs, (const cf *)M, (cf *)A,
                              (cf *)B, pl->status, fs, nr, rs);
    if (!patched)
      patched = launch_m2l_patch<R>(p, H, 2, leaf_m2l_done ? H - 1 : H, dg,
                                    (const cpx<R> *)pl->t_m2l_pad, logs, M, A, B, pl->status, fs,
                                    nr, rs, pl->leaf_start, tw ? 0 : 1);
    pass_end(pl, fs, PASS_M2L_FREE, patched ? (tc_m2l ? H - 1 : 1) : 0);
  }
  // the leaf level's M2L joins the chain here (the mirror M2L below adds to
  // its result, when it runs in place)
  if (leaf_m2l_apart) HP_CUDA(cudaStreamWaitEvent(fs, pl->ev_m2lh, 0));
  if (leaf_m2l_apart && !leaf_m2l_done) {
    set_last_error("leaf-level M2L: no patch kernel for p = %d", p);
    return HPFMM_EUNSUPPORTED;
  }
  if (mw && !patched) {
    set_last_error("multi-RHS passes need the patch M2L kernel (2 <= p <= %d)", HPFMM_MAX_P);
    return HPFMM_EUNSUPPORTED;
  }
  for (int l = 1; l <= H; ++l) {
    if (l >= 2 && !patched) {
      dim3 g(cdiv_u(int64_t(1) << (2 * (l - 1)), 32), 4);
      pass_begin(pl, fs, PASS_M2L_FREE);
      k_m2l_free<R><<<g, 128, shfree, fs>>>(l, p, dg, Tfree, logs, M, A, B);
      pass_end(pl, fs, PASS_M2L_FREE, 1);
    }
  }
  // otherwise the mirror M2L of all levels, after the free-space M2L it adds
  // to; it reads the reaction tables of the last rebuild
  if (!mirror_apart) {
    HP_TRY(plan_join_tables(pl, fs));
    pass_begin(pl, fs, PASS_M2L_MIRROR);
    unsigned nb = (unsigned)(4 * ((1 << H) - 1));  // sum over l of 2 * 2^l boxes
    size_t sm = sizeof(cpx<R>) * (4 * 3 * P1 + 4 * P1);
    k_m2l_mirror_all<R><<<dim3(nb, nr), 128, sm, fs>>>(H, p, dg, Timg, logs + 49, Treact, M, A,
                                                         B, rs, nullptr, nullptr);
    pass_end(pl, fs, PASS_M2L_MIRROR, 1);
  }
  // downward pass: L2L from level 1 to the leaves, each block of subtrees
  // forming its root's expansion from its ancestors.  Split single precision:
  // after the near field has joined, the same kernel evaluates the leaf
  // expansions at the points (on the caller's stream); otherwise the leaf
  // expansions go to memory for the leaf kernels below.
  const DownEval noev{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (split) {
    HP_CUDA(cudaEventRecord(pl->ev_join, fs));
    HP_CUDA(cudaStreamWaitEvent(st, pl->ev_join, 0));
    int kd = H - 1 < 3 ? H - 1 : 3;  // subtrees of 64 leaves: 4^(H-3) blocks
    while (kd > 0 && downward_smem<R>(p, kd, true) > kFusedSmem) --kd;
    pass_begin(pl, st, PASS_L2L);
    const DownEval ev{pl->loc32, pl->near, pl->perm, pl->keys, dg, pot, grad};
    k_downward<R, true><<<dim3((unsigned)(int64_t(1) << (2 * (H - kd))), 1), 256,
                          downward_smem<R>(p, kd, true), st>>>(
        H, kd, p, Tl2l, A, B, rs, pl->leaf_start, 1, ev,
        mirror_apart ? (const cpx<R> *)pl->mir_A : nullptr,
        mirror_apart ? (const cpx<R> *)pl->mir_B : nullptr);
    pass_end(pl, st, PASS_L2L, 1);
    HP_LAUNCH_CHECK();
    return HPFMM_OK;
  }
  pass_begin(pl, fs, PASS_L2L);
  if (ksub > 0)
    k_downward<R, false><<<dim3((unsigned)(int64_t(1) << (2 * l0)), nr), 256,
                           downward_smem<R>(p, ksub, false), fs>>>(H, ksub, p, Tl2l, A, B, rs,
                                                                   pl->leaf_start, tw ? 0 : 1,
                                                                   noev, nullptr, nullptr);
  pass_end(pl, fs, PASS_L2L, ksub > 0 ? 1 : 0);
  pass_begin(pl, st, PASS_EVAL);
  // evaluation at the leaves + near field
  cd kappa = mk(pl->kre, pl->kim);
  if (tw) {
    if (tw->nt > 0)
      k_eval_targets<R><<<cdiv_u(tw->nt, 256), 256, 0, st>>>(
          tw->xt, tw->yt, tw->nt, pl->xs, pl->ys, pl->loc32, (const R *)qs, pl->leaf_start, H,
          pl->x0, pl->side, pl->qscale, p, kappa, A, B, pot, grad);
    pass_end(pl, st, PASS_EVAL, tw->nt > 0 ? 1 : 0);
    if (sizeof(R) == 4 && tw->nbottom > 0) {
      pass_begin(pl, st, PASS_NEAR_MIRROR);
      const float tau = pl->prec == HPFMM_MIXED ? (float)pl->tau_fp64 : 0.f;
      k_mirror_targets<<<(unsigned)tw->nbottom, 32 * kEvWarps, 0, st>>>(
          tw->blist, tw->xt, tw->yt, pl->loc32, pl->yabs, (const float *)qs, pl->leaf_start, H,
          pl->x0, pl->side, pl->qscale, kappa_log(pl->kre, pl->kim), tau, pot, grad);
      pass_end(pl, st, PASS_NEAR_MIRROR, 1);
    }
    HP_LAUNCH_CHECK();
    return HPFMM_OK;
  }
  if (sizeof(R) == 8) {
    k_eval64<<<cdiv_u(pl->nleaf, kWarpsPerBlock), 32 * kWarpsPerBlock, 0, st>>>(
        pl->xs, pl->ys, (const double *)qs, pl->perm, pl->leaf_start, H, dg, p,
        kappa, (const cd *)A, (const cd *)B, pot, grad);
  } else {
    float tau = pl->prec == HPFMM_MIXED ? (float)pl->tau_fp64 : 0.f;
    if (mw) {
      k_eval32m<kRhsChunk><<<dim3(cdiv_u(pl->nleaf, kEvWarps), mw->rp / kRhsChunk),
                             32 * kEvWarps, 0, st>>>(
          pl->loc32, (const float *)mw->qsm, mw->rp, nr, pl->perm, pl->leaf_start, H, dg, p,
          (const cf *)A, (const cf *)B, rs, pot, grad);
    } else {
      set_last_error("single-RHS single-precision evaluation outside the split path");
      return HPFMM_ECUDA;
    }
    pass_end(pl, st, PASS_EVAL, 1);
    pass_begin(pl, st, PASS_NEAR_MIRROR);
    k_mirror32<<<dim3((unsigned)(1 << H), nr, kMirSplit), 32 * kEvWarps, 0, st>>>(
        pl->loc32, pl->yabs, (const float *)qs, pl->perm, pl->leaf_start, H, dg,
        kappa_log(pl->kre, pl->kim), tau, pot, grad, rs, 0);
    pass_end(pl, st, PASS_NEAR_MIRROR, 1);
  }
  if (sizeof(R) == 8) pass_end(pl, st, PASS_EVAL, 1);
  HP_LAUNCH_CHECK();
  return HPFMM_OK;
}

}  // namespace

size_t fmm_shared_bytes_max(int p, bool fp64) {
  size_t c = fp64 ? sizeof(cd) : sizeof(cf);
  size_t P1 = p + 1;
  size_t a = c * P1 * 33 * kWarpsPerBlock, b = c * (P1 * P1 + P1 * 33);
  return a > b ? a : b;
}

hpfmm_status fmm_set_smem_limits(int p) {
  size_t s64 = fmm_shared_bytes_max(p, true), s32 = fmm_shared_bytes_max(p, false);
  HP_CUDA(cudaFuncSetAttribute(k_p2m<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64));
  HP_CUDA(cudaFuncSetAttribute(k_p2m<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32));
  HP_CUDA(cudaFuncSetAttribute(k_m2l_free<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64));
  HP_CUDA(cudaFuncSetAttribute(k_near32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTpSmem));
  HP_CUDA(cudaFuncSetAttribute(k_upward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kFusedSmem));
  HP_CUDA(cudaFuncSetAttribute(k_upward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kFusedSmem));
  HP_CUDA(cudaFuncSetAttribute(k_downward<double, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem));
  HP_CUDA(cudaFuncSetAttribute(k_downward<float, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem));
  HP_CUDA(cudaFuncSetAttribute(k_downward<float, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem));
  HP_CUDA(cudaFuncSetAttribute(k_m2l_free<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32));
  return HPFMM_OK;
}

hpfmm_status fmm_prepare() { return special_init_here(); }

hpfmm_status fmm_eval(hpfmm_plan *pl, const double *q, double *pot, double *grad,
                      cudaStream_t st) {
  if (pl->adaptive) return adaptive_eval(pl, q, pot, grad, st);
  HP_TRY(special_init_here());
  if (pl->prec == HPFMM_FP64) return run_passes<double>(pl, q, pot, grad, st, nullptr);
  return run_passes<float>(pl, q, pot, grad, st, nullptr);
}

bool fmm_multi_supported(const hpfmm_plan *pl) {
  return !pl->adaptive && pl->prec != HPFMM_FP64 && pl->H >= 2 && pl->p >= 2 &&
         pl->p <= HPFMM_MAX_P;
}

int fmm_multi_rp(int nr) { return (nr + kRhsChunk - 1) / kRhsChunk * kRhsChunk; }

hpfmm_status fmm_eval_targets(hpfmm_plan *pl, const double *q, const double *xt,
                              const double *yt, int64_t nt, const int64_t *blist,
                              int64_t nbottom, double *pot, double *grad, cudaStream_t st) {
  HP_TRY(special_init_here());
  const TargetWork tw{xt, yt, nt, blist, nbottom};
  if (pl->prec == HPFMM_FP64) return run_passes<double>(pl, q, pot, grad, st, nullptr, &tw);
  return run_passes<float>(pl, q, pot, grad, st, nullptr, &tw);
}

hpfmm_status fmm_eval_multi(hpfmm_plan *pl, const double *q, int nr, double *pot, double *grad,
                            void *qs, void *qsm, void *M, void *A, void *B, cudaStream_t st) {
  HP_TRY(special_init_here());
  if (!fmm_multi_supported(pl)) {
    set_last_error("multi-RHS passes need single precision, >= 2 levels and p >= 2");
    return HPFMM_EUNSUPPORTED;
  }
  const MultiWork mw{nr, fmm_multi_rp(nr), qs, qsm, M, A, B};
  return run_passes<float>(pl, q, pot, grad, st, &mw);
}
