// adaptive.cu -- the FMM of Algorithms 1 and 2 on an adaptive quadtree, in
// single precision (MIXED adds double-precision reaction pairs near the
// boundary).
//
// Tree.  tree.cu first puts the points in Morton order (stable by key and
// index).  Box (l, k) -- level l, Morton key k of its cell -- holds the points
// whose 60-bit key has the prefix k: a contiguous range of that order.  The
// root holds every point; a box is split, while it holds more than leaf_size
// points and l < H, into its non-empty children.  Boxes are stored level by
// level (levels in order, Morton order within a level).  A dense per-level
// table maps a cell key to its box; an entry is checked against the box's
// key when read, so the table is never cleared.
//
// Interactions -- the paper's adaptive tree over the points and their images,
// whose leaf rule and lists it does not state, read as the classic U, V, W and
// X lists:
//   free V-list of a box t at level l >= 2: the existing children of the
//     neighbours of parent(t) that do not touch t.  They are on t's level, so
//     the 40 translation classes and tables of the uniform tree apply;
//   mirror V-list (boxes of rows 0 and 1): the same rule for t and the mirror
//     images of the boxes, as in the uniform tree, with its per-level tables;
//   near field of a leaf D at level l_D: every leaf C whose ancestor at level
//     min(l_C, l_D) touches the ancestor of D there (image and reaction
//     parts: touches its mirror image, i.e. both in row 0 and at most one
//     cell apart).  With l_C >= l_D these are the leaves inside the 3 x 3
//     cells around D (U-list and W-list), with l_C < l_D the leaves next to
//     an ancestor of D (U-list and X-list).  W and X pairs are summed
//     directly instead of through M2P and P2L.
// Every pair of leaves outside the near field is then covered exactly once:
// by the V-lists of the first level at which their ancestors stop touching.
#include <math.h>

#include "common.cuh"
#include "fsplit.cuh"
#include "near32.cuh"
#include "special.cuh"

namespace {

constexpr int kScanB = 1024;
constexpr int kAdWarps = 8;
// the leaf kernel looks up 8 cells per ancestor level in at most four rounds of 32 lanes
static_assert(8 * kAdaptiveMaxLevel <= 4 * 32, "ancestor-cell lookups exceed four rounds");

inline unsigned cdiv_u(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

struct AdGeom {  // per-level box side (as float hi + lo), its reciprocal and log
  float d[16], dlo[16], invd[16];
  double logd[16];
};
AdGeom ad_geom(double side) {
  AdGeom g;
  for (int l = 0; l < 16; ++l) {
    const double d = ldexp(side, -l);
    g.d[l] = (float)d;
    g.dlo[l] = (float)(d - (double)g.d[l]);
    g.invd[l] = (float)(1.0 / d);
    g.logd[l] = log(d);
  }
  return g;
}

// the box of cell (cx, cy) at level l, or -1
__device__ __forceinline__ int ad_lookup(const int *__restrict__ idx,
                                         const uint64_t *__restrict__ key,
                                         const int *__restrict__ lev, int nbox, int l, int cx,
                                         int cy) {
  const int nx = 1 << l;
  if (cx < 0 || cy < 0 || cx >= nx || cy >= nx) return -1;
  const uint64_t k = box_morton(cx, cy);
  const int b = idx[level_offset(l) + (int64_t)k];
  return (b >= lev[l] && b < lev[l + 1] && b < nbox && key[b] == k) ? b : -1;
}

__device__ __forceinline__ bool is_leaf(int4 c) {
  return c.x < 0 && c.y < 0 && c.z < 0 && c.w < 0;
}

__device__ __forceinline__ int block_scan(int v, int *ws, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  int wpre = 0, tot = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    if (w < warp) wpre += ws[w];
    tot += ws[w];
  }
  __syncthreads();
  total = tot;
  return wpre + x - v;  // exclusive
}

// ---------------------------------------------------------------------------
// tree build

__global__ void k_ad_root(int n, uint64_t *key, int *lo, int *hi, int *parent, int *lvl,
                          int *lev) {
  key[0] = 0;
  lo[0] = 0;
  hi[0] = n;
  parent[0] = -1;
  lvl[0] = 0;
  lev[0] = 0;
  lev[1] = 1;
}

// boxes of level l: index entry, split decision and the split points of the
// range between the four children: the first points of the child cells, read
// from the sort's cell offsets down to its bucket level Hs, below that lower
// bounds of the child key prefixes
__global__ void __launch_bounds__(256)
k_ad_split(int l, int H, int cap, int acap, int maxlev, const uint64_t *__restrict__ pkeys,
           const int *__restrict__ cell_start, int Hs, const int *__restrict__ lev,
           const uint64_t *__restrict__ key,
           const int *__restrict__ lo, const int *__restrict__ hi, int4 *__restrict__ cut,
           int *__restrict__ nch, int4 *__restrict__ child, int *__restrict__ idx) {
  const int b0 = lev[l], b1 = min(min(lev[l + 1], acap), b0 + maxlev);
  for (int b = b0 + (int)(blockIdx.x * blockDim.x + threadIdx.x); b < b1;
       b += (int)(gridDim.x * blockDim.x)) {
    const uint64_t k = key[b];
    if (k < (uint64_t(1) << (2 * l))) idx[level_offset(l) + (int64_t)k] = b;
    child[b] = make_int4(-1, -1, -1, -1);
    const int a = lo[b], e = hi[b];
    int nc = 0;
    int4 ct = make_int4(0, 0, 0, 0);
    if (e - a > cap && l < H) {
      const int sh = 2 * (30 - (l + 1));
      int c[5];
      c[0] = a;
      c[4] = e;
      for (int t = 1; t <= 3; ++t) {
        if (l + 1 <= Hs) {  // a cell of the sort's buckets or above: its first point
          c[t] = cell_start[((k << 2) | (uint64_t)t) << (2 * (Hs - l - 1))];
          continue;
        }
        const uint64_t v = ((k << 2) | (uint64_t)t) << sh;
        int L = c[t - 1], R = e;
        while (L < R) {
          const int m = (L + R) >> 1;
          if (pkeys[m] < v) L = m + 1;
          else R = m;
        }
        c[t] = L;
      }
      for (int t = 0; t < 4; ++t) nc += c[t + 1] > c[t] ? 1 : 0;
      ct = make_int4(c[1], c[2], c[3], 1);
    }
    cut[b] = ct;
    nch[b - b0] = nc;
  }
}

// exclusive scan of the child counts of level l (block partial scans, block
// totals scanned by one block, which also sets the end of level l + 1)
__global__ void __launch_bounds__(kScanB)
k_ad_scan_part(const int *__restrict__ lev, int l, int maxlev, int *__restrict__ v,
               int *__restrict__ btot) {
  __shared__ int ws[32];
  const int n = min(lev[l + 1] - lev[l], maxlev);
  if ((int)(blockIdx.x * kScanB) >= n) return;
  const int i = blockIdx.x * kScanB + threadIdx.x;
  const int x = i < n ? v[i] : 0;
  int tot;
  const int ex = block_scan(x, ws, tot);
  if (i < n) v[i] = ex;
  if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanB)
k_ad_scan_top(int *__restrict__ lev, int l, int maxlev, int *__restrict__ btot) {
  __shared__ int ws[32];
  const int n = max(min(lev[l + 1] - lev[l], maxlev), 0);
  const int nb = (n + kScanB - 1) / kScanB;
  int carry = 0;
  for (int base = 0; base < nb; base += kScanB) {
    const int i = base + threadIdx.x;
    const int x = i < nb ? btot[i] : 0;
    int tot;
    const int ex = block_scan(x, ws, tot);
    if (i < nb) btot[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) lev[l + 2] = lev[l + 1] + carry;
}

// the non-empty children of the split boxes of level l, in Morton order
__global__ void __launch_bounds__(256)
k_ad_children(int l, int acap, int maxlev, const int *__restrict__ lev,
              const int *__restrict__ off, const int *__restrict__ btot,
              uint64_t *__restrict__ key, int *__restrict__ lo, int *__restrict__ hi,
              const int4 *__restrict__ cut, int4 *__restrict__ child, int *__restrict__ parent,
              int *__restrict__ lvl) {
  const int b0 = lev[l], b1 = min(min(lev[l + 1], acap), b0 + maxlev);
  for (int b = b0 + (int)(blockIdx.x * blockDim.x + threadIdx.x); b < b1;
       b += (int)(gridDim.x * blockDim.x)) {
    const int4 ct = cut[b];
    if (ct.w == 0) continue;
    const int r = b - b0;
    int o = b1 + btot[r / kScanB] + off[r];
    const int c[5] = {lo[b], ct.x, ct.y, ct.z, hi[b]};
    const uint64_t k = key[b];
    int ch[4];
    for (int t = 0; t < 4; ++t) {
      if (c[t + 1] > c[t] && o < acap) {
        key[o] = (k << 2) | (uint64_t)t;
        lo[o] = c[t];
        hi[o] = c[t + 1];
        parent[o] = b;
        lvl[o] = l + 1;
        ch[t] = o++;
      } else {
        ch[t] = -1;
      }
    }
    child[b] = make_int4(ch[0], ch[1], ch[2], ch[3]);
  }
}

// leaves in tree order: flag each leaf's first point; after an exclusive scan
// over the points, the leaves of any box are the ranks [E[lo], E[hi])
__global__ void __launch_bounds__(256)
k_ad_leafflag(const int *__restrict__ lev, int H, int acap, int n,
              const int4 *__restrict__ child, const int *__restrict__ lo, int *__restrict__ flag) {
  const int nb = min(lev[H + 1], acap);
  for (int b = (int)(blockIdx.x * blockDim.x + threadIdx.x); b < nb;
       b += (int)(gridDim.x * blockDim.x))
    if (is_leaf(child[b]) && lo[b] >= 0 && lo[b] < n) flag[lo[b]] = 1;
}

__global__ void __launch_bounds__(kScanB)
k_ad_pscan_part(int *__restrict__ v, int cnt, int *__restrict__ btot) {
  __shared__ int ws[32];
  const int i = blockIdx.x * kScanB + threadIdx.x;
  const int x = i < cnt ? v[i] : 0;
  int tot;
  const int ex = block_scan(x, ws, tot);
  if (i < cnt) v[i] = ex;
  if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanB)
k_ad_pscan_top(int *__restrict__ btot, int nb) {
  __shared__ int ws[32];
  int carry = 0;
  for (int base = 0; base < nb; base += kScanB) {
    const int i = base + threadIdx.x;
    const int x = i < nb ? btot[i] : 0;
    int tot;
    const int ex = block_scan(x, ws, tot);
    if (i < nb) btot[i] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanB)
k_ad_pscan_add(int *__restrict__ v, int cnt, const int *__restrict__ btot) {
  const int i = blockIdx.x * kScanB + threadIdx.x;
  if (i < cnt) v[i] += btot[blockIdx.x];
}

__global__ void __launch_bounds__(256)
k_ad_leafrank(const int *__restrict__ lev, int H, int acap, int n, int leafcap,
              const int4 *__restrict__ child, const int *__restrict__ lo,
              const int *__restrict__ rank, int *__restrict__ leaf) {
  const int nb = min(lev[H + 1], acap);
  for (int b = (int)(blockIdx.x * blockDim.x + threadIdx.x); b < nb;
       b += (int)(gridDim.x * blockDim.x)) {
    if (!is_leaf(child[b]) || lo[b] < 0 || lo[b] >= n) continue;
    const int r = rank[lo[b]];
    if (r >= 0 && r < leafcap) leaf[r] = b;
  }
}

// single-precision leaf frames: (x, y) relative to the centre of the point's
// own leaf, and y itself; one warp per leaf
__global__ void __launch_bounds__(256)
k_ad_frames(const double *__restrict__ x, const double *__restrict__ y,
            const int64_t *__restrict__ perm, const int *__restrict__ rank, int n, int leafcap,
            const int *__restrict__ leaf, const uint64_t *__restrict__ key,
            const int *__restrict__ lo, const int *__restrict__ hi, const int *__restrict__ lvl,
            double x0, double side, float2 *__restrict__ loc, float2 *__restrict__ loclo,
            float *__restrict__ yabs) {
  const int lane = threadIdx.x & 31;
  const int nl = min(rank[n], leafcap);
  for (int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < nl;
       r += (int)((gridDim.x * blockDim.x) >> 5)) {
    const int b = leaf[r];
    const uint64_t k = key[b];
    const double2 c = leaf_centre_at(x0, ldexp(side, -lvl[b]), box_ix(k), box_iy(k));
    const int e = min(hi[b], n);
    for (int i = max(lo[b], 0) + lane; i < e; i += 32) {
      const int64_t j = perm[i];
      const double a = x[j], v = y[j];
      // the leaf-frame position as float hi + lo, by integer operations
      const FsPair sx = fs_split(a - c.x), sy = fs_split(v - c.y);
      loc[i] = make_float2(sx.hi, sy.hi);
      loclo[i] = make_float2(sx.lo, sy.lo);
      yabs[i] = fs_round(v);
    }
  }
}

// ---------------------------------------------------------------------------
// passes

__global__ void k_ad_gather_q(const double *__restrict__ q, const int64_t *__restrict__ perm,
                              int n, float *__restrict__ qs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) qs[i] = (float)q[perm[i]];
}

// S2M at the leaves (Eq. MEcoefficients, power moments scaled by the leaf
// side): one thread per leaf and group of four orders, compensated sums
constexpr int kG = 4;
__global__ void __launch_bounds__(256)
k_ad_s2m(const float2 *__restrict__ loc, const float *__restrict__ qs,
         const int *__restrict__ leaf, int nleaf, const int *__restrict__ lo,
         const int *__restrict__ hi, const int *__restrict__ lvl, AdGeom g, int p,
         cf *__restrict__ M) {
  const int P1 = p + 1, NB = (P1 + kG - 1) / kG;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nleaf * NB) return;
  const int r = (int)(t / NB), nb = (int)(t % NB), n0 = kG * nb;
  const int b = leaf[r];
  const float invd = g.invd[lvl[b]];
  cf acc[kG], cmp[kG];
#pragma unroll
  for (int e = 0; e < kG; ++e) acc[e] = cmp[e] = mk(0.f, 0.f);
  for (int j = lo[b]; j < hi[b]; ++j) {
    const float2 v = loc[j];
    const cf w = mk(v.x * invd, v.y * invd);
    const cf w2 = w * w, w4 = w2 * w2;
    cf wn = mk(qs[j], 0.f);
    for (int i = 0; i < nb; ++i) wn = wn * w4;
#pragma unroll
    for (int e = 0; e < kG; ++e) {
      const cf yv = wn - cmp[e];
      const cf tv = acc[e] + yv;
      cmp[e] = (tv - acc[e]) - yv;
      acc[e] = tv;
      wn = wn * w;
    }
  }
#pragma unroll
  for (int e = 0; e < kG; ++e)
    if (n0 + e < P1) M[(size_t)b * P1 + n0 + e] = acc[e];
}

// M2M (Eq. metome) of the split boxes of level l from their children
__global__ void __launch_bounds__(256)
k_ad_m2m(int b0, int nb, int p, const cf *__restrict__ Tm2m, const int4 *__restrict__ child,
         cf *__restrict__ M) {
  const int P1 = p + 1;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nb * P1) return;
  const int b = b0 + (int)(e / P1), n = (int)(e % P1);
  const int4 c4 = child[b];
  if (is_leaf(c4)) return;
  const int ch[4] = {c4.x, c4.y, c4.z, c4.w};
  cf acc = mk(0.f, 0.f);
  for (int c = 0; c < 4; ++c) {
    if (ch[c] < 0) continue;
    const cf *Tc = Tm2m + (size_t)c * P1 * P1 + (size_t)n * P1;
    const cf *Mc = M + (size_t)ch[c] * P1;
    for (int m = 0; m <= n; ++m) cfma(acc, Tc[m], Mc[m]);
  }
  M[(size_t)b * P1 + n] = acc;
}

// free-space M2L over the V-list (same level): one warp per target box, lane
// n accumulates output coefficient n; the source vector is broadcast from
// lane k by shuffles.  Adds L/2 to A and conj(L)/2 to B.
__global__ void __launch_bounds__(kAdWarps * 32)
k_ad_m2l(int bfirst, int blast, int nbox, int p, AdGeom g, const cf *__restrict__ Tfree,
         const cd *__restrict__ logt, const int *__restrict__ idx, const uint64_t *__restrict__ key,
         const int *__restrict__ lev, const int *__restrict__ lvl, const cf *__restrict__ M,
         cf *__restrict__ A, cf *__restrict__ B) {
  const int lane = threadIdx.x & 31;
  const int b = bfirst + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b >= blast) return;
  const int P1 = p + 1, l = lvl[b];
  const uint64_t k = key[b];
  const int ix = box_ix(k), iy = box_iy(k), px = ix >> 1, py = iy >> 1;
  const float logd = (float)g.logd[l];
  cf acc = mk(0.f, 0.f);
  for (int sy = 2 * (py - 1); sy <= 2 * (py + 1) + 1; ++sy) {
    for (int sx = 2 * (px - 1); sx <= 2 * (px + 1) + 1; ++sx) {
      const int dx = sx - ix, dy = sy - iy;
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
      const int s = ad_lookup(idx, key, lev, nbox, l, sx, sy);
      if (s < 0) continue;
      const int cls = (dy + 3) * 7 + (dx + 3);
      const cf mine = lane < P1 ? M[(size_t)s * P1 + lane] : mk(0.f, 0.f);
      const cf *Tr = Tfree + (size_t)cls * P1 * P1 + (size_t)(lane < P1 ? lane : 0) * P1;
      for (int kk = 0; kk < P1; ++kk) {
        cf mv;
        mv.x = __shfl_sync(0xffffffffu, mine.x, kk);
        mv.y = __shfl_sync(0xffffffffu, mine.y, kk);
        if (lane < P1) cfma(acc, Tr[kk], mv);
      }
      // M_0 log(t d) term of L_0 (M_0 is real for real charges)
      const float m0 = __shfl_sync(0xffffffffu, mine.x, 0);
      if (lane == 0) acc.x += m0 * ((float)logt[cls].x + logd);
    }
  }
  if (lane >= P1) return;
  const cf v = (float)(-0.5 / HP_TWO_PI) * acc;
  const size_t e = (size_t)b * P1 + lane;
  A[e] = A[e] + v;
  B[e] = B[e] + conj(v);
}

// Free-space M2L in Hankel form (even p up to 20): moments scaled by 16^k/k!,
// T'[r][k] = g_{r+k} of the offset class (scaled by 16^-(r+k) in the table),
// outputs scaled by (-1)^{r+1} 16^r/r!
// (the uniform tree's class vectors, staged in shared memory).  A block of
// four warps takes 32 parent boxes and warp w their children of type w, so
// that the lanes of a warp share every source offset and class vector (a
// broadcast read); each lane accumulates its target's P1 outputs in
// registers.  Parents of every level in one launch.
__device__ __forceinline__ int ad_slot(int cls) {  // 7 x 7 offset class -> 0..39
  const int r = cls / 7, c = cls % 7;
  const int near_before = r < 2 ? 0 : (r > 4 ? 9 : (r - 2) * 3 + min(max(c - 2, 0), 3));
  return cls - near_before;
}

template <int P1>
__global__ void __launch_bounds__(128)
k_ad_m2l_hk(int pfirst, int plast, int nbox, AdGeom g, const cf *__restrict__ Tpad,
            const cd *__restrict__ logt, const int *__restrict__ idx,
            const uint64_t *__restrict__ key, const int *__restrict__ lev,
            const int *__restrict__ lvl, const int4 *__restrict__ child,
            const cf *__restrict__ M, cf *__restrict__ A, cf *__restrict__ B) {
  constexpr int GP = 2 * P1;
  __shared__ cf Gs[40 * GP];
  __shared__ float fac_in[P1], fac_out[P1], lgt[49];
  for (int e = threadIdx.x; e < 40 * GP; e += blockDim.x)
    Gs[e] = Tpad[(size_t)(e / GP) * 2 * GP + e % GP];
  if (threadIdx.x < P1) {
    double f = 1.0;
    for (int i = 2; i <= (int)threadIdx.x; ++i) f *= (double)i;
    // the table's entries carry 16^-j (the single-precision range scaling of
    // m2l_patch.cuh), so the moment and output factors carry 16^k and 16^r
    const double rr = ldexp(1.0, kHankelLog2R * (int)threadIdx.x);
    fac_in[threadIdx.x] = (float)(rr / f);
    fac_out[threadIdx.x] = (float)(((threadIdx.x & 1) ? rr : -rr) / f);
  }
  for (int c = threadIdx.x; c < 49; c += blockDim.x) lgt[c] = (float)logt[c].x;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = pfirst + (int)blockIdx.x * 32 + lane;
  int c = -1;
  if (P < plast) {
    const int4 ch = child[P];
    c = warp == 0 ? ch.x : (warp == 1 ? ch.y : (warp == 2 ? ch.z : ch.w));
  }
  if (!__any_sync(0xffffffffu, c >= 0)) return;
  const int a = warp & 1, bb = warp >> 1;
  int l = 2, ix = 0, iy = 0;
  if (c >= 0) {
    const uint64_t k = key[c];
    l = lvl[c];
    ix = box_ix(k);
    iy = box_iy(k);
  }
  const float logd = (float)g.logd[l];
  cf acc[P1];
#pragma unroll
  for (int r = 0; r < P1; ++r) acc[r] = mk(0.f, 0.f);
  for (int dy = -2 - bb; dy <= 3 - bb; ++dy) {
    for (int dx = -2 - a; dx <= 3 - a; ++dx) {
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
      const int s = c >= 0 ? ad_lookup(idx, key, lev, nbox, l, ix + dx, iy + dy) : -1;
      if (!__any_sync(0xffffffffu, s >= 0)) continue;
      if (s < 0) continue;
      const int cls = (dy + 3) * 7 + (dx + 3);
      const cf *G = Gs + ad_slot(cls) * GP;
      cf m[P1];
#pragma unroll
      for (int k = 0; k < P1; ++k) m[k] = fac_in[k] * M[(size_t)s * P1 + k];
      // anti-diagonals j = r + k: each g_j read once
#pragma unroll
      for (int j = 0; j < 2 * P1 - 1; ++j) {
        const cf gj = G[j];
#pragma unroll
        for (int r = (j - P1 + 1 > 0 ? j - P1 + 1 : 0); r <= (j < P1 - 1 ? j : P1 - 1); ++r)
          cfma(acc[r], gj, m[j - r]);
      }
      // M_0 ln|t d| on Re L_0 (in the scaled outputs L_0 = -L'_0)
      acc[0].x -= m[0].x * (lgt[cls] + logd);
    }
  }
  if (c < 0) return;
  const float s = (float)(-0.5 / HP_TWO_PI);
  const size_t e0 = (size_t)c * P1;
#pragma unroll
  for (int r = 0; r < P1; ++r) {
    const cf v = (s * fac_out[r]) * acc[r];
    A[e0 + r] = A[e0 + r] + v;
    B[e0 + r] = B[e0 + r] + conj(v);
  }
}

template <int P1>
void launch_ad_m2l_hk(int pfirst, int plast, int nbox, const AdGeom &g, const cf *Tpad,
                      const cd *logt, const hpfmm_plan *pl, const cf *M, cf *A, cf *B,
                      cudaStream_t st) {
  k_ad_m2l_hk<P1><<<cdiv_u(plast - pfirst, 32), 128, 0, st>>>(
      pfirst, plast, nbox, g, Tpad, logt, pl->ab_idx, pl->ab_key, pl->ab_lev, pl->ab_lvl,
      pl->ab_child, M, A, B);
}

// mirror M2L (image log and the reaction parts Phi_2^+ and Phi_2^-, Eqs.
// metoleimage and truncatedM2Lcoef) for the boxes of rows 0 and 1, with the
// tables of the uniform tree (21 classes per level)
__global__ void __launch_bounds__(kAdWarps * 32)
k_ad_mirror(int bfirst, int blast, int nbox, int p, AdGeom g, const cf *__restrict__ Timg,
            const cd *__restrict__ logimg, const cf *__restrict__ Treact,
            const int *__restrict__ idx, const uint64_t *__restrict__ key,
            const int *__restrict__ lev, const int *__restrict__ lvl, const cf *__restrict__ M,
            cf *__restrict__ A, cf *__restrict__ B) {
  const int lane = threadIdx.x & 31;
  const int b = bfirst + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b >= blast) return;
  const uint64_t k = key[b];
  const int ixt = box_ix(k), iyt = box_iy(k);
  if (iyt > 1) return;
  const int P1 = p + 1, l = lvl[b], px = ixt >> 1;
  const int nx = 1 << l;
  const float logd = (float)g.logd[l];
  const int row = lane < P1 ? lane : 0;
  cf aL = mk(0.f, 0.f), aC = aL, aD = aL;
  for (int iys = 0; iys <= 1; ++iys) {
    for (int ixs = 2 * (px - 1); ixs <= 2 * (px + 1) + 1; ++ixs) {
      if (ixs < 0 || ixs >= nx) continue;
      if (iyt == 0 && iys == 0 && abs(ixs - ixt) <= 1) continue;
      const int s = ad_lookup(idx, key, lev, nbox, l, ixs, iys);
      if (s < 0) continue;
      const int dx = ixs - ixt, ysum = iyt + iys + 1;
      const int cls = (ysum - 1) * 7 + (dx + 3);
      const cf mine = lane < P1 ? M[(size_t)s * P1 + lane] : mk(0.f, 0.f);
      const cf *Ti = Timg + (size_t)cls * P1 * P1 + (size_t)row * P1;
      const cf *Tp = Treact + ((size_t)((l - 1) * 21 + cls) * 2) * P1 * P1 + (size_t)row * P1;
      const cf *Tm = Tp + (size_t)P1 * P1;
      for (int kk = 0; kk < P1; ++kk) {
        cf mv;
        mv.x = __shfl_sync(0xffffffffu, mine.x, kk);
        mv.y = __shfl_sync(0xffffffffu, mine.y, kk);
        if (lane < P1) {
          const cf mc = conj(mv);
          cfma(aL, Ti[kk], mc);
          cfma(aC, Tp[kk], mc);
          cfma(aD, Tm[kk], mv);
        }
      }
      const float m0 = __shfl_sync(0xffffffffu, mine.x, 0);
      if (lane == 0) aL.x += m0 * ((float)logimg[cls].x + logd);  // M_0 ln|t d|
    }
  }
  if (lane >= P1) return;
  const cf L = (float)(0.5 / HP_TWO_PI) * aL;
  const size_t e = (size_t)b * P1 + lane;
  A[e] = A[e] + L + aC;
  B[e] = B[e] + conj(L) + aD;
}

// L2L (Eq. letole1) into the boxes of level l + 1 from their parents
__global__ void __launch_bounds__(256)
k_ad_l2l(int b0, int nb, int p, const cf *__restrict__ Tl2l, const int *__restrict__ parent,
         const uint64_t *__restrict__ key, cf *__restrict__ A, cf *__restrict__ B) {
  const int P1 = p + 1;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nb * P1) return;
  const int b = b0 + (int)(e / P1), m = (int)(e % P1);
  const int pa = parent[b], c = (int)(key[b] & 3);
  const cf *Tc = Tl2l + (size_t)c * P1 * P1 + (size_t)m * P1;
  const size_t pe = (size_t)pa * P1, ce = (size_t)b * P1;
  cf sa = A[ce + m], sb = B[ce + m];
  for (int n = m; n < P1; ++n) {
    cfma(sa, Tc[n], A[pe + n]);
    cfma(sb, conj(Tc[n]), B[pe + n]);
  }
  A[ce + m] = sa;
  B[ce + m] = sb;
}

// offset of the centre of box (l, cx, cy) from the centre of box (lt, tx, ty)
// in single precision: an exact integer multiple of half the finer side.
// With levels <= 13 both products stay below 2^28 and the difference of two
// touching boxes' centres below 2^15 half-sides, so 32-bit integers and the
// conversion to float are exact (no 64-bit conversions on the FP64 pipe).
__device__ __forceinline__ float2 ad_offset(const AdGeom &g, int l, int cx, int cy, int lt,
                                            int tx, int ty) {
  const int m = l > lt ? l : lt;
  const int nx = (2 * cx + 1) * (1 << (m - l)) - (2 * tx + 1) * (1 << (m - lt));
  const int ny = (2 * cy + 1) * (1 << (m - l)) - (2 * ty + 1) * (1 << (m - lt));
  const float h = 0.5f * g.d[m];
  return make_float2((float)nx * h, (float)ny * h);
}

// the offset ad_offset() gives, as float hi + lo of its exact value n d_m / 2
// (n the integer of ad_offset, d_m = d + dlo the level's side in two parts)
__device__ __forceinline__ float4 ad_offset_hilo(const AdGeom &g, int l, int cx, int cy, int lt,
                                                 int tx, int ty) {
  const int m = l > lt ? l : lt;
  const float nx = (float)((2 * cx + 1) * (1 << (m - l)) - (2 * tx + 1) * (1 << (m - lt)));
  const float ny = (float)((2 * cy + 1) * (1 << (m - l)) - (2 * ty + 1) * (1 << (m - lt)));
  const float h = 0.5f * g.d[m], hl = 0.5f * g.dlo[m];
  const float oxh = nx * h, oyh = ny * h;
  // the products' rounding errors (exact by FMA) plus the low part of the side
  const float oxl = fmaf(nx, h, -oxh) + nx * hl, oyl = fmaf(ny, h, -oyh) + ny * hl;
  return make_float4(oxh, oyh, oxl, oyl);
}

// (h, l) - (oh, ol) as hi + lo: the two-sum of h and -oh (exact for any
// magnitudes), the low parts added
__device__ __forceinline__ void ad_sub_hilo(float h, float l, float oh, float ol, float &sh,
                                            float &sl) {
  sh = h - oh;
  const float bb = sh - h;
  sl = ((h - (sh - bb)) + (-oh - bb)) + (l - ol);
}

// the free-space pairs of one target (its position in the source leaf's frame
// as hi + lo pairs mh, ml) with the points lo .. hi - 1 of that leaf (frames
// loc + loclo), the target's own index `self` skipped; the differences
// (hi - hi) + (lo - lo) and the sums as paired FP32 instructions
__device__ __forceinline__ void ad_free_range(const float2 *__restrict__ loc,
                                              const float2 *__restrict__ loclo,
                                              const float *__restrict__ qs, int lo, int hi,
                                              int self, f2p mh, f2p ml, float &lf, f2p &g) {
  for (int k = lo; k < hi; ++k) {
    if (k == self) continue;
    const float2 v = loc[k], w = loclo[k];
    const float q = qs[k];
    const f2p d = f2_add(f2_sub(mh, f2_pack(v.x, v.y)), f2_sub(ml, f2_pack(w.x, w.y)));
    float dx, dy;
    f2_unpack(d, dx, dy);
    const float r2 = fmaf(dx, dx, dy * dy);
    const float qi = q * fast_rcp(r2);
    lf = fmaf(q, fast_lg2(r2), lf);
    g = f2_fma(f2_pack(qi, qi), d, g);
  }
}

__global__ void __launch_bounds__(kAdWarps * 32)
k_ad_eval(const float2 *__restrict__ loc, const float2 *__restrict__ loclo,
          const float *__restrict__ qs,
          const int64_t *__restrict__ perm,
          const int *__restrict__ leaf, int nleaf, int nbox, const int *__restrict__ rank,
          const int *__restrict__ idx, const uint64_t *__restrict__ key,
          const int *__restrict__ lev, const int *__restrict__ lo, const int *__restrict__ hi,
          const int *__restrict__ lvl, const int4 *__restrict__ child, AdGeom g, int p,
          const cf *__restrict__ A, const cf *__restrict__ B,
          double *__restrict__ pot, double *__restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (r >= nleaf) return;
  const int D = leaf[r], l = lvl[D];
  const uint64_t kD = key[D];
  const int ix = box_ix(kD), iy = box_iy(kD);
  const int P1 = p + 1;
  const float d = g.d[l], invd = g.invd[l];
  const float c4 = (float)(0.69314718055994530942 / (4.0 * HP_PI));
  const float i2pi = (float)(1.0 / HP_TWO_PI);
  (void)d;
  // the near-field sources of D, looked up by the lanes in parallel: lane
  // j < 9 takes cell j of the 3 x 3 around D (all leaves below it); the
  // 8 cells around each ancestor of D (leaves only) in rounds of 32 lanes
  const int nbA = lane < 9 ? ad_lookup(idx, key, lev, nbox, l, ix + lane % 3 - 1,
                                       iy + lane / 3 - 1)
                           : -1;
  const unsigned maskA = __ballot_sync(0xffffffffu, nbA >= 0);
  int candB[4];
  unsigned maskB[4];
#pragma unroll
  for (int rd = 0; rd < 4; ++rd) {
    const int j = rd * 32 + lane;
    int cb = -1;
    if (j < 8 * l) {
      const int la = l - 1 - j / 8, o = j % 8, o9 = o < 4 ? o : o + 1;
      const int C = ad_lookup(idx, key, lev, nbox, la, (ix >> (l - la)) + o9 % 3 - 1,
                              (iy >> (l - la)) + o9 / 3 - 1);
      if (C >= 0 && is_leaf(child[C])) cb = C;
    }
    candB[rd] = cb;
    maskB[rd] = __ballot_sync(0xffffffffu, cb >= 0);
  }
  for (int tb = lo[D]; tb < hi[D]; tb += 32) {
    const int i = tb + lane;
    const bool act = i < hi[D];
    const float2 me = act ? loc[i] : make_float2(0.f, 0.f);
    const float2 mel = act ? loclo[i] : make_float2(0.f, 0.f);
    f2p gsum = f2_pack(0.f, 0.f);
    NearAcc a;
    a.lf = a.gx = a.gy = a.li = a.gix = a.giy = 0.f;
    a.ur = a.grx = a.gry = mk(0.f, 0.f);
    // leaves at level >= l inside the 3 x 3 cells around D
    for (unsigned mA = maskA; mA; mA &= mA - 1) {
      const int jc = __ffs(mA) - 1;
      const int nb = __shfl_sync(0xffffffffu, nbA, jc);
      const int r1 = min(rank[hi[nb]], nleaf);
      for (int rr = rank[lo[nb]]; rr < r1; ++rr) {
        const int C = leaf[rr];
        const uint64_t kC = key[C];
        const float4 o = ad_offset_hilo(g, lvl[C], box_ix(kC), box_iy(kC), l, ix, iy);
        if (act) {
          float sxh, sxl, syh, syl;
          ad_sub_hilo(me.x, mel.x, o.x, o.z, sxh, sxl);
          ad_sub_hilo(me.y, mel.y, o.y, o.w, syh, syl);
          ad_free_range(loc, loclo, qs, lo[C], hi[C], i, f2_pack(sxh, syh), f2_pack(sxl, syl),
                        a.lf, gsum);
        }
      }
    }
    // coarser leaves next to an ancestor of D
#pragma unroll
    for (int rd = 0; rd < 4; ++rd) {
      for (unsigned mB = maskB[rd]; mB; mB &= mB - 1) {
        const int jl = __ffs(mB) - 1;
        const int C = __shfl_sync(0xffffffffu, candB[rd], jl);
        const int j = rd * 32 + jl;
        const int la = l - 1 - j / 8, o = j % 8, o9 = o < 4 ? o : o + 1;
        const int cy = (iy >> (l - la)) + o9 / 3 - 1;
        const float4 off = ad_offset_hilo(g, la, (ix >> (l - la)) + o9 % 3 - 1, cy, l, ix, iy);
        if (act) {
          float sxh, sxl, syh, syl;
          ad_sub_hilo(me.x, mel.x, off.x, off.z, sxh, sxl);
          ad_sub_hilo(me.y, mel.y, off.y, off.w, syh, syl);
          ad_free_range(loc, loclo, qs, lo[C], hi[C], -1, f2_pack(sxh, syh), f2_pack(sxl, syl),
                        a.lf, gsum);
        }
      }
    }
    if (!act) continue;
    f2_unpack(gsum, a.gx, a.gy);
    // far field: L2P with the leaf's expansions
    const cf *Al = A + (size_t)D * P1;
    const cf *Bl = B + (size_t)D * P1;
    const cf w = mk(me.x * invd, me.y * invd), wb = conj(w);
    cf va = Al[p], da = mk(0.f, 0.f), vb = Bl[p], db = mk(0.f, 0.f);
    for (int n = p - 1; n >= 0; --n) {
      da = da * w + va;
      va = va * w + Al[n];
      db = db * wb + vb;
      vb = vb * wb + Bl[n];
    }
    const float ur = va.x + vb.x - a.lf * c4;
    const float ui = va.y + vb.y;
    const cf gxo = invd * (da + db) + mk(-a.gx * i2pi, 0.f);
    const cf gyo = invd * (mul_i(da) - mul_i(db)) + mk(-a.gy * i2pi, 0.f);
    const int64_t o = perm[i];
    pot[2 * o] = f2d(ur);
    pot[2 * o + 1] = f2d(ui);
    if (grad) {
      grad[4 * o + 0] = f2d(gxo.x);
      grad[4 * o + 1] = f2d(gxo.y);
      grad[4 * o + 2] = f2d(gyo.x);
      grad[4 * o + 3] = f2d(gyo.y);
    }
  }
}

// Image and reaction near field on the adaptive tree, added to the outputs of
// k_ad_eval.  A leaf D of row 0 takes the leaves below the row-0 cells on both
// sides of it at its level; every leaf takes the row-0 leaves next to its
// row-0 ancestors (the near-field rule with the mirror image).  One warp per
// leaf, one target per lane; a leaf without such sources returns after its
// lookups (at most 3 + 2 per ancestor level, one round of the lanes).  Kept
// apart from k_ad_eval, whose register count the double-precision branch of
// the pair would otherwise raise.
__global__ void __launch_bounds__(kAdWarps * 32)
k_ad_mirror_near(const float2 *__restrict__ loc, const float *__restrict__ yabs,
                 const float *__restrict__ qs, const int64_t *__restrict__ perm,
                 const int *__restrict__ leaf, int nleaf, int nbox, const int *__restrict__ rank,
                 const int *__restrict__ idx, const uint64_t *__restrict__ key,
                 const int *__restrict__ lev, const int *__restrict__ lo,
                 const int *__restrict__ hi, const int *__restrict__ lvl,
                 const int4 *__restrict__ child, AdGeom g, KappaLog K, float tau,
                 double *__restrict__ pot, double *__restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (r >= nleaf) return;
  const int D = leaf[r], l = lvl[D];
  const uint64_t kD = key[D];
  const int ix = box_ix(kD), iy = box_iy(kD);
  // row-0 cells beside D at its level (lanes 0..2), row-0 leaves beside its
  // row-0 ancestors (lane j: level l - 1 - j/2, side -1 or +1)
  const int nbA = (iy == 0 && lane < 3) ? ad_lookup(idx, key, lev, nbox, l, ix + lane - 1, 0) : -1;
  const unsigned maskA = __ballot_sync(0xffffffffu, nbA >= 0);
  int cb = -1;
  if (lane < 2 * l) {
    const int la = l - 1 - lane / 2, dx = (lane & 1) ? 1 : -1;
    if ((iy >> (l - la)) == 0) {
      const int C = ad_lookup(idx, key, lev, nbox, la, (ix >> (l - la)) + dx, 0);
      if (C >= 0 && is_leaf(child[C])) cb = C;
    }
  }
  const unsigned maskB = __ballot_sync(0xffffffffu, cb >= 0);
  if (!maskA && !maskB) return;
  const cf kap = mk((float)K.kappa.x, (float)K.kappa.y);
  const float c4 = (float)(0.69314718055994530942 / (4.0 * HP_PI));
  const float i2pi = (float)(1.0 / HP_TWO_PI);
  for (int tb = lo[D]; tb < hi[D]; tb += 32) {
    const int i = tb + lane;
    const bool act = i < hi[D];
    const float mx = act ? loc[i].x : 0.f, my = act ? yabs[i] : 0.f;
    NearAcc a;
    a.lf = a.gx = a.gy = a.li = a.gix = a.giy = 0.f;
    a.ur = a.grx = a.gry = mk(0.f, 0.f);
    for (unsigned m = maskA; m; m &= m - 1) {
      const int nb = __shfl_sync(0xffffffffu, nbA, __ffs(m) - 1);
      const int r1 = min(rank[hi[nb]], nleaf);
      for (int rr = rank[lo[nb]]; rr < r1; ++rr) {
        const int C = leaf[rr];
        const uint64_t kC = key[C];
        const float ox = ad_offset(g, lvl[C], box_ix(kC), box_iy(kC), l, ix, iy).x;
        if (act)
          for (int kk = lo[C]; kk < hi[C]; ++kk)
            mirror_pair(make_float4(loc[kk].x + ox, yabs[kk], qs[kk], 0.f), mx, my, kap, K, tau,
                        a);
      }
    }
    for (unsigned m = maskB; m; m &= m - 1) {
      const int j = __ffs(m) - 1;
      const int C = __shfl_sync(0xffffffffu, cb, j);
      const int la = l - 1 - j / 2, dx = (j & 1) ? 1 : -1;
      const float ox = ad_offset(g, la, (ix >> (l - la)) + dx, 0, l, ix, iy).x;
      if (act)
        for (int kk = lo[C]; kk < hi[C]; ++kk)
          mirror_pair(make_float4(loc[kk].x + ox, yabs[kk], qs[kk], 0.f), mx, my, kap, K, tau, a);
    }
    if (!act) continue;
    const int64_t o = perm[i];
    pot[2 * o] += (double)(a.li * c4 + a.ur.x * i2pi);
    pot[2 * o + 1] += (double)(a.ur.y * i2pi);
    if (grad) {
      grad[4 * o + 0] += (double)((a.gix + a.grx.x) * i2pi);
      grad[4 * o + 1] += (double)(a.grx.y * i2pi);
      grad[4 * o + 2] += (double)((a.giy + a.gry.x) * i2pi);
      grad[4 * o + 3] += (double)(a.gry.y * i2pi);
    }
  }
}

// boxes that level l can hold: 4^l, and at most four children per split box
// of level l - 1, which holds more than cap points
int64_t level_bound(int l, int64_t n, int cap) {
  const int64_t full = int64_t(1) << (2 * l);
  if (l == 0) return 1;
  const int64_t split = 4 * (n / (cap + 1));
  return full < split ? full : (split > 0 ? split : 1);
}

}  // namespace

hpfmm_status adaptive_alloc(hpfmm_plan *pl) {
  const int H = pl->H;
  const int64_t n = pl->n;
  int64_t acap = 1, maxlev = 1;
  for (int l = 1; l <= H; ++l) {
    const int64_t b = level_bound(l, n, pl->leaf_cap);
    acap += b;
    if (b > maxlev) maxlev = b;
  }
  pl->acap = acap;
  pl->ad_maxlev = maxlev;
  const int64_t nsb = (maxlev + kScanB - 1) / kScanB, npb = (n + 1 + kScanB - 1) / kScanB;
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_key, sizeof(uint64_t) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_lo, sizeof(int) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_hi, sizeof(int) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_parent, sizeof(int) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_lvl, sizeof(int) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_child, sizeof(int4) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_cut, sizeof(int4) * acap));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_off, sizeof(int) * maxlev));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_idx, sizeof(int) * level_offset(H + 1)));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_lev, sizeof(int) * 32));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_btot, sizeof(int) * (nsb > npb ? nsb : npb)));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_lrank, sizeof(int) * (n + 1)));
  HP_TRY(plan_dalloc(pl, (void **)&pl->ab_leaf, sizeof(int) * (n < acap ? n : acap)));
  return HPFMM_OK;
}

hpfmm_status adaptive_build(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st) {
  const int H = pl->H, cap = pl->leaf_cap;
  const int n = (int)pl->n;
  const int acap = (int)pl->acap, maxlev = (int)pl->ad_maxlev;
  const int leafcap = (int)(pl->n < pl->acap ? pl->n : pl->acap);
  pass_begin(pl, st, PASS_TREE);
  int launches = 0;
  k_ad_root<<<1, 1, 0, st>>>(n, pl->ab_key, pl->ab_lo, pl->ab_hi, pl->ab_parent, pl->ab_lvl,
                             pl->ab_lev);
  ++launches;
  for (int l = 0; l <= H; ++l) {
    const int64_t bound = level_bound(l, pl->n, cap);
    const unsigned gs = cdiv_u(bound, 256) < 4096 ? cdiv_u(bound, 256) : 4096;
    k_ad_split<<<gs, 256, 0, st>>>(l, H, cap, acap, maxlev, pl->keys, pl->leaf_start, pl->Hsort,
                                   pl->ab_lev, pl->ab_key, pl->ab_lo, pl->ab_hi, pl->ab_cut,
                                   pl->ab_off, pl->ab_child, pl->ab_idx);
    ++launches;
    if (l == H) break;
    k_ad_scan_part<<<cdiv_u(bound, kScanB), kScanB, 0, st>>>(pl->ab_lev, l, maxlev, pl->ab_off,
                                                             pl->ab_btot);
    k_ad_scan_top<<<1, kScanB, 0, st>>>(pl->ab_lev, l, maxlev, pl->ab_btot);
    k_ad_children<<<gs, 256, 0, st>>>(l, acap, maxlev, pl->ab_lev, pl->ab_off, pl->ab_btot,
                                      pl->ab_key, pl->ab_lo, pl->ab_hi, pl->ab_cut,
                                      pl->ab_child, pl->ab_parent, pl->ab_lvl);
    launches += 3;
  }
  // leaves in tree order, and the single-precision frames of their points
  const unsigned gb = cdiv_u(pl->acap, 256) < 8192 ? cdiv_u(pl->acap, 256) : 8192;
  HP_CUDA(cudaMemsetAsync(pl->ab_lrank, 0, sizeof(int) * (size_t)(n + 1), st));
  k_ad_leafflag<<<gb, 256, 0, st>>>(pl->ab_lev, H, acap, n, pl->ab_child, pl->ab_lo,
                                    pl->ab_lrank);
  const int np = n + 1, npb = (int)cdiv_u(np, kScanB);
  k_ad_pscan_part<<<npb, kScanB, 0, st>>>(pl->ab_lrank, np, pl->ab_btot);
  k_ad_pscan_top<<<1, kScanB, 0, st>>>(pl->ab_btot, npb);
  k_ad_pscan_add<<<npb, kScanB, 0, st>>>(pl->ab_lrank, np, pl->ab_btot);
  k_ad_leafrank<<<gb, 256, 0, st>>>(pl->ab_lev, H, acap, n, leafcap, pl->ab_child, pl->ab_lo,
                                    pl->ab_lrank, pl->ab_leaf);
  k_ad_frames<<<cdiv_u(n, 256 / 32) < 8192 ? cdiv_u(n, 256 / 32) : 8192, 256, 0, st>>>(
      x, y, pl->perm, pl->ab_lrank, n, leafcap, pl->ab_leaf, pl->ab_key, pl->ab_lo, pl->ab_hi,
      pl->ab_lvl,
      pl->x0, pl->side, pl->loc32, pl->loclo, pl->yabs);
  launches += 6;
  pass_end(pl, st, PASS_TREE, launches);
  HP_LAUNCH_CHECK();
  // level extents and the number of leaves, for the launch sizes of the passes
  int hl[34];
  HP_CUDA(cudaMemcpyAsync(hl, pl->ab_lev, sizeof(int) * (H + 2), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaMemcpyAsync(hl + 33, pl->ab_lrank + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  for (int l = 0; l <= H + 1; ++l) pl->ad_lev[l] = hl[l];
  pl->ad_nbox = hl[H + 1];
  pl->ad_nleaf = hl[33];
  pl->ad_depth = 0;
  for (int l = 0; l <= H; ++l)
    if (hl[l + 1] > hl[l]) pl->ad_depth = l;
  if (pl->ad_nbox < 1 || pl->ad_nbox > pl->acap || pl->ad_nleaf < 1 || pl->ad_nleaf > n) {
    set_last_error("adaptive tree: inconsistent box counts (%lld boxes, %d leaves)",
                   (long long)pl->ad_nbox, pl->ad_nleaf);
    return HPFMM_ECUDA;
  }
  // expansion arrays for the boxes of this tree
  if (pl->ad_nbox > pl->ad_mcap) {
    const int64_t cap2 = pl->ad_nbox + pl->ad_nbox / 4;
    const size_t bytes = sizeof(cf) * (size_t)cap2 * (pl->p + 1);
    for (void **b : {(void **)&pl->M, (void **)&pl->A, (void **)&pl->B}) {
      if (*b) {
        cudaFree(*b);
        pl->workspace_bytes -= (int64_t)(sizeof(cf) * (size_t)pl->ad_mcap * (pl->p + 1));
        *b = nullptr;
      }
    }
    pl->ad_mcap = 0;
    HP_TRY(plan_dalloc(pl, (void **)&pl->M, bytes));
    HP_TRY(plan_dalloc(pl, (void **)&pl->A, bytes));
    HP_TRY(plan_dalloc(pl, (void **)&pl->B, bytes));
    pl->ad_mcap = cap2;
  }
  pl->nbox = pl->ad_nbox;
  return HPFMM_OK;
}

hpfmm_status adaptive_prepare() { return special_init_here(); }

hpfmm_status adaptive_eval(hpfmm_plan *pl, const double *q, double *pot, double *grad,
                           cudaStream_t st) {
  HP_TRY(special_init_here());
  HP_TRY(plan_join_tables(pl, st));  // the mirror M2L reads the reaction tables
  const int p = pl->p, P1 = p + 1, n = (int)pl->n, H = pl->H, depth = pl->ad_depth;
  const size_t m2 = (size_t)P1 * P1;
  const AdGeom g = ad_geom(pl->side);
  // single-precision copies of the tables follow the double block
  auto tab = [&](void *base, size_t count) { return (const cf *)((cd *)base + count); };
  const cf *Tm2m = tab(pl->t_m2m, 4 * m2);
  const cf *Tl2l = tab(pl->t_l2l, 4 * m2);
  const cf *Tfree = tab(pl->t_m2l, 49 * m2);
  const cf *Timg = tab(pl->t_rlog, 21 * m2);
  const cf *Treact = tab(pl->t_refl, (size_t)H * 42 * m2);
  const cd *logs = (const cd *)pl->t_rlog0;
  cf *M = (cf *)pl->M, *A = (cf *)pl->A, *B = (cf *)pl->B;
  float *qs = (float *)pl->qs;
  const int *lev = pl->ad_lev;
  const int nleaf = pl->ad_nleaf, nbox = (int)pl->ad_nbox;

  pass_begin(pl, st, PASS_GATHER);
  k_ad_gather_q<<<cdiv_u(n, 256), 256, 0, st>>>(q, pl->perm, n, qs);
  pass_end(pl, st, PASS_GATHER, 1);
  pass_begin(pl, st, PASS_P2M);
  const int NB = (P1 + kG - 1) / kG;
  k_ad_s2m<<<cdiv_u((int64_t)nleaf * NB, 256), 256, 0, st>>>(
      pl->loc32, qs, pl->ab_leaf, nleaf, pl->ab_lo, pl->ab_hi, pl->ab_lvl, g, p, M);
  pass_end(pl, st, PASS_P2M, 1);
  pass_begin(pl, st, PASS_M2M);
  int nl = 0;
  for (int l = depth - 1; l >= 0; --l) {
    const int nb = lev[l + 1] - lev[l];
    if (nb == 0) continue;
    k_ad_m2m<<<cdiv_u((int64_t)nb * P1, 256), 256, 0, st>>>(lev[l], nb, p, Tm2m, pl->ab_child, M);
    ++nl;
  }
  pass_end(pl, st, PASS_M2M, nl);
  HP_CUDA(cudaMemsetAsync(A, 0, sizeof(cf) * (size_t)pl->ad_nbox * P1, st));
  HP_CUDA(cudaMemsetAsync(B, 0, sizeof(cf) * (size_t)pl->ad_nbox * P1, st));
  pass_begin(pl, st, PASS_M2L_FREE);
  const int all0 = depth >= 2 ? lev[2] : 0, all1 = depth >= 2 ? lev[depth + 1] : 0;
  // Hankel form over the parents of levels 1 .. depth - 1 (even p <= 20),
  // else the dense form over the boxes of levels 2 .. depth
  const int par0 = depth >= 2 ? lev[1] : 0, par1 = depth >= 2 ? lev[depth] : 0;
  bool hankel = false;
  if (all1 > all0 && p % 2 == 0 && p >= 4 && p <= 20) {
    const cf *Tpad = (const cf *)pl->t_m2l_pad;
    hankel = true;
    switch (P1) {
#define HP_AD_CASE(Q) \
  case Q: launch_ad_m2l_hk<Q>(par0, par1, nbox, g, Tpad, logs, pl, M, A, B, st); break;
      HP_AD_CASE(5) HP_AD_CASE(7) HP_AD_CASE(9) HP_AD_CASE(11) HP_AD_CASE(13)
      HP_AD_CASE(15) HP_AD_CASE(17) HP_AD_CASE(19) HP_AD_CASE(21)
#undef HP_AD_CASE
      default: hankel = false;
    }
  }
  if (all1 > all0 && !hankel)
    k_ad_m2l<<<cdiv_u((int64_t)(all1 - all0) * 32, kAdWarps * 32), kAdWarps * 32, 0, st>>>(
        all0, all1, nbox, p, g, Tfree, logs, pl->ab_idx, pl->ab_key, pl->ab_lev, pl->ab_lvl, M, A,
        B);
  pass_end(pl, st, PASS_M2L_FREE, all1 > all0 ? 1 : 0);
  pass_begin(pl, st, PASS_M2L_MIRROR);
  const int m0 = depth >= 1 ? lev[1] : 0, m1 = depth >= 1 ? lev[depth + 1] : 0;
  if (m1 > m0)
    k_ad_mirror<<<cdiv_u((int64_t)(m1 - m0) * 32, kAdWarps * 32), kAdWarps * 32, 0, st>>>(
        m0, m1, nbox, p, g, Timg, logs + 49, Treact, pl->ab_idx, pl->ab_key, pl->ab_lev, pl->ab_lvl,
        M, A, B);
  pass_end(pl, st, PASS_M2L_MIRROR, m1 > m0 ? 1 : 0);
  pass_begin(pl, st, PASS_L2L);
  nl = 0;
  for (int l = 1; l < depth; ++l) {
    const int nb = lev[l + 2] - lev[l + 1];
    if (nb == 0) continue;
    k_ad_l2l<<<cdiv_u((int64_t)nb * P1, 256), 256, 0, st>>>(lev[l + 1], nb, p, Tl2l,
                                                             pl->ab_parent, pl->ab_key, A, B);
    ++nl;
  }
  pass_end(pl, st, PASS_L2L, nl);
  pass_begin(pl, st, PASS_EVAL);
  const float tau = pl->prec == HPFMM_MIXED ? (float)pl->tau_fp64 : 0.f;
  k_ad_eval<<<cdiv_u((int64_t)nleaf * 32, kAdWarps * 32), kAdWarps * 32, 0, st>>>(
      pl->loc32, pl->loclo, qs, pl->perm, pl->ab_leaf, nleaf, nbox, pl->ab_lrank, pl->ab_idx,
      pl->ab_key, pl->ab_lev, pl->ab_lo, pl->ab_hi, pl->ab_lvl, pl->ab_child, g, p, A, B, pot,
      grad);
  pass_end(pl, st, PASS_EVAL, 1);
  pass_begin(pl, st, PASS_NEAR_MIRROR);
  k_ad_mirror_near<<<cdiv_u((int64_t)nleaf * 32, kAdWarps * 32), kAdWarps * 32, 0, st>>>(
      pl->loc32, pl->yabs, qs, pl->perm, pl->ab_leaf, nleaf, nbox, pl->ab_lrank, pl->ab_idx,
      pl->ab_key, pl->ab_lev, pl->ab_lo, pl->ab_hi, pl->ab_lvl, pl->ab_child, g,
      kappa_log(pl->kre, pl->kim), tau, pot, grad);
  pass_end(pl, st, PASS_NEAR_MIRROR, 1);
  HP_LAUNCH_CHECK();
  return HPFMM_OK;
}

extern "C" hpfmm_status hpfmm_get_adaptive_counts(const hpfmm_plan *pl, int maxlev,
                                                  int64_t *boxes, int64_t *leaves, int *depth,
                                                  void *stream) {
  if (!pl || maxlev < 0 || !boxes || !leaves) {
    set_last_error("hpfmm_get_adaptive_counts: null argument or maxlev < 0");
    return HPFMM_EINVAL;
  }
  if (!pl->adaptive) {
    set_last_error("hpfmm_get_adaptive_counts: not an adaptive plan");
    return HPFMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)pl->ad_nbox;
  int *hlvl = new int[nb];
  int4 *hch = new int4[nb];
  cudaError_t e = cudaMemcpyAsync(hlvl, pl->ab_lvl, sizeof(int) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hch, pl->ab_child, sizeof(int4) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete[] hlvl;
    delete[] hch;
    set_last_error("hpfmm_get_adaptive_counts: %s", cudaGetErrorString(e));
    return HPFMM_ECUDA;
  }
  for (int l = 0; l <= maxlev; ++l) boxes[l] = leaves[l] = 0;
  for (int b = 0; b < nb; ++b) {
    const int l = hlvl[b];
    if (l > maxlev) continue;
    ++boxes[l];
    if (hch[b].x < 0 && hch[b].y < 0 && hch[b].z < 0 && hch[b].w < 0) ++leaves[l];
  }
  delete[] hlvl;
  delete[] hch;
  if (depth) *depth = pl->ad_depth;
  return HPFMM_OK;
}
