// tree.cu -- tree construction of Algorithm 1 ("generate an adaptive
// hierarchical tree structure with target points and image source points"):
// the points define a square [x0, x0+L] x [0, L] whose lower edge is the
// boundary y = 0; the image sources fill its mirror [x0, x0+L] x [-L, 0], so
// one quadtree over the points serves both (the mirror tree is its
// reflection).  Steps: validation and bounding square (reduction), 60-bit
// Morton keys (30 bits per axis, bit-exact rule), stable LSD radix sort of
// (key, index), leaf offsets of the uniform level-H grid, gathers.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "fsplit.cuh"

namespace {

struct Geom {
  double xmin, xmax, ymax;
  int bad;  // non-finite or y <= 0 seen
};

constexpr int kRedThreads = 256;

// order-preserving integer image of a finite double (a < b <=> key(a) < key(b),
// key = b >= 0 ? b : b ^ 0x7ff..f), so the min / max reductions run on the
// integer pipe; dkey_inv maps a key back to its double
__device__ __forceinline__ double dkey_inv(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
}

__global__ void bbox_partial(const double *__restrict__ x, const double *__restrict__ y,
                             int64_t n, Geom *__restrict__ part) {
  __shared__ long long s0[kRedThreads], s1[kRedThreads], s2[kRedThreads];
  __shared__ int sb[kRedThreads];
  long long xmn = LLONG_MAX, xmx = LLONG_MIN, ymx = LLONG_MIN;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const long long a = __double_as_longlong(x[i]), b = __double_as_longlong(y[i]);
    // finite: exponent field below 0x7ff; y > 0: sign clear and not +0
    const bool fin = ((a >> 52) & 0x7ff) != 0x7ff && ((b >> 52) & 0x7ff) != 0x7ff;
    if (!fin || b <= 0) bad = 1;
    const long long ka = a >= 0 ? a : (a ^ 0x7fffffffffffffffll);
    xmn = min(xmn, ka);
    xmx = max(xmx, ka);
    ymx = max(ymx, b);  // y > 0: the bit pattern orders like the value
  }
  s0[threadIdx.x] = xmn;
  s1[threadIdx.x] = xmx;
  s2[threadIdx.x] = ymx;
  sb[threadIdx.x] = bad;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s0[threadIdx.x] = min(s0[threadIdx.x], s0[threadIdx.x + w]);
      s1[threadIdx.x] = max(s1[threadIdx.x], s1[threadIdx.x + w]);
      s2[threadIdx.x] = max(s2[threadIdx.x], s2[threadIdx.x + w]);
      sb[threadIdx.x] |= sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    part[blockIdx.x] = Geom{dkey_inv(s0[0]), dkey_inv(s1[0]), dkey_inv(s2[0]), sb[0]};
}

// final reduction (one block); geo[0] = x0, geo[1] = L (side), geo[2] = bad
// flag, geo[3] = 2^30 / L rounded (the fast-path quantisation scale)
__global__ void __launch_bounds__(kRedThreads)
bbox_final(const Geom *__restrict__ part, int nb, double *__restrict__ geo, double root_x0,
           double root_side) {
  __shared__ double s0[kRedThreads], s1[kRedThreads], s2[kRedThreads];
  __shared__ int sb[kRedThreads];
  double xmn = INFINITY, xmx = -INFINITY, ymx = -INFINITY;
  int bad = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    xmn = fmin(xmn, part[b].xmin);
    xmx = fmax(xmx, part[b].xmax);
    ymx = fmax(ymx, part[b].ymax);
    bad |= part[b].bad;
  }
  s0[threadIdx.x] = xmn;
  s1[threadIdx.x] = xmx;
  s2[threadIdx.x] = ymx;
  sb[threadIdx.x] = bad;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s0[threadIdx.x] = fmin(s0[threadIdx.x], s0[threadIdx.x + w]);
      s1[threadIdx.x] = fmax(s1[threadIdx.x], s1[threadIdx.x + w]);
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
      sb[threadIdx.x] |= sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double w = __dsub_rn(s1[0], s0[0]);
  double L = (w > s2[0]) ? w : s2[0];
  L = __dmul_rn(L, 1.0 + 0x1p-40);
  geo[0] = s0[0];
  geo[1] = L;
  geo[2] = sb[0] ? 1.0 : 0.0;
  if (root_side > 0) {  // caller's root square: it must contain the points
    const bool inside = root_x0 <= s0[0] && s1[0] <= root_x0 + root_side && s2[0] <= root_side;
    if (!inside && !sb[0]) geo[2] = 2.0;
    geo[0] = root_x0;
    geo[1] = L = root_side;
  }
  geo[3] = __ddiv_rn(1073741824.0, L);
}


// keys, and the point count of each level-H leaf (the atomic's return value
// is the point's slot inside its leaf bucket; the order within a bucket is
// fixed later by the per-leaf sort)
__global__ void morton_keys(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                            const double *__restrict__ geo, int H, uint64_t *__restrict__ keys,
                            int *__restrict__ idx, int *__restrict__ leaf_count,
                            int *__restrict__ slot) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x0 = geo[0], L = geo[1], sc = geo[3];
  uint64_t ix = quantise(__dsub_rn(x[i], x0), L, sc);
  uint64_t iy = quantise(y[i], L, sc);
  uint64_t k = spread1((uint32_t)ix) | (spread1((uint32_t)iy) << 1);
  keys[i] = k;
  idx[i] = (int)i;
  if (leaf_count) slot[i] = atomicAdd(&leaf_count[k >> (60 - 2 * H)], 1);
}

// exclusive scan of the leaf counts into leaf_start, in three phases: block
// partial scans (1024 leaves per block) with block totals and maxima, a scan
// of the totals (one block), the block offsets added back
__device__ __forceinline__ int block_scan_1024(int v, int *ws, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  int wpre = 0, tot = 0;
  for (int w = 0; w < 32; ++w) {
    if (w < warp) wpre += ws[w];
    tot += ws[w];
  }
  __syncthreads();
  total = tot;
  return wpre + x - v;  // exclusive
}

__global__ void __launch_bounds__(1024)
scan_part(const int *__restrict__ count, int nleaf, int *__restrict__ start,
          int *__restrict__ btot, int *__restrict__ bmax) {
  __shared__ int ws[32];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const int v = i < nleaf ? count[i] : 0;
  int tot;
  const int ex = block_scan_1024(v, ws, tot);
  if (i < nleaf) start[i] = ex;
  int m = v;
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int mm = 0;
    for (int w = 0; w < 32; ++w) mm = max(mm, ws[w]);
    btot[blockIdx.x] = tot;
    bmax[blockIdx.x] = mm;
  }
}

__global__ void __launch_bounds__(1024)
scan_top(int *__restrict__ btot, const int *__restrict__ bmax, int nb, int nleaf,
         int *__restrict__ start, int *__restrict__ maxleaf) {
  __shared__ int ws[32];
  int carry = 0, mx = 0;
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? btot[i] : 0;
    if (i < nb) mx = max(mx, bmax[i]);
    int tot;
    const int ex = block_scan_1024(v, ws, tot);
    if (i < nb) btot[i] = carry + ex;
    carry += tot;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < 32; ++w) m = max(m, ws[w]);
    *maxleaf = m;
    start[nleaf] = carry;
  }
}

__global__ void scan_add(const int *__restrict__ btot, int nleaf, int *__restrict__ start) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < nleaf) start[i] += btot[blockIdx.x];
}

__global__ void bucket_scatter(const uint64_t *__restrict__ keys, const int *__restrict__ slot,
                               int64_t n, int H, const int *__restrict__ start,
                               uint64_t *__restrict__ kout, int *__restrict__ vout) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k = keys[i];
  int pos = start[k >> (60 - 2 * H)] + slot[i];
  kout[pos] = k;
  vout[pos] = (int)i;
}

// sort the leaf buckets of at most 128 points by (key, index): one warp per
// leaf, E = 1, 2 or 4 elements per lane (element i = e * 32 + lane), bitonic
// network with shuffles for partner distances < 32 and register swaps above
__device__ __forceinline__ bool kv_less(uint64_t ka, int va, uint64_t kb, int vb) {
  return ka < kb || (ka == kb && va < vb);
}
__device__ __forceinline__ void kv_cas(uint64_t &ka, int &va, uint64_t &kb, int &vb, bool asc) {
  // after the call (ka, va) <= (kb, vb) when asc, >= otherwise
  const bool gt = kv_less(kb, vb, ka, va);
  if (gt == asc) {
    uint64_t tk = ka; ka = kb; kb = tk;
    int tv = va; va = vb; vb = tv;
  }
}

template <int E>
__device__ __forceinline__ void warp_bitonic(uint64_t (&k)[E], int (&v)[E], int lane) {
  constexpr int N = 32 * E;
  for (int kk = 2; kk <= N; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j < 32) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint64_t ok = __shfl_xor_sync(0xffffffffu, k[e], j);
          const int ov = __shfl_xor_sync(0xffffffffu, v[e], j);
          const int i = e * 32 + lane;
          const bool self_less = kv_less(k[e], v[e], ok, ov);
          const bool want_min = ((i & j) == 0) == ((i & kk) == 0);
          if (want_min != self_less) {
            k[e] = ok;
            v[e] = ov;
          }
        }
      } else if (E >= 2 && j == 32) {
#pragma unroll
        for (int e = 0; e < E; e += 2)
          kv_cas(k[e], v[e], k[e + 1], v[e + 1], ((e * 32 + lane) & kk) == 0);
      } else if (E >= 4 && j == 64) {
        kv_cas(k[0], v[0], k[2 % E], v[2 % E], (lane & kk) == 0);
        kv_cas(k[1 % E], v[1 % E], k[3 % E], v[3 % E], ((32 + lane) & kk) == 0);
      }
    }
  }
}

// Points of a sorted leaf into tree order: the permutation, the leaf-centred
// single-precision coordinates and (double precision) the sorted coordinates.
// Done by the warp or block that sorted the leaf, from the sorted indices it
// holds.  x == nullptr: order only (no gather).
struct LeafGather {
  const double *x, *y, *geo;
  int H;
  double *xs, *ys;
  int64_t *perm;
  float2 *loc32;
  float *yabs;    // y rounded to single precision (with loc32)
  float2 *loclo;  // with loc32: the rest of the leaf-frame position
};

// centre of a leaf (double precision; the leaf side d = side / 2^H is exact)
__device__ __forceinline__ double2 leaf_centre(const LeafGather &g, int leaf) {
  return leaf_centre_at(g.geo[0], ldexp(g.geo[1], -g.H), box_ix(leaf), box_iy(leaf));
}

__device__ __forceinline__ void gather_one(const LeafGather &g, double2 c, int k, int j) {
  const double a = g.x[j], b = g.y[j];
  if (g.xs) {
    g.xs[k] = a;
    g.ys[k] = b;
  }
  g.perm[k] = j;
  if (g.loc32) {
    // the leaf-frame position as a pair of floats (hi + lo), so that
    // differences of nearby points keep their relative precision
    const double rx = a - c.x, ry = b - c.y;
    const float hx = (float)rx, hy = (float)ry;
    g.loc32[k] = make_float2(hx, hy);
    if (g.loclo) g.loclo[k] = make_float2((float)(rx - (double)hx), (float)(ry - (double)hy));
    g.yabs[k] = (float)b;
  }
}

// a warp's leaf centre: computed by lane 0 and broadcast (the double-precision
// pipe is slow; the other lanes would compute the same value)
__device__ __forceinline__ double2 warp_leaf_centre(const LeafGather &g, int leaf, int lane) {
  double2 c = make_double2(0.0, 0.0);
  if (lane == 0 && g.loc32) c = leaf_centre(g, leaf);
  c.x = __shfl_sync(0xffffffffu, c.x, 0);
  c.y = __shfl_sync(0xffffffffu, c.y, 0);
  return c;
}

template <int E>
__device__ __forceinline__ void warp_sort_leaf(int b0, int m, int lane, uint64_t *keys,
                                               int *vals, const LeafGather &g, int leaf) {
  uint64_t k[E];
  int v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    k[e] = i < m ? keys[b0 + i] : ~0ull;
    v[e] = i < m ? vals[b0 + i] : 0x7fffffff;
  }
  warp_bitonic<E>(k, v, lane);
  const double2 c = g.x ? warp_leaf_centre(g, leaf, lane) : make_double2(0.0, 0.0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    if (i < m) {
      keys[b0 + i] = k[e];
      vals[b0 + i] = v[e];
      if (g.x) gather_one(g, c, b0 + i, v[e]);
    }
  }
}

// one leaf of at most 128 points by one warp; larger leaves are appended to
// big[] (count in *nbig) for the block sort
__device__ __forceinline__ void sort_small_leaf(int leaf, int lane, const int *__restrict__ start,
                                                uint64_t *__restrict__ keys, int *__restrict__ vals,
                                                int *__restrict__ big, int *__restrict__ nbig,
                                                const LeafGather &g) {
  const int b0 = start[leaf], m = start[leaf + 1] - b0;
  if (m > 128) {
    if (lane == 0 && big) big[atomicAdd(nbig, 1)] = leaf;
    return;
  }
  if (m == 0) return;
  if (m == 1) {
    if (lane == 0 && g.x) gather_one(g, g.loc32 ? leaf_centre(g, leaf) : make_double2(0, 0), b0, vals[b0]);
    return;
  }
  if (m <= 32) warp_sort_leaf<1>(b0, m, lane, keys, vals, g, leaf);
  else if (m <= 64) warp_sort_leaf<2>(b0, m, lane, keys, vals, g, leaf);
  else warp_sort_leaf<4>(b0, m, lane, keys, vals, g, leaf);
}

__global__ void __launch_bounds__(256)
leaf_sort_warp(const int *__restrict__ start, int nleaf, uint64_t *__restrict__ keys,
               int *__restrict__ vals, int *__restrict__ big, int *__restrict__ nbig,
               LeafGather g) {
  const int lane = threadIdx.x & 31;
  const int leaf = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (leaf >= nleaf) return;
  sort_small_leaf(leaf, lane, start, keys, vals, big, nbig, g);
}

// sort the leaf buckets of more than 128 points, one block per leaf (blocks
// skip the small leaves): up to kLeafSort points by a bitonic sort in shared
// memory; larger leaves in place in global memory by the bitonic network whose
// comparators all put the minimum at the lower index (each merge starts by
// comparing an element with its mirror in the block), so that the virtual
// +infinity padding up to the next power of two never moves into the leaf
// and comparators that touch it are skipped
constexpr int kLeafSort = 1024;

__device__ __forceinline__ void cmp_lo_hi(uint64_t *__restrict__ keys, int *__restrict__ vals,
                                          int lo, int hi) {
  const uint64_t ka = keys[lo], kb = keys[hi];
  const int va = vals[lo], vb = vals[hi];
  if (ka > kb || (ka == kb && va > vb)) {
    keys[lo] = kb;
    keys[hi] = ka;
    vals[lo] = vb;
    vals[hi] = va;
  }
}

__device__ void sort_leaf_global(uint64_t *__restrict__ keys, int *__restrict__ vals, int m) {
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  for (int kk = 2; kk <= np2; kk <<= 1) {
    // merge: element e of the lower half of each kk-block against its mirror
    for (int e = threadIdx.x; e < np2 / 2; e += blockDim.x) {
      const int lo = (e / (kk >> 1)) * kk + (e % (kk >> 1));
      const int hi = lo ^ (kk - 1);
      if (hi < m) cmp_lo_hi(keys, vals, lo, hi);
    }
    __threadfence_block();
    __syncthreads();
    for (int j = kk >> 2; j > 0; j >>= 1) {
      for (int e = threadIdx.x; e < np2 / 2; e += blockDim.x) {
        const int lo = (e / j) * 2 * j + (e % j);
        const int hi = lo + j;
        if (hi < m) cmp_lo_hi(keys, vals, lo, hi);
      }
      __threadfence_block();
      __syncthreads();
    }
  }
}
// one leaf of more than 128 points by the whole block (sk, sv: kLeafSort
// entries of shared memory)
__device__ void sort_big_leaf(int leaf, const int *__restrict__ start, uint64_t *__restrict__ keys,
                              int *__restrict__ vals, const LeafGather &g, uint64_t *sk, int *sv) {
  const int b0 = start[leaf], b1 = start[leaf + 1], m = b1 - b0;
  if (m <= 128) return;
  if (m > kLeafSort) {
    __syncthreads();
    sort_leaf_global(keys + b0, vals + b0, m);
    if (g.x) {
      const double2 c = g.loc32 ? leaf_centre(g, leaf) : make_double2(0, 0);
      for (int e = threadIdx.x; e < m; e += blockDim.x) gather_one(g, c, b0 + e, vals[b0 + e]);
    }
    return;
  }
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  __syncthreads();
  for (int e = threadIdx.x; e < np2; e += blockDim.x) {
    sk[e] = e < m ? keys[b0 + e] : ~0ull;
    sv[e] = e < m ? vals[b0 + e] : 0x7fffffff;
  }
  __syncthreads();
  for (int kk = 2; kk <= np2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int e = threadIdx.x; e < np2; e += blockDim.x) {
        int o = e ^ j;
        if (o > e) {
          bool up = (e & kk) == 0;
          uint64_t ka = sk[e], kb = sk[o];
          int va = sv[e], vb = sv[o];
          bool gt = ka > kb || (ka == kb && va > vb);
          if (gt == up) {
            sk[e] = kb; sk[o] = ka;
            sv[e] = vb; sv[o] = va;
          }
        }
      }
      __syncthreads();
    }
  }
  const double2 c = (g.x && g.loc32) ? leaf_centre(g, leaf) : make_double2(0, 0);
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    keys[b0 + e] = sk[e];
    vals[b0 + e] = sv[e];
    if (g.x) gather_one(g, c, b0 + e, sv[e]);
  }
}

__global__ void __launch_bounds__(256)
leaf_sort(const int *__restrict__ start, const int *__restrict__ big, const int *__restrict__ nbig,
          uint64_t *__restrict__ keys, int *__restrict__ vals, LeafGather g) {
  __shared__ uint64_t sk[kLeafSort];
  __shared__ int sv[kLeafSort];
  const int nb = *nbig;
  for (int bi = blockIdx.x; bi < nb; bi += gridDim.x) sort_big_leaf(big[bi], start, keys, vals, g, sk, sv);
}

// ---------------------------------------------------------------------------
// The tree build: six kernels at full occupancy, one thread per point or
// bucket, with nothing waiting for the host.  Buckets are the boxes of a
// level Hb >= H chosen so that they hold about four points each, so that
// sorting a bucket is a few comparisons in one thread.
//   k_tb_bbox     bounding-square partials per block (4 points a thread, warp
//                 shuffle reductions); the last block to finish
//                 reduces them, publishes the root square and the level
//                 geometry (and, for asynchronous rebuilds, the validity flags
//                 in the status word); the bucket counters are cleared
//   k_tb_keys     Morton keys; bucket counts (the atomic's return value is the
//                 point's slot in its bucket)
//   k_tb_scan     exclusive scan of the counts within chunks of kScanChunk
//                 buckets, chunk totals and maxima
//   k_tb_scatter  one thread per point, bucket and leaf: chunk offsets (each
//                 block scans the chunk totals); the point scattered into its
//                 bucket with its coordinates; bucket and leaf starts; leaf centres
//   k_tb_sort     one thread per point: its rank by (key, index) within its
//                 bucket of up to kTinyBucket points, then its outputs in tree
//                 order; larger buckets listed
//   k_tb_big      the listed buckets: a warp each up to 128 points, else a block
constexpr int kTinyBucket = 16;
constexpr int kScanChunk = 4096;  // buckets per block of the scan (1024 threads x 4)
constexpr int kBboxThreads = 256;
constexpr int kBboxPer = 8;  // points per thread and grid-stride step of k_tb_bbox

// a point in its bucket: one 32-byte record (a single full-sector store by
// the scatter, contiguous reads by the sort)
struct alignas(32) BRec {
  uint64_t key;
  int v, pad;  // caller index
  double x, y;
};
// key and caller index of a record: one 16-byte load
__device__ __forceinline__ void rec_kv(const BRec *r, uint64_t &k, int &v) {
  const uint4 u = *reinterpret_cast<const uint4 *>(r);
  k = ((uint64_t)u.y << 32) | u.x;
  v = (int)u.z;
}

struct TreeBuild {
  const double *x, *y;
  int64_t n;
  int H, nleaf;         // leaf level of the outputs, 4^H
  int Hb, nbucket;      // bucket level (>= H), 4^Hb
  int nchunk;           // nbucket / kScanChunk, rounded up
  double root_x0, root_side;
  double kabs;          // |kappa|: the I_n range check of an asynchronous rebuild
  int report;           // record invalid input / range in the status word
  double *geo;          // x0, side, invalid flag, 2^30 / side, largest bucket (int)
  DevGeom *dg;          // level geometry
  uint64_t *keys;       // sorted keys
  int *leaf_start;      // nleaf + 1
  LeafGather g;
  Geom *part;           // [bbox grid]
  unsigned *ticket;     // last-block counter of k_tb_bbox
  uint64_t *kb;         // [n] keys in input order
  BRec *rec;            // [n] the points bucketed: key, coordinates, caller index
  int *slot;            // [n] slot in the bucket
  int *bcount;          // [nbucket + 1]: counts, then chunk prefixes; [nbucket]: big buckets
  int *bstart;          // [nbucket + 1] bucket starts
  double2 *centre;      // [nleaf] leaf centres
  int *ctot;            // [2 nchunk]: chunk totals, chunk maxima
  int *big;             // [nbucket]
  int *status;
};

// one point into tree order, its coordinates (a, b) given (the leaf centre
// precomputed)
__device__ __forceinline__ void place_point(const LeafGather &g, double2 c, int k, int j, double a,
                                            double b) {
  if (g.xs) {
    g.xs[k] = a;
    g.ys[k] = b;
  }
  g.perm[k] = j;
  if (g.loc32) {
    const FsPair sx = fs_split(a - c.x), sy = fs_split(b - c.y);
    g.loc32[k] = make_float2(sx.hi, sy.hi);
    g.loclo[k] = make_float2(sx.lo, sy.lo);
    g.yabs[k] = fs_round(b);
  }
}

// the same, reading the coordinates of caller index j
__device__ __forceinline__ void gather_point(const LeafGather &g, double2 c, int k, int j) {
  place_point(g, c, k, j, g.x[j], g.y[j]);
}

// block-wide reduction of the bounding-square partials (warp shuffles, then
// the warps' results in shared memory); the block's result in lane 0 of warp 0
struct BoxAcc {
  long long xmn, xmx, ymx;
  int bad;
};
__device__ __forceinline__ BoxAcc box_reduce(BoxAcc v, BoxAcc *ws) {
  for (int o = 16; o > 0; o >>= 1) {
    v.xmn = min(v.xmn, __shfl_xor_sync(0xffffffffu, v.xmn, o));
    v.xmx = max(v.xmx, __shfl_xor_sync(0xffffffffu, v.xmx, o));
    v.ymx = max(v.ymx, __shfl_xor_sync(0xffffffffu, v.ymx, o));
    v.bad |= __shfl_xor_sync(0xffffffffu, v.bad, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? ws[lane] : BoxAcc{LLONG_MAX, LLONG_MIN, LLONG_MIN, 0};
    for (int o = 16; o > 0; o >>= 1) {
      v.xmn = min(v.xmn, __shfl_xor_sync(0xffffffffu, v.xmn, o));
      v.xmx = max(v.xmx, __shfl_xor_sync(0xffffffffu, v.xmx, o));
      v.ymx = max(v.ymx, __shfl_xor_sync(0xffffffffu, v.ymx, o));
      v.bad |= __shfl_xor_sync(0xffffffffu, v.bad, o);
    }
  }
  return v;
}

__global__ void __launch_bounds__(kBboxThreads)
k_tb_bbox(TreeBuild a) {
  __shared__ BoxAcc ws[kBboxThreads / 32];
  __shared__ int s_last;
  __shared__ double sg[4];
  pdl_trigger();
  const int64_t T = (int64_t)gridDim.x * kBboxThreads;
  const int64_t tid = (int64_t)blockIdx.x * kBboxThreads + threadIdx.x;
  // the bucket counters start at zero for k_tb_keys
  for (int64_t l = tid; l <= a.nbucket; l += T) a.bcount[l] = 0;
  // partials: order-preserving integer images of the doubles (min / max on
  // the integer pipe); kBboxPer independent loads a thread
  BoxAcc v{LLONG_MAX, LLONG_MIN, LLONG_MIN, 0};
  for (int64_t i0 = tid; i0 < a.n; i0 += T * kBboxPer) {
    long long u[kBboxPer], w[kBboxPer];
#pragma unroll
    for (int j = 0; j < kBboxPer; ++j) {
      const int64_t i = i0 + j * T;
      u[j] = i < a.n ? __double_as_longlong(a.x[i]) : 0ll;
      w[j] = i < a.n ? __double_as_longlong(a.y[i]) : 0x3ff0000000000000ll;  // 1.0
    }
#pragma unroll
    for (int j = 0; j < kBboxPer; ++j) {
      if (i0 + j * T >= a.n) continue;
      const bool fin = ((u[j] >> 52) & 0x7ff) != 0x7ff && ((w[j] >> 52) & 0x7ff) != 0x7ff;
      if (!fin || w[j] <= 0) v.bad = 1;
      const long long ku = u[j] >= 0 ? u[j] : (u[j] ^ 0x7fffffffffffffffll);
      v.xmn = min(v.xmn, ku);
      v.xmx = max(v.xmx, ku);
      v.ymx = max(v.ymx, w[j]);
    }
  }
  v = box_reduce(v, ws);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = Geom{dkey_inv(v.xmn), dkey_inv(v.xmx), dkey_inv(v.ymx), v.bad};
    __threadfence();
    s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // the last block: all partials, read past L1
  __threadfence();
  v = BoxAcc{LLONG_MAX, LLONG_MIN, LLONG_MIN, 0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kBboxThreads) {
    const volatile Geom *pg = a.part + b;
    const long long u = __double_as_longlong(pg->xmin), w = __double_as_longlong(pg->xmax);
    v.xmn = min(v.xmn, u >= 0 ? u : (u ^ 0x7fffffffffffffffll));
    v.xmx = max(v.xmx, w >= 0 ? w : (w ^ 0x7fffffffffffffffll));
    v.ymx = max(v.ymx, __double_as_longlong(pg->ymax));
    v.bad |= pg->bad;
  }
  __syncthreads();
  v = box_reduce(v, ws);
  if (threadIdx.x == 0) {
    *a.ticket = 0;  // ready for the next build
    const double xmin = dkey_inv(v.xmn), xmax = dkey_inv(v.xmx), ymax = dkey_inv(v.ymx);
    const double w = __dsub_rn(xmax, xmin);
    double L = (w > ymax) ? w : ymax;
    L = __dmul_rn(L, 1.0 + 0x1p-40);
    double x0 = xmin, flag = v.bad ? 1.0 : 0.0;
    if (a.root_side > 0) {  // caller's root square: it must contain the points
      const bool inside = a.root_x0 <= xmin && xmax <= a.root_x0 + a.root_side &&
                          ymax <= a.root_side;
      if (!inside && flag == 0.0) flag = 2.0;
      x0 = a.root_x0;
      L = a.root_side;
    }
    sg[0] = x0;
    sg[1] = L;
    sg[2] = flag;
    sg[3] = __ddiv_rn(1073741824.0, L);
    if (a.report) {
      if (flag != 0.0) atomicOr(a.status, HPFMM_DEV_EINVAL);
      else if (a.kabs * sqrt(5.0) * L > 60.0) atomicOr(a.status, HPFMM_DEV_RANGE);
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) a.geo[threadIdx.x] = sg[threadIdx.x];
  if (a.dg && threadIdx.x < 16) {
    const int l = threadIdx.x;
    const double d = ldexp(sg[1], -l);
    const float dh = (float)d;
    a.dg->d[l] = dh;
    a.dg->dlo[l] = (float)(d - (double)dh);
    a.dg->invd[l] = (float)(1.0 / d);
    a.dg->logd[l] = log(d);
    if (l == 0) {
      a.dg->x0 = sg[0];
      a.dg->side = sg[1];
      a.dg->qscale = sg[3];
    }
  }
}

__global__ void __launch_bounds__(256)
k_tb_keys(TreeBuild a) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double x0 = a.geo[0], L = a.geo[1], sc = a.geo[3];
  const uint64_t ix = quantise(__dsub_rn(a.x[i], x0), L, sc);
  const uint64_t iy = quantise(a.y[i], L, sc);
  const uint64_t k = spread1((uint32_t)ix) | (spread1((uint32_t)iy) << 1);
  a.kb[i] = k;
  a.slot[i] = atomicAdd(&a.bcount[k >> (60 - 2 * a.Hb)], 1);
}

__global__ void __launch_bounds__(1024)
k_tb_scan(TreeBuild a) {
  pdl_wait();
  pdl_trigger();
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kScanChunk + 4 * threadIdx.x;
  int v[4], sum = 0, mx = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = c0 + j < a.nbucket ? a.bcount[c0 + j] : 0;
    sum += v[j];
    mx = max(mx, v[j]);
  }
  int x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  int wpre = 0, tot = 0;
  for (int w = 0; w < 32; ++w) {
    if (w < warp) wpre += ws[w];
    tot += ws[w];
  }
  __syncthreads();
  if (lane == 0) ws[warp] = mx;
  __syncthreads();
  int run = wpre + x - sum;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (c0 + j < a.nbucket) a.bcount[c0 + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < 32; ++w) m = max(m, ws[w]);
    a.ctot[blockIdx.x] = tot;
    a.ctot[a.nchunk + blockIdx.x] = m;
  }
}

// chunk offsets in shared memory: the exclusive scan of the chunk totals
// (every block, nchunk <= kMaxChunks); returns the grand total, *mx the
// largest bucket
constexpr int kMaxChunks = 4096;
__device__ int chunk_offsets(const TreeBuild &a, int *off, int *ws, int *mx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (a.nchunk + blockDim.x - 1) / blockDim.x;
  const int t0 = min((int)threadIdx.x * per, a.nchunk), t1 = min(t0 + per, a.nchunk);
  int sum = 0, m = 0;
  for (int c = t0; c < t1; ++c) {
    sum += a.ctot[c];
    m = max(m, a.ctot[a.nchunk + c]);
  }
  int x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 31) ws[warp] = x;
  if (lane == 0) ws[32 + warp] = m;
  __syncthreads();
  int wpre = 0, tot = 0, mm = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < warp) wpre += ws[w];
    tot += ws[w];
    mm = max(mm, ws[32 + w]);
  }
  int run = wpre + x - sum;
  for (int c = t0; c < t1; ++c) {
    off[c] = run;
    run += a.ctot[c];
  }
  __syncthreads();
  *mx = mm;
  return tot;
}

__global__ void __launch_bounds__(256)
k_tb_scatter(TreeBuild a) {
  pdl_wait();
  pdl_trigger();
  __shared__ int off[kMaxChunks];
  __shared__ int ws[64];
  int maxbucket;
  const int total = chunk_offsets(a, off, ws, &maxbucket);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // point t into its bucket, with its coordinates
  if (t < a.n) {
    const uint64_t k = a.kb[t];
    const int bk = (int)(k >> (60 - 2 * a.Hb));
    const int pos = a.bcount[bk] + off[bk / kScanChunk] + a.slot[t];
    BRec r;
    r.key = k;
    r.x = a.x[t];
    r.y = a.y[t];
    r.v = (int)t;
    r.pad = 0;
    a.rec[pos] = r;
  }
  // bucket t's start (and its leaf's, for the first bucket of a leaf)
  const int lsh = 2 * (a.Hb - a.H);
  if (t < a.nbucket) {
    const int s0 = a.bcount[t] + off[t / kScanChunk];
    a.bstart[t] = s0;
    if ((t & ((1 << lsh) - 1)) == 0) a.leaf_start[t >> lsh] = s0;
  }
  if (t == 0) {
    a.bstart[a.nbucket] = total;
    a.leaf_start[a.nleaf] = total;
    int *mxp = (int *)(a.geo + 4);
    *mxp = maxbucket;
  }
  // leaf t's centre (double precision, explicit roundings)
  if (a.g.loc32 && t < a.nleaf)
    a.centre[t] = leaf_centre_at(a.geo[0], ldexp(a.geo[1], -a.H), box_ix((uint64_t)t),
                                 box_iy((uint64_t)t));
}

__global__ void __launch_bounds__(256)
k_tb_sort(TreeBuild a) {
  pdl_wait();
  pdl_trigger();
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // bucketed position
  if (q >= a.n) return;
  const BRec rq = a.rec[q];
  const uint64_t kq = rq.key;
  const int vq = rq.v;
  const int64_t bk = (int64_t)(kq >> (60 - 2 * a.Hb));
  const int b0 = a.bstart[bk], m = a.bstart[bk + 1] - b0;
  if (m > kTinyBucket) {  // listed once, by its first position
    if (q == b0) a.big[atomicAdd(a.bcount + a.nbucket, 1)] = (int)bk;
    return;
  }
  // rank by (key, index) among the bucket's points
  int r = 0;
  for (int i = b0; i < b0 + m; ++i) {
    uint64_t ki;
    int vi;
    rec_kv(a.rec + i, ki, vi);
    r += (ki < kq || (ki == kq && vi < vq)) ? 1 : 0;
  }
  const int k = b0 + r;
  a.keys[k] = kq;
  const double2 c = a.g.loc32 ? a.centre[kq >> (60 - 2 * a.H)] : make_double2(0.0, 0.0);
  place_point(a.g, c, k, vq, rq.x, rq.y);
}

// buckets of more than kTinyBucket points: sorted by a warp (up to 128
// points, bitonic network in registers) or by the block (up to kLeafSort in
// shared memory, larger ones in place in global memory, in the input-order
// key and slot arrays, free by then), then the sorted keys written and the
// points gathered into tree order
template <int E>
__device__ __forceinline__ void warp_sort_bucket(int b0, int m, int lane, const BRec *rec,
                                                 uint64_t *kout, const LeafGather &g,
                                                 const double2 *centre, int sh) {
  uint64_t k[E];
  int v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    k[e] = ~0ull;
    v[e] = 0x7fffffff;
    if (i < m) rec_kv(rec + b0 + i, k[e], v[e]);
  }
  warp_bitonic<E>(k, v, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    if (i < m) {
      kout[b0 + i] = k[e];
      gather_point(g, g.loc32 ? centre[k[e] >> sh] : make_double2(0.0, 0.0), b0 + i, v[e]);
    }
  }
}

__global__ void __launch_bounds__(256)
k_tb_big(TreeBuild a) {
  pdl_wait();
  pdl_trigger();  // the evaluation's charge gather may follow on the stream
  __shared__ uint64_t sk[kLeafSort];
  __shared__ int sv[kLeafSort];
  const int *maxb = (const int *)(a.geo + 4);
  if (*maxb <= kTinyBucket) return;
  const int nbig = a.bcount[a.nbucket];
  const int sh = 60 - 2 * a.H;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t bi = gw; bi < nbig; bi += nw) {
    const int bk = a.big[bi];
    const int b0 = a.bstart[bk], m = a.bstart[bk + 1] - b0;
    if (m > 128) continue;
    if (m <= 32) warp_sort_bucket<1>(b0, m, lane, a.rec, a.keys, a.g, a.centre, sh);
    else if (m <= 64) warp_sort_bucket<2>(b0, m, lane, a.rec, a.keys, a.g, a.centre, sh);
    else warp_sort_bucket<4>(b0, m, lane, a.rec, a.keys, a.g, a.centre, sh);
  }
  for (int bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
    const int bk = a.big[bi];
    const int b0 = a.bstart[bk], m = a.bstart[bk + 1] - b0;
    if (m <= 128) continue;
    __syncthreads();
    if (m > kLeafSort) {
      uint64_t *kw = a.kb + b0;
      int *vw = a.slot + b0;
      for (int e = threadIdx.x; e < m; e += blockDim.x) {
        rec_kv(a.rec + b0 + e, kw[e], vw[e]);
      }
      __threadfence_block();
      __syncthreads();
      sort_leaf_global(kw, vw, m);
      for (int e = threadIdx.x; e < m; e += blockDim.x) {
        const uint64_t k = kw[e];
        a.keys[b0 + e] = k;
        gather_point(a.g, a.g.loc32 ? a.centre[k >> sh] : make_double2(0.0, 0.0), b0 + e, vw[e]);
      }
      continue;
    }
    int np2 = 1;
    while (np2 < m) np2 <<= 1;
    for (int e = threadIdx.x; e < np2; e += blockDim.x) {
      sk[e] = ~0ull;
      sv[e] = 0x7fffffff;
      if (e < m) {
        uint64_t kk;
        int vv;
        rec_kv(a.rec + b0 + e, kk, vv);
        sk[e] = kk;
        sv[e] = vv;
      }
    }
    __syncthreads();
    for (int kk = 2; kk <= np2; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int e = threadIdx.x; e < np2; e += blockDim.x) {
          const int o = e ^ j;
          if (o > e) {
            const bool up = (e & kk) == 0;
            const uint64_t ka = sk[e], kb = sk[o];
            const int va = sv[e], vb = sv[o];
            const bool gt = ka > kb || (ka == kb && va > vb);
            if (gt == up) {
              sk[e] = kb; sk[o] = ka;
              sv[e] = vb; sv[o] = va;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
      a.keys[b0 + e] = sk[e];
      gather_point(a.g, a.g.loc32 ? a.centre[sk[e] >> sh] : make_double2(0.0, 0.0), b0 + e,
                   sv[e]);
    }
  }
}

}  // namespace

// Build (or rebuild) the tree of pl for the n points (x, y) (device pointers):
// the six kernels above on `st`.  Leaves pl->keys, perm, leaf_start, the
// tree-order coordinates (loc32 / loclo / yabs or xs / ys), pl->geo and
// pl->dgeom filled on the device.  The temporaries live in one workspace of
// the plan, allocated by the first build.  The host copies of the root square
// are set by tree_finish.
namespace {
struct TreeTmp {
  char *base = nullptr;
  Geom *part;
  uint64_t *kb;
  BRec *rec;
  int *slot, *bcount, *bstart, *ctot, *big;
  double2 *centre;
  int nbbox, Hb, nchunk;
};

// bucket level: about four points per bucket (level round(log4 n) - 1), at
// least the leaf level, at most level 11 (4M buckets) unless the leaves are
// deeper
int bucket_level(int64_t n, int H) {
  int hb = (int)floor(log((double)(n > 1 ? n : 1)) / log(4.0) + 0.5) - 1;
  if (hb > 11) hb = 11;
  return hb > H ? hb : H;
}
}  // namespace

static hpfmm_status tree_alloc(hpfmm_plan *pl, TreeTmp &t, cudaStream_t st) {
  const int64_t n = pl->n;
  const int nleaf = pl->nleaf;
  t.Hb = bucket_level(n, pl->Hsort);
  const size_t nb = size_t(1) << (2 * t.Hb);
  t.nchunk = (int)((nb + kScanChunk - 1) / kScanChunk);
  if (t.nchunk > kMaxChunks) {
    set_last_error("tree build: %d leaf levels exceed the bucket scan", pl->Hsort);
    return HPFMM_EUNSUPPORTED;
  }
  // one wave of bounding-square blocks: kBboxPer points a thread, at most
  // four blocks per SM (a grid-stride loop covers the rest)
  int64_t nbb = (n + kBboxPer * kBboxThreads - 1) / (kBboxPer * kBboxThreads);
  const int64_t cap = 4 * (int64_t)(pl->sms > 0 ? pl->sms : 1);
  t.nbbox = (int)(nbb < 1 ? 1 : (nbb > cap ? cap : nbb));
  size_t bytes = sizeof(Geom) * t.nbbox + sizeof(uint64_t) * n + sizeof(BRec) * n +
                 sizeof(int) * n +
                 sizeof(int) * (3 * nb + 3) + sizeof(double2) * (size_t)nleaf +
                 2 * sizeof(int) * (size_t)t.nchunk;
  bytes += 14 * 256;
  // the workspace stays with the plan: rebuilds of the same size reuse it
  if (!pl->tree_tmp || pl->tree_tmp_bytes < (int64_t)bytes) {
    if (pl->tree_tmp) {
      HP_CUDA(cudaStreamSynchronize(st));
      cudaFree(pl->tree_tmp);
      pl->workspace_bytes -= pl->tree_tmp_bytes;
      pl->tree_tmp = nullptr;
      pl->tree_tmp_bytes = 0;
    }
    HP_TRY(plan_dalloc(pl, &pl->tree_tmp, bytes));
    pl->tree_tmp_bytes = (int64_t)bytes;
  }
  t.base = (char *)pl->tree_tmp;
  char *c = t.base;
  auto carve = [&](size_t b) {
    char *r = c;
    c += (b + 255) & ~size_t(255);
    return r;
  };
  t.part = (Geom *)carve(sizeof(Geom) * t.nbbox);
  t.kb = (uint64_t *)carve(sizeof(uint64_t) * n);
  t.rec = (BRec *)carve(sizeof(BRec) * n);
  t.slot = (int *)carve(sizeof(int) * n);
  t.bcount = (int *)carve(sizeof(int) * (nb + 1));
  t.bstart = (int *)carve(sizeof(int) * (nb + 1));
  t.big = (int *)carve(sizeof(int) * (nb + 1));
  t.centre = (double2 *)carve(sizeof(double2) * (size_t)nleaf);
  t.ctot = (int *)carve(2 * sizeof(int) * (size_t)t.nchunk);
  return HPFMM_OK;
}

hpfmm_status tree_build(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st) {
  TreeTmp t;
  HP_TRY(tree_alloc(pl, t, st));
  TreeBuild a;
  a.x = x;
  a.y = y;
  a.n = pl->n;
  a.H = pl->Hsort;
  a.nleaf = pl->nleaf;
  a.Hb = t.Hb;
  a.nbucket = 1 << (2 * t.Hb);
  a.nchunk = t.nchunk;
  a.root_x0 = pl->root_x0;
  a.root_side = pl->root_side;
  a.kabs = sqrt(pl->kre * pl->kre + pl->kim * pl->kim);
  a.report = pl->async_update;
  a.geo = pl->geo;
  a.dg = pl->dgeom;
  a.keys = pl->keys;
  a.leaf_start = pl->leaf_start;
  // the sorts also put the points into tree order (permutation, coordinates);
  // adaptive plans: only the permutation, their leaf frames follow the
  // adaptive build
  a.g = pl->adaptive ? LeafGather{x, y, pl->geo, a.H, nullptr, nullptr, pl->perm, nullptr, nullptr,
                                  nullptr}
                     : LeafGather{x, y, pl->geo, a.H, pl->xs, pl->ys, pl->perm, pl->loc32,
                                  pl->yabs, pl->loclo};
  a.part = t.part;
  a.ticket = pl->tree_ctr;
  a.kb = t.kb;
  a.rec = t.rec;
  a.slot = t.slot;
  a.bcount = t.bcount;
  a.bstart = t.bstart;
  a.centre = t.centre;
  a.ctot = t.ctot;
  a.big = t.big;
  a.status = pl->status;
  const int64_t n = pl->n;
  const unsigned gp = (unsigned)((n + 255) / 256);
  const int64_t nitem = n > a.nbucket ? n : (int64_t)a.nbucket;
  const unsigned gs = (unsigned)((nitem + 255) / 256);
  pass_begin(pl, st, PASS_TREE);
  k_tb_bbox<<<t.nbbox, kBboxThreads, 0, st>>>(a);
  // the rest of the chain by programmatic dependent launches: each kernel is
  // scheduled while its predecessor's last blocks run and waits for it
  // (griddepcontrol) before reading its results
  cudaError_t le = launch_dependent(k_tb_keys, dim3(gp), dim3(256), 0, st, a);
  if (le == cudaSuccess) le = launch_dependent(k_tb_scan, dim3(t.nchunk), dim3(1024), 0, st, a);
  if (le == cudaSuccess) le = launch_dependent(k_tb_scatter, dim3(gs), dim3(256), 0, st, a);
  if (le == cudaSuccess) le = launch_dependent(k_tb_sort, dim3(gp), dim3(256), 0, st, a);
  if (le == cudaSuccess) le = launch_dependent(k_tb_big, dim3(608), dim3(256), 0, st, a);
  if (le != cudaSuccess) {
    set_last_error("tree_build launch: %s", cudaGetErrorString(le));
    return HPFMM_ECUDA;
  }
  // the reaction tables and the host copy of the root square start on the
  // table stream once the build is done: run during the build, their
  // FP64-bound blocks slowed its short kernels by a third; after it they
  // share the SMs with the near field, which leaves the FP64 pipe idle
  if (pl->ev_tree) {
    cudaError_t e = cudaEventRecord(pl->ev_tree, st);
    if (e != cudaSuccess) {
      set_last_error("tree_build: %s", cudaGetErrorString(e));
      return HPFMM_ECUDA;
    }
  }
  pass_end(pl, st, PASS_TREE, 6);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("tree_build launch: %s", cudaGetErrorString(e));
    return HPFMM_ECUDA;
  }
  return HPFMM_OK;
}

// With hgeo != nullptr (the geometry has reached the host): the invalid-input
// check and the host copies of the root square.  The build's workspace stays
// with the plan (freed with it).
hpfmm_status tree_finish(hpfmm_plan *pl, const double *hgeo, cudaStream_t) {
  hpfmm_status s = HPFMM_OK;
  if (hgeo) {
    if (hgeo[2] != 0.0) {
      set_last_error(hgeo[2] == 2.0 ? "the root square does not contain the points"
                                    : "points must be finite with y > 0");
      s = HPFMM_EINVAL;
    } else {
      pl->x0 = hgeo[0];
      pl->side = hgeo[1];
      pl->qscale = hgeo[3];
    }
  }
  return s;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the tree ordering, for callers that cannot call
// cudaMalloc (an embedding runtime that owns every device allocation and
// forbids others, or code that must not grow the device's memory use).  It
// runs the multi-kernel form of the ordering (bounding square, keys, leaf
// counts, scan, bucket scatter, per-leaf sorts; leaves of any size are sorted
// on the device) on up to kNoAllocMaxN points, with every temporary carved
// from one file-scope device array of kNoAllocBytes.  That array is part of
// the library image, so every GPU on which the library is loaded holds it
// until the process exits.
namespace {
constexpr int64_t kNoAllocMaxN = 65536;
constexpr int kNoAllocMaxLevels = 8;
constexpr size_t kNoAllocBytes = (size_t)2560 * 1024;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void write_perm(const int *__restrict__ v, int64_t n, int64_t *__restrict__ perm) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) perm[k] = v[k];
}

// device address of g_noalloc_scratch on device `dev` (current when called;
// host code only sees a host-side stand-in for the symbol); looked up once
// per device
void *noalloc_scratch_address(int dev) {
  static std::mutex mu;
  static void *addr[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

// device of a device pointer, -1 for anything else
int pointer_device(const void *p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? at.device : -1;
}
}  // namespace

extern "C" hpfmm_status hpfmm_tree_order_noalloc(const double *x, const double *y, int64_t n,
                                                 int levels, uint64_t *keys, int64_t *perm,
                                                 void *stream) {
  if (!x || !y || !keys || !perm || n < 1) {
    set_last_error("hpfmm_tree_order_noalloc: null pointer or n < 1");
    return HPFMM_EINVAL;
  }
  if (n > kNoAllocMaxN || levels < 1 || levels > kNoAllocMaxLevels) {
    set_last_error("hpfmm_tree_order_noalloc: needs n <= %lld and 1 <= levels <= %d "
                   "(got n = %lld, levels = %d)",
                   (long long)kNoAllocMaxN, kNoAllocMaxLevels, (long long)n, levels);
    return HPFMM_EINVAL;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("hpfmm_tree_order_noalloc: no current device");
    return HPFMM_ECUDA;
  }
  const int dx = pointer_device(x), dy = pointer_device(y), dk = pointer_device(keys),
            dp = pointer_device(perm);
  if (dx < 0 || dy < 0 || dk < 0 || dp < 0) {
    set_last_error("hpfmm_tree_order_noalloc: x, y, keys and perm must be device memory");
    return HPFMM_EINVAL;
  }
  if (dx != cur || dy != cur || dk != cur || dp != cur) {
    set_last_error("hpfmm_tree_order_noalloc: x, y, keys and perm must be on the current "
                   "device (%d)", cur);
    return HPFMM_EINVAL;
  }
  char *base = (char *)noalloc_scratch_address(cur);
  if (!base) {
    set_last_error("hpfmm_tree_order_noalloc: cannot resolve the scratch array's device address");
    return HPFMM_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int H = levels, nleaf = 1 << (2 * H);
  const int nbR = (int)((n + kRedThreads - 1) / kRedThreads);
  const int nsb = (nleaf + 1023) / 1024;
  char *c = base;
  auto carve = [&](size_t b) {
    char *r = c;
    c += (b + 255) & ~size_t(255);
    return r;
  };
  Geom *part = (Geom *)carve(sizeof(Geom) * nbR);
  double *geo = (double *)carve(8 * sizeof(double));
  uint64_t *kb = (uint64_t *)carve(sizeof(uint64_t) * n);
  int *va = (int *)carve(sizeof(int) * n);
  int *vb = (int *)carve(sizeof(int) * n);
  int *slot = (int *)carve(sizeof(int) * n);
  int *lcount = (int *)carve(sizeof(int) * ((size_t)nleaf + 1));  // [nleaf]: big-leaf count
  int *big = (int *)carve(sizeof(int) * ((size_t)nleaf + 1));
  int *lstart = (int *)carve(sizeof(int) * ((size_t)nleaf + 1));
  int *btot = (int *)carve(sizeof(int) * nsb);
  int *bmax = (int *)carve(sizeof(int) * nsb);
  if ((size_t)(c - base) > kNoAllocBytes) {
    set_last_error("hpfmm_tree_order_noalloc: scratch layout exceeds %zu bytes", kNoAllocBytes);
    return HPFMM_EUNSUPPORTED;
  }
  const unsigned gb = (unsigned)((n + 255) / 256);
  // the array keeps the previous call's contents: clear what must start at 0
  HP_CUDA(cudaMemsetAsync(lcount, 0, sizeof(int) * ((size_t)nleaf + 1), st));
  bbox_partial<<<nbR, kRedThreads, 0, st>>>(x, y, n, part);
  bbox_final<<<1, kRedThreads, 0, st>>>(part, nbR, geo, 0.0, 0.0);
  morton_keys<<<gb, 256, 0, st>>>(x, y, n, geo, H, kb, va, lcount, slot);
  scan_part<<<nsb, 1024, 0, st>>>(lcount, nleaf, lstart, btot, bmax);
  scan_top<<<1, 1024, 0, st>>>(btot, bmax, nsb, nleaf, lstart, (int *)(geo + 4));
  scan_add<<<nsb, 1024, 0, st>>>(btot, nleaf, lstart);
  bucket_scatter<<<gb, 256, 0, st>>>(kb, slot, n, H, lstart, keys, vb);
  // leaves of any size are sorted here: up to 128 points by a warp, up to
  // kLeafSort in shared memory, larger ones in place in global memory
  const LeafGather none{nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                        nullptr};
  leaf_sort_warp<<<(unsigned)(((int64_t)nleaf * 32 + 255) / 256), 256, 0, st>>>(
      lstart, nleaf, keys, vb, big, lcount + nleaf, none);
  leaf_sort<<<160, 256, 0, st>>>(lstart, big, lcount + nleaf, keys, vb, none);
  write_perm<<<gb, 256, 0, st>>>(vb, n, perm);
  HP_LAUNCH_CHECK();
  // the validity flag of the points comes back to the host: the call waits
  // for the stream
  double hgeo[5];
  HP_CUDA(cudaMemcpyAsync(hgeo, geo, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  if (hgeo[2] != 0.0) {
    set_last_error("hpfmm_tree_order_noalloc: points must be finite with y > 0");
    return HPFMM_EINVAL;
  }
  return HPFMM_OK;
}
