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
  float *yabs;  // y rounded to single precision (with loc32)
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
    g.loc32[k] = make_float2((float)(a - c.x), (float)(b - c.y));
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

__global__ void __launch_bounds__(256)
leaf_sort_warp(const int *__restrict__ start, int nleaf, uint64_t *__restrict__ keys,
               int *__restrict__ vals, int *__restrict__ big, int *__restrict__ nbig,
               LeafGather g) {
  const int lane = threadIdx.x & 31;
  const int leaf = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (leaf >= nleaf) return;
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
__global__ void __launch_bounds__(256)
leaf_sort(const int *__restrict__ start, const int *__restrict__ big, const int *__restrict__ nbig,
          uint64_t *__restrict__ keys, int *__restrict__ vals, LeafGather g) {
  __shared__ uint64_t sk[kLeafSort];
  __shared__ int sv[kLeafSort];
  const int nb = *nbig;
  for (int bi = blockIdx.x; bi < nb; bi += gridDim.x) {
    const int leaf = big[bi];
    int b0 = start[leaf], b1 = start[leaf + 1], m = b1 - b0;
    if (m <= 128) continue;
    if (m > kLeafSort) {
      __syncthreads();
      sort_leaf_global(keys + b0, vals + b0, m);
      if (g.x) {
        const double2 c = g.loc32 ? leaf_centre(g, leaf) : make_double2(0, 0);
        for (int e = threadIdx.x; e < m; e += blockDim.x) gather_one(g, c, b0 + e, vals[b0 + e]);
      }
      continue;
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
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint64 key, int value), 8-bit digits.
// A tile of kTile = 256 x 8 elements per block; elements are taken in rounds
// of 256 (one per thread, in order), so ranking by (round, warp, lane) keeps
// the input order among equal digits.
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kTile = kSortThreads * kSortRounds;
constexpr int kWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads)
radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int nblocks,
           unsigned *__restrict__ counts) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];  // digit-major
}

// exclusive scan of the per-block counts of each digit (block d scans row d of
// the digit-major table in place) and the digit totals
__global__ void __launch_bounds__(256)
radix_scan_digit(unsigned *__restrict__ counts, int nblocks, unsigned *__restrict__ totals) {
  __shared__ unsigned ws[8];
  unsigned *row = counts + (int64_t)blockIdx.x * nblocks;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned carry = 0;
  for (int base = 0; base < nblocks; base += 256) {
    int i = base + threadIdx.x;
    unsigned v = (i < nblocks) ? row[i] : 0u;
    unsigned x = v;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    unsigned wpre = 0, tot = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < warp) wpre += ws[w];
      tot += ws[w];
    }
    if (i < nblocks) row[i] = carry + wpre + x - v;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter(const uint64_t *__restrict__ kin, const int *__restrict__ vin, int64_t n, int shift,
              int nblocks, const unsigned *__restrict__ offs, const unsigned *__restrict__ totals,
              uint64_t *__restrict__ kout, int *__restrict__ vout) {
  __shared__ unsigned base_off[256];
  __shared__ unsigned whist[kWarps][256];
  __shared__ unsigned wsum[kWarps];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {  // digit base = exclusive prefix of the digit totals
    unsigned t = totals[threadIdx.x], x = t;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned pre = 0;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    base_off[threadIdx.x] = pre + x - t + offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  }
  int64_t tile = (int64_t)blockIdx.x * kTile;
  unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    for (int w = 0; w < kWarps; ++w) whist[w][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = tile + r * kSortThreads + threadIdx.x;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0;
    int val = valid ? vin[i] : 0;
    unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 256u;  // 256: no digit
    unsigned same = __match_any_sync(0xffffffffu, d);
    unsigned rank_in_warp = __popc(same & lt_mask);
    if (valid && rank_in_warp == 0) whist[warp][d] = __popc(same);
    __syncthreads();
    if (valid) {
      unsigned before = 0;
      for (int w = 0; w < warp; ++w) before += whist[w][d];
      unsigned pos = base_off[d] + before + rank_in_warp;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    unsigned tot = 0;
    for (int w = 0; w < kWarps; ++w) tot += whist[w][threadIdx.x];
    base_off[threadIdx.x] += tot;
    __syncthreads();
  }
}



}  // namespace

// Build (or rebuild) the tree of pl for the n points (x, y) (device pointers).
// Leaves pl->xs, ys, perm, keys, leaf_start, loc32 filled and pl->geo (x0,
// side, invalid flag, 2^30/side, largest leaf) on the device, and a copy of
// geo in the plan's pinned host buffer followed by the event ev_geo; the host
// values pl->x0 / side are set by tree_finish once that event has completed.
//
// Order: keys and leaf counts -> leaf offsets (scan) -> points bucketed by leaf
// -> each bucket sorted by (key, index).  The result is the stable order by
// (key, index) over all points.  Nothing waits for the host: leaves of any
// size are sorted on the device.
namespace {
struct TreeTmp {
  char *base = nullptr;
  Geom *part;
  uint64_t *kb;
  int *va, *vb, *slot, *lcount, *btot, *bmax, *big;
  unsigned *counts, *totals;
  int nbR, nblocks;
};
}  // namespace

static hpfmm_status tree_alloc(hpfmm_plan *pl, TreeTmp &t, cudaStream_t st) {
  const int64_t n = pl->n;
  const int nleaf = pl->nleaf;
  int64_t nbR64 = (n + kRedThreads - 1) / kRedThreads;
  t.nbR = nbR64 < 1024 ? (int)nbR64 : 1024;
  t.nblocks = (int)((n + kTile - 1) / kTile);
  const int nsb = (nleaf + 1023) / 1024;
  size_t bytes = sizeof(Geom) * t.nbR + sizeof(uint64_t) * n + 4 * sizeof(int) * n +
                 sizeof(int) * (2 * (size_t)nleaf + 2) + 2 * sizeof(int) * nsb +
                 sizeof(unsigned) * 256 * ((size_t)t.nblocks + 1);
  HP_CUDA(cudaMallocAsync((void **)&t.base, bytes + 13 * 256, st));
  char *c = t.base;
  auto carve = [&](size_t b) {
    char *r = c;
    c += (b + 255) & ~size_t(255);
    return r;
  };
  t.part = (Geom *)carve(sizeof(Geom) * t.nbR);
  t.kb = (uint64_t *)carve(sizeof(uint64_t) * n);
  t.va = (int *)carve(sizeof(int) * n);
  t.vb = (int *)carve(sizeof(int) * n);
  t.slot = (int *)carve(sizeof(int) * n);
  t.lcount = (int *)carve(sizeof(int) * ((size_t)nleaf + 1));  // [nleaf] = big-leaf count
  t.big = (int *)carve(sizeof(int) * ((size_t)nleaf + 1));
  t.btot = (int *)carve(sizeof(int) * nsb);
  t.bmax = (int *)carve(sizeof(int) * nsb);
  t.counts = (unsigned *)carve(sizeof(unsigned) * 256 * (size_t)t.nblocks);
  t.totals = (unsigned *)carve(sizeof(unsigned) * 256);
  return HPFMM_OK;
}

hpfmm_status tree_build(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st) {
  const int64_t n = pl->n;
  const int H = pl->Hsort, nleaf = pl->nleaf;
  TreeTmp t;
  HP_TRY(tree_alloc(pl, t, st));
  pl->tree_tmp_bytes = 0;
  int tb = 256;
  unsigned gb = (unsigned)((n + tb - 1) / tb);
  const int nsb = (nleaf + 1023) / 1024;
  double *geo = pl->geo;
  int *maxleaf = (int *)(geo + 4);
  pass_begin(pl, st, PASS_TREE);
  bbox_partial<<<t.nbR, kRedThreads, 0, st>>>(x, y, n, t.part);
  bbox_final<<<1, kRedThreads, 0, st>>>(t.part, t.nbR, geo, pl->root_x0, pl->root_side);
  // the geometry, for the host and for the table stream, is known from here on
  cudaError_t e = cudaSuccess;
  if (pl->hgeo) e = cudaMemcpyAsync(pl->hgeo, geo, 5 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && pl->ev_geo) e = cudaEventRecord(pl->ev_geo, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.lcount, 0, sizeof(int) * ((size_t)nleaf + 1), st);
  morton_keys<<<gb, tb, 0, st>>>(x, y, n, geo, H, t.kb, t.va, t.lcount, t.slot);
  scan_part<<<nsb, 1024, 0, st>>>(t.lcount, nleaf, pl->leaf_start, t.btot, t.bmax);
  scan_top<<<1, 1024, 0, st>>>(t.btot, t.bmax, nsb, nleaf, pl->leaf_start, maxleaf);
  scan_add<<<nsb, 1024, 0, st>>>(t.btot, nleaf, pl->leaf_start);
  bucket_scatter<<<gb, tb, 0, st>>>(t.kb, t.slot, n, H, pl->leaf_start, pl->keys, t.vb);
  // the leaf sorts also put the points into tree order (permutation, coordinates)
  // (adaptive plans: only the permutation; their leaf frames follow the adaptive build)
  const LeafGather lg = pl->adaptive
                            ? LeafGather{x, y, geo, H, nullptr, nullptr, pl->perm, nullptr, nullptr}
                            : LeafGather{x, y, geo, H, pl->xs, pl->ys, pl->perm, pl->loc32, pl->yabs};
  leaf_sort_warp<<<(unsigned)(((int64_t)nleaf * 32 + 255) / 256), 256, 0, st>>>(
      pl->leaf_start, nleaf, pl->keys, t.vb, t.big, t.lcount + nleaf, lg);
  leaf_sort<<<160, 256, 0, st>>>(pl->leaf_start, t.big, t.lcount + nleaf, pl->keys, t.vb, lg);
  pass_end(pl, st, PASS_TREE, 9);
  if (e == cudaSuccess) e = cudaGetLastError();
  // released (stream-ordered) by tree_finish
  pl->tree_tmp = t.base;
  if (e != cudaSuccess) {
    set_last_error("tree_build launch: %s", cudaGetErrorString(e));
    return HPFMM_ECUDA;
  }
  return HPFMM_OK;
}

// Once the geometry has reached the host (hgeo): invalid-input check, host
// copies of the root square, stream-ordered release of the temporaries.  Leaves
// of any size are sorted on the device, so nothing here waits for the sort.
hpfmm_status tree_finish(hpfmm_plan *pl, const double *hgeo, cudaStream_t st) {
  hpfmm_status s = HPFMM_OK;
  if (hgeo[2] != 0.0) {
    set_last_error(hgeo[2] == 2.0 ? "the root square does not contain the points"
                                  : "points must be finite with y > 0");
    s = HPFMM_EINVAL;
  } else {
    pl->x0 = hgeo[0];
    pl->side = hgeo[1];
    pl->qscale = hgeo[3];
  }
  if (pl->tree_tmp) cudaFreeAsync(pl->tree_tmp, st);
  pl->tree_tmp = nullptr;
  return s;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the tree ordering, for callers that cannot call
// cudaMalloc (for example code running inside a CUDA-graph capture that must
// not allocate, or an embedding runtime that owns every device allocation and
// forbids others).  It runs the same kernels as tree_build on up to
// kNoAllocMaxN points, with every temporary carved from one file-scope device
// array of kNoAllocBytes.  That array is part of the library image, so every
// GPU on which the library is loaded holds it until the process exits.
namespace {
constexpr int64_t kNoAllocMaxN = 65536;
constexpr int kNoAllocMaxLevels = 8;
constexpr size_t kNoAllocBytes = (size_t)2560 * 1024;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void write_perm(const int *__restrict__ v, int64_t n, int64_t *__restrict__ perm) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) perm[k] = v[k];
}

// device address of g_noalloc_scratch on the current device (host code only
// sees a host-side stand-in for the symbol); looked up once per device
void *noalloc_scratch_address() {
  static std::mutex mu;
  static void *addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
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
  if (!is_device_pointer(x) || !is_device_pointer(y) || !is_device_pointer(keys) ||
      !is_device_pointer(perm)) {
    set_last_error("hpfmm_tree_order_noalloc: x, y, keys and perm must be device memory");
    return HPFMM_EINVAL;
  }
  char *base = (char *)noalloc_scratch_address();
  if (!base) {
    set_last_error("hpfmm_tree_order_noalloc: cannot resolve the scratch array's device address");
    return HPFMM_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int H = levels, nleaf = 1 << (2 * H);
  const int nbR = (int)((n + kRedThreads - 1) / kRedThreads);
  const int nblocks = (int)((n + kTile - 1) / kTile);
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
  unsigned *counts = (unsigned *)carve(sizeof(unsigned) * 256 * (size_t)nblocks);
  unsigned *totals = (unsigned *)carve(sizeof(unsigned) * 256);
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
  const LeafGather none{nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
  leaf_sort_warp<<<(unsigned)(((int64_t)nleaf * 32 + 255) / 256), 256, 0, st>>>(
      lstart, nleaf, keys, vb, big, lcount + nleaf, none);
  leaf_sort<<<160, 256, 0, st>>>(lstart, big, lcount + nleaf, keys, vb, none);
  HP_LAUNCH_CHECK();
  double hgeo[5];
  HP_CUDA(cudaMemcpyAsync(hgeo, geo, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  HP_CUDA(cudaStreamSynchronize(st));
  if (hgeo[2] != 0.0) {
    set_last_error("hpfmm_tree_order_noalloc: points must be finite with y > 0");
    return HPFMM_EINVAL;
  }
  int hmax = 0;
  memcpy(&hmax, &hgeo[4], sizeof(int));
  const int *sorted = vb;
  if (hmax > kLeafSort) {  // a leaf too large for the in-block sort: full radix sort
    morton_keys<<<gb, 256, 0, st>>>(x, y, n, geo, H, kb, va, nullptr, nullptr);
    uint64_t *kin = kb, *kout = keys;
    int *vin = va, *vout = vb;
    for (int shift = 0; shift < 60; shift += 8) {
      radix_hist<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, nblocks, counts);
      radix_scan_digit<<<256, 256, 0, st>>>(counts, nblocks, totals);
      radix_scatter<<<nblocks, kSortThreads, 0, st>>>(kin, vin, n, shift, nblocks, counts, totals,
                                                       kout, vout);
      uint64_t *tk = kin; kin = kout; kout = tk;
      int *tv = vin; vin = vout; vout = tv;
    }
    HP_CUDA(cudaMemcpyAsync(keys, kb, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
    sorted = va;
  }
  write_perm<<<gb, 256, 0, st>>>(sorted, n, perm);
  HP_LAUNCH_CHECK();
  return HPFMM_OK;
}
