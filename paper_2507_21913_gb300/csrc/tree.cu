// tree.cu -- tree construction of Algorithm 1 ("generate an adaptive
// hierarchical tree structure with target points and image source points"):
// the points define a square [x0, x0+L] x [0, L] whose lower edge is the
// boundary y = 0; the image sources fill its mirror [x0, x0+L] x [-L, 0], so
// one quadtree over the points serves both (the mirror tree is its
// reflection).  Steps: validation and bounding square (reduction), 60-bit
// Morton keys (30 bits per axis, bit-exact rule), stable LSD radix sort of
// (key, index), leaf offsets of the uniform level-H grid, gathers.
#include <math.h>

#include "common.cuh"

namespace {

struct Geom {
  double xmin, xmax, ymax;
  int bad;  // non-finite or y <= 0 seen
};

constexpr int kRedThreads = 256;

__global__ void bbox_partial(const double *__restrict__ x, const double *__restrict__ y,
                             int64_t n, Geom *__restrict__ part) {
  __shared__ double s0[kRedThreads], s1[kRedThreads], s2[kRedThreads];
  __shared__ int sb[kRedThreads];
  double xmn = INFINITY, xmx = -INFINITY, ymx = -INFINITY;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double a = x[i], b = y[i];
    if (!isfinite(a) || !isfinite(b) || !(b > 0.0)) bad = 1;
    xmn = fmin(xmn, a);
    xmx = fmax(xmx, a);
    ymx = fmax(ymx, b);
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
  if (threadIdx.x == 0) part[blockIdx.x] = Geom{s0[0], s1[0], s2[0], sb[0]};
}

// final reduction; geo[0] = x0, geo[1] = L (side), ((int*)(geo+2))[0] = bad
__global__ void bbox_final(const Geom *__restrict__ part, int nb, double *__restrict__ geo) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Geom g{INFINITY, -INFINITY, -INFINITY, 0};
  for (int b = 0; b < nb; ++b) {
    g.xmin = fmin(g.xmin, part[b].xmin);
    g.xmax = fmax(g.xmax, part[b].xmax);
    g.ymax = fmax(g.ymax, part[b].ymax);
    g.bad |= part[b].bad;
  }
  double w = __dsub_rn(g.xmax, g.xmin);
  double L = (w > g.ymax) ? w : g.ymax;
  L = __dmul_rn(L, 1.0 + 0x1p-40);
  geo[0] = g.xmin;
  geo[1] = L;
  geo[2] = g.bad ? 1.0 : 0.0;
}

// ix = min(floor((x - x0) / L * 2^30), 2^30 - 1), every operation correctly
// rounded and uncontracted so that the result matches a plain IEEE host
// computation bit for bit
__device__ __forceinline__ uint64_t quantise(double v, double L) {
  double q = __ddiv_rn(v, L);
  double s = __dmul_rn(q, 1073741824.0);
  double f = floor(s);
  f = fmax(f, 0.0);
  f = fmin(f, 1073741823.0);
  return (uint64_t)f;
}

__global__ void morton_keys(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                            const double *__restrict__ geo, uint64_t *__restrict__ keys,
                            int *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x0 = geo[0], L = geo[1];
  uint64_t ix = quantise(__dsub_rn(x[i], x0), L);
  uint64_t iy = quantise(y[i], L);
  keys[i] = spread1((uint32_t)ix) | (spread1((uint32_t)iy) << 1);
  idx[i] = (int)i;
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

// leaf_start[b] = first sorted position whose level-H box index is >= b
__global__ void leaf_offsets(const uint64_t *__restrict__ keys, int64_t n, int H, int nleaf,
                             int *__restrict__ start) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > nleaf) return;
  int shift = 60 - 2 * H;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)(keys[mid] >> shift) < b) lo = mid + 1;
    else hi = mid;
  }
  start[b] = (int)lo;
}

__global__ void gather_points(const double *__restrict__ x, const double *__restrict__ y,
                              const int *__restrict__ idx, const uint64_t *__restrict__ keys,
                              int64_t n, int H, const double *__restrict__ geo,
                              double *__restrict__ xs, double *__restrict__ ys,
                              int64_t *__restrict__ perm, float2 *__restrict__ loc32) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int j = idx[k];
  double a = x[j], b = y[j];
  xs[k] = a;
  ys[k] = b;
  perm[k] = j;
  if (loc32) {
    uint64_t leaf = keys[k] >> (60 - 2 * H);
    double d = geo[1] / (double)(1 << H);
    double cx = geo[0] + (box_ix(leaf) + 0.5) * d, cy = (box_iy(leaf) + 0.5) * d;
    loc32[k] = make_float2((float)(a - cx), (float)(b - cy));
  }
}

}  // namespace

// Build (or rebuild) the tree of pl for the n points (x, y) (device pointers).
// Leaves pl->xs, ys, perm, keys, leaf_start, loc32 filled and pl->x0, side set;
// returns EINVAL (synchronously) for non-finite input or y <= 0.
hpfmm_status tree_build(hpfmm_plan *pl, const double *x, const double *y, cudaStream_t st) {
  const int64_t n = pl->n;
  int64_t nbR64 = (n + kRedThreads - 1) / kRedThreads;
  int nbR = nbR64 < 1024 ? (int)nbR64 : 1024;
  Geom *part = nullptr;
  double *geo = nullptr;
  uint64_t *kb = nullptr;
  int *va = nullptr, *vb = nullptr;
  unsigned *counts = nullptr;
  int nblocks = (int)((n + kTile - 1) / kTile);
  size_t bytes = sizeof(Geom) * nbR + 4 * sizeof(double) + sizeof(uint64_t) * n +
                 2 * sizeof(int) * n + sizeof(unsigned) * 256 * ((size_t)nblocks + 1);
  char *tmp = nullptr;
  HP_CUDA(cudaMallocAsync((void **)&tmp, bytes + 7 * 256, st));
  char *c = tmp;
  auto carve = [&](size_t b) {
    char *r = c;
    c += (b + 255) & ~size_t(255);
    return r;
  };
  part = (Geom *)carve(sizeof(Geom) * nbR);
  geo = (double *)carve(4 * sizeof(double));
  kb = (uint64_t *)carve(sizeof(uint64_t) * n);
  va = (int *)carve(sizeof(int) * n);
  vb = (int *)carve(sizeof(int) * n);
  counts = (unsigned *)carve(sizeof(unsigned) * 256 * (size_t)nblocks);
  unsigned *totals = (unsigned *)carve(sizeof(unsigned) * 256);

  hpfmm_status status = HPFMM_OK;
  double hgeo[3];
  pass_begin(pl, st, PASS_TREE);
  bbox_partial<<<nbR, kRedThreads, 0, st>>>(x, y, n, part);
  bbox_final<<<1, 32, 0, st>>>(part, nbR, geo);
  cudaError_t e = cudaMemcpyAsync(hgeo, geo, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error("tree_build: %s", cudaGetErrorString(e));
    cudaFreeAsync(tmp, st);
    return HPFMM_ECUDA;
  }
  if (hgeo[2] != 0.0) {
    pass_end(pl, st, PASS_TREE, 2);
    set_last_error("points must be finite with y > 0");
    cudaFreeAsync(tmp, st);
    return HPFMM_EINVAL;
  }
  pl->x0 = hgeo[0];
  pl->side = hgeo[1];
  if (!(pl->side > 0)) pl->side = 1.0;  // single point: any square will do

  int tb = 256;
  unsigned gb = (unsigned)((n + tb - 1) / tb);
  morton_keys<<<gb, tb, 0, st>>>(x, y, n, geo, pl->keys, va);
  uint64_t *kin = pl->keys, *kout = kb;
  int *vin = va, *vout = vb;
  for (int shift = 0; shift < 60; shift += 8) {
    radix_hist<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, nblocks, counts);
    radix_scan_digit<<<256, 256, 0, st>>>(counts, nblocks, totals);
    radix_scatter<<<nblocks, kSortThreads, 0, st>>>(kin, vin, n, shift, nblocks, counts, totals,
                                                     kout, vout);
    uint64_t *tk = kin; kin = kout; kout = tk;
    int *tv = vin; vin = vout; vout = tv;
  }
  // 8 passes: the sorted data is back in pl->keys / va
  leaf_offsets<<<(pl->nleaf + 1 + 255) / 256, 256, 0, st>>>(pl->keys, n, pl->H, pl->nleaf,
                                                            pl->leaf_start);
  gather_points<<<gb, tb, 0, st>>>(x, y, vin, pl->keys, n, pl->H, geo, pl->xs, pl->ys, pl->perm,
                                   pl->loc32);
  pass_end(pl, st, PASS_TREE, 2 + 1 + 3 * 8 + 2);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("tree_build launch: %s", cudaGetErrorString(e));
    status = HPFMM_ECUDA;
  }
  cudaFreeAsync(tmp, st);
  return status;
}
