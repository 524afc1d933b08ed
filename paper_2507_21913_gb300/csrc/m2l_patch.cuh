// m2l_patch.cuh -- the patch form of the free-space M2L (Eq. truncatedM2Lcoef
// for the log kernel, the classic 2-D form the paper's Remark reduces to),
// shared by the translation units that instantiate it for each expansion
// order (single precision: m2l_patch_lo.cu for p <= kPatchSplitP,
// m2l_patch_hi.cu for the higher orders; double precision: m2l_patch_64.cu),
// so that the instances compile in parallel.
#pragma once

#include <mutex>

#include "common.cuh"
#include "special.cuh"

// strides between the right-hand sides of a multi-RHS evaluation (blockIdx.y
// = RHS index): q in charges, m in expansion coefficients, out in doubles of
// the potential (the gradient has twice that)
struct RhsStride {
  int64_t q, m, out;
};

// orders up to kPatchSplitP are instantiated in m2l_patch_lo.cu, the rest up
// to HPFMM_MAX_P in m2l_patch_hi.cu; both return false when the order has no
// instance or its shared memory does not fit
constexpr int kPatchSplitP = 20;
// (levels lmin .. lmax of a tree with leaf level H in one launch)
bool m2l_patch_launch_lo(int p, int H, int lmin, int lmax, const DevGeom *dg, const cf *Tpad,
                         const cd *logt, const cf *M, cf *A, cf *B, int *status, cudaStream_t st,
                         int nr, RhsStride rs, const int *leaf_start, int skip_empty);
bool m2l_patch_launch_hi(int p, int H, int lmin, int lmax, const DevGeom *dg, const cf *Tpad,
                         const cd *logt, const cf *M, cf *A, cf *B, int *status, cudaStream_t st,
                         int nr, RhsStride rs, const int *leaf_start, int skip_empty);
// double precision, every order 2 .. HPFMM_MAX_P (m2l_patch_64.cu)
bool m2l_patch_launch_64(int p, int H, int lmin, int lmax, const DevGeom *dg, const cd *Tpad,
                         const cd *logt, const cd *M, cd *A, cd *B, int *status, cudaStream_t st,
                         int nr, RhsStride rs, const int *leaf_start, int skip_empty);

namespace {

// A block owns a patch of kPatch x kPatchRows parent boxes of one level;
// their four children of each type are its 128 targets, one per thread (warp
// w: child type w).  The block stages the (2 kPatch + 4) x (2 kPatchRows + 4)
// source boxes' multipoles and the 40 translation vectors once; then each
// thread applies the 27 V-list offsets of its child type to its target.
//
// A class translation in Hankel form is L'_r += sum_k g_{r+k} M'_k.  A
// thread holds its source's moments and a chunk of its outputs in registers
// and walks the anti-diagonals j = r + k: each g_j is read once per chunk (a
// warp-uniform broadcast, two per 16-byte load) and applied to every (r, k)
// of the chunk with r + k = j, the loop fully unrolled at compile time.  The
// output orders are split into chunks of at most about kDiagCmacs / (p + 1)
// rows, processed one after the other (each over all 27 offsets), so that the
// unrolled body stays small enough for the instruction cache at any order.
// All levels lmin..lmax are processed by one launch.
constexpr int kPatch = 8;      // parents per block in x
constexpr int kPatchRows = 4;  // parents per block in y
constexpr int kPatchThreads = 128;
constexpr int kDiagCmacs = 400;  // complex multiply-adds a chunk of output orders, per offset
constexpr int kPatchSrc = 2 * kPatch + 4;  // source boxes per block in x
constexpr int kSrcRows = 2 * kPatchRows + 4;  // source boxes per block in y
// 7 x 7 offset class (dy + 3) * 7 + (dx + 3) -> its index among the 40 far
// classes, -1 for the near 3 x 3
__constant__ signed char c_slot[49] = {
    0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15, -1, -1, -1, 16, 17, 18, 19, -1, -1,
    -1, 20, 21, 22, 23, -1, -1, -1, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39};

// output-order chunks of an order: about kDiagCmacs / P1 rows each (half that
// in double precision, whose values take twice the registers), balanced
template <typename R, int P1>
constexpr int diag_chunks() {
  constexpr int cm = sizeof(R) == 4 ? kDiagCmacs : kDiagCmacs / 2;
  constexpr int rows = cm / P1 > 0 ? cm / P1 : 1;
  return (P1 + rows - 1) / rows;
}

// the translations of one target for its output orders R0 .. R1 - 1, then
// their scaled values written to A and B (see k_m2l_free_patch)
template <typename R, int P1, int R0, int R1>
__device__ __forceinline__ void patch_target_rows(
    int a, int bb, int txA, int tyA, bool vA, bool skip_warp, bool skip_empty, int sx0, int sy0,
    const cpx<R> *Mp, const cpx<R> *Ts, const R *lg, const unsigned char *sempty,
    const R *fac_out, int64_t off, cpx<R> *__restrict__ A, cpx<R> *__restrict__ B) {
  constexpr int PP = (P1 + 1) & ~1;
  constexpr int PS = ((PP / 2) & 1) ? PP : PP + 2;
  constexpr int GP = 2 * P1;
  constexpr int HALF = kPatchSrc / 2;
  constexpr int NR = R1 - R0;
  cpx<R> acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = mk<R>(0, 0);
  for (int dy = -2 - bb; dy <= 3 - bb && !skip_warp; ++dy) {
    for (int dx = -2 - a; dx <= 3 - a; ++dx) {
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
      const int slot = c_slot[(dy + 3) * 7 + (dx + 3)];
      const int colA = txA + dx - sx0;
      const int cpA = (colA & 1) * HALF + (colA >> 1);
      const int sbA = (tyA + dy - sy0) * kPatchSrc + cpA;
      if (skip_empty && __all_sync(0xffffffffu, sempty[sbA])) continue;
      const cpx<R> *mA = Mp + sbA * PS;
      cpx<R> m[P1];
#pragma unroll
      for (int k = 0; k < P1; ++k) m[k] = mA[k];
      const cpx<R> *G = Ts + slot * GP;
      // anti-diagonals j = r + k of these rows, in aligned pairs
#pragma unroll
      for (int j = R0 & ~1; j <= R1 + P1 - 2; j += 2) {
        const cpx<R> g0 = G[j], g1 = G[j + 1];  // one 16-byte broadcast read
#pragma unroll
        for (int r = R0; r < R1; ++r) {
          if (j - r >= 0 && j - r < P1) cfma(acc[r - R0], g0, m[j - r]);
          if (j + 1 - r >= 0 && j + 1 - r < P1) cfma(acc[r - R0], g1, m[j + 1 - r]);
        }
      }
      // M_0 ln|t d| on Re L_0, in the scaled outputs (L_0 = -L'_0; M'_0 = M_0)
      if (R0 == 0) acc[0].x -= m[0].x * lg[slot];
    }
  }
  const R s = (R)(-0.5 / HP_TWO_PI);
  if (vA) {
    const size_t e0 = (size_t)(off + box_morton(txA, tyA)) * P1;
#pragma unroll
    for (int r = R0; r < R1; ++r) {
      const cpx<R> v = (s * fac_out[r]) * acc[r - R0];
      A[e0 + r] = v;
      B[e0 + r] = conj(v);
    }
  }
}

template <typename R, int P1, int NCH, int C>
__device__ __forceinline__ void patch_target_chunks(
    int a, int bb, int txA, int tyA, bool vA, bool skip_warp, bool skip_empty, int sx0, int sy0,
    const cpx<R> *Mp, const cpx<R> *Ts, const R *lg, const unsigned char *sempty,
    const R *fac_out, int64_t off, cpx<R> *__restrict__ A, cpx<R> *__restrict__ B) {
  patch_target_rows<R, P1, C * P1 / NCH, (C + 1) * P1 / NCH>(
      a, bb, txA, tyA, vA, skip_warp, skip_empty, sx0, sy0, Mp, Ts, lg, sempty, fac_out, off, A, B);
  if constexpr (C + 1 < NCH)
    patch_target_chunks<R, P1, NCH, C + 1>(a, bb, txA, tyA, vA, skip_warp, skip_empty, sx0, sy0,
                                           Mp, Ts, lg, sempty, fac_out, off, A, B);
}

template <typename R, int P1>
__global__ void __launch_bounds__(kPatchThreads)
k_m2l_free_patch(int H, int lmin, int lmax, const DevGeom *__restrict__ dg,
                 const cpx<R> *__restrict__ Tpad,
                 const cd *__restrict__ logt, const cpx<R> *__restrict__ M,
                 cpx<R> *__restrict__ A, cpx<R> *__restrict__ B, int *__restrict__ status,
                 RhsStride rs, const int *__restrict__ leaf_start, int skip_empty) {
  M += blockIdx.y * rs.m;
  A += blockIdx.y * rs.m;
  B += blockIdx.y * rs.m;
  // The translation of each class is applied in its Hankel form (see the
  // table builder): moments scaled by 16^k/k! when staged, T'[l][k] = g_{l+k},
  // outputs scaled by (-1)^{l+1} 16^l/l!.  Moment rows are padded to an even length
  // PP so that k, k+1 pairs are one 16-byte (single precision) shared-memory
  // load, and so are the (g_j, g_{j+1}) pairs of even j the anti-diagonal walk
  // reads.  The source patch is stored with even columns first, so that the
  // sources of a warp's x-consecutive targets (all of one column parity) are
  // consecutive boxes.  The row stride PS is an odd number of 16-byte units,
  // so that the 8 lanes of a quarter-warp (consecutive source boxes) hit 8
  // different bank groups with their 16-byte (k, k+1) loads.
  constexpr int PP = (P1 + 1) & ~1;
  constexpr int PS = ((PP / 2) & 1) ? PP : PP + 2;
  constexpr int GP = 2 * P1;
  constexpr int HALF = kPatchSrc / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ R fac_in[P1], fac_out[P1];  // 16^k / k!, (-1)^{l+1} 16^l / l!
  __shared__ unsigned char sempty[kPatchSrc * kSrcRows];  // source box holds no point
  cpx<R> *Ts = reinterpret_cast<cpx<R> *>(smem_raw);      // [40][GP]
  cpx<R> *Mp = Ts + 40 * GP;                               // [12][20][PS]
  R *lg = reinterpret_cast<R *>(Mp + kPatchSrc * kSrcRows * PS);  // [40] ln|t d|
  // level and patch of this block: kPatch x kPatchRows parents, whose four
  // children of each type are the block's targets (one per thread)
  int b = blockIdx.x, l = lmin;
  for (; l <= lmax; ++l) {
    const int nps = 1 << (l - 1);
    const int npx = nps / kPatch < 1 ? 1 : nps / kPatch, npy = nps / kPatchRows < 1 ? 1 : nps / kPatchRows;
    if (b < npx * npy) break;
    b -= npx * npy;
  }
  const int npx = (1 << (l - 1)) / kPatch < 1 ? 1 : (1 << (l - 1)) / kPatch;
  const int px0 = (b % npx) * kPatch, py0 = (b / npx) * kPatchRows;
  const int nparent_side = 1 << (l - 1), nside = 1 << l;
  const int64_t off = level_offset(l);
  const R logd = (R)dg->logd[l];
  // the 40 Hankel vectors by bulk copies (TMA) from the table ([40][2][GP]):
  // copy 0 of each class (16 p + 16 bytes, 16-byte aligned)
  const unsigned tbytes = (unsigned)(sizeof(cpx<R>) * 40 * GP);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, tbytes);
    for (int c = 0; c < 40; ++c)
      bulk_g2s(Ts + c * GP, Tpad + (size_t)c * 2 * GP, (unsigned)(sizeof(cpx<R>) * GP), &bar);
  }
  for (int c = threadIdx.x; c < 49; c += blockDim.x)
    if (c_slot[c] >= 0) lg[c_slot[c]] = (R)logt[c].x + logd;
  if (threadIdx.x < P1) {
    double f = 1.0;
    for (int i = 2; i <= (int)threadIdx.x; ++i) f *= (double)i;
    const double r = ldexp(1.0, kHankelLog2R * (int)threadIdx.x);
    fac_in[threadIdx.x] = (R)(r / f);
    fac_out[threadIdx.x] = (R)(((threadIdx.x & 1) ? r : -r) / f);
  }
  __syncthreads();
  // source patch: one box per thread and iteration, P1 independent loads each
  const int sx0 = 2 * px0 - 2, sy0 = 2 * py0 - 2;
  for (int sb = threadIdx.x; sb < kPatchSrc * kSrcRows; sb += blockDim.x) {
    const int row = sb / kPatchSrc, colp = sb % kPatchSrc;  // colp: parity-split column
    const int col = (colp < HALF) ? 2 * colp : 2 * (colp - HALF) + 1;
    const int sx = sx0 + col, sy = sy0 + row;
    cpx<R> *dst = Mp + (size_t)sb * PS;
    bool empty = true;
    if (sx >= 0 && sy >= 0 && sx < nside && sy < nside) {
      // points of the box: its leaves are contiguous in Morton order
      const uint64_t mb = box_morton(sx, sy);
      const int sh = 2 * (H - l);
      empty = leaf_start[(mb + 1) << sh] == leaf_start[mb << sh];
    }
    sempty[sb] = empty ? 1 : 0;
    if (sx >= 0 && sy >= 0 && sx < nside && sy < nside) {
      const cpx<R> *src = M + (size_t)(off + box_morton(sx, sy)) * P1;
      cpx<R> v[P1];
#pragma unroll
      for (int k = 0; k < P1; ++k) v[k] = src[k];
#pragma unroll
      for (int k = 0; k < P1; ++k) dst[k] = fac_in[k] * v[k];
    } else {
#pragma unroll
      for (int k = 0; k < P1; ++k) dst[k] = mk<R>(0, 0);
    }
    if (PP > P1) dst[PP - 1] = mk<R>(0, 0);
  }
  __syncthreads();  // also publishes the mbarrier initialisation
  if (!mbar_wait_bounded(&bar, 0)) {
    if (threadIdx.x == 0) atomicOr(status, HPFMM_DEV_TIMEOUT);
    mbar_wait_bounded(&bar, 0);  // give the copy a second bounded chance to land
    return;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = warp & 1, bb = warp >> 1;  // child type handled by this warp
  const int pxA = px0 + (lane & 7), pyA = py0 + (lane >> 3);
  const bool vA = pxA < nparent_side && pyA < nparent_side;
  const int txA = 2 * pxA + a, tyA = 2 * pyA + bb;
  // boxes holding no point need no local expansion (nothing is evaluated in
  // them or below them); a warp whose targets are all empty skips the
  // translations, and so does a warp whose sources of a class are all empty
  // (their moments are zero).  Not for evaluation at separate targets, which
  // may lie in empty boxes.
  bool tempty = true;
  if (skip_empty && vA) {
    const int sh = 2 * (H - l);
    const uint64_t mb = box_morton(txA, tyA);
    tempty = leaf_start[(mb + 1) << sh] == leaf_start[mb << sh];
  }
  const bool skip_warp = skip_empty && __all_sync(0xffffffffu, tempty);
  patch_target_chunks<R, P1, diag_chunks<R, P1>(), 0>(a, bb, txA, tyA, vA, skip_warp, skip_empty,
                                                   sx0, sy0, Mp, Ts, lg, sempty, fac_out, off, A,
                                                   B);
}

template <typename R, int P1>
size_t patch_smem() {
  constexpr int PP = (P1 + 1) & ~1;
  constexpr int PS = ((PP / 2) & 1) ? PP : PP + 2;
  return sizeof(cpx<R>) * (40 * 2 * P1 + kPatchSrc * kSrcRows * PS) + sizeof(R) * 40;
}

int patch_blocks(int lmin, int lmax) {
  int nb = 0;
  for (int l = lmin; l <= lmax; ++l) {
    const int nps = 1 << (l - 1);
    const int npx = nps / kPatch < 1 ? 1 : nps / kPatch, npy = nps / kPatchRows < 1 ? 1 : nps / kPatchRows;
    nb += npx * npy;
  }
  return nb;
}

// one order: sets the kernel's shared-memory limit once per device and
// launches; false when it does not fit
template <typename R, int P1>
bool patch_launch_order(int H, int lmin, int lmax, const DevGeom *dg, const cpx<R> *Tpad,
                        const cd *logt, const cpx<R> *M, cpx<R> *A, cpx<R> *B, int *status,
                        cudaStream_t st, int nr, RhsStride rs, const int *leaf_start,
                        int skip_empty) {
  static std::mutex mu;
  static signed char attr[64] = {};  // per device: 0 unknown, 1 set, -1 failed
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  const size_t sm = patch_smem<R, P1>();
  if (sm > 227 * 1024) return false;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (attr[dev] == 0) {
      const bool ok = cudaFuncSetAttribute(k_m2l_free_patch<R, P1>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm) == cudaSuccess;
      if (!ok) cudaGetLastError();
      attr[dev] = ok ? 1 : -1;
    }
    if (attr[dev] < 0) return false;
  }
  if (lmin < 2) lmin = 2;
  if (lmax < lmin) return true;  // no level to translate
  k_m2l_free_patch<R, P1><<<dim3(patch_blocks(lmin, lmax), nr), kPatchThreads, sm, st>>>(
      H, lmin, lmax, dg, Tpad, logt, M, A, B, status, rs, leaf_start, skip_empty);
  return true;
}

}  // namespace
