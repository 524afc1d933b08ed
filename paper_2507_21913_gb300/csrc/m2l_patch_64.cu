// m2l_patch_64.cu -- double-precision instances of the patch free-space M2L
// (see m2l_patch.cuh) for p = 2 .. HPFMM_MAX_P: the plain double-precision
// path's M2L in Hankel form.
#include <mutex>
#include <utility>

#include "m2l_patch.cuh"

namespace {
template <int... Ps>
bool launch_64(int p, std::integer_sequence<int, Ps...>, int H, int lmin, int lmax,
               const DevGeom *dg, const cd *Tpad, const cd *logt, const cd *M, cd *A, cd *B,
               int *status, cudaStream_t st, int nr, RhsStride rs, const int *leaf_start,
               int skip_empty) {
  bool r = false;
  // orders 2 + Ps: the instance whose expansion length P1 = p + 1 matches
  (void)((p == Ps + 2 ? (r = patch_launch_order<double, Ps + 3>(H, lmin, lmax, dg, Tpad, logt, M,
                                                                A, B, status, st, nr, rs,
                                                                leaf_start, skip_empty),
                         true)
                      : false) ||
         ...);
  return r;
}
}  // namespace

bool m2l_patch_launch_64(int p, int H, int lmin, int lmax, const DevGeom *dg, const cd *Tpad,
                         const cd *logt, const cd *M, cd *A, cd *B, int *status, cudaStream_t st,
                         int nr, RhsStride rs, const int *leaf_start, int skip_empty) {
  if (!Tpad || p < 2 || p > HPFMM_MAX_P) return false;
  return launch_64(p, std::make_integer_sequence<int, HPFMM_MAX_P - 1>{}, H, lmin, lmax, dg,
                   Tpad, logt, M, A, B, status, st, nr, rs, leaf_start, skip_empty);
}
