// m2l_patch_lo.cu -- instances of the patch free-space M2L for p = 2 .. kPatchSplitP
// (see m2l_patch.cuh).
#include <mutex>

#include "m2l_patch.cuh"

bool m2l_patch_launch_lo(int p, int H, int lmin, int lmax, const DevGeom *dg, const cf *Tpad,
                         const cd *logt, const cf *M, cf *A, cf *B, int *status, cudaStream_t st,
                         int nr, RhsStride rs, const int *leaf_start, int skip_empty) {
  if (!Tpad) return false;
  switch (p) {
    case 2: return patch_launch_order<float, 3>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 3: return patch_launch_order<float, 4>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 4: return patch_launch_order<float, 5>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 5: return patch_launch_order<float, 6>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 6: return patch_launch_order<float, 7>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 7: return patch_launch_order<float, 8>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 8: return patch_launch_order<float, 9>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 9: return patch_launch_order<float, 10>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 10: return patch_launch_order<float, 11>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 11: return patch_launch_order<float, 12>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 12: return patch_launch_order<float, 13>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 13: return patch_launch_order<float, 14>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 14: return patch_launch_order<float, 15>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 15: return patch_launch_order<float, 16>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 16: return patch_launch_order<float, 17>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 17: return patch_launch_order<float, 18>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 18: return patch_launch_order<float, 19>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 19: return patch_launch_order<float, 20>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 20: return patch_launch_order<float, 21>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    default: return false;
  }
}
