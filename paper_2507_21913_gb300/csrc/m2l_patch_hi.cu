// m2l_patch_hi.cu -- instances of the patch free-space M2L for p = kPatchSplitP + 1 .. HPFMM_MAX_P
// (see m2l_patch.cuh).
#include <mutex>

#include "m2l_patch.cuh"

bool m2l_patch_launch_hi(int p, int H, int lmin, int lmax, const DevGeom *dg, const cf *Tpad,
                         const cd *logt, const cf *M, cf *A, cf *B, int *status, cudaStream_t st,
                         int nr, RhsStride rs, const int *leaf_start, int skip_empty) {
  if (!Tpad) return false;
  switch (p) {
    case 21: return patch_launch_order<float, 22>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 22: return patch_launch_order<float, 23>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 23: return patch_launch_order<float, 24>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 24: return patch_launch_order<float, 25>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 25: return patch_launch_order<float, 26>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 26: return patch_launch_order<float, 27>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 27: return patch_launch_order<float, 28>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 28: return patch_launch_order<float, 29>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 29: return patch_launch_order<float, 30>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 30: return patch_launch_order<float, 31>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 31: return patch_launch_order<float, 32>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 32: return patch_launch_order<float, 33>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 33: return patch_launch_order<float, 34>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 34: return patch_launch_order<float, 35>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 35: return patch_launch_order<float, 36>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 36: return patch_launch_order<float, 37>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 37: return patch_launch_order<float, 38>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 38: return patch_launch_order<float, 39>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 39: return patch_launch_order<float, 40>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    case 40: return patch_launch_order<float, 41>(H, lmin, lmax, dg, Tpad, logt, M, A, B, status, st,
                                           nr, rs, leaf_start, skip_empty);
    default: return false;
  }
}
