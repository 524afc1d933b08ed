// Adjoint of the interaction sum u = G q (Section 2.2, Eq. 1.2 with the
// image and reaction parts of Eq. reactioncomp1/reactioncomp2).
//
// For a real functional L of the complex potentials with cotangent
// g_i = dL/dRe u_i + i dL/dIm u_i, the gradient with respect to the real
// charges and positions is
//
//   dL/dq_j = sum_i Re(conj(g_i) G(r_i, r_j))
//   dL/dr_k = Re(conj(g_k) grad_k u[q](r_k)) + q_k sum_i Re(conj(g_i) grad_2 G(r_i, r_k)).
//
// The kernel is symmetric, G(r, r') = G(r', r) (Eq. greensfunsymm), so the
// transpose sums are forward sums with the real charge vectors Re g and Im g:
//
//   dL/dq_j = Re u[Re g](r_j) + Im u[Im g](r_j)
//   dL/dr_k = Re(conj(g_k) grad u[q](r_k)) + q_k (Re grad u[Re g](r_k) + Im grad u[Im g](r_k)).
//
// The self convention carries over: the free part skips i = j in both
// directions, the image and reaction parts keep the diagonal, whose
// derivative in r_k is the sum of the derivatives in both arguments (equal by
// symmetry).  So one adjoint is two (or, without the forward field, three)
// FMM evaluations on the plan's tree plus one elementwise combination.
#include "common.cuh"

namespace {

__global__ void k_adj_split(const double2 *__restrict__ g, int64_t n, double *__restrict__ gr,
                            double *__restrict__ gi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = g[i];
  gr[i] = v.x;
  gi[i] = v.y;
}

// pot_*: complex u[Re g], u[Im g]; grad_*: complex (d/dx, d/dy) of the same and
// of u[q]; all in caller (input) order
__global__ void k_adj_combine(int64_t n, const double *__restrict__ q,
                              const double2 *__restrict__ g, const double2 *__restrict__ gq,
                              const double2 *__restrict__ pot_r, const double2 *__restrict__ pot_i,
                              const double2 *__restrict__ grad_r,
                              const double2 *__restrict__ grad_i, double *__restrict__ dq,
                              double2 *__restrict__ dxy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (dq) dq[i] = pot_r[i].x + pot_i[i].y;
  if (dxy) {
    const double2 gv = g[i];
    const double qi = q[i];
    const double2 ax = gq[2 * i], ay = gq[2 * i + 1];
    const double2 rx = grad_r[2 * i], ry = grad_r[2 * i + 1];
    const double2 ix = grad_i[2 * i], iy = grad_i[2 * i + 1];
    double2 o;
    o.x = gv.x * ax.x + gv.y * ax.y + qi * (rx.x + ix.y);
    o.y = gv.x * ay.x + gv.y * ay.y + qi * (ry.x + iy.y);
    dxy[i] = o;
  }
}

}  // namespace

extern "C" hpfmm_status hpfmm_eval_adjoint(hpfmm_plan *pl, const double *q, const double *g,
                                           const double *grad_q, double *dq, double *dxy,
                                           void *stream) {
  if (!pl || !g || (!dq && !dxy) || (dxy && !q)) {
    set_last_error("hpfmm_eval_adjoint: need plan, g, an output, and q when dxy is wanted");
    return HPFMM_EINVAL;
  }
  const void *ptrs[] = {q, g, grad_q, dq, dxy};
  for (const void *p : ptrs)
    if (p && !is_device_pointer(p)) {
      set_last_error("hpfmm_eval_adjoint: all arrays must be device memory");
      return HPFMM_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = pl->n;
  if (!pl->adj) HP_TRY(plan_dalloc(pl, (void **)&pl->adj, sizeof(double) * 20 * (size_t)n));
  double *gr = pl->adj, *gi = gr + n;
  double *pot_r = gi + n, *pot_i = pot_r + 2 * n;
  double *grad_r = pot_i + 2 * n, *grad_i = grad_r + 4 * n;
  double *gq = grad_i + 4 * n, *pot_q = gq + 4 * n;
  const unsigned nb = (unsigned)((n + 255) / 256);
  k_adj_split<<<nb, 256, 0, st>>>((const double2 *)g, n, gr, gi);
  HP_LAUNCH_CHECK();
  // transpose sums = forward sums with the real charge vectors Re g, Im g
  HP_TRY(fmm_eval(pl, gr, pot_r, dxy ? grad_r : nullptr, st));
  HP_TRY(fmm_eval(pl, gi, pot_i, dxy ? grad_i : nullptr, st));
  if (dxy && !grad_q) {  // the forward field was not supplied: one more pass
    HP_TRY(fmm_eval(pl, q, pot_q, gq, st));
    grad_q = gq;
  }
  k_adj_combine<<<nb, 256, 0, st>>>(n, q, (const double2 *)g, (const double2 *)grad_q,
                                    (const double2 *)pot_r, (const double2 *)pot_i,
                                    (const double2 *)grad_r, (const double2 *)grad_i, dq,
                                    (double2 *)dxy);
  HP_LAUNCH_CHECK();
  return HPFMM_OK;
}
