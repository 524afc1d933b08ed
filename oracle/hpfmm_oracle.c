/*
 * hpfmm_oracle.c -- plain, slow, FP64 CPU oracle for the half-plane Robin
 * Laplace interaction sum (arXiv 2507.21913).  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA path.
 *
 * What it computes (Section 2.2, Eqs. potential1 / 1.2 / reactioncomp1 /
 * reactioncomp2):
 *
 *   u(r_i) =  sum_{j != i} Q_j (-1/2pi) ln|r_i - r_j|            (free part)
 *          +  sum_j        Q_j (+1/2pi) ln|r_i - r_j^im|         (image part)
 *          +  sum_j        Q_j [ I_0(X, Y) + I_0(-X, Y) ]        (reaction)
 *   X = x_i - x_j,  Y = y_i + y_j,  r_j^im = (x_j, -y_j)
 *
 * with I_n from Eq. generalintegral,
 *   I_n(x, y) = 1/(2 pi n!) int_0^inf e^{-lambda (y - i x)} lambda^n /
 *               (lambda - kappa) d lambda,
 * where for real kappa the lambda path passes below the pole (limiting
 * absorption, Eq. dzGreensfunimplossless).
 *
 * I_n is evaluated by adaptive Gauss-Kronrod (7/15) quadrature after the
 * substitution t = lambda s, s = y - i x, used in the proof of Lemma 3.2 and
 * in Appendix A:  I_n = J_n(P) / (2 pi n! s^n),  P = kappa s,
 *   J_n(P) = int_S t^n e^{-t} / (t - P) dt
 *          = int_0^inf t^n e^{-t}/(t - P) dt + 2 pi i H(P) P^n e^{-P},
 * H = 1 if Im P < 0 (the pole lies between S and the real axis, Appendix A
 * case (d)), 1/2 if Im P = 0 (the lossless path passes below the pole:
 * principal value plus half residue, Appendix A case (c)), 0 if Im P > 0.
 * When the pole is close to the positive real axis it is subtracted on
 * [0, 2 Re P] so that the integrand stays smooth.
 *
 * The Morton ordering (bounding square, 30-bit quantisation per axis,
 * bit-interleaved key, stable sort by (key, index)) is the tree ordering of
 * Algorithm 1's tree-building step; it is written here independently so that
 * the device ordering can be checked bit for bit.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (see build.py).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define TWO_PI 6.283185307179586476925286766559
#define PI_ 3.141592653589793238462643383280

/* ------------------------------------------------------------------------ */
/* Gauss-Kronrod 7/15 rule on [-1, 1]: Kronrod abscissae (the odd-indexed ones
 * are the 7-point Gauss abscissae), Kronrod weights, Gauss weights.  These
 * are the standard published values; the test suite checks the rules'
 * polynomial exactness (degree 22 for Kronrod, 13 for Gauss).               */
static const double gk_x[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double gk_wk[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

/* exported so the tests can check the rule itself */
void hpo_gk15_rule(double *x, double *wk, double *wg) {
  memcpy(x, gk_x, sizeof gk_x);
  memcpy(wk, gk_wk, sizeof gk_wk);
  memcpy(wg, gk_wg, sizeof gk_wg);
}

/* Vector integrand: m complex components, one per order n in [n0, n0+m). */
typedef struct {
  cplx P;       /* pole position kappa * s                               */
  cplx fP[96];  /* P^n e^{-P} for the subtracted form                     */
  cplx eP;      /* e^{-P}                                                 */
  int n0, m;
  int subtract; /* integrand (f(t) - f(P))/(t - P) instead of f(t)/(t-P) */
  int capped;   /* set when the panel budget ran out                      */
} integrand_t;

/* phi(h) = (e^{-h} - 1)/h, by its Taylor series when |h| is small. */
static cplx phi_em1(cplx h) {
  if (cabs(h) < 0.1) {
    cplx s = 0.0;
    double f = 1.0;
    for (int k = 15; k >= 1; --k) {
      f = 1.0;
      for (int j = 2; j <= k; ++j) f *= j; /* k! */
      s = s * h + ((k & 1) ? -1.0 : 1.0) / f;
    }
    return s;
  }
  return (cexp(-h) - 1.0) / h;
}

static void eval_integrand(const integrand_t *g, double t, cplx *out) {
  int nmax = g->n0 + g->m - 1;
  if (g->subtract && cabs(t - g->P) < 1.0) {
    /* Close to the pole:
     * (t^n e^{-t} - P^n e^{-P}) / (t - P)
     *   = t^n e^{-P} phi(t - P) + e^{-P} S_n,  S_n = sum_{k<n} t^k P^{n-1-k},
     * which has no cancellation as t approaches P (the two terms differ in
     * size by at most a factor e^{|t-P|}).                                 */
    cplx E = g->eP * phi_em1(t - g->P);
    double tn = 1.0;
    cplx S = 0.0, Pn = 1.0;
    for (int n = 0; n <= nmax; ++n) {
      if (n >= g->n0) out[n - g->n0] = tn * E + g->eP * S;
      S = Pn + t * S;
      Pn *= g->P;
      tn *= t;
    }
    return;
  }
  if (g->subtract) { /* away from the pole: the plain divided difference */
    double e = exp(-t);
    double tn = (g->n0 == 0) ? 1.0 : pow(t, (double)g->n0);
    cplx inv = 1.0 / (t - g->P);
    for (int c = 0; c < g->m; ++c) {
      out[c] = (tn * e - g->fP[c]) * inv;
      tn *= t;
    }
    return;
  }
  double e = exp(-t);
  double tn = (g->n0 == 0) ? 1.0 : pow(t, (double)g->n0);
  cplx inv = 1.0 / (t - g->P);
  for (int c = 0; c < g->m; ++c) {
    out[c] = (tn * e) * inv; /* t^n e^{-t} / (t - P) */
    tn *= t;
  }
}

static void gk15(const integrand_t *g, double a, double b, cplx *K, cplx *G) {
  double h = 0.5 * (b - a), c = 0.5 * (a + b);
  cplx f1[96], f2[96];
  int m = g->m;
  for (int k = 0; k < m; ++k) { K[k] = 0; G[k] = 0; }
  for (int i = 0; i < 7; ++i) {
    double dx = h * gk_x[i];
    eval_integrand(g, c - dx, f1);
    eval_integrand(g, c + dx, f2);
    for (int k = 0; k < m; ++k) {
      cplx s = f1[k] + f2[k];
      K[k] += gk_wk[i] * s;
      if (i & 1) G[k] += gk_wg[i >> 1] * s;
    }
  }
  eval_integrand(g, c, f1);
  for (int k = 0; k < m; ++k) {
    K[k] += gk_wk[7] * f1[k];
    G[k] += gk_wg[3] * f1[k];
    K[k] *= h;
    G[k] *= h;
  }
}

/* Recursive bisection: accept a panel when every component's Gauss/Kronrod
 * difference is below rtol*|K| or below the absolute floor for that
 * component.  Depth is capped; the cap is never reached for the tested
 * arguments (the tests compare against closed forms to ~1e-13).           */
static void adapt(const integrand_t *g, double a, double b, const double *floor_,
                  int depth, long *budget, cplx *acc) {
  cplx K[96], G[96];
  gk15(g, a, b, K, G);
  --*budget;
  int ok = 1;
  for (int k = 0; k < g->m && ok; ++k) {
    double err = cabs(K[k] - G[k]);
    if (err > 1e-14 * cabs(K[k]) && err > floor_[k]) ok = 0;
  }
  if (ok || depth >= 60 || *budget <= 0) {
    for (int k = 0; k < g->m; ++k) acc[k] += K[k];
    return;
  }
  double mid = 0.5 * (a + b);
  adapt(g, a, mid, floor_, depth + 1, budget, acc);
  adapt(g, mid, b, floor_, depth + 1, budget, acc);
}

/* Integrate over consecutive breakpoints; the absolute floor for each
 * component is 1e-17 times a first coarse estimate of its magnitude.  At
 * most 200000 panels per call: g->capped records that the budget ran out
 * (never observed for the tested arguments).                             */
static void integrate(integrand_t *g, const double *bp, int nbp, cplx *acc) {
  long budget = 200000;
  cplx K[96], G[96];
  double floor_[96];
  for (int k = 0; k < g->m; ++k) { acc[k] = 0; floor_[k] = 0; }
  for (int i = 0; i + 1 < nbp; ++i) {
    gk15(g, bp[i], bp[i + 1], K, G);
    for (int k = 0; k < g->m; ++k) floor_[k] += cabs(K[k]);
  }
  for (int k = 0; k < g->m; ++k) floor_[k] *= 1e-17;
  for (int i = 0; i + 1 < nbp; ++i) {
    if (bp[i + 1] > bp[i]) adapt(g, bp[i], bp[i + 1], floor_, 0, &budget, acc);
  }
  if (budget <= 0) g->capped = 1;
}

/* Sorted, de-duplicated breakpoints in [lo, hi]: lo, hi, the given interior
 * points, and the powers of two in between (so that panels near t = 0, where
 * e^{-t} lives, are never coarser than the distance to the origin).        */
static int make_bp(double lo, double hi, const double *extra, int nextra, double *bp) {
  int n = 0;
  bp[n++] = lo;
  bp[n++] = hi;
  for (int i = 0; i < nextra; ++i)
    if (extra[i] > lo && extra[i] < hi) bp[n++] = extra[i];
  for (double p2 = 1.0; p2 < hi; p2 *= 2.0)
    if (p2 > lo) bp[n++] = p2;
  for (int i = 1; i < n; ++i) { /* insertion sort */
    double v = bp[i];
    int j = i - 1;
    while (j >= 0 && bp[j] > v) { bp[j + 1] = bp[j]; --j; }
    bp[j + 1] = v;
  }
  int m = 1;
  for (int i = 1; i < n; ++i)
    if (bp[i] > bp[m - 1]) bp[m++] = bp[i];
  return m;
}

/* J_n(P) for n = n0 .. n0+m-1 (see the header comment). */
static int jn_quad(cplx P, int n0, int m, cplx *J) {
  integrand_t g;
  g.capped = 0;
  g.P = P;
  g.n0 = n0;
  g.m = m;
  int nmax = n0 + m - 1;
  double a = creal(P), b = cimag(P);
  /* upper limit: t^nmax e^{-t} is below 1e-30 of its peak well before T */
  double T = 2.0 * (nmax + cabs(P)) + 80.0;
  double H = (b < 0) ? 1.0 : ((b == 0) ? 0.5 : 0.0);
  double nn = nmax > 1 ? (double)nmax : 1.0;
  g.subtract = (a > 0 && fabs(b) <= fmin(0.5, a * sqrt(2.0 / nn)));
  cplx tail[96];
  if (g.subtract) {
    /* int_0^{2a} (f(t)-f(P))/(t-P) dt + f(P) [log(2a-P) - log(-P) + 2 pi i H]
     * + int_{2a}^T f(t)/(t-P) dt.  The bracket is the exact integral of
     * 1/(t-P) over [0,2a] plus the residue rule; it equals i pi when P is
     * real (principal value + half residue).                              */
    cplx ePn = cexp(-P);
    g.eP = ePn;
    for (int c = 0; c < m; ++c) g.fP[c] = cpow(P, n0 + c) * ePn;
    if (n0 == 0) g.fP[0] = ePn;
    double bp1[96], ex1[2] = {0.5 * a, a};
    int nb1 = make_bp(0.0, 2.0 * a, ex1, 2, bp1);
    integrate(&g, bp1, nb1, J);
    cplx br;
    if (b == 0)
      br = I * PI_;
    else
      br = clog(2.0 * a - P) - clog(-P) + I * TWO_PI * H;
    for (int c = 0; c < m; ++c) J[c] += g.fP[c] * br;
    g.subtract = 0;
    double bp2[96], ex2[1] = {(double)nmax};
    int nb = make_bp(2.0 * a, T, ex2, 1, bp2);
    integrate(&g, bp2, nb, tail);
    for (int c = 0; c < m; ++c) J[c] += tail[c];
  } else {
    double bp[96], ex[2] = {a, (double)nmax};
    int nb = make_bp(0.0, T, ex, 2, bp);
    integrate(&g, bp, nb, J);
    if (H != 0) {
      cplx ePn = cexp(-P);
      for (int c = 0; c < m; ++c) J[c] += I * TWO_PI * H * cpow(P, n0 + c) * ePn;
    }
  }
  return g.capped;
}

/* I_n(x, y), n = 0..nmax, for kappa = kre + i kim (Eq. generalintegral). */
int hpo_In(double x, double y, double kre, double kim, int nmax, double *out) {
  if (nmax < 0 || nmax > 95 || !(y > 0)) return -1;
  cplx s = y - I * x;
  cplx P = (kre + I * kim) * s;
  cplx J[96];
  int capped = jn_quad(P, 0, nmax + 1, J);
  cplx fac = 1.0 / TWO_PI; /* 1/(2 pi n! s^n) */
  for (int n = 0; n <= nmax; ++n) {
    if (n > 0) fac /= (n * s);
    cplx v = J[n] * fac;
    out[2 * n] = creal(v);
    out[2 * n + 1] = cimag(v);
  }
  return capped ? 1 : 0;
}

/* I_0 and I_1 at one argument, by one joint quadrature. */
static void i01(double x, double y, cplx kappa, cplx *I0, cplx *I1) {
  cplx s = y - I * x;
  cplx J[2];
  jn_quad(kappa * s, 0, 2, J);
  *I0 = J[0] / TWO_PI;
  *I1 = J[1] / (TWO_PI * s);
}

/* Neumaier-compensated complex accumulator */
typedef struct { double s, c; } kacc;
static inline void kadd(kacc *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static inline double kval(const kacc *a) { return a->s + a->c; }

/*
 * Direct O(Nt * Ns) sum (sources y_j > 0, targets y_i >= 0).  parts: bit 0 free, bit 1 image, bit 2 reaction
 * I_0(X,Y) ("plus"), bit 3 reaction I_0(-X,Y) ("minus").  self_index[i] is
 * the source index equal to target i (excluded from the free part, Eq. 1.2)
 * or -1; self_index may be NULL (no exclusion).  u: 2*nt doubles (re, im).
 * grad (may be NULL): 4*nt doubles (d/dx re, im, d/dy re, im) of u with
 * respect to the target position.
 * Gradients: d/dx_i of ln|r_i - r| = (x_i - x)/|r_i - r|^2 etc.;
 * d/dx I_0(X,Y) = i I_1(X,Y), d/dx I_0(-X,Y) = -i I_1(-X,Y),
 * d/dy I_0(+-X,Y) = -I_1(+-X,Y)  (differentiate Eq. generalintegral).
 */
int hpo_direct(long ns, const double *xs, const double *ys, const double *qs,
               long nt, const double *xt, const double *yt, const long *self_index,
               double kre, double kim, int parts, int nthreads, double *u, double *grad) {
  cplx kappa = kre + I * kim;
  for (long j = 0; j < ns; ++j)
    if (!(ys[j] > 0)) return -1;
  for (long i = 0; i < nt; ++i)
    if (!(yt[i] >= 0)) return -1; /* targets may lie on the boundary y = 0 */
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (long i = 0; i < nt; ++i) {
    kacc ur = {0, 0}, ui = {0, 0}, gxr = {0, 0}, gxi = {0, 0}, gyr = {0, 0}, gyi = {0, 0};
    long self = self_index ? self_index[i] : -1;
    for (long j = 0; j < ns; ++j) {
      double q = qs[j];
      double X = xt[i] - xs[j];
      if ((parts & 1) && j != self) {
        double dy = yt[i] - ys[j];
        double r2 = X * X + dy * dy;
        kadd(&ur, -q * 0.5 * log(r2) / TWO_PI);
        if (grad) {
          kadd(&gxr, -q * X / (r2 * TWO_PI));
          kadd(&gyr, -q * dy / (r2 * TWO_PI));
        }
      }
      double Y = yt[i] + ys[j];
      if (parts & 2) {
        double r2 = X * X + Y * Y;
        kadd(&ur, q * 0.5 * log(r2) / TWO_PI);
        if (grad) {
          kadd(&gxr, q * X / (r2 * TWO_PI));
          kadd(&gyr, q * Y / (r2 * TWO_PI));
        }
      }
      if (parts & 4) {
        cplx I0, I1;
        i01(X, Y, kappa, &I0, &I1);
        kadd(&ur, q * creal(I0));
        kadd(&ui, q * cimag(I0));
        if (grad) {
          cplx gx = I * I1, gy = -I1;
          kadd(&gxr, q * creal(gx)); kadd(&gxi, q * cimag(gx));
          kadd(&gyr, q * creal(gy)); kadd(&gyi, q * cimag(gy));
        }
      }
      if (parts & 8) {
        cplx I0, I1;
        i01(-X, Y, kappa, &I0, &I1);
        kadd(&ur, q * creal(I0));
        kadd(&ui, q * cimag(I0));
        if (grad) {
          cplx gx = -I * I1, gy = -I1;
          kadd(&gxr, q * creal(gx)); kadd(&gxi, q * cimag(gx));
          kadd(&gyr, q * creal(gy)); kadd(&gyi, q * cimag(gy));
        }
      }
    }
    u[2 * i] = kval(&ur);
    u[2 * i + 1] = kval(&ui);
    if (grad) {
      grad[4 * i + 0] = kval(&gxr);
      grad[4 * i + 1] = kval(&gxi);
      grad[4 * i + 2] = kval(&gyr);
      grad[4 * i + 3] = kval(&gyi);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tree ordering (Algorithm 1, tree-building step).
 * Bounding square: x0 = min x, L = max(max x - x0, max y) * (1 + 2^-40); the
 * square [x0, x0+L] x [0, L] has y = 0 as its lower edge.  Quantisation:
 * ix = min(floor((x - x0) / L * 2^30), 2^30 - 1), iy likewise with y / L.
 * Key bit 2b is bit b of ix, key bit 2b+1 is bit b of iy.                   */
void hpo_bbox(long n, const double *x, const double *y, double *x0_out, double *L_out) {
  double xmin = x[0], xmax = x[0], ymax = y[0];
  for (long i = 1; i < n; ++i) {
    if (x[i] < xmin) xmin = x[i];
    if (x[i] > xmax) xmax = x[i];
    if (y[i] > ymax) ymax = y[i];
  }
  double w = xmax - xmin;
  double L = (w > ymax) ? w : ymax;
  L = L * (1.0 + ldexp(1.0, -40));
  *x0_out = xmin;
  *L_out = L;
}

static uint64_t quantise(double v, double L) {
  volatile double q = v / L;         /* correctly rounded division */
  volatile double s = q * 1073741824.0; /* exact scaling by 2^30    */
  double f = floor(s);
  if (f < 0) f = 0;
  if (f > 1073741823.0) f = 1073741823.0;
  return (uint64_t)f;
}

void hpo_morton_keys(long n, const double *x, const double *y, double x0, double L,
                     uint64_t *keys) {
  for (long i = 0; i < n; ++i) {
    volatile double dx = x[i] - x0;
    uint64_t ix = quantise(dx, L), iy = quantise(y[i], L);
    uint64_t k = 0;
    for (int b = 0; b < 30; ++b) {
      k |= ((ix >> b) & 1ull) << (2 * b);
      k |= ((iy >> b) & 1ull) << (2 * b + 1);
    }
    keys[i] = k;
  }
}

typedef struct { uint64_t key; long idx; } kv_t;
static int kv_cmp(const void *a, const void *b) {
  const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return (p->idx > q->idx) - (p->idx < q->idx);
}

/* Sorted keys and the permutation perm[k] = input index of k-th point. */
void hpo_morton_order(long n, const double *x, const double *y, uint64_t *keys_sorted,
                      long *perm, double *x0_out, double *L_out) {
  double x0, L;
  hpo_bbox(n, x, y, &x0, &L);
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)n);
  hpo_morton_keys(n, x, y, x0, L, keys);
  for (long i = 0; i < n; ++i) { kv[i].key = keys[i]; kv[i].idx = i; }
  qsort(kv, (size_t)n, sizeof(kv_t), kv_cmp);
  for (long i = 0; i < n; ++i) { keys_sorted[i] = kv[i].key; perm[i] = kv[i].idx; }
  free(keys);
  free(kv);
  *x0_out = x0;
  *L_out = L;
}

int hpo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
