/*
 * mra_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * A plain, slow, FP64 CPU restatement of what the GPU library computes:
 * projection of a Gaussian sum onto the Legendre scaling-function basis,
 * the trapezoid Gaussian fit of 1/r and exp(-mu r)/r, the 1-D operator
 * blocks, the norm screen and the separated operator apply by direct
 * summation, and the non-standard form apply on uniform trees.  Every routine follows the paper (Harrison et al., "MADNESS: A
 * Multiresolution, Adaptive Numerical Environment for Scientific Simulation",
 * arXiv 1507.01888) section or equation it cites.  It shares no code, header,
 * table or constant with the CUDA library; only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load it.
 *
 * Conventions (the same readings the library documents):
 *   cell [-L, L]^3, level n has 2^n boxes per dimension of width h_n = 2L/2^n;
 *   box key = level<<57 | x<<38 | y<<19 | z  (19 bits per translation);
 *   coefficient tensor s[ix][iy][iz], ix slowest, k^3 doubles per box;
 *   phi_i(x) = sqrt(2i+1) P_i(2x-1) on (0,1)                (Sec. 2.1, eq. scalingfunc)
 *   phi^n_{b,i}(x) = h_n^{-1/2} phi_i((x+L)/h_n - b)         (Sec. 2.1, scaled to the cell)
 *
 * Compiled with -ffp-contract=off so that no FMA contraction happens here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_MAXK 32
#define GLQ 20 /* points per panel in the composite Gauss-Legendre rules */

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and Gauss-Legendre nodes                             */
/* ------------------------------------------------------------------------ */

/* P_0..P_{n-1}(x) by the three-term recurrence (n+1)P_{n+1} = (2n+1)xP_n - nP_{n-1}. */
static void legendre_upto(int n, double x, double *p) {
  if (n <= 0) return;
  p[0] = 1.0;
  if (n == 1) return;
  p[1] = x;
  for (int m = 1; m + 1 < n; ++m)
    p[m + 1] = ((2.0 * m + 1.0) * x * p[m] - (double)m * p[m - 1]) / (m + 1.0);
}

/* Scaling functions phi_i(x) = sqrt(2i+1) P_i(2x-1), i < k, for x in [0,1]
 * (Sec. 2.1, eq. scalingfunc).  Outside [0,1] they are zero. */
void orc_phi_all(int k, double x, double *out) {
  if (x < 0.0 || x > 1.0) {
    for (int i = 0; i < k; ++i) out[i] = 0.0;
    return;
  }
  double p[ORC_MAXK];
  legendre_upto(k, 2.0 * x - 1.0, p);
  for (int i = 0; i < k; ++i) out[i] = sqrt(2.0 * i + 1.0) * p[i];
}

/* n-point Gauss-Legendre rule on [-1,1]: Newton iteration on P_n from the
 * usual cosine starting guesses; weights 2/((1-x^2) P_n'(x)^2). */
void orc_gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 1; m < n; ++m) {
        double p2 = ((2.0 * m + 1.0) * z * p1 - (double)m * p0) / (m + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      /* p1 = P_n(z), p0 = P_{n-1}(z) */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int m = 1; m < n; ++m) {
        double p2 = ((2.0 * m + 1.0) * z * p1 - (double)m * p0) / (m + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static double GLX[GLQ], GLW[GLQ];
static int gl_ready = 0;
static void gl_init(void) {
  if (!gl_ready) {
    orc_gauss_legendre(GLQ, GLX, GLW);
    gl_ready = 1;
  }
}

/* ------------------------------------------------------------------------ */
/* Graded composite quadrature of a Gaussian against the scaling functions   */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Break points on [a,b] graded geometrically away from the peak p (in [a,b])
 * with first width delta, and no panel wider than 1/8.  Returns count. */
static int graded_breaks(double a, double b, double p, double delta, double *bp, int cap) {
  int n = 0;
  bp[n++] = a;
  bp[n++] = b;
  if (p > a && p < b && n < cap) bp[n++] = p;
  for (double d = delta; n + 2 < cap; d *= 2.0) {
    int added = 0;
    if (p + d < b) { bp[n++] = p + d; added = 1; }
    if (p - d > a) { bp[n++] = p - d; added = 1; }
    if (!added) break;
  }
  qsort(bp, n, sizeof(double), cmp_double);
  /* subdivide wide gaps uniformly */
  int m = n;
  for (int i = 0; i + 1 < n; ++i) {
    double gap = bp[i + 1] - bp[i];
    int pieces = (int)ceil(gap / 0.125);
    for (int q = 1; q < pieces && m < cap; ++q) bp[m++] = bp[i] + gap * q / pieces;
  }
  qsort(bp, m, sizeof(double), cmp_double);
  int u = 0;
  for (int i = 0; i < m; ++i)
    if (u == 0 || bp[i] > bp[u - 1]) bp[u++] = bp[i];
  return u;
}

/* out[j] = int_0^1 exp(-T (u-uc)^2) phi_j(u) du, j < k, with uc = base + x
 * (base an integer, so that the distance from uc to the nearer end of [0,1]
 * is formed without cancellation).
 * The integrand is negligible (below e^-46 of its maximum on [0,1]) outside
 * |u-uc| <= sqrt(dmin^2 + 46/T), dmin = dist(uc,[0,1]); inside, composite
 * 20-point Gauss-Legendre panels graded from the point p of [0,1] closest to
 * uc.  Nodes are placed by their offset from p, and u - uc = off + (p - uc). */
static void gauss_phi_integral(int k, double T, double base, double x, double *out) {
  gl_init();
  for (int j = 0; j < k; ++j) out[j] = 0.0;
  double uc = base + x;
  double p, e; /* peak point in [0,1] and e = p - uc */
  if (uc <= 0.0) { p = 0.0; e = (0.0 - base) - x; }
  else if (uc >= 1.0) { p = 1.0; e = (1.0 - base) - x; }
  else { p = uc; e = 0.0; }
  double dmin = fabs(e);
  double a = 0.0, b = 1.0, delta;
  if (T > 0.0) {
    double W = sqrt(dmin * dmin + 46.0 / T);
    /* the relevant interval around uc, intersected with [0,1] */
    if (p - e - W > a) a = p - e - W;
    if (p - e + W < b) b = p - e + W;
    if (a >= b) return;
    double s1 = 1.0 / sqrt(T);
    double s2 = dmin > 0.0 ? 1.0 / (2.0 * T * dmin) : s1;
    delta = (s1 < s2 ? s1 : s2) / 16.0;
  } else {
    delta = 0.125;
  }
  if (p < a) p = a;
  if (p > b) p = b;
  double bp[512];
  /* break points as offsets from p */
  int nb = graded_breaks(a - p, b - p, 0.0, delta, bp, 512);
  double ph[ORC_MAXK];
  double epk = (p - uc); /* equals e unless p was moved onto the relevant interval */
  if (p == 0.0 || p == 1.0) epk = e;
  for (int q = 0; q + 1 < nb; ++q) {
    double lo = bp[q], hi = bp[q + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int g = 0; g < GLQ; ++g) {
      double off = mid + half * GLX[g];
      double w = off + epk;
      double ex = exp(-T * w * w) * half * GLW[g];
      orc_phi_all(k, p + off, ph);
      for (int j = 0; j < k; ++j) out[j] += ex * ph[j];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Two-scale matrices (Sec. 2.2: P^{n+1} = P^n + Q^n)                        */
/* ------------------------------------------------------------------------ */

/* U^{(c)}[i][j] = 2^{-1/2} int_0^1 phi_i(y) phi_j((y+c)/2) dy: the level-(n+1)
 * coefficient i, in child c, of the level-n scaling function j. */
void orc_two_scale(int k, double *U0, double *U1) {
  int nq = k + 2;
  double x[64], w[64], pi_[ORC_MAXK], pj[ORC_MAXK];
  orc_gauss_legendre(nq, x, w);
  for (int c = 0; c < 2; ++c) {
    double *U = c == 0 ? U0 : U1;
    for (int i = 0; i < k * k; ++i) U[i] = 0.0;
    for (int q = 0; q < nq; ++q) {
      double y = 0.5 * (x[q] + 1.0), wy = 0.5 * w[q];
      orc_phi_all(k, y, pi_);
      orc_phi_all(k, 0.5 * (y + c), pj);
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) U[i * k + j] += wy * pi_[i] * pj[j] / sqrt(2.0);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Gaussian fit of the kernel (Sec. 2.3)                                     */
/* ------------------------------------------------------------------------ */

/* Trapezoid rule with step h from s_lo on
 *   exp(-mu r)/r = (2/sqrt(pi)) int exp(-r^2 e^{2s} - mu^2 e^{-2s}/4 + s) ds
 * (mu = 0 is the 1/r identity printed in Sec. 2.3):
 *   c_m = (2/sqrt(pi)) h exp(s_m - mu^2 e^{-2 s_m}/4),  t_m = e^{2 s_m}. */
void orc_fit_coeffs(double mu, int M, double h, double s_lo, double *c, double *t) {
  for (int m = 0; m < M; ++m) {
    double s = s_lo + m * h;
    c[m] = 2.0 / sqrt(ORC_PI) * h * exp(s - mu * mu * exp(-2.0 * s) / 4.0);
    t[m] = exp(2.0 * s);
  }
}

static double fit_r_point(double r_lo, double r_hi, int p, int npts) {
  return r_lo * pow(r_hi / r_lo, (double)p / (double)(npts - 1));
}

/* max over npts log-spaced r in [r_lo, r_hi] of |sum c e^{-t r^2} - K(r)| / K(r). */
double orc_fit_maxerr(double mu, int M, const double *c, const double *t, double r_lo, double r_hi,
                      int npts) {
  double worst = 0.0;
  for (int p = 0; p < npts; ++p) {
    double r = fit_r_point(r_lo, r_hi, p, npts);
    double K = exp(-mu * r) / r, sum = 0.0;
    for (int m = 0; m < M; ++m) sum += c[m] * exp(-t[m] * r * r);
    double e = fabs(sum - K) / K;
    if (e > worst) worst = e;
  }
  return worst;
}

/* Grid search: h = (5+i)/100, i = 0..115 (0.05..1.20); s_lo = (j-100)/4,
 * j = 0..112 (-25..3).  Minimise the max relative error on 3000 log-spaced
 * points; the first strict minimum in (i, j) order wins, so ties go to the
 * smaller h. */
int orc_fit_search(double mu, int M, double r_lo, double r_hi, double *h_out, double *slo_out,
                   double *err_out, int nthreads) {
  const int NH = 116, NS = 113, NP = 3000;
  double *errs = (double *)malloc(sizeof(double) * NH * NS);
  if (!errs) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
#endif
  for (int cand = 0; cand < NH * NS; ++cand) {
    int i = cand / NS, j = cand % NS;
    double h = (5.0 + i) / 100.0, s_lo = (j - 100.0) / 4.0;
    double c[512], t[512];
    orc_fit_coeffs(mu, M, h, s_lo, c, t);
    errs[cand] = orc_fit_maxerr(mu, M, c, t, r_lo, r_hi, NP);
  }
  int best = 0;
  for (int cand = 1; cand < NH * NS; ++cand)
    if (errs[cand] < errs[best]) best = cand;
  *h_out = (5.0 + best / NS) / 100.0;
  *slo_out = (best % NS - 100.0) / 4.0;
  *err_out = errs[best];
  free(errs);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Operator blocks (Sec. 2.2 Toeplitz property, Sec. 2.3 separated form)     */
/* ------------------------------------------------------------------------ */

/* R[i][j] = h int_0^1 du phi_i(u) int_0^1 dv phi_j(v) exp(-T (u - v + l)^2),
 * the 1-D block connecting source box b to target box b+l at a level of
 * width h for one Gaussian exp(-t x^2), T = t h^2.  Iterated (u outer,
 * v inner) composite Gauss-Legendre; the outer panels are graded around the
 * points where the Gaussian ridge u - v + l = 0 enters or leaves the square. */
void orc_block(int k, double h, double T, long l, double *R) {
  gl_init();
  for (int i = 0; i < k * k; ++i) R[i] = 0.0;
  /* The ridge v = u + l meets v=0 at u=-l and v=1 at u=1-l.  Each of the two
   * points, clamped to [0,1], anchors graded outer panels whose nodes are
   * placed by their offset from the anchor (u = anchor + off, and the inner
   * integral receives u + l = (anchor + l) + off with anchor + l an integer). */
  double pts[2] = {(double)-l, 1.0 - (double)l};
  double anc[2], dl[2];
  for (int q = 0; q < 2; ++q) {
    double p = pts[q];
    dl[q] = p < 0.0 ? -p : (p > 1.0 ? p - 1.0 : 0.0);
    anc[q] = p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
  }
  int nseg = (anc[0] == anc[1]) ? 1 : 2;
  double G[ORC_MAXK], ph[ORC_MAXK];
  for (int sg = 0; sg < nseg; ++sg) {
    double A = anc[sg], d = dl[sg];
    if (nseg == 1 && dl[1] < d) d = dl[1];
    /* segment of [0,1] served by this anchor */
    double lo_u = 0.0, hi_u = 1.0;
    if (nseg == 2) {
      double m = 0.5 * (anc[0] + anc[1]);
      if (A <= m) hi_u = m; else lo_u = m;
    }
    double delta;
    if (T > 0.0) {
      double s1 = 1.0 / sqrt(T);
      double s2 = d > 0.0 ? 1.0 / (2.0 * T * d) : s1;
      delta = (s1 < s2 ? s1 : s2) / 16.0;
    } else {
      delta = 0.125;
    }
    double bp[512];
    int nb = graded_breaks(lo_u - A, hi_u - A, 0.0, delta, bp, 512);
    double base = A + (double)l;
    for (int q = 0; q + 1 < nb; ++q) {
      double lo = bp[q], hi = bp[q + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
      for (int g = 0; g < GLQ; ++g) {
        double off = mid + half * GLX[g];
        gauss_phi_integral(k, T, base, off, G);
        orc_phi_all(k, A + off, ph);
        double wq = h * half * GLW[g];
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j) R[i * k + j] += wq * ph[i] * G[j];
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Keys                                                                      */
/* ------------------------------------------------------------------------ */

static uint64_t make_key(int n, long x, long y, long z) {
  return ((uint64_t)n << 57) | ((uint64_t)x << 38) | ((uint64_t)y << 19) | (uint64_t)z;
}
static void split_key(uint64_t key, int *n, long *x, long *y, long *z) {
  *n = (int)(key >> 57);
  *x = (long)((key >> 38) & 0x7FFFF);
  *y = (long)((key >> 19) & 0x7FFFF);
  *z = (long)(key & 0x7FFFF);
}
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}
static long find_key(const uint64_t *keys, long n, uint64_t key) {
  long lo = 0, hi = n - 1;
  while (lo <= hi) {
    long mid = (lo + hi) / 2;
    if (keys[mid] == key) return mid;
    if (keys[mid] < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 2.1, eq. projection, and the adaptive refinement text)   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int ng;
  const double *coef, *expnt, *cx, *cy, *cz;
} orc_gsum;

/* s^n_b = int f phi^n_b, exactly (to quadrature rounding), for the Gaussian
 * sum f = sum_g coef_g exp(-a_g |x - c_g|^2); separable per Gaussian:
 * s[ix][iy][iz] = sum_g coef_g X_g[ix] Y_g[iy] Z_g[iz] with
 * X_g[i] = h^{1/2} int_0^1 exp(-a_g h^2 (u - uc)^2) phi_i(u) du. */
static void project_box(const orc_gsum *f, int k, double L, int n, long bx, long by, long bz,
                        double *s) {
  double h = 2.0 * L / (double)(1L << n);
  double sh = sqrt(h);
  double X[ORC_MAXK], Y[ORC_MAXK], Z[ORC_MAXK];
  int k3 = k * k * k;
  for (int i = 0; i < k3; ++i) s[i] = 0.0;
  for (int g = 0; g < f->ng; ++g) {
    double a = f->expnt[g], T = a * h * h;
    gauss_phi_integral(k, T, (double)-bx, (f->cx[g] + L) / h, X);
    gauss_phi_integral(k, T, (double)-by, (f->cy[g] + L) / h, Y);
    gauss_phi_integral(k, T, (double)-bz, (f->cz[g] + L) / h, Z);
    double cf = f->coef[g] * sh * sh * sh;
    for (int ix = 0; ix < k; ++ix)
      for (int iy = 0; iy < k; ++iy)
        for (int iz = 0; iz < k; ++iz) s[(ix * k + iy) * k + iz] += cf * X[ix] * Y[iy] * Z[iz];
  }
}

typedef struct {
  uint64_t key;
  long idx;
} keyidx;
static int cmp_keyidx(const void *a, const void *b) {
  uint64_t x = ((const keyidx *)a)->key, y = ((const keyidx *)b)->key;
  return (x > y) - (x < y);
}

/* Projection onto a uniform level (uniform_level >= 0) or adaptive refinement:
 * start from every box at level init_level-1 as a parent; project the parent
 * and its 8 children exactly; d = s_children - U s_parent (two-scale, tensor
 * product); if ||d||_F <= thresh, or the children are at max_level, the
 * children become leaves, else every child becomes a parent.  Output keys are
 * sorted ascending.  min_margin = min |(||d|| - thresh)/thresh| over the
 * refinement decisions that were not forced by max_level. */
int orc_project(int ng, const double *coef, const double *expnt, const double *cx,
                const double *cy, const double *cz, int k, double L, double thresh, int init_level,
                int max_level, int uniform_level, long cap, uint64_t *keys, double *coeffs,
                long *n_out, double *min_margin, int nthreads) {
  orc_gsum f = {ng, coef, expnt, cx, cy, cz};
  int k3 = k * k * k;
  if (k < 1 || k > ORC_MAXK) return -1;
  gl_init(); /* before any parallel region */
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  *min_margin = INFINITY;
  if (uniform_level >= 0) {
    long nb = 1L << uniform_level, total = nb * nb * nb;
    if (total > cap) return -2;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (long b = 0; b < total; ++b) {
      long bx = b / (nb * nb), by = (b / nb) % nb, bz = b % nb;
      keys[b] = make_key(uniform_level, bx, by, bz);
      project_box(&f, k, L, uniform_level, bx, by, bz, coeffs + b * k3);
    }
    *n_out = total;
    return 0;
  }
  if (init_level < 1 || max_level < init_level || max_level > 19) return -1;
  double U[2][ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U[0], U[1]);
  /* parent list at level init_level-1 */
  int pl = init_level - 1;
  long np = 1L << (3 * pl);
  uint64_t *par = (uint64_t *)malloc(sizeof(uint64_t) * (np > 0 ? np : 1));
  for (long b = 0; b < np; ++b) {
    long nb = 1L << pl;
    par[b] = make_key(pl, b / (nb * nb), (b / nb) % nb, b % nb);
  }
  long nleaf = 0;
  int err = 0;
  double margin = INFINITY;
  while (np > 0 && !err) {
    uint64_t *next = (uint64_t *)malloc(sizeof(uint64_t) * 8 * np);
    char *refine = (char *)malloc(np);
    double *child = (double *)malloc(sizeof(double) * 8 * k3 * np);
    double *pmarg = (double *)malloc(sizeof(double) * np);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (long p = 0; p < np; ++p) {
      int n;
      long x, y, z;
      split_key(par[p], &n, &x, &y, &z);
      double *sp = (double *)malloc(sizeof(double) * k3);
      double *t1 = (double *)malloc(sizeof(double) * k3);
      double *t2 = (double *)malloc(sizeof(double) * k3);
      project_box(&f, k, L, n, x, y, z, sp);
      double dn2 = 0.0;
      for (int c = 0; c < 8; ++c) {
        int cxb = (c >> 2) & 1, cyb = (c >> 1) & 1, czb = c & 1;
        double *sc = child + ((long)p * 8 + c) * k3;
        project_box(&f, k, L, n + 1, 2 * x + cxb, 2 * y + cyb, 2 * z + czb, sc);
        /* (U^{cx} x U^{cy} x U^{cz}) s_parent, one mode at a time */
        for (int ix = 0; ix < k; ++ix)
          for (int jy = 0; jy < k; ++jy)
            for (int jz = 0; jz < k; ++jz) {
              double acc = 0.0;
              for (int jx = 0; jx < k; ++jx)
                acc += U[cxb][ix * k + jx] * sp[(jx * k + jy) * k + jz];
              t1[(ix * k + jy) * k + jz] = acc;
            }
        for (int ix = 0; ix < k; ++ix)
          for (int iy = 0; iy < k; ++iy)
            for (int jz = 0; jz < k; ++jz) {
              double acc = 0.0;
              for (int jy = 0; jy < k; ++jy)
                acc += U[cyb][iy * k + jy] * t1[(ix * k + jy) * k + jz];
              t2[(ix * k + iy) * k + jz] = acc;
            }
        for (int ix = 0; ix < k; ++ix)
          for (int iy = 0; iy < k; ++iy)
            for (int iz = 0; iz < k; ++iz) {
              double acc = 0.0;
              for (int jz = 0; jz < k; ++jz)
                acc += U[czb][iz * k + jz] * t2[(ix * k + iy) * k + jz];
              double d = sc[(ix * k + iy) * k + iz] - acc;
              dn2 += d * d;
            }
      }
      double dn = sqrt(dn2);
      int forced = (n + 1 >= max_level);
      refine[p] = (!forced && dn > thresh) ? 1 : 0;
      pmarg[p] = forced ? INFINITY : fabs(dn - thresh) / thresh;
      free(sp);
      free(t1);
      free(t2);
    }
    long nn = 0;
    for (long p = 0; p < np; ++p) {
      if (pmarg[p] < margin) margin = pmarg[p];
      int n;
      long x, y, z;
      split_key(par[p], &n, &x, &y, &z);
      for (int c = 0; c < 8; ++c) {
        int cxb = (c >> 2) & 1, cyb = (c >> 1) & 1, czb = c & 1;
        uint64_t ck = make_key(n + 1, 2 * x + cxb, 2 * y + cyb, 2 * z + czb);
        if (refine[p]) {
          next[nn++] = ck;
        } else {
          if (nleaf >= cap) { err = -2; break; }
          keys[nleaf] = ck;
          memcpy(coeffs + nleaf * k3, child + ((long)p * 8 + c) * k3, sizeof(double) * k3);
          ++nleaf;
        }
      }
      if (err) break;
    }
    free(refine);
    free(child);
    free(pmarg);
    free(par);
    par = next;
    np = nn;
  }
  free(par);
  if (err) return err;
  /* sort leaves by key */
  keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * (nleaf > 0 ? nleaf : 1));
  for (long i = 0; i < nleaf; ++i) { ki[i].key = keys[i]; ki[i].idx = i; }
  qsort(ki, nleaf, sizeof(keyidx), cmp_keyidx);
  double *tmp = (double *)malloc(sizeof(double) * k3 * (nleaf > 0 ? nleaf : 1));
  for (long i = 0; i < nleaf; ++i) {
    keys[i] = ki[i].key;
    memcpy(tmp + i * k3, coeffs + ki[i].idx * k3, sizeof(double) * k3);
  }
  memcpy(coeffs, tmp, sizeof(double) * k3 * nleaf);
  free(tmp);
  free(ki);
  *n_out = nleaf;
  *min_margin = margin;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Separated operator apply by direct summation (Sec. 2.3)                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n, D;        /* level, max |l_d| */
  double h;
  double *R;       /* [M][2D+1][k*k] */
  double *N;       /* [M][2D+1] Frobenius norms */
} level_blocks;

/* Result: for every source box b (level n), every displacement l in D(b) with
 * b+l inside the cell, and every Gaussian term mu that passes the screen
 *   B = |c_mu| * ||R^n_{mu,lx}||_F ||R^n_{mu,ly}||_F ||R^n_{mu,lz}||_F * ||s_b||_F >= tau,
 *   r_{n,b+l}[ix iy iz] += c_mu sum_j Rx[ix][jx] Ry[iy][jy] Rz[iz][jz] s_b[jx jy jz]
 * with the three mode products done one after another (Sec. 2.3).
 * D(b): stencil=1 -> all |l|_inf <= min(1, 2^n-1); stencil=0 -> shells
 * d = 0,1,2,... of |l|_inf up to min(max_disp, 2^n-1), stopping after the
 * first shell in which no term is kept.
 * If n_sample > 0 only the destination keys listed in sample_keys that are in
 * the destination set are computed (in that order, skipping the others).
 * Per destination: out_bound = sum of B over kept terms, out_marginal = sum of
 * B over terms whose B is within 1e-9 relative of tau (decisions that rounding
 * could flip).  stats: [0] (source,l) pairs with a kept term, [1] kept terms,
 * [2] screened terms (within D(b)), [3] sources whose last allowed shell still
 * kept terms (truncated by max_disp), [4] destinations and [5] kept terms of the
 * whole job (whatever the sample). */
int orc_apply(int k, double L, long n_in, const uint64_t *keys, const double *coeffs, int M,
              const double *c, const double *t, int stencil, int max_disp, double tau,
              long n_sample, const uint64_t *sample_keys, long cap, uint64_t *out_keys,
              double *out_coeffs, double *out_bound, double *out_marginal, long *n_out,
              long *stats, int nthreads) {
  int k2 = k * k, k3 = k * k * k;
  if (k < 1 || k > ORC_MAXK || M < 1) return -1;
  gl_init(); /* before any parallel region */
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (long i = 1; i < n_in; ++i)
    if (keys[i] <= keys[i - 1]) return -1; /* input keys must be sorted and unique */
  /* levels present */
  int present[20] = {0};
  for (long i = 0; i < n_in; ++i) {
    int n = (int)(keys[i] >> 57);
    if (n > 19) return -1;
    present[n] = 1;
  }
  level_blocks lb[20];
  memset(lb, 0, sizeof(lb));
  for (int n = 0; n < 20; ++n) {
    if (!present[n]) continue;
    long nb = 1L << n;
    int D = stencil == 1 ? 1 : max_disp;
    if (D > nb - 1) D = (int)(nb - 1);
    if (D < 0) D = 0;
    lb[n].n = n;
    lb[n].D = D;
    lb[n].h = 2.0 * L / (double)nb;
    int nl = 2 * D + 1;
    lb[n].R = (double *)malloc(sizeof(double) * (size_t)M * nl * k2);
    lb[n].N = (double *)malloc(sizeof(double) * (size_t)M * nl);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (int q = 0; q < M * nl; ++q) {
      int mu = q / nl, li = q % nl;
      double *R = lb[n].R + (size_t)q * k2;
      double h = lb[n].h;
      orc_block(k, h, t[mu] * h * h, (long)(li - D), R);
      double s = 0.0;
      for (int i = 0; i < k2; ++i) s += R[i] * R[i];
      lb[n].N[q] = sqrt(s);
    }
  }
  /* source norms and shell radii */
  double *snorm = (double *)malloc(sizeof(double) * (n_in > 0 ? n_in : 1));
  int *dstop = (int *)malloc(sizeof(int) * (n_in > 0 ? n_in : 1));
  long truncated = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) reduction(+ : truncated)
#endif
  for (long b = 0; b < n_in; ++b) {
    const double *s = coeffs + b * k3;
    double a = 0.0;
    for (int i = 0; i < k3; ++i) a += s[i] * s[i];
    snorm[b] = sqrt(a);
    int n;
    long x, y, z;
    split_key(keys[b], &n, &x, &y, &z);
    long nb = 1L << n;
    int D = lb[n].D, nl = 2 * D + 1;
    if (stencil == 1) {
      dstop[b] = D + 1;
      continue;
    }
    int d;
    for (d = 0; d <= D; ++d) {
      int kept = 0;
      for (int lx = -d; lx <= d && !kept; ++lx)
        for (int ly = -d; ly <= d && !kept; ++ly)
          for (int lz = -d; lz <= d && !kept; ++lz) {
            int m = abs(lx) > abs(ly) ? abs(lx) : abs(ly);
            if (abs(lz) > m) m = abs(lz);
            if (m != d) continue;
            if (x + lx < 0 || x + lx >= nb || y + ly < 0 || y + ly >= nb || z + lz < 0 ||
                z + lz >= nb)
              continue;
            for (int mu = 0; mu < M && !kept; ++mu) {
              double B = fabs(c[mu]) * lb[n].N[mu * nl + lx + D] * lb[n].N[mu * nl + ly + D] *
                         lb[n].N[mu * nl + lz + D] * snorm[b];
              if (B >= tau) kept = 1;
            }
          }
      if (!kept) break;
    }
    dstop[b] = d; /* shells 0..d-1 are in D(b) */
    if (d == D + 1) truncated += 1;
  }
  /* destination set */
  long maxd = 0;
  for (long b = 0; b < n_in; ++b) {
    long w = 2L * dstop[b] - 1;
    if (w > 0) maxd += w * w * w;
  }
  uint64_t *dest = (uint64_t *)malloc(sizeof(uint64_t) * (maxd > 0 ? maxd : 1));
  long nd = 0, total_terms = 0;
  for (long b = 0; b < n_in; ++b) {
    int n;
    long x, y, z;
    split_key(keys[b], &n, &x, &y, &z);
    long nb = 1L << n;
    int D = lb[n].D, nl = 2 * D + 1, r = dstop[b] - 1;
    for (int lx = -r; lx <= r; ++lx)
      for (int ly = -r; ly <= r; ++ly)
        for (int lz = -r; lz <= r; ++lz) {
          if (x + lx < 0 || x + lx >= nb || y + ly < 0 || y + ly >= nb || z + lz < 0 ||
              z + lz >= nb)
            continue;
          int any = 0;
          for (int mu = 0; mu < M; ++mu) {
            double B = fabs(c[mu]) * lb[n].N[mu * nl + lx + D] * lb[n].N[mu * nl + ly + D] *
                       lb[n].N[mu * nl + lz + D] * snorm[b];
            if (B >= tau) { any = 1; total_terms += 1; }
          }
          if (any) dest[nd++] = make_key(n, x + lx, y + ly, z + lz);
        }
  }
  qsort(dest, nd, sizeof(uint64_t), cmp_u64);
  long nu = 0;
  for (long i = 0; i < nd; ++i)
    if (nu == 0 || dest[i] != dest[nu - 1]) dest[nu++] = dest[i];
  /* which destinations to compute */
  uint64_t *todo = dest;
  long ntodo = nu;
  uint64_t *sel = NULL;
  if (n_sample > 0) {
    sel = (uint64_t *)malloc(sizeof(uint64_t) * n_sample);
    ntodo = 0;
    for (long i = 0; i < n_sample; ++i)
      if (find_key(dest, nu, sample_keys[i]) >= 0) sel[ntodo++] = sample_keys[i];
    todo = sel;
  }
  if (ntodo > cap) {
    *n_out = ntodo; /* tell the caller how much room is needed */
    free(dest); free(sel); free(snorm); free(dstop);
    for (int n = 0; n < 20; ++n) { free(lb[n].R); free(lb[n].N); }
    return -2;
  }
  long pairs = 0, kept_terms = 0, screened = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) reduction(+ : pairs, kept_terms, screened)
#endif
  for (long di = 0; di < ntodo; ++di) {
    int n;
    long x, y, z;
    split_key(todo[di], &n, &x, &y, &z);
    long nb = 1L << n;
    int D = lb[n].D, nl = 2 * D + 1;
    double *r = out_coeffs + di * k3;
    double *t1 = (double *)malloc(sizeof(double) * k3);
    double *t2 = (double *)malloc(sizeof(double) * k3);
    for (int i = 0; i < k3; ++i) r[i] = 0.0;
    double bsum = 0.0, msum = 0.0;
    for (int lx = -D; lx <= D; ++lx)
      for (int ly = -D; ly <= D; ++ly)
        for (int lz = -D; lz <= D; ++lz) {
          long sx = x - lx, sy = y - ly, sz = z - lz;
          if (sx < 0 || sx >= nb || sy < 0 || sy >= nb || sz < 0 || sz >= nb) continue;
          long b = find_key(keys, n_in, make_key(n, sx, sy, sz));
          if (b < 0) continue;
          int m = abs(lx) > abs(ly) ? abs(lx) : abs(ly);
          if (abs(lz) > m) m = abs(lz);
          if (m >= dstop[b]) continue;
          const double *s = coeffs + b * k3;
          int any = 0;
          for (int mu = 0; mu < M; ++mu) {
            const double *Rx = lb[n].R + ((size_t)mu * nl + lx + D) * k2;
            const double *Ry = lb[n].R + ((size_t)mu * nl + ly + D) * k2;
            const double *Rz = lb[n].R + ((size_t)mu * nl + lz + D) * k2;
            double B = fabs(c[mu]) * lb[n].N[mu * nl + lx + D] * lb[n].N[mu * nl + ly + D] *
                       lb[n].N[mu * nl + lz + D] * snorm[b];
            if (!(B >= tau)) {
              screened += 1;
              continue;
            }
            any = 1;
            kept_terms += 1;
            bsum += B;
            if (tau > 0.0 && fabs(B - tau) <= 1e-9 * tau) msum += B;
            /* t1 = s x_1 Rx */
            for (int ix = 0; ix < k; ++ix)
              for (int jy = 0; jy < k; ++jy)
                for (int jz = 0; jz < k; ++jz) {
                  double acc = 0.0;
                  for (int jx = 0; jx < k; ++jx) acc += Rx[ix * k + jx] * s[(jx * k + jy) * k + jz];
                  t1[(ix * k + jy) * k + jz] = acc;
                }
            /* t2 = t1 x_2 Ry */
            for (int ix = 0; ix < k; ++ix)
              for (int iy = 0; iy < k; ++iy)
                for (int jz = 0; jz < k; ++jz) {
                  double acc = 0.0;
                  for (int jy = 0; jy < k; ++jy)
                    acc += Ry[iy * k + jy] * t1[(ix * k + jy) * k + jz];
                  t2[(ix * k + iy) * k + jz] = acc;
                }
            /* r += c_mu (t2 x_3 Rz) */
            for (int ix = 0; ix < k; ++ix)
              for (int iy = 0; iy < k; ++iy)
                for (int iz = 0; iz < k; ++iz) {
                  double acc = 0.0;
                  for (int jz = 0; jz < k; ++jz)
                    acc += Rz[iz * k + jz] * t2[(ix * k + iy) * k + jz];
                  r[(ix * k + iy) * k + iz] += c[mu] * acc;
                }
          }
          if (any) pairs += 1;
        }
    out_keys[di] = todo[di];
    if (out_bound) out_bound[di] = bsum;
    if (out_marginal) out_marginal[di] = msum;
    free(t1);
    free(t2);
  }
  *n_out = ntodo;
  if (stats) {
    stats[0] = pairs;
    stats[1] = kept_terms;
    stats[2] = screened;
    stats[3] = truncated;
    stats[4] = nu;          /* destinations of the whole job */
    stats[5] = total_terms; /* kept terms of the whole job */
  }
  free(dest);
  free(sel);
  free(snorm);
  free(dstop);
  for (int n = 0; n < 20; ++n) {
    free(lb[n].R);
    free(lb[n].N);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Non-standard form apply on a uniform tree (Sec. 2.2)                      */
/* ------------------------------------------------------------------------ */

/* Level-n boxes of a uniform level are stored densely: box (x, y, z) at ((x nb) + y) nb + z.
 *
 * Two-scale relation (Sec. 2.2, P^{n+1} = P^n + Q^n): with Ubar[(c,i)][j] = U^(c)[i][j]
 * (orc_two_scale), the children of a box hold S = (Ubar x Ubar x Ubar) s for a function
 * of the parent space, and the parent's scaling coefficients of any children tensor S are
 * s = (Ubar^T x Ubar^T x Ubar^T) S.  S is stored as the (2k)^3 tensor with index (c, i) =
 * c k + i in every dimension.
 *
 * The operator blocks of the 2k basis of level n are those of level n+1 between the
 * children: R2k^n_{m,l}[(ci,i)][(cj,j)] = R^{n+1}_{m, 2l+ci-cj}[i][j].
 *
 * Non-standard form: T^{n+1} = T^n + A^n + B^n + C^n, so on a uniform level N
 *   T^N s^N = T^{n0} s^{n0} + sum_{n=n0}^{N-1} (A^n + B^n + C^n) s,
 * with (A + B + C)^n = T2k^n - Ubar T^n Ubar^T on level n's 2k basis.  The apply takes
 * T^{n0} with every displacement of level n0 and the level-n differences with |l|_inf <= D,
 * then sums down: r^{n+1} = Ubar (r^n - Z^n) + Y^n per box (Y^n = T2k^n S^n,
 * Z^n = T^n s^n), split into the children.  With D covering every displacement the
 * result equals the plain level-N apply T^N s^N. */

/* out[target] = sum_{l, m} c_m (R_{m,lx} x R_{m,ly} x R_{m,lz}) in[target - l] on a dense level
 * of nb^3 boxes of kk^3 coefficients; R holds [M][2D+1][kk*kk] blocks (index l + D). */
static void apply_level_dense(int kk, long nb, const double *in, const double *R, const double *c, int M,
                              int D, double *out) {
  long nbox = nb * nb * nb;
  int kk2 = kk * kk, kk3 = kk2 * kk, nl = 2 * D + 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
  for (long tb = 0; tb < nbox; ++tb) {
    long tx = tb / (nb * nb), ty = (tb / nb) % nb, tz = tb % nb;
    double *o = out + tb * kk3;
    double *t1 = (double *)malloc(sizeof(double) * kk3 * 3);
    double *t2 = t1 + kk3, *t3 = t2 + kk3;
    for (int i = 0; i < kk3; ++i) o[i] = 0.0;
    for (int lx = -D; lx <= D; ++lx)
      for (int ly = -D; ly <= D; ++ly)
        for (int lz = -D; lz <= D; ++lz) {
          long sx = tx - lx, sy = ty - ly, sz = tz - lz;
          if (sx < 0 || sx >= nb || sy < 0 || sy >= nb || sz < 0 || sz >= nb) continue;
          const double *s = in + ((sx * nb + sy) * nb + sz) * kk3;
          for (int m = 0; m < M; ++m) {
            const double *Rx = R + ((size_t)m * nl + lx + D) * kk2;
            const double *Ry = R + ((size_t)m * nl + ly + D) * kk2;
            const double *Rz = R + ((size_t)m * nl + lz + D) * kk2;
            /* t1[ix][jy][jz] = sum_jx Rx[ix][jx] s[jx][jy][jz] */
            for (int ix = 0; ix < kk; ++ix)
              for (int q = 0; q < kk2; ++q) {
                double a = 0.0;
                for (int jx = 0; jx < kk; ++jx) a += Rx[ix * kk + jx] * s[jx * kk2 + q];
                t1[ix * kk2 + q] = a;
              }
            /* t2[ix][iy][jz] = sum_jy Ry[iy][jy] t1[ix][jy][jz] */
            for (int ix = 0; ix < kk; ++ix)
              for (int iy = 0; iy < kk; ++iy)
                for (int jz = 0; jz < kk; ++jz) {
                  double a = 0.0;
                  for (int jy = 0; jy < kk; ++jy) a += Ry[iy * kk + jy] * t1[(ix * kk + jy) * kk + jz];
                  t2[(ix * kk + iy) * kk + jz] = a;
                }
            /* t3[ix][iy][iz] = sum_jz Rz[iz][jz] t2[ix][iy][jz] */
            for (int q = 0; q < kk2; ++q)
              for (int iz = 0; iz < kk; ++iz) {
                double a = 0.0;
                for (int jz = 0; jz < kk; ++jz) a += Rz[iz * kk + jz] * t2[q * kk + jz];
                t3[q * kk + iz] = a;
              }
            for (int i = 0; i < kk3; ++i) o[i] += c[m] * t3[i];
          }
        }
    free(t1);
  }
}

/* k x k blocks of level n for l in [-D, D] (Sec. 2.2 Toeplitz blocks, Sec. 2.3 terms). */
static double *blocks_level(int k, double L, int n, int M, const double *t, int D) {
  int nl = 2 * D + 1, k2 = k * k;
  double h = 2.0 * L / (double)(1L << n);
  double *R = (double *)malloc(sizeof(double) * (size_t)M * nl * k2);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
  for (int q = 0; q < M * nl; ++q) orc_block(k, h, t[q / nl] * h * h, (long)(q % nl - D), R + (size_t)q * k2);
  return R;
}

/* 2k x 2k blocks of level n from the level-(n+1) blocks between the children. */
static double *blocks_level_2k(int k, double L, int n, int M, const double *t, int D) {
  int Dc = 2 * D + 1, nlc = 2 * Dc + 1, nl = 2 * D + 1, kk = 2 * k, kk2 = kk * kk;
  double *Rc = blocks_level(k, L, n + 1, M, t, Dc);
  double *R = (double *)malloc(sizeof(double) * (size_t)M * nl * kk2);
  for (int m = 0; m < M; ++m)
    for (int li = 0; li < nl; ++li) {
      int l = li - D;
      double *B = R + ((size_t)m * nl + li) * kk2;
      for (int ci = 0; ci < 2; ++ci)
        for (int cj = 0; cj < 2; ++cj) {
          const double *C = Rc + ((size_t)m * nlc + (2 * l + ci - cj) + Dc) * k * k;
          for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) B[(ci * k + i) * kk + cj * k + j] = C[i * k + j];
        }
    }
  free(Rc);
  return R;
}

/* (Ubar x Ubar x Ubar) v: k^3 -> (2k)^3, Ubar[(c,i)][j] = U^(c)[i][j]. */
static void unfilter3(int k, const double *Ub, const double *v, double *S) {
  int kk = 2 * k;
  double *a = (double *)malloc(sizeof(double) * kk * k * k);
  double *b = (double *)malloc(sizeof(double) * kk * kk * k);
  for (int I = 0; I < kk; ++I)
    for (int q = 0; q < k * k; ++q) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += Ub[I * k + j] * v[j * k * k + q];
      a[I * k * k + q] = s;
    }
  for (int I = 0; I < kk; ++I)
    for (int J = 0; J < kk; ++J)
      for (int l = 0; l < k; ++l) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += Ub[J * k + j] * a[(I * k + j) * k + l];
        b[(I * kk + J) * k + l] = s;
      }
  for (int q = 0; q < kk * kk; ++q)
    for (int Lq = 0; Lq < kk; ++Lq) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += Ub[Lq * k + j] * b[q * k + j];
      S[q * kk + Lq] = s;
    }
  free(a);
  free(b);
}

/* (Ubar^T x Ubar^T x Ubar^T) S: (2k)^3 -> k^3. */
static void filter3(int k, const double *Ub, const double *S, double *v) {
  int kk = 2 * k;
  double *a = (double *)malloc(sizeof(double) * k * kk * kk);
  double *b = (double *)malloc(sizeof(double) * k * k * kk);
  for (int i = 0; i < k; ++i)
    for (int q = 0; q < kk * kk; ++q) {
      double s = 0.0;
      for (int I = 0; I < kk; ++I) s += Ub[I * k + i] * S[I * kk * kk + q];
      a[i * kk * kk + q] = s;
    }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j)
      for (int Lq = 0; Lq < kk; ++Lq) {
        double s = 0.0;
        for (int J = 0; J < kk; ++J) s += Ub[J * k + j] * a[(i * kk + J) * kk + Lq];
        b[(i * k + j) * kk + Lq] = s;
      }
  for (int q = 0; q < k * k; ++q)
    for (int l = 0; l < k; ++l) {
      double s = 0.0;
      for (int Lq = 0; Lq < kk; ++Lq) s += Ub[Lq * k + l] * b[q * kk + Lq];
      v[q * k + l] = s;
    }
  free(a);
  free(b);
}

/* children of box (x,y,z) of level n (dense level n+1 array `fine`) as one (2k)^3 tensor */
static void gather_children(int k, long nb, long x, long y, long z, const double *fine, double *S) {
  int kk = 2 * k, k3 = k * k * k;
  long nf = 2 * nb;
  for (int cx = 0; cx < 2; ++cx)
    for (int cy = 0; cy < 2; ++cy)
      for (int cz = 0; cz < 2; ++cz) {
        const double *s = fine + (((2 * x + cx) * nf + 2 * y + cy) * nf + 2 * z + cz) * k3;
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j)
            for (int l = 0; l < k; ++l) S[((cx * k + i) * kk + cy * k + j) * kk + cz * k + l] = s[(i * k + j) * k + l];
      }
}

int orc_apply_ns(int k, double L, int N, int n0, const double *s_in, int M, const double *c, const double *t,
                 int D, double *r_out, int nthreads) {
  if (k < 1 || 2 * k > ORC_MAXK || n0 < 0 || n0 > N || N > 10 || M < 1 || D < 0) return -1;
  gl_init();
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  int k3 = k * k * k, kk = 2 * k, kk3 = kk * kk * kk;
  double U0[ORC_MAXK * ORC_MAXK], U1[ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U0, U1);
  double *Ub = (double *)malloc(sizeof(double) * kk * k);
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ub[(cc * k + i) * k + j] = (cc == 0 ? U0 : U1)[i * k + j];
  /* compress: s^n and S^n for n = N-1 .. n0 */
  double *s[11], *S[11];
  memset(s, 0, sizeof(s));
  memset(S, 0, sizeof(S));
  long nbN = 1L << N;
  s[N] = (double *)malloc(sizeof(double) * nbN * nbN * nbN * k3);
  memcpy(s[N], s_in, sizeof(double) * nbN * nbN * nbN * k3);
  for (int n = N - 1; n >= n0; --n) {
    long nb = 1L << n, nbox = nb * nb * nb;
    s[n] = (double *)malloc(sizeof(double) * nbox * k3);
    S[n] = (double *)malloc(sizeof(double) * nbox * kk3);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (long b = 0; b < nbox; ++b) {
      gather_children(k, nb, b / (nb * nb), (b / nb) % nb, b % nb, s[n + 1], S[n] + b * kk3);
      filter3(k, Ub, S[n] + b * kk3, s[n] + b * k3);
    }
  }
  /* coarsest level: T^{n0} with every displacement */
  long nb0 = 1L << n0;
  int D0 = (int)(nb0 - 1);
  double *R0 = blocks_level(k, L, n0, M, t, D0);
  double *r = (double *)malloc(sizeof(double) * nb0 * nb0 * nb0 * k3);
  apply_level_dense(k, nb0, s[n0], R0, c, M, D0, r);
  free(R0);
  /* levels n0 .. N-1: r^{n+1} = Ubar (r^n - Z^n) + Y^n */
  for (int n = n0; n < N; ++n) {
    long nb = 1L << n, nbox = nb * nb * nb, nf = 2 * nb;
    int Dn = D < nb - 1 ? D : (int)(nb - 1);
    double *Rk = blocks_level(k, L, n, M, t, Dn);
    double *R2 = blocks_level_2k(k, L, n, M, t, Dn);
    double *Y = (double *)malloc(sizeof(double) * nbox * kk3);
    double *Z = (double *)malloc(sizeof(double) * nbox * k3);
    apply_level_dense(kk, nb, S[n], R2, c, M, Dn, Y);
    apply_level_dense(k, nb, s[n], Rk, c, M, Dn, Z);
    double *rn = (double *)malloc(sizeof(double) * nf * nf * nf * k3);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
    for (long b = 0; b < nbox; ++b) {
      double *dv = (double *)malloc(sizeof(double) * (k3 + kk3));
      double *U = dv + k3;
      for (int i = 0; i < k3; ++i) dv[i] = r[b * k3 + i] - Z[b * k3 + i];
      unfilter3(k, Ub, dv, U);
      for (int i = 0; i < kk3; ++i) U[i] += Y[b * kk3 + i];
      long x = b / (nb * nb), y = (b / nb) % nb, z = b % nb;
      for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy)
          for (int cz = 0; cz < 2; ++cz) {
            double *o = rn + (((2 * x + cx) * nf + 2 * y + cy) * nf + 2 * z + cz) * k3;
            for (int i = 0; i < k; ++i)
              for (int j = 0; j < k; ++j)
                for (int l = 0; l < k; ++l) o[(i * k + j) * k + l] = U[((cx * k + i) * kk + cy * k + j) * kk + cz * k + l];
          }
      free(dv);
    }
    free(Rk);
    free(R2);
    free(Y);
    free(Z);
    free(r);
    r = rn;
  }
  memcpy(r_out, r, sizeof(double) * nbN * nbN * nbN * k3);
  free(r);
  for (int n = 0; n <= 10; ++n) {
    free(s[n]);
    free(S[n]);
  }
  free(Ub);
  return 0;
}

/* The two-scale transforms alone, for the pins: S = (Ubar x3) v and v = (Ubar^T x3) S. */
void orc_unfilter3(int k, const double *v, double *S) {
  double U0[ORC_MAXK * ORC_MAXK], U1[ORC_MAXK * ORC_MAXK], Ub[2 * ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U0, U1);
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ub[(cc * k + i) * k + j] = (cc == 0 ? U0 : U1)[i * k + j];
  unfilter3(k, Ub, v, S);
}
void orc_filter3(int k, const double *S, double *v) {
  double U0[ORC_MAXK * ORC_MAXK], U1[ORC_MAXK * ORC_MAXK], Ub[2 * ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U0, U1);
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ub[(cc * k + i) * k + j] = (cc == 0 ? U0 : U1)[i * k + j];
  filter3(k, Ub, S, v);
}

/* ------------------------------------------------------------------------ */
/* Non-standard form apply on an adaptive tree (Sec. 2.2)                    */
/* ------------------------------------------------------------------------ */

/* The input is a complete octree partition of the cell: leaves (sorted keys, k^3
 * coefficients each) at levels > n0, every interior node with its eight children.
 * Sources of level n are the interior nodes I_n with S_b = their children's coefficients as
 * one (2k)^3 tensor (a child is a leaf or an interior node, whose s = filter(S) comes from
 * below) and s_b = (Ubar^T)^{x3} S_b.  The result tree is built from the top: R_{n0} = every
 * box of level n0 with r = T^{n0} s^{n0} (every displacement); at level n the nodes of R_n
 * that a level-n apply reaches (Y^n = T2k^n S^n, Z^n = T^n s^n, |l|_inf <= D) are refined,
 * their children getting Ubar^{x3} (r_p - Z_p) + Y_p; the others are result leaves.  Every
 * node of R at the deepest leaf level is a result leaf.  A leaf f_b of level n reaches the
 * result through T^n (its parent's 2k apply telescopes T^{n0} + sum (T^{m+1} - T^m)), so with
 * every displacement the result is, as a function, the leaf-level apply with every
 * displacement. */

typedef struct {
  long n;
  uint64_t *keys;
  double *v; /* n x len */
} orc_set;

static int cmp_u64v(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y);
}

/* out[t] = sum_{l, m, src = t - l in the source set} c_m (R x R x R) in[src]; the targets are
 * every in-cell box within |l|_inf <= D of a source (sorted). */
static orc_set apply_level_sparse(int kk, int n, long ns, const uint64_t *skeys, const double *sin,
                                  const double *R, const double *c, int M, int D) {
  long nb = 1L << n;
  int kk2 = kk * kk, kk3 = kk2 * kk, nl = 2 * D + 1;
  long cap = ns * nl * nl * nl;
  uint64_t *cand = (uint64_t *)malloc(sizeof(uint64_t) * (cap > 0 ? cap : 1));
  long nc = 0;
  for (long i = 0; i < ns; ++i) {
    int lv;
    long x, y, z;
    split_key(skeys[i], &lv, &x, &y, &z);
    for (int lx = -D; lx <= D; ++lx)
      for (int ly = -D; ly <= D; ++ly)
        for (int lz = -D; lz <= D; ++lz) {
          long a = x + lx, b = y + ly, e = z + lz;
          if (a < 0 || a >= nb || b < 0 || b >= nb || e < 0 || e >= nb) continue;
          cand[nc++] = make_key(n, a, b, e);
        }
  }
  qsort(cand, nc, sizeof(uint64_t), cmp_u64v);
  long nt = 0;
  for (long i = 0; i < nc; ++i)
    if (i == 0 || cand[i] != cand[i - 1]) cand[nt++] = cand[i];
  orc_set out;
  out.n = nt;
  out.keys = cand;
  out.v = (double *)calloc((size_t)(nt > 0 ? nt : 1) * kk3, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
  for (long ti = 0; ti < nt; ++ti) {
    int lv;
    long tx, ty, tz;
    split_key(cand[ti], &lv, &tx, &ty, &tz);
    double *o = out.v + ti * kk3;
    double *t1 = (double *)malloc(sizeof(double) * kk3 * 3);
    double *t2 = t1 + kk3, *t3 = t2 + kk3;
    for (int lx = -D; lx <= D; ++lx)
      for (int ly = -D; ly <= D; ++ly)
        for (int lz = -D; lz <= D; ++lz) {
          long sx = tx - lx, sy = ty - ly, sz = tz - lz;
          if (sx < 0 || sx >= nb || sy < 0 || sy >= nb || sz < 0 || sz >= nb) continue;
          long si = find_key(skeys, ns, make_key(n, sx, sy, sz));
          if (si < 0) continue;
          const double *s = sin + si * kk3;
          for (int m = 0; m < M; ++m) {
            const double *Rx = R + ((size_t)m * nl + lx + D) * kk2;
            const double *Ry = R + ((size_t)m * nl + ly + D) * kk2;
            const double *Rz = R + ((size_t)m * nl + lz + D) * kk2;
            for (int ix = 0; ix < kk; ++ix)
              for (int q = 0; q < kk2; ++q) {
                double a = 0.0;
                for (int jx = 0; jx < kk; ++jx) a += Rx[ix * kk + jx] * s[jx * kk2 + q];
                t1[ix * kk2 + q] = a;
              }
            for (int ix = 0; ix < kk; ++ix)
              for (int iy = 0; iy < kk; ++iy)
                for (int jz = 0; jz < kk; ++jz) {
                  double a = 0.0;
                  for (int jy = 0; jy < kk; ++jy) a += Ry[iy * kk + jy] * t1[(ix * kk + jy) * kk + jz];
                  t2[(ix * kk + iy) * kk + jz] = a;
                }
            for (int q = 0; q < kk2; ++q)
              for (int iz = 0; iz < kk; ++iz) {
                double a = 0.0;
                for (int jz = 0; jz < kk; ++jz) a += Rz[iz * kk + jz] * t2[q * kk + jz];
                t3[q * kk + iz] = a;
              }
            for (int i = 0; i < kk3; ++i) o[i] += c[m] * t3[i];
          }
        }
    free(t1);
  }
  return out;
}

int orc_apply_ns_tree(int k, double L, long n_leaf, const uint64_t *lkeys, const double *lcoeffs, int n0, int M,
                      const double *c, const double *t, int D, long cap, uint64_t *out_keys, double *out_coeffs,
                      long *n_out, int nthreads) {
  if (k < 1 || 2 * k > ORC_MAXK || n0 < 0 || M < 1 || D < 0 || n_leaf < 1) return -1;
  gl_init();
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (long i = 1; i < n_leaf; ++i)
    if (lkeys[i] <= lkeys[i - 1]) return -1;
  int Nmax = 0;
  for (long i = 0; i < n_leaf; ++i) {
    int lv = (int)(lkeys[i] >> 57);
    if (lv <= n0 || lv > 19) return -1; /* every leaf below the coarsest level */
    if (lv > Nmax) Nmax = lv;
  }
  int k3 = k * k * k, kk = 2 * k, kk3 = kk * kk * kk;
  double U0[ORC_MAXK * ORC_MAXK], U1[ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U0, U1);
  double *Ub = (double *)malloc(sizeof(double) * kk * k);
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ub[(cc * k + i) * k + j] = (cc == 0 ? U0 : U1)[i * k + j];
  /* interior nodes per level: the ancestors of the leaves */
  orc_set I[20], Ssrc[20];
  memset(I, 0, sizeof(I));
  memset(Ssrc, 0, sizeof(Ssrc));
  for (int n = n0; n < Nmax; ++n) {
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * n_leaf);
    long na = 0;
    for (long i = 0; i < n_leaf; ++i) {
      int lv;
      long x, y, z;
      split_key(lkeys[i], &lv, &x, &y, &z);
      if (lv <= n) continue;
      a[na++] = make_key(n, x >> (lv - n), y >> (lv - n), z >> (lv - n));
    }
    qsort(a, na, sizeof(uint64_t), cmp_u64v);
    long u = 0;
    for (long i = 0; i < na; ++i)
      if (i == 0 || a[i] != a[i - 1]) a[u++] = a[i];
    I[n].n = u;
    I[n].keys = a;
    I[n].v = (double *)malloc(sizeof(double) * (u > 0 ? u : 1) * k3); /* s of interior nodes */
    Ssrc[n].n = u;
    Ssrc[n].keys = a;
    Ssrc[n].v = (double *)malloc(sizeof(double) * (u > 0 ? u : 1) * kk3); /* S of interior nodes */
  }
  if (I[n0].n != (1L << (3 * n0))) return -2; /* level n0 must be complete */
  int err = 0;
  /* compress, from the deepest interior level up */
  for (int n = Nmax - 1; n >= n0 && !err; --n) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) reduction(| : err)
#endif
    for (long b = 0; b < I[n].n; ++b) {
      int lv;
      long x, y, z;
      split_key(I[n].keys[b], &lv, &x, &y, &z);
      double *S = Ssrc[n].v + b * kk3;
      for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy)
          for (int cz = 0; cz < 2; ++cz) {
            uint64_t ck = make_key(n + 1, 2 * x + cx, 2 * y + cy, 2 * z + cz);
            const double *src = NULL;
            long li = find_key(lkeys, n_leaf, ck);
            if (li >= 0) src = lcoeffs + li * k3;
            else if (n + 1 < Nmax) {
              long ii = find_key(I[n + 1].keys, I[n + 1].n, ck);
              if (ii >= 0) src = I[n + 1].v + ii * k3;
            }
            if (!src) {
              err = 1; /* not a complete octree */
              continue;
            }
            for (int i = 0; i < k; ++i)
              for (int j = 0; j < k; ++j)
                for (int l = 0; l < k; ++l) S[((cx * k + i) * kk + cy * k + j) * kk + cz * k + l] = src[(i * k + j) * k + l];
          }
      filter3(k, Ub, S, I[n].v + b * k3);
    }
  }
  long nout = 0;
  int rc = 0;
  /* coarsest level: every box, T^{n0} with every displacement */
  long nb0 = 1L << n0;
  int D0 = (int)(nb0 - 1);
  orc_set R;
  R.n = I[n0].n;
  R.keys = (uint64_t *)malloc(sizeof(uint64_t) * R.n);
  memcpy(R.keys, I[n0].keys, sizeof(uint64_t) * R.n);
  R.v = (double *)malloc(sizeof(double) * R.n * k3);
  if (!err) {
    double *R0 = blocks_level(k, L, n0, M, t, D0);
    apply_level_dense(k, nb0, I[n0].v, R0, c, M, D0, R.v);
    free(R0);
  }
  for (int n = n0; n < Nmax && !err; ++n) {
    int Dn = D < (1L << n) - 1 ? D : (int)((1L << n) - 1);
    double *Rk = blocks_level(k, L, n, M, t, Dn);
    double *R2 = blocks_level_2k(k, L, n, M, t, Dn);
    orc_set Y = apply_level_sparse(kk, n, Ssrc[n].n, Ssrc[n].keys, Ssrc[n].v, R2, c, M, Dn);
    orc_set Z = apply_level_sparse(k, n, I[n].n, I[n].keys, I[n].v, Rk, c, M, Dn);
    free(Rk);
    free(R2);
    /* every target must be a node of R_n */
    for (long i = 0; i < Y.n; ++i)
      if (find_key(R.keys, R.n, Y.keys[i]) < 0) err = 2;
    /* refine the reached nodes, emit the others */
    long nref = 0;
    for (long p = 0; p < R.n; ++p)
      if (find_key(Y.keys, Y.n, R.keys[p]) >= 0) ++nref;
    orc_set Rn;
    Rn.n = 8 * nref;
    Rn.keys = (uint64_t *)malloc(sizeof(uint64_t) * (Rn.n > 0 ? Rn.n : 1));
    Rn.v = (double *)malloc(sizeof(double) * (Rn.n > 0 ? Rn.n : 1) * k3);
    long q = 0;
    double *dv = (double *)malloc(sizeof(double) * (k3 + kk3));
    double *U = dv + k3;
    for (long p = 0; p < R.n && !err; ++p) {
      long yi = find_key(Y.keys, Y.n, R.keys[p]);
      if (yi < 0) {
        if (nout < cap) {
          out_keys[nout] = R.keys[p];
          memcpy(out_coeffs + nout * k3, R.v + p * k3, sizeof(double) * k3);
        }
        ++nout;
        continue;
      }
      long zi = find_key(Z.keys, Z.n, R.keys[p]);
      for (int i = 0; i < k3; ++i) dv[i] = R.v[p * k3 + i] - (zi >= 0 ? Z.v[zi * k3 + i] : 0.0);
      unfilter3(k, Ub, dv, U);
      for (int i = 0; i < kk3; ++i) U[i] += Y.v[yi * kk3 + i];
      int lv;
      long x, y, z;
      split_key(R.keys[p], &lv, &x, &y, &z);
      for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy)
          for (int cz = 0; cz < 2; ++cz, ++q) {
            Rn.keys[q] = make_key(n + 1, 2 * x + cx, 2 * y + cy, 2 * z + cz);
            double *o = Rn.v + q * k3;
            for (int i = 0; i < k; ++i)
              for (int j = 0; j < k; ++j)
                for (int l = 0; l < k; ++l) o[(i * k + j) * k + l] = U[((cx * k + i) * kk + cy * k + j) * kk + cz * k + l];
          }
    }
    free(dv);
    free(Y.keys);
    free(Y.v);
    free(Z.keys);
    free(Z.v);
    /* the children in key order */
    long *perm = (long *)malloc(sizeof(long) * (Rn.n > 0 ? Rn.n : 1));
    for (long i = 0; i < Rn.n; ++i) perm[i] = i;
    for (long i = 1; i < Rn.n; ++i) { /* insertion sort by key (plain; sizes are small here) */
      long pi = perm[i], j = i - 1;
      while (j >= 0 && Rn.keys[perm[j]] > Rn.keys[pi]) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = pi;
    }
    orc_set Rs;
    Rs.n = Rn.n;
    Rs.keys = (uint64_t *)malloc(sizeof(uint64_t) * (Rs.n > 0 ? Rs.n : 1));
    Rs.v = (double *)malloc(sizeof(double) * (Rs.n > 0 ? Rs.n : 1) * k3);
    for (long i = 0; i < Rs.n; ++i) {
      Rs.keys[i] = Rn.keys[perm[i]];
      memcpy(Rs.v + i * k3, Rn.v + perm[i] * k3, sizeof(double) * k3);
    }
    free(perm);
    free(Rn.keys);
    free(Rn.v);
    free(R.keys);
    free(R.v);
    R = Rs;
  }
  if (!err) {
    for (long p = 0; p < R.n; ++p) { /* the deepest level: all leaves */
      if (nout < cap) {
        out_keys[nout] = R.keys[p];
        memcpy(out_coeffs + nout * k3, R.v + p * k3, sizeof(double) * k3);
      }
      ++nout;
    }
  }
  free(R.keys);
  free(R.v);
  for (int n = 0; n < 20; ++n) {
    free(I[n].keys);
    free(I[n].v);
    free(Ssrc[n].v);
  }
  free(Ub);
  *n_out = nout;
  if (err) return -3;
  if (nout > cap) rc = -4;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Reconstruct: a multi-level sum of boxes as disjoint leaves (Sec. 2.2)     */
/* ------------------------------------------------------------------------ */

/* The input boxes (sorted, unique keys, any levels, a box and its descendants both allowed)
 * represent f = sum_b f_b.  Sum-down (the reconstruction half of the fast wavelet transform):
 * a box that has input boxes below it is interior; so is every box on the path from it to
 * them; every interior box passes its accumulated coefficients to its eight children through
 * the two-scale relation (S = Ubar^{x3} s), and the boxes that are not interior are the
 * leaves of the result, which hold f restricted to them.  A box with no input box above it
 * is a top of the result. */
int orc_reconstruct(int k, long n_in, const uint64_t *keys, const double *coeffs, long cap, uint64_t *out_keys,
                    double *out_coeffs, long *n_out) {
  if (k < 1 || 2 * k > ORC_MAXK || n_in < 0) return -1;
  for (long i = 1; i < n_in; ++i)
    if (keys[i] <= keys[i - 1]) return -1;
  int k3 = k * k * k, kk = 2 * k, kk3 = kk * kk * kk;
  double U0[ORC_MAXK * ORC_MAXK], U1[ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U0, U1);
  double Ub[2 * ORC_MAXK * ORC_MAXK];
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ub[(cc * k + i) * k + j] = (cc == 0 ? U0 : U1)[i * k + j];
  /* top level of every input box: the shallowest input box above it or itself */
  int *top = (int *)malloc(sizeof(int) * (n_in > 0 ? n_in : 1));
  int nmin = 20, nmax = -1;
  for (long b = 0; b < n_in; ++b) {
    int lv;
    long x, y, z;
    split_key(keys[b], &lv, &x, &y, &z);
    top[b] = lv;
    for (int m = 0; m < lv; ++m)
      if (find_key(keys, n_in, make_key(m, x >> (lv - m), y >> (lv - m), z >> (lv - m))) >= 0) {
        top[b] = m;
        break;
      }
    if (lv < nmin) nmin = lv;
    if (lv > nmax) nmax = lv;
  }
  long nout = 0;
  /* R: the result's boxes of the current level with their accumulated coefficients */
  orc_set R = {0, NULL, NULL};
  for (int n = nmin; n <= nmax; ++n) {
    /* interior boxes of level n: ancestors (at level n) of deeper input boxes with top <= n */
    uint64_t *I = (uint64_t *)malloc(sizeof(uint64_t) * (n_in > 0 ? n_in : 1));
    long nI = 0;
    for (long b = 0; b < n_in; ++b) {
      int lv;
      long x, y, z;
      split_key(keys[b], &lv, &x, &y, &z);
      if (lv > n && top[b] <= n) I[nI++] = make_key(n, x >> (lv - n), y >> (lv - n), z >> (lv - n));
    }
    qsort(I, nI, sizeof(uint64_t), cmp_u64v);
    long u = 0;
    for (long i = 0; i < nI; ++i)
      if (i == 0 || I[i] != I[i - 1]) I[u++] = I[i];
    nI = u;
    /* R_n = children passed down from level n-1 (already in R) plus the tops of level n */
    long ntop = 0;
    for (long b = 0; b < n_in; ++b)
      if ((int)(keys[b] >> 57) == n && top[b] == n) ++ntop;
    orc_set Rn;
    Rn.n = R.n + ntop;
    Rn.keys = (uint64_t *)malloc(sizeof(uint64_t) * (Rn.n > 0 ? Rn.n : 1));
    Rn.v = (double *)malloc(sizeof(double) * (Rn.n > 0 ? Rn.n : 1) * k3);
    long q = 0;
    for (long i = 0; i < R.n; ++i, ++q) {
      Rn.keys[q] = R.keys[i];
      memcpy(Rn.v + q * k3, R.v + i * k3, sizeof(double) * k3);
    }
    for (long b = 0; b < n_in; ++b)
      if ((int)(keys[b] >> 57) == n && top[b] == n) {
        Rn.keys[q] = keys[b];
        memcpy(Rn.v + q * k3, coeffs + b * k3, sizeof(double) * k3);
        ++q;
      }
    /* key order */
    long *perm = (long *)malloc(sizeof(long) * (Rn.n > 0 ? Rn.n : 1));
    for (long i = 0; i < Rn.n; ++i) perm[i] = i;
    for (long i = 1; i < Rn.n; ++i) {
      long pi = perm[i], j = i - 1;
      while (j >= 0 && Rn.keys[perm[j]] > Rn.keys[pi]) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = pi;
    }
    orc_set Rs;
    Rs.n = Rn.n;
    Rs.keys = (uint64_t *)malloc(sizeof(uint64_t) * (Rs.n > 0 ? Rs.n : 1));
    Rs.v = (double *)malloc(sizeof(double) * (Rs.n > 0 ? Rs.n : 1) * k3);
    for (long i = 0; i < Rs.n; ++i) {
      Rs.keys[i] = Rn.keys[perm[i]];
      memcpy(Rs.v + i * k3, Rn.v + perm[i] * k3, sizeof(double) * k3);
    }
    free(perm);
    free(Rn.keys);
    free(Rn.v);
    /* the input boxes of level n below a top add their own coefficients */
    for (long b = 0; b < n_in; ++b)
      if ((int)(keys[b] >> 57) == n && top[b] < n) {
        long p = find_key(Rs.keys, Rs.n, keys[b]);
        if (p < 0) { /* cannot happen: its parent is interior */
          free(I);
          free(Rs.keys);
          free(Rs.v);
          free(R.keys);
          free(R.v);
          free(top);
          return -3;
        }
        for (int i = 0; i < k3; ++i) Rs.v[p * k3 + i] += coeffs[b * k3 + i];
      }
    /* leaves out, interior boxes down */
    long nnext = 0;
    for (long p = 0; p < Rs.n; ++p)
      if (find_key(I, nI, Rs.keys[p]) >= 0) ++nnext;
    orc_set Nx;
    Nx.n = 8 * nnext;
    Nx.keys = (uint64_t *)malloc(sizeof(uint64_t) * (Nx.n > 0 ? Nx.n : 1));
    Nx.v = (double *)malloc(sizeof(double) * (Nx.n > 0 ? Nx.n : 1) * k3);
    double *S = (double *)malloc(sizeof(double) * kk3);
    long c = 0;
    for (long p = 0; p < Rs.n; ++p) {
      if (find_key(I, nI, Rs.keys[p]) < 0) {
        if (nout < cap) {
          out_keys[nout] = Rs.keys[p];
          memcpy(out_coeffs + nout * k3, Rs.v + p * k3, sizeof(double) * k3);
        }
        ++nout;
        continue;
      }
      unfilter3(k, Ub, Rs.v + p * k3, S);
      int lv;
      long x, y, z;
      split_key(Rs.keys[p], &lv, &x, &y, &z);
      for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy)
          for (int cz = 0; cz < 2; ++cz, ++c) {
            Nx.keys[c] = make_key(n + 1, 2 * x + cx, 2 * y + cy, 2 * z + cz);
            double *o = Nx.v + c * k3;
            for (int i = 0; i < k; ++i)
              for (int j = 0; j < k; ++j)
                for (int l = 0; l < k; ++l) o[(i * k + j) * k + l] = S[((cx * k + i) * kk + cy * k + j) * kk + cz * k + l];
          }
    }
    free(S);
    free(I);
    free(Rs.keys);
    free(Rs.v);
    free(R.keys);
    free(R.v);
    R = Nx;
  }
  free(R.keys);
  free(R.v);
  free(top);
  *n_out = nout;
  return nout > cap ? -4 : 0;
}

/* Truncate (Sec. 2.1 refinement test run backwards): on disjoint leaves, from the deepest level
 * up, eight sibling leaves whose detail d = S - Ubar^{x3} s (s = the parent's filter of their
 * tensor S) has ||d||_F <= thresh are replaced by their parent holding s.  A merged parent can
 * merge again one level up.  Since d is orthogonal to the parent's space, the L2 error is
 * sqrt(sum ||d||^2) over the merges, returned in *err2 as sum ||d||^2. */
int orc_truncate(int k, long n_in, const uint64_t *keys, const double *coeffs, double thresh, long cap,
                 uint64_t *out_keys, double *out_coeffs, long *n_out, double *err2) {
  if (k < 1 || 2 * k > ORC_MAXK || n_in < 0) return -1;
  for (long i = 1; i < n_in; ++i)
    if (keys[i] <= keys[i - 1]) return -1;
  int k3 = k * k * k, kk = 2 * k, kk3 = kk * kk * kk;
  double U0[ORC_MAXK * ORC_MAXK], U1[ORC_MAXK * ORC_MAXK];
  orc_two_scale(k, U0, U1);
  double Ub[2 * ORC_MAXK * ORC_MAXK];
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ub[(cc * k + i) * k + j] = (cc == 0 ? U0 : U1)[i * k + j];
  /* leaves by level */
  orc_set lev[20];
  memset(lev, 0, sizeof(lev));
  for (long i = 0; i < n_in; ++i) {
    int n = (int)(keys[i] >> 57);
    if (n > 19) return -1;
    lev[n].n++;
  }
  for (int n = 0; n < 20; ++n) {
    lev[n].keys = (uint64_t *)malloc(sizeof(uint64_t) * (lev[n].n + 1) * 2);
    lev[n].v = (double *)malloc(sizeof(double) * (lev[n].n + 1) * 2 * k3);
    lev[n].n = 0;
  }
  /* room for merged parents: at most one per eight leaves of the level below */
  long room[20];
  for (int n = 0; n < 20; ++n) room[n] = 0;
  for (long i = 0; i < n_in; ++i) {
    int n = (int)(keys[i] >> 57);
    orc_set *L = &lev[n];
    L->keys[L->n] = keys[i];
    memcpy(L->v + L->n * k3, coeffs + i * k3, sizeof(double) * k3);
    L->n++;
  }
  for (int n = 0; n < 20; ++n) room[n] = lev[n].n;
  /* grow the parent levels' arrays to hold merges coming from below */
  for (int n = 18; n >= 0; --n) {
    long extra = 0;
    for (int m = n + 1; m < 20; ++m) extra += room[m] / 8 + 1;
    lev[n].keys = (uint64_t *)realloc(lev[n].keys, sizeof(uint64_t) * (room[n] + extra + 1));
    lev[n].v = (double *)realloc(lev[n].v, sizeof(double) * (room[n] + extra + 1) * k3);
  }
  double e2 = 0.0;
  double *S = (double *)malloc(sizeof(double) * kk3), *B = (double *)malloc(sizeof(double) * kk3);
  double *s = (double *)malloc(sizeof(double) * k3);
  char *gone = NULL;
  for (int n = 19; n >= 1; --n) {
    orc_set *L = &lev[n];
    if (L->n == 0) continue;
    /* the level's leaves in key order (merges from below were appended) */
    long *perm = (long *)malloc(sizeof(long) * L->n);
    for (long i = 0; i < L->n; ++i) perm[i] = i;
    for (long i = 1; i < L->n; ++i) {
      long pi = perm[i], j = i - 1;
      while (j >= 0 && L->keys[perm[j]] > L->keys[pi]) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = pi;
    }
    uint64_t *sk = (uint64_t *)malloc(sizeof(uint64_t) * L->n);
    double *sv = (double *)malloc(sizeof(double) * L->n * k3);
    for (long i = 0; i < L->n; ++i) {
      sk[i] = L->keys[perm[i]];
      memcpy(sv + i * k3, L->v + perm[i] * k3, sizeof(double) * k3);
    }
    free(perm);
    memcpy(L->keys, sk, sizeof(uint64_t) * L->n);
    memcpy(L->v, sv, sizeof(double) * L->n * k3);
    free(sk);
    free(sv);
    gone = (char *)calloc(L->n, 1);
    for (long i = 0; i < L->n; ++i) {
      int lv;
      long x, y, z;
      split_key(L->keys[i], &lv, &x, &y, &z);
      if ((x & 1) || (y & 1) || (z & 1)) continue; /* each parent once, from its first child */
      long idx[8];
      int all = 1;
      for (int c = 0; c < 8 && all; ++c) {
        idx[c] = find_key(L->keys, L->n, make_key(n, x + (c >> 2), y + ((c >> 1) & 1), z + (c & 1)));
        if (idx[c] < 0) all = 0;
      }
      if (!all) continue;
      for (int c = 0; c < 8; ++c) {
        int cx = c >> 2, cy = (c >> 1) & 1, cz = c & 1;
        const double *v = L->v + idx[c] * k3;
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b)
            for (int d = 0; d < k; ++d) S[((cx * k + a) * kk + cy * k + b) * kk + cz * k + d] = v[(a * k + b) * k + d];
      }
      filter3(k, Ub, S, s);
      unfilter3(k, Ub, s, B);
      double dn = 0.0;
      for (int q = 0; q < kk3; ++q) dn += (S[q] - B[q]) * (S[q] - B[q]);
      if (sqrt(dn) > thresh) continue;
      e2 += dn;
      for (int c = 0; c < 8; ++c) gone[idx[c]] = 1;
      orc_set *P = &lev[n - 1];
      P->keys[P->n] = make_key(n - 1, x >> 1, y >> 1, z >> 1);
      memcpy(P->v + P->n * k3, s, sizeof(double) * k3);
      P->n++;
    }
    long w = 0;
    for (long i = 0; i < L->n; ++i)
      if (!gone[i]) {
        L->keys[w] = L->keys[i];
        memmove(L->v + w * k3, L->v + i * k3, sizeof(double) * k3);
        ++w;
      }
    L->n = w;
    free(gone);
  }
  /* level 0 may also have received merges: sort it too */
  {
    orc_set *L = &lev[0];
    for (long i = 1; i < L->n; ++i)
      for (long j = i; j > 0 && L->keys[j - 1] > L->keys[j]; --j) {
        uint64_t tk = L->keys[j];
        L->keys[j] = L->keys[j - 1];
        L->keys[j - 1] = tk;
        for (int q = 0; q < k3; ++q) {
          double tv = L->v[j * k3 + q];
          L->v[j * k3 + q] = L->v[(j - 1) * k3 + q];
          L->v[(j - 1) * k3 + q] = tv;
        }
      }
  }
  long nout = 0;
  for (int n = 0; n < 20; ++n)
    for (long i = 0; i < lev[n].n; ++i, ++nout)
      if (nout < cap) {
        out_keys[nout] = lev[n].keys[i];
        memcpy(out_coeffs + nout * k3, lev[n].v + i * k3, sizeof(double) * k3);
      }
  for (int n = 0; n < 20; ++n) {
    free(lev[n].keys);
    free(lev[n].v);
  }
  free(S);
  free(B);
  free(s);
  *n_out = nout;
  *err2 = e2;
  return nout > cap ? -4 : 0;
}
