/*
 * psht_oracle.c -- plain FP64 CPU oracle for partial-sky spin-s synthesis general
 * and its adjoint (Carron & Reinecke, "Fast partial-sky spherical harmonic transforms").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, imports or calls this
 * file; only the test suite, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every routine is the plain definition, written for a reader to check against the paper:
 *   - Wigner small-d columns d^l_{m,m'}(beta), l = 0..lmax, by the textbook three-term
 *     recurrence in l (Edmonds), seeded by Wigner's closed form for l0 = max(|m|,|m'|),
 *     in exact "mantissa x 2^e" arithmetic (no value is ever flushed on purpose: results are
 *     ldexp'ed at the end, so only genuine double underflow loses anything).
 *   - sY_lm(theta, phi) = sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi}   (appendix, eq. Ylm)
 *   - ring Fourier coefficients F(theta)[m] = -sum_l (g+ic)_lm sY_lm(theta, 0)   (eq. syn)
 *     with the reality rule a_{l,-m} = (-1)^m a*_lm for g and c separately     (Sec. I)
 *   - their exact transpose, followed by the projection onto (g~, c~) of the adjoint
 *     synthesis general equation (Sec. I).
 *   - ES-kernel interpolation (type-2) and spreading (type-1) on a periodic 2-D grid
 *     (Barnett, Magland & af Klinteberg 2019, the NUFFT the paper defers to, Sec. I.B, II.E).
 *
 * Complex arrays are interleaved (re, im) doubles.  Harmonic coefficients use the packed
 * m-major layout idx(l, m) = m(2 lmax + 1 - m)/2 + l, 0 <= m <= l <= lmax.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_RESCALE_EXP 256          /* renormalise the mantissa pair when |d| > 2^256 */

static inline int64_t alm_idx(int lmax, int l, int m) {
  return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

/* log2 of sqrt(binomial(n, k)) in long double. */
static long double log2_sqrt_binom(int n, int k) {
  long double v = lgammal((long double)n + 1.0L) - lgammal((long double)k + 1.0L) -
                  lgammal((long double)(n - k) + 1.0L);
  return 0.5L * v / logl(2.0L);
}

/*
 * Wigner small-d column: out[l] = d^l_{m,mp}(beta) for l = 0..lmax, with m >= 0 and any mp.
 * cb = cos(beta), ch = cos(beta/2), sh = sin(beta/2) are passed in so the caller controls
 * how they are rounded (half-angle values are not recomputed from cb).
 *
 * Seed (Wigner's closed form):
 *   if m >= |mp|: l0 = m,    d^m_{m,mp}  = (-1)^(m-mp) sqrt(C(2m, m+mp)) ch^(m+mp) sh^(m-mp)
 *   else:         l0 = |mp|, use d^j_{m,mp} = d^j_{-mp,-m} (mp < 0) or
 *                 d^j_{m,mp} = (-1)^(mp-m) d^j_{mp,m} (mp > 0) and the same closed form.
 * Recurrence (l >= l0, d^{l0-1} = 0):
 *   d^{l+1} = (l+1)(2l+1)/sqrt(((l+1)^2-m^2)((l+1)^2-mp^2))
 *             * [ (cb - m mp/(l(l+1))) d^l - sqrt((l^2-m^2)(l^2-mp^2))/(l(2l+1)) d^{l-1} ]
 */
void orc_wigner_d_column(int lmax, int m, int mp, double cb, double ch, double sh, double* out) {
  int amp = mp < 0 ? -mp : mp;
  int l0 = m > amp ? m : amp;
  for (int l = 0; l <= lmax && l < l0; ++l) out[l] = 0.0;
  if (l0 > lmax) return;
  /* closed-form seed: sign * sqrt(C(2 l0, p)) * ch^p * sh^q with p + q = 2 l0 */
  int p, q, sign;
  if (m >= amp) {
    p = m + mp; q = m - mp; sign = ((m - mp) & 1) ? -1 : 1;
  } else if (mp < 0) {
    /* d^j_{m,mp} = d^j_{-mp,-m}: top index j = -mp, second index -m */
    p = amp - m; q = amp + m; sign = ((amp + m) & 1) ? -1 : 1;
  } else {
    /* d^j_{m,mp} = (-1)^(mp-m) d^j_{mp,m}: top index j = mp, second index m */
    /* the two factors (-1)^(mp-m) and (-1)^(j-m) with j = mp cancel */
    p = amp + m; q = amp - m; sign = 1;
  }
  double mant; int e;
  if ((p > 0 && ch == 0.0) || (q > 0 && sh == 0.0)) {
    for (int l = l0; l <= lmax; ++l) out[l] = 0.0;
    return;
  }
  {
    long double lg = log2_sqrt_binom(2 * l0, p);
    if (p > 0) lg += (long double)p * log2l(fabsl((long double)ch));
    if (q > 0) lg += (long double)q * log2l(fabsl((long double)sh));
    long double fl = floorl(lg);
    e = (int)fl;
    mant = (double)exp2l(lg - fl);
    /* signs of ch, sh (beta may lie outside [0, pi] in tests) */
    if (p > 0 && ch < 0 && (p & 1)) sign = -sign;
    if (q > 0 && sh < 0 && (q & 1)) sign = -sign;
    mant *= sign;
  }
  double dprev = 0.0, dcur = mant;
  out[l0] = ldexp(dcur, e);
  const double m2 = (double)m * m, mp2 = (double)mp * mp, mmp = (double)m * mp;
  const double big = ldexp(1.0, ORC_RESCALE_EXP);
  for (int l = l0; l < lmax; ++l) {
    double lp1 = l + 1.0;
    double a = lp1 * (2.0 * l + 1.0) / sqrt((lp1 * lp1 - m2) * (lp1 * lp1 - mp2));
    double shift = (l == 0) ? 0.0 : mmp / ((double)l * (l + 1.0));
    double c = (l == 0) ? 0.0 : sqrt(((double)l * l - m2) * ((double)l * l - mp2)) / ((double)l * (2.0 * l + 1.0));
    double dnext = a * ((cb - shift) * dcur - c * dprev);
    dprev = dcur; dcur = dnext;
    if (fabs(dcur) > big) {
      dcur = ldexp(dcur, -ORC_RESCALE_EXP);
      dprev = ldexp(dprev, -ORC_RESCALE_EXP);
      e += ORC_RESCALE_EXP;
    }
    out[l + 1] = ldexp(dcur, e);
  }
}

static inline void half_angles(double beta, double* cb, double* ch, double* sh) {
  *cb = cos(beta); *ch = cos(0.5 * beta); *sh = sin(0.5 * beta);
}

/*
 * Ring Fourier coefficients of the synthesis general map at colatitude theta:
 *   F[m] = -sum_{l} u_lm N_l d^l_{m,-s}(theta),  u = g + i c,  |m| <= mmax,
 * so that f(theta, phi) = sum_m F[m] e^{i m phi}.  For m > 0 the negative order uses
 *   u_{l,-m} N_l d^l_{-m,-s} = (-1)^s (g*_lm + i c*_lm) N_l d^l_{m,s}.
 * Im(g_l0), Im(c_l0) and l < s are ignored.  Output F[(m + mmax)], interleaved complex.
 * d1, d2 are caller scratch of length lmax+1.
 */
static void ring_coeffs_one(int lmax, int s, int mmax, const double* g, const double* c, double theta,
                            double* F, double* d1, double* d2) {
  double cb, ch, sh; half_angles(theta, &cb, &ch, &sh);
  int mtop = mmax < lmax ? mmax : lmax;
  memset(F, 0, sizeof(double) * 2 * (2 * mmax + 1));
  double sgn_s = (s & 1) ? -1.0 : 1.0;
  for (int m = 0; m <= mtop; ++m) {
    orc_wigner_d_column(lmax, m, -s, cb, ch, sh, d1);
    if (s != 0) orc_wigner_d_column(lmax, m, s, cb, ch, sh, d2);
    const double* dd2 = s != 0 ? d2 : d1;
    double pr = 0, pi = 0, qr = 0, qi = 0;
    for (int l = (m > s ? m : s); l <= lmax; ++l) {
      int64_t k = alm_idx(lmax, l, m);
      double gr = g[2 * k], gi = (m == 0) ? 0.0 : g[2 * k + 1];
      double cr = c ? c[2 * k] : 0.0, ci = (c && m != 0) ? c[2 * k + 1] : 0.0;
      double nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
      /* u = g + i c = (gr - ci) + i (gi + cr);  v = g* + i c* = (gr + ci) + i (cr - gi) */
      pr += nl * d1[l] * (gr - ci);
      pi += nl * d1[l] * (gi + cr);
      qr += nl * dd2[l] * (gr + ci);
      qi += nl * dd2[l] * (cr - gi);
    }
    F[2 * (mmax + m)] = -pr;
    F[2 * (mmax + m) + 1] = -pi;
    if (m > 0) {
      F[2 * (mmax - m)] = -sgn_s * qr;
      F[2 * (mmax - m) + 1] = -sgn_s * qi;
    }
  }
}

/* F[k][m + mmax] for nr rings at colatitudes theta[k].  OpenMP over rings. */
void orc_ring_synthesis(int lmax, int s, int mmax, const double* g, const double* c, int64_t nr,
                        const double* theta, double* F) {
  int64_t stride = 2 * (2 * (int64_t)mmax + 1);
#pragma omp parallel
  {
    double* d1 = (double*)malloc(sizeof(double) * (lmax + 1));
    double* d2 = (double*)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (int64_t k = 0; k < nr; ++k) ring_coeffs_one(lmax, s, mmax, g, c, theta[k], F + k * stride, d1, d2);
    free(d1); free(d2);
  }
}

/*
 * Transpose of orc_ring_synthesis followed by the adjoint projection:
 *   ut_{l,m}  = -sum_k N_l d^l_{m,-s}(theta_k) G_k[m]
 *   ut_{l,-m} = -sum_k N_l d^l_{-m,-s}(theta_k) G_k[-m] = -(-1)^(m-s) sum_k N_l d^l_{m,s}(theta_k) G_k[-m]
 *   g~_lm = (ut_lm + (-1)^m conj(ut_{l,-m}))/2,  c~_lm = (ut_lm - (-1)^m conj(ut_{l,-m}))/(2i)
 * (equivalent to the adjoint synthesis general formula via sY*_lm = (-1)^(s+m) _{-s}Y_{l,-m}).
 * G is [k][m + mmax] interleaved.  gt, ct (nullable) receive packed coefficients; l < s and
 * Im at m = 0 are written as 0.  OpenMP over m.
 */
void orc_ring_adjoint(int lmax, int s, int mmax, int64_t nr, const double* theta, const double* G,
                      double* gt, double* ct) {
  int64_t nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  memset(gt, 0, sizeof(double) * 2 * nalm);
  if (ct) memset(ct, 0, sizeof(double) * 2 * nalm);
  int64_t stride = 2 * (2 * (int64_t)mmax + 1);
  int mtop = mmax < lmax ? mmax : lmax;
#pragma omp parallel
  {
    double* d1 = (double*)malloc(sizeof(double) * (lmax + 1));
    double* d2 = (double*)malloc(sizeof(double) * (lmax + 1));
    double* up = (double*)malloc(sizeof(double) * 2 * (lmax + 1));
    double* um = (double*)malloc(sizeof(double) * 2 * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (int m = 0; m <= mtop; ++m) {
      memset(up, 0, sizeof(double) * 2 * (lmax + 1));
      memset(um, 0, sizeof(double) * 2 * (lmax + 1));
      int l0 = m > s ? m : s;
      for (int64_t k = 0; k < nr; ++k) {
        double cb, ch, sh; half_angles(theta[k], &cb, &ch, &sh);
        orc_wigner_d_column(lmax, m, -s, cb, ch, sh, d1);
        if (s != 0) orc_wigner_d_column(lmax, m, s, cb, ch, sh, d2);
        const double* dd2 = s != 0 ? d2 : d1;
        const double* Gk = G + k * stride;
        double gpr = Gk[2 * (mmax + m)], gpi = Gk[2 * (mmax + m) + 1];
        double gmr = Gk[2 * (mmax - m)], gmi = Gk[2 * (mmax - m) + 1];
        for (int l = l0; l <= lmax; ++l) {
          up[2 * l] += d1[l] * gpr; up[2 * l + 1] += d1[l] * gpi;
          um[2 * l] += dd2[l] * gmr; um[2 * l + 1] += dd2[l] * gmi;
        }
      }
      double sg = (((m - s) % 2) != 0) ? -1.0 : 1.0;  /* (-1)^(m-s) */
      double sm = (m & 1) ? -1.0 : 1.0;                /* (-1)^m */
      for (int l = l0; l <= lmax; ++l) {
        double nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
        double a_r = -nl * up[2 * l], a_i = -nl * up[2 * l + 1];             /* ut_{l,m}  */
        double b_r = -sg * nl * um[2 * l], b_i = -sg * nl * um[2 * l + 1];   /* ut_{l,-m} */
        /* w = (-1)^m conj(ut_{l,-m}) */
        double w_r = sm * b_r, w_i = -sm * b_i;
        int64_t idx = alm_idx(lmax, l, m);
        if (m == 0) {
          gt[2 * idx] = a_r; gt[2 * idx + 1] = 0.0;
          if (ct) { ct[2 * idx] = a_i; ct[2 * idx + 1] = 0.0; }
        } else {
          gt[2 * idx] = 0.5 * (a_r + w_r); gt[2 * idx + 1] = 0.5 * (a_i + w_i);
          /* (x)/(2i) = -i x / 2 : (xr + i xi)(-i)/2 = (xi - i xr)/2 */
          double xr = a_r - w_r, xi = a_i - w_i;
          if (ct) { ct[2 * idx] = 0.5 * xi; ct[2 * idx + 1] = -0.5 * xr; }
        }
      }
    }
    free(d1); free(d2); free(up); free(um);
  }
}

/* Direct summation of synthesis general at points: f_p = sum_m F(theta_p)[m] e^{i m phi_p}. */
void orc_direct_synthesis(int lmax, int s, const double* g, const double* c, int64_t npts,
                          const double* theta, const double* phi, double* f) {
  int64_t stride = 2 * (2 * (int64_t)lmax + 1);
#pragma omp parallel
  {
    double* d1 = (double*)malloc(sizeof(double) * (lmax + 1));
    double* d2 = (double*)malloc(sizeof(double) * (lmax + 1));
    double* F = (double*)malloc(sizeof(double) * stride);
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < npts; ++p) {
      ring_coeffs_one(lmax, s, lmax, g, c, theta[p], F, d1, d2);
      double fr = 0, fi = 0;
      for (int m = -lmax; m <= lmax; ++m) {
        double cr = cos(m * phi[p]), si = sin(m * phi[p]);
        double ar = F[2 * (lmax + m)], ai = F[2 * (lmax + m) + 1];
        fr += ar * cr - ai * si; fi += ar * si + ai * cr;
      }
      f[2 * p] = fr; f[2 * p + 1] = fi;
    }
    free(d1); free(d2); free(F);
  }
}

/* Direct adjoint synthesis general at points: G_p[m] = f_p e^{-i m phi_p}, then orc_ring_adjoint. */
void orc_direct_adjoint(int lmax, int s, int64_t npts, const double* theta, const double* phi,
                        const double* f, double* gt, double* ct) {
  int64_t stride = 2 * (2 * (int64_t)lmax + 1);
  double* G = (double*)malloc(sizeof(double) * stride * (npts > 0 ? npts : 1));
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < npts; ++p) {
    for (int m = -lmax; m <= lmax; ++m) {
      double cr = cos(m * phi[p]), si = -sin(m * phi[p]);
      G[p * stride + 2 * (lmax + m)] = f[2 * p] * cr - f[2 * p + 1] * si;
      G[p * stride + 2 * (lmax + m) + 1] = f[2 * p] * si + f[2 * p + 1] * cr;
    }
  }
  orc_ring_adjoint(lmax, s, lmax, npts, theta, G, gt, ct);
  free(G);
}

/* ES kernel psi(z) = exp(beta (sqrt(1 - z^2) - 1)) for |z| <= 1, else 0. */
static inline double es_kernel(double z, double beta) {
  if (z < -1.0 || z > 1.0) return 0.0;
  return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}

/*
 * Type-2 interpolation at points with fractional grid coordinates (t_p, u_p):
 *   r0 = ceil(t - W/2), q0 = ceil(u - W/2)
 *   f_p = sum_{i,k<W} psi(2(t - r0 - i)/W) psi(2(u - q0 - k)/W) grid[r0 + i - r_lo][(q0 + k) mod nphi]
 * grid is [nrows][nphi] interleaved complex holding rows r_lo .. r_lo + nrows - 1.
 */
void orc_interp(int64_t npts, const double* t, const double* u, int W, double beta, int64_t r_lo,
                int64_t nrows, int64_t nphi, const double* grid, double* f) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < npts; ++p) {
    int64_t r0 = (int64_t)ceil(t[p] - 0.5 * W), q0 = (int64_t)ceil(u[p] - 0.5 * W);
    double fr = 0, fi = 0;
    for (int i = 0; i < W; ++i) {
      double wr = es_kernel(2.0 * (t[p] - (double)(r0 + i)) / W, beta);
      int64_t row = r0 + i - r_lo;
      if (row < 0 || row >= nrows) continue; /* never happens when rows cover the points */
      for (int k = 0; k < W; ++k) {
        double wq = es_kernel(2.0 * (u[p] - (double)(q0 + k)) / W, beta);
        int64_t q = ((q0 + k) % nphi + nphi) % nphi;
        const double* gv = grid + 2 * (row * nphi + q);
        fr += wr * wq * gv[0]; fi += wr * wq * gv[1];
      }
    }
    f[2 * p] = fr; f[2 * p + 1] = fi;
  }
}

/*
 * Type-1 spreading, the transpose of orc_interp: grid[r][q] = sum_p psi psi f_p over the same
 * windows.  Written cell-by-row: each grid row sums the points whose window covers it, so no
 * two threads write the same row.  order[] lists the points sorted by r0 ascending.
 */
void orc_spread(int64_t npts, const double* t, const double* u, const int64_t* order, int W, double beta,
                int64_t r_lo, int64_t nrows, int64_t nphi, const double* f, double* grid) {
  memset(grid, 0, sizeof(double) * 2 * nrows * nphi);
  int64_t* r0s = (int64_t*)malloc(sizeof(int64_t) * (npts > 0 ? npts : 1));
  for (int64_t i = 0; i < npts; ++i) r0s[i] = (int64_t)ceil(t[order[i]] - 0.5 * W);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t row = 0; row < nrows; ++row) {
    int64_t r = row + r_lo;
    /* points with r0 in [r - W + 1, r] */
    int64_t lo = 0, hi = npts;
    while (lo < hi) { int64_t mid = (lo + hi) / 2; if (r0s[mid] < r - W + 1) lo = mid + 1; else hi = mid; }
    for (int64_t ii = lo; ii < npts && r0s[ii] <= r; ++ii) {
      int64_t p = order[ii];
      double wr = es_kernel(2.0 * (t[p] - (double)r) / W, beta);
      int64_t q0 = (int64_t)ceil(u[p] - 0.5 * W);
      for (int k = 0; k < W; ++k) {
        double wq = es_kernel(2.0 * (u[p] - (double)(q0 + k)) / W, beta);
        int64_t q = ((q0 + k) % nphi + nphi) % nphi;
        double* gv = grid + 2 * (row * nphi + q);
        gv[0] += wr * wq * f[2 * p]; gv[1] += wr * wq * f[2 * p + 1];
      }
    }
  }
  free(r0s);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel regions (timing runs on fewer cores than the machine has). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/*
 * Selected outputs of the direct adjoint synthesis general: for each (l_k, m_k), m_k >= 0,
 *   ut_{l,m}  = -sum_p f_p N_l d^l_{m,-s}(theta_p) e^{-i m phi_p}
 *   ut_{l,-m} = -(-1)^(m-s) sum_p f_p N_l d^l_{m,s}(theta_p) e^{+i m phi_p}
 * projected as in orc_ring_adjoint.  Cost per point O(l_k - max(m_k, s)), so the full point set
 * of a large workload can be summed for coefficients close to the diagonal or of low degree.
 */
void orc_direct_adjoint_lm(int s, int64_t npts, const double* theta, const double* phi, const double* f, int nsel,
                           const int* ls, const int* ms, double* gt, double* ct) {
  for (int k = 0; k < nsel; ++k) {
    const int l = ls[k], m = ms[k];
    double ar = 0, ai = 0, br = 0, bi = 0;
    if (l >= (m > s ? m : s)) {
#pragma omp parallel reduction(+ : ar, ai, br, bi)
      {
        double* d1 = (double*)malloc(sizeof(double) * (l + 1));
        double* d2 = (double*)malloc(sizeof(double) * (l + 1));
#pragma omp for schedule(static)
        for (int64_t p = 0; p < npts; ++p) {
          double cb, ch, sh; half_angles(theta[p], &cb, &ch, &sh);
          orc_wigner_d_column(l, m, -s, cb, ch, sh, d1);
          orc_wigner_d_column(l, m, s, cb, ch, sh, d2);
          const double cr = cos(m * phi[p]), si = sin(m * phi[p]);
          const double fr = f[2 * p], fi = f[2 * p + 1];
          /* f e^{-i m phi} and f e^{+i m phi} */
          ar += d1[l] * (fr * cr + fi * si); ai += d1[l] * (fi * cr - fr * si);
          br += d2[l] * (fr * cr - fi * si); bi += d2[l] * (fi * cr + fr * si);
        }
        free(d1); free(d2);
      }
    }
    const double nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
    const double sg = (((m - s) % 2) != 0) ? -1.0 : 1.0, sm = (m & 1) ? -1.0 : 1.0;
    const double a_r = -nl * ar, a_i = -nl * ai, b_r = -sg * nl * br, b_i = -sg * nl * bi;
    const double w_r = sm * b_r, w_i = -sm * b_i;
    if (l < s) { gt[2 * k] = gt[2 * k + 1] = ct[2 * k] = ct[2 * k + 1] = 0.0; continue; }
    if (m == 0) {
      gt[2 * k] = a_r; gt[2 * k + 1] = 0.0; ct[2 * k] = a_i; ct[2 * k + 1] = 0.0;
    } else {
      gt[2 * k] = 0.5 * (a_r + w_r); gt[2 * k + 1] = 0.5 * (a_i + w_i);
      ct[2 * k] = 0.5 * (a_i - w_i); ct[2 * k + 1] = -0.5 * (a_r - w_r);
    }
  }
}

/*
 * Rotation of one harmonic coefficient set (a real field's g or c) by the Euler angles
 * (alpha, beta, gamma) of R = R_z(alpha) R_y(beta) R_z(gamma), plain definition:
 *   a'_{l,m} = sum_{m'=-l}^{l} e^{-i m alpha} d^l_{m,m'}(beta) e^{-i m' gamma} a_{l,m'},   m >= 0,
 * with a_{l,-m'} = (-1)^{m'} a*_{l,m'}; Im(a_l0) is ignored.  The rotated field is the original
 * one carried along by R (scalar case: f'(n) = f(R^-1 n)); the appendix's Wigner small-d is the
 * one used everywhere in this file.  nsel < 0 computes every (l, m); otherwise only the nsel
 * pairs (ls[k], ms[k]), written to out[k] (each costs O(l^2), so single coefficients of a large
 * band limit stay cheap).  Cost of the full form O(lmax^3).
 */
static void rot_one_m(int lmax, int m, int lsel, double alpha, double gamma, double cb, double ch, double sh,
                      const double* a, double* acc /* 2*(lmax+1) */, double* d) {
  const int lhi = lsel >= 0 ? lsel : lmax;
  for (int l = 0; l <= lhi; ++l) acc[2 * l] = acc[2 * l + 1] = 0.0;
  for (int mp = -lhi; mp <= lhi; ++mp) {
    const int amp = mp < 0 ? -mp : mp;
    orc_wigner_d_column(lhi, m, mp, cb, ch, sh, d);
    /* e^{-i m alpha} e^{-i mp gamma} */
    const double ph = -(double)m * alpha - (double)mp * gamma;
    const double er = cos(ph), ei = sin(ph);
    const int l0 = m > amp ? m : amp;
    for (int l = (lsel >= 0 ? lsel : l0); l <= lhi; ++l) {
      if (l < l0) continue;
      const int64_t k = alm_idx(lmax, l, amp);
      double ar = a[2 * k], ai = (amp == 0) ? 0.0 : a[2 * k + 1];
      if (mp < 0) { /* a_{l,-|mp|} = (-1)^|mp| conj(a_{l,|mp|}) */
        const double sg = (amp & 1) ? -1.0 : 1.0;
        ar = sg * ar; ai = -sg * ai;
      }
      const double tr = er * ar - ei * ai, ti = er * ai + ei * ar;
      acc[2 * l] += d[l] * tr;
      acc[2 * l + 1] += d[l] * ti;
    }
  }
}

void orc_rotate_alm(int lmax, double alpha, double beta, double gamma, const double* a, int nsel, const int* ls,
                    const int* ms, double* out) {
  double cb, ch, sh; half_angles(beta, &cb, &ch, &sh);
  if (nsel < 0) {
#pragma omp parallel
    {
      double* acc = (double*)malloc(sizeof(double) * 2 * (lmax + 1));
      double* d = (double*)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
      for (int m = 0; m <= lmax; ++m) {
        rot_one_m(lmax, m, -1, alpha, gamma, cb, ch, sh, a, acc, d);
        for (int l = m; l <= lmax; ++l) {
          const int64_t k = alm_idx(lmax, l, m);
          out[2 * k] = acc[2 * l];
          out[2 * k + 1] = (m == 0) ? 0.0 : acc[2 * l + 1];
        }
      }
      free(acc); free(d);
    }
    return;
  }
#pragma omp parallel
  {
    double* acc = (double*)malloc(sizeof(double) * 2 * (lmax + 1));
    double* d = (double*)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (int k = 0; k < nsel; ++k) {
      rot_one_m(lmax, ms[k], ls[k], alpha, gamma, cb, ch, sh, a, acc, d);
      out[2 * k] = acc[2 * ls[k]];
      out[2 * k + 1] = (ms[k] == 0) ? 0.0 : acc[2 * ls[k] + 1];
    }
    free(acc); free(d);
  }
}
