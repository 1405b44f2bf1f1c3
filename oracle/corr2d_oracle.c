/*
 * FP64 CPU oracle for generalized two-dimensional correlation analysis
 * (Geitner et al., "corr2D: Implementation of Two-Dimensional Correlation
 * Analysis in R", arXiv:1808.00685).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent, slow, obviously
 * correct statement of what the GPU path computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * library never does, and the two share no code, headers or tables.
 *
 * Everything is plain double arithmetic, straight loops, no blocking, no
 * fusion, no FFT.  Each function names the passage of the paper it follows.
 * Where the paper is silent or inconsistent the reading taken is written next
 * to the code (readings R1..R13):
 *
 *  R1  Eq. disint2d sums over all m frequencies; for real input that sum is
 *      real (Eq. symmeFT), so the asynchronous part would vanish.  The package
 *      (Sec. 4.2, FFT snippet) keeps only the half spectrum and counts every
 *      frequency except omega = 0 twice.  That half-spectrum sum is used.
 *  R2  The retained index set is ((1:(m-1)) %/% 2) + 1 in R, i.e. omega =
 *      0..K with K = floor((m-1)/2); omega = 0 once, omega = 1..K twice; for
 *      even m the Nyquist bin m/2 is never used.
 *  R3  Default normalisation 1/(pi (m-1)) (Eq. disint2d and Sec. 4.2); a caller
 *      may override it.
 *  R4  Eqs. pearsonsyn..scaleasyn print a negative exponent in the denominator; the
 *      text says the spectra are DIVIDED by (sigma1 sigma2)^alpha.  The text is
 *      followed: Phi_scaled = Phi / (sigma1 sigma2)^alpha.
 *  R5  sigma is per spectral variable (Eq. stdev), not per spectrum.
 *  R6  sigma uses the chosen reference literally (Eq. stdev), so a user
 *      reference gives sum((y - ref)^2)/(m-1).
 *  R7  sigma = 0 with alpha > 0: the scale factor is taken as 0 (the row and
 *      column of that variable are exactly 0) instead of 0/0.
 *  R8  In hetero correlation each stack defaults to its own mean.
 *  R9  Row index = stack 1 (nu1), column = stack 2 (nu2),
 *      Z = sum_omega w Y1 conj(Y2); DFT sign e^{-i...} (Eq. disFT).
 *  R10 The DC term is kept with weight 1.
 *  R11 The perturbation values do not enter the discrete formula; equal
 *      spacing is assumed (Sec. 2, before Eq. disFT).
 *  R12 Spectral-axis preprocessing: linear interpolation onto
 *      x_k = x_0 + k (x_last - x_0)/(n_out - 1), k = 0..n_out-1, last point
 *      set to x_last exactly; x must be strictly increasing.
 *  R13 Perturbation-axis interpolation (Sec. 4.2): the linear function
 *      (approxfun) and the package's default, splinefun, read as R's default
 *      spline method "fmm" (Forsythe, Malcolm and Moler, 1977): the C^2
 *      interpolating cubic spline whose third derivative on the first and
 *      last interval equals that of the cubic through the first and last four
 *      points; with three points those third derivatives are taken as 0 (the
 *      interpolating parabola), with two points the spline is the line.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* Number of frequencies kept by the half-spectrum sum (reading R2). */
int oracle_num_freq(int m) { return (m - 1) / 2 + 1; }

/* Weight of frequency omega in the half-spectrum sum (readings R1, R2, R10). */
double oracle_weight(int omega) { return omega == 0 ? 1.0 : 2.0; }

/* Default normalisation factor 1/(pi (m-1)) (Eq. disint2d, reading R3). */
double oracle_default_norm(int m) { return 1.0 / (ORACLE_PI * (double)(m - 1)); }

/*
 * Reference spectrum as the perturbation mean (Eq. ref; the package's
 * column mean in Sec. 4.2).  y is m x n row-major with leading dimension ld:
 * row j = perturbation step t_j, column = spectral variable nu.
 */
void oracle_reference_mean(int m, int n, const float* y, long ld, double* ref) {
  for (int v = 0; v < n; ++v) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += (double)y[(long)j * ld + v];
    ref[v] = s / (double)m;
  }
}

/* Dynamic spectra y~ = y - ref inside the perturbation window (Eq. dynspec).
 * Output ydyn is m x n row-major, contiguous. */
void oracle_dynamic(int m, int n, const float* y, long ld, const double* ref, double* ydyn) {
  for (int j = 0; j < m; ++j)
    for (int v = 0; v < n; ++v) ydyn[(long)j * n + v] = (double)y[(long)j * ld + v] - ref[v];
}

/* Standard deviation per spectral variable (Eq. stdev; readings R5, R6). */
void oracle_sigma(int m, int n, const double* ydyn, double* sigma) {
  for (int v = 0; v < n; ++v) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
      double d = ydyn[(long)j * n + v];
      s += d * d;
    }
    sigma[v] = sqrt(s / (double)(m - 1));
  }
}

/* Scale factor applied to one spectral variable: sigma^-alpha, 1 without
 * scaling, 0 for sigma = 0 (Eqs. scalesyn/scaleasyn; readings R4, R7). */
double oracle_scale_factor(double sigma, double alpha) {
  if (!(alpha > 0.0)) return 1.0;
  if (sigma == 0.0) return 0.0;
  return pow(sigma, -alpha);
}

/*
 * Discrete Fourier transform along the perturbation axis (Eq. disFT), kept
 * for omega = 0..K only (reading R2).  Direct O(m^2) sum, no FFT:
 *   Y(nu, omega) = sum_{j=0}^{m-1} y~(nu, t_j) exp(-i 2 pi omega j / m).
 * The angle's integer part omega*j is reduced modulo m before the division so
 * that cos/sin see an argument in [0, 2 pi).  Output Yre/Yim are n x nfreq.
 */
void oracle_dft(int m, int n, const double* ydyn, int nfreq, double* Yre, double* Yim) {
  for (int v = 0; v < n; ++v) {
    for (int w = 0; w < nfreq; ++w) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < m; ++j) {
        long r = ((long)w * (long)j) % (long)m;
        double theta = 2.0 * ORACLE_PI * (double)r / (double)m;
        double d = ydyn[(long)j * n + v];
        re += d * cos(theta);
        im -= d * sin(theta);
      }
      Yre[(long)v * nfreq + w] = re;
      Yim[(long)v * nfreq + w] = im;
    }
  }
}

/*
 * Complex correlation (Eq. disint2d with readings R1, R2, R9):
 *   Z(nu1, nu2) = sum_{omega=0}^{K} w_omega Y1(nu1, omega) conj(Y2(nu2, omega)),
 *   Phi = norm * s1[nu1] * s2[nu2] * Re Z,  Psi = norm * s1 * s2 * Im Z.
 * Only the rows listed in rows[0..nrows) are produced (all rows when rows is
 * NULL and nrows = n1); output row r of phi/psi holds nu1 = rows[r] and has
 * n2 entries.  nthreads > 1 spreads output rows over OpenMP threads.
 */
void oracle_cross_spectrum(int n1, int n2, int nfreq, const double* Yre1, const double* Yim1,
                           const double* Yre2, const double* Yim2, double norm,
                           const double* s1, const double* s2, int nrows, const int* rows,
                           double* phi, double* psi, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int r = 0; r < nrows; ++r) {
    int a = rows ? rows[r] : r;
    for (int b = 0; b < n2; ++b) {
      double zr = 0.0, zi = 0.0;
      for (int w = 0; w < nfreq; ++w) {
        double xr = Yre1[(long)a * nfreq + w], xi = Yim1[(long)a * nfreq + w];
        double yr = Yre2[(long)b * nfreq + w], yi = Yim2[(long)b * nfreq + w];
        double wt = oracle_weight(w);
        /* (xr + i xi) * (yr - i yi) */
        zr += wt * (xr * yr + xi * yi);
        zi += wt * (xi * yr - xr * yi);
      }
      double f = norm * s1[a] * s2[b];
      phi[(long)r * n2 + b] = f * zr;
      psi[(long)r * n2 + b] = f * zi;
    }
  }
  (void)n1;
}

/*
 * Whole corr2d() computation (Sec. 2 three-step summary; Sec. 4.2 order:
 * reference, dynamic spectra, scaling, FT, correlation).
 *   y2 == NULL selects homo correlation (stack 2 := stack 1).
 *   ref_mode 0: each stack uses its own perturbation mean (R8);
 *   ref_mode 1: ref1/ref2 are caller-supplied reference spectra.
 *   norm <= 0 selects the default 1/(pi (m-1)).
 *   alpha > 0 divides by (sigma1 sigma2)^alpha.
 *   rows/nrows select output rows (see oracle_cross_spectrum).
 *   sigma1/sigma2 (nullable) receive the per-variable standard deviations.
 * Returns 0 on success, 1 on invalid arguments, 2 on allocation failure.
 */
int oracle_corr2d(int m, int n1, const float* y1, long ld1, int n2, const float* y2, long ld2,
                  int ref_mode, const float* ref1, const float* ref2, double norm, double alpha,
                  int nrows, const int* rows, double* phi, double* psi, double* sigma1,
                  double* sigma2, int nthreads) {
  if (m < 2 || n1 < 1 || !y1 || !phi || !psi || ld1 < n1) return 1;
  int homo = (y2 == NULL);
  if (homo) {
    n2 = n1;
    ld2 = ld1;
    ref2 = ref1;
  } else if (n2 < 1 || ld2 < n2) {
    return 1;
  }
  if (ref_mode == 1 && (!ref1 || (!homo && !ref2))) return 1;
  if (!rows) nrows = n1;
  for (int r = 0; r < nrows && rows; ++r)
    if (rows[r] < 0 || rows[r] >= n1) return 1;

  int nfreq = oracle_num_freq(m);
  if (!(norm > 0.0)) norm = oracle_default_norm(m);

  double *r1 = malloc(sizeof(double) * n1), *r2 = malloc(sizeof(double) * n2);
  double *d1 = malloc(sizeof(double) * (size_t)m * n1), *d2 = malloc(sizeof(double) * (size_t)m * n2);
  double *sg1 = malloc(sizeof(double) * n1), *sg2 = malloc(sizeof(double) * n2);
  double *sc1 = malloc(sizeof(double) * n1), *sc2 = malloc(sizeof(double) * n2);
  double *Yr1 = malloc(sizeof(double) * (size_t)n1 * nfreq), *Yi1 = malloc(sizeof(double) * (size_t)n1 * nfreq);
  double *Yr2 = malloc(sizeof(double) * (size_t)n2 * nfreq), *Yi2 = malloc(sizeof(double) * (size_t)n2 * nfreq);
  int rc = 0;
  if (!r1 || !r2 || !d1 || !d2 || !sg1 || !sg2 || !sc1 || !sc2 || !Yr1 || !Yi1 || !Yr2 || !Yi2) {
    rc = 2;
    goto done;
  }

  /* Step 1: reference spectra and dynamic spectra (Eqs. ref, dynspec). */
  if (ref_mode == 1) {
    for (int v = 0; v < n1; ++v) r1[v] = (double)ref1[v];
  } else {
    oracle_reference_mean(m, n1, y1, ld1, r1);
  }
  oracle_dynamic(m, n1, y1, ld1, r1, d1);
  if (homo) {
    memcpy(r2, r1, sizeof(double) * n1);
    memcpy(d2, d1, sizeof(double) * (size_t)m * n1);
  } else {
    if (ref_mode == 1) {
      for (int v = 0; v < n2; ++v) r2[v] = (double)ref2[v];
    } else {
      oracle_reference_mean(m, n2, y2, ld2, r2);
    }
    oracle_dynamic(m, n2, y2, ld2, r2, d2);
  }

  /* Scaling factors from the standard deviations (Eqs. stdev, scale*). */
  oracle_sigma(m, n1, d1, sg1);
  oracle_sigma(m, n2, d2, sg2);
  for (int v = 0; v < n1; ++v) sc1[v] = oracle_scale_factor(sg1[v], alpha);
  for (int v = 0; v < n2; ++v) sc2[v] = oracle_scale_factor(sg2[v], alpha);

  /* Step 2: DFT along the perturbation axis (Eq. disFT). */
  oracle_dft(m, n1, d1, nfreq, Yr1, Yi1);
  oracle_dft(m, n2, d2, nfreq, Yr2, Yi2);

  /* Step 3: correlation (Eq. disint2d) with normalisation and scaling. */
  oracle_cross_spectrum(n1, n2, nfreq, Yr1, Yi1, Yr2, Yi2, norm, sc1, sc2, nrows, rows, phi, psi,
                        nthreads);
  if (sigma1) memcpy(sigma1, sg1, sizeof(double) * n1);
  if (sigma2) memcpy(sigma2, sg2, sizeof(double) * n2);

done:
  free(r1); free(r2); free(d1); free(d2); free(sg1); free(sg2); free(sc1); free(sc2);
  free(Yr1); free(Yi1); free(Yr2); free(Yi2);
  return rc;
}

/*
 * Preprocessing onto a common, equally spaced spectral axis (reading R12):
 * the interpolation mechanism of Sec. 4.2 (target grid seq(min, max,
 * length.out = N), evaluated from a per-row interpolating function), here
 * with linear interpolation and applied along the spectral axis.  Each of the
 * m rows of y_raw (n_raw values at strictly increasing positions x_raw) is
 * evaluated at the n_out grid points.  ref (nullable, length n_out) is
 * subtracted into dyn_out (nullable) as in Eq. dynspec.
 * Returns 0 on success, 1 on invalid arguments.
 */
int oracle_interp_linear(int m, int n_raw, const double* x_raw, const float* y_raw, long ld_raw,
                         int n_out, double* y_out, const float* ref, double* dyn_out) {
  if (m < 1 || n_raw < 2 || n_out < 2 || !x_raw || !y_raw || !y_out || ld_raw < n_raw) return 1;
  for (int i = 1; i < n_raw; ++i)
    if (!(x_raw[i] > x_raw[i - 1])) return 1;
  double x0 = x_raw[0], x1 = x_raw[n_raw - 1];
  double step = (x1 - x0) / (double)(n_out - 1);
  int seg = 0;
  for (int k = 0; k < n_out; ++k) {
    double x = (k == n_out - 1) ? x1 : x0 + (double)k * step;
    /* segment [x_raw[seg], x_raw[seg+1]] containing x (grid is increasing) */
    while (seg < n_raw - 2 && x_raw[seg + 1] < x) ++seg;
    double xa = x_raw[seg], xb = x_raw[seg + 1];
    double t = (x - xa) / (xb - xa);
    for (int j = 0; j < m; ++j) {
      double ya = (double)y_raw[(long)j * ld_raw + seg];
      double yb = (double)y_raw[(long)j * ld_raw + seg + 1];
      double val = ya + t * (yb - ya);
      y_out[(long)j * n_out + k] = val;
      if (dyn_out) dyn_out[(long)j * n_out + k] = val - (ref ? (double)ref[k] : 0.0);
    }
  }
  return 0;
}

/*
 * Interpolation along the perturbation axis (Sec. 4.2, interpolation
 * snippet): new perturbation values T_k = seq(min(Time), max(Time),
 * length.out = N), i.e. T_k = t_0 + k (t_last - t_0)/(N - 1) with the last
 * value t_last exactly, then every spectral variable (column nu of the m x n
 * matrix) is evaluated at the T_k through an interpolating function of its
 * values over Time.  The package offers approxfun (linear) and splinefun; this
 * is the linear function (reading R13; the spline is oracle_interp_spline).  Time must be
 * strictly increasing.  Output: N x n row-major.  Returns 0, or 1 on invalid
 * arguments.
 */
int oracle_interp_perturbation(int m, int n, const double* time, const float* y, long ld, int N,
                               double* out) {
  if (m < 2 || n < 1 || N < 2 || !time || !y || !out || ld < n) return 1;
  for (int j = 1; j < m; ++j)
    if (!(time[j] > time[j - 1])) return 1;
  double t0 = time[0], t1 = time[m - 1];
  double step = (t1 - t0) / (double)(N - 1);
  int seg = 0;
  for (int k = 0; k < N; ++k) {
    double T = (k == N - 1) ? t1 : t0 + (double)k * step;
    while (seg < m - 2 && time[seg + 1] < T) ++seg;
    double ta = time[seg], tb = time[seg + 1];
    double u = (T - ta) / (tb - ta);
    for (int v = 0; v < n; ++v) {
      double ya = (double)y[(long)seg * ld + v];
      double yb = (double)y[(long)(seg + 1) * ld + v];
      out[(long)k * n + v] = ya + u * (yb - ya);
    }
  }
  return 0;
}

/*
 * Perturbation-axis interpolation through the default interpolating function
 * of the package, splinefun (Sec. 4.2; reading R13: R's "fmm" spline).  Same
 * new perturbation values as oracle_interp_perturbation.  For each spectral
 * variable the spline s is cubic on every [t_i, t_i+1], s(t_i) = y_i, and s is
 * twice continuously differentiable.  With M_i = s''(t_i), h_i = t_i+1 - t_i
 * and D_i = (y_i+1 - y_i)/h_i the continuity of s' at the inner knots gives
 *   h_i-1 M_i-1 + 2 (h_i-1 + h_i) M_i + h_i M_i+1 = 6 (D_i - D_i-1),
 * i = 1..m-2, and the end conditions fix the third derivative of s on the
 * first and last interval:
 *   (M_1 - M_0) / h_0 = 6 f[t_0, t_1, t_2, t_3],
 *   (M_m-1 - M_m-2) / h_m-2 = 6 f[t_m-4, ..., t_m-1]
 * (f[...] the divided differences: 6 f[four points] is the third derivative
 * of the cubic through them); with m = 3 both are 0, with m = 2 M = 0.  The
 * tridiagonal system is solved by Gaussian elimination in knot order, then
 *   s(T) = (M_s A^3 + M_s+1 B^3) / (6 h) + (y_s - M_s h^2/6) A / h
 *        + (y_s+1 - M_s+1 h^2/6) B / h,   A = t_s+1 - T, B = T - t_s, h = h_s
 * on the segment s of T chosen as in the linear case.  Output N x n
 * row-major; returns 0, or 1 on invalid arguments.
 */
static double oracle_third_divided_difference(const double* t, const double* y) {
  double f01 = (y[1] - y[0]) / (t[1] - t[0]);
  double f12 = (y[2] - y[1]) / (t[2] - t[1]);
  double f23 = (y[3] - y[2]) / (t[3] - t[2]);
  double f012 = (f12 - f01) / (t[2] - t[0]);
  double f123 = (f23 - f12) / (t[3] - t[1]);
  return (f123 - f012) / (t[3] - t[0]);
}

int oracle_interp_spline(int m, int n, const double* time, const float* y, long ld, int N,
                         double* out) {
  if (m < 2 || n < 1 || N < 2 || !time || !y || !out || ld < n) return 1;
  for (int j = 1; j < m; ++j)
    if (!(time[j] > time[j - 1])) return 1;
  double* yv = malloc(sizeof(double) * (size_t)m);
  double* M = malloc(sizeof(double) * (size_t)m);
  double* sub = malloc(sizeof(double) * (size_t)m);
  double* dia = malloc(sizeof(double) * (size_t)m);
  double* sup = malloc(sizeof(double) * (size_t)m);
  double* rhs = malloc(sizeof(double) * (size_t)m);
  if (!yv || !M || !sub || !dia || !sup || !rhs) {
    free(yv); free(M); free(sub); free(dia); free(sup); free(rhs);
    return 1;
  }
  const double t0 = time[0], t1 = time[m - 1];
  const double step = (t1 - t0) / (double)(N - 1);
  for (int v = 0; v < n; ++v) {
    for (int i = 0; i < m; ++i) yv[i] = (double)y[(long)i * ld + v];
    if (m == 2) {
      M[0] = M[1] = 0.0;
    } else {
      /* rows of the tridiagonal system: sub M_i-1 + dia M_i + sup M_i+1 = rhs */
      for (int i = 1; i < m - 1; ++i) {
        double hl = time[i] - time[i - 1], hr = time[i + 1] - time[i];
        sub[i] = hl;
        dia[i] = 2.0 * (hl + hr);
        sup[i] = hr;
        rhs[i] = 6.0 * ((yv[i + 1] - yv[i]) / hr - (yv[i] - yv[i - 1]) / hl);
      }
      double g0 = 0.0, g1 = 0.0;  /* third derivatives at the two ends */
      if (m >= 4) {
        g0 = 6.0 * oracle_third_divided_difference(time, yv);
        g1 = 6.0 * oracle_third_divided_difference(time + (m - 4), yv + (m - 4));
      }
      sub[0] = 0.0; dia[0] = -1.0; sup[0] = 1.0;
      rhs[0] = g0 * (time[1] - time[0]);
      sub[m - 1] = -1.0; dia[m - 1] = 1.0; sup[m - 1] = 0.0;
      rhs[m - 1] = g1 * (time[m - 1] - time[m - 2]);
      /* Gaussian elimination, rows in order, then back substitution */
      for (int i = 1; i < m; ++i) {
        double l = sub[i] / dia[i - 1];
        dia[i] -= l * sup[i - 1];
        rhs[i] -= l * rhs[i - 1];
      }
      M[m - 1] = rhs[m - 1] / dia[m - 1];
      for (int i = m - 2; i >= 0; --i) M[i] = (rhs[i] - sup[i] * M[i + 1]) / dia[i];
    }
    int seg = 0;
    for (int k = 0; k < N; ++k) {
      double T = (k == N - 1) ? t1 : t0 + (double)k * step;
      while (seg < m - 2 && time[seg + 1] < T) ++seg;
      double h = time[seg + 1] - time[seg];
      double A = time[seg + 1] - T, B = T - time[seg];
      out[(long)k * n + v] = (M[seg] * A * A * A + M[seg + 1] * B * B * B) / (6.0 * h) +
                             (yv[seg] - M[seg] * h * h / 6.0) * A / h +
                             (yv[seg + 1] - M[seg + 1] * h * h / 6.0) * B / h;
    }
  }
  free(yv); free(M); free(sub); free(dia); free(sup); free(rhs);
  return 0;
}

/*
 * Hilbert-transform approach (Sec. 2, Eqs. disHTsyn, disHT, HilbNoda,
 * disHTasyn), given dynamic spectra d1 (m x n1) and d2 (m x n2):
 *   Phi = 1/(m-1) sum_j d1(nu1, j) d2(nu2, j)
 *   z(nu2, j) = sum_k N_jk d2(nu2, k),  N_jk = 0 (j = k), 1/(pi (k - j)) else
 *   Psi = 1/(m-1) sum_j d1(nu1, j) z(nu2, j)
 * Outputs are n1 x n2.
 */
void oracle_hilbert_noda(int m, int n1, const double* d1, int n2, const double* d2, double* phi,
                         double* psi) {
  double* z = malloc(sizeof(double) * (size_t)m * n2);
  if (!z) return;
  for (int b = 0; b < n2; ++b)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k)
        if (k != j) s += d2[(long)k * n2 + b] / (ORACLE_PI * (double)(k - j));
      z[(long)j * n2 + b] = s;
    }
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) {
      double sp = 0.0, sq = 0.0;
      for (int j = 0; j < m; ++j) {
        sp += d1[(long)j * n1 + a] * d2[(long)j * n2 + b];
        sq += d1[(long)j * n1 + a] * z[(long)j * n2 + b];
      }
      phi[(long)a * n2 + b] = sp / (double)(m - 1);
      psi[(long)a * n2 + b] = sq / (double)(m - 1);
    }
  free(z);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
