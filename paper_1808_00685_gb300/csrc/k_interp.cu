// Preprocessing onto a common, equally spaced spectral (or perturbation) axis: the interpolation
// mechanism of Sec. 4.2 (target grid seq(min, max, length.out = N), each row
// evaluated through an interpolating function), here linear and applied along
// the spectral axis, followed by reference subtraction (Eq. dynspec).
//
// One thread per output grid point and slab of rows: it locates its segment
// of the raw axis (FP64: a galloping search from where an equally spaced axis
// would put the point), then blends the two neighbouring raw values of each row
// in FP64 with explicitly rounded operations, so each output is the correctly
// rounded FP32 value of the plain double formula.  The same launch checks that
// the raw axis is strictly increasing and finite (raising the context's error
// word if not).  Slabs get fewer rows on small grids so that the launch fills
// the GPU.  Bound by the FP64 pipe (about six FP64 operations per output) on
// large grids; reads m x n_raw, writes m x n_out (twice with a reference).
#include "internal.h"

namespace c2d {

__global__ void k_check_axis(int n_raw, const double* __restrict__ x, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 < n_raw) {
    const double a = x[i], b = x[i + 1];
    if (!(b > a) || !isfinite(a) || !isfinite(b)) atomicCAS(err, 0, DEV_BAD_AXIS);
  }
}

// Segment s of grid value xk: the largest index in [0, n_raw - 2] with
// x[s] < xk (0 if none).  The search starts at `e` (any start gives the same
// segment), gallops outwards to a bracket and bisects it: a few steps on
// nearly uniform axes, O(log n_raw) on any increasing one.
__device__ __forceinline__ int find_segment(const double* __restrict__ x, int n_raw, double xk,
                                            int e) {
  const int top = n_raw - 2;
  e = e < 0 ? 0 : (e > top ? top : e);
  int lo, hi;  // the answer lies in [lo, hi]
  if (x[e] < xk) {
    lo = e;
    hi = top;
    for (int step = 1; lo + step <= top; step <<= 1) {
      if (x[lo + step] < xk) {
        lo += step;
      } else {
        hi = lo + step - 1;
        break;
      }
    }
  } else {
    hi = e > 0 ? e - 1 : 0;
    lo = 0;
    for (int step = 1; e - step > 0; step <<= 1) {
      if (x[e - step] < xk) {
        lo = e - step;
        break;
      }
      hi = e - step - 1;
    }
  }
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (x[mid] < xk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_interp(int m, int n_raw, const double* __restrict__ x,
                                                const float* __restrict__ y, int n_out,
                                                int rows_per_block, float* __restrict__ out,
                                                const float* __restrict__ ref,
                                                float* __restrict__ dyn, int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.y == 0)  // the axis check, pair (i, i + 1), spread over the first slab
    for (int i = k; i + 1 < n_raw; i += gridDim.x * blockDim.x) {
      const double a = x[i], b = x[i + 1];
      if (!(b > a) || !isfinite(a) || !isfinite(b)) atomicCAS(err, 0, DEV_BAD_AXIS);
    }
  if (k >= n_out) return;
  const double x0 = x[0], x1 = x[n_raw - 1];
  const double step = __ddiv_rn(__dsub_rn(x1, x0), (double)(n_out - 1));
  // explicit roundings (no FMA contraction) keep the grid and the blend
  // identical to a plain double evaluation of the same formulas
  const double xk = (k == n_out - 1) ? x1 : __dadd_rn(x0, __dmul_rn((double)k, step));
  const int e = (int)((float)k * ((float)(n_raw - 2) / (float)(n_out - 1)));  // FP32 start
  const int s = find_segment(x, n_raw, xk, e);
  const double xa = x[s], xb = x[s + 1];
  const double t = __ddiv_rn(__dsub_rn(xk, xa), __dsub_rn(xb, xa));
  const double r = ref ? (double)ref[k] : 0.0;
  const int j0 = blockIdx.y * rows_per_block;
  const int j1 = min(m, j0 + rows_per_block);
  for (int j = j0; j < j1; ++j) {
    const double ya = (double)y[(size_t)j * n_raw + s];
    const double yb = (double)y[(size_t)j * n_raw + s + 1];
    const double val = __dadd_rn(ya, __dmul_rn(t, __dsub_rn(yb, ya)));
    out[(size_t)j * n_out + k] = (float)val;
    if (dyn) dyn[(size_t)j * n_out + k] = (float)__dsub_rn(val, r);
  }
}

// Interpolation along the perturbation axis (Sec. 4.2: new perturbation values
// seq(min(Time), max(Time), length.out = N), every spectral variable evaluated
// there through a linear interpolating function of its values over Time).
// One thread per (new step k, variable nu); the segment of Time containing
// T_k is the same for all variables of a row, so reads and writes are
// coalesced along nu.  Same explicitly rounded FP64 blend as k_interp.
__global__ void __launch_bounds__(256) k_interp_t(int m, int n, const double* __restrict__ t,
                                                  const float* __restrict__ y, long ld, int N,
                                                  float* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (v >= n) return;
  const double t0 = t[0], t1 = t[m - 1];
  const double step = __ddiv_rn(__dsub_rn(t1, t0), (double)(N - 1));
  const double T = (k == N - 1) ? t1 : __dadd_rn(t0, __dmul_rn((double)k, step));
  int lo = 0, hi = m - 2;  // largest s in [0, m-2] with t[s] < T (0 if none)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t[mid] < T) lo = mid; else hi = mid - 1;
  }
  const double ta = t[lo], tb = t[lo + 1];
  const double u = __ddiv_rn(__dsub_rn(T, ta), __dsub_rn(tb, ta));
  const double ya = (double)y[(size_t)lo * ld + v];
  const double yb = (double)y[(size_t)(lo + 1) * ld + v];
  out[(size_t)k * n + v] = (float)__dadd_rn(ya, __dmul_rn(u, __dsub_rn(yb, ya)));
}

// ---------------------------------------------------------------------------
// Spline interpolation along the perturbation axis: splinefun, the package's
// default interpolating function (Sec. 4.2), with R's default "fmm" end
// conditions.  For each spectral variable the C^2 cubic spline through
// (t_i, y_i) has second derivatives M_i solving the tridiagonal system
//   row 0:       -M_0 + M_1 = h_0 g0
//   rows 1..m-2:  h_i-1 M_i-1 + 2 (h_i-1 + h_i) M_i + h_i M_i+1
//                   = 6 ((y_i+1 - y_i)/h_i - (y_i - y_i-1)/h_i-1)
//   row m-1:     -M_m-2 + M_m-1 = h_m-2 g1
// with g0, g1 the third derivatives of the cubics through the first and the
// last four points (6 x their third divided differences; 0 when m = 3); m = 2
// is the line.  The matrix depends on the knots only, so one thread factors
// it once (pivots, multipliers, reciprocals); one thread per variable then
// builds its right-hand side, runs the substitutions and stores M in an FP64
// workspace [i][nu] (coalesced across variables).  On the segment s of the new
// value T (A = t_s+1 - T, B = T - t_s, h = t_s+1 - t_s) the spline is
//   y_s A/h + y_s+1 B/h - M_s A B (A + h)/(6h) - M_s+1 A B (B + h)/(6h),
// the usual form with A^3 - h^2 A written as -A B (A + h) (no cancellation);
// its four weights per new value are tabulated once.  All FP64.
// ---------------------------------------------------------------------------
struct SplineTab {
  double* mul;    // m: elimination multipliers l_i (row i minus l_i x row i-1)
  double* rpiv;   // m: reciprocal pivots 1 / u_i
  double* sup;    // m: super-diagonal of row i
  double* rh;     // m: 1 / h_i (i < m - 1)
  double* w;      // 4 N: weights of y_s, y_s+1, M_s, M_s+1 for new value k
  int* seg;       // N: segment s of new value k
};

__global__ void k_spline_setup(int m, const double* __restrict__ t, SplineTab tab) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i + 1 < m; ++i) tab.rh[i] = 1.0 / (t[i + 1] - t[i]);
  if (m < 3) return;  // the line: no system
  double u = -1.0;    // row 0: -M_0 + M_1
  tab.mul[0] = 0.0;
  tab.rpiv[0] = 1.0 / u;
  tab.sup[0] = 1.0;
  for (int i = 1; i < m; ++i) {
    double sub, dia, sup;
    if (i < m - 1) {
      const double hl = t[i] - t[i - 1], hr = t[i + 1] - t[i];
      sub = hl; dia = 2.0 * (hl + hr); sup = hr;
    } else {
      sub = -1.0; dia = 1.0; sup = 0.0;
    }
    const double l = sub / u;
    u = dia - l * tab.sup[i - 1];
    tab.mul[i] = l;
    tab.rpiv[i] = 1.0 / u;
    tab.sup[i] = sup;
  }
}

// Segment and weights of every new perturbation value (same grid and segment
// rule as the linear interpolation).
__global__ void k_spline_grid(int m, const double* __restrict__ t, int N, SplineTab tab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double t0 = t[0], t1 = t[m - 1];
  const double step = (t1 - t0) / (double)(N - 1);
  const double T = (k == N - 1) ? t1 : t0 + (double)k * step;
  int lo = 0, hi = m - 2;  // largest s in [0, m-2] with t[s] < T (0 if none)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t[mid] < T) lo = mid; else hi = mid - 1;
  }
  const double h = t[lo + 1] - t[lo], A = t[lo + 1] - T, B = T - t[lo];
  const double rh = 1.0 / h, r6h = rh / 6.0;
  tab.seg[k] = lo;
  tab.w[4 * k + 0] = A * rh;
  tab.w[4 * k + 1] = B * rh;
  tab.w[4 * k + 2] = (m < 3) ? 0.0 : -A * B * (A + h) * r6h;
  tab.w[4 * k + 3] = (m < 3) ? 0.0 : -A * B * (B + h) * r6h;
}

__device__ __forceinline__ double third_divided_difference(const double* t, double y0, double y1,
                                                           double y2, double y3) {
  const double f01 = (y1 - y0) / (t[1] - t[0]);
  const double f12 = (y2 - y1) / (t[2] - t[1]);
  const double f23 = (y3 - y2) / (t[3] - t[2]);
  const double f012 = (f12 - f01) / (t[2] - t[0]);
  const double f123 = (f23 - f12) / (t[3] - t[1]);
  return (f123 - f012) / (t[3] - t[0]);
}

__global__ void __launch_bounds__(256) k_spline_solve(int m, int n, const double* __restrict__ t,
                                                      const float* __restrict__ y, long ld,
                                                      SplineTab tab, double* __restrict__ M) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const float* yv = y + v;
  double g0 = 0.0, g1 = 0.0;
  if (m >= 4) {
    g0 = 6.0 * third_divided_difference(t, yv[0], yv[ld], yv[2 * ld], yv[3 * ld]);
    g1 = 6.0 * third_divided_difference(t + (m - 4), yv[(m - 4) * ld], yv[(m - 3) * ld],
                                        yv[(m - 2) * ld], yv[(m - 1) * ld]);
  }
  // forward elimination; the reduced right-hand sides go to M
  double rp = g0 * (t[1] - t[0]);
  M[v] = rp;
  double ya = yv[0], yb = yv[ld];
  double da = (yb - ya) * tab.rh[0];  // slope of segment i - 1
  for (int i = 1; i < m; ++i) {
    double r;
    if (i < m - 1) {
      const double yc = yv[(long)(i + 1) * ld];
      const double db = (yc - yb) * tab.rh[i];
      r = 6.0 * (db - da);
      da = db;
      yb = yc;
    } else {
      r = g1 * (t[m - 1] - t[m - 2]);
    }
    rp = r - tab.mul[i] * rp;
    M[(size_t)i * n + v] = rp;
  }
  // back substitution
  double mi = rp * tab.rpiv[m - 1];
  M[(size_t)(m - 1) * n + v] = mi;
  for (int i = m - 2; i >= 0; --i) {
    mi = (M[(size_t)i * n + v] - tab.sup[i] * mi) * tab.rpiv[i];
    M[(size_t)i * n + v] = mi;
  }
}

__global__ void __launch_bounds__(256) k_spline_eval(int m, int n, const float* __restrict__ y,
                                                     long ld, const double* __restrict__ M,
                                                     SplineTab tab, int N,
                                                     float* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (v >= n) return;
  const int s = tab.seg[k];
  const double wa = tab.w[4 * k], wb = tab.w[4 * k + 1];
  double val = (double)y[(size_t)s * ld + v] * wa + (double)y[(size_t)(s + 1) * ld + v] * wb;
  if (m >= 3)
    val += M[(size_t)s * n + v] * tab.w[4 * k + 2] + M[(size_t)(s + 1) * n + v] * tab.w[4 * k + 3];
  out[(size_t)k * n + v] = (float)val;
}

size_t spline_workspace_bytes(int m, int n, int N) {
  const size_t tab = (size_t)4 * m * sizeof(double) + (size_t)4 * N * sizeof(double) +
                     (size_t)N * sizeof(int);
  return ((tab + 255) / 256) * 256 + (m >= 3 ? (size_t)m * n * sizeof(double) : 0);
}

cudaError_t launch_spline_t(int m, int n, const double* t, const float* y, long ld, int N,
                            float* out, void* ws, int* err, cudaStream_t s) {
  uint8_t* p = (uint8_t*)ws;
  SplineTab tab;
  tab.mul = (double*)p;
  tab.rpiv = tab.mul + m;
  tab.sup = tab.rpiv + m;
  tab.rh = tab.sup + m;
  tab.w = tab.rh + m;
  tab.seg = (int*)(tab.w + 4 * N);
  const size_t tab_bytes = (size_t)4 * m * sizeof(double) + (size_t)4 * N * sizeof(double) +
                           (size_t)N * sizeof(int);
  double* M = (double*)(p + ((tab_bytes + 255) / 256) * 256);
  k_check_axis<<<(m + 255) / 256, 256, 0, s>>>(m, t, err);
  k_spline_setup<<<1, 32, 0, s>>>(m, t, tab);
  k_spline_grid<<<(N + 127) / 128, 128, 0, s>>>(m, t, N, tab);
  if (m >= 3) k_spline_solve<<<(n + 255) / 256, 256, 0, s>>>(m, n, t, y, ld, tab, M);
  k_spline_eval<<<dim3((n + 255) / 256, N), 256, 0, s>>>(m, n, y, ld, M, tab, N, out);
  return cudaGetLastError();
}

cudaError_t launch_interp_t(int m, int n, const double* t, const float* y, long ld, int N,
                            float* out, int* err, cudaStream_t s) {
  k_check_axis<<<(m + 255) / 256, 256, 0, s>>>(m, t, err);
  k_interp_t<<<dim3((n + 255) / 256, N), 256, 0, s>>>(m, n, t, y, ld, N, out);
  return cudaGetLastError();
}

cudaError_t launch_interp(int m, int n_raw, const double* x, const float* y, int n_out,
                          float* out, const float* ref, float* dyn, int* err, cudaStream_t s) {
  // rows per slab: 16, or fewer (down to 4) until the launch has at least two
  // blocks per SM of a 152-SM GPU (each slab repeats its grid points' search)
  const int kblocks = (n_out + 127) / 128;
  int rows = 16;
  while (rows > 4 && (long)kblocks * ((m + rows - 1) / rows) < 304) rows >>= 1;
  dim3 grid(kblocks, (m + rows - 1) / rows);
  k_interp<<<grid, 128, 0, s>>>(m, n_raw, x, y, n_out, rows, out, ref, dyn, err);
  return cudaGetLastError();
}

}  // namespace c2d
