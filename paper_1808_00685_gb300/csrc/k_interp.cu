// Preprocessing onto a common, equally spaced spectral axis: the interpolation
// mechanism of Sec. 4.2 (target grid seq(min, max, length.out = N), each row
// evaluated through an interpolating function), here linear and applied along
// the spectral axis, followed by reference subtraction (Eq. dynspec).
//
// One thread per output grid point and 16-row slab of the stack: it locates
// its segment of the raw axis by binary search (FP64), then blends the two
// neighbouring raw values of each row in FP64 with explicitly rounded
// operations, so each output is the correctly rounded FP32 value of the plain
// double formula.  A separate pass checks that
// the raw axis is strictly increasing and raises the context's error word if
// it is not.  HBM-bound: reads m x n_raw, writes m x n_out (twice with a
// reference).
#include "internal.h"

namespace c2d {

constexpr int INTERP_ROWS = 16;

__global__ void k_check_axis(int n_raw, const double* __restrict__ x, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 < n_raw) {
    const double a = x[i], b = x[i + 1];
    if (!(b > a) || !isfinite(a) || !isfinite(b)) atomicCAS(err, 0, DEV_BAD_AXIS);
  }
}

__global__ void __launch_bounds__(128) k_interp(int m, int n_raw, const double* __restrict__ x,
                                                const float* __restrict__ y, int n_out,
                                                float* __restrict__ out,
                                                const float* __restrict__ ref,
                                                float* __restrict__ dyn) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_out) return;
  const double x0 = x[0], x1 = x[n_raw - 1];
  const double step = __ddiv_rn(__dsub_rn(x1, x0), (double)(n_out - 1));
  // explicit roundings (no FMA contraction) keep the grid and the blend
  // identical to a plain double evaluation of the same formulas
  const double xk = (k == n_out - 1) ? x1 : __dadd_rn(x0, __dmul_rn((double)k, step));
  // segment s: largest index in [0, n_raw - 2] with x[s] < xk (0 if none)
  int lo = 0, hi = n_raw - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (x[mid] < xk) lo = mid; else hi = mid - 1;
  }
  const int s = lo;
  const double xa = x[s], xb = x[s + 1];
  const double t = __ddiv_rn(__dsub_rn(xk, xa), __dsub_rn(xb, xa));
  const double r = ref ? (double)ref[k] : 0.0;
  const int j0 = blockIdx.y * INTERP_ROWS;
  const int j1 = min(m, j0 + INTERP_ROWS);
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

cudaError_t launch_interp_t(int m, int n, const double* t, const float* y, long ld, int N,
                            float* out, int* err, cudaStream_t s) {
  k_check_axis<<<(m + 255) / 256, 256, 0, s>>>(m, t, err);
  k_interp_t<<<dim3((n + 255) / 256, N), 256, 0, s>>>(m, n, t, y, ld, N, out);
  return cudaGetLastError();
}

cudaError_t launch_interp(int m, int n_raw, const double* x, const float* y, int n_out,
                          float* out, const float* ref, float* dyn, int* err, cudaStream_t s) {
  k_check_axis<<<(n_raw + 255) / 256, 256, 0, s>>>(n_raw, x, err);
  dim3 grid((n_out + 127) / 128, (m + INTERP_ROWS - 1) / INTERP_ROWS);
  k_interp<<<grid, 128, 0, s>>>(m, n_raw, x, y, n_out, out, ref, dyn);
  return cudaGetLastError();
}

}  // namespace c2d
