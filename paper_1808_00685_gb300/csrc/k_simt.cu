// Plain FP32 CUDA-core cross-spectrum (Eq. disint2d, half spectrum of
// Sec. 4.2): the baseline the tensor-core path is measured against.
//
// 128 x 128 output tile per CTA, 256 threads, each thread an 8 x 8 block of
// (Phi, Psi) pairs accumulated with FP32 FMAs over the retained frequencies.
// Operands are frequency-major planes (Re, Im of stack 1; weighted Re, Im of
// stack 2), staged through shared memory 8 frequencies at a time.  For homo
// problems only tiles with ti <= tj run and each thread also writes its
// transposed block (Phi symmetric, Psi antisymmetric).
#include "internal.h"

namespace c2d {

constexpr int ST = 128;  // tile edge
constexpr int SK = 8;    // frequencies per stage

__global__ void __launch_bounds__(256) k_xspec_simt(int kp1, int n1, int n2,
                                                    const float* __restrict__ yr1,
                                                    const float* __restrict__ yi1,
                                                    const float* __restrict__ yr2,
                                                    const float* __restrict__ yi2,
                                                    const float* __restrict__ s1,
                                                    const float* __restrict__ s2, float norm,
                                                    float* __restrict__ phi,
                                                    float* __restrict__ psi, long ldo,
                                                    int mirror, int ntile) {
  __shared__ __align__(16) float sar[SK][ST], sai[SK][ST], sbr[SK][ST], sbi[SK][ST];
  int ti, tj;
  if (mirror) {
    // linear index over the upper triangle, row by row
    int t = blockIdx.x;
    ti = 0;
    int rowlen = ntile;
    while (t >= rowlen) { t -= rowlen; ++ti; --rowlen; }
    tj = ti + t;
  } else {
    ti = blockIdx.y;
    tj = blockIdx.x;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = ti * ST + ty * 8, c0 = tj * ST + tx * 8;
  float ap[8][8], aq[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) ap[i][j] = aq[i][j] = 0.f;

  for (int k0 = 0; k0 < kp1; k0 += SK) {
    // stage 8 frequencies x 128 variables of each plane (coalesced along nu)
    for (int e = threadIdx.x; e < SK * ST; e += 256) {
      const int kk = e / ST, v = e % ST, k = k0 + kk;
      const int a = ti * ST + v, b = tj * ST + v;
      const bool ka = k < kp1;
      sar[kk][v] = (ka && a < n1) ? yr1[(size_t)k * n1 + a] : 0.f;
      sai[kk][v] = (ka && a < n1) ? yi1[(size_t)k * n1 + a] : 0.f;
      sbr[kk][v] = (ka && b < n2) ? yr2[(size_t)k * n2 + b] : 0.f;
      sbi[kk][v] = (ka && b < n2) ? yi2[(size_t)k * n2 + b] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SK; ++kk) {
      float xr[8], xi[8], zr[8], zi[8];
      *(float4*)&xr[0] = *(const float4*)&sar[kk][ty * 8];
      *(float4*)&xr[4] = *(const float4*)&sar[kk][ty * 8 + 4];
      *(float4*)&xi[0] = *(const float4*)&sai[kk][ty * 8];
      *(float4*)&xi[4] = *(const float4*)&sai[kk][ty * 8 + 4];
      *(float4*)&zr[0] = *(const float4*)&sbr[kk][tx * 8];
      *(float4*)&zr[4] = *(const float4*)&sbr[kk][tx * 8 + 4];
      *(float4*)&zi[0] = *(const float4*)&sbi[kk][tx * 8];
      *(float4*)&zi[4] = *(const float4*)&sbi[kk][tx * 8 + 4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          ap[i][j] = fmaf(xr[i], zr[j], fmaf(xi[i], zi[j], ap[i][j]));
          aq[i][j] = fmaf(xi[i], zr[j], fmaf(-xr[i], zi[j], aq[i][j]));
        }
    }
    __syncthreads();
  }
  // epilogue: scale and store (and the mirrored block for homo tiles)
  float rsc[8], csc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    rsc[i] = (r0 + i < n1) ? norm * s1[r0 + i] : 0.f;
    csc[i] = (c0 + i < n2) ? s2[c0 + i] : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      ap[i][j] = ap[i][j] * rsc[i] * csc[j];
      aq[i][j] = aq[i][j] * rsc[i] * csc[j];
    }
  // On a diagonal homo tile, 8x8 block (ty, tx) with tx > ty writes itself and
  // its mirror, tx == ty writes its upper triangle and mirrors it, tx < ty is
  // left to block (tx, ty): the output is exactly (anti)symmetric.
  const bool diag = mirror && ti == tj;
  if (diag && tx < ty) return;
  const bool tri = diag && tx == ty;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + i;
    if (r >= n1) break;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (c0 + j < n2 && (!tri || j >= i)) {
        phi[(size_t)r * ldo + c0 + j] = ap[i][j];
        psi[(size_t)r * ldo + c0 + j] = (tri && j == i) ? 0.f : aq[i][j];
      }
    }
  }
  if (tri) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = c0 + j;
      if (r >= n2) break;
#pragma unroll
      for (int i = 0; i < j; ++i) {
        if (r0 + i < n1) {
          phi[(size_t)r * ldo + r0 + i] = ap[i][j];
          psi[(size_t)r * ldo + r0 + i] = -aq[i][j];
        }
      }
    }
  }
  if (mirror && !tri) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = c0 + j;  // mirrored row
      if (r >= n2) break;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (r0 + i < n1) {
          phi[(size_t)r * ldo + r0 + i] = ap[i][j];
          psi[(size_t)r * ldo + r0 + i] = -aq[i][j];
        }
      }
    }
  }
}

cudaError_t launch_xspec_simt(int kp1, int n1, int n2, const float* yr1, const float* yi1,
                              const float* yr2w, const float* yi2w, const float* s1,
                              const float* s2, float norm, float* phi, float* psi, long ldo,
                              bool mirror, cudaStream_t s) {
  const int nt1 = (n1 + ST - 1) / ST, nt2 = (n2 + ST - 1) / ST;
  if (mirror) {
    const int nt = nt1;
    const long ntri = (long)nt * (nt + 1) / 2;
    k_xspec_simt<<<dim3((unsigned)ntri, 1), 256, 0, s>>>(kp1, n1, n2, yr1, yi1, yr2w, yi2w, s1,
                                                         s2, norm, phi, psi, ldo, 1, nt);
  } else {
    k_xspec_simt<<<dim3(nt2, nt1), 256, 0, s>>>(kp1, n1, n2, yr1, yi1, yr2w, yi2w, s1, s2, norm,
                                               phi, psi, ldo, 0, nt2);
  }
  return cudaGetLastError();
}

}  // namespace c2d
