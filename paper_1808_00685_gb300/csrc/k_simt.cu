// Plain FP32 CUDA-core cross-spectrum (Eq. disint2d, half spectrum of
// Sec. 4.2): the baseline the tensor-core path is measured against.
//
// 128 x 128 output tile per CTA, 256 threads (16 x 16), each thread 8 x 8
// (Phi, Psi) pairs accumulated with FP32 FMAs over the retained frequencies.
// Thread (ty, tx) owns tile rows {4 ty .. 4 ty + 3, 64 + 4 ty .. 64 + 4 ty + 3}
// and columns {4 tx .., 64 + 4 tx ..}: consecutive threads read consecutive
// 16-byte words of the staged operands (no bank conflicts) and store
// consecutive 16-byte words of an output row.  Operands are frequency-major
// planes (Re, Im of stack 1; weighted Re, Im of stack 2; rows padded to a
// multiple of 4 floats) staged 8 frequencies at a time into a two-slot
// shared-memory ring by cp.async, the next stage in flight while the current
// one is multiplied.  Homo problems run only tiles with ti <= tj and each
// thread also writes the transposed pairs (Phi symmetric, Psi antisymmetric).
#include "internal.h"

namespace c2d {

constexpr int ST = 128;  // tile edge
constexpr int SK = 8;    // frequencies per stage

// 16-byte global -> shared copy; bytes < 16 zero-fills the rest (0: all zeros).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Local tile coordinate of owned row/column index i (0..7) of thread t (0..15).
__device__ __forceinline__ int own(int t, int i) { return (i < 4) ? 4 * t + i : 60 + 4 * t + i; }

__global__ void __launch_bounds__(256) k_xspec_simt(int kp1, int n1, int n2, int ldp1, int ldp2,
                                                    const float* __restrict__ yr1,
                                                    const float* __restrict__ yi1,
                                                    const float* __restrict__ yr2,
                                                    const float* __restrict__ yi2,
                                                    const float* __restrict__ s1,
                                                    const float* __restrict__ s2, float norm,
                                                    float* __restrict__ phi,
                                                    float* __restrict__ psi, long ldo,
                                                    int mirror, int ntile) {
  // [slot][plane: Re1, Im1, Re2, Im2][frequency][variable]
  __shared__ __align__(16) float sb[2][4][SK][ST];
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
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  // one stage: 4 planes x 8 frequencies x 32 words of 4 variables = 1024
  // words, four per thread; words past kp1 or past n are zero-filled
  auto load_stage = [&](int slot, int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int plane = e >> 8, kk = (e >> 5) & 7, word = e & 31;
      const int k = k0 + kk;
      const bool s1p = plane < 2;
      const int var = (s1p ? ti : tj) * ST + word * 4;
      const int n = s1p ? n1 : n2;
      const float* base = plane == 0 ? yr1 : plane == 1 ? yi1 : plane == 2 ? yr2 : yi2;
      int bytes = 0;
      const float* src = base;  // any valid address for a zero-fill
      if (k < kp1 && var < n) {
        bytes = (n - var >= 4) ? 16 : (n - var) * 4;
        src = base + (size_t)k * (size_t)(s1p ? ldp1 : ldp2) + var;
      }
      cp_async16(&sb[slot][plane][kk][word * 4], src, bytes);
    }
    cp_async_commit();
  };

  float ap[8][8], aq[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) ap[i][j] = aq[i][j] = 0.f;

  const int nstage = (kp1 + SK - 1) / SK;
  load_stage(0, 0);
  for (int st = 0; st < nstage; ++st) {
    const int slot = st & 1;
    if (st + 1 < nstage) {
      load_stage(slot ^ 1, (st + 1) * SK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SK; ++kk) {
      float xr[8], xi[8], zr[8], zi[8];
      *(float4*)&xr[0] = *(const float4*)&sb[slot][0][kk][4 * ty];
      *(float4*)&xr[4] = *(const float4*)&sb[slot][0][kk][64 + 4 * ty];
      *(float4*)&xi[0] = *(const float4*)&sb[slot][1][kk][4 * ty];
      *(float4*)&xi[4] = *(const float4*)&sb[slot][1][kk][64 + 4 * ty];
      *(float4*)&zr[0] = *(const float4*)&sb[slot][2][kk][4 * tx];
      *(float4*)&zr[4] = *(const float4*)&sb[slot][2][kk][64 + 4 * tx];
      *(float4*)&zi[0] = *(const float4*)&sb[slot][3][kk][4 * tx];
      *(float4*)&zi[4] = *(const float4*)&sb[slot][3][kk][64 + 4 * tx];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          ap[i][j] = fmaf(xr[i], zr[j], fmaf(xi[i], zi[j], ap[i][j]));
          aq[i][j] = fmaf(xi[i], zr[j], fmaf(-xr[i], zi[j], aq[i][j]));
        }
    }
    __syncthreads();  // the slot is refilled two stages later
  }

  // epilogue: scale, store the owned pairs (and the transposed ones for homo)
  const int rt = ti * ST, ct = tj * ST;
  float rsc[8], csc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = rt + own(ty, i), c = ct + own(tx, i);
    rsc[i] = (r < n1) ? norm * s1[r] : 0.f;
    csc[i] = (c < n2) ? s2[c] : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      ap[i][j] = ap[i][j] * rsc[i] * csc[j];
      aq[i][j] = aq[i][j] * rsc[i] * csc[j];
    }
  const bool diag = mirror && ti == tj;
  if (diag) {
    // Each unordered pair {R, C} of the diagonal tile is written, both ways,
    // by the thread owning (min, max): the output is exactly (anti)symmetric.
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int R = own(ty, i);
      if (rt + R >= n1) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int C = own(tx, j);
        if (ct + C >= n2 || R > C) continue;
        phi[(size_t)(rt + R) * ldo + ct + C] = ap[i][j];
        psi[(size_t)(rt + R) * ldo + ct + C] = (R == C) ? 0.f : aq[i][j];
        if (R < C) {
          phi[(size_t)(ct + C) * ldo + rt + R] = ap[i][j];
          psi[(size_t)(ct + C) * ldo + rt + R] = -aq[i][j];
        }
      }
    }
    return;
  }
  // 16-byte stores where four owned columns are inside n2 and the row is
  // 16-byte aligned; element by element otherwise
  const bool vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(phi) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(psi) & 15) == 0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = rt + own(ty, i);
    if (r >= n1) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = ct + own(tx, 4 * h);
      float* pp = phi + (size_t)r * ldo + c;
      float* pq = psi + (size_t)r * ldo + c;
      if (vec_ok && c + 3 < n2) {
        *(float4*)pp = make_float4(ap[i][4 * h], ap[i][4 * h + 1], ap[i][4 * h + 2], ap[i][4 * h + 3]);
        *(float4*)pq = make_float4(aq[i][4 * h], aq[i][4 * h + 1], aq[i][4 * h + 2], aq[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (c + e < n2) {
            pp[e] = ap[i][4 * h + e];
            pq[e] = aq[i][4 * h + e];
          }
      }
    }
  }
  if (mirror) {
    // transposed pairs: output row = owned column, four owned rows per word
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = ct + own(tx, j);
      if (r >= n2) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = rt + own(ty, 4 * h);
        float* pp = phi + (size_t)r * ldo + c;
        float* pq = psi + (size_t)r * ldo + c;
        if (vec_ok && c + 3 < n1) {
          *(float4*)pp = make_float4(ap[4 * h][j], ap[4 * h + 1][j], ap[4 * h + 2][j], ap[4 * h + 3][j]);
          *(float4*)pq = make_float4(-aq[4 * h][j], -aq[4 * h + 1][j], -aq[4 * h + 2][j],
                                     -aq[4 * h + 3][j]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (c + e < n1) {
              pp[e] = ap[4 * h + e][j];
              pq[e] = -aq[4 * h + e][j];
            }
        }
      }
    }
  }
}

cudaError_t launch_xspec_simt(int kp1, int n1, int n2, int ldp1, int ldp2, const float* yr1,
                              const float* yi1, const float* yr2w, const float* yi2w,
                              const float* s1, const float* s2, float norm, float* phi,
                              float* psi, long ldo, bool mirror, cudaStream_t s) {
  if ((ldp1 & 3) || (ldp2 & 3)) return cudaErrorInvalidValue;  // 16-byte aligned plane rows
  const int nt1 = (n1 + ST - 1) / ST, nt2 = (n2 + ST - 1) / ST;
  if (mirror) {
    const int nt = nt1;
    const long ntri = (long)nt * (nt + 1) / 2;
    k_xspec_simt<<<dim3((unsigned)ntri, 1), 256, 0, s>>>(kp1, n1, n2, ldp1, ldp2, yr1, yi1, yr2w,
                                                         yi2w, s1, s2, norm, phi, psi, ldo, 1, nt);
  } else {
    k_xspec_simt<<<dim3(nt2, nt1), 256, 0, s>>>(kp1, n1, n2, ldp1, ldp2, yr1, yi1, yr2w, yi2w, s1,
                                               s2, norm, phi, psi, ldo, 0, nt2);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 FMA throughput probe: the measured ceiling of the CUDA-core path.
// Every thread runs FMA_CHAINS independent chains x <- x * a + b (latency
// hidden by the chains and by 32 warps per SM), so the kernel is bound by the
// FP32 pipe alone; 2 flop per FMA.  The result is stored only under a
// condition the host makes false, so no chain can be removed.
// ---------------------------------------------------------------------------
constexpr int FMA_CHAINS = 8;

__global__ void __launch_bounds__(256) k_fma_probe(float* out, int iters, float a, float b,
                                                   float never) {
  float x[FMA_CHAINS];
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
  }
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) acc += x[k];
  if (acc == never) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_fma_probe(float* out, int blocks, int iters, cudaStream_t s) {
  k_fma_probe<<<blocks, 256, 0, s>>>(out, iters, 0.999f, 1e-4f, -1.0f);
  return cudaGetLastError();
}

double fma_probe_flops(int blocks, int iters) {
  return 2.0 * FMA_CHAINS * (double)iters * (double)blocks * 256.0;
}

}  // namespace c2d
