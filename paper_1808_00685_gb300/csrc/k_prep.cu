// Reference spectrum, dynamic spectra, standard deviation and the truncated
// DFT along the perturbation axis (Eqs. ref, dynspec, stdev, disFT; the half
// spectrum of Sec. 4.2), producing the operand rows of the cross-spectrum.
//
// Tensor-core kernel (k_prep_tc): one CTA of 256 threads per 128 spectral
// variables (two CTAs per SM); two threads share a variable's perturbation
// steps.
//   1. Reference (perturbation mean or the caller's spectrum) as a
//      double-float pair rh + rl: the sum of y is accumulated with TwoSum
//      into a (hi, lo) FP32 pair (each addition adds an error of order
//      2^-47 of the running sum), then divided by m with an exact remainder.
//      FP32 extremes of y give the range of y - ref.
//   2. Centering y - rh - rl with TwoSum (the result is y - ref rounded once
//      to FP32, up to a rounding of the 2^-48-sized tail), scaled by a power
//      of two and split into 16-bit planes (FP16 hi/lo, or one BF16 plane),
//      written to shared memory as the A operand (variables x steps, K-major,
//      128-byte swizzle), 64 steps at a time; compensated FP32 sum of squares.
//   3. tcgen05.mma contracts them with the twiddle matrix W (rows: cos and
//      -sin of 2 pi ((omega j) mod m) / m, FP64-built, split likewise) into
//      TMEM: D(nu, c) = sum_j y~(nu, j) W(c, j); with planes hi*hi + hi*lo +
//      lo*hi.  The twiddle chunks arrive by bulk copy.
//   4. Epilogue (8 warps, two per TMEM lane quadrant): row maximum,
//      power-of-two rescale, the square root of the half-spectrum weight
//      (w = 1 / 2), split into planes, operand rows, scale sigma^-alpha 2^-E,
//      sigma.
// No FP64 arithmetic runs per element: GB300's FP64 pipe retires about one
// operation per clock per SM, so the FP64 conversions and subtraction of a
// plain FP64 centering bound the kernel; double-float FP32 arithmetic gives
// the same FP32 results at the FP32 rate.
#include <cmath>
#include "internal.h"
#include "ptx.cuh"

namespace c2d {

constexpr int PREP_THREADS = 256;
constexpr int PREP_GROUPS = PREP_THREADS / PREP_ROWS;  // threads per variable (2)
constexpr int PREP_JG = 8 / PREP_GROUPS;               // 8-step groups per thread per chunk
// reduction scratch: double-float sums (2 x 2 x 128 floats), FP32 min / max /
// sum of squares (3 x 2 x 128; the min slots are reused for the epilogue row
// maxima), per-row exponent (128 ints) and double-float reference (128 pairs)
constexpr int PREP_SCRATCH = PREP_GROUPS * PREP_ROWS * (8 + 4 + 4 + 4) + PREP_ROWS * (4 + 8);
constexpr uint32_t PREP_STAGING = (PREP_THREADS / 32) * 4096;  // epilogue staging boxes

// Error-free sum of two floats: a + b = s + e exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += x + r, with x exact and r a small correction: TwoSum of hi and
// x, the low parts added to its error, renormalised by TwoSum.
__device__ __forceinline__ void df_acc(float& hi, float& lo, float x, float r) {
  float s, e;
  two_sum(hi, x, s, e);
  e += lo + r;
  two_sum(s, e, hi, lo);
}

// 16 consecutive TMEM columns of this warp's lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}
__device__ __forceinline__ uint32_t pack_b2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// FP32 -> FP16 hi/lo of 8 values: hi = fp16(v), lo = fp16(v - hi), two
// values per conversion instruction (each rounded to nearest on its own).
__device__ __forceinline__ void split8_f32(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __half2 hh = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
    h[e] = *reinterpret_cast<const uint32_t*>(&hh);
    l[e] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ uint4 bf16x8_f32(const float* v) {
  uint32_t h[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    h[e] = *reinterpret_cast<const uint32_t*>(&b);
  }
  return make_uint4(h[0], h[1], h[2], h[3]);
}

__host__ __device__ __forceinline__ uint32_t tmem_cols_for(int ncomp) {
  uint32_t c = 32;
  while ((int)c < ncomp) c <<= 1;
  return c;
}

// One operand chunk (g frequencies of Re and Im, already scaled) as planes:
// SPLIT [Re_hi Im_hi Re_lo Im_lo] (16 each), BF16 [Re Im] (32 each).
template <int P>
__device__ __forceinline__ void pack_chunk(const float* re, const float* im, uint4 (&outv)[8]) {
  if (P == 2) {
    split8_f32(re, outv[0], outv[4]);
    split8_f32(re + 8, outv[1], outv[5]);
    split8_f32(im, outv[2], outv[6]);
    split8_f32(im + 8, outv[3], outv[7]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) outv[q] = bf16x8_f32(re + 8 * q);
#pragma unroll
    for (int q = 0; q < 4; ++q) outv[4 + q] = bf16x8_f32(im + 8 * q);
  }
}

// Chunk c of the warp's 32 operand rows (row nu0 + lane holds pk) to global
// memory through the warp's 4 KB staging box.  The rows lie rowlen elements
// apart, so each thread storing its own row would touch 32 lines per store
// instruction; restaged (XOR-swizzled, conflict-free), every instruction
// writes four whole 128-byte lines.
__device__ __forceinline__ void store_rows_chunk(uint8_t* stg, const uint4 (&pk)[8], uint16_t* out,
                                                 long rowlen, int nu0, int n, int c, int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) *(uint4*)(stg + lane * 128 + ((k ^ (lane & 7)) << 4)) = pk[k];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int rr = i * 4 + (lane >> 3), pc = lane & 7;
    const uint4 v = *(const uint4*)(stg + rr * 128 + ((pc ^ (rr & 7)) << 4));
    if (nu0 + rr < n)
      *(uint4*)((uint8_t*)(out + (size_t)(nu0 + rr) * rowlen) + c * 128 + pc * 16) = v;
  }
  __syncwarp();
}

// One centred step of the second pass: d = y - rh - rl (0 when !in_range),
// d^2 added to the Kahan sum (ss, ss_c); returns d fy.
__device__ __forceinline__ float center_step(float y, float2 ref, float fy, float& ss,
                                             float& ss_c, bool in_range) {
  float d = 0.f;
  if (in_range) {
    float ds, de;
    two_sum(y, -ref.x, ds, de);
    d = ds + (de - ref.y);
  }
  const float sq = fmaf(d, d, -ss_c);
  const float tsum = ss + sq;
  ss_c = (tsum - ss) - sq;
  ss = tsum;
  return d * fy;
}

// One round of the first pass over a thread's steps j0, j0 + 2, ..., j0 + 62
// (PREP_GROUPS = 2 threads per variable): the 32 loads are in flight before
// the first is used.  SUMS: each four values are summed exactly as
// s4 + (e1 + e2 + e3) by TwoSum (the residuals are below half an ulp of s4,
// their FP32 sum is off by ~2^-48 s4) and the pair joins the running (sh, sl)
// sum.  FULL: every step is below m; otherwise the steps past m read as zeros
// (they add nothing to the sums) and stay out of the extremes.
template <bool FULL, bool SUMS>
__device__ __forceinline__ void first_pass_round(const float* __restrict__ y, long ld, long col,
                                                 int j0, int m, float& sh, float& sl, float& mn,
                                                 float& mx) {
  static_assert(PREP_GROUPS == 2, "step interleave of the first pass");
  float v[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    const int j = j0 + e * PREP_GROUPS;
    v[e] = (FULL || j < m) ? __ldg(y + (long)j * ld + col) : 0.f;
  }
  if (SUMS) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (!FULL && j0 + 4 * q * PREP_GROUPS >= m) break;  // warp-uniform
      const float a = v[4 * q], b = v[4 * q + 1], c = v[4 * q + 2], d = v[4 * q + 3];
      float s1, e1, s2, e2, s4, e3;
      two_sum(a, b, s1, e1);
      two_sum(c, d, s2, e2);
      two_sum(s1, s2, s4, e3);
      df_acc(sh, sl, s4, (e1 + e2) + e3);
    }
  }
#pragma unroll
  for (int e = 0; e < 32; ++e)
    if (FULL || j0 + e * PREP_GROUPS < m) {
      mn = fminf(mn, v[e]);
      mx = fmaxf(mx, v[e]);
    }
}

template <int P>
__global__ void __launch_bounds__(PREP_THREADS, 2) k_prep_tc(const PrepJob* __restrict__ jobs,
                                                          const PrepItem* __restrict__ items,
                                                          int* err, unsigned long long limit_ns) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // The cross-spectrum launch behind this one may start its setup on free SMs
  // now; it waits for this launch to complete before it reads anything.
  griddep_launch_dependents();
  const PrepItem item = items[blockIdx.x];
  const PrepJob& job = jobs[item.job];
  const int m = job.m, n = job.n, kp = job.kp;
  const int ncomp = 2 * kp;  // rows of W: cos block then -sin block
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int r = t % PREP_ROWS, g = t / PREP_ROWS;  // variable row, step group
  const int nu = item.tile * PREP_ROWS + r;
  const bool valid = nu < n;
  const WaitCtl wc{err, limit_ns};

  // shared memory: A planes (128 rows x 128 B each), W planes (ncomp rows x
  // 128 B each) -- after the last MMA the epilogue's staging boxes (8 warps x
  // 4 KB) -- then reduction scratch and barriers
  uint8_t* sA = base;
  uint8_t* sW = base + P * PREP_ROWS * 128;
  const uint32_t wbytes = (uint32_t)ncomp * 128u;
  const uint32_t tiles = P * PREP_ROWS * 128 + P * wbytes;
  float* red_sh = (float*)(base + (tiles > PREP_STAGING ? tiles : PREP_STAGING));  // [2][128] sums, high
  float* red_sl = red_sh + PREP_GROUPS * PREP_ROWS;        // [2][128] sums, low parts
  float* red_mn = red_sl + PREP_GROUPS * PREP_ROWS;
  float* red_mx = red_mn + PREP_GROUPS * PREP_ROWS;
  float* red_ss = red_mx + PREP_GROUPS * PREP_ROWS;        // Kahan partials
  float* red_max = red_mn;                                 // epilogue row maxima (reuse)
  float2* row_ref = (float2*)(red_ss + PREP_GROUPS * PREP_ROWS);  // (rh, rl)
  int* row_ey = (int*)(row_ref + PREP_ROWS);
  uint64_t* bars = (uint64_t*)(row_ey + PREP_ROWS);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2);
  const uint32_t wbar = smem_u32(&bars[0]), mbar = smem_u32(&bars[1]);
  const uint32_t ncols = tmem_cols_for(ncomp);

  if (t == 0) {
    mbar_init(wbar, 1);
    mbar_init(mbar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), ncols);
    tmem_relinquish();
  }
  // ---- 1. double-float partial sums over steps j = g, g+2, ..., FP32 extremes
  // Rows past n read the last column (their results are never stored), so
  // no load needs a row predicate.
  const float* y = job.y;
  const long col = (long)(valid ? nu : n - 1) * (job.cstride_m1 + 1);  // column of variable nu in y
  const long ld = job.ld;
  {
    float sh = 0.f, sl = 0.f;
    float mn = __int_as_float(0x7f800000), mx = -__int_as_float(0x7f800000);
    // Rounds of 32 steps per thread (64 per variable) with every step below
    // m run without predicates; the last, partial round reads the steps past
    // m as zeros.
    int j0 = g;
    if (job.ref) {  // the caller's reference: extremes only
      for (; j0 + 31 * PREP_GROUPS < m; j0 += 32 * PREP_GROUPS)
        first_pass_round<true, false>(y, ld, col, j0, m, sh, sl, mn, mx);
      if (j0 < m) first_pass_round<false, false>(y, ld, col, j0, m, sh, sl, mn, mx);
    } else {
      for (; j0 + 31 * PREP_GROUPS < m; j0 += 32 * PREP_GROUPS)
        first_pass_round<true, true>(y, ld, col, j0, m, sh, sl, mn, mx);
      if (j0 < m) first_pass_round<false, true>(y, ld, col, j0, m, sh, sl, mn, mx);
    }
    red_sh[g * PREP_ROWS + r] = sh;
    red_sl[g * PREP_ROWS + r] = sl;
    red_mn[g * PREP_ROWS + r] = mn;
    red_mx[g * PREP_ROWS + r] = mx;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (g == 0) {
    float rh = 0.f, rl = 0.f, amax = 0.f;
    {  // rows past n repeat the last variable
      float mn = red_mn[r], mx = red_mx[r];
      float sh = red_sh[r], sl = red_sl[r];
      for (int k = 1; k < PREP_GROUPS; ++k) {
        df_acc(sh, sl, red_sh[k * PREP_ROWS + r], red_sl[k * PREP_ROWS + r]);
        mn = fminf(mn, red_mn[k * PREP_ROWS + r]);
        mx = fmaxf(mx, red_mx[k * PREP_ROWS + r]);
      }
      if (job.ref) {
        rh = job.ref[col];
      } else {
        // (sh + sl) / m: the remainder sh - q1 m of the rounded quotient q1 is
        // exact in FP32 and is computed exactly by the FMA
        const float fm = (float)m;
        const float q1 = __fdiv_rn(sh, fm);
        const float q2 = __fdiv_rn(fmaf(-q1, fm, sh) + sl, fm);
        two_sum(q1, q2, rh, rl);
      }
      amax = fmaxf((mx - rh) - rl, (rh - mn) + rl);  // extremes of |y - ref|
    }
    int ey = 0;
    if (amax > 0.f) {
      int e;
      frexpf(amax, &e);  // amax < 2^e
      ey = 14 - e;      // scaled maximum in [2^13, 2^14)
      if (ey > 126) ey = 126;  // keep 2^ey a normal FP32 number (data below ~1e-34)
    }
    row_ref[r] = make_float2(rh, rl);
    row_ey[r] = ey;
  }
  __syncthreads();
  const uint32_t tmem = *tmem_slot;
  const float2 ref = row_ref[r];
  const float fy = ldexpf(1.0f, row_ey[r]);
  float ss = 0.f, ss_c = 0.f;  // Kahan sum of (y - ref)^2 over this thread's steps
  bool ok = true;

  // ---- 2./3. A chunks of 64 perturbation steps, MMA with the twiddle chunk
  const int jchunks = job.jchunks;
  const int nhalf = ncomp > 256 ? 2 : 1;
  const int nfirst = ncomp > 256 ? 256 : ncomp;
  const uint32_t id0 = idesc_f16(128, nfirst, P == 1, false);
  const uint32_t id1 = idesc_f16(128, ncomp - 256 > 0 ? ncomp - 256 : 16, P == 1, false);
  int w_armed = 0, m_committed = 0;  // thread 0: async operations started
  for (int kc = 0; kc < jchunks; ++kc) {
    // this thread's groups of 8 steps: jg = g, g + 2, g + 4, g + 6; the loads
    // are issued before waiting for the previous chunk's MMAs
    // (groups of 8 steps below m load without predicates; warp-uniform)
    float yv[PREP_JG][8];
#pragma unroll
    for (int h = 0; h < PREP_JG; ++h) {
      const int jb = kc * 64 + (g + PREP_GROUPS * h) * 8;
      if (jb + 8 <= m) {
#pragma unroll
        for (int e = 0; e < 8; ++e) yv[h][e] = __ldg(y + (long)(jb + e) * ld + col);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          yv[h][e] = (jb + e < m) ? __ldg(y + (long)(jb + e) * ld + col) : 0.f;
      }
    }
    if (kc > 0) ok = ok && mbar_wait(mbar, (kc - 1) & 1, wc);  // smem free again
    if (t == 0 && ok) {
      mbar_arrive_expect_tx(wbar, P * wbytes);
      ++w_armed;
      for (int p = 0; p < P; ++p)
        bulk_load(smem_u32(sW + p * wbytes), job.wtab + ((size_t)kc * P + p) * wbytes, wbytes,
                  wbar);
    }
#pragma unroll
    for (int h = 0; h < PREP_JG; ++h) {
      const int jg = g + PREP_GROUPS * h;
      const uint32_t off = sw128_off((uint32_t)r, (uint32_t)jg);
      if (kc * 64 + jg * 8 >= m) {  // steps past m (warp-uniform): zeros
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        *(uint4*)(sA + off) = z;
        if (P == 2) *(uint4*)(sA + PREP_ROWS * 128 + off) = z;
        continue;
      }
      // centering y - rh - rl (steps past m: 0); scaling by 2^ey is exact
      float v[8];
      if (kc * 64 + jg * 8 + 8 <= m) {  // warp-uniform
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = center_step(yv[h][e], ref, fy, ss, ss_c, true);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          v[e] = center_step(yv[h][e], ref, fy, ss, ss_c, kc * 64 + jg * 8 + e < m);
      }
      if (P == 2) {
        uint4 hi, lo;
        split8_f32(v, hi, lo);
        *(uint4*)(sA + off) = hi;
        *(uint4*)(sA + PREP_ROWS * 128 + off) = lo;
      } else {
        *(uint4*)(sA + off) = bf16x8_f32(v);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0 && ok) {
      ok = mbar_wait(wbar, kc & 1, wc);
      if (ok) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), w0 = smem_u32(sW);
        const int ncombo = P == 2 ? 3 : 1;
        // (A plane, W plane) products: the small hi*lo and lo*hi of all four
        // 16-step slices first, hi*hi last, so that fewer of the accumulator's
        // (truncating) additions happen at its full size
#pragma unroll 1
        for (int o = 0; o < 4 * ncombo; ++o) {
          const int cb = (ncombo == 3) ? (o < 8 ? 1 + (o & 1) : 0) : 0;
          const int ks = (ncombo == 3) ? (o < 8 ? o >> 1 : o - 8) : o;
          const int pa = (cb == 2) ? 1 : 0, pw = (cb == 1) ? 1 : 0;
          const uint64_t ad = sw128_desc(a0 + pa * PREP_ROWS * 128 + ks * 32);
          const uint32_t acc = (kc > 0 || o > 0) ? 1u : 0u;
          for (int hh = 0; hh < nhalf; ++hh) {
            const uint64_t bd = sw128_desc(w0 + pw * wbytes + hh * 256 * 128 + ks * 32);
            mma_f16(tmem + hh * 256, ad, bd, hh ? id1 : id0, acc);
          }
        }
        mma_commit(mbar);
        ++m_committed;
      }
    }
  }
  red_ss[g * PREP_ROWS + r] = ss;
  ok = ok && mbar_wait(mbar, (jchunks - 1) & 1, wc);
  tc_fence_after();

  // ---- 4. epilogue: warp w reads TMEM lane quadrant q = w % 4 and column
  // part w / 4 (PREP_GROUPS parts)
  const int q = warp & 3, part = warp >> 2;
  const int lr = q * 32 + lane;                       // tile row (TMEM lane)
  const int nu_e = item.tile * PREP_ROWS + lr;
  const bool valid_e = nu_e < n;
  const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
  float dmax = 0.f;
  for (int b = part; b < ncomp / 16; b += PREP_GROUPS) {
    float v[16];
    tmem_ld16(trow + b * 16, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) dmax = fmaxf(dmax, fabsf(v[i]));
  }
  red_max[part * PREP_ROWS + lr] = dmax;
  __syncthreads();
  dmax = red_max[lr];
  for (int k = 1; k < PREP_GROUPS; ++k) dmax = fmaxf(dmax, red_max[k * PREP_ROWS + lr]);
  int eY = 0;
  if (dmax > 0.f) {
    int e;
    frexpf(dmax, &e);
    eY = 14 - e;
  }
  const float fY = ldexpf(1.0f, eY);
  const int gsz = (P == 2) ? 16 : 32;
  const int nch = kp / gsz;
  uint8_t* stg = base + warp * 4096;  // the operand tiles are free after the last MMA
  const int nu0 = item.tile * PREP_ROWS + q * 32;
  // The half-spectrum weight w (1 at omega = 0, the first element of chunk
  // 0; 2 otherwise) enters both operands as sqrt(w), so that every product
  // of a stack-1 and a stack-2 row carries w and a homo problem needs one row
  // set for both.  The Hilbert variant has weight 1 everywhere.  fY is a
  // power of two, so one product by fY sqrt(w) rounds as (x fY) sqrt(w) does.
  const float fYw = job.plain_weights ? fY : fY * 1.41421356f;
  for (int c = part; c < nch; c += PREP_GROUPS) {
    float re[32], im[32];
    if (P == 2) {
      float a[16], b[16];
      tmem_ld16(trow + c * 16, a);
      tmem_ld16(trow + kp + c * 16, b);
#pragma unroll
      for (int i = 0; i < 16; ++i) { re[i] = a[i] * fYw; im[i] = b[i] * fYw; }
      if (c == 0) { re[0] = a[0] * fY; im[0] = b[0] * fY; }
    } else {
      float a[32], b[32];
      tmem_ld32(trow + c * 32, a);
      tmem_ld32(trow + kp + c * 32, b);
#pragma unroll
      for (int i = 0; i < 32; ++i) { re[i] = a[i] * fYw; im[i] = b[i] * fYw; }
      if (c == 0) { re[0] = a[0] * fY; im[0] = b[0] * fY; }
    }
    uint4 pk[8];
    pack_chunk<P>(re, im, pk);
    if (job.outA) store_rows_chunk(stg, pk, job.outA, job.rowlen, nu0, n, c, lane);
    if (job.outB && job.outB != job.outA)
      store_rows_chunk(stg, pk, job.outB, job.rowlen, nu0, n, c, lane);
  }
  if (part == 0 && valid_e) {
    float s2sum = red_ss[lr];
    for (int k = 1; k < PREP_GROUPS; ++k) s2sum += red_ss[k * PREP_ROWS + lr];
    const float sigma = sqrtf(__fdiv_rn(s2sum, (float)(m - 1)));
    float sc = 1.f;
    int ex = 0;
    if (job.alpha > 0.0) {
      if (sigma == 0.f) {
        sc = 0.f;
      } else if (job.alpha <= 64.0) {
        // sigma^-alpha = f^-alpha 2^(-alpha k) with sigma = f 2^k, f in
        // [0.5, 1): f^-alpha <= 2^64 cannot overflow, and -alpha k is split
        // into integer and fraction in FP64 (two operations per variable)
        int k;
        const float f = frexpf(sigma, &k);
        const double tk = fmin(fmax(-job.alpha * (double)k, -1024.0), 1024.0);
        const double ti = floor(tk);
        sc = powf(f, (float)-job.alpha) * exp2f((float)(tk - ti));
        ex = (int)ti;
      } else {
        const double p = pow((double)sigma, -job.alpha);
        int k;
        sc = (float)frexp(p, &k);
        ex = k;
      }
    }
    job.scale[nu_e] = ldexpf(sc, ex - (row_ey[lr] + eY));
    if (job.sigma_out) job.sigma_out[nu_e] = sigma;
  }
  if (t == 0 && !ok) {  // abort: let started copies and MMAs finish
    if (w_armed > 0) mbar_wait_drain(wbar, (w_armed - 1) & 1, limit_ns);
    if (m_committed > 0) mbar_wait_drain(mbar, (m_committed - 1) & 1, limit_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

static size_t prep_smem_bytes(int planes, int max_kp) {
  size_t tiles = (size_t)planes * PREP_ROWS * 128 + (size_t)planes * 2 * max_kp * 128;
  if (tiles < PREP_STAGING) tiles = PREP_STAGING;
  size_t bytes = 1024 + tiles + PREP_SCRATCH + 64;
  // Keep (CTAs per SM) x (TMEM columns per CTA) <= 512 so allocation never waits.
  const uint32_t cols = tmem_cols_for(2 * max_kp);
  const size_t sm_smem = 233472;  // shared memory per SM
  const size_t max_cta = 512 / cols;
  const size_t floor_bytes = sm_smem / (max_cta + 1) + 1024;
  return bytes > floor_bytes ? bytes : floor_bytes;
}

cudaError_t launch_prep_tc(const PrepJob* d_jobs, const PrepItem* d_items, int nitems, int planes,
                           int max_kp, int* err, unsigned long long limit_ns, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  size_t smem = prep_smem_bytes(planes, max_kp);
  if (planes == 2)
    k_prep_tc<2><<<nitems, PREP_THREADS, smem, s>>>(d_jobs, d_items, err, limit_ns);
  else
    k_prep_tc<1><<<nitems, PREP_THREADS, smem, s>>>(d_jobs, d_items, err, limit_ns);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core DFT (the plain GPU baseline).  One CTA per 32 variables, 8
// warps; lane = variable, warps stride over frequencies.  FP64 reference and
// centering, then FP32 values in shared memory and FP32 twiddles indexed by
// (omega j) mod m.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prep_simt(SimtPrepJob job) {
  extern __shared__ float sm[];
  const int m = job.m, n = job.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nu = blockIdx.x * 32 + lane;
  const bool valid = nu < n;
  float* tw = sm;              // 2m
  float* yt = sm + 2 * m;      // m x 32 centred values
  double* red = (double*)(yt + (size_t)m * 32);  // 8 x 32 partial sums
  for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) tw[i] = job.tw[i];
  // reference (FP64)
  double part = 0.0;
  if (!job.ref && valid)
    for (int j = warp; j < m; j += 8) part += (double)job.y[(long)j * job.ld + nu];
  red[warp * 32 + lane] = part;
  __syncthreads();
  double ref;
  if (job.ref) {
    ref = valid ? (double)job.ref[nu] : 0.0;
  } else {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w * 32 + lane];
    ref = s / (double)m;
  }
  __syncthreads();
  part = 0.0;
  for (int j = warp; j < m; j += 8) {
    double d = valid ? (double)job.y[(long)j * job.ld + nu] - ref : 0.0;
    part += d * d;
    yt[(size_t)j * 32 + lane] = (float)d;
  }
  red[warp * 32 + lane] = part;
  __syncthreads();
  if (warp == 0 && valid) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w * 32 + lane];
    double sigma = sqrt(s / (double)(m - 1));
    double sc = (job.alpha > 0.0) ? (sigma == 0.0 ? 0.0 : pow(sigma, -job.alpha)) : 1.0;
    job.scale[nu] = (float)sc;
    if (job.sigma_out) job.sigma_out[nu] = (float)sigma;
  }
  for (int w = warp; w < job.kp1; w += 8) {
    float re = 0.f, im = 0.f;
    int rr = 0;  // (w * j) mod m, advanced incrementally
    for (int j = 0; j < m; ++j) {
      float d = yt[(size_t)j * 32 + lane];
      re = fmaf(d, tw[2 * rr], re);
      im = fmaf(-d, tw[2 * rr + 1], im);
      rr += w;
      if (rr >= m) rr -= m;
    }
    if (valid) {
      const size_t at = (size_t)w * job.ldp + nu;
      if (job.yr) {
        job.yr[at] = re;
        job.yi[at] = im;
      }
      if (job.yrw) {
        float wt = (w == 0) ? 1.f : 2.f;
        job.yrw[at] = wt * re;
        job.yiw[at] = wt * im;
      }
    }
  }
}

static size_t simt_prep_smem_bytes(int m) {
  return (size_t)2 * m * 4 + (size_t)m * 32 * 4 + 8 * 32 * 8;
}

cudaError_t init_prep_kernels() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_prep_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_prep_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_prep_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

cudaError_t launch_prep_simt(const SimtPrepJob& job, cudaStream_t s) {
  size_t smem = simt_prep_smem_bytes(job.m);
  if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  k_prep_simt<<<(job.n + 31) / 32, 256, smem, s>>>(job);
  return cudaGetLastError();
}

}  // namespace c2d
