// Complex cross-spectrum with the stack-1 operand held in TMEM: the same
// product as k_xspec_tc (Eq. disint2d with the half-spectrum weights of
// Sec. 4.2), organised so that each tensor-core instruction reads only the
// stack-2 operand from shared memory.
//
// A work unit is a row segment: the 128 stack-1 rows of tile row ti against
// up to ntj column tiles of 128 stack-2 rows.  The segment's stack-1 chunks
// (at most 8: m <= 256 in split precision) are copied once into TMEM columns
// 0..255 with tcgen05.cp; the tiles then stream their stack-2 chunks through
// shared memory, and every MMA takes A from TMEM.  Per tile this removes the
// stack-1 operand's shared-memory reads (half of the MMAs' operand traffic),
// the largest item of the single-CTA kernel's shared-memory budget.
//
// TMEM: A chunk c at columns 32c .. 32c + 31 (four 16-element K slices of 8
// columns: Re_hi, Im_hi, Re_lo, Im_lo in split precision); one accumulator
// set, Phi at 256 and Psi at 384 (128 columns each).  With a single set the
// epilogue first moves a tile's accumulators into registers (4 x 32 values
// per thread), hands TMEM back, and then scales and stores while the MMAs of
// the next tile run.  Roles, tile order and the mirrored boxes of homo
// problems are those of k_xspec_tc: warp 0 TMA producer, warp 1 MMA issuer
// (one thread), warps 2..9 epilogue (Phi / Psi x TMEM lane quadrant).
#include "internal.h"
#include "ptx.cuh"

namespace c2d {

constexpr int TA_STAGES = 8;
constexpr int TA_STAGE_BYTES = TILE_M * 128;  // one 128-row chunk of either operand
constexpr int TA_EPI_WARPS = 8;
constexpr int TA_BOX_BYTES = 32 * 32 * 4;
constexpr int TA_EPI_SLOTS = 2;
constexpr int TA_THREADS = 64 + 32 * TA_EPI_WARPS;
constexpr size_t TA_SMEM = 1024 + (size_t)TA_STAGES * TA_STAGE_BYTES +
                           (size_t)TA_EPI_WARPS * TA_EPI_SLOTS * TA_BOX_BYTES +
                           (size_t)TA_EPI_WARPS * TILE_N * 4 + 256;
static_assert(TA_SMEM <= (size_t)kMaxDynSmem, "TMEM-operand kernel shared memory exceeds the limit");
constexpr uint32_t TA_ACC_COL = 256;  // Phi at 256, Psi at 384
static_assert(32 * TA_MAX_CHUNKS <= (int)TA_ACC_COL, "operand columns overlap the accumulators");

template <int P>
__device__ __forceinline__ void issue_chunk_mmas_ta(uint32_t d_phi, uint32_t d_psi, uint32_t ta,
                                                    uint32_t b0, uint32_t acc, uint32_t ID,
                                                    uint32_t IDN) {
  // ta: TMEM column of the chunk's A slices (8 columns each); b0: shared B chunk.
  // Products and order as issue_chunk_mmas (k_xspec.cu): corrections first.
  if (P == 2) {
    // slices: Re_hi @ta, Im_hi @ta+8, Re_lo @ta+16, Im_lo @ta+24
    mma_f16_ta(d_phi, ta + 0, sw128_desc(b0 + 64), ID, acc);     // Rh Rl
    mma_f16_ta(d_phi, ta + 8, sw128_desc(b0 + 96), ID, 1);       // Ih Il
    mma_f16_ta(d_phi, ta + 16, sw128_desc(b0 + 0), ID, 1);       // Rl Rh
    mma_f16_ta(d_phi, ta + 24, sw128_desc(b0 + 32), ID, 1);      // Il Ih
    mma_f16_ta(d_phi, ta + 0, sw128_desc(b0 + 0), ID, 1);        // Rh Rh
    mma_f16_ta(d_phi, ta + 8, sw128_desc(b0 + 32), ID, 1);       // Ih Ih
    mma_f16_ta(d_psi, ta + 8, sw128_desc(b0 + 64), ID, acc);     // Ih Rl
    mma_f16_ta(d_psi, ta + 0, sw128_desc(b0 + 96), IDN, 1);      // -Rh Il
    mma_f16_ta(d_psi, ta + 24, sw128_desc(b0 + 0), ID, 1);       // Il Rh
    mma_f16_ta(d_psi, ta + 16, sw128_desc(b0 + 32), IDN, 1);     // -Rl Ih
    mma_f16_ta(d_psi, ta + 8, sw128_desc(b0 + 0), ID, 1);        // Ih Rh
    mma_f16_ta(d_psi, ta + 0, sw128_desc(b0 + 32), IDN, 1);      // -Rh Ih
  } else {
    // slices: Re[0:16] @ta, Re[16:32] @ta+8, Im[0:16] @ta+16, Im[16:32] @ta+24
    mma_f16_ta(d_phi, ta + 0, sw128_desc(b0 + 0), ID, acc);
    mma_f16_ta(d_phi, ta + 8, sw128_desc(b0 + 32), ID, 1);
    mma_f16_ta(d_phi, ta + 16, sw128_desc(b0 + 64), ID, 1);
    mma_f16_ta(d_phi, ta + 24, sw128_desc(b0 + 96), ID, 1);
    mma_f16_ta(d_psi, ta + 16, sw128_desc(b0 + 0), ID, acc);
    mma_f16_ta(d_psi, ta + 24, sw128_desc(b0 + 32), ID, 1);
    mma_f16_ta(d_psi, ta + 0, sw128_desc(b0 + 64), IDN, 1);
    mma_f16_ta(d_psi, ta + 8, sw128_desc(b0 + 96), IDN, 1);
  }
}

template <int P>
__global__ void __launch_bounds__(TA_THREADS, 1)
    k_xspec_ta(const XProblem* __restrict__ probs, const XSeg* __restrict__ segs, int nsegs,
               int* err, unsigned long long limit_ns, int inject) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* stages = base;
  uint8_t* epi = base + TA_STAGES * TA_STAGE_BYTES;
  float* s2stage = (float*)(epi + TA_EPI_WARPS * TA_EPI_SLOTS * TA_BOX_BYTES);
  uint64_t* bars = (uint64_t*)(s2stage + TA_EPI_WARPS * TILE_N);
  // bars: full[S], empty[S], tfull, tempty, abar
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * TA_STAGES + 3);
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[TA_STAGES + s]); };
  const uint32_t tfull = smem_u32(&bars[2 * TA_STAGES]);
  const uint32_t tempty = smem_u32(&bars[2 * TA_STAGES + 1]);
  const uint32_t abar = smem_u32(&bars[2 * TA_STAGES + 2]);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WaitCtl wc{err, limit_ns};

  if (threadIdx.x == 0) {
    for (int s = 0; s < TA_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, TA_EPI_WARPS);
    mbar_init(abar, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[TA_STAGES];
      uint32_t armed_phase[TA_STAGES];
      for (int s = 0; s < TA_STAGES; ++s) armed[s] = 0, armed_phase[s] = 0;
      bool ok = (inject & 1) == 0;  // inject & 1: issue nothing (time-out test)
      const uint64_t keep = l2_policy_evict_last();
      for (int k = 0; ok; ++k) {
        const int si = k * (int)gridDim.x + (int)blockIdx.x;
        if (si >= nsegs) break;
        const XSeg sg = segs[si];
        const XProblem* pr = probs + sg.prob;
        const int nch = pr->nchunks;
        // the segment's stack-1 chunks, then each tile's stack-2 chunks from
        // the highest frequencies down
        const int nload = nch * (1 + (int)sg.ntj);
        for (int l = 0; l < nload; ++l) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, wc)) { ok = false; break; }
          mbar_arrive_expect_tx(full_bar(stage), TILE_M * 128u);
          armed[stage] = 1;
          armed_phase[stage] = phase;
          const uint32_t dst = smem_u32(stages + stage * TA_STAGE_BYTES);
          if (l < nch) {
            tma_load_2d_hint(dst, &pr->tmA, l * CHUNK_ELEMS, (int)sg.ti * TILE_M, full_bar(stage),
                             keep);
          } else {
            const int t = (l - nch) / nch, c = nch - 1 - (l - nch) % nch;
            tma_load_2d_hint(dst, &pr->tmB, c * CHUNK_ELEMS, ((int)sg.tj0 + t) * TILE_N,
                             full_bar(stage), keep);
          }
          if (++stage == TA_STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      for (int s = 0; s < TA_STAGES; ++s)
        if (armed[s]) mbar_wait_drain(full_bar(s), armed_phase[s], limit_ns);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0, committed = 0, nseg = 0;
      uint32_t last_bar = 0, last_parity = 0;
      bool ok = true;
      const uint32_t id = idesc_f16(TILE_M, TILE_N, P == 1, false);
      const uint32_t idn = idesc_f16(TILE_M, TILE_N, P == 1, true);
      const uint32_t d_phi = tmem + TA_ACC_COL, d_psi = d_phi + 128u;
      for (int k = 0; ok; ++k) {
        const int si = k * (int)gridDim.x + (int)blockIdx.x;
        if (si >= nsegs) break;
        const XSeg sg = segs[si];
        const int nch = probs[sg.prob].nchunks;
        // abar completes twice per segment (copies landed; MMAs done).  The
        // previous segment's MMAs read the columns about to be overwritten.
        if (nseg > 0 && !mbar_wait(abar, 1u, wc)) { ok = false; break; }
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(full_bar(stage), phase, wc)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stages + stage * TA_STAGE_BYTES);
#pragma unroll
          for (int sl = 0; sl < 4; ++sl)
            tmem_cp_128x256b(tmem + (uint32_t)(32 * c + 8 * sl), sw128_desc(a0 + 32 * sl));
          mma_commit(empty_bar(stage));
          ++committed;
          last_bar = empty_bar(stage);
          last_parity = phase;
          if (++stage == TA_STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(abar);
        if (!mbar_wait(abar, 0u, wc)) { ok = false; break; }
        tc_fence_after();
        for (int t = 0; t < (int)sg.ntj && ok; ++t, ++lt) {
          // the epilogue has moved the previous tile's accumulators out
          if (!mbar_wait(tempty, ((uint32_t)lt & 1u) ^ 1u, wc)) { ok = false; break; }
          tc_fence_after();
          for (int j = 0; j < nch; ++j) {
            const int c = nch - 1 - j;  // high frequencies first
            if (!mbar_wait(full_bar(stage), phase, wc)) { ok = false; break; }
            tc_fence_after();
            const uint32_t b0 = smem_u32(stages + stage * TA_STAGE_BYTES);
            issue_chunk_mmas_ta<P>(d_phi, d_psi, tmem + (uint32_t)(32 * c), b0, j > 0 ? 1u : 0u,
                                   id, idn);
            mma_commit(empty_bar(stage));
            ++committed;
            last_bar = empty_bar(stage);
            last_parity = phase;
            if (++stage == TA_STAGES) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          mma_commit(tfull);
        }
        if (!ok) break;
        mma_commit(abar);
        ++nseg;
      }
      if (committed > 0) mbar_wait_drain(last_bar, last_parity, limit_ns);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int half = ew >> 2;     // 0: Phi, 1: Psi
    const int q = warp & 3;       // TMEM lane quadrant
    const float sgn = half ? -1.f : 1.f;
    const uint64_t stream_out = l2_policy_evict_first();
    uint8_t* ring = epi + ew * TA_EPI_SLOTS * TA_BOX_BYTES;
    float* s2w = s2stage + ew * TILE_N;
    int lt = 0;
    int slot = 0;
    bool alive = true;
    for (int k = 0; alive; ++k) {
      const int si = k * (int)gridDim.x + (int)blockIdx.x;
      if (si >= nsegs) break;
      const XSeg sg = segs[si];
      const XProblem* pr = probs + sg.prob;
      const CUtensorMap* tm = half ? &pr->tmPsi : &pr->tmPhi;
      const int n1 = pr->n1, n2 = pr->n2, pmirror = pr->mirror, upper = pr->upper_only;
      const int row0 = (int)sg.ti * TILE_M + q * 32;
      const int row = row0 + lane;
      const float rs = (row < n1) ? pr->norm * __ldg(pr->s1 + row) : 0.f;
      const bool rows_in = row0 < n1;
      for (int t = 0; t < (int)sg.ntj; ++t, ++lt) {
        const int tj = (int)sg.tj0 + t;
        const int colt = tj * TILE_N;
        {
          const int c = colt + lane * 4;
          float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (c + 3 < n2) {
            sv = __ldg((const float4*)(pr->s2 + c));
          } else {
            if (c < n2) sv.x = __ldg(pr->s2 + c);
            if (c + 1 < n2) sv.y = __ldg(pr->s2 + c + 1);
            if (c + 2 < n2) sv.z = __ldg(pr->s2 + c + 2);
          }
          *(float4*)(s2w + lane * 4) = sv;
        }
        __syncwarp();
        if (!mbar_wait(tfull, (uint32_t)lt & 1u, wc)) { alive = false; break; }
        tc_fence_after();
        float v[4][32];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) +
                        (TA_ACC_COL + (uint32_t)(half * 128 + cc * 32)),
                    v[cc]);
        // accumulators are in registers: TMEM is free for the next tile
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty);
        if (!rows_in) continue;
        // mirrored problems as in k_xspec_tc: on the diagonal tile box cc > q
        // stores itself and its mirror, cc == q its upper triangle mirrored,
        // cc < q nothing
        const bool diag = pmirror && ((int)sg.ti == tj);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int col0 = colt + cc * 32;
          if (col0 >= n2) break;  // warp-uniform
          if (diag && cc < q) continue;
          const bool mirror = pmirror && !upper && (!diag || cc > q);
          const bool tri = diag && cc == q;
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 s4 = *(const float4*)(s2w + cc * 32 + i);
            v[cc][i] = v[cc][i] * rs * s4.x;
            v[cc][i + 1] = v[cc][i + 1] * rs * s4.y;
            v[cc][i + 2] = v[cc][i + 2] * rs * s4.z;
            v[cc][i + 3] = v[cc][i + 3] * rs * s4.w;
          }
          const bool two = mirror && !tri;
          if (lane == 0) {
            if (two)
              bulk_wait_read<TA_EPI_SLOTS - 2>();
            else
              bulk_wait_read<TA_EPI_SLOTS - 1>();
          }
          __syncwarp();
          uint8_t* slot0 = ring + slot * TA_BOX_BYTES;
          uint8_t* slot1 = ring + ((slot + 1) % TA_EPI_SLOTS) * TA_BOX_BYTES;
          if (!tri) {
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4)
              *(float4*)(slot0 + sw128_off(lane, c4)) =
                  make_float4(v[cc][4 * c4], v[cc][4 * c4 + 1], v[cc][4 * c4 + 2],
                              v[cc][4 * c4 + 3]);
            if (mirror) {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                *(float*)(slot1 + sw128_off(i, lane >> 2) + (lane & 3) * 4) = sgn * v[cc][i];
            }
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (c > lane) {
                *(float*)(slot0 + sw128_off(lane, c >> 2) + (c & 3) * 4) = v[cc][c];
                *(float*)(slot0 + sw128_off(c, lane >> 2) + (lane & 3) * 4) = sgn * v[cc][c];
              } else if (c == lane) {
                *(float*)(slot0 + sw128_off(lane, c >> 2) + (c & 3) * 4) = half ? 0.f : v[cc][c];
              }
            }
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d_hint(tm, col0, row0, smem_u32(slot0), stream_out);
            bulk_commit();
            if (two) {
              tma_store_2d_hint(tm, row0, col0, smem_u32(slot1), stream_out);
              bulk_commit();
            }
          }
          slot = (slot + (two ? 2 : 1)) % TA_EPI_SLOTS;
        }
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

cudaError_t init_xspec_ta_kernels() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_xspec_ta<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TA_SMEM)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_xspec_ta<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TA_SMEM);
}

cudaError_t launch_xspec_ta(const XProblem* d_probs, const XSeg* d_segs, int nsegs, int planes,
                            int grid, int* err, unsigned long long limit_ns, cudaStream_t s,
                            int inject) {
  if (nsegs <= 0) return cudaSuccess;
  if (grid > nsegs) grid = nsegs;
  if (planes == 2)
    k_xspec_ta<2><<<grid, TA_THREADS, TA_SMEM, s>>>(d_probs, d_segs, nsegs, err, limit_ns, inject);
  else
    k_xspec_ta<1><<<grid, TA_THREADS, TA_SMEM, s>>>(d_probs, d_segs, nsegs, err, limit_ns, inject);
  return cudaGetLastError();
}

}  // namespace c2d
