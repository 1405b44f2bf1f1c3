// Complex cross-spectrum on CTA pairs (tcgen05 cta_group::2), the same
// product as k_xspec_tc (Eq. disint2d with the half-spectrum weights of
// Sec. 4.2):
//   Phi(nu1, nu2) = norm s1[nu1] s2[nu2] sum_w w (Re1 Re2 + Im1 Im2)
//   Psi(nu1, nu2) = norm s1[nu1] s2[nu2] sum_w w (Im1 Re2 - Re1 Im2)
//
// A work item is a 256 x 128 tile: rows 256a .. 256a + 255 of stack 1 and
// columns 128 tj .. 128 tj + 127 of stack 2.  Each CTA of a two-CTA cluster
// holds its own 128 stack-1 rows and half (64) of the 128 stack-2 rows; one
// MMA instruction issued by the even CTA multiplies the 256 rows by all 128
// columns, each CTA receiving its 128 x 128 accumulators in its own TMEM.
// Against one CTA per 128 x 128 tile this halves the stack-2 operand bytes a
// CTA loads and reads from shared memory per output (four shared-memory bytes
// per output byte become three for the operands).  Measured on GB300 the
// coupling of the two SMs (an MMA waits for both operand halves, a TMEM buffer
// for both epilogues) costs more than the saved traffic: the kernel runs 2-20 %
// slower than k_xspec_tc, so the library uses it only on request
// (CORR2D_XSPEC=pair or =any).
//
// Roles (320 threads per CTA, as in k_xspec_tc):
//   warp 0      TMA producer of this CTA's operand halves; both CTAs' loads
//               signal the even CTA's "full" barrier, which the even CTA arms
//               with the bytes of both halves
//   warp 1      even CTA: MMA issuer (one thread); its commits arrive on the
//               barriers of both CTAs (operand slot free, accumulators ready)
//   warps 2..9  epilogue of this CTA's 128 rows; after reading a TMEM buffer
//               every epilogue warp of both CTAs arrives on the even CTA's
//               "accumulators free" barrier
// Homo problems compute items with tj >= 2a: the odd CTA's tile (2a+1, 2a) of
// the item (a, 2a) lies below the diagonal and stores nothing (its transpose
// is stored by the even CTA of item (a, 2a+1)); everything else follows the
// mirror rules of k_xspec_tc.
#include "internal.h"
#include "ptx.cuh"

namespace c2d {

// operand stages and staging slots per epilogue warp (build-time overrides
// for sweeps; 4 stages measured 13 % slower, 6 stages or 3 slots no faster)
#ifndef C2D_XP_STAGES
#define C2D_XP_STAGES 5
#endif
#ifndef C2D_XP_SLOTS
#define C2D_XP_SLOTS 2
#endif
constexpr int XP_STAGES = C2D_XP_STAGES;
constexpr int XP_A_BYTES = TILE_M * 128;            // this CTA's 128 stack-1 rows of a chunk
constexpr int XP_B_BYTES = (TILE_N / 2) * 128;      // this CTA's 64 stack-2 rows of a chunk
constexpr int XP_STAGE_BYTES = XP_A_BYTES + XP_B_BYTES;
constexpr int XP_EPI_WARPS = 8;
constexpr int XP_BOX_BYTES = 32 * 32 * 4;
constexpr int XP_EPI_SLOTS = C2D_XP_SLOTS;
static_assert(XP_EPI_SLOTS >= 2, "a box and its mirror need two staging slots");
static_assert(XP_A_BYTES % 1024 == 0 && XP_STAGE_BYTES % 1024 == 0, "swizzle atoms are 1 KB");
constexpr int XP_THREADS = 64 + 32 * XP_EPI_WARPS;
constexpr size_t XP_SMEM = 1024 + (size_t)XP_STAGES * XP_STAGE_BYTES +
                           (size_t)XP_EPI_WARPS * XP_EPI_SLOTS * XP_BOX_BYTES +
                           (size_t)XP_EPI_WARPS * TILE_N * 4 + 256;
static_assert(XP_SMEM <= (size_t)kMaxDynSmem, "pair kernel shared memory exceeds the limit");

template <int P>
__device__ __forceinline__ void issue_chunk_mmas_pair(uint32_t d_phi, uint32_t d_psi, uint32_t a0,
                                                      uint32_t b0, uint32_t acc, uint32_t ID,
                                                      uint32_t IDN) {
  // same operand chunk layout, products and order as issue_chunk_mmas (k_xspec.cu)
  if (P == 2) {
    mma_f16_pair(d_phi, sw128_desc(a0 + 0), sw128_desc(b0 + 64), ID, acc);    // Rh Rl
    mma_f16_pair(d_phi, sw128_desc(a0 + 32), sw128_desc(b0 + 96), ID, 1);     // Ih Il
    mma_f16_pair(d_phi, sw128_desc(a0 + 64), sw128_desc(b0 + 0), ID, 1);      // Rl Rh
    mma_f16_pair(d_phi, sw128_desc(a0 + 96), sw128_desc(b0 + 32), ID, 1);     // Il Ih
    mma_f16_pair(d_phi, sw128_desc(a0 + 0), sw128_desc(b0 + 0), ID, 1);       // Rh Rh
    mma_f16_pair(d_phi, sw128_desc(a0 + 32), sw128_desc(b0 + 32), ID, 1);     // Ih Ih
    mma_f16_pair(d_psi, sw128_desc(a0 + 32), sw128_desc(b0 + 64), ID, acc);   // Ih Rl
    mma_f16_pair(d_psi, sw128_desc(a0 + 0), sw128_desc(b0 + 96), IDN, 1);     // -Rh Il
    mma_f16_pair(d_psi, sw128_desc(a0 + 96), sw128_desc(b0 + 0), ID, 1);      // Il Rh
    mma_f16_pair(d_psi, sw128_desc(a0 + 64), sw128_desc(b0 + 32), IDN, 1);    // -Rl Ih
    mma_f16_pair(d_psi, sw128_desc(a0 + 32), sw128_desc(b0 + 0), ID, 1);      // Ih Rh
    mma_f16_pair(d_psi, sw128_desc(a0 + 0), sw128_desc(b0 + 32), IDN, 1);     // -Rh Ih
  } else {
    mma_f16_pair(d_phi, sw128_desc(a0 + 0), sw128_desc(b0 + 0), ID, acc);
    mma_f16_pair(d_phi, sw128_desc(a0 + 32), sw128_desc(b0 + 32), ID, 1);
    mma_f16_pair(d_phi, sw128_desc(a0 + 64), sw128_desc(b0 + 64), ID, 1);
    mma_f16_pair(d_phi, sw128_desc(a0 + 96), sw128_desc(b0 + 96), ID, 1);
    mma_f16_pair(d_psi, sw128_desc(a0 + 64), sw128_desc(b0 + 0), ID, acc);
    mma_f16_pair(d_psi, sw128_desc(a0 + 96), sw128_desc(b0 + 32), ID, 1);
    mma_f16_pair(d_psi, sw128_desc(a0 + 0), sw128_desc(b0 + 64), IDN, 1);
    mma_f16_pair(d_psi, sw128_desc(a0 + 32), sw128_desc(b0 + 96), IDN, 1);
  }
}

// The k-th work item of this cluster (runs of `chunk` list entries, as item_at).
__device__ __forceinline__ int pair_item_at(int k, int chunk) {
  const int ncl = (int)gridDim.x >> 1, cid = (int)blockIdx.x >> 1;
  return (k / chunk) * ncl * chunk + cid * chunk + (k % chunk);
}

template <int P>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(XP_THREADS, 1)
    k_xspec_pair(const XProblem* __restrict__ probs, const XItem* __restrict__ items, int nitems,
                 int* err, unsigned long long limit_ns, int inject, int chunk) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* stages = base;
  uint8_t* epi = base + XP_STAGES * XP_STAGE_BYTES;
  float* s2stage = (float*)(epi + XP_EPI_WARPS * XP_EPI_SLOTS * XP_BOX_BYTES);
  uint64_t* bars = (uint64_t*)(s2stage + XP_EPI_WARPS * TILE_N);
  // bars: full[S], empty[S], tfull[2], tempty[2]
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * XP_STAGES + 4);
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[XP_STAGES + s]); };
  auto tfull_bar = [&](int b) { return smem_u32(&bars[2 * XP_STAGES + b]); };
  auto tempty_bar = [&](int b) { return smem_u32(&bars[2 * XP_STAGES + 2 + b]); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();  // 0: issues the MMAs, 1: its peer
  const WaitCtl wc{err, limit_ns};
  // copies and MMAs finish in microseconds: abort-path drains need no more
  const unsigned long long drain_ns = limit_ns < 20000000ull ? limit_ns : 20000000ull;

  if (threadIdx.x == 0) {
    for (int s = 0; s < XP_STAGES; ++s) {
      mbar_init(full_bar(s), 1);    // even CTA: arm with both halves' bytes
      mbar_init(empty_bar(s), 1);   // one multicast commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);                  // one multicast commit
      mbar_init(tempty_bar(b), 2 * XP_EPI_WARPS);  // even CTA: epilogue warps of both CTAs
    }
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_slot), 512);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated in both
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[XP_STAGES];
      uint32_t armed_phase[XP_STAGES];
      for (int s = 0; s < XP_STAGES; ++s) armed[s] = 0, armed_phase[s] = 0;
      bool ok = (inject & 1) == 0;  // inject & 1: issue nothing (time-out test)
      bool issued = false;
      const uint64_t keep = l2_policy_evict_last();
      int cur_prob = -1, nch = 0, bn = 0;
      for (int k = 0; ok; ++k) {
        const int it = pair_item_at(k, chunk);
        if (it >= nitems) break;
        const XItem w = items[it];
        const XProblem* pr = probs + w.prob;
        if (w.prob != cur_prob) {
          cur_prob = w.prob;
          nch = pr->nchunks;
          bn = pr->bn;
        }
        {
          const int nx = pair_item_at(k + 1, chunk);
          if (nx < nitems) {
            const int np = items[nx].prob;
            if (np != w.prob) {
              tma_prefetch_desc(&probs[np].tmA);
              tma_prefetch_desc(&probs[np].tmB);
            }
          }
        }
        const int arow = ((int)w.ti * 2 + (int)rank) * TILE_M;
        const int brow = (int)w.tj * bn + (int)rank * (bn / 2);
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, wc)) { ok = false; break; }
          if (rank == 0) {
            mbar_arrive_expect_tx(full_bar(stage), 2u * (uint32_t)(TILE_M + bn / 2) * 128u);
            armed[stage] = 1;
            armed_phase[stage] = phase;
          }
          const uint32_t lead_full = map_shared_rank(full_bar(stage), 0);
          const uint32_t sa = smem_u32(stages + stage * XP_STAGE_BYTES);
          const int cx = (nch - 1 - c) * CHUNK_ELEMS;  // high frequencies first
          tma_load_2d_pair(sa, &pr->tmA, cx, arow, lead_full, keep);
          tma_load_2d_pair(sa + XP_A_BYTES, &pr->tmB, cx, brow, lead_full, keep);
          issued = true;
          if (++stage == XP_STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (rank == 0) {
        // both halves of every armed slot have landed before shared memory is released
        for (int s = 0; s < XP_STAGES; ++s)
          if (armed[s]) mbar_wait_cluster_drain(full_bar(s), armed_phase[s], drain_ns);
      } else if (!ok && issued) {
        // aborted: this CTA's copies signal the even CTA's barriers, which may
        // not have been armed for them; give copies in flight time to land
        const unsigned long long t0 = globaltimer();
        while (globaltimer() - t0 < 200000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0 && rank == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0, committed = 0;
      uint32_t last_bar = 0, last_parity = 0;
      bool ok = true;
      int cur_prob = -1, nch = 0;
      uint32_t id = 0, idn = 0;
      for (int k = 0; ok; ++k, ++lt) {
        const int it = pair_item_at(k, chunk);
        if (it >= nitems) break;
        const XItem w = items[it];
        if (w.prob != cur_prob) {
          cur_prob = w.prob;
          nch = probs[w.prob].nchunks;
          const int bn = probs[w.prob].bn;
          id = idesc_f16(2 * TILE_M, bn, P == 1, false);
          idn = idesc_f16(2 * TILE_M, bn, P == 1, true);
        }
        const int buf = lt & 1;
        const uint32_t tpar = (uint32_t)(lt >> 1) & 1u;
        if (!mbar_wait_cluster(tempty_bar(buf), tpar ^ 1u, wc)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_phi = tmem + (uint32_t)buf * 256u;
        const uint32_t d_psi = d_phi + 128u;
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(full_bar(stage), phase, wc)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stages + stage * XP_STAGE_BYTES);
          issue_chunk_mmas_pair<P>(d_phi, d_psi, a0, a0 + XP_A_BYTES, c > 0 ? 1u : 0u, id, idn);
          mma_commit_pair(empty_bar(stage));
          ++committed;
          last_bar = empty_bar(stage);
          last_parity = phase;
          if (++stage == XP_STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit_pair(tfull_bar(buf));
      }
      // every MMA has completed (so no operand read of either CTA's shared
      // memory and no TMEM write is pending) before the pair tears down
      if (committed > 0) mbar_wait_cluster_drain(last_bar, last_parity, drain_ns);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int half = ew >> 2;     // 0: Phi, 1: Psi
    const int q = warp & 3;       // TMEM lane quadrant
    const float sg = half ? -1.f : 1.f;
    const uint64_t stream_out = l2_policy_evict_first();
    uint8_t* ring = epi + ew * XP_EPI_SLOTS * XP_BOX_BYTES;
    float* s2w = s2stage + ew * TILE_N;
    int lt = 0;
    int slot = 0;
    int cur_prob = -1;
    const CUtensorMap* tm = nullptr;
    const float* s1p = nullptr;
    const float* s2p = nullptr;
    int n1 = 0, n2 = 0, bn = 0, pmirror = 0, orow_off = 0, upper = 0;
    float norm = 0.f;
    for (int k = 0;; ++k, ++lt) {
      const int it = pair_item_at(k, chunk);
      if (it >= nitems) break;
      const XItem w = items[it];
      if (w.prob != cur_prob) {
        cur_prob = w.prob;
        const XProblem* pr = probs + w.prob;
        tm = half ? &pr->tmPsi : &pr->tmPhi;
        s1p = pr->s1;
        s2p = pr->s2;
        n1 = pr->n1;
        n2 = pr->n2;
        bn = pr->bn;
        pmirror = pr->mirror;
        upper = pr->upper_only;
        orow_off = pr->out_row_tile0 * TILE_M;
        norm = pr->norm;
      }
      const int ti = (int)w.ti * 2 + (int)rank;    // this CTA's 128-row tile
      const int row0 = ti * TILE_M + q * 32;
      const int row = row0 + lane;
      const int colt = (int)w.tj * bn;
      const float rs = (row < n1) ? norm * __ldg(s1p + row) : 0.f;
      {
        const int c = colt + lane * 4;
        float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane * 4 < bn) {
          if (c + 3 < n2) {
            sv = __ldg((const float4*)(s2p + c));
          } else {
            if (c < n2) sv.x = __ldg(s2p + c);
            if (c + 1 < n2) sv.y = __ldg(s2p + c + 1);
            if (c + 2 < n2) sv.z = __ldg(s2p + c + 2);
          }
          *(float4*)(s2w + lane * 4) = sv;
        }
      }
      __syncwarp();
      const int buf = lt & 1;
      const uint32_t tpar = (uint32_t)(lt >> 1) & 1u;
      if (!mbar_wait(tfull_bar(buf), tpar, wc)) break;
      tc_fence_after();
      // a homo tile below the diagonal (odd CTA of item (a, 2a)) stores nothing
      const bool below = pmirror && ((int)w.tj < ti);
      const bool diag = pmirror && ((int)w.tj == ti);
      const bool rows_in = row0 < n1 && !below;
      const int nbox = bn / 32;
      for (int cc = diag ? q : 0; cc < nbox; ++cc) {
        const int col0 = colt + cc * 32;
        if (col0 >= n2) break;
        const bool mirror = pmirror && !upper && (!diag || cc > q);
        const bool tri = diag && cc == q;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256 + half * 128 + cc * 32),
                  v);
        if (!rows_in) continue;
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 s4 = *(const float4*)(s2w + cc * 32 + i);
          v[i] = v[i] * rs * s4.x;
          v[i + 1] = v[i + 1] * rs * s4.y;
          v[i + 2] = v[i + 2] * rs * s4.z;
          v[i + 3] = v[i + 3] * rs * s4.w;
        }
        const bool two = mirror && !tri;
        if (lane == 0) {
          if (two)
            bulk_wait_read<XP_EPI_SLOTS - 2>();
          else
            bulk_wait_read<XP_EPI_SLOTS - 1>();
        }
        __syncwarp();
        uint8_t* slot0 = ring + slot * XP_BOX_BYTES;
        uint8_t* slot1 = ring + ((slot + 1) % XP_EPI_SLOTS) * XP_BOX_BYTES;
        if (!tri) {
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4)
            *(float4*)(slot0 + sw128_off(lane, c4)) =
                make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
          if (mirror) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              *(float*)(slot1 + sw128_off(i, lane >> 2) + (lane & 3) * 4) = sg * v[i];
          }
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            if (c > lane) {
              *(float*)(slot0 + sw128_off(lane, c >> 2) + (c & 3) * 4) = v[c];
              *(float*)(slot0 + sw128_off(c, lane >> 2) + (lane & 3) * 4) = sg * v[c];
            } else if (c == lane) {
              *(float*)(slot0 + sw128_off(lane, c >> 2) + (c & 3) * 4) = half ? 0.f : v[c];
            }
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d_hint(tm, col0, row0 - orow_off, smem_u32(slot0), stream_out);
          bulk_commit();
          if (two) {
            tma_store_2d_hint(tm, row0, col0, smem_u32(slot1), stream_out);
            bulk_commit();
          }
        }
        slot = (slot + (two ? 2 : 1)) % XP_EPI_SLOTS;
      }
      // this CTA's half of the accumulators is consumed: tell the MMA issuer
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          mbar_arrive(tempty_bar(buf));
        else
          mbar_arrive_cluster(map_shared_rank(tempty_bar(buf), 0));
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  __syncwarp();
  tc_fence_before();
  cluster_sync_all();  // no MMA, copy or TMEM read of either CTA is pending
  tc_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem, 512);
}

cudaError_t init_xspec_pair_kernels() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_xspec_pair<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)XP_SMEM)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_xspec_pair<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)XP_SMEM);
}

// Clusters of the pair kernel that fit on the device at once (0 on failure).
int xspec_pair_max_clusters() {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(XP_THREADS, 1, 1);
  cfg.dynamicSmemBytes = XP_SMEM;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_xspec_pair<2>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_xspec_pair(const XProblem* d_probs, const XItem* d_items, int nitems,
                              int planes, int clusters, int* err, unsigned long long limit_ns,
                              cudaStream_t s, int inject, int chunk) {
  if (nitems <= 0) return cudaSuccess;
  if (chunk < 1) chunk = 1;
  if (clusters < 1) clusters = 1;
  if ((long)clusters * chunk > nitems) clusters = (nitems + chunk - 1) / chunk;
  const dim3 grid(2 * clusters);
  if (planes == 2)
    k_xspec_pair<2><<<grid, XP_THREADS, XP_SMEM, s>>>(d_probs, d_items, nitems, err, limit_ns,
                                                      inject, chunk);
  else
    k_xspec_pair<1><<<grid, XP_THREADS, XP_SMEM, s>>>(d_probs, d_items, nitems, err, limit_ns,
                                                      inject, chunk);
  return cudaGetLastError();
}

}  // namespace c2d
