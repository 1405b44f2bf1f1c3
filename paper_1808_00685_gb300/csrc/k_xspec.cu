// Complex cross-spectrum on tcgen05 tensor cores (Eq. disint2d with the
// half-spectrum weights of Sec. 4.2):
//   Phi(nu1, nu2) = norm s1[nu1] s2[nu2] sum_w w (Re1 Re2 + Im1 Im2)
//   Psi(nu1, nu2) = norm s1[nu1] s2[nu2] sum_w w (Im1 Re2 - Re1 Im2)
// The weight w is already in the operand rows (each carries sqrt(w); a homo
// problem's two operands are one row set); s1, s2 carry sigma^-alpha and the
// power-of-two operand scaling.
//
// Persistent, warp-specialised kernel, one CTA per SM, 320 threads:
//   warp 0      TMA producer: operand chunks of stack 1 (128 rows) and
//               stack 2 (bn rows) into a shared-memory ring of 4 or 5
//               stages (the tuner's choice: 5 helps full tiles, 4 mirrored)
//   warp 1      MMA issuer (one thread): per chunk, Phi and Psi accumulate in
//               TMEM (128 lanes x bn columns each); the Re*Im term of Psi
//               uses the instruction's negate-A bit.  With FP16 hi/lo planes
//               the products are hi*hi + hi*lo + lo*hi.
//   warps 2..9  epilogue, two warps per TMEM lane quadrant (one for Phi, one
//               for Psi): TMEM -> registers, scale, 128-byte-swizzled staging
//               box, TMA store of 32x32 FP32 boxes (BF16 boxes of 64-byte
//               rows with CORR2D_FLAG_OUTPUT_BF16).  For homo problems the
//               mirrored box is stored too (Phi symmetric, Psi antisymmetric),
//               so only tiles with ti <= tj are computed.  Each warp stages
//               its boxes in a ring of XS_EPI_SLOTS slots, one bulk group per
//               box, and waits only for the group that last read the slot it
//               is about to overwrite.
// TMEM holds two accumulator sets (2 x 256 columns): the MMAs of tile i+1
// run while the epilogue of tile i streams its stores.
//
// Work distribution: each CTA's first run of `chunk` list entries is its own
// (blockIdx.x); later runs come from a counter in global memory (atomicAdd),
// so CTAs that finish early take more tiles and all finish within about one
// tile of each other.  The producer reads each run one run ahead and publishes
// every tile to the MMA thread and the epilogue warps through a ring of
// XS_SCHED shared-memory slots (sfull / sempty barriers); a slot holding
// prob < 0 ends the loop.  The last CTA to finish resets the counter for the
// next launch (graph replays included).
#include "internal.h"
#include "ptx.cuh"

namespace c2d {

constexpr int XS_STAGES = 5;  // ring slots allocated; a launch uses 4 or 5 of them
constexpr int XS_STAGE_BYTES = 2 * TILE_M * 128;  // A chunk + B chunk (bn <= 128 rows)
constexpr int XS_EPI_WARPS = 8;
constexpr int XS_BOX_BYTES = 32 * 32 * 4;
constexpr int XS_EPI_SLOTS = 2;                   // staging boxes per epilogue warp (ring)
static_assert(XS_EPI_SLOTS >= 2, "a box and its mirror need two staging slots");
constexpr int XS_THREADS = 64 + 32 * XS_EPI_WARPS;
constexpr int XS_SCHED = 8;  // tile-schedule ring slots (> the tiles the producer runs ahead)
static_assert((XS_SCHED & (XS_SCHED - 1)) == 0 && XS_SCHED > XS_STAGES,
              "the schedule ring must outrun the operand ring");
// barriers (full/empty per stage, tfull/tempty per TMEM buffer, sfull/sempty
// per schedule slot), the TMEM base address, then the schedule ring
constexpr int XS_NBARS = 2 * XS_STAGES + 4 + 2 * XS_SCHED;
constexpr size_t XS_CTRL = 512;
static_assert(XS_NBARS * 8 + 8 + (XS_SCHED + 1) * sizeof(XItem) <= XS_CTRL, "control block");
constexpr size_t XS_SMEM = 1024 + (size_t)XS_STAGES * XS_STAGE_BYTES +
                           (size_t)XS_EPI_WARPS * XS_EPI_SLOTS * XS_BOX_BYTES +
                           (size_t)2 * TILE_N * 4 + XS_CTRL;

// Accumulation order.  Tensor-core FP32 accumulation truncates each addition,
// so its error grows with the number of MMAs added while the accumulator is
// large.  Chunks therefore run from the highest frequencies to the lowest
// (spectral energy sits at low frequencies), and within a chunk the small
// hi*lo / lo*hi products go before hi*hi: on smooth spectra this halves the
// error (m = 512: 1.1e-5 -> 5e-6 relative).
template <int P>
__device__ __forceinline__ void issue_chunk_mmas(uint32_t d_phi, uint32_t d_psi, uint32_t a0,
                                                 uint32_t b0, uint32_t acc, uint32_t ID,
                                                 uint32_t IDN) {
  // ID / IDN: M = 128, N = bn, FP16 (split planes) or BF16, IDN with negate-A.
  if (P == 2) {
    // chunk bytes: Re_hi @0, Im_hi @32, Re_lo @64, Im_lo @96 (16 frequencies each)
    mma_f16(d_phi, sw128_desc(a0 + 0), sw128_desc(b0 + 64), ID, acc);    // Rh Rl
    mma_f16(d_phi, sw128_desc(a0 + 32), sw128_desc(b0 + 96), ID, 1);     // Ih Il
    mma_f16(d_phi, sw128_desc(a0 + 64), sw128_desc(b0 + 0), ID, 1);      // Rl Rh
    mma_f16(d_phi, sw128_desc(a0 + 96), sw128_desc(b0 + 32), ID, 1);     // Il Ih
    mma_f16(d_phi, sw128_desc(a0 + 0), sw128_desc(b0 + 0), ID, 1);       // Rh Rh
    mma_f16(d_phi, sw128_desc(a0 + 32), sw128_desc(b0 + 32), ID, 1);     // Ih Ih
    mma_f16(d_psi, sw128_desc(a0 + 32), sw128_desc(b0 + 64), ID, acc);   // Ih Rl
    mma_f16(d_psi, sw128_desc(a0 + 0), sw128_desc(b0 + 96), IDN, 1);     // -Rh Il
    mma_f16(d_psi, sw128_desc(a0 + 96), sw128_desc(b0 + 0), ID, 1);      // Il Rh
    mma_f16(d_psi, sw128_desc(a0 + 64), sw128_desc(b0 + 32), IDN, 1);    // -Rl Ih
    mma_f16(d_psi, sw128_desc(a0 + 32), sw128_desc(b0 + 0), ID, 1);      // Ih Rh
    mma_f16(d_psi, sw128_desc(a0 + 0), sw128_desc(b0 + 32), IDN, 1);     // -Rh Ih
  } else {
    // chunk bytes: Re @0 (two K=16 steps: 0, 32), Im @64 (64, 96)
    mma_f16(d_phi, sw128_desc(a0 + 0), sw128_desc(b0 + 0), ID, acc);
    mma_f16(d_phi, sw128_desc(a0 + 32), sw128_desc(b0 + 32), ID, 1);
    mma_f16(d_phi, sw128_desc(a0 + 64), sw128_desc(b0 + 64), ID, 1);
    mma_f16(d_phi, sw128_desc(a0 + 96), sw128_desc(b0 + 96), ID, 1);
    mma_f16(d_psi, sw128_desc(a0 + 64), sw128_desc(b0 + 0), ID, acc);
    mma_f16(d_psi, sw128_desc(a0 + 96), sw128_desc(b0 + 32), ID, 1);
    mma_f16(d_psi, sw128_desc(a0 + 0), sw128_desc(b0 + 64), IDN, 1);
    mma_f16(d_psi, sw128_desc(a0 + 32), sw128_desc(b0 + 96), IDN, 1);
  }
}

// Runs of `chunk` consecutive list entries: the first run of a CTA starts at
// blockIdx.x * chunk, the later ones at gridDim.x * chunk + (the counter's old
// value), the counter advancing by chunk per run.  chunk > 1 keeps a CTA on
// one problem for several tiles in a batch of small problems.
__device__ __forceinline__ int next_run(int* ctr, int chunk) {
  return (int)gridDim.x * chunk + atomicAdd(ctr, chunk);
}

// A tile published in the schedule ring (read after its sfull barrier).
__device__ __forceinline__ XItem read_sched(const XItem* p) {
  const volatile XItem* v = p;
  XItem w;
  w.prob = v->prob;
  w.ti = v->ti;
  w.tj = v->tj;
  return w;
}

template <int P>
__global__ void __launch_bounds__(XS_THREADS, 1)
    k_xspec_tc(const XProblem* __restrict__ plist, const XItem* __restrict__ items, int nitems,
               int* err, unsigned long long limit_ns, int inject, int chunk, int nst,
               int nprobs, const __grid_constant__ XProblem p0) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* stages = base;
  uint8_t* epi = base + XS_STAGES * XS_STAGE_BYTES;
  float* s2stage = (float*)(epi + XS_EPI_WARPS * XS_EPI_SLOTS * XS_BOX_BYTES);
  uint64_t* bars = (uint64_t*)(s2stage + 2 * TILE_N);
  // bars: full[S], empty[S], tfull[2], tempty[2], sfull[R], sempty[R]
  uint32_t* tmem_slot = (uint32_t*)(bars + XS_NBARS);
  XItem* sched = (XItem*)(tmem_slot + 2);  // schedule ring (8-byte aligned)
  XItem* first_sm = sched + XS_SCHED;      // this CTA's first tile
  // A launch with one problem takes it (tensor maps included) from the kernel
  // parameters, which arrive with the launch; the descriptor list in global
  // memory may have been evicted from L2, and the first TMA copies would wait
  // for its DRAM reads.
  const bool one = nprobs == 1;
  const XProblem* probs = one ? &p0 : plist;
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[XS_STAGES + s]); };
  auto tfull_bar = [&](int b) { return smem_u32(&bars[2 * XS_STAGES + b]); };
  auto tempty_bar = [&](int b) { return smem_u32(&bars[2 * XS_STAGES + 2 + b]); };
  auto sfull_bar = [&](int r) { return smem_u32(&bars[2 * XS_STAGES + 4 + r]); };
  auto sempty_bar = [&](int r) { return smem_u32(&bars[2 * XS_STAGES + 4 + XS_SCHED + r]); };
  int* ctr = err + XS_COUNTER_WORD;  // [0] next run, [1] CTAs finished

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WaitCtl wc{err, limit_ns};

  // The first tile is known now: an epilogue warp fetches it and warms the TMA
  // unit's descriptor cache while thread 0 sets up the barriers and warp 1 TMEM.
  const int first_it = (int)blockIdx.x * chunk;
  if (threadIdx.x == 64) {
    XItem f{-1, 0, 0};
    if (first_it < nitems) {
      f = items[first_it];
      if (!one) {
        tma_prefetch_desc(&probs[f.prob].tmA);
        tma_prefetch_desc(&probs[f.prob].tmB);
        tma_prefetch_desc(&probs[f.prob].tmPhi);
        tma_prefetch_desc(&probs[f.prob].tmPsi);
      }
    }
    *first_sm = f;
  }
  if (threadIdx.x == 96 && one) {  // in parallel with the list read above
    tma_prefetch_desc(&probs[0].tmA);
    tma_prefetch_desc(&probs[0].tmB);
    tma_prefetch_desc(&probs[0].tmPhi);
    tma_prefetch_desc(&probs[0].tmPsi);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < XS_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), XS_EPI_WARPS);
    }
    for (int r = 0; r < XS_SCHED; ++r) {
      mbar_init(sfull_bar(r), 1);
      mbar_init(sempty_bar(r), 1 + XS_EPI_WARPS);  // the MMA thread and every epilogue warp
    }
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
  // Launched behind the DFT kernel with programmatic serialization, the setup
  // above overlaps its tail; operand rows, scales and the work counter are
  // touched only after it has completed.
  griddep_wait();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[XS_STAGES];
      uint32_t armed_phase[XS_STAGES];
      for (int s = 0; s < XS_STAGES; ++s) armed[s] = 0, armed_phase[s] = 0;
      // inject & 1: a host-requested fault for tests -- the producer issues
      // nothing, so the MMA and epilogue waits run out and report a time-out.
      bool ok = (inject & 1) == 0;
      const uint64_t keep = l2_policy_evict_last();  // operand rows are re-read by every CTA
      int cur_prob = -1, nch = 0, bn = 0;
      // current run [run, run + chunk) and the next one, read a run ahead
      int run = first_it, pos = 0;
      int ahead = (ok && run < nitems) ? next_run(ctr, chunk) : nitems;
      XItem w = *first_sm;
      for (int lt = 0; ok; ++lt) {
        // this tile: the next entry of the current run, else of the next run
        int it = run + pos;
        if (pos == chunk || it >= nitems) {
          run = ahead;
          pos = 0;
          it = run;
          if (run < nitems) ahead = next_run(ctr, chunk);
        }
        const bool done = it >= nitems;
        if (!done && lt > 0) w = items[it];
        ++pos;
        // publish it (prob < 0 ends the other roles' loops)
        const int ss = lt & (XS_SCHED - 1);
        if (!mbar_wait(sempty_bar(ss), ((uint32_t)(lt / XS_SCHED) & 1u) ^ 1u, wc)) break;
        sched[ss] = done ? XItem{-1, 0, 0} : w;
        mbar_arrive(sfull_bar(ss));
        if (done) break;
        const XProblem* pr = probs + w.prob;
        if (w.prob != cur_prob) {
          cur_prob = w.prob;
          nch = pr->nchunks;
          bn = pr->bn;
        }
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, wc)) { ok = false; break; }
          mbar_arrive_expect_tx(full_bar(stage), (uint32_t)(TILE_M + bn) * 128u);
          armed[stage] = 1;
          armed_phase[stage] = phase;
          const uint32_t sa = smem_u32(stages + stage * XS_STAGE_BYTES);
          const int cx = (nch - 1 - c) * CHUNK_ELEMS;  // high frequencies first
          tma_load_2d_hint(sa, &pr->tmA, cx, (int)w.ti * TILE_M, full_bar(stage), keep);
          tma_load_2d_hint(sa + TILE_M * 128, &pr->tmB, cx, (int)w.tj * bn, full_bar(stage), keep);
          if (++stage == nst) { stage = 0; phase ^= 1u; }
        }
        // Warm the TMA unit's descriptor cache for the next problem.  This
        // comes after the tile's loads: at the first tile the next run is the
        // result of the work-counter atomic, and waiting for it (and for the
        // list entry it names) before the first loads delayed them ~1.5 us.
        if (ok) {
          const int nx = (pos < chunk && it + 1 < nitems) ? it + 1 : ahead;
          if (nx < nitems) {
            const int np = items[nx].prob;
            if (np != w.prob) {
              tma_prefetch_desc(&probs[np].tmA);
              tma_prefetch_desc(&probs[np].tmB);
            }
          }
        }
      }
      // every load this thread started has landed before shared memory is released
      for (int s = 0; s < XS_STAGES; ++s)
        if (armed[s]) mbar_wait_drain(full_bar(s), armed_phase[s], limit_ns);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0, committed = 0;
      uint32_t last_bar = 0, last_parity = 0;
      bool ok = true;
      int cur_prob = -1, nch = 0;
      uint32_t id = 0, idn = 0;
      for (;; ++lt) {
        const int ss = lt & (XS_SCHED - 1);
        if (!mbar_wait(sfull_bar(ss), (uint32_t)(lt / XS_SCHED) & 1u, wc)) { ok = false; break; }
        const XItem w = read_sched(sched + ss);
        mbar_arrive(sempty_bar(ss));
        if (w.prob < 0) break;
        if (w.prob != cur_prob) {
          cur_prob = w.prob;
          nch = probs[w.prob].nchunks;
          const int bn = probs[w.prob].bn;
          id = idesc_f16(128, bn, P == 1, false);
          idn = idesc_f16(128, bn, P == 1, true);
        }
        const int buf = lt & 1;
        const uint32_t tpar = (uint32_t)(lt >> 1) & 1u;
        if (!mbar_wait(tempty_bar(buf), tpar ^ 1u, wc)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_phi = tmem + (uint32_t)buf * 256u;
        const uint32_t d_psi = d_phi + 128u;
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(full_bar(stage), phase, wc)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stages + stage * XS_STAGE_BYTES);
          issue_chunk_mmas<P>(d_phi, d_psi, a0, a0 + TILE_M * 128, c > 0 ? 1u : 0u, id, idn);
          mma_commit(empty_bar(stage));
          ++committed;
          last_bar = empty_bar(stage);
          last_parity = phase;
          if (++stage == nst) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull_bar(buf));
      }
      // all MMAs this thread issued complete before TMEM is released
      if (committed > 0) mbar_wait_drain(last_bar, last_parity, limit_ns);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;      // epilogue warp 0..7
    const int half = ew >> 2;     // 0: Phi, 1: Psi
    const int q = warp & 3;       // TMEM lane quadrant this warp may access
    const float sg = half ? -1.f : 1.f;
    const uint64_t stream_out = l2_policy_evict_first();  // written once, never re-read here
    uint8_t* ring = epi + ew * XS_EPI_SLOTS * XS_BOX_BYTES;
    int lt = 0;
    int slot = 0;  // next slot of this warp's staging ring
    int cur_prob = -1;
    const CUtensorMap* tm = nullptr;
    const float* s1p = nullptr;
    const float* s2p = nullptr;
    int n1 = 0, n2 = 0, bn = 0, pmirror = 0, orow_off = 0, upper = 0, obf = 0;
    float norm = 0.f;
    for (;; ++lt) {
      const int ss = lt & (XS_SCHED - 1);
      if (!mbar_wait(sfull_bar(ss), (uint32_t)(lt / XS_SCHED) & 1u, wc)) break;
      const XItem w = read_sched(sched + ss);
      __syncwarp();
      if (lane == 0) mbar_arrive(sempty_bar(ss));
      if (w.prob < 0) break;
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
        obf = pr->out_bf16;
        orow_off = pr->out_row_tile0 * TILE_M;
        norm = pr->norm;
      }
      const int row0 = (int)w.ti * TILE_M + q * 32;  // first nu1 of this warp's rows
      const int row = row0 + lane;
      const int colt = (int)w.tj * bn;                // first nu2 of the tile
      // tile constants while the MMAs finish: row scale, column scales in smem
      const float rs = (row < n1) ? norm * __ldg(s1p + row) : 0.f;
      // column scales of the tile, loaded while the MMAs finish; stored into
      // the tile-parity half of the buffer all epilogue warps share once the
      // accumulators are ready (every warp has then left the tile two back,
      // the last one to use that half; all warps store the same values)
      float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
      {
        const int c = colt + lane * 4;
        if (lane * 4 < bn) {
          if (c + 3 < n2) {
            sv = __ldg((const float4*)(s2p + c));
          } else {
            if (c < n2) sv.x = __ldg(s2p + c);
            if (c + 1 < n2) sv.y = __ldg(s2p + c + 1);
            if (c + 2 < n2) sv.z = __ldg(s2p + c + 2);
          }
        }
      }
      __syncwarp();
      const int buf = lt & 1;
      const uint32_t tpar = (uint32_t)(lt >> 1) & 1u;
      if (!mbar_wait(tfull_bar(buf), tpar, wc)) break;
      tc_fence_after();
      float* s2w = s2stage + (lt & 1) * TILE_N;
      if (lane * 4 < bn) *(float4*)(s2w + lane * 4) = sv;
      __syncwarp();
      // Homo tiles off the diagonal store each box and its mirror.  On a
      // diagonal tile, box (q, cc) with cc > q stores itself and its mirror,
      // cc == q stores its upper triangle and mirrors it into the lower one,
      // cc < q is left to box (cc, q): the output is then exactly symmetric
      // (Phi) / antisymmetric with zero diagonal (Psi).
      const bool diag = pmirror && (w.ti == w.tj);
      const bool rows_in = row0 < n1;
      const int nbox = bn / 32;
      for (int cc = diag ? q : 0; cc < nbox; ++cc) {
        const int col0 = colt + cc * 32;
        if (col0 >= n2) break;  // warp-uniform
        // upper-triangle output: no mirrored boxes (diagonal boxes stay whole)
        const bool mirror = pmirror && !upper && (!diag || cc > q);
        const bool tri = diag && cc == q;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256 + half * 128 + cc * 32),
                  v);
        if (!rows_in) continue;  // rows beyond n1 (their mirror columns are beyond n2 too)
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 s4 = *(const float4*)(s2w + cc * 32 + i);
          v[i] = v[i] * rs * s4.x;
          v[i + 1] = v[i + 1] * rs * s4.y;
          v[i + 2] = v[i + 2] * rs * s4.z;
          v[i + 3] = v[i + 3] * rs * s4.w;
        }
        // The slots about to be written were last read by the group committed
        // XS_EPI_SLOTS (second slot: XS_EPI_SLOTS - 1) groups ago; lane 0
        // committed them, so lane 0 waits.
        const bool two = mirror && !tri;
        if (lane == 0) {
          if (two)
            bulk_wait_read<XS_EPI_SLOTS - 2>();
          else
            bulk_wait_read<XS_EPI_SLOTS - 1>();
        }
        __syncwarp();
        uint8_t* slot0 = ring + slot * XS_BOX_BYTES;
        uint8_t* slot1 = ring + ((slot + 1) % XS_EPI_SLOTS) * XS_BOX_BYTES;
        if (obf) {
          // BF16 output: the same FP32 values rounded to nearest (ties to
          // even), boxes of 32 rows x 64 bytes with the 64-byte swizzle
          if (!tri) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t w[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
                w[e] = *reinterpret_cast<const uint32_t*>(&b2);
              }
              *(uint4*)(slot0 + sw64_off(lane, q)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            if (mirror) {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                *(__nv_bfloat16*)(slot1 + sw64_off(i, lane >> 3) + (lane & 7) * 2) =
                    __float2bfloat16_rn(sg * v[i]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (c > lane) {
                *(__nv_bfloat16*)(slot0 + sw64_off(lane, c >> 3) + (c & 7) * 2) =
                    __float2bfloat16_rn(v[c]);
                *(__nv_bfloat16*)(slot0 + sw64_off(c, lane >> 3) + (lane & 7) * 2) =
                    __float2bfloat16_rn(sg * v[c]);
              } else if (c == lane) {
                *(__nv_bfloat16*)(slot0 + sw64_off(lane, c >> 3) + (c & 7) * 2) =
                    __float2bfloat16_rn(half ? 0.f : v[c]);
              }
            }
          }
        } else if (!tri) {
          // box (rows row0.., cols col0..): row = lane, 8 swizzled 16-byte chunks
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4)
            *(float4*)(slot0 + sw128_off(lane, c4)) =
                make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
          if (mirror) {
            // transposed box (rows col0.., cols row0..): element (i, lane)
#pragma unroll
            for (int i = 0; i < 32; ++i)
              *(float*)(slot1 + sw128_off(i, lane >> 2) + (lane & 3) * 4) = sg * v[i];
          }
        } else {
          // element (lane, c) for c >= lane, its mirror (c, lane) for c > lane
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
        slot = (slot + (two ? 2 : 1)) % XS_EPI_SLOTS;
      }
      // this tile's accumulators are consumed: hand the TMEM buffer back
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(buf));
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 512);
  // every role of this CTA has stopped taking runs: count the CTA as finished;
  // the last one resets the counters for the next launch on this stream
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1) == (int)gridDim.x - 1) {
      ctr[0] = 0;
      ctr[1] = 0;
      __threadfence();
    }
  }
}

static_assert(XS_SMEM <= (size_t)kMaxDynSmem, "cross-spectrum shared memory exceeds the limit");

cudaError_t init_xspec_kernels() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_xspec_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XS_SMEM)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_xspec_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XS_SMEM);
}

cudaError_t launch_xspec_tc(const XProblem* d_probs, const XItem* d_items, int nitems, int planes,
                            int grid, int* err, unsigned long long limit_ns, cudaStream_t s,
                            int inject, int chunk, int stages, int nprobs, bool pdl,
                            const XProblem* h_p0) {
  static const XProblem kNone{};
  if (nitems <= 0) return cudaSuccess;
  if (chunk < 1) chunk = 1;
  if (stages != XS_STAGES) stages = 4;
  if ((long)grid * chunk > nitems) grid = (nitems + chunk - 1) / chunk;
  // a one-problem launch needs the problem itself as a parameter
  if (nprobs == 1 && !h_p0) nprobs = 0;
  const XProblem* p0 = (nprobs == 1) ? h_p0 : &kNone;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(XS_THREADS);
  cfg.dynamicSmemBytes = XS_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  if (planes == 2)
    return cudaLaunchKernelEx(&cfg, k_xspec_tc<2>, d_probs, d_items, nitems, err, limit_ns, inject,
                              chunk, stages, nprobs, *p0);
  return cudaLaunchKernelEx(&cfg, k_xspec_tc<1>, d_probs, d_items, nitems, err, limit_ns, inject,
                            chunk, stages, nprobs, *p0);
}

}  // namespace c2d
