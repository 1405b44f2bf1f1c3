// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace c2d {

// ----------------------------------------------------------------------------
// Operand layout of the tensor-core path.
//
// Each spectral variable nu gets one operand row of `rowlen` 16-bit elements
// holding its half spectrum Y(nu, omega), omega = 0..K'p-1 (K'p = K+1 rounded
// up to a multiple of g), scaled by a power of two 2^E(nu) that puts the row
// maximum in [2^13, 2^14).  The row is a sequence of 128-byte chunks, each
// covering g frequencies:
//   SPLIT (FP16 hi/lo, g = 16): [Re_hi(16) Im_hi(16) Re_lo(16) Im_lo(16)]
//   BF16  (g = 32):             [Re(32) Im(32)]
// with hi = fp16(v), lo = fp16(v - hi).  Both operands carry the square root
// of the half-spectrum weight w (1 for omega = 0, else 2), so a stack-1 row
// times a stack-2 row carries w, and a homo problem uses one row set for both
// operands.  A chunk is exactly one 128-byte swizzle row, so one TMA
// box of 64 elements x rows lands in shared memory ready for tcgen05.mma.
// ----------------------------------------------------------------------------
constexpr int CHUNK_ELEMS = 64;   // 16-bit elements per 128-byte chunk
constexpr int TILE_M = 128;       // nu1 rows per MMA tile (TMEM lanes)
constexpr int TILE_N = 128;       // nu2 columns per tile (Phi and Psi each)
constexpr int PREP_ROWS = 128;    // spectral variables per DFT tile
constexpr int MAX_M_TC = 512;     // largest m accepted by the tensor-core path
constexpr int kMaxDynSmem = 232448;  // dynamic shared memory per CTA (227 KB)
constexpr int MAX_M_FP32 = 1600;     // FP32 DFT keeps m x 32 centred values in smem

inline int freq_count(int m) { return (m - 1) / 2 + 1; }          // K + 1
inline int freq_group(int planes) { return planes == 2 ? 16 : 32; }
inline int freq_padded(int m, int planes) {
  int g = freq_group(planes);
  return (freq_count(m) + g - 1) / g * g;
}
inline int chunks_for(int m, int planes) { return freq_padded(m, planes) / freq_group(planes); }

// Contraction applied along the perturbation axis by the prep kernel.  The
// operand row of a variable holds two blocks of components ("Re", "Im"):
//   XF_DFT      Re = cos, Im = -sin of 2 pi omega j / m, omega = 0..K  (Eq. disFT)
//   XF_HT_A     Re = y~ (identity), Im = 0                     (stack 1 of the
//   XF_HT_B     Re = y~ (identity), Im = -N y~ (Eq. HilbNoda)   Hilbert variant)
// With these rows the cross-spectrum kernel's Phi = <Re1,Re2> + <Im1,Im2> and
// Psi = <Im1,Re2> - <Re1,Im2> become Eqs. disHTsyn and disHTasyn.
enum TransformKind : int { XF_DFT = 0, XF_HT_A = 1, XF_HT_B = 2 };
constexpr int MAX_M_HT = 256;     // the Hilbert variant keeps 2 m components in TMEM
inline int comps_padded(int m, int planes, bool hilbert) {
  const int g = freq_group(planes);
  return hilbert ? (m + g - 1) / g * g : freq_padded(m, planes);
}
// Table of the contraction matrix of `kind` for m steps, pre-swizzled for
// tcgen05 (rows = components, 64 steps per 128-byte row, one block per
// 64-step chunk and plane).  Returns its size; fills `out` when non-null.
size_t make_transform(int m, int planes, int kind, uint8_t* out);

// One stack's DFT job (tensor-core prep kernel).
struct PrepJob {
  const float* y;          // m x n, leading dimension ld
  const float* ref;        // user reference (nullable -> perturbation mean)
  uint16_t* outA;          // operand rows of stack 1 (nullable)
  uint16_t* outB;          // operand rows of stack 2 (nullable; may equal outA)
  float* scale;            // n: sigma^-alpha * 2^-E(nu)
  float* sigma_out;        // n (nullable)
  const uint8_t* wtab;     // pre-swizzled twiddles of this m (see make_twiddles)
  long ld;
  int m, n;
  int kp;                  // K'p
  int jchunks;             // ceil(m / 64)
  int rowlen;              // operand row length in elements
  int plain_weights;       // 1: weight 1 everywhere (Hilbert variant); 0: rows
                           // carry sqrt of the half-spectrum weights 1 / 2
  int cstride_m1;          // column stride of y (and ref) minus 1: variable nu is
                           // column nu * (cstride_m1 + 1) (decimated preview)
  int pad2_;
  double alpha;
};

// One work item of the prep kernel: (job, 128-variable tile).
struct PrepItem {
  int job;
  int tile;
};

// One correlation problem of the cross-spectrum kernel.  Tensor maps first:
// they must be 64-byte aligned.
struct alignas(128) XProblem {
  CUtensorMap tmA;     // operand rows of stack 1: {rowlen, n1}, box {64, 128}
  CUtensorMap tmB;     // operand rows of stack 2: {rowlen, n2}, box {64, bn}
  CUtensorMap tmPhi;   // output {n2, n1}, box {32, 32}, 128-byte swizzle
  CUtensorMap tmPsi;
  const float* s1;     // scale vectors (stack 1 / stack 2)
  const float* s2;
  float norm;
  int n1, n2;
  int nchunks;         // operand chunks per row
  int mirror;          // 1: homo tile with its mirror written too (bn == 128)
  int bn;              // nu2 columns per tile: 64 or 128
  int out_row_tile0;   // output rows are shifted up by out_row_tile0 * 128
  int upper_only;      // 1: mirrored problem storing only nu2 >= nu1 (no mirror boxes)
  int out_bf16;        // 1: Phi and Psi stored as BF16 (tmPhi/tmPsi: BF16, 64-byte swizzle)
  int pad_[1];
};

// One tile of the cross-spectrum kernel: problem index and tile coordinates.
struct XItem {
  int prob;
  uint16_t ti, tj;
};

// Host side: build the pre-swizzled twiddle table for m (FP64 angles with
// the integer part reduced modulo m, split into 16-bit planes).  Returns the
// table size in bytes; writes it into `out` when non-null.
size_t make_twiddles(int m, int planes, uint8_t* out);

// One-time kernel attribute setup (dynamic shared memory limits); called when
// a context is created, so that later launches may be captured in graphs.
cudaError_t init_prep_kernels();
cudaError_t init_xspec_kernels();

// Launchers (return cudaGetLastError()).
cudaError_t launch_prep_tc(const PrepJob* d_jobs, const PrepItem* d_items, int nitems, int planes,
                           int max_kp, int* err, unsigned long long limit_ns, cudaStream_t s);
// inject & 1 makes the producer issue nothing (host-requested fault for the
// time-out test); 0 in normal operation.  Each CTA takes runs of `chunk`
// consecutive work items; `stages` (4 or 5) operand stages are in flight.
// Programmatic dependent launch of the cross-spectrum kernel behind the DFT
// kernel: its launch latency and setup then overlap the DFT's tail.  Measured
// on GB300 per call without per-launch events (which serialise the two):
// homo m = 64 n = 4096 42.0-42.6 -> 39.9-41.0 us, hetero m = 128 8192 x 2048
// 48.5-49.8 -> 45.1 us, homo m = 256 n = 8192 125.9 -> 122.5-122.9 us,
// n = 16384 374.7-375.6 -> 371.5-372.7 us, but n = 32768 (8.6 GB of output)
// 1.39-1.45 -> 1.42-1.53 ms, that long launch running at lower SM clocks.  By
// default it is used up to this much output.
constexpr double kPdlMaxOutBytes = 4.0 * 1024.0 * 1024.0 * 1024.0;

cudaError_t launch_xspec_tc(const XProblem* d_probs, const XItem* d_items, int nitems,
                            int planes, int grid, int* err, unsigned long long limit_ns,
                            cudaStream_t s, int inject = 0, int chunk = 1, int stages = 4,
                            int nprobs = 0, bool pdl = false, const XProblem* h_p0 = nullptr);
// nprobs: problems in the list (0: unknown); with nprobs == 1, h_p0 is a host
// copy of d_probs[0], passed as a kernel parameter.  pdl: launch with
// programmatic stream serialization, only when the DFT kernel is the launch
// just ahead of it in the stream (its setup then overlaps the DFT's tail).

// Row segment of the TMEM-operand cross-spectrum kernel: tiles (ti, tj0 ..
// tj0 + ntj - 1) of 128 x 128 outputs that share their stack-1 rows.
struct XSeg {
  int prob;
  uint16_t ti, tj0, ntj, pad_;
};
// Cross-spectrum with the stack-1 operand in TMEM (k_xspec_ta): segments
// instead of tiles, stack-2 tensor maps with 64-row boxes, problems with at
// most 8 operand chunks (m <= 256 in split precision).
cudaError_t init_xspec_ta_kernels();
cudaError_t launch_xspec_ta(const XProblem* d_probs, const XSeg* d_segs, int nsegs, int planes,
                            int grid, int* err, unsigned long long limit_ns, cudaStream_t s,
                            int inject = 0);
constexpr int TA_MAX_CHUNKS = 8;

// Cross-spectrum on CTA pairs (clusters of two, tcgen05 cta_group::2): items
// are 256 x 128 tiles (XItem.ti = index of a 256-row pair of tiles), stack-2
// tensor maps have 64-row boxes.  `clusters` pairs run persistently.
cudaError_t init_xspec_pair_kernels();
int xspec_pair_max_clusters();
cudaError_t launch_xspec_pair(const XProblem* d_probs, const XItem* d_items, int nitems,
                              int planes, int clusters, int* err, unsigned long long limit_ns,
                              cudaStream_t s, int inject = 0, int chunk = 1);

// FP32 CUDA-core path.
struct SimtPrepJob {
  const float* y;
  const float* ref;
  float* yr;      // kp1 x n, frequency-major (A: unweighted; nullable)
  float* yi;
  float* yrw;     // weighted copies (nullable when not needed)
  float* yiw;
  float* scale;   // n: sigma^-alpha
  float* sigma_out;
  const float* tw;  // 2*m: cos(2 pi r/m), sin(2 pi r/m)
  long ld;
  int m, n, kp1;
  int ldp;        // plane row pitch (>= n, a multiple of 32: 16-byte aligned rows)
  double alpha;
};
cudaError_t launch_prep_simt(const SimtPrepJob& job, cudaStream_t s);
// Planes: kp1 rows of pitch ldp1 (stack 1) / ldp2 (stack 2), multiples of 4.
cudaError_t launch_xspec_simt(int kp1, int n1, int n2, int ldp1, int ldp2, const float* yr1,
                              const float* yi1, const float* yr2w, const float* yi2w,
                              const float* s1, const float* s2, float norm, float* phi,
                              float* psi, long ldo, bool mirror, cudaStream_t s);

// FP32 FMA throughput probe (measured ceiling of the FP32 path): `blocks` CTAs
// of 256 threads, `iters` iterations of independent FMA chains; the flops one
// launch performs.  `out` (blocks x 256 floats) is never written in practice.
cudaError_t launch_fma_probe(float* out, int blocks, int iters, cudaStream_t s);
double fma_probe_flops(int blocks, int iters);

// Preprocessing.
cudaError_t launch_interp(int m, int n_raw, const double* x, const float* y, int n_out,
                          float* out, const float* ref, float* dyn, int* err, cudaStream_t s);
cudaError_t launch_interp_t(int m, int n, const double* t, const float* y, long ld, int N,
                            float* out, int* err, cudaStream_t s);
size_t spline_workspace_bytes(int m, int n, int N);
cudaError_t launch_spline_t(int m, int n, const double* t, const float* y, long ld, int N,
                            float* out, void* ws, int* err, cudaStream_t s);

// Codes of the device error word: a bounded wait ran out, or the
// preprocessing axis check failed.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_AXIS = 2 };

// The error word `err` every launcher takes is the first int of a 256-byte,
// zero-initialised block; ints XS_COUNTER_WORD and XS_COUNTER_WORD + 1 of that
// block are the work counters of k_xspec_tc (next run, CTAs finished).  They
// are zero between launches: the kernel's last CTA resets them, so launches on
// one stream (and graph replays) may share the block.
constexpr int XS_COUNTER_WORD = 32;
constexpr int ERR_BLOCK_BYTES = 256;

}  // namespace c2d
