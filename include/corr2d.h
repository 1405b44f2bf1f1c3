/*
 * corr2d.h -- C ABI of the GB300 (sm_103a) implementation of generalized
 * two-dimensional correlation analysis (Geitner et al., arXiv:1808.00685,
 * the corr2D R package).
 *
 * The library computes, for one or two stacks of m spectra sampled along a
 * shared perturbation axis, the synchronous (Phi) and asynchronous (Psi)
 * correlation spectra:
 *
 *   1. reference spectrum and dynamic spectra          (Eqs. ref, dynspec)
 *   2. DFT along the perturbation axis, half spectrum   (Eqs. disFT, symmeFT)
 *   3. Phi + i Psi = Norm sum_w w_w Y1 conj(Y2)          (Eq. disint2d, Sec. 4.2)
 *   4. optional scaling by (sigma1 sigma2)^-alpha       (Eqs. stdev, scalesyn,
 *                                                        scaleasyn)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Stacks are row-major FP32 matrices, m rows (row j = perturbation step t_j)
 *   by n columns (spectral variables nu), leading dimension ld >= n elements:
 *   the layout of the paper's input matrix (Sec. 3, "m perturbation values by
 *   rows and n spectral values by columns").
 * - Outputs Phi and Psi are row-major FP32 n1 x n2 matrices with leading
 *   dimension ldo (elements): row = nu1 of stack 1, column = nu2 of stack 2
 *   (Sec. 4.2: FT matrix built with byrow = TRUE over the columns of ft1).
 * - Every pointer argument that names device memory must point to memory of
 *   the context's device (cudaMalloc, torch CUDA tensors); host pointers are
 *   only accepted where a comment says "host".  The caller owns all input and
 *   output buffers; the library keeps no pointer after a call returns.
 * - Work is enqueued on the context's CUDA stream and the call returns before
 *   the GPU finishes.  Results are valid once the stream has been
 *   synchronised; corr2d_synchronize() does that and also reports device-side
 *   wait time-outs.
 * - The work of one context must not overlap on the GPU: its calls share the
 *   context's workspace (operand rows, descriptors) and the cross-spectrum
 *   kernel's work counters.  Calls on one stream are ordered; before switching
 *   streams with corr2d_set_stream, let the old stream's work finish (or order
 *   the streams with an event).  Use one context per concurrent stream.
 * - No function throws or aborts.  Each returns a corr2d_status; on failure
 *   corr2d_last_error() describes the first problem found.  Arguments are
 *   validated before anything is launched, so a rejected call leaves outputs
 *   untouched.
 * - Half-spectrum weights (Sec. 4.2 and Eq. symmeFT): omega = 0 .. K with
 *   K = floor((m-1)/2), weight 1 for omega = 0 and 2 otherwise; for even m the
 *   Nyquist bin m/2 is not used.
 */
#ifndef CORR2D_H
#define CORR2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CORR2D_OK = 0,
  CORR2D_EINVAL = 1,       /* bad shape, pointer, alignment or parameter */
  CORR2D_ENOMEM = 2,       /* device workspace could not be allocated */
  CORR2D_ECUDA = 3,        /* a CUDA runtime/driver call failed */
  CORR2D_ETIMEOUT = 4,     /* a device-side wait ran past its limit */
  CORR2D_EUNSUPPORTED = 5  /* valid request outside what this build supports */
} corr2d_status;

/* Arithmetic of the DFT and of the cross-spectrum contraction.  The
 * reference mean and the centering subtraction are computed in FP64 (FP32
 * precision) or in double-float FP32 arithmetic, an unevaluated (hi, lo) pair
 * accurate to about 2^-44 relative (tensor-core precisions); the centred
 * values are then rounded to FP32, and every product accumulates in FP32. */
typedef enum {
  CORR2D_PREC_FP32 = 0,  /* CUDA-core FP32 FMA (the plain GPU baseline) */
  CORR2D_PREC_SPLIT = 1, /* tcgen05 FP16 hi/lo split: hi*hi + hi*lo + lo*hi */
  CORR2D_PREC_BF16 = 2   /* tcgen05 plain BF16 operands */
} corr2d_precision;

typedef enum {
  CORR2D_REF_MEAN = 0, /* perturbation-mean reference per stack (Eq. ref) */
  CORR2D_REF_USER = 1  /* caller-supplied reference spectra ref1/ref2 */
} corr2d_ref_mode;

/* Homo correlation computes tiles with nu1-block <= nu2-block and writes each
 * tile and its mirror (Phi symmetric, Psi antisymmetric: Sec. 3 and Sec. 4.3).
 * This flag forces every tile to be computed instead. */
#define CORR2D_FLAG_NO_MIRROR 1u
/* Homo correlation: the tile tuner may pick full (unmirrored) tiles when they
 * are faster; the result then agrees with the mirrored one to rounding but is
 * not bit-for-bit symmetric.  This flag keeps the mirrored tiles, so Phi is
 * exactly symmetric and Psi exactly antisymmetric with a zero diagonal. */
#define CORR2D_FLAG_EXACT_SYMMETRY 2u
/* Hilbert-transform approach instead of the Fourier-transform one (Sec. 2,
 * Eqs. disHTsyn, disHT, HilbNoda, disHTasyn):
 *   Phi = Norm sum_j y~1(t_j) y~2(t_j),  Psi = Norm sum_j y~1(t_j) z~2(t_j),
 *   z~2 = N y~2 with the Hilbert-Noda matrix N_jk = 1/(pi (k - j)), N_jj = 0,
 * default Norm 1/(m - 1).  Tensor-core precisions only, m <= 256. */
#define CORR2D_FLAG_HILBERT 4u
/* Homo correlation: store only the upper triangle (nu2 >= nu1) of Phi and Psi,
 * the half that determines the rest (Phi symmetric, Psi antisymmetric); half
 * the output traffic.  Elements with nu2 < nu1 are unspecified: those within
 * 32 rows of the diagonal hold their mirrored values, the others are not
 * written.  Ignored for hetero problems. */
#define CORR2D_FLAG_UPPER_TRIANGLE 8u
/* Store Phi and Psi as BF16 (bfloat16: FP32's exponent range, 8 significant
 * bits) instead of FP32: half the output bytes of a store-bound computation
 * (the precision half of the output compaction that the symmetry facts of
 * Sec. 3 and Sec. 4.3 motivate).  Each element is the FP32 result rounded to
 * the nearest BF16 (ties to even): relative rounding error at most 2^-8
 * (3.9e-3; about 2e-3 relative Frobenius error on a whole map).  phi and psi
 * then point to 16-bit elements (passed as float* all the same), ldo counts
 * 16-bit elements and must be a multiple of 8, and phi/psi stay 16-byte
 * aligned.  Tensor-core precisions only (the FP32 path returns
 * CORR2D_EUNSUPPORTED), and not for corr2d_compute_host or the
 * allocation-free entry point, which return CORR2D_EUNSUPPORTED. */
#define CORR2D_FLAG_OUTPUT_BF16 16u

typedef struct {
  int ref_mode;       /* corr2d_ref_mode */
  const float* ref1;  /* device, n1 values; used when ref_mode == CORR2D_REF_USER */
  const float* ref2;  /* device, n2 values; hetero + user reference only */
  double norm;        /* <= 0 selects the default 1/(pi (m-1)) (Eq. disint2d) */
  double alpha;       /* 0: no scaling; 1: Pearson; 0.5: Pareto (Eqs. scale*) */
  int precision;      /* corr2d_precision */
  unsigned flags;     /* CORR2D_FLAG_*; other bits are rejected with CORR2D_EINVAL */
} corr2d_params;

typedef struct corr2d_ctx corr2d_ctx; /* opaque: device, stream, workspace, tuning cache */

/* Fill *p with the defaults: mean reference, default norm, alpha 0, SPLIT. */
corr2d_status corr2d_params_default(corr2d_params* p);

/* Create a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context; the caller releases it with corr2d_destroy. */
corr2d_status corr2d_create(corr2d_ctx** out, int device, void* cuda_stream);

/* Release a context and its device workspace (synchronises its stream). */
corr2d_status corr2d_destroy(corr2d_ctx* ctx);

/* Change the stream later calls enqueue on (the context's earlier work must
 * not overlap the later calls' on the GPU: see the conventions above). */
corr2d_status corr2d_set_stream(corr2d_ctx* ctx, void* cuda_stream);

/* Text of the last failure on this context ("" after success). NULL ctx
 * gives the last failure of corr2d_create. */
const char* corr2d_last_error(const corr2d_ctx* ctx);

/* Wait for the context's stream, then report ETIMEOUT if a kernel gave up on
 * a bounded wait since the previous call, or ECUDA on an asynchronous error. */
corr2d_status corr2d_synchronize(corr2d_ctx* ctx);

/*
 * Preprocessing onto a common, equally spaced spectral axis, then reference
 * subtraction (the interpolation mechanism of Sec. 4.2, applied along the
 * spectral axis, followed by Eq. dynspec).
 *   m       rows (perturbation steps) of y_raw, >= 1
 *   n_raw   raw points per row, >= 2
 *   x_raw   device, n_raw FP64 positions, strictly increasing and finite;
 *           a kernel checks this and the next corr2d_synchronize() returns
 *           EINVAL if it does not hold (the outputs are then meaningless)
 *   y_raw   device, m x n_raw FP32, leading dimension n_raw
 *   n_out   points of the target grid x_k = x_0 + k (x_last - x_0)/(n_out - 1),
 *           last point x_last exactly; >= 2
 *   y_out   device, m x n_out FP32 (linear interpolation, weights in FP64)
 *   ref     device, n_out FP32 reference spectrum, or NULL
 *   dyn_out device, m x n_out FP32 receiving y_out - ref, or NULL
 */
corr2d_status corr2d_preprocess(corr2d_ctx* ctx, int m, int n_raw, const double* x_raw,
                                const float* y_raw, int n_out, float* y_out, const float* ref,
                                float* dyn_out);

/*
 * Interpolation along the perturbation axis onto N equidistant perturbation
 * values (Sec. 4.2: the FT approach needs evenly spaced perturbation values;
 * the new values are seq(min(Time), max(Time), length.out = N) and every
 * spectral variable is evaluated there through an interpolating function of
 * its values over Time -- here the linear one, approxfun).
 *   m      perturbation steps of y, >= 2
 *   n      spectral variables, >= 1
 *   time   device, m FP64 perturbation values, strictly increasing and finite
 *          (checked by a kernel; corr2d_synchronize() reports EINVAL)
 *   y, ld  device, m x n FP32 stack, leading dimension ld >= n
 *   N      new number of perturbation steps, >= 2 (powers of two suit the FFT
 *          of the paper; any N works here)
 *   y_out  device, N x n FP32, leading dimension n
 */
corr2d_status corr2d_preprocess_perturbation(corr2d_ctx* ctx, int m, int n, const double* time,
                                             const float* y, int ld, int N, float* y_out);

/* Interpolating functions for corr2d_interpolate_perturbation (Sec. 4.2: the
 * package's Int argument; approxfun and its default, splinefun). */
typedef enum {
  CORR2D_INTERP_LINEAR = 0, /* approxfun: piecewise linear */
  CORR2D_INTERP_SPLINE = 1  /* splinefun with R's default method "fmm": the C^2
                               interpolating cubic spline whose third derivative on
                               the first / last interval is that of the cubic through
                               the first / last four points (3 points: the parabola,
                               2 points: the line) */
} corr2d_interp_method;

/*
 * corr2d_preprocess_perturbation with a choice of interpolating function
 * (same grid, arguments and errors; the linear method gives identical
 * results).  The spline keeps an FP64 workspace of m x n second derivatives
 * in the context (allocated on first use; ENOMEM if that fails).  An unknown
 * method is EINVAL.
 */
corr2d_status corr2d_interpolate_perturbation(corr2d_ctx* ctx, int method, int m, int n,
                                             const double* time, const float* y, int ld, int N,
                                             float* y_out);

/*
 * Synchronous and asynchronous correlation spectra of one problem.
 *   m          perturbation steps shared by both stacks, >= 2 (the
 *              normalisation divides by m - 1); tensor-core precisions
 *              accept m <= 512, FP32 accepts m <= 1600 (EUNSUPPORTED beyond)
 *   y1, ld1    device stack 1, m x n1, ld1 >= n1
 *   y2, ld2    device stack 2, m x n2, or y2 == NULL for homo correlation
 *              (stack 2 := stack 1, n2 and ld2 ignored)
 *   params     NULL for the defaults (corr2d_params_default)
 *   phi, psi   device outputs, n1 x n2 FP32, leading dimension ldo >= n2;
 *              tensor-core precisions need ldo % 4 == 0 and 16-byte aligned
 *              phi/psi (TMA stores), else EINVAL.  ldo % 32 == 0 with 128-byte
 *              aligned phi/psi is fastest: every stored row segment is then
 *              whole 128-byte lines (no partial-sector writes)
 *   sigma1_out, sigma2_out  device, n1 / n2 FP32 standard deviations
 *              (Eq. stdev with the chosen reference), or NULL
 * A spectral variable with sigma = 0 and alpha > 0 gets scale factor 0: its
 * row and column of Phi and Psi are 0 (instead of 0/0).
 * The first call for a shape (m, n1, n2, homo, precision, flags) tunes the
 * tile choice on the caller's buffers: each candidate (mirrored or full tiles,
 * tile order) runs three times and the fastest cross-spectrum launch wins;
 * later calls reuse it.  CORR2D_NO_TUNE=1 takes the first candidate;
 * CORR2D_TILES=bn:mirror:group:chunk[:seg] forces one choice (bn 64 or 128,
 * mirror 0/1, group 0 for row-major or G for G x G super-blocks, chunk >= 1
 * list entries per CTA at a time; seg > 0 runs the kernel that keeps the
 * stack-1 operand in TMEM, on row segments of seg 128 x 128 tiles, when the
 * problem has at most 8 frequency chunks).  The two launches of a call with at
 * most 4 GiB of output are programmatically dependent: the cross-spectrum
 * launch's setup overlaps the DFT launch's tail, and it reads the operand
 * rows only after the DFT launch has completed (CORR2D_PDL=off or =always
 * overrides the size rule; timing events recorded between the two launches,
 * see corr2d_set_profiling, serialise them).  Repeated calls with the same
 * buffers and arguments (up to four recent sets) launch from descriptors
 * already on the device.  The launches use the context's workspace, which a later call with
 * other shapes may reallocate: do not capture corr2d_compute into a CUDA
 * graph that outlives such calls.  To replay one problem with the least host
 * work, pass it to corr2d_batch as a batch of one: the batch records its own
 * graph over buffers of its own.
 */
corr2d_status corr2d_compute(corr2d_ctx* ctx, int m, int n1, const float* y1, int ld1, int n2,
                             const float* y2, int ld2, const corr2d_params* params, float* phi,
                             float* psi, long ldo, float* sigma1_out, float* sigma2_out);

/*
 * Reduced map for display (Sec. 4.3: plot_corr2din3d's `reduce` argument
 * resamples the matrix at the 1-based indices divisible by `reduce` with a
 * box kernel, i.e. it keeps every reduce-th row and column).  Computes
 *   phi_r[i][j] = Phi(nu1 = reduce (i + 1) - 1, nu2 = reduce (j + 1) - 1)
 * (and psi_r alike) for i < n1 / reduce, j < n2 / reduce, directly: only the
 * sampled variables are transformed and correlated, so the full n1 x n2 map
 * is never formed.  The reference, sigma and scaling of each sampled variable
 * are those of the full problem.  reduce >= 1; ldr >= n2 / reduce, a multiple
 * of 4; tensor-core precisions.  Other arguments as corr2d_compute.
 */
corr2d_status corr2d_compute_reduced(corr2d_ctx* ctx, int m, int n1, const float* y1, int ld1,
                                     int n2, const float* y2, int ld2,
                                     const corr2d_params* params, int reduce, float* phi_r,
                                     float* psi_r, long ldr);

/*
 * One row slab of the correlation: output rows nu1 in [row_begin, row_begin +
 * row_count) of Phi and Psi, written to phi/psi as a row_count x n2 matrix
 * (leading dimension ldo).  Slabs are independent -- this is how the work is
 * split over several GPUs (one context and slab per GPU, no communication):
 * every slab needs both whole stacks and recomputes their DFT, which is cheap
 * next to the n1 x n2 output.  row_begin must be a multiple of 128 (the tile
 * height); row_count >= 1 with row_begin + row_count <= n1.  Tensor-core
 * precisions; all tiles of the slab are computed (no mirroring).  Other
 * arguments as corr2d_compute.
 */
corr2d_status corr2d_compute_rows(corr2d_ctx* ctx, int m, int n1, const float* y1, int ld1,
                                  int n2, const float* y2, int ld2, const corr2d_params* params,
                                  int row_begin, int row_count, float* phi, float* psi,
                                  long ldo);

/*
 * One part of the output tiles, for splitting one problem over several GPUs
 * while keeping the homo mirror (the cross-spectrum of Eq. disint2d split by
 * output tiles; the paper's own parallel scheme, Sec. 4.2, splits the matrix
 * product over column blocks on CPU cores).  The problem's 128 x 128 output
 * tiles are listed in a fixed order -- homo problems: mirrored tiles (nu1-block
 * <= nu2-block, each writing itself and its transpose) in 64 x 64 super-blocks,
 * unless CORR2D_FLAG_NO_MIRROR; hetero problems: row-major -- and the list is cut
 * into `nparts` contiguous parts of about equal cost (a tile costs its stored
 * 128 x 128 blocks, two for an off-diagonal mirrored tile, plus one for its
 * tensor-core work).  This call computes part `part` (0 <= part < nparts): every
 * tile of the part and, for mirrored tiles, its mirrored block, written at their
 * places in the full n1 x n2 phi/psi (leading dimension ldo); nothing else of
 * phi/psi is written.  The parts of one problem cover every output exactly
 * once, so phi/psi of the nparts calls (one per GPU, each into its own buffer)
 * combine by taking each element from the part that wrote it
 * (corr2d_plan_part names the tiles).  Each call transforms both whole stacks
 * (cheap next to its share of the output); the parts need no communication.
 * The order is not tuned, so every process builds the same list.  Tensor-core
 * precisions; flags as corr2d_compute (UPPER_TRIANGLE drops the mirrored
 * blocks).  Other arguments and errors as corr2d_compute; a part with no tiles
 * (nparts larger than the tile count) writes nothing.
 */
corr2d_status corr2d_compute_part(corr2d_ctx* ctx, int m, int n1, const float* y1, int ld1,
                                  int n2, const float* y2, int ld2, const corr2d_params* params,
                                  int part, int nparts, float* phi, float* psi, long ldo);

/*
 * Host-only companion of corr2d_compute_part (no GPU, no context): the tiles of
 * part `part` of `nparts` of an n1 x n2 problem (homo != 0: n2 is ignored and
 * the mirrored list is used unless `flags` holds CORR2D_FLAG_NO_MIRROR), in list
 * order.  *count receives the number of tiles; when tiles is not NULL it
 * receives 2 * count ints (ti, tj): tile (ti, tj) covers rows 128 ti .. and
 * columns 128 tj .. of the map, and a mirrored tile with ti != tj also the
 * transposed block.  EINVAL for a bad shape or part, or cap < count (tiles
 * not NULL); corr2d_last_error(NULL) describes the failure.
 */
corr2d_status corr2d_plan_part(int n1, int n2, int homo, unsigned flags, int part, int nparts,
                               int* tiles, int cap, int* count);

/*
 * Same computation with every buffer in HOST memory: the library copies the
 * stacks to its device workspace, computes, and copies Phi and Psi back in
 * row slabs so that copies overlap the kernels.  Blocks until the results are
 * in phi/psi.  y2 == NULL selects homo correlation.  Pinned host memory gives
 * the fastest copies; pageable memory works.
 */
corr2d_status corr2d_compute_host(corr2d_ctx* ctx, int m, int n1, const float* y1, int n2,
                                  const float* y2, const corr2d_params* params, float* phi,
                                  float* psi, long ldo);

/* One problem of a batch (device pointers, same conventions as
 * corr2d_compute; y2 == NULL selects homo). */
typedef struct {
  int m, n1, n2;
  const float* y1;
  const float* y2;
  float* phi;
  float* psi;
  long ldo;
} corr2d_problem;

/*
 * Many independent correlations of uneven m, n1, n2: one batched DFT launch
 * and one persistent cross-spectrum launch over a cost-ordered tile list, with
 * per-problem tile shapes from the tuner; the launches are captured once in a
 * CUDA graph per batch layout and replayed, the cross-spectrum launch
 * programmatically dependent on the DFT launch (its setup overlaps the DFT's
 * last wave; while profiling is on, the two run as separate graphs with the
 * timing events between them).  host_problems is a host array of
 * `count` descriptors.  shared_params (NULL = defaults) applies to every
 * problem; its ref_mode must be CORR2D_REF_MEAN and its precision a
 * tensor-core precision.  A call whose problem list and parameters equal the
 * previous call's (same shapes and pointers) replays the recorded graph
 * without querying the pointers again: the buffers it names must still be
 * allocated.
 */
corr2d_status corr2d_batch(corr2d_ctx* ctx, int count, const corr2d_problem* host_problems,
                           const corr2d_params* shared_params);

/*
 * Host-only (no GPU, no context; the paper runs one problem at a time and has
 * no counterpart): which problems of a batch go to part `part` of `nparts`,
 * for running one batch over several GPUs -- one process per GPU, each calling
 * corr2d_batch on its part, no communication.  Problem i has m[i] perturbation
 * steps, n1[i] spectral variables in stack 1 and n2[i] in stack 2 (n2[i] == 0:
 * homo, stack 2 = stack 1).  Its cost, in units of one output pair, is
 *   n1 n2 + 3 m (n1 + n2)      (homo: n1 n1 + 3 m n1),
 * the stored pair against the DFT work per input element (about 3 pairs' worth
 * each: the batch of 512 ragged problems took 1.3 ps per output pair in its
 * cross-spectrum launch and 4.1 ps per input element in its DFT launch on one
 * GB300).  Problems are taken by decreasing cost (ties: lower index first) and
 * each goes to the part with the smallest total so far (ties: lower part), so
 * the largest part exceeds the mean by less than the largest single cost.  The
 * assignment depends on the shapes alone, so every process computes the same
 * one.  *count receives the number of problems of the part; indices, when not
 * NULL, receives their indices in increasing order (room for cap ints).
 * EINVAL for count < 0, NULL arrays with count > 0, a bad part, a problem with
 * m < 2, n1 < 1 or n2 < 0, or cap < *count; corr2d_last_error(NULL) describes
 * the failure.
 */
corr2d_status corr2d_plan_batch_part(int count, const int* m, const int* n1, const int* n2,
                                     int part, int nparts, int* indices, int cap, int* count_out);

/* Per-kernel timing of the last corr2d_compute / corr2d_batch call on this
 * context, from CUDA events recorded on the context's stream around each
 * kernel while profiling is on (the paper profiles its own steps the same
 * way, Sec. 4.3).  corr2d_get_timings waits for those events.  The events
 * serialise the two launches, which otherwise overlap (programmatic dependent
 * launch), so a call with profiling on can take a few microseconds longer.
 *   prep_ms   reference, centering, sigma and DFT kernel(s)
 *   xspec_ms  cross-spectrum kernel
 * Returns EINVAL when profiling is off or nothing was recorded yet. */
corr2d_status corr2d_set_profiling(corr2d_ctx* ctx, int on);
corr2d_status corr2d_get_timings(corr2d_ctx* ctx, float* prep_ms, float* xspec_ms);

/* Library introspection (the paper has no counterpart): which cross-spectrum
 * kernel the last corr2d_compute / corr2d_batch call on this context launched
 * (CORR2D_XSPEC_* below), and how many CTA pairs the device runs at once (0:
 * the CTA-pair kernel is unavailable).  Either output may be NULL (host
 * ints otherwise); EINVAL for a NULL context.  The tuner times the single-CTA
 * kernel's tile shapes and orders, and for upper-triangle output of a homo
 * problem also the kernel that holds the stack-1 operand in TMEM (up to 8
 * frequency chunks: split m <= 256, BF16 m <= 512); the environment variable
 * CORR2D_XSPEC=pair makes it use the CTA-pair kernel instead, =ta the TMEM
 * one (the single-CTA kernel beyond 8 chunks), =any lets it time every kind,
 * =single holds it to the single-CTA kernel. */
enum { CORR2D_XSPEC_NONE = 0, CORR2D_XSPEC_TC = 1, CORR2D_XSPEC_TC_PAIR = 2,
       CORR2D_XSPEC_FP32 = 3, CORR2D_XSPEC_TC_TA = 4 };
corr2d_status corr2d_get_kernel_info(corr2d_ctx* ctx, int* last_xspec, int* pair_clusters);

/*
 * Allocation-free variant of corr2d_compute.  The paper has no counterpart:
 * this entry point exists for callers of this library that must not allocate
 * GPU memory -- a program whose memory planner already owns the whole device,
 * a plugin whose host framework forbids hidden allocations, a latency-critical
 * loop that cannot pay the implicit synchronisation of cudaMalloc/cudaFree,
 * or code without a library context (corr2d_create allocates).
 *
 * It takes no context.  The caller passes the device, a stream (cudaStream_t,
 * NULL = legacy default stream), the stacks and the Phi/Psi outputs exactly as
 * for corr2d_compute (device memory of `device`; ldo % 4 == 0; 16-byte
 * aligned outputs).  All intermediates live in one static device array of
 * CORR2D_NOALLOC_SCRATCH_BYTES that the library declares; every GPU that
 * loads the library keeps that array until the process exits.  The call
 * allocates no device memory: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *
 * - Precisions: CORR2D_PREC_SPLIT and CORR2D_PREC_BF16 (FP32: EUNSUPPORTED).
 * - Flags: CORR2D_FLAG_HILBERT selects the Hilbert-transform approach as in
 *   corr2d_compute (m <= 256, default norm 1/(m - 1)); CORR2D_FLAG_UPPER_TRIANGLE
 *   stores only the upper triangle of a homo problem as in corr2d_compute;
 *   CORR2D_FLAG_NO_MIRROR computes every tile.  Without NO_MIRROR a homo
 *   problem always runs on mirrored tiles (no tuner here), so its Phi is
 *   exactly symmetric and Psi exactly antisymmetric with a zero diagonal --
 *   what CORR2D_FLAG_EXACT_SYMMETRY asks of corr2d_compute.
 *   CORR2D_FLAG_OUTPUT_BF16 is not available here (CORR2D_EUNSUPPORTED).
 * - Size limit: a problem needs about rows * rowbytes + twiddles, with rows =
 *   n1 for a homo problem (its two operands share one row set; the Hilbert
 *   variant keeps two: 2 n1) and n1 + n2 for a hetero one, rowbytes = 1 KB for
 *   m <= 257 in SPLIT (2 KB for m <= 513; the Hilbert variant: 2 m bytes
 *   rounded up to 128); anything larger than the array returns EUNSUPPORTED
 *   with the byte counts in `msg`, before any work is enqueued.  Example: homo
 *   n = 30000 at m = 256 in SPLIT fits, homo n = 40000 does not.
 * - The first call on a device does a one-time set-up there: it looks up the
 *   array's device address with cudaGetSymbolAddress, which also loads the
 *   library module that holds the array, so the array's device memory is
 *   committed on that device by this first call (and kept until the process
 *   exits), and it sets kernel attributes.  Make that first call at start-up:
 *   before a memory planner claims the device, and before any stream capture
 *   begins.
 * - The call is synchronous: it returns after the results are in phi/psi
 *   (it waits for `cuda_stream`) and reports CORR2D_ETIMEOUT if a device-side
 *   wait ran out (limit 2 s, or CORR2D_WAIT_LIMIT_MS milliseconds).
 * - All calls share the one array and it keeps the last call's contents.
 *   Calls that overlap on the GPU (from several host threads or streams) race
 *   on it; serialise them.
 * - msg (nullable, msg_len bytes) receives the reason for a failure.
 */
#define CORR2D_NOALLOC_SCRATCH_BYTES (32u << 20)
corr2d_status corr2d_compute_noalloc(int device, void* cuda_stream, int m, int n1,
                                     const float* y1, int ld1, int n2, const float* y2, int ld2,
                                     const corr2d_params* params, float* phi, float* psi,
                                     long ldo, char* msg, size_t msg_len);

/* Measured FP32 FMA throughput of the context's device in TFLOP/s (the
 * paper has no counterpart: it is the ceiling against which the CUDA-core
 * FP32 path, CORR2D_PREC_FP32, is reported).  A probe kernel of independent
 * FMA chains (4 CTAs of 256 threads per SM) runs four times on the context's
 * stream, the first as a warm-up; *tflops receives the best of the other three
 * (2 flop per FMA).  Synchronous; allocates and frees a small device buffer.
 * EINVAL for a NULL argument, ECUDA if the launch fails. */
corr2d_status corr2d_measure_fp32_peak(corr2d_ctx* ctx, double* tflops);

/* Library version string. */
const char* corr2d_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CORR2D_H */
