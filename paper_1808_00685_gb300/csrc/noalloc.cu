// corr2d_compute_noalloc: the correlation of corr2d_compute for callers that
// must not allocate GPU memory.
//
// Who needs this: code that runs where a device allocation is not allowed or
// not wanted -- a process whose memory planner has already handed out the
// whole GPU, a plugin inside a host framework that owns every allocation, a
// real-time loop that cannot afford the implicit device synchronisation of
// cudaMalloc/cudaFree, or a caller that has no library context (creating one
// allocates).  The caller still provides the stacks and the Phi/Psi outputs;
// every intermediate (operand rows, scale vectors, contraction tables,
// descriptors, error word) lives in one fixed array of device memory that the
// library declares at file scope.
//
// When the array is committed: the library is built without relocatable
// device code, so this file is a module of its own that holds only the array,
// and CUDA loads modules lazily.  The array's memory is therefore committed on
// a device by the first call there (its cudaGetSymbolAddress loads the
// module), not when the library is loaded, and stays committed until the
// process exits.  A caller whose memory planner will own the device should
// make that first call at start-up, before the planner claims the memory.
//
// The kernels are the ones corr2d_compute uses (k_prep_tc, k_xspec_tc); only
// where their scratch lives differs.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "corr2d.h"
#include "internal.h"

namespace {

using namespace c2d;

constexpr size_t kScratchBytes = (size_t)CORR2D_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr double kPi = 3.14159265358979323846264338327950288;

// The shared scratch.  Device code could name it directly; host code must use
// the address cudaGetSymbolAddress returns for the current device (the name
// itself is only a host-side stand-in).
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                             const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                             const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct DeviceSetup {
  bool done = false;
  uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sm_count = 0;
};

std::mutex g_setup_lock;
DeviceSetup g_setup[kMaxDevices];
EncodeFn g_encode = nullptr;

corr2d_status say(char* msg, size_t len, corr2d_status st, const char* fmt, ...) {
  if (msg && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, len, fmt, ap);
    va_end(ap);
  }
  return st;
}

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev;
  return a.type == cudaMemoryTypeManaged;
}

// One-time set-up on the current device: the scratch address, kernel
// attributes and the tensor-map encoder.  Runs on the first call per device.
corr2d_status setup_device(int dev, DeviceSetup** out, char* msg, size_t len) {
  std::lock_guard<std::mutex> lk(g_setup_lock);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return say(msg, len, CORR2D_ECUDA, "cudaGetSymbolAddress of the scratch failed: %s",
                 cudaGetErrorString(e));
    if ((e = init_prep_kernels()) != cudaSuccess || (e = init_xspec_kernels()) != cudaSuccess)
      return say(msg, len, CORR2D_ECUDA, "kernel attribute setup failed: %s",
                 cudaGetErrorString(e));
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                           cudaEnableDefault, &q) != cudaSuccess || !fn)
        return say(msg, len, CORR2D_ECUDA, "cuTensorMapEncodeTiled unavailable");
      g_encode = (EncodeFn)fn;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
      return say(msg, len, CORR2D_ECUDA, "cannot query device %d", dev);
    if (prop.major != 10 || prop.minor != 3)
      return say(msg, len, CORR2D_EUNSUPPORTED, "device %d is sm_%d%d, not sm_103a", dev,
                 prop.major, prop.minor);
    s.scratch = (uint8_t*)p;
    s.sm_count = prop.multiProcessorCount;
    s.done = true;
  }
  *out = &s;
  return CORR2D_OK;
}

bool encode(CUtensorMap* tm, CUtensorMapDataType dt, void* base, uint64_t inner, uint64_t rows,
            uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_rows) {
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_encode(tm, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B,
                  dt == CU_TENSOR_MAP_DATA_TYPE_FLOAT32 ? CU_TENSOR_MAP_L2_PROMOTION_NONE
                                                        : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct RestoreDevice {
  int prev = -1;
  explicit RestoreDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~RestoreDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" corr2d_status corr2d_compute_noalloc(int device, void* cuda_stream, int m, int n1,
                                                const float* y1, int ld1, int n2,
                                                const float* y2, int ld2,
                                                const corr2d_params* params, float* phi,
                                                float* psi, long ldo, char* msg,
                                                size_t msg_len) {
  if (msg && msg_len) msg[0] = '\0';
  corr2d_params p;
  if (params) {
    p = *params;
  } else {
    memset(&p, 0, sizeof p);
    p.ref_mode = CORR2D_REF_MEAN;
    p.precision = CORR2D_PREC_SPLIT;
  }
  const bool homo = (y2 == nullptr);
  if (homo) { n2 = n1; ld2 = ld1; }
  // ---- arguments (nothing is launched unless all of them are acceptable)
  if (m < 2) return say(msg, msg_len, CORR2D_EINVAL, "m = %d: at least 2 perturbation steps", m);
  if (m > MAX_M_TC) return say(msg, msg_len, CORR2D_EUNSUPPORTED, "m = %d > %d", m, MAX_M_TC);
  if (n1 < 1 || n2 < 1 || !y1 || ld1 < n1 || ld2 < n2 || !phi || !psi || ldo < n2)
    return say(msg, msg_len, CORR2D_EINVAL, "bad shapes or NULL buffers");
  if (ldo % 4 != 0 || ((uintptr_t)phi & 15) || ((uintptr_t)psi & 15))
    return say(msg, msg_len, CORR2D_EINVAL, "TMA stores need ldo %% 4 == 0 and 16-byte aligned outputs");
  if (p.precision != CORR2D_PREC_SPLIT && p.precision != CORR2D_PREC_BF16)
    return say(msg, msg_len, CORR2D_EUNSUPPORTED, "only the tensor-core precisions run without allocation");
  if (p.ref_mode != CORR2D_REF_MEAN && p.ref_mode != CORR2D_REF_USER)
    return say(msg, msg_len, CORR2D_EINVAL, "bad ref_mode");
  if (p.ref_mode == CORR2D_REF_USER && (!p.ref1 || (!homo && !p.ref2)))
    return say(msg, msg_len, CORR2D_EINVAL, "user reference mode needs ref1 (and ref2)");
  if (!std::isfinite(p.norm) || !(p.alpha >= 0.0) || !std::isfinite(p.alpha))
    return say(msg, msg_len, CORR2D_EINVAL, "norm and alpha must be finite, alpha >= 0");
  if (p.flags & CORR2D_FLAG_OUTPUT_BF16)
    return say(msg, msg_len, CORR2D_EUNSUPPORTED, "BF16 output needs corr2d_compute");
  if (p.flags & ~(CORR2D_FLAG_NO_MIRROR | CORR2D_FLAG_EXACT_SYMMETRY | CORR2D_FLAG_HILBERT |
                  CORR2D_FLAG_UPPER_TRIANGLE))
    return say(msg, msg_len, CORR2D_EINVAL, "unknown flag bits");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
      device >= kMaxDevices) {
    cudaGetLastError();
    return say(msg, msg_len, CORR2D_EINVAL, "device %d is not available", device);
  }

  const bool hilbert = (p.flags & CORR2D_FLAG_HILBERT) != 0;
  if (hilbert && m > MAX_M_HT)
    return say(msg, msg_len, CORR2D_EUNSUPPORTED,
               "the Hilbert-transform variant supports m <= %d", MAX_M_HT);

  // ---- scratch plan: everything must fit the static array
  // Operand rows: stack 1 and stack 2; a homo FT problem uses one row set for
  // both operands (each row carries the square root of the half-spectrum
  // weight), the Hilbert variant's two operands come from different matrices
  // ([I; 0] and [I; -N]) and keep two.
  const int planes = p.precision == CORR2D_PREC_SPLIT ? 2 : 1;
  const int kp = comps_padded(m, planes, hilbert);
  const int nch = kp / freq_group(planes);
  const int rowlen = nch * CHUNK_ELEMS;
  const bool shared_rows = homo && !hilbert;
  const size_t tw_bytes = make_transform(m, planes, hilbert ? XF_HT_A : XF_DFT, nullptr);
  const size_t tw2_bytes = hilbert ? make_transform(m, planes, XF_HT_B, nullptr) : 0;
  const int nt1 = (n1 + TILE_M - 1) / TILE_M, nt2 = (n2 + TILE_N - 1) / TILE_N;
  const bool mirror = homo && !(p.flags & CORR2D_FLAG_NO_MIRROR);
  const long nitems = mirror ? (long)nt1 * (nt1 + 1) / 2 : (long)nt1 * nt2;
  const int njobs = shared_rows ? 1 : 2;
  const int npitems = nt1 + (shared_rows ? 0 : (n2 + PREP_ROWS - 1) / PREP_ROWS);
  size_t off = ERR_BLOCK_BYTES;  // error word and the cross-spectrum work counters
  const size_t off_tw = off; off = up(off + tw_bytes, 1024);
  const size_t off_tw2 = off; off = up(off + tw2_bytes, 1024);
  const size_t off_a = off;  off = up(off + (size_t)n1 * rowlen * 2, 1024);
  const size_t off_b = off;  off = up(off + (shared_rows ? 0 : (size_t)n2 * rowlen * 2), 1024);
  const size_t off_s1 = off; off = up(off + (size_t)n1 * 4, 256);
  const size_t off_s2 = off; off = up(off + (shared_rows ? 0 : (size_t)n2 * 4), 256);
  const size_t off_jobs = off; off = up(off + njobs * sizeof(PrepJob), 128);
  const size_t off_pit = off; off = up(off + npitems * sizeof(PrepItem), 128);
  const size_t off_prob = off; off = up(off + sizeof(XProblem), 128);
  const size_t off_xit = off; off = up(off + nitems * sizeof(XItem), 128);
  if (off > kScratchBytes)
    return say(msg, msg_len, CORR2D_EUNSUPPORTED,
               "problem needs %zu bytes of scratch; the allocation-free entry point has %zu "
               "(use corr2d_compute)", off, kScratchBytes);
  if (nt1 > 65535 || nt2 > 65535) return say(msg, msg_len, CORR2D_EUNSUPPORTED, "n too large");

  RestoreDevice rd(device);
  for (const void* q : {(const void*)y1, (const void*)y2, (const void*)phi, (const void*)psi,
                        (const void*)(p.ref_mode == CORR2D_REF_USER ? p.ref1 : nullptr),
                        (const void*)(p.ref_mode == CORR2D_REF_USER && !homo ? p.ref2 : nullptr)})
    if (q && !on_device(q, device))
      return say(msg, msg_len, CORR2D_EINVAL, "buffers must be device memory of device %d", device);
  DeviceSetup* ds = nullptr;
  corr2d_status st = setup_device(device, &ds, msg, msg_len);
  if (st != CORR2D_OK) return st;
  uint8_t* S = ds->scratch;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // ---- host-side descriptors
  std::vector<uint8_t> tw(tw_bytes), tw2(tw2_bytes);
  make_transform(m, planes, hilbert ? XF_HT_A : XF_DFT, tw.data());
  if (hilbert) make_transform(m, planes, XF_HT_B, tw2.data());
  uint16_t* opA = (uint16_t*)(S + off_a);
  uint16_t* opB = shared_rows ? opA : (uint16_t*)(S + off_b);
  float* s1 = (float*)(S + off_s1);
  // each row's scale carries its operand's power-of-two rescale, which differs
  // between the Hilbert variant's two matrices: a scale array per operand
  float* s2 = shared_rows ? s1 : (float*)(S + off_s2);
  const float* ref1 = p.ref_mode == CORR2D_REF_USER ? p.ref1 : nullptr;
  const float* ref2 = p.ref_mode == CORR2D_REF_USER ? (homo ? p.ref1 : p.ref2) : nullptr;
  std::vector<PrepJob> jobs(njobs);
  std::vector<PrepItem> pit;
  for (int jn = 0; jn < njobs; ++jn) {
    // job 0: stack 1 -> opA (and opB when the rows are shared); job 1: the
    // stack-2 operand (stack 1 again for a homo Hilbert problem) -> opB
    PrepJob& j = jobs[jn];
    memset(&j, 0, sizeof j);
    const bool second = jn == 1;
    const bool from_y2 = second && !homo;
    j.y = from_y2 ? y2 : y1;
    j.ld = from_y2 ? ld2 : ld1;
    j.n = from_y2 ? n2 : n1;
    j.ref = from_y2 ? ref2 : ref1;
    j.outA = second ? nullptr : opA;
    j.outB = second ? opB : nullptr;  // job 0 with shared rows: opB == opA
    j.scale = second ? s2 : s1;
    j.sigma_out = nullptr;
    j.wtab = S + ((second && hilbert) ? off_tw2 : off_tw);
    j.m = m;
    j.kp = kp;
    j.jchunks = (m + 63) / 64;
    j.rowlen = rowlen;
    j.alpha = p.alpha;
    j.plain_weights = hilbert ? 1 : 0;
    for (int t = 0; t < (j.n + PREP_ROWS - 1) / PREP_ROWS; ++t) pit.push_back(PrepItem{jn, t});
  }
  XProblem xp;
  memset(&xp, 0, sizeof xp);
  const CUtensorMapDataType odt =
      planes == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (!encode(&xp.tmA, odt, opA, rowlen, n1, (uint64_t)rowlen * 2, CHUNK_ELEMS, TILE_M) ||
      !encode(&xp.tmB, odt, opB, rowlen, n2, (uint64_t)rowlen * 2, CHUNK_ELEMS, TILE_N) ||
      !encode(&xp.tmPhi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, phi, n2, n1, (uint64_t)ldo * 4, 32, 32) ||
      !encode(&xp.tmPsi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, psi, n2, n1, (uint64_t)ldo * 4, 32, 32))
    return say(msg, msg_len, CORR2D_ECUDA, "tensor map encoding failed");
  xp.s1 = s1;
  xp.s2 = s2;
  // Norm: the caller's, else 1/(pi (m-1)) (Eq. disint2d) or, for the Hilbert
  // approach, 1/(m-1) (Eqs. disHTsyn, disHTasyn)
  xp.norm = (float)(p.norm > 0.0 ? p.norm
                                 : hilbert ? 1.0 / (double)(m - 1)
                                           : 1.0 / (kPi * (double)(m - 1)));
  xp.n1 = n1;
  xp.n2 = n2;
  xp.nchunks = nch;
  xp.mirror = mirror ? 1 : 0;
  xp.bn = TILE_N;
  xp.out_row_tile0 = 0;
  xp.upper_only = (mirror && (p.flags & CORR2D_FLAG_UPPER_TRIANGLE)) ? 1 : 0;
  std::vector<XItem> items;
  items.reserve(nitems);
  for (int ti = 0; ti < nt1; ++ti)
    for (int tj = mirror ? ti : 0; tj < nt2; ++tj) items.push_back(XItem{0, (uint16_t)ti, (uint16_t)tj});

  // ---- enqueue: the error word and the work counters start at zero; the rest
  // is written before it is read
  cudaError_t e = cudaMemsetAsync(S, 0, ERR_BLOCK_BYTES, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + off_tw, tw.data(), tw_bytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && hilbert)
    e = cudaMemcpyAsync(S + off_tw2, tw2.data(), tw2_bytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + off_jobs, jobs.data(), njobs * sizeof(PrepJob), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + off_pit, pit.data(), pit.size() * sizeof(PrepItem), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + off_prob, &xp, sizeof xp, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + off_xit, items.data(), items.size() * sizeof(XItem), cudaMemcpyHostToDevice, stream);
  int* err = (int*)S;
  // bounded device-side waits: 2 s, or CORR2D_WAIT_LIMIT_MS as for contexts
  unsigned long long limit_ns = 2000000000ull;
  if (const char* lim = getenv("CORR2D_WAIT_LIMIT_MS")) {
    const long v = atol(lim);
    if (v > 0) limit_ns = (unsigned long long)v * 1000000ull;
  }
  if (e == cudaSuccess)
    e = launch_prep_tc((const PrepJob*)(S + off_jobs), (const PrepItem*)(S + off_pit),
                       (int)pit.size(), planes, kp, err, limit_ns, stream);
  if (e == cudaSuccess)
    e = launch_xspec_tc((const XProblem*)(S + off_prob), (const XItem*)(S + off_xit),
                        (int)items.size(), planes, ds->sm_count, err, limit_ns, stream, 0, 1, 4,
                        1, 8.0 * n1 * n2 <= kPdlMaxOutBytes, &xp);
  // The host-side descriptors above must outlive the copies: wait for the stream.
  cudaError_t es = cudaStreamSynchronize(stream);
  if (e != cudaSuccess || es != cudaSuccess)
    return say(msg, msg_len, CORR2D_ECUDA, "CUDA error: %s",
               cudaGetErrorString(e != cudaSuccess ? e : es));
  int word = 0;
  if ((e = cudaMemcpy(&word, S, sizeof word, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return say(msg, msg_len, CORR2D_ECUDA, "reading the error word failed: %s", cudaGetErrorString(e));
  if (word != DEV_OK)
    return say(msg, msg_len, CORR2D_ETIMEOUT, "a device-side wait exceeded its limit");
  return CORR2D_OK;
}
