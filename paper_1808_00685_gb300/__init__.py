"""Python binding of libcorr2d, the GB300 (sm_103a) generalized 2D correlation library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/corr2d.h``.  The functions
``corr2d_*`` mirror the C entry points one to one (raw pointers and sizes);
``Context`` wraps them for torch CUDA tensors.  Importing works without a GPU;
loading the library fails loudly if it has not been built, and there is no
CPU fallback.

The method: Geitner et al., arXiv:1808.00685 (the corr2D R package) --
dynamic spectra (Eq. dynspec), DFT along the perturbation axis (Eq. disFT),
half-spectrum complex correlation Phi + i Psi (Eq. disint2d, Sec. 4.2) and
optional scaling (Eqs. scalesyn, scaleasyn).
"""
from __future__ import annotations

import ctypes
import os
import threading

from ._build import build, lib_path

__all__ = [
    "Corr2dError", "Context", "BatchPlan", "load", "build", "lib_path", "EXPORTED_SYMBOLS",
    "PREC_FP32", "PREC_SPLIT", "PREC_BF16", "REF_MEAN", "REF_USER", "FLAG_NO_MIRROR",
]

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}
PREC_FP32, PREC_SPLIT, PREC_BF16 = 0, 1, 2
REF_MEAN, REF_USER = 0, 1
FLAG_NO_MIRROR = 1
FLAG_EXACT_SYMMETRY = 2
FLAG_HILBERT = 4
FLAG_UPPER_TRIANGLE = 8
FLAG_OUTPUT_BF16 = 16
_PREC_BY_NAME = {"fp32": PREC_FP32, "split": PREC_SPLIT, "bf16": PREC_BF16}
INTERP_LINEAR, INTERP_SPLINE = 0, 1
_INTERP_BY_NAME = {"linear": INTERP_LINEAR, "spline": INTERP_SPLINE}

EXPORTED_SYMBOLS = (
    "corr2d_params_default", "corr2d_create", "corr2d_destroy", "corr2d_set_stream",
    "corr2d_last_error", "corr2d_synchronize", "corr2d_preprocess", "corr2d_compute",
    "corr2d_compute_host", "corr2d_batch", "corr2d_version", "corr2d_set_profiling",
    "corr2d_get_timings", "corr2d_compute_noalloc", "corr2d_preprocess_perturbation",
    "corr2d_compute_rows", "corr2d_compute_reduced", "corr2d_interpolate_perturbation",
    "corr2d_get_kernel_info", "corr2d_measure_fp32_peak", "corr2d_compute_part",
    "corr2d_plan_part", "corr2d_plan_batch_part",
)
XSPEC_NONE, XSPEC_TC, XSPEC_TC_PAIR, XSPEC_FP32, XSPEC_TC_TA = range(5)


class corr2d_params(ctypes.Structure):
    _fields_ = [("ref_mode", ctypes.c_int), ("ref1", ctypes.c_void_p), ("ref2", ctypes.c_void_p),
                ("norm", ctypes.c_double), ("alpha", ctypes.c_double),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint)]


class corr2d_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("y1", ctypes.c_void_p), ("y2", ctypes.c_void_p), ("phi", ctypes.c_void_p),
                ("psi", ctypes.c_void_p), ("ldo", ctypes.c_long)]


class Corr2dError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libcorr2d (built by ``build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"libcorr2d is not built ({p}); run paper_1808_00685_gb300.build()")
        lib = ctypes.CDLL(p)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "corr2d_params_default": (i, [ctypes.POINTER(corr2d_params)]),
            "corr2d_create": (i, [ctypes.POINTER(vp), i, vp]),
            "corr2d_destroy": (i, [vp]),
            "corr2d_set_stream": (i, [vp, vp]),
            "corr2d_last_error": (ctypes.c_char_p, [vp]),
            "corr2d_synchronize": (i, [vp]),
            "corr2d_preprocess": (i, [vp, i, i, vp, vp, i, vp, vp, vp]),
            "corr2d_preprocess_perturbation": (i, [vp, i, i, vp, vp, i, i, vp]),
            "corr2d_interpolate_perturbation": (i, [vp, i, i, i, vp, vp, i, i, vp]),
            "corr2d_compute_rows": (i, [vp, i, i, vp, i, i, vp, i, ctypes.POINTER(corr2d_params),
                                        i, i, vp, vp, ctypes.c_long]),
            "corr2d_compute_reduced": (i, [vp, i, i, vp, i, i, vp, i,
                                           ctypes.POINTER(corr2d_params), i, vp, vp,
                                           ctypes.c_long]),
            "corr2d_compute": (i, [vp, i, i, vp, i, i, vp, i, ctypes.POINTER(corr2d_params), vp,
                                   vp, ctypes.c_long, vp, vp]),
            "corr2d_compute_host": (i, [vp, i, i, vp, i, vp, ctypes.POINTER(corr2d_params), vp,
                                        vp, ctypes.c_long]),
            "corr2d_batch": (i, [vp, i, ctypes.POINTER(corr2d_problem),
                                 ctypes.POINTER(corr2d_params)]),
            "corr2d_version": (ctypes.c_char_p, []),
            "corr2d_compute_noalloc": (i, [i, vp, i, i, vp, i, i, vp, i,
                                           ctypes.POINTER(corr2d_params), vp, vp, ctypes.c_long,
                                           ctypes.c_char_p, ctypes.c_size_t]),
            "corr2d_set_profiling": (i, [vp, i]),
            "corr2d_get_timings": (i, [vp, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float)]),
            "corr2d_get_kernel_info": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
            "corr2d_measure_fp32_peak": (i, [vp, ctypes.POINTER(d)]),
            "corr2d_compute_part": (i, [vp, i, i, vp, i, i, vp, i, ctypes.POINTER(corr2d_params),
                                        i, i, vp, vp, ctypes.c_long]),
            "corr2d_plan_part": (i, [i, i, i, ctypes.c_uint, i, i, ctypes.POINTER(i), i,
                                     ctypes.POINTER(i)]),
            "corr2d_plan_batch_part": (i, [i, ctypes.POINTER(i), ctypes.POINTER(i),
                                           ctypes.POINTER(i), i, i, ctypes.POINTER(i), i,
                                           ctypes.POINTER(i)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _ = d
        _lib = lib
        return lib


# ------------------------------------------------------------ C-ABI mirrors
def corr2d_params_default() -> corr2d_params:
    p = corr2d_params()
    load().corr2d_params_default(ctypes.byref(p))
    return p


def corr2d_create(device: int = 0, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    st = load().corr2d_create(ctypes.byref(h), device, stream)
    if st != OK:
        raise Corr2dError(st, load().corr2d_last_error(None).decode())
    return h.value


def corr2d_last_error(ctx: int | None) -> str:
    return load().corr2d_last_error(ctx).decode()


def _check(ctx, st):
    if st != OK:
        raise Corr2dError(st, corr2d_last_error(ctx))


def corr2d_destroy(ctx: int) -> None:
    _check(None, load().corr2d_destroy(ctx))


def corr2d_set_stream(ctx: int, stream: int | None) -> None:
    _check(ctx, load().corr2d_set_stream(ctx, stream))


def corr2d_synchronize(ctx: int) -> None:
    _check(ctx, load().corr2d_synchronize(ctx))


def corr2d_preprocess_perturbation(ctx, m, n, time, y, ld, N, y_out) -> None:
    _check(ctx, load().corr2d_preprocess_perturbation(ctx, m, n, time, y, ld, N, y_out))


def corr2d_interpolate_perturbation(ctx, method, m, n, time, y, ld, N, y_out) -> None:
    _check(ctx, load().corr2d_interpolate_perturbation(ctx, method, m, n, time, y, ld, N, y_out))


def corr2d_preprocess(ctx, m, n_raw, x_raw, y_raw, n_out, y_out, ref=None, dyn_out=None) -> None:
    _check(ctx, load().corr2d_preprocess(ctx, m, n_raw, x_raw, y_raw, n_out, y_out, ref, dyn_out))


def corr2d_compute(ctx, m, n1, y1, ld1, n2, y2, ld2, params, phi, psi, ldo, sigma1=None,
                   sigma2=None) -> None:
    pp = ctypes.byref(params) if params is not None else None
    _check(ctx, load().corr2d_compute(ctx, m, n1, y1, ld1, n2, y2, ld2, pp, phi, psi, ldo,
                                      sigma1, sigma2))


def corr2d_compute_rows(ctx, m, n1, y1, ld1, n2, y2, ld2, params, row_begin, row_count, phi,
                        psi, ldo) -> None:
    pp = ctypes.byref(params) if params is not None else None
    _check(ctx, load().corr2d_compute_rows(ctx, m, n1, y1, ld1, n2, y2, ld2, pp, row_begin,
                                           row_count, phi, psi, ldo))


def corr2d_compute_reduced(ctx, m, n1, y1, ld1, n2, y2, ld2, params, reduce, phi_r, psi_r,
                           ldr) -> None:
    pp = ctypes.byref(params) if params is not None else None
    _check(ctx, load().corr2d_compute_reduced(ctx, m, n1, y1, ld1, n2, y2, ld2, pp, reduce,
                                              phi_r, psi_r, ldr))


def corr2d_compute_part(ctx, m, n1, y1, ld1, n2, y2, ld2, params, part, nparts, phi, psi,
                        ldo) -> None:
    pp = ctypes.byref(params) if params is not None else None
    _check(ctx, load().corr2d_compute_part(ctx, m, n1, y1, ld1, n2, y2, ld2, pp, part, nparts,
                                           phi, psi, ldo))


def corr2d_plan_part(n1: int, n2: int, homo: bool, flags: int, part: int, nparts: int):
    """Tiles (ti, tj) of part `part` of `nparts` of an n1 x n2 problem, in list order
    (host only; the tile split corr2d_compute_part uses)."""
    lib = load()
    cnt = ctypes.c_int()
    _check(None, lib.corr2d_plan_part(n1, n2, 1 if homo else 0, flags, part, nparts, None, 0,
                                      ctypes.byref(cnt)))
    buf = (ctypes.c_int * max(2 * cnt.value, 1))()
    _check(None, lib.corr2d_plan_part(n1, n2, 1 if homo else 0, flags, part, nparts, buf,
                                      cnt.value, ctypes.byref(cnt)))
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(cnt.value)]


def plan_batch_part(shapes, part: int, nparts: int):
    """Indices (increasing) of the problems of a batch that go to part `part` of
    `nparts` (host only; corr2d_plan_batch_part's cost-balanced split).  shapes:
    (m, n1, n2, homo) per problem; a homo problem's n2 is ignored."""
    lib = load()
    k = len(shapes)
    arr = lambda vals: (ctypes.c_int * max(k, 1))(*vals)
    m = arr([s[0] for s in shapes])
    n1 = arr([s[1] for s in shapes])
    n2 = arr([0 if s[3] else s[2] for s in shapes])
    cnt = ctypes.c_int()
    out = (ctypes.c_int * max(k, 1))()
    _check(None, lib.corr2d_plan_batch_part(k, m, n1, n2, part, nparts, out, k, ctypes.byref(cnt)))
    return [out[i] for i in range(cnt.value)]


def shard_rows(n1: int, world: int, rank: int, tile: int = 128):
    """Row slab (row_begin, row_count) of rank `rank` when the n1 output rows are
    split over `world` GPUs in whole 128-row tiles (corr2d_compute_rows)."""
    ntiles = (n1 + tile - 1) // tile
    per, extra = divmod(ntiles, world)
    t0 = rank * per + min(rank, extra)
    t1 = t0 + per + (1 if rank < extra else 0)
    r0, r1 = t0 * tile, min(n1, t1 * tile)
    return r0, max(0, r1 - r0)


def corr2d_compute_host(ctx, m, n1, y1, n2, y2, params, phi, psi, ldo) -> None:
    pp = ctypes.byref(params) if params is not None else None
    _check(ctx, load().corr2d_compute_host(ctx, m, n1, y1, n2, y2, pp, phi, psi, ldo))


def corr2d_batch(ctx, problems, params=None) -> None:
    arr = (corr2d_problem * len(problems))(*problems)
    pp = ctypes.byref(params) if params is not None else None
    _check(ctx, load().corr2d_batch(ctx, len(problems), arr, pp))


def corr2d_version() -> str:
    return load().corr2d_version().decode()


def corr2d_compute_noalloc(device, stream, m, n1, y1, ld1, n2, y2, ld2, params, phi, psi,
                           ldo) -> None:
    """Allocation-free correlation (no context, static device scratch; synchronous).

    For callers that must not allocate GPU memory; see include/corr2d.h for
    the size limit and the rule that calls must not overlap on the GPU."""
    buf = ctypes.create_string_buffer(512)
    pp = ctypes.byref(params) if params is not None else None
    st = load().corr2d_compute_noalloc(device, stream, m, n1, y1, ld1, n2, y2, ld2, pp, phi, psi,
                                       ldo, buf, len(buf))
    if st != OK:
        raise Corr2dError(st, buf.value.decode())


def corr2d_set_profiling(ctx: int, on: bool) -> None:
    _check(ctx, load().corr2d_set_profiling(ctx, 1 if on else 0))


def corr2d_get_timings(ctx: int):
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(ctx, load().corr2d_get_timings(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def corr2d_measure_fp32_peak(ctx: int) -> float:
    """Measured FP32 FMA throughput of the context's device, TFLOP/s."""
    t = ctypes.c_double()
    _check(ctx, load().corr2d_measure_fp32_peak(ctx, ctypes.byref(t)))
    return t.value


class BatchPlan:
    """corr2d_batch arguments for one list of problems (torch tensors), built
    once.  The tensors must stay alive while the plan is run."""

    def __init__(self, ctx: "Context", problems, params: corr2d_params):
        self.ctx = ctx
        self.count = len(problems)
        self.arr = (corr2d_problem * max(self.count, 1))()
        for i, (y1, y2, phi, psi) in enumerate(problems):
            m, n1 = y1.shape
            n2 = n1 if y2 is None else y2.shape[1]
            self.arr[i] = corr2d_problem(m, n1, n2, _ptr(y1), _ptr(y2), _ptr(phi), _ptr(psi),
                                         phi.stride(0))
        self.params = params
        self._keep = problems

    def run(self) -> None:
        _check(self.ctx.handle, load().corr2d_batch(self.ctx.handle, self.count, self.arr,
                                                    ctypes.byref(self.params)))


def corr2d_get_kernel_info(ctx: int):
    """(last cross-spectrum kernel: XSPEC_*, co-resident CTA pairs)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().corr2d_get_kernel_info(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ------------------------------------------------------------ torch helpers
def _ptr(t):
    return None if t is None else t.data_ptr()


def make_params(precision="split", alpha=0.0, norm=0.0, ref1=None, ref2=None,
                no_mirror=False, exact_symmetry=False, hilbert=False,
                upper_triangle=False, output_bf16=False) -> corr2d_params:
    p = corr2d_params_default()
    p.precision = _PREC_BY_NAME[precision] if isinstance(precision, str) else int(precision)
    p.alpha = float(alpha)
    p.norm = float(norm)
    if ref1 is not None:
        p.ref_mode = REF_USER
        p.ref1 = _ptr(ref1)
        p.ref2 = _ptr(ref2)
    p.flags = ((FLAG_NO_MIRROR if no_mirror else 0) | (FLAG_EXACT_SYMMETRY if exact_symmetry else 0)
               | (FLAG_HILBERT if hilbert else 0) | (FLAG_UPPER_TRIANGLE if upper_triangle else 0)
               | (FLAG_OUTPUT_BF16 if output_bf16 else 0))
    return p


class Context:
    """A library context on one CUDA device and stream (torch tensors in, out)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.handle = corr2d_create(device, stream.cuda_stream)

    def close(self):
        if self.handle:
            corr2d_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        corr2d_synchronize(self.handle)

    def set_stream(self, stream):
        """Enqueue later calls on `stream` (a torch.cuda.Stream)."""
        self.stream = stream
        corr2d_set_stream(self.handle, stream.cuda_stream)

    def set_profiling(self, on: bool = True):
        corr2d_set_profiling(self.handle, on)

    def timings(self):
        """(prep_ms, xspec_ms) of the last call (profiling must be on)."""
        return corr2d_get_timings(self.handle)

    def fp32_peak_tflops(self) -> float:
        """Measured FP32 FMA throughput of this device (TFLOP/s)."""
        return corr2d_measure_fp32_peak(self.handle)

    def kernel_info(self):
        """(last cross-spectrum kernel: XSPEC_*, co-resident CTA pairs)."""
        return corr2d_get_kernel_info(self.handle)

    @staticmethod
    def alloc_out(n1, n2, device, ld=None, bf16=False):
        """Phi/Psi buffers whose rows start on 128-byte boundaries (ld a multiple of
        32 floats, or 64 BF16 elements with bf16=True): every stored box row is then
        one whole 128-byte line.  With rows only 16-byte aligned, half the rows of an
        odd-width matrix split their lines into partial 32-byte sectors, which DRAM
        writes read-modify-write (batches of ragged problems ran ~20 % slower)."""
        import torch
        q = 64 if bf16 else 32
        ldo = ld or (n2 + q - 1) // q * q
        dt = torch.bfloat16 if bf16 else torch.float32
        phi = torch.empty((n1, ldo), dtype=dt, device=device)
        psi = torch.empty((n1, ldo), dtype=dt, device=device)
        return phi, psi, ldo

    def compute(self, y1, y2=None, precision="split", alpha=0.0, norm=0.0, ref1=None, ref2=None,
                no_mirror=False, out=None, want_sigma=False, exact_symmetry=False,
                hilbert=False, upper_triangle=False, output_bf16=False):
        """Phi, Psi (n1 x n2 views) of the m x n1 stack y1 (and y2, or homo); BF16
        tensors with output_bf16 (each the FP32 result rounded to nearest)."""
        import torch
        assert y1.is_cuda and y1.dtype == torch.float32 and y1.dim() == 2
        m, n1 = y1.shape
        if y2 is not None:
            assert y2.is_cuda and y2.dtype == torch.float32 and y2.shape[0] == m
        n2 = n1 if y2 is None else y2.shape[1]
        if out is None:
            phi, psi, ldo = self.alloc_out(n1, n2, y1.device, bf16=output_bf16)
        else:
            phi, psi = out
            ldo = phi.stride(0)
        s1 = torch.empty(n1, dtype=torch.float32, device=y1.device) if want_sigma else None
        s2 = (torch.empty(n2, dtype=torch.float32, device=y1.device)
              if (want_sigma and y2 is not None) else None)
        params = make_params(precision, alpha, norm, ref1, ref2, no_mirror, exact_symmetry,
                             hilbert, upper_triangle, output_bf16)
        corr2d_compute(self.handle, m, n1, _ptr(y1), y1.stride(0), n2, _ptr(y2),
                       y2.stride(0) if y2 is not None else 0, params, _ptr(phi), _ptr(psi), ldo,
                       _ptr(s1), _ptr(s2))
        res = (phi[:, :n2], psi[:, :n2])
        if want_sigma:
            return res + (s1, s2 if s2 is not None else s1)
        return res

    def preprocess_perturbation(self, time, y, N, method="linear"):
        """Resample the m x n stack y along the perturbation axis onto N equidistant
        steps with the linear or the (fmm) spline interpolating function."""
        import torch
        m, n = y.shape
        out = torch.empty((N, n), dtype=torch.float32, device=y.device)
        corr2d_interpolate_perturbation(self.handle, _INTERP_BY_NAME[method], m, n, _ptr(time),
                                        _ptr(y), y.stride(0), N, _ptr(out))
        return out

    def preprocess(self, x_raw, y_raw, n_out, ref=None):
        import torch
        m, n_raw = y_raw.shape
        out = torch.empty((m, n_out), dtype=torch.float32, device=y_raw.device)
        dyn = torch.empty_like(out) if ref is not None else None
        corr2d_preprocess(self.handle, m, n_raw, _ptr(x_raw), _ptr(y_raw), n_out, _ptr(out),
                          _ptr(ref), _ptr(dyn))
        return out, dyn

    def batch(self, problems, precision="split", alpha=0.0, norm=0.0, no_mirror=False,
              hilbert=False, output_bf16=False):
        """problems: list of (y1, y2 or None, phi, psi) torch tensors (phi/psi n1 x ldo,
        BF16 with output_bf16)."""
        self.batch_plan(problems, precision, alpha, norm, no_mirror, hilbert, output_bf16).run()

    def batch_plan(self, problems, precision="split", alpha=0.0, norm=0.0, no_mirror=False,
                   hilbert=False, output_bf16=False) -> "BatchPlan":
        """The descriptor array of a batch, marshalled once; ``run()`` submits it
        (repeated runs of the same list replay the library's recorded graph)."""
        return BatchPlan(self, problems, make_params(precision, alpha, norm, None, None,
                                                     no_mirror, hilbert=hilbert,
                                                     output_bf16=output_bf16))

    def compute_reduced(self, y1, y2, reduce, precision="split", alpha=0.0, norm=0.0,
                        hilbert=False, ref1=None, ref2=None, output_bf16=False):
        """Every reduce-th row and column of Phi and Psi (plot_corr2din3d's `reduce`)."""
        m, n1 = y1.shape
        n2 = n1 if y2 is None else y2.shape[1]
        phi, psi, ldr = self.alloc_out(n1 // reduce, n2 // reduce, y1.device, bf16=output_bf16)
        params = make_params(precision, alpha, norm, ref1, ref2, hilbert=hilbert,
                             output_bf16=output_bf16)
        corr2d_compute_reduced(self.handle, m, n1, _ptr(y1), y1.stride(0), n2, _ptr(y2),
                               y2.stride(0) if y2 is not None else 0, params, reduce, _ptr(phi),
                               _ptr(psi), ldr)
        return phi[:, :n2 // reduce], psi[:, :n2 // reduce]

    def compute_rows(self, y1, y2, row_begin, row_count, precision="split", alpha=0.0, norm=0.0,
                     hilbert=False, output_bf16=False):
        """Rows [row_begin, row_begin + row_count) of Phi and Psi (row_begin % 128 == 0)."""
        m, n1 = y1.shape
        n2 = n1 if y2 is None else y2.shape[1]
        phi, psi, ldo = self.alloc_out(row_count, n2, y1.device, bf16=output_bf16)
        params = make_params(precision, alpha, norm, hilbert=hilbert, output_bf16=output_bf16)
        corr2d_compute_rows(self.handle, m, n1, _ptr(y1), y1.stride(0), n2, _ptr(y2),
                            y2.stride(0) if y2 is not None else 0, params, row_begin, row_count,
                            _ptr(phi), _ptr(psi), ldo)
        return phi[:, :n2], psi[:, :n2]

    def compute_part(self, y1, y2, part, nparts, precision="split", alpha=0.0, norm=0.0,
                     no_mirror=False, upper_triangle=False, hilbert=False, out=None,
                     output_bf16=False):
        """Part `part` of `nparts` of the output tiles (and their mirrors) of Phi and Psi,
        written at their places in full n1 x n2 buffers; other elements are untouched."""
        m, n1 = y1.shape
        n2 = n1 if y2 is None else y2.shape[1]
        if out is None:
            phi, psi, ldo = self.alloc_out(n1, n2, y1.device, bf16=output_bf16)
        else:
            phi, psi = out
            ldo = phi.stride(0)
        params = make_params(precision, alpha, norm, no_mirror=no_mirror,
                             upper_triangle=upper_triangle, hilbert=hilbert,
                             output_bf16=output_bf16)
        corr2d_compute_part(self.handle, m, n1, _ptr(y1), y1.stride(0), n2, _ptr(y2),
                            y2.stride(0) if y2 is not None else 0, params, part, nparts,
                            _ptr(phi), _ptr(psi), ldo)
        return phi[:, :n2], psi[:, :n2]

    def compute_host(self, y1, y2=None, precision="split", alpha=0.0, norm=0.0, out=None):
        """Host (CPU) tensors in and out; copies overlap the kernels inside the library."""
        import torch
        m, n1 = y1.shape
        n2 = n1 if y2 is None else y2.shape[1]
        if out is None:
            phi = torch.empty((n1, n2), dtype=torch.float32)
            psi = torch.empty((n1, n2), dtype=torch.float32)
        else:
            phi, psi = out
        params = make_params(precision, alpha, norm)
        corr2d_compute_host(self.handle, m, n1, _ptr(y1), n2, _ptr(y2), params, _ptr(phi),
                            _ptr(psi), phi.stride(0))
        return phi, psi
