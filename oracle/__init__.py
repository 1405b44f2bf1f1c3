"""FP64 CPU oracle for generalized 2D correlation analysis (arXiv:1808.00685).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
(``paper_1808_00685_gb300``) never imports this package and shares no code
with it.

The arithmetic lives in ``corr2d_oracle.c`` (plain double loops, direct
O(m^2) DFT, no FFT); this module compiles it with the host C compiler on first
use and exposes it through ctypes with numpy arrays.  Every function cites the
passage of the paper it states; the readings taken where the paper is silent
or inconsistent are listed at the top of the C file (R1..R13); ``reduce_map`` states its
own (R14) in its docstring.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force by a second formula, library special cases, Parseval, closed
forms, invariants, the Noda sign rules, and for ``hilbert_noda`` the matrix
written out by hand, the sawtooth series and FT/HT agreement); the module
docstring there names the pins of each function.  None is "parity unpinned".
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corr2d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)


def lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP, no FP contraction) in-tree."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _configure(lib):
    lib.oracle_num_freq.restype = ctypes.c_int
    lib.oracle_num_freq.argtypes = [ctypes.c_int]
    lib.oracle_weight.restype = ctypes.c_double
    lib.oracle_weight.argtypes = [ctypes.c_int]
    lib.oracle_default_norm.restype = ctypes.c_double
    lib.oracle_default_norm.argtypes = [ctypes.c_int]
    lib.oracle_scale_factor.restype = ctypes.c_double
    lib.oracle_scale_factor.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.oracle_reference_mean.argtypes = [ctypes.c_int, ctypes.c_int, _fp, ctypes.c_long, _dp]
    lib.oracle_dynamic.argtypes = [ctypes.c_int, ctypes.c_int, _fp, ctypes.c_long, _dp, _dp]
    lib.oracle_sigma.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
    lib.oracle_dft.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
    lib.oracle_cross_spectrum.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double,
        _dp, _dp, ctypes.c_int, _ip, _dp, _dp, ctypes.c_int]
    lib.oracle_corr2d.restype = ctypes.c_int
    lib.oracle_corr2d.argtypes = [
        ctypes.c_int, ctypes.c_int, _fp, ctypes.c_long, ctypes.c_int, _fp, ctypes.c_long,
        ctypes.c_int, _fp, _fp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _ip,
        _dp, _dp, _dp, _dp, ctypes.c_int]
    lib.oracle_interp_linear.restype = ctypes.c_int
    lib.oracle_interp_linear.argtypes = [
        ctypes.c_int, ctypes.c_int, _dp, _fp, ctypes.c_long, ctypes.c_int, _dp, _fp, _dp]
    lib.oracle_hilbert_noda.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                        _dp, _dp]
    lib.oracle_interp_perturbation.restype = ctypes.c_int
    lib.oracle_interp_perturbation.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _fp,
                                               ctypes.c_long, ctypes.c_int, _dp]
    lib.oracle_interp_spline.restype = ctypes.c_int
    lib.oracle_interp_spline.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _fp, ctypes.c_long,
                                         ctypes.c_int, _dp]
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
        return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every call to another build of the oracle source.

    Used by the mutation tests, which compile copies of the C file with a
    planted mistake and check that the pins reject them."""
    global _lib
    _load()
    saved = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def compile_source(src: str, out: str) -> str:
    """Compile a C source text (a copy of the oracle) to a shared library."""
    cpath = out + ".c"
    with open(cpath, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", cpath, "-o", out, "-lm"], check=True)
    return out


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_fp)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def num_freq(m: int) -> int:
    """Number K+1 of retained frequencies omega = 0..floor((m-1)/2) (Sec. 4.2 FFT index)."""
    return _load().oracle_num_freq(m)


def weight(omega: int) -> float:
    """Half-spectrum weight: 1 for omega = 0, else 2 (Sec. 4.2, Eq. symmeFT)."""
    return _load().oracle_weight(omega)


def default_norm(m: int) -> float:
    """Default normalisation 1/(pi (m-1)) (Eq. disint2d)."""
    return _load().oracle_default_norm(m)


def scale_factor(sigma: float, alpha: float) -> float:
    """sigma^-alpha, 1 without scaling, 0 for sigma = 0 (Eqs. scale*)."""
    return _load().oracle_scale_factor(sigma, alpha)


def max_threads() -> int:
    return _load().oracle_max_threads()


def reference_mean(y: np.ndarray) -> np.ndarray:
    """Perturbation-mean reference spectrum (Eq. ref). y is m x n (rows = t_j)."""
    y, yp = _f32(y)
    m, n = y.shape
    ref = np.empty(n, np.float64)
    _load().oracle_reference_mean(m, n, yp, n, ref.ctypes.data_as(_dp))
    return ref


def dynamic(y: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Dynamic spectra y - ref (Eq. dynspec)."""
    y, yp = _f32(y)
    m, n = y.shape
    ref, rp = _f64(ref)
    out = np.empty((m, n), np.float64)
    _load().oracle_dynamic(m, n, yp, n, rp, out.ctypes.data_as(_dp))
    return out


def sigma(ydyn: np.ndarray) -> np.ndarray:
    """Per-variable standard deviation with (m-1) denominator (Eq. stdev)."""
    ydyn, dp = _f64(ydyn)
    m, n = ydyn.shape
    out = np.empty(n, np.float64)
    _load().oracle_sigma(m, n, dp, out.ctypes.data_as(_dp))
    return out


def dft(ydyn: np.ndarray):
    """Truncated DFT along the perturbation axis (Eq. disFT), omega = 0..K.

    Returns complex Y of shape (n, K+1)."""
    ydyn, dp = _f64(ydyn)
    m, n = ydyn.shape
    nf = num_freq(m)
    yr = np.empty((n, nf), np.float64)
    yi = np.empty((n, nf), np.float64)
    _load().oracle_dft(m, n, dp, nf, yr.ctypes.data_as(_dp), yi.ctypes.data_as(_dp))
    return yr + 1j * yi


def cross_spectrum(Y1: np.ndarray, Y2: np.ndarray, norm: float, s1=None, s2=None, rows=None,
                   nthreads: int = 1):
    """Half-spectrum complex correlation (Eq. disint2d, Sec. 4.2) -> (Phi, Psi)."""
    n1, nf = Y1.shape
    n2 = Y2.shape[0]
    yr1, p1 = _f64(Y1.real)
    yi1, q1 = _f64(Y1.imag)
    yr2, p2 = _f64(Y2.real)
    yi2, q2 = _f64(Y2.imag)
    s1, sp1 = _f64(np.ones(n1) if s1 is None else s1)
    s2, sp2 = _f64(np.ones(n2) if s2 is None else s2)
    if rows is None:
        nrows, rp = n1, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        nrows, rp = len(rows), rows.ctypes.data_as(_ip)
    phi = np.empty((nrows, n2), np.float64)
    psi = np.empty((nrows, n2), np.float64)
    _load().oracle_cross_spectrum(n1, n2, nf, p1, q1, p2, q2, float(norm), sp1, sp2, nrows, rp,
                                  phi.ctypes.data_as(_dp), psi.ctypes.data_as(_dp), nthreads)
    return phi, psi


def corr2d(y1: np.ndarray, y2: np.ndarray | None = None, ref1=None, ref2=None, norm: float = 0.0,
           alpha: float = 0.0, rows=None, nthreads: int = 1):
    """Whole correlation: reference, dynamic spectra, scaling, DFT, correlation.

    y1 (m x n1) and optional y2 (m x n2) are FP32 stacks (rows = perturbation
    steps).  Returns (phi, psi, sigma1, sigma2) in FP64; phi/psi are
    len(rows) x n2 (all n1 rows when rows is None)."""
    y1, p1 = _f32(y1)
    m, n1 = y1.shape
    if y2 is not None:
        y2, p2 = _f32(y2)
        if y2.shape[0] != m:
            raise ValueError("both stacks need the same number of perturbation steps")
        n2 = y2.shape[1]
    else:
        p2, n2 = None, n1
    ref_mode = 0
    rp1 = rp2 = None
    if ref1 is not None:
        ref_mode = 1
        ref1, rp1 = _f32(ref1)
        if y2 is not None:
            if ref2 is None:
                raise ValueError("hetero correlation with a user reference needs ref2")
            ref2, rp2 = _f32(ref2)
    if rows is None:
        nrows, rows_p = n1, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        nrows, rows_p = len(rows), rows.ctypes.data_as(_ip)
    phi = np.empty((nrows, n2), np.float64)
    psi = np.empty((nrows, n2), np.float64)
    s1 = np.empty(n1, np.float64)
    s2 = np.empty(n2, np.float64)
    rc = _load().oracle_corr2d(m, n1, p1, n1, n2, p2, n2, ref_mode, rp1, rp2, float(norm),
                               float(alpha), nrows, rows_p, phi.ctypes.data_as(_dp),
                               psi.ctypes.data_as(_dp), s1.ctypes.data_as(_dp),
                               s2.ctypes.data_as(_dp), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_corr2d rejected its arguments (code {rc})")
    return phi, psi, s1, s2


def interp_linear(x_raw: np.ndarray, y_raw: np.ndarray, n_out: int, ref=None):
    """Linear resampling onto seq(x_first, x_last, length.out = n_out) (reading R12).

    Returns (y_out, dyn_out) in FP64; dyn_out is None without ref."""
    x_raw, xp = _f64(x_raw)
    y_raw, yp = _f32(y_raw)
    m, n_raw = y_raw.shape
    out = np.empty((m, n_out), np.float64)
    dyn = np.empty((m, n_out), np.float64) if ref is not None else None
    rp = None
    if ref is not None:
        ref, rp = _f32(ref)
    rc = _load().oracle_interp_linear(m, n_raw, xp, yp, n_raw, n_out, out.ctypes.data_as(_dp), rp,
                                      dyn.ctypes.data_as(_dp) if dyn is not None else None)
    if rc != 0:
        raise ValueError("oracle_interp_linear rejected its arguments")
    return out, dyn


def interp_perturbation(time: np.ndarray, y: np.ndarray, N: int,
                        method: str = "linear") -> np.ndarray:
    """Resampling along the perturbation axis onto N equidistant values (Sec. 4.2
    interpolation snippet, reading R13): method "linear" (approxfun) or "spline"
    (splinefun's default fmm spline).  y is m x n; returns N x n FP64."""
    time, tp = _f64(time)
    y, yp = _f32(y)
    m, n = y.shape
    out = np.empty((N, n), np.float64)
    fn = {"linear": _load().oracle_interp_perturbation,
          "spline": _load().oracle_interp_spline}[method]
    rc = fn(m, n, tp, yp, n, N, out.ctypes.data_as(_dp))
    if rc != 0:
        raise ValueError(f"oracle {method} interpolation rejected its arguments")
    return out


def reduce_map(M: np.ndarray, reduce: int) -> np.ndarray:
    """plot_corr2din3d's `reduce` (Sec. 4.3, reading R14): rows and columns whose
    1-based index i satisfies i %% reduce == 0, sampled with a box kernel at those
    grid points, i.e. their values themselves."""
    rows = [i - 1 for i in range(1, M.shape[0] + 1) if i % reduce == 0]
    cols = [j - 1 for j in range(1, M.shape[1] + 1) if j % reduce == 0]
    out = np.empty((len(rows), len(cols)), dtype=M.dtype)
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            out[a, b] = M[i, j]
    return out


def hilbert_noda(d1: np.ndarray, d2: np.ndarray):
    """Hilbert-transform approach on dynamic spectra (Eqs. disHTsyn..disHTasyn)."""
    d1, q1 = _f64(d1)
    d2, q2 = _f64(d2)
    m, n1 = d1.shape
    n2 = d2.shape[1]
    phi = np.empty((n1, n2), np.float64)
    psi = np.empty((n1, n2), np.float64)
    _load().oracle_hilbert_noda(m, n1, q1, n2, q2, phi.ctypes.data_as(_dp),
                                psi.ctypes.data_as(_dp))
    return phi, psi
