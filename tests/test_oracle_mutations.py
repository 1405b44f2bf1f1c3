"""Planted mistakes: each test compiles a copy of the oracle's C source with one
plausible error and checks that the pins of ``test_oracle_pins.py`` reject it.

This shows the pins are discriminating: a dropped term, a wrong sign, a wrong
index or weight, a conjugate on the wrong operand, a wrong denominator or a
misread scaling exponent each fail at least one independent check.  The
mistakes are planted on the CPU, in the oracle only.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
import test_oracle_pins as pins
from test_oracle_pins import _brute, _dense_fmm_spline, _grid, _rel

MUTATIONS = {
    "weights_all_one": ("return omega == 0 ? 1.0 : 2.0;", "return 1.0;"),
    "dc_doubled": ("return omega == 0 ? 1.0 : 2.0;", "return 2.0;"),
    "nyquist_kept": ("return (m - 1) / 2 + 1;", "return m / 2 + 1;"),
    "dft_sign": ("im -= d * sin(theta);", "im += d * sin(theta);"),
    "conj_on_first": ("zi += wt * (xi * yr - xr * yi);", "zi += wt * (xr * yi - xi * yr);"),
    "dropped_term": ("zr += wt * (xr * yr + xi * yi);", "zr += wt * (xr * yr);"),
    "sigma_over_m": ("sigma[v] = sqrt(s / (double)(m - 1));", "sigma[v] = sqrt(s / (double)m);"),
    "scaling_exponent_sign": ("return pow(sigma, -alpha);", "return pow(sigma, alpha);"),
    "norm_over_m": ("return 1.0 / (ORACLE_PI * (double)(m - 1));",
                    "return 1.0 / (ORACLE_PI * (double)m);"),
    "mean_over_m_minus_1": ("ref[v] = s / (double)m;", "ref[v] = s / (double)(m - 1);"),
    "dft_index_shift": ("long r = ((long)w * (long)j) % (long)m;",
                        "long r = ((long)w * (long)(j + 1)) % (long)m;"),
    "user_ref_ignored": ("for (int v = 0; v < n1; ++v) r1[v] = (double)ref1[v];",
                         "for (int v = 0; v < n1; ++v) r1[v] = 0.0;"),
    "interp_weight": ("double t = (x - xa) / (xb - xa);", "double t = (x - xa) / (xb - x0);"),
    "psi_unscaled": ("psi[(long)r * n2 + b] = f * zi;", "psi[(long)r * n2 + b] = norm * zi;"),
    "perturbation_grid": ("double t0 = time[0], t1 = time[m - 1];\n  double step = (t1 - t0) / (double)(N - 1);",
                          "double t0 = time[0], t1 = time[m - 1];\n  double step = (t1 - t0) / (double)N;"),
    "spline_zero_end_third_derivative": ("g0 = 6.0 * oracle_third_divided_difference(time, yv);",
                                         "g0 = 0.0;"),
    "spline_interior_rhs_factor": ("rhs[i] = 6.0 * ((yv[i + 1] - yv[i]) / hr - (yv[i] - yv[i - 1]) / hl);",
                                   "rhs[i] = 3.0 * ((yv[i + 1] - yv[i]) / hr - (yv[i] - yv[i - 1]) / hl);"),
    "spline_end_interval_width": ("rhs[m - 1] = g1 * (time[m - 1] - time[m - 2]);",
                                  "rhs[m - 1] = g1 * (time[m - 2] - time[m - 3]);"),
    "spline_eval_weight": ("(yv[seg] - M[seg] * h * h / 6.0) * A / h",
                           "(yv[seg] - M[seg] * h * h / 6.0) * B / h"),
    "dyn_out_ref_sign": ("dyn_out[(long)j * n_out + k] = val - (ref ? (double)ref[k] : 0.0);",
                         "dyn_out[(long)j * n_out + k] = val + (ref ? (double)ref[k] : 0.0);"),
    "hilbert_pi_dropped": ("if (k != j) s += d2[(long)k * n2 + b] / (ORACLE_PI * (double)(k - j));",
                           "if (k != j) s += d2[(long)k * n2 + b] / ((double)(k - j));"),
    "hilbert_transposed": ("if (k != j) s += d2[(long)k * n2 + b] / (ORACLE_PI * (double)(k - j));",
                           "if (k != j) s += d2[(long)k * n2 + b] / (ORACLE_PI * (double)(j - k));"),
    "hilbert_psi_over_m": ("psi[(long)a * n2 + b] = sq / (double)(m - 1);",
                           "psi[(long)a * n2 + b] = sq / (double)m;"),
    "hilbert_phi_over_m": ("phi[(long)a * n2 + b] = sp / (double)(m - 1);",
                           "phi[(long)a * n2 + b] = sp / (double)m;"),
    "hilbert_on_stack_1": (
        """  double* z = malloc(sizeof(double) * (size_t)m * n2);
  if (!z) return;
  for (int b = 0; b < n2; ++b)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k)
        if (k != j) s += d2[(long)k * n2 + b] / (ORACLE_PI * (double)(k - j));
      z[(long)j * n2 + b] = s;
    }
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) {
      double sp = 0.0, sq = 0.0;
      for (int j = 0; j < m; ++j) {
        sp += d1[(long)j * n1 + a] * d2[(long)j * n2 + b];
        sq += d1[(long)j * n1 + a] * z[(long)j * n2 + b];
      }""",
        """  double* z = malloc(sizeof(double) * (size_t)m * n1);
  if (!z) return;
  for (int a = 0; a < n1; ++a)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k)
        if (k != j) s += d1[(long)k * n1 + a] / (ORACLE_PI * (double)(k - j));
      z[(long)j * n1 + a] = s;
    }
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) {
      double sp = 0.0, sq = 0.0;
      for (int j = 0; j < m; ++j) {
        sp += d1[(long)j * n1 + a] * d2[(long)j * n2 + b];
        sq += z[(long)j * n1 + a] * d2[(long)j * n2 + b];
      }"""),
}


def _battery():
    """Run the independent pins; return the names of those that fail."""
    failed = []

    def check(name, fn):
        try:
            if not fn():
                failed.append(name)
        except Exception:  # a mutant may also trip an argument check
            failed.append(name)

    y1 = workloads.random_stack(6, 5, seed=1, offset=0.5)
    y2 = workloads.random_stack(6, 4, seed=2, offset=-1.0)
    y3 = workloads.random_stack(5, 4, seed=3)

    def brute_homo():
        p, q, _, _ = oracle.corr2d(y1, alpha=0.5)
        bp, bq = _brute(y1, alpha=0.5)
        return _rel(p, bp) < 1e-12 and np.abs(q - bq).max() <= 1e-12 * np.abs(bp).max()

    def brute_hetero_odd():
        p, q, _, _ = oracle.corr2d(y3, workloads.random_stack(5, 3, seed=9))
        bp, bq = _brute(y3, workloads.random_stack(5, 3, seed=9))
        return _rel(p, bp) < 1e-12 and _rel(q, bq) < 1e-12

    def brute_user_ref():
        p, q, _, _ = oracle.corr2d(y1, y2, ref1=y1[0], ref2=y2[-1], alpha=1.0)
        bp, bq = _brute(y1, y2, ref1=y1[0], ref2=y2[-1], alpha=1.0)
        return _rel(p, bp) < 1e-12 and _rel(q, bq) < 1e-12

    def parseval_even():
        m = 8
        a = workloads.random_stack(m, 6, seed=4)
        p, _, _, _ = oracle.corr2d(a)
        d = a.astype(np.float64) - a.astype(np.float64).mean(0)
        alt = (-1.0) ** np.arange(m)
        rhs = m * d.T @ d - np.outer(alt @ d, alt @ d)
        return _rel(math.pi * (m - 1) * p, rhs) < 1e-12

    def pearson_diag():
        p, _, _, _ = oracle.corr2d(workloads.random_stack(9, 5, seed=5), alpha=1.0)
        return np.allclose(np.diag(p), 9 / math.pi, rtol=1e-12)

    def closed_form():
        m, n = 8, 32
        y, c, g, a = workloads.sinusoid_bands(m, n, [0.0, 50.0], seed=6)
        p, q, _, _ = oracle.corr2d(y)
        nu = np.arange(n, dtype=np.float64)
        L = 1.0 / (1.0 + ((nu[None, :] - c[:, None]) / g[:, None]) ** 2)
        E = ((a[:, None] * L) * np.exp(1j * np.deg2rad([0.0, 50.0]))[:, None]).sum(0)
        Z = (m * m / 2.0) * np.outer(E, np.conj(E)) / (math.pi * (m - 1))
        return _rel(p, Z.real) < 1e-5 and np.abs(q - Z.imag).max() < 1e-5 * np.abs(Z).max()

    def dft_numpy():
        d = np.random.default_rng(7).standard_normal((9, 4))
        return np.abs(oracle.dft(d) - np.fft.fft(d, axis=0)[:5].T).max() < 1e-12

    def sigma_numpy():
        a = workloads.random_stack(7, 5, seed=8, offset=1.0)
        d = oracle.dynamic(a, oracle.reference_mean(a))
        return np.allclose(oracle.sigma(d), a.astype(np.float64).std(0, ddof=1), rtol=1e-12)

    def interp_numpy():
        x = workloads.jittered_axis(40, 0.0, 29.0, np.random.default_rng(1))
        yy = workloads.random_stack(2, 40, seed=2)
        out, _ = oracle.interp_linear(x, yy, 30)
        g = np.linspace(0.0, 29.0, 30)
        return all(np.allclose(out[j], np.interp(g, x, yy[j].astype(np.float64)), atol=1e-12)
                   for j in range(2))

    def interp_t_numpy():
        t = np.sort(np.random.default_rng(5).uniform(0, 3, 9))
        yy = workloads.random_stack(9, 3, seed=6)
        out = oracle.interp_perturbation(t, yy, 13)
        g = np.linspace(t[0], t[-1], 13)
        return all(np.allclose(out[:, v], np.interp(g, t, yy[:, v].astype(np.float64)),
                               atol=1e-12) for v in range(3))

    def spline_cubic():
        t = np.array([0.0, 0.5, 1.25, 2.0, 3.5, 4.0, 5.75, 6.0])
        c = (0.5, -1.25, 0.75, 2.0)
        yy = np.polyval(c, t)[:, None].astype(np.float32)
        out = oracle.interp_perturbation(t, yy, 23, method="spline")
        return np.allclose(out[:, 0], np.polyval(c, _grid(t, 23)), rtol=0, atol=1e-10)

    def spline_dense():
        t = np.cumsum(np.random.default_rng(11).uniform(0.2, 1.5, 7))
        yy = workloads.random_stack(7, 2, seed=12)
        out = oracle.interp_perturbation(t, yy, 19, method="spline")
        g = _grid(t, 19)
        return all(np.allclose(out[:, v], _dense_fmm_spline(t, yy[:, v].astype(np.float64), g),
                               atol=1e-9) for v in range(2))

    def interp_dyn_out():
        pins.test_interp_dyn_out_is_the_dynamic_spectrum_of_the_correlation()
        return True

    def hilbert_by_hand():
        for m in (3, 4):
            pins.test_hilbert_noda_matrix_written_out_by_hand(m)
        return True

    def hilbert_hetero():
        pins.test_hilbert_noda_hetero_applies_the_matrix_to_stack_2()
        return True

    def hilbert_sinusoid():
        pins.test_hilbert_noda_of_a_sinusoid_is_the_cosine_times_the_kernel_gain(0.7)
        return True

    def ft_ht_tone():
        pins.test_ft_and_ht_async_spectra_agree_on_a_single_tone(513, 20)
        return True

    for name, fn in [("brute_homo", brute_homo), ("brute_hetero_odd", brute_hetero_odd),
                     ("brute_user_ref", brute_user_ref), ("parseval_even", parseval_even),
                     ("pearson_diag", pearson_diag), ("closed_form", closed_form),
                     ("dft_numpy", dft_numpy), ("sigma_numpy", sigma_numpy),
                     ("interp_numpy", interp_numpy), ("interp_t_numpy", interp_t_numpy),
                     ("spline_cubic", spline_cubic), ("spline_dense", spline_dense),
                     ("interp_dyn_out", interp_dyn_out), ("hilbert_by_hand", hilbert_by_hand),
                     ("hilbert_hetero", hilbert_hetero), ("hilbert_sinusoid", hilbert_sinusoid),
                     ("ft_ht_tone", ft_ht_tone)]:
        check(name, fn)
    return failed


def test_unmutated_oracle_passes_battery():
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    lib = oracle.compile_source(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    with oracle.use_library(lib):
        failed = _battery()
    assert failed, f"planted mistake {name} passed every pin"
