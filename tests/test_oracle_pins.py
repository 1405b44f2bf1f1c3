"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Nothing here re-types the oracle's own formulas: each check uses a second,
independent route (a time-domain kernel, numpy's FFT, Parseval's identity, a
closed form for sinusoidal bands, an exact invariance, the Noda sign rules or
the R index expression of the paper's FFT snippet).  A dropped term, a wrong
sign or index, a transposed operand or a wrong weight in the oracle fails at
least one of them.

The pins of each oracle function (``oracle/__init__.py``):

  num_freq, weight          test_kept_frequencies_follow_r_index_expression,
                            test_parseval_links_frequency_sum_to_covariance
  default_norm              test_pearson_diagonal_is_m_over_pi_for_odd_m,
                            test_closed_form_sinusoidal_bands, test_norm_override_and_constant_variable
  scale_factor, sigma       test_reference_and_sigma_match_numpy, test_amplitude_scaling,
                            test_norm_override_and_constant_variable
  reference_mean, dynamic   test_reference_and_sigma_match_numpy, test_baseline_offset_invariance
  dft                       test_dft_is_numpy_fft_truncated
  cross_spectrum, corr2d    test_brute_force_*, test_parseval_*, test_closed_form_*,
                            test_fig1_*, the invariance tests, test_noda_sign_rules_*,
                            test_row_subset_matches_full, test_sampled_columns_give_those_entries
  interp_linear (y_out)     test_interp_matches_numpy_interp_and_endpoints,
                            test_interp_reproduces_linear_functions_and_subtracts_reference
  interp_linear (dyn_out)   test_interp_dyn_out_is_the_dynamic_spectrum_of_the_correlation
  interp_perturbation       test_perturbation_interp_* (linear), test_spline_* (spline)
  reduce_map                test_reduce_map_is_decimation
  hilbert_noda              test_hilbert_noda_matrix_written_out_by_hand,
                            test_hilbert_noda_hetero_applies_the_matrix_to_stack_2,
                            test_hilbert_noda_of_a_sinusoid_is_the_cosine_times_the_kernel_gain,
                            test_ft_and_ht_async_spectra_agree_on_a_single_tone,
                            test_odd_m_ft_equals_ht_synchronous_up_to_m_over_pi,
                            test_hilbert_noda_async_sign_agrees_with_ft
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _furanmale():
    rows = []
    with open(os.path.join(GOLDEN, "furanmale_excerpt.txt")) as f:
        for line in f:
            if line.startswith("#") or line.startswith("nu"):
                continue
            vals = line.split()
            if vals:
                rows.append([float(v) for v in vals[1:]])
    return np.array(rows, dtype=np.float32)


def _brute(y1, y2=None, ref1=None, ref2=None, alpha=0.0, norm=None):
    """Time-domain evaluation of the half-spectrum correlation.

    With d = y - ref, summing w_omega e^{i 2 pi omega (k - j)/m} over the kept
    frequencies gives, for each pair of perturbation steps (j, k), the kernels
      c(j,k) = 1 + 2 sum_{omega=1}^{K} cos(2 pi omega (k - j)/m)
      s(j,k) =     2 sum_{omega=1}^{K} sin(2 pi omega (k - j)/m)
    and Phi + i Psi = norm * sum_{j,k} d1(j) d2(k) (c + i s).  No DFT is formed.
    """
    y1 = y1.astype(np.float64)
    m, n1 = y1.shape
    homo = y2 is None
    y2 = y1 if homo else y2.astype(np.float64)
    n2 = y2.shape[1]
    r1 = y1.mean(axis=0) if ref1 is None else np.asarray(ref1, np.float64)
    if homo:
        r2 = r1
    else:
        r2 = y2.mean(axis=0) if ref2 is None else np.asarray(ref2, np.float64)
    d1 = y1 - r1
    d2 = y2 - r2
    K = (m - 1) // 2
    c = np.empty((m, m))
    s = np.empty((m, m))
    for j in range(m):
        for k in range(m):
            cc, ss = 1.0, 0.0
            for w in range(1, K + 1):
                ang = 2.0 * math.pi * w * (k - j) / m
                cc += 2.0 * math.cos(ang)
                ss += 2.0 * math.sin(ang)
            c[j, k], s[j, k] = cc, ss
    if norm is None:
        norm = 1.0 / (math.pi * (m - 1))
    phi = np.zeros((n1, n2))
    psi = np.zeros((n1, n2))
    for a in range(n1):
        for b in range(n2):
            pr = pi = 0.0
            for j in range(m):
                for k in range(m):
                    pr += d1[j, a] * d2[k, b] * c[j, k]
                    pi += d1[j, a] * d2[k, b] * s[j, k]
            phi[a, b] = norm * pr
            psi[a, b] = norm * pi
    if alpha > 0:
        sd1 = np.sqrt((d1 ** 2).sum(axis=0) / (m - 1))
        sd2 = np.sqrt((d2 ** 2).sum(axis=0) / (m - 1))
        f = np.outer(sd1 ** -alpha, sd2 ** -alpha)
        phi, psi = phi * f, psi * f
    return phi, psi


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- frequencies

@pytest.mark.parametrize("m", range(2, 14))
def test_kept_frequencies_follow_r_index_expression(m):
    """Sec. 4.2 FFT snippet: fft(x)[1:(NROW - 1) %/% 2 + 1] (R precedence: ':' first).

    The snippet picks frequencies with repetition; the product with Conj() then
    sums every pick, so the pick count is the weight.  For even m that count is
    the weight exactly.  For odd m the expression picks the top bin K = (m-1)/2
    once, while the text (every omega != 0 used twice) and the Hermitian pairing
    of K with m-K (Eq. symmeFT) count it twice; the text's reading is taken."""
    idx_1based = [(k // 2) + 1 for k in range(1, m)]  # (1:(m-1)) %/% 2 + 1
    counts = {}
    for i in idx_1based:
        counts[i - 1] = counts.get(i - 1, 0) + 1
    K = (m - 1) // 2
    assert sorted(counts) == list(range(oracle.num_freq(m)))
    for omega, cnt in counts.items():
        if m % 2 == 1 and omega == K and K > 0:
            assert cnt == 1 and oracle.weight(omega) == 2.0
        else:
            assert oracle.weight(omega) == cnt
    if m % 2 == 0:
        assert m // 2 not in counts  # Nyquist bin never used


# ----------------------------------------------------------------------- DFT

@pytest.mark.parametrize("m", [2, 3, 5, 8, 11, 16, 31, 64])
def test_dft_is_numpy_fft_truncated(m):
    rng = np.random.default_rng(m)
    d = rng.standard_normal((m, 7))
    Y = oracle.dft(d)
    ref = np.fft.fft(d, axis=0)[: (m - 1) // 2 + 1].T
    assert np.max(np.abs(Y - ref)) < 1e-12 * max(1.0, np.abs(ref).max())


def test_reference_and_sigma_match_numpy():
    y = workloads.random_stack(9, 13, seed=3, offset=2.0)
    ref = oracle.reference_mean(y)
    assert np.allclose(ref, y.astype(np.float64).mean(axis=0), rtol=0, atol=1e-14)
    d = oracle.dynamic(y, ref)
    assert np.array_equal(d, y.astype(np.float64) - ref)
    assert np.allclose(oracle.sigma(d), y.astype(np.float64).std(axis=0, ddof=1), rtol=1e-13)


# ------------------------------------------------------------- brute force

@pytest.mark.parametrize("m,n1,n2", [(2, 3, 3), (3, 4, 4), (4, 5, 3), (5, 6, 6), (8, 4, 5),
                                     (9, 8, 8)])
def test_brute_force_time_domain(m, n1, n2):
    y1 = workloads.random_stack(m, n1, seed=10 + m, offset=0.5)
    phi, psi, _, _ = oracle.corr2d(y1)
    bphi, bpsi = _brute(y1)
    assert np.max(np.abs(phi - bphi)) < 1e-13 * max(1, np.abs(bphi).max())
    assert np.max(np.abs(psi - bpsi)) < 1e-13 * max(1, np.abs(bphi).max())
    y2 = workloads.random_stack(m, n2, seed=20 + m, offset=-1.0)
    phi, psi, _, _ = oracle.corr2d(y1, y2, alpha=0.5)
    bphi, bpsi = _brute(y1, y2, alpha=0.5)
    assert _rel(phi, bphi) < 1e-13 and np.max(np.abs(psi - bpsi)) <= 1e-13 * np.abs(bphi).max()


def test_brute_force_user_reference_and_norm():
    y1 = workloads.random_stack(7, 5, seed=4)
    y2 = workloads.random_stack(7, 6, seed=5)
    ref1, ref2 = y1[0].copy(), y2[-1].copy()  # first / last spectrum as reference
    phi, psi, s1, s2 = oracle.corr2d(y1, y2, ref1=ref1, ref2=ref2, norm=0.25, alpha=1.0)
    bphi, bpsi = _brute(y1, y2, ref1=ref1, ref2=ref2, norm=0.25, alpha=1.0)
    assert _rel(phi, bphi) < 1e-13 and _rel(psi, bpsi) < 1e-13
    # Eq. stdev with the chosen reference, not re-centred on the mean
    assert np.allclose(s1, np.sqrt(((y1.astype(np.float64) - ref1.astype(np.float64)) ** 2).sum(0) / 6), rtol=1e-13)


def test_brute_force_paper_excerpt():
    """Real data printed in the paper (FuranMale, 6 temperatures x 5 wavenumbers)."""
    y = _furanmale()
    assert y.shape == (6, 5)
    phi, psi, _, _ = oracle.corr2d(y)
    bphi, bpsi = _brute(y)
    assert _rel(phi, bphi) < 1e-12
    assert np.max(np.abs(psi - bpsi)) < 1e-12 * np.abs(bphi).max()
    assert np.all(np.diag(phi) > 0)


# ---------------------------------------------------------------- Parseval

@pytest.mark.parametrize("m", [3, 4, 7, 10, 33, 64])
def test_parseval_links_frequency_sum_to_covariance(m):
    """sum over all m bins of Y1 conj(Y2) = m sum_j d1 d2; pairing bins omega and m-omega
    (Eq. symmeFT) leaves pi (m-1) Phi = m sum_j d1 d2 - [m even] Y1(m/2) Y2(m/2)."""
    y1 = workloads.random_stack(m, 11, seed=m)
    y2 = workloads.random_stack(m, 9, seed=m + 1, offset=3.0)
    phi, _, _, _ = oracle.corr2d(y1, y2)
    d1 = y1.astype(np.float64) - y1.astype(np.float64).mean(0)
    d2 = y2.astype(np.float64) - y2.astype(np.float64).mean(0)
    rhs = m * d1.T @ d2
    if m % 2 == 0:
        alt = (-1.0) ** np.arange(m)
        rhs -= np.outer(alt @ d1, alt @ d2)
    assert _rel(math.pi * (m - 1) * phi, rhs) < 1e-12


@pytest.mark.parametrize("m", [5, 9, 15])
def test_odd_m_ft_equals_ht_synchronous_up_to_m_over_pi(m):
    """Sec. 2: FT and HT give the same spectra; exactly Phi_FT = (m/pi) Phi_HT for odd m."""
    y = workloads.random_stack(m, 6, seed=m)
    phi, _, _, _ = oracle.corr2d(y)
    d = oracle.dynamic(y, oracle.reference_mean(y))
    hphi, _ = oracle.hilbert_noda(d, d)
    assert _rel(phi, (m / math.pi) * hphi) < 1e-12


def test_pearson_diagonal_is_m_over_pi_for_odd_m():
    m = 13
    y = workloads.random_stack(m, 10, seed=1, offset=5.0)
    phi, psi, _, _ = oracle.corr2d(y, alpha=1.0)
    assert np.allclose(np.diag(phi), m / math.pi, rtol=1e-12)
    assert np.allclose(np.diag(psi), 0.0, atol=1e-12)


# ------------------------------------------------------------- closed form

@pytest.mark.parametrize("m", [3, 8, 11, 64])
def test_closed_form_sinusoidal_bands(m):
    """t_j = j/m, y = sum_b L_b(nu) a_b sin(2 pi t + phi_b): only bin 1 is non-zero,
    Y_b(1) = a_b m e^{i phi_b}/(2i), so Phi + i Psi = norm (m^2/2) sum_bc L_b L_c a_b a_c
    e^{i (phi_b - phi_c)}."""
    n = 64
    phases = [0.0, 30.0, 60.0, 90.0]
    y, c, g, a = workloads.sinusoid_bands(m, n, phases, seed=7)
    phi, psi, _, _ = oracle.corr2d(y)
    nu = np.arange(n, dtype=np.float64)
    L = 1.0 / (1.0 + ((nu[None, :] - c[:, None]) / g[:, None]) ** 2)  # bands x n
    ph = np.deg2rad(phases)
    E = (a[:, None] * L) * np.exp(1j * ph)[:, None]  # bands x n
    Z = (m * m / 2.0) * (E.sum(0)[:, None] * np.conj(E.sum(0))[None, :])
    Z /= math.pi * (m - 1)
    # inputs are rounded to FP32, so agreement is at FP32 level
    assert _rel(phi, Z.real) < 3e-6
    assert np.max(np.abs(psi - Z.imag)) < 3e-6 * np.abs(Z).max()


def test_fig1_cases_pure_sync_and_pure_async():
    """Fig. 1 (a): identical response -> Psi = 0; (b) pi/2 lag -> Phi = 0 (Sec. 2)."""
    m = 16
    t = np.arange(m) / m
    s0 = np.sin(2 * np.pi * t)
    s90 = np.sin(2 * np.pi * t + np.pi / 2)
    y = np.stack([s0, s0, s90], axis=1).astype(np.float32)
    phi, psi, _, _ = oracle.corr2d(y)
    scale = abs(phi[0, 0])
    assert abs(psi[0, 1]) < 1e-7 * scale and phi[0, 1] > 0
    assert abs(phi[0, 2]) < 1e-7 * scale
    # column 2 leads column 0 by 90 deg: Psi(2, 0) > 0 (Noda rule 3)
    assert psi[2, 0] > 0.99 * scale and psi[0, 2] < 0


# --------------------------------------------------------------- invariants

def test_homo_symmetry_and_autopeaks():
    y = workloads.c1()
    phi, psi, _, _ = oracle.corr2d(y)
    assert np.array_equal(phi, phi.T)
    assert np.array_equal(psi, -psi.T)
    assert np.all(np.diag(psi) == 0.0)
    assert np.all(np.diag(phi) >= 0.0)


def _quantised(m, n, seed):
    """Values on a 2^-10 grid in [-4, 4): adding 8 stays exact in FP32."""
    rng = np.random.default_rng(seed)
    return (rng.integers(-4096, 4096, (m, n)) / 1024.0).astype(np.float32)


def test_baseline_offset_invariance():
    y = _quantised(12, 9, seed=2)
    base = np.float32(8.0) + np.arange(9, dtype=np.float32)  # per-variable constant
    p0, q0, _, _ = oracle.corr2d(y)
    p1, q1, _, _ = oracle.corr2d(y + base)
    assert _rel(p1, p0) < 1e-13 and np.max(np.abs(q1 - q0)) < 1e-13 * np.abs(p0).max()


@pytest.mark.parametrize("m,shift", [(10, 3), (11, 4)])
def test_circular_shift_invariance(m, shift):
    y = workloads.random_stack(m, 8, seed=m)
    p0, q0, _, _ = oracle.corr2d(y)
    p1, q1, _, _ = oracle.corr2d(np.roll(y, shift, axis=0))
    assert _rel(p1, p0) < 1e-12 and np.max(np.abs(q1 - q0)) < 1e-12 * np.abs(p0).max()


def test_time_reversal_flips_async_sign():
    y = workloads.random_stack(9, 8, seed=9)
    p0, q0, _, _ = oracle.corr2d(y)
    p1, q1, _, _ = oracle.corr2d(y[::-1].copy())
    assert _rel(p1, p0) < 1e-12 and _rel(q1, -q0) < 1e-12


def test_hetero_swap_and_self_hetero_equals_homo():
    y1 = workloads.random_stack(10, 7, seed=1)
    y2 = workloads.random_stack(10, 5, seed=2)
    p12, q12, _, _ = oracle.corr2d(y1, y2)
    p21, q21, _, _ = oracle.corr2d(y2, y1)
    assert _rel(p21, p12.T) < 1e-13 and _rel(q21, -q12.T) < 1e-13
    ph, qh, _, _ = oracle.corr2d(y1)
    ps, qs, _, _ = oracle.corr2d(y1, y1.copy())
    assert np.array_equal(ph, ps) and np.array_equal(qh, qs)


def test_amplitude_scaling():
    y = _quantised(8, 6, seed=5)
    p0, q0, _, _ = oracle.corr2d(y)
    p1, q1, _, _ = oracle.corr2d(y * np.float32(4.0))
    assert _rel(p1, 16 * p0) < 1e-14 and _rel(q1, 16 * q0) < 1e-14
    # Pearson scaling removes the amplitude (Eq. pearsonsyn)
    p2, q2, _, _ = oracle.corr2d(y, alpha=1.0)
    p3, q3, _, _ = oracle.corr2d(y * np.float32(4.0), alpha=1.0)
    assert _rel(p3, p2) < 1e-13 and _rel(q3, q2) < 1e-13
    # Pareto (alpha = 0.5) leaves a factor c^2 / c
    p4, _, _, _ = oracle.corr2d(y, alpha=0.5)
    p5, _, _, _ = oracle.corr2d(y * np.float32(4.0), alpha=0.5)
    assert _rel(p5, 4 * p4) < 1e-13


def test_norm_override_and_constant_variable():
    y = workloads.random_stack(6, 5, seed=8)
    y[:, 2] = 3.25  # constant variable: sigma = 0
    p0, q0, s, _ = oracle.corr2d(y)
    p1, _, _, _ = oracle.corr2d(y, norm=1.0)
    assert _rel(p1, p0 * math.pi * 5) < 1e-13
    assert s[2] == 0.0
    p2, q2, _, _ = oracle.corr2d(y, alpha=0.5)
    assert np.all(p2[2, :] == 0) and np.all(p2[:, 2] == 0) and np.all(q2[2, :] == 0)
    assert np.all(np.isfinite(p2))


def test_row_subset_matches_full():
    y = workloads.random_stack(10, 40, seed=3)
    p, q, _, _ = oracle.corr2d(y)
    rows = np.array([0, 5, 17, 39], np.int32)
    ps, qs, _, _ = oracle.corr2d(y, rows=rows, nthreads=2)
    assert np.array_equal(ps, p[rows]) and np.array_equal(qs, q[rows])


@pytest.mark.parametrize("alpha", [0.0, 0.5])
def test_sampled_columns_give_those_entries(alpha):
    """Reference, centering, sigma (one per spectral variable, reading R5) and
    the DFT act on each spectral variable alone, so correlating the sampled
    columns of the stacks gives exactly the sampled entries of the full maps.
    A per-spectrum sigma, or a reference shared between variables, breaks it.
    (The GPU test of the full batch of 512 problems checks sampled outputs this way.)"""
    y1 = workloads.random_stack(23, 90, seed=61, offset=2.0)
    y2 = workloads.random_stack(23, 70, seed=62, offset=-1.0)
    rows = np.array([0, 7, 44, 89])
    cols = np.array([0, 3, 31, 32, 68, 69])
    p, q, _, _ = oracle.corr2d(y1, y2, alpha=alpha)
    ps, qs, _, _ = oracle.corr2d(np.ascontiguousarray(y1[:, rows]),
                                 np.ascontiguousarray(y2[:, cols]), alpha=alpha)
    assert np.array_equal(ps, p[np.ix_(rows, cols)]) and np.array_equal(qs, q[np.ix_(rows, cols)])
    ph, qh, _, _ = oracle.corr2d(y1, alpha=alpha)
    ps, qs, _, _ = oracle.corr2d(np.ascontiguousarray(y1[:, rows]),
                                 np.ascontiguousarray(y1[:, cols]), alpha=alpha)
    assert np.array_equal(ps, ph[np.ix_(rows, cols)]) and np.array_equal(qs, qh[np.ix_(rows, cols)])


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.corr2d(np.zeros((1, 4), np.float32))  # m < 2: Norm divides by m - 1
    with pytest.raises(ValueError):
        oracle.corr2d(np.zeros((3, 4), np.float32), np.zeros((4, 4), np.float32))


# ---------------------------------------------------------- Noda sign rules

def test_noda_sign_rules_on_phase_lagged_bands():
    """Sec. 3 rules 1-4 on the 0/30/60 deg three-band input: at band centres
    sign(Phi) = sign(cos(dphi)) and sign(Psi(nu_b, nu_c)) = sign(sin(phi_b - phi_c))."""
    y, c, g, a = workloads.sinusoid_bands(11, 500, [0.0, 30.0, 60.0], seed=0, noise=0.01,
                                          centers=[100.0, 250.0, 400.0], widths=[8, 8, 8])
    phi, psi, _, _ = oracle.corr2d(y)
    ph = np.deg2rad([0.0, 30.0, 60.0])
    idx = [100, 250, 400]
    for b in range(3):
        for cc in range(3):
            if b == cc:
                continue
            assert np.sign(phi[idx[b], idx[cc]]) == np.sign(math.cos(ph[b] - ph[cc]))
            assert np.sign(psi[idx[b], idx[cc]]) == np.sign(math.sin(ph[b] - ph[cc]))


def test_hilbert_noda_async_sign_agrees_with_ft():
    """Eq. HilbNoda: antisymmetric matrix -> homo Psi_HT antisymmetric; its sign pattern
    on lagged bands matches the FT approach (rule 3)."""
    y, c, g, a = workloads.sinusoid_bands(32, 60, [0.0, 45.0], seed=1,
                                          centers=[15.0, 45.0], widths=[4, 4])
    d = oracle.dynamic(y, oracle.reference_mean(y))
    hphi, hpsi = oracle.hilbert_noda(d, d)
    assert np.max(np.abs(hpsi + hpsi.T)) < 1e-13 * np.abs(hphi).max()
    _, psi, _, _ = oracle.corr2d(y)
    assert np.sign(hpsi[45, 15]) == np.sign(psi[45, 15]) == 1.0


# Eq. HilbNoda worked out by hand for m = 3 and m = 4: the entries of pi * N
# (row j, column k), pi N_jk = 1/(k - j) off the diagonal, 0 on it.
_F = Fraction
_PI_TIMES_N = {
    3: [[_F(0), _F(1), _F(1, 2)],
        [_F(-1), _F(0), _F(1)],
        [_F(-1, 2), _F(-1), _F(0)]],
    4: [[_F(0), _F(1), _F(1, 2), _F(1, 3)],
        [_F(-1), _F(0), _F(1), _F(1, 2)],
        [_F(-1, 2), _F(-1), _F(0), _F(1)],
        [_F(-1, 3), _F(-1, 2), _F(-1), _F(0)]],
}


@pytest.mark.parametrize("m", [3, 4])
def test_hilbert_noda_matrix_written_out_by_hand(m):
    """Unit-impulse dynamic spectra pick single terms of Eqs. disHTsyn, disHT and
    disHTasyn: with d1 = d2 = the m x m identity (variable a is an impulse at step a),
    (m - 1) Phi = I and (m - 1) Psi[a, b] = sum_j d1(j, a) sum_k N_jk d2(k, b) = N_ab.
    Pins the 1/pi of Eq. HilbNoda, the 1/(m - 1) of both spectra and the orientation
    of N (a transposed N, or N applied to stack 1, flips every sign)."""
    eye = np.eye(m)
    phi, psi = oracle.hilbert_noda(eye, eye)
    assert np.array_equal((m - 1) * phi, eye)
    pin = np.array([[float(v) for v in row] for row in _PI_TIMES_N[m]])
    assert np.max(np.abs(math.pi * (m - 1) * psi - pin)) < 1e-14


def test_hilbert_noda_hetero_applies_the_matrix_to_stack_2():
    """Hetero Eq. disHTasyn: Psi = d1^T (N d2) / (m - 1), N acting on the perturbation
    steps of stack 2.  Exact rational evaluation with the hand-written pi N of m = 4
    and small integer dynamic spectra."""
    m = 4
    d1 = np.array([[1, 0, 2], [0, -1, 1], [3, 1, 0], [-2, 2, -1]], dtype=np.float64)
    d2 = np.array([[2, -1], [1, 0], [0, 3], [-1, 1]], dtype=np.float64)
    piN = _PI_TIMES_N[m]
    want_psi = [[sum(_F(int(d1[j, a])) * piN[j][k] * _F(int(d2[k, b]))
                     for j in range(m) for k in range(m)) for b in range(2)] for a in range(3)]
    want_phi = [[sum(_F(int(d1[j, a])) * _F(int(d2[j, b])) for j in range(m))
                 for b in range(2)] for a in range(3)]
    phi, psi = oracle.hilbert_noda(d1, d2)
    assert np.allclose((m - 1) * phi, np.array(want_phi, dtype=np.float64), rtol=0, atol=1e-14)
    assert np.allclose(math.pi * (m - 1) * psi, np.array(want_psi, dtype=np.float64), rtol=0,
                       atol=1e-13)
    # stack 2 swapped in: N then acts on the other stack, i.e. the transposed pairing
    _, psi21 = oracle.hilbert_noda(d2, d1)
    assert np.allclose(psi21, -psi.T, rtol=0, atol=1e-14)


@pytest.mark.parametrize("w", [0.3, 0.7, 1.5, 2.5])
def test_hilbert_noda_of_a_sinusoid_is_the_cosine_times_the_kernel_gain(w):
    """Eq. HT: with the paper's (1/pi) PV int y(t')/(t' - t) dt', the Hilbert transform
    of sin(w t) is cos(w t).  The discrete kernel of Eq. HilbNoda, summed over the lags
    l = k - j on both sides of a step, gives
      z(t_j) = (2/pi) cos(w j + p) sum_{l=1}^{L} sin(w l)/l
    for y = sin(w k + p), and the sawtooth Fourier series sum_{l>=1} sin(w l)/l =
    (pi - w)/2 (0 < w < 2 pi) leaves z = (1 - w/pi) cos(w j + p) up to the series tail
    beyond the window, |tail| <= 1/((L + 1) sin(w/2)).  An impulse d1 at the centre
    step j0 reads z(t_j0) out of Psi."""
    m, j0 = 2001, 1000
    L = min(j0, m - 1 - j0)
    k = np.arange(m)
    d2 = np.stack([np.sin(w * k + 0.3), np.cos(w * k - 1.1)], axis=1)  # cos = sin(. + pi/2)
    d1 = np.zeros((m, 1))
    d1[j0, 0] = 1.0
    _, psi = oracle.hilbert_noda(d1, d2)
    z = (m - 1) * psi[0]
    want = (1.0 - w / math.pi) * np.array([np.cos(w * j0 + 0.3), -np.sin(w * j0 - 1.1)])
    bound = (2.0 / math.pi) / ((L + 1) * math.sin(w / 2.0))
    assert np.max(np.abs(z - want)) <= bound


@pytest.mark.parametrize("m,f", [(513, 20), (1025, 40)])
def test_ft_and_ht_async_spectra_agree_on_a_single_tone(m, f):
    """Sec. 2: the FT and HT approaches give the same spectra.  For bands varying as
    sin(2 pi f j/m + phase) (f whole periods in the window) the FT's Psi is the closed
    form Norm (m^2/2) a b sin(phase difference) and, far from the window edges, the HT's
    is (m/2) a b (1 - w/pi) sin(...) / (m - 1) with w = 2 pi f/m (the previous pin): so
    Psi_FT / Psi_HT = (m/pi) / (1 - w/pi) up to the edges' share, ~1/(m w) (below 1 %
    here), while Phi_FT / Phi_HT = m/pi exactly (odd m)."""
    t = np.arange(m)
    nu = np.arange(40.0)
    L1 = 1.0 / (1.0 + ((nu - 10.0) / 4.0) ** 2)
    L2 = 1.0 / (1.0 + ((nu - 30.0) / 4.0) ** 2)
    y = (np.outer(np.sin(2 * np.pi * f * t / m), L1) +
         np.outer(np.sin(2 * np.pi * f * t / m + np.deg2rad(50.0)), L2)).astype(np.float32)
    phi, psi, _, _ = oracle.corr2d(y)
    d = oracle.dynamic(y, oracle.reference_mean(y))
    hphi, hpsi = oracle.hilbert_noda(d, d)
    w = 2 * np.pi * f / m
    gain = (m / math.pi) / (1.0 - w / math.pi)
    assert abs(psi[30, 10] / hpsi[30, 10] / gain - 1.0) < 0.02
    assert psi[30, 10] > 0 and hpsi[30, 10] > 0  # band 2 leads band 1 (rule 3)
    assert abs(phi[30, 10] / hphi[30, 10] / (m / math.pi) - 1.0) < 1e-12


# ------------------------------------------------------------ interpolation

def test_interp_matches_numpy_interp_and_endpoints():
    rng = np.random.default_rng(0)
    x = workloads.jittered_axis(130, 0.0, 99.0, rng)
    y = workloads.random_stack(4, 130, seed=1)
    out, dyn = oracle.interp_linear(x, y, 100, ref=np.zeros(100, np.float32))
    grid = np.linspace(0.0, 99.0, 100)
    for j in range(4):
        assert np.allclose(out[j], np.interp(grid, x, y[j].astype(np.float64)), rtol=0,
                           atol=1e-12)
    assert np.array_equal(out[:, 0], y[:, 0].astype(np.float64))
    assert np.array_equal(out[:, -1], y[:, -1].astype(np.float64))
    assert np.array_equal(dyn, out)


def test_interp_reproduces_linear_functions_and_subtracts_reference():
    rng = np.random.default_rng(3)
    x = workloads.jittered_axis(50, -2.0, 7.0, rng)
    y = np.stack([1.5 + 0.25 * x, -3.0 * x]).astype(np.float32)
    out, _ = oracle.interp_linear(x.astype(np.float64), y.astype(np.float64).astype(np.float32), 37)
    grid = np.linspace(-2.0, 7.0, 37)
    # FP32 inputs: linear up to the rounding of the knots
    assert np.allclose(out[0], 1.5 + 0.25 * grid, atol=5e-6)
    assert np.allclose(out[1], -3.0 * grid, atol=5e-5)
    ref = np.linspace(0, 1, 37).astype(np.float32)
    out2, dyn = oracle.interp_linear(x, y, 37, ref=ref)
    assert np.array_equal(dyn, out2 - ref.astype(np.float64))


def test_interp_dyn_out_is_the_dynamic_spectrum_of_the_correlation():
    """Eq. dynspec after the spectral-axis preprocessing: correlating dyn_out as the
    stack (user reference 0) equals correlating y_out against the reference itself;
    the reference subtraction inside oracle.corr2d is pinned by the brute force of a
    second formula (test_brute_force_user_reference_and_norm).  dyn_out of the
    reference row itself is zero."""
    rng = np.random.default_rng(8)
    x = workloads.jittered_axis(90, 0.0, 40.0, rng)
    y = workloads.random_stack(7, 90, seed=9, offset=1.5)
    out0, _ = oracle.interp_linear(x, y, 64)
    ref = out0[2].astype(np.float32)
    out, dyn = oracle.interp_linear(x, y, 64, ref=ref)
    zero = np.zeros(64, np.float32)
    pa, qa, _, _ = oracle.corr2d(dyn.astype(np.float32), ref1=zero)
    pb, qb, _, _ = oracle.corr2d(out.astype(np.float32), ref1=ref)
    assert _rel(pa, pb) < 1e-6 and np.abs(qa - qb).max() < 1e-6 * np.abs(pb).max()
    assert np.abs(dyn[2]).max() <= 1e-6 * np.abs(out[2]).max()


def test_perturbation_interp_matches_numpy_per_variable():
    """Sec. 4.2: TIME <- seq(min(Time), max(Time), length.out = N), each column
    evaluated through approxfun over Time (library special case: numpy.interp)."""
    rng = np.random.default_rng(4)
    time = np.sort(rng.uniform(0, 10, 12))
    y = workloads.random_stack(12, 7, seed=2)
    out = oracle.interp_perturbation(time, y, 16)
    grid = np.linspace(time[0], time[-1], 16)
    for v in range(7):
        assert np.allclose(out[:, v], np.interp(grid, time, y[:, v].astype(np.float64)),
                           rtol=0, atol=1e-12)
    assert np.array_equal(out[0], y[0].astype(np.float64))
    assert np.array_equal(out[-1], y[-1].astype(np.float64))


def test_perturbation_interp_identity_and_linear_signal():
    time = np.arange(9, dtype=np.float64) * 0.5
    y = workloads.random_stack(9, 5, seed=3)
    assert np.allclose(oracle.interp_perturbation(time, y, 9), y.astype(np.float64), atol=1e-15)
    t = np.array([0.0, 0.3, 1.1, 2.0, 4.5])
    lin = (2.0 + 3.0 * t)[:, None] * np.ones((1, 4))
    out = oracle.interp_perturbation(t, lin.astype(np.float32), 10)
    assert np.allclose(out, (2.0 + 3.0 * np.linspace(0, 4.5, 10))[:, None], atol=1e-5)
    with pytest.raises(ValueError):
        oracle.interp_perturbation(np.array([0.0, 1.0, 1.0]), np.zeros((3, 2), np.float32), 4)


def _grid(t, N):
    g = t[0] + np.arange(N) * ((t[-1] - t[0]) / (N - 1))
    g[-1] = t[-1]
    return g


def test_spline_reproduces_cubic_polynomials():
    """fmm end conditions (reading R13): the third derivative at each end is that
    of the cubic through four end points, so any cubic is reproduced exactly --
    natural or zero-third-derivative ends would bend it.  Dyadic knots and
    coefficients keep the FP32 inputs exact."""
    t = np.array([0.0, 0.5, 1.25, 2.0, 3.5, 4.0, 5.75, 6.0])
    coeffs = [(1.0, 0.0, 0.0, 0.0), (0.5, -1.25, 0.75, 2.0), (-0.25, 2.0, 0.0, -1.0),
              (0.0, 1.5, -0.5, 0.25), (0.0, 0.0, 3.0, 1.0)]
    y = np.stack([np.polyval(c, t) for c in coeffs], axis=1)
    assert np.array_equal(y.astype(np.float32).astype(np.float64), y)
    out = oracle.interp_perturbation(t, y.astype(np.float32), 29, method="spline")
    g = _grid(t, 29)
    for v, c in enumerate(coeffs):
        assert np.allclose(out[:, v], np.polyval(c, g), rtol=0, atol=1e-12 * 300)


def test_spline_with_three_and_two_points():
    """m = 3: zero end third derivatives leave the interpolating parabola;
    m = 2: the line (fmm's short-input cases, reading R13)."""
    t = np.array([1.0, 1.75, 3.0])
    y = np.array([[2.0, -1.0], [0.5, 4.0], [3.25, 0.0]], np.float32)
    out = oracle.interp_perturbation(t, y, 11, method="spline")
    g = _grid(t, 11)
    for v in range(2):
        par = np.polyfit(t, y[:, v].astype(np.float64), 2)
        assert np.allclose(out[:, v], np.polyval(par, g), atol=1e-12)
    t2 = np.array([0.0, 2.0])
    y2 = np.array([[1.0], [5.0]], np.float32)
    assert np.allclose(oracle.interp_perturbation(t2, y2, 5, method="spline")[:, 0],
                       1.0 + 2.0 * _grid(t2, 5), atol=1e-14)


def _dense_fmm_spline(t, y, g):
    """The same spline written as one dense linear system in the 4 (m-1)
    polynomial coefficients p_i(x) = a + b (x - t_i) + c (x - t_i)^2 + d (x - t_i)^3:
    interpolation at both ends of every interval, matching first and second
    derivatives at inner knots, and 6 d on the first / last interval equal to the
    third derivative of numpy.polyfit's cubic through the four end points."""
    m = len(t)
    nu = 4 * (m - 1)
    A = np.zeros((nu, nu))
    b = np.zeros(nu)
    r = 0
    for i in range(m - 1):
        h = t[i + 1] - t[i]
        A[r, 4 * i] = 1.0; b[r] = y[i]; r += 1
        A[r, 4 * i:4 * i + 4] = [1.0, h, h * h, h ** 3]; b[r] = y[i + 1]; r += 1
    for i in range(m - 2):
        h = t[i + 1] - t[i]
        A[r, 4 * i:4 * i + 4] = [0.0, 1.0, 2 * h, 3 * h * h]; A[r, 4 * (i + 1) + 1] = -1.0; r += 1
        A[r, 4 * i:4 * i + 4] = [0.0, 0.0, 2.0, 6 * h]; A[r, 4 * (i + 1) + 2] = -2.0; r += 1
    A[r, 3] = 6.0; b[r] = 6.0 * np.polyfit(t[:4], y[:4], 3)[0]; r += 1
    A[r, 4 * (m - 2) + 3] = 6.0; b[r] = 6.0 * np.polyfit(t[-4:], y[-4:], 3)[0]; r += 1
    coef = np.linalg.solve(A, b)
    s = np.clip(np.searchsorted(t, g, side="left") - 1, 0, m - 2)
    dx = g - t[s]
    a, bb, c, d = (coef[4 * s + k] for k in range(4))
    return a + bb * dx + c * dx ** 2 + d * dx ** 3


@pytest.mark.parametrize("m", [4, 6, 11])
def test_spline_matches_dense_piecewise_cubic_solve(m):
    rng = np.random.default_rng(m)
    t = np.cumsum(rng.uniform(0.2, 1.5, m))
    y = workloads.random_stack(m, 6, seed=m + 40)
    out = oracle.interp_perturbation(t, y, 37, method="spline")
    g = _grid(t, 37)
    for v in range(6):
        ref = _dense_fmm_spline(t, y[:, v].astype(np.float64), g)
        assert np.allclose(out[:, v], ref, rtol=0, atol=1e-9 * max(1.0, np.abs(ref).max()))


def test_spline_knots_and_fourth_order_convergence():
    """The grid hits every knot when N = 2m - 1 on equidistant knots: values equal
    y exactly there; on a smooth signal the error falls ~16x per halving of h."""
    t = np.arange(9, dtype=np.float64) * 0.25
    y = workloads.random_stack(9, 4, seed=77)
    out = oracle.interp_perturbation(t, y, 17, method="spline")
    assert np.allclose(out[::2], y.astype(np.float64), atol=1e-12)
    errs = []
    for m in (17, 33, 65):
        tt = np.linspace(0.0, 1.0, m)
        f = np.sin(2 * np.pi * tt) + 0.5 * np.cos(5 * tt)
        g = _grid(tt, 1001)
        o = oracle.interp_perturbation(tt, f[:, None].astype(np.float32), 1001, method="spline")
        # FP32 inputs: compare with the spline-interpolation error, not below FP32 rounding
        errs.append(np.abs(o[:, 0] - (np.sin(2 * np.pi * g) + 0.5 * np.cos(5 * g))).max())
    assert errs[0] / errs[1] > 10.0 and errs[1] / errs[2] > 10.0


@pytest.mark.parametrize("reduce", [1, 2, 3, 7])
def test_reduce_map_is_decimation(reduce):
    """Sec. 4.3 `reduce`: 1-based indices divisible by reduce == numpy slicing from reduce-1."""
    M = np.arange(23 * 17, dtype=np.float64).reshape(23, 17)
    assert np.array_equal(oracle.reduce_map(M, reduce), M[reduce - 1::reduce, reduce - 1::reduce])


def test_interp_rejects_non_increasing_axis():
    x = np.array([0.0, 1.0, 1.0, 2.0])
    with pytest.raises(ValueError):
        oracle.interp_linear(x, np.zeros((2, 4), np.float32), 3)
