"""The seeded synthetic inputs: determinism, shapes and the recipe's statistics.

Every GPU parity test and the benchmark read these arrays, so they must be the
same on every machine and run (FP64 draws from numpy's default generator,
rounded once to FP32) and have the shapes and structure the workload recipe
states.  CPU only."""
import math

import numpy as np

import workloads


def test_generators_are_deterministic_fp32_and_seed_dependent():
    for make in (workloads.c1, workloads.c2):
        a, b = make(), make()
        assert a.dtype == np.float32 and np.array_equal(a, b)
    assert not np.array_equal(workloads.c2(seed=1), workloads.c2(seed=5))
    r1, r2 = workloads.c3(), workloads.c3()
    assert np.array_equal(r1.y1, r2.y1) and np.array_equal(r1.x2, r2.x2)
    s1 = workloads.random_stack(7, 9, seed=3)
    assert np.array_equal(s1, workloads.random_stack(7, 9, seed=3))


def test_configuration_shapes():
    assert workloads.c1().shape == (11, 500)
    assert workloads.c2().shape == (64, 4096)
    raw = workloads.c3()
    assert raw.y1.shape[0] == raw.y2.shape[0] == 128
    assert (raw.n1_out, raw.n2_out) == (8192, 2048)
    assert raw.y1.shape[1] == round(1.3 * 8192) and raw.y2.shape[1] == round(1.3 * 2048)
    assert raw.alpha == 0.5


def test_c2_baseline_and_noise_levels():
    y = workloads.c2().astype(np.float64)
    # baseline 10 under bands of amplitude <= 1 per band
    assert 9.99 < np.median(y[0]) < 12.0 and y.min() > 9.9
    # the noise floor: successive differences far from every band are ~ sqrt(2) 1e-3
    d = np.diff(y, axis=0)
    assert 0.5e-3 < np.median(np.abs(d)) < 0.2


def test_raw_axes_are_strictly_increasing_with_fixed_endpoints():
    raw = workloads.c3()
    for x, n_out in ((raw.x1, raw.n1_out), (raw.x2, raw.n2_out)):
        assert np.all(np.diff(x) > 0)
        assert x[0] == 0.0 and x[-1] == float(n_out - 1)
        h = (n_out - 1) / (len(x) - 1)
        assert np.max(np.abs(np.diff(x) - h)) < 0.81 * h  # jitter within +-0.4 h per point


def test_c5_spec_follows_the_recipe():
    spec = workloads.c5_spec()
    assert len(spec.problems) == 512
    ms = np.array([p.m for p in spec.problems])
    n1 = np.array([p.n1 for p in spec.problems])
    assert ms.min() >= 8 and ms.max() <= 200 and 80 < ms.mean() < 130
    assert n1.min() >= 256 and n1.max() <= 8192
    # log-uniform: the median of log n sits near the middle of [log 256, log 8192]
    mid = 0.5 * (math.log(256) + math.log(8192))
    assert abs(np.median(np.log(n1)) - mid) < 0.35
    for i, p in enumerate(spec.problems):
        assert p.homo == (i % 2 == 0)
        if p.homo:
            assert p.n2 == p.n1
    assert spec.total_outputs == sum(p.n1 * p.n2 for p in spec.problems)
    assert spec.total_outputs == workloads.c5_spec().total_outputs


def test_sample_rows_are_sorted_distinct_and_include_the_edges():
    r = workloads.sample_rows(1000, 50, seed=4)
    assert np.all(np.diff(r) > 0) and r[0] == 0 and r[-1] == 999 and len(r) == 50
    assert np.array_equal(r, workloads.sample_rows(1000, 50, seed=4))
    assert np.array_equal(workloads.sample_rows(3, 10, seed=1), np.array([0, 1, 2]))


def test_c5_fixed_n_keeps_the_m_mix():
    full, small = workloads.c5_spec(), workloads.c5_spec(n_fixed=768)
    assert [p.m for p in full.problems] == [p.m for p in small.problems]
    assert [p.homo for p in full.problems] == [p.homo for p in small.problems]
    assert all(p.n1 == p.n2 == 768 for p in small.problems)
    assert small.total_outputs == 512 * 768 * 768


def test_step_stack_puts_the_hilbert_transform_in_a_higher_binade():
    """The step-response stack exists to make the Hilbert variant's two operands
    (the dynamic spectrum d and its transform N d, Eq. HilbNoda) have their largest
    entries in different powers of two for most variables; the oracle's
    Hilbert-Noda product with the identity as stack 1 gives N d / (m - 1)."""
    import oracle
    m, n = 124, 300
    y = workloads.step_stack(m, n, seed=7)
    assert y.dtype == np.float32 and np.array_equal(y, workloads.step_stack(m, n, seed=7))
    d = oracle.dynamic(y, oracle.reference_mean(y))
    _, nd = oracle.hilbert_noda(np.eye(m), d)
    nd *= m - 1
    e_d = np.frexp(np.abs(d).max(axis=0))[1]
    e_nd = np.frexp(np.abs(nd).max(axis=0))[1]
    assert (e_nd > e_d).mean() > 0.9
