"""Host-side logic of bench.py, on the CPU: where the forms' errors are sampled,
how a batch's algorithmic bytes are counted, and that the CPU-baseline leg's
error report catches a planted error in the "GPU" values it is given."""
import numpy as np
import pytest

import bench
import workloads


@pytest.mark.parametrize("n", [300, 4096, 32768])
def test_sampled_blocks_include_the_edges_and_the_upper_form_stays_above_the_diagonal(n):
    rows, cols = bench.sample_block(n)
    assert rows[0] == 0 and rows[-1] == n - 1 and cols[0] == 0 and cols[-1] == n - 1
    assert len(set(rows)) == len(rows) == min(n, 256)
    rows, cols = bench.sample_block(n, upper=True)
    assert rows.max() < cols.min()  # every sampled entry has nu2 > nu1
    assert rows[0] == 0 and cols[-1] == n - 1


def test_batch_bytes_are_outputs_plus_operand_rows_read_once():
    spec = workloads.c5_spec(count=6, seed=3, n_lo=40, n_hi=500)
    want = 0.0
    for p in spec.problems:
        kp = ((p.m - 1) // 2 + 1 + 15) // 16 * 16  # split: 16 frequencies per chunk
        rowlen = kp // 16 * 64
        rows = p.n1 if p.homo else p.n1 + p.n2
        want += 8.0 * p.n1 * p.n2 + 2.0 * rows * rowlen
    assert bench.batch_bytes(spec, "split") == pytest.approx(want, rel=0, abs=0.5)
    assert bench.rowlen_elems(256, "split") == 512 and bench.rowlen_elems(256, "bf16") == 256


def test_cpu_baseline_leg_reports_the_error_of_what_it_is_given():
    class Args:
        no_cpu_baseline = True
        cpu_sample_n = 0
    y = workloads.random_stack(12, 200, seed=5, offset=3.0)
    rows, cols = bench.sample_block(200)
    exact = bench.oracle_at(y, None, rows, cols)
    planted = exact[0].copy()
    planted[3, 7] += 1e-3 * np.abs(exact[0]).max()  # one wrong entry
    checks = {"exact": [(y, None, rows, cols, 0.0, exact)],
              "planted": [(y, None, rows, cols, 0.0, (planted, exact[1]))]}
    cpu, errors = bench.cpu_baseline_leg(Args(), y, 0.0, checks)
    assert cpu is None
    assert errors["exact"]["rel_err_phi"] == 0.0 and errors["exact"]["max_abs_psi"] == 0.0
    e = errors["planted"]
    assert e["max_abs_phi"] == pytest.approx(1e-3 * e["largest_magnitude"], rel=1e-9)
    assert e["rel_err_phi"] > 0 and e["rel_err_psi"] == 0.0
