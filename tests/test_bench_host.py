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


def test_tensor_flops_count_the_split_products_and_the_binding_bound_leads():
    # homo m = 256 (K' = 128) over the 32768 x 32768 map's unique pairs, three products each
    pairs = 32768 * 32769 / 2
    fl = bench.tensor_flops(256, "split", pairs)
    assert fl == 3 * 8 * 128 * pairs
    assert bench.tensor_flops(256, "bf16", pairs) == fl / 3
    assert bench.tensor_flops(2, "split", 1) == 24  # m = 2: K' = 1 (omega = 0 only)
    peak, _ = bench.measured_tensor_peak()
    # the full map's kernel time: HBM binds and leads, the tensor figures sit beside it
    hbm = {"bound": "hbm", "achieved": 6450.0, "peak": 6792.1, "unit": "GB/s", "frac": 0.95,
           "algorithmic_bytes_per_launch": 8.6e9}
    r = bench.with_tensor_bound(hbm, fl, 1.334)
    assert r["bound"] == "hbm" and r["tensor"]["bound"] == "tensor"
    assert r["tensor"]["achieved"] == pytest.approx(fl / 1.334e-3 / 1e12, abs=0.05)
    # half the stores for the same products: the tensor bound binds and leads
    hbm_u = dict(hbm, achieved=3785.0, frac=0.557)
    r = bench.with_tensor_bound(hbm_u, fl, 1.133)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["hbm"]["frac"] == 0.557
    assert r["frac"] == pytest.approx(fl / 1.133e-3 / 1e12 / peak, abs=1e-4)
