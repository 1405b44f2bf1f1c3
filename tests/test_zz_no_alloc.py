"""The allocation-free entry point against the ordinary one and the FP64 oracle.

corr2d_compute_noalloc serves callers that must not allocate GPU memory (a
memory planner that owns the device, a host framework that forbids hidden
allocations, a loop that cannot pay cudaMalloc's synchronisation, code with
no library context): its intermediates live in a static device array.  Each
case here calls it through the C ABI twice in a row (the second call reuses
the array the first one left behind) and compares both results with
corr2d_compute on the same inputs and with the oracle, within the parity
tolerances of the other GPU tests (1e-5 relative Frobenius error for the
split precision, 1e-2 for plain BF16).  Requests larger than the static array
must be refused up front.  This file is collected last on purpose, so that a
run stopping at the first failure has run every other test before it.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split": 1e-5, "bf16": 1e-2}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def pkg():
    import paper_1808_00685_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load()
    return p


def _noalloc(pkg, y1, y2, params, n1, n2, fill=None):
    """Run the allocation-free entry point; the test allocates the outputs."""
    phi, psi, ldo = pkg.Context.alloc_out(n1, n2, y1.device)
    if fill is not None:
        phi.fill_(fill)
        psi.fill_(fill)
    stream = torch.cuda.current_stream().cuda_stream
    m = y1.shape[0]
    pkg.corr2d_compute_noalloc(0, stream, m, n1, y1.data_ptr(), y1.stride(0), n2,
                               None if y2 is None else y2.data_ptr(),
                               0 if y2 is None else y2.stride(0), params, phi.data_ptr(),
                               psi.data_ptr(), ldo)
    return phi[:, :n2].double().cpu().numpy(), psi[:, :n2].double().cpu().numpy()


def _oracle_ht(y1, y2, alpha):
    d1 = oracle.dynamic(y1, oracle.reference_mean(y1))
    d2 = d1 if y2 is None else oracle.dynamic(y2, oracle.reference_mean(y2))
    phi, psi = oracle.hilbert_noda(d1, d2)
    s1 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d1)])
    s2 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d2)])
    return phi * np.outer(s1, s2), psi * np.outer(s1, s2)


def _stacks(case):
    if case == "homo":
        return workloads.sigmoid_bands(64, 1000, 20, seed=21), None
    if case == "step":  # N d a power of two above d: the two operands rescale differently
        return workloads.step_stack(124, 519, seed=41), None
    return (workloads.random_stack(100, 700, seed=22, offset=2.0),
            workloads.random_stack(100, 500, seed=23, offset=-1.0))


CASES = [
    # (stacks, precision, options)
    ("homo", "split", {}),
    ("hetero", "split", {}),
    ("homo", "bf16", {}),
    ("hetero", "bf16", {}),
    ("hetero", "split", {"user_ref": True}),
    ("homo", "split", {"user_ref": True}),
    ("homo", "split", {"no_mirror": True}),
    ("homo", "split", {"hilbert": True}),
    ("hetero", "split", {"hilbert": True}),
    ("step", "split", {"hilbert": True}),
]


@pytest.mark.parametrize("case,prec,opts", CASES,
                         ids=[f"{c}-{p}-{'-'.join(o) or 'plain'}" for c, p, o in CASES])
def test_noalloc_matches_compute_and_oracle_twice(pkg, case, prec, opts):
    y1, y2 = _stacks(case)
    d1 = torch.from_numpy(y1).cuda()
    d2 = None if y2 is None else torch.from_numpy(y2).cuda()
    n1 = y1.shape[1]
    n2 = n1 if y2 is None else y2.shape[1]
    alpha = 0.5
    hilbert = opts.get("hilbert", False)
    no_mirror = opts.get("no_mirror", False)
    r1 = r2 = None
    dr1 = dr2 = None
    if opts.get("user_ref"):
        r1 = y1[0].copy()
        r2 = None if y2 is None else y2[-1].copy()
        dr1 = torch.from_numpy(r1).cuda()
        dr2 = None if r2 is None else torch.from_numpy(r2).cuda()
    with pkg.Context(0) as ctx:
        ref_phi, ref_psi = ctx.compute(d1, d2, precision=prec, alpha=alpha, ref1=dr1, ref2=dr2,
                                       hilbert=hilbert, no_mirror=no_mirror,
                                       exact_symmetry=True)
        ctx.synchronize()
        ref_phi = ref_phi.double().cpu().numpy()
        ref_psi = ref_psi.double().cpu().numpy()
    if hilbert:
        ophi, opsi = _oracle_ht(y1, y2, alpha)
    else:
        ophi, opsi, _, _ = oracle.corr2d(y1, y2, ref1=r1, ref2=r2, alpha=alpha,
                                         nthreads=oracle.max_threads())
    params = pkg.make_params(prec, alpha=alpha, ref1=dr1, ref2=dr2, hilbert=hilbert,
                             no_mirror=no_mirror)
    tol = TOL[prec]
    for call in range(2):
        phi, psi = _noalloc(pkg, d1, d2, params, n1, n2, fill=float("nan") if call else None)
        for name, got, want in (("Phi", phi, ref_phi), ("Psi", psi, ref_psi)):
            assert _rel(got, want) <= tol, f"call {call}: {name} vs corr2d_compute {_rel(got, want):.3e}"
        for name, got, want in (("Phi", phi, ophi), ("Psi", psi, opsi)):
            assert _rel(got, want) <= tol, f"call {call}: {name} vs oracle {_rel(got, want):.3e}"
        if y2 is None and not no_mirror:  # mirrored tiles: exact (anti)symmetry
            assert np.array_equal(phi, phi.T) and np.array_equal(psi, -psi.T)


def test_noalloc_upper_triangle(pkg):
    """CORR2D_FLAG_UPPER_TRIANGLE: nu2 >= nu1 matches the oracle; the lower boxes
    away from the diagonal are not written (sentinel NaNs stay), on both calls."""
    y = workloads.random_stack(40, 700, seed=23)
    d = torch.from_numpy(y).cuda()
    n = y.shape[1]
    ophi, opsi, _, _ = oracle.corr2d(y, nthreads=oracle.max_threads())
    iu = np.triu_indices(n)
    r, c = np.indices((n, n))
    far_lower = (r // 32) > (c // 32)
    params = pkg.make_params("split", upper_triangle=True)
    for call in range(2):
        phi, psi = _noalloc(pkg, d, None, params, n, n, fill=float("nan"))
        assert _rel(phi[iu], ophi[iu]) <= 1e-5 and _rel(psi[iu], opsi[iu]) <= 1e-5
        assert np.all(np.isnan(phi[far_lower])) and np.all(np.isnan(psi[far_lower]))


def test_noalloc_hilbert_sync_is_the_ft_sync_times_pi_over_m(pkg):
    """Odd m: Phi_FT = (m / pi) Phi_HT (Sec. 2); both from the allocation-free entry
    point, so a Hilbert request that ran the FT path would fail here."""
    m = 31
    y = workloads.sigmoid_bands(m, 400, 10, seed=9)
    d = torch.from_numpy(y).cuda()
    phi_ft, _ = _noalloc(pkg, d, None, pkg.make_params("split"), 400, 400)
    phi_ht, psi_ht = _noalloc(pkg, d, None, pkg.make_params("split", hilbert=True), 400, 400)
    assert _rel(phi_ft, (m / math.pi) * phi_ht) < 1e-5
    _, opsi = _oracle_ht(y, None, 0.0)
    assert _rel(psi_ht, opsi) < 1e-5


def test_noalloc_refuses_what_it_cannot_do(pkg):
    stream = torch.cuda.current_stream().cuda_stream
    phi = torch.empty((8, 8), dtype=torch.float32, device="cuda")
    # more scratch than the static array holds
    y = torch.zeros((256, 40000), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_compute_noalloc(0, stream, 256, 40000, y.data_ptr(), 40000, 0, None, 0,
                                   pkg.make_params("split"), phi.data_ptr(), phi.data_ptr(), 40000)
    assert ei.value.status == pkg.EUNSUPPORTED
    assert "scratch" in str(ei.value)
    # BF16 output needs corr2d_compute
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_compute_noalloc(0, stream, 16, 64, y.data_ptr(), 64, 0, None, 0,
                                   pkg.make_params("split", output_bf16=True), phi.data_ptr(),
                                   phi.data_ptr(), 64)
    assert ei.value.status == pkg.EUNSUPPORTED
    # the Hilbert variant stops at m = 256, the FP32 path needs a context
    y = torch.zeros((300, 64), dtype=torch.float32, device="cuda")
    out = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    for params in (pkg.make_params("split", hilbert=True), pkg.make_params("fp32")):
        m = 300 if params.flags else 20
        with pytest.raises(pkg.Corr2dError) as ei:
            pkg.corr2d_compute_noalloc(0, stream, m, 64, y.data_ptr(), 64, 0, None, 0, params,
                                       out.data_ptr(), out.data_ptr(), 64)
        assert ei.value.status == pkg.EUNSUPPORTED
