"""The cross-spectrum launch overlapping the DFT launch's tail (programmatic
dependent launch) must not change a single output bit.

The cross-spectrum kernel waits for the DFT kernel to complete before it reads
operand rows, scales or the work counter; every tile's arithmetic is the same
whichever CTA computes it.  So a context with the overlap forced on
(CORR2D_PDL=always) and one with it off (CORR2D_PDL=off) give identical Phi
and Psi, and the batch's graph holding both launches with the
programmatic edge (replayed when no timings are recorded) gives what its two
separate graphs give (replayed when they are).  Both contexts take the tuner's
first tile candidate, so that they run the same tile layout.  Every FT case is
also held to the FP64 oracle at the parity tolerance (1e-5 relative Frobenius
error; 1e-2 with BF16 operands).
"""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def one_tile_choice():
    """Both contexts take the same tile layout (the tuner's first candidate): each
    context tunes on its own, and full and mirrored tiles may differ in the last FP32
    bit of the mirrored half."""
    old = os.environ.get("CORR2D_NO_TUNE")
    os.environ["CORR2D_NO_TUNE"] = "1"
    yield
    if old is None:
        del os.environ["CORR2D_NO_TUNE"]
    else:
        os.environ["CORR2D_NO_TUNE"] = old


@pytest.fixture(scope="module")
def pkg():
    import paper_1808_00685_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load()
    return p


def _context(pkg, mode):
    """A context created with CORR2D_PDL=mode (the variable is read at creation)."""
    old = os.environ.get("CORR2D_PDL")
    os.environ["CORR2D_PDL"] = mode
    try:
        return pkg.Context(0)
    finally:
        if old is None:
            del os.environ["CORR2D_PDL"]
        else:
            os.environ["CORR2D_PDL"] = old


def _host(t):
    return t.double().cpu().numpy()


CASES = [
    ("homo m=64 n=4096", (64, 4096, None), {}),
    ("hetero m=128 1000 x 700 alpha 0.5", (128, 1000, 700), {"alpha": 0.5}),
    ("homo m=33 n=517 bf16", (33, 517, None), {"precision": "bf16"}),
    ("homo m=40 n=600 Hilbert", (40, 600, None), {"hilbert": True}),
    ("homo m=96 n=1500 upper triangle", (96, 1500, None), {"upper_triangle": True}),
    ("homo m=3 n=33", (3, 33, None), {}),
    ("hetero m=257 140 x 1", (257, 140, 1), {}),
]


@pytest.mark.parametrize("name,shape,kw", CASES, ids=[c[0] for c in CASES])
def test_overlapped_and_serialised_launches_are_bit_identical(pkg, name, shape, kw):
    m, n1, n2 = shape
    y1 = workloads.random_stack(m, n1, seed=m + n1, offset=2.0)
    y2 = None if n2 is None else workloads.random_stack(m, n2, seed=m + n2 + 1, offset=-1.0)
    d1 = torch.from_numpy(y1).cuda()
    d2 = None if y2 is None else torch.from_numpy(y2).cuda()
    # the upper-triangle output leaves the boxes below the diagonal unwritten
    iu = np.triu_indices(n1) if kw.get("upper_triangle") else None

    def sel(a):
        return a[iu] if iu is not None else a

    got = {}
    for mode in ("off", "always"):
        ctx = _context(pkg, mode)
        try:
            outs = []
            for _ in range(2):  # the second call replays the cached descriptors
                phi, psi = ctx.compute(d1, d2, **kw)
                ctx.synchronize()
                outs.append((sel(_host(phi)), sel(_host(psi))))
            assert all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1])), name
            got[mode] = outs[1]
        finally:
            ctx.close()
    for a, b in zip(got["off"], got["always"]):
        assert np.array_equal(a, b), name
    if not kw.get("hilbert"):  # the overlapped launch against the oracle, too
        ophi, opsi, _, _ = oracle.corr2d(y1, y2, alpha=kw.get("alpha", 0.0),
                                         nthreads=oracle.max_threads())
        phi, psi = got["always"]
        tol = 1e-2 if kw.get("precision") == "bf16" else 1e-5
        if np.linalg.norm(ophi) > 0:
            assert np.linalg.norm(phi - sel(ophi)) / np.linalg.norm(sel(ophi)) <= tol, name
            assert np.linalg.norm(psi - sel(opsi)) / np.linalg.norm(sel(opsi)) <= tol, name


def test_batch_graphs_with_and_without_timing_events_are_bit_identical(pkg):
    spec = workloads.c5_spec(count=12, seed=21, m_lo=8, m_hi=200, n_lo=100, n_hi=1500)
    ins = workloads.batch_inputs(spec, nbands=6)
    ctx = pkg.Context(0)
    try:
        probs = []
        for (y1, y2), p in zip(ins, spec.problems):
            d1 = torch.from_numpy(y1).cuda()
            d2 = None if y2 is None else torch.from_numpy(y2).cuda()
            phi, psi, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
            probs.append((d1, d2, phi, psi))
        plan = ctx.batch_plan(probs, precision="split")
        results = []
        for profile in (False, True, False):
            for _, _, phi, psi in probs:
                phi.fill_(float("nan"))
                psi.fill_(float("nan"))
            ctx.set_profiling(profile)
            plan.run()
            ctx.synchronize()
            if profile:
                prep_ms, xspec_ms = ctx.timings()
                assert prep_ms > 0 and xspec_ms > 0
            results.append([(_host(phi[:, :p.n2]), _host(psi[:, :p.n2]))
                            for (_, _, phi, psi), p in zip(probs, spec.problems)])
        ctx.set_profiling(False)
        for r in results[1:]:
            for (a, b), (c, d) in zip(results[0], r):
                assert np.array_equal(a, c) and np.array_equal(b, d)
        (y1, y2), p = ins[0], spec.problems[0]
        ophi, opsi, _, _ = oracle.corr2d(y1, y2, nthreads=oracle.max_threads())
        phi, psi = results[0][0]
        assert np.linalg.norm(phi - ophi) / np.linalg.norm(ophi) <= 1e-5
        assert np.linalg.norm(psi - opsi) / np.linalg.norm(opsi) <= 1e-5
    finally:
        ctx.close()
