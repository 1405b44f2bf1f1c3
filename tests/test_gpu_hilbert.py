"""GPU parity of the Hilbert-transform approach (Sec. 2, Eqs. disHTsyn, disHT,
HilbNoda, disHTasyn) against the FP64 oracle's direct evaluation.

Phi = 1/(m-1) sum_j d1 d2 and Psi = 1/(m-1) sum_j d1 (N d2) with the
Hilbert-Noda matrix; scaling by (sigma1 sigma2)^-alpha as for the FT approach.
Tolerance: 1e-5 relative Frobenius error (split), 1e-2 (plain BF16).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1808_00685_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    c = pkg.Context(0)
    yield c
    c.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle_ht(y1, y2=None, alpha=0.0):
    d1 = oracle.dynamic(y1, oracle.reference_mean(y1))
    d2 = d1 if y2 is None else oracle.dynamic(y2, oracle.reference_mean(y2))
    phi, psi = oracle.hilbert_noda(d1, d2)
    if alpha > 0:
        s1 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d1)])
        s2 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d2)])
        phi, psi = phi * np.outer(s1, s2), psi * np.outer(s1, s2)
    return phi, psi


def _gpu(ctx, y1, y2=None, **kw):
    d1 = torch.from_numpy(y1).cuda()
    d2 = None if y2 is None else torch.from_numpy(y2).cuda()
    phi, psi = ctx.compute(d1, d2, hilbert=True, **kw)
    ctx.synchronize()
    return phi.double().cpu().numpy(), psi.double().cpu().numpy()


@pytest.mark.parametrize("m,n", [(2, 40), (7, 150), (16, 300), (33, 129), (128, 260), (256, 200)])
def test_hilbert_homo(ctx, m, n):
    y = workloads.random_stack(m, n, seed=m + n, offset=2.0)
    phi, psi = _gpu(ctx, y)
    ophi, opsi = _oracle_ht(y)
    assert _rel(phi, ophi) < 1e-5
    assert np.abs(psi - opsi).max() <= 1e-5 * np.abs(ophi).max()
    if m > 2:
        assert _rel(psi, opsi) < 1e-5


@pytest.mark.parametrize("prec,tol", [("split", 1e-5), ("bf16", 1e-2)])
def test_hilbert_hetero_scaled(ctx, prec, tol):
    y1 = workloads.random_stack(40, 333, seed=5, offset=-1.0)
    y2 = workloads.random_stack(40, 170, seed=6, offset=3.0)
    phi, psi = _gpu(ctx, y1, y2, precision=prec, alpha=0.5)
    ophi, opsi = _oracle_ht(y1, y2, alpha=0.5)
    assert _rel(phi, ophi) < tol and _rel(psi, opsi) < tol


def test_hilbert_sync_matches_ft_for_odd_m(ctx):
    """Odd m: Phi_FT = (m / pi) Phi_HT (Parseval; Sec. 2 'results are identical')."""
    m = 31
    y = workloads.sigmoid_bands(m, 400, 10, seed=9)
    phi_ht, _ = _gpu(ctx, y)
    d = torch.from_numpy(y).cuda()
    phi_ft, _ = ctx.compute(d)
    ctx.synchronize()
    assert _rel(phi_ft.double().cpu().numpy(), (m / math.pi) * phi_ht) < 1e-5


def test_hilbert_rejected_where_unsupported(ctx):
    import paper_1808_00685_gb300 as pkg
    y = torch.from_numpy(workloads.random_stack(300, 64, seed=1)).cuda()
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.compute(y, hilbert=True)  # m > 256
    assert ei.value.status == pkg.EUNSUPPORTED
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.compute(y[:20], hilbert=True, precision="fp32")
    assert ei.value.status == pkg.EUNSUPPORTED


def _oracle_ht_ref(y1, y2, r1, r2, alpha=0.0):
    """Hilbert approach with caller-supplied references (Eq. dynspec with the chosen
    reference; sigma from the same dynamic spectra, Eq. stdev)."""
    d1 = oracle.dynamic(y1, r1.astype(np.float64))
    d2 = d1 if y2 is None else oracle.dynamic(y2, r2.astype(np.float64))
    phi, psi = oracle.hilbert_noda(d1, d2)
    if alpha > 0:
        s1 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d1)])
        s2 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d2)])
        phi, psi = phi * np.outer(s1, s2), psi * np.outer(s1, s2)
    return phi, psi


def test_hilbert_with_user_reference_and_scaling(ctx):
    y1 = workloads.random_stack(24, 300, seed=31, offset=1.0)
    y2 = workloads.random_stack(24, 170, seed=32, offset=-2.0)
    r1, r2 = y1[0].copy(), y2[-1].copy()
    phi, psi = _gpu(ctx, y1, y2, ref1=torch.from_numpy(r1).cuda(), ref2=torch.from_numpy(r2).cuda(),
                    alpha=1.0)
    ophi, opsi = _oracle_ht_ref(y1, y2, r1, r2, alpha=1.0)
    assert _rel(phi, ophi) < 1e-5 and _rel(psi, opsi) < 1e-5


def test_hilbert_batch_matches_oracle(ctx):
    """corr2d_batch with the Hilbert flag: homo and hetero problems of uneven m and n."""
    import paper_1808_00685_gb300 as pkg
    spec = workloads.c5_spec(count=8, seed=12, m_lo=3, m_hi=200, n_lo=40, n_hi=600)
    ins = workloads.batch_inputs(spec, nbands=5)
    probs = []
    for (y1, y2), p in zip(ins, spec.problems):
        d1 = torch.from_numpy(y1).cuda()
        d2 = None if y2 is None else torch.from_numpy(y2).cuda()
        phi, psi, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
        probs.append((d1, d2, phi, psi))
    for rep in range(2):
        ctx.batch(probs, precision="split", hilbert=True)
        ctx.synchronize()
        for (y1, y2), p, (_, _, phi, psi) in zip(ins, spec.problems, probs):
            ophi, opsi = _oracle_ht(y1, y2)
            gp = phi[:, :p.n2].double().cpu().numpy()
            gq = psi[:, :p.n2].double().cpu().numpy()
            assert _rel(gp, ophi) < 1e-5, f"rep {rep} m={p.m} n1={p.n1} n2={p.n2}"
            assert _rel(gq, opsi) < 1e-5, f"rep {rep} m={p.m} n1={p.n1} n2={p.n2}"


def test_hilbert_rows_parts_reduced_and_upper_triangle(ctx):
    """The Hilbert flag through row slabs, tile parts, the reduced map and the
    upper-triangle output."""
    import paper_1808_00685_gb300 as pkg
    n = 600
    y = workloads.random_stack(40, n, seed=33, offset=0.5)
    y2 = workloads.random_stack(40, 250, seed=34, offset=1.5)
    d, d2 = torch.from_numpy(y).cuda(), torch.from_numpy(y2).cuda()
    ophi, opsi = _oracle_ht(y)
    hphi, hpsi = _oracle_ht(y, y2)
    # row slabs of the hetero problem
    parts = [ctx.compute_rows(d, d2, *pkg.shard_rows(n, 3, r), hilbert=True) for r in range(3)]
    ctx.synchronize()
    phi = np.concatenate([p.double().cpu().numpy() for p, _ in parts])
    psi = np.concatenate([q.double().cpu().numpy() for _, q in parts])
    assert _rel(phi, hphi) < 1e-5 and _rel(psi, hpsi) < 1e-5
    # tile parts of the homo problem, each into its own NaN-filled buffers
    got = []
    for part in range(3):
        a, b, _ = pkg.Context.alloc_out(n, n, d.device)
        a.fill_(float("nan"))
        b.fill_(float("nan"))
        pa, pb = ctx.compute_part(d, None, part, 3, hilbert=True, out=(a, b))
        ctx.synchronize()
        got.append((pa.double().cpu().numpy(), pb.double().cpu().numpy()))
    w = np.stack([~np.isnan(a) for a, _ in got])
    assert np.all(w.sum(0) == 1)
    phi = np.where(w, np.stack([a for a, _ in got]), 0.0).sum(0)
    psi = np.where(w, np.stack([b for _, b in got]), 0.0).sum(0)
    assert _rel(phi, ophi) < 1e-5 and _rel(psi, opsi) < 1e-5
    assert np.array_equal(psi, -psi.T)
    # reduced map: every 4th variable
    pr, qr = ctx.compute_reduced(d, None, 4, hilbert=True)
    ctx.synchronize()
    assert _rel(pr.double().cpu().numpy(), oracle.reduce_map(ophi, 4)) < 1e-5
    assert _rel(qr.double().cpu().numpy(), oracle.reduce_map(opsi, 4)) < 1e-5
    # upper triangle
    a, b, _ = pkg.Context.alloc_out(n, n, d.device)
    pa, pb = ctx.compute(d, hilbert=True, upper_triangle=True, out=(a, b))
    ctx.synchronize()
    iu = np.triu_indices(n)
    assert _rel(pa.double().cpu().numpy()[iu], ophi[iu]) < 1e-5
    assert _rel(pb.double().cpu().numpy()[iu], opsi[iu]) < 1e-5


def test_hilbert_step_dynamics_every_route(ctx):
    """Step responses: the transform N d of these dynamic spectra has its
    largest entries a power of two above those of d for most variables, so the
    two operands of a homo problem get different power-of-two rescales and each
    needs its own scale array.  Through compute (mirrored, unmirrored, BF16),
    the hetero form, the batch and tile parts."""
    import paper_1808_00685_gb300 as pkg
    m, n = 124, 519
    y = workloads.step_stack(m, n, seed=41)
    y2 = workloads.step_stack(m, 300, seed=42, offset=-1.0)
    ys = workloads.step_stack(m, 150, seed=43)
    d, d2, ds = (torch.from_numpy(a).cuda() for a in (y, y2, ys))
    ophi, opsi = _oracle_ht(y)
    for kw, tol in (({}, 1e-5), ({"no_mirror": True}, 1e-5), ({"precision": "bf16"}, 1e-2)):
        phi, psi = _gpu(ctx, y, **kw)
        assert _rel(phi, ophi) < tol and _rel(psi, opsi) < tol, kw
    phi, psi = _gpu(ctx, y, y2, alpha=0.5)
    hphi, hpsi = _oracle_ht(y, y2, alpha=0.5)
    assert _rel(phi, hphi) < 1e-5 and _rel(psi, hpsi) < 1e-5
    # batch: the homo problem, the hetero one and a small homo one (64-wide tiles)
    shapes = [(d, None, n, n), (d, d2, n, 300), (ds, None, 150, 150)]
    probs = []
    for a, b, n1, n2 in shapes:
        p, q, _ = pkg.Context.alloc_out(n1, n2, a.device)
        probs.append((a, b, p, q))
    ctx.batch(probs, precision="split", hilbert=True)
    ctx.synchronize()
    want = [_oracle_ht(y), _oracle_ht(y, y2), _oracle_ht(ys)]
    for (_, _, n1, n2), (_, _, p, q), (wp, wq) in zip(shapes, probs, want):
        assert _rel(p[:, :n2].double().cpu().numpy(), wp) < 1e-5, (n1, n2)
        assert _rel(q[:, :n2].double().cpu().numpy(), wq) < 1e-5, (n1, n2)
    # tile parts of the homo problem
    acc_p, acc_q = np.zeros((n, n)), np.zeros((n, n))
    for part in range(3):
        a, b, _ = pkg.Context.alloc_out(n, n, d.device)
        a.zero_()
        b.zero_()
        pa, pb = ctx.compute_part(d, None, part, 3, hilbert=True, out=(a, b))
        ctx.synchronize()
        acc_p += pa.double().cpu().numpy()
        acc_q += pb.double().cpu().numpy()
    assert _rel(acc_p, ophi) < 1e-5 and _rel(acc_q, opsi) < 1e-5
