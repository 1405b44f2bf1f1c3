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
