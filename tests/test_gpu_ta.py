"""GPU parity of the TMEM-operand cross-spectrum kernel (stack-1 operand in TMEM).

The tuner is restricted to that kernel (CORR2D_XSPEC=ta), or one of its
segment lengths is forced (CORR2D_TILES=128:mirror:0:1:seg); every case is
checked against the FP64 oracle (relative Frobenius error of Phi and Psi, 1e-5
for the FP16 hi/lo split, 1e-2 for plain BF16), homo outputs for exact
symmetry, and against the single-CTA kernel.  Shapes cover ragged tails in
both directions, a single tile, odd numbers of tiles, segments of
one tile and segments longer than a row, every chunk count up to the TMEM
limit (m = 256 in split precision: 8 chunks) and the fallback beyond it.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split": 1e-5, "bf16": 1e-2}


class _Env:
    """Sets environment variables for the duration of a with-block."""

    def __init__(self, **env):
        self.env = env

    def __enter__(self):
        self.saved = {k: os.environ.get(k) for k in self.env}
        for k, v in self.env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def __exit__(self, *exc):
        for k, v in self.saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def ctx():
    import paper_1808_00685_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    c = pkg.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def run(ctx, y1, y2=None, kind="ta", tiles=None, expect=None, **kw):
    import paper_1808_00685_gb300 as pkg
    with _Env(CORR2D_XSPEC=kind, CORR2D_TILES=tiles):
        phi, psi = ctx.compute(dev(y1), None if y2 is None else dev(y2), **kw)
        ctx.synchronize()
    want = pkg.XSPEC_TC_TA if expect is None else expect
    assert ctx.kernel_info()[0] == want
    return host(phi), host(psi)


def check(phi, psi, ophi, opsi, tol, what):
    """Relative Frobenius error within tol, and every element within 4 x tol x the
    largest oracle magnitude of the pair (as in test_gpu_parity.check)."""
    ep, eq = rel(phi, ophi), rel(psi, opsi)
    mp, mq = np.abs(phi - ophi).max(), np.abs(psi - opsi).max()
    big = max(np.abs(ophi).max(), np.abs(opsi).max())
    msg = (f"{what}: rel Phi {ep:.3e} Psi {eq:.3e}; max-abs Phi {mp:.3e} Psi {mq:.3e} "
           f"(largest magnitude {big:.3e})")
    assert ep <= tol and eq <= tol, msg
    assert mp <= 4.0 * tol * big and mq <= 4.0 * tol * big, msg


@pytest.mark.parametrize("m,n", [(11, 100), (64, 64), (33, 200), (64, 300), (200, 384),
                                 (256, 513), (16, 1000), (128, 1280)])
@pytest.mark.parametrize("prec", ["split", "bf16"])
def test_ta_homo_mirrored_matches_oracle_and_is_exactly_symmetric(ctx, m, n, prec):
    y = workloads.random_stack(m, n, seed=2000 + m + n)
    phi, psi = run(ctx, y, precision=prec, exact_symmetry=True)
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(phi, psi, ophi, opsi, TOL[prec], f"ta homo mirrored m={m} n={n} {prec}")
    assert np.array_equal(phi, phi.T) and np.array_equal(psi, -psi.T)
    assert np.all(np.diag(psi) == 0.0)


@pytest.mark.parametrize("m,n", [(11, 100), (64, 300), (256, 513)])
@pytest.mark.parametrize("prec", ["split", "bf16"])
def test_ta_homo_full_tiles_match_oracle(ctx, m, n, prec):
    y = workloads.random_stack(m, n, seed=2100 + m + n)
    phi, psi = run(ctx, y, precision=prec, no_mirror=True)
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(phi, psi, ophi, opsi, TOL[prec], f"ta homo full m={m} n={n} {prec}")


@pytest.mark.parametrize("m,n1,n2", [(33, 130, 70), (128, 1000, 257), (256, 129, 640),
                                     (7, 64, 64), (100, 2, 1)])
@pytest.mark.parametrize("prec", ["split", "bf16"])
def test_ta_hetero_matches_oracle(ctx, m, n1, n2, prec):
    y1 = workloads.random_stack(m, n1, seed=2200 + n1)
    y2 = workloads.random_stack(m, n2, seed=2300 + n2)
    phi, psi = run(ctx, y1, y2, precision=prec, alpha=0.5)
    ophi, opsi, _, _ = oracle.corr2d(y1, y2, alpha=0.5)
    check(phi, psi, ophi, opsi, TOL[prec], f"ta hetero m={m} {n1}x{n2} {prec}")


@pytest.mark.parametrize("seg", [1, 3, 4, 4096])
@pytest.mark.parametrize("mirror", [0, 1])
def test_ta_every_segment_length_gives_the_same_map(ctx, seg, mirror):
    """Segment boundaries only change which CTA computes a tile and when the
    stack-1 operand is reloaded: the maps are bit-identical for every length."""
    y = workloads.random_stack(96, 900, seed=2400)
    ref = run(ctx, y, tiles=f"128:{mirror}:0:1:2")
    got = run(ctx, y, tiles=f"128:{mirror}:0:1:{seg}")
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(got[0], got[1], ophi, opsi, 1e-5, f"ta seg={seg} mirror={mirror}")


@pytest.mark.parametrize("m", [16, 100, 256])
def test_ta_matches_the_single_cta_kernel(ctx, m):
    """Same products in the same order per output element: the two kernels
    agree far below the split's error bar."""
    import paper_1808_00685_gb300 as pkg
    y1 = workloads.random_stack(m, 900, seed=2500 + m)
    y2 = workloads.random_stack(m, 333, seed=2600 + m)
    a = run(ctx, y1, y2)
    b = run(ctx, y1, y2, kind="single", expect=pkg.XSPEC_TC)
    scale = np.abs(b[0]).max()
    assert np.abs(a[0] - b[0]).max() <= 1e-6 * scale
    assert np.abs(a[1] - b[1]).max() <= 1e-6 * scale


def test_ta_falls_back_beyond_the_tmem_operand_limit(ctx):
    """m = 257 needs 9 split chunks (more than TMEM holds beside the
    accumulators): the single-CTA kernel runs instead."""
    import paper_1808_00685_gb300 as pkg
    y = workloads.random_stack(257, 300, seed=2700)
    phi, psi = run(ctx, y, expect=pkg.XSPEC_TC)
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(phi, psi, ophi, opsi, 1e-5, "m=257 fallback")
    # BF16 keeps 32 frequencies per chunk: m = 257 fits
    phi, psi = run(ctx, y, precision="bf16")
    check(phi, psi, ophi, opsi, 1e-2, "m=257 bf16")


def test_ta_upper_triangle(ctx):
    n = 300
    y = workloads.random_stack(40, n, seed=2800)
    import paper_1808_00685_gb300 as pkg
    phi_t, psi_t, _ = pkg.Context.alloc_out(n, n, torch.device("cuda"))
    phi_t.fill_(7.0)
    psi_t.fill_(7.0)
    with _Env(CORR2D_XSPEC="ta", CORR2D_TILES=None):
        ctx.compute(dev(y), out=(phi_t, psi_t), upper_triangle=True)
        ctx.synchronize()
    assert ctx.kernel_info()[0] == pkg.XSPEC_TC_TA
    phi, psi = host(phi_t)[:, :n], host(psi_t)[:, :n]
    ophi, opsi, _, _ = oracle.corr2d(y)
    iu = np.triu_indices(n)
    check(phi[iu], psi[iu], ophi[iu], opsi[iu], 1e-5, "ta upper triangle")
    il = np.tril_indices(n, -32)
    assert np.all(phi[il] == 7.0) and np.all(psi[il] == 7.0)


def test_ta_stalled_producer_times_out_and_context_survives():
    import paper_1808_00685_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    y = dev(workloads.random_stack(16, 300, seed=3))
    with _Env(CORR2D_FAULT="stall", CORR2D_WAIT_LIMIT_MS="200"):
        bad = pkg.Context(0)
    try:
        with _Env(CORR2D_TILES="128:1:0:1:8"):
            bad.compute(y, precision="split")
        with pytest.raises(pkg.Corr2dError) as ei:
            bad.synchronize()
        assert ei.value.status == pkg.ETIMEOUT
        assert bad.kernel_info()[0] == pkg.XSPEC_TC_TA
        bad.synchronize()
    finally:
        bad.close()
    with pkg.Context(0) as ok:
        with _Env(CORR2D_XSPEC="ta"):
            phi, psi = ok.compute(y, precision="split")
            ok.synchronize()
        assert ok.kernel_info()[0] == pkg.XSPEC_TC_TA
        ophi, opsi, _, _ = oracle.corr2d(y.cpu().numpy())
        check(host(phi), host(psi), ophi, opsi, 1e-5, "after time-out")


def _oracle_hilbert(y1, y2=None, alpha=0.0):
    d1 = oracle.dynamic(y1, oracle.reference_mean(y1))
    d2 = d1 if y2 is None else oracle.dynamic(y2, oracle.reference_mean(y2))
    phi, psi = oracle.hilbert_noda(d1, d2)
    if alpha > 0:
        s1 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d1)])
        s2 = np.array([oracle.scale_factor(s, alpha) for s in oracle.sigma(d2)])
        phi, psi = phi * np.outer(s1, s2), psi * np.outer(s1, s2)
    return phi, psi


@pytest.mark.parametrize("m,n1,n2", [(16, 300, None), (100, 260, None), (40, 333, 170)])
def test_ta_runs_the_hilbert_variant_when_forced(ctx, m, n1, n2):
    """The Hilbert-transform operands (two row sets even for homo problems, up
    to 8 chunks of 16 steps) through the TMEM-operand kernel."""
    y1 = workloads.random_stack(m, n1, seed=2900 + m, offset=2.0)
    y2 = None if n2 is None else workloads.random_stack(m, n2, seed=2950 + m, offset=-1.0)
    alpha = 0.0 if n2 is None else 0.5
    phi, psi = run(ctx, y1, y2, tiles="128:0:0:1:3", hilbert=True, alpha=alpha)
    ophi, opsi = _oracle_hilbert(y1, y2, alpha=alpha)
    assert rel(phi, ophi) < 1e-5
    assert np.abs(psi - opsi).max() <= 1e-5 * np.abs(ophi).max()


def test_ta_row_slabs_use_the_single_cta_kernel(ctx):
    """A row slab is not a whole problem: the single-CTA kernel computes it,
    and its rows equal those of the whole map."""
    import paper_1808_00685_gb300 as pkg
    y = workloads.random_stack(64, 700, seed=3000)
    full = run(ctx, y, no_mirror=True)
    with _Env(CORR2D_XSPEC="ta", CORR2D_TILES=None):
        phi, psi = ctx.compute_rows(dev(y), None, 256, 300)
        ctx.synchronize()
    assert ctx.kernel_info()[0] == pkg.XSPEC_TC
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(host(phi), host(psi), ophi[256:556], opsi[256:556], 1e-5, "ta row slab")
    assert np.abs(host(phi) - full[0][256:556]).max() <= 1e-6 * np.abs(full[0]).max()
