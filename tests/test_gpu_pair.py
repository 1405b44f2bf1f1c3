"""GPU parity of the CTA-pair cross-spectrum kernel (tcgen05 cta_group::2).

The tuner is restricted to the pair kernel (CORR2D_XSPEC=pair) in one context
and to the single-CTA kernel in another; every case is checked against the
FP64 oracle (relative Frobenius error of Phi and Psi, 1e-5 for the FP16 hi/lo
split, 1e-2 for plain BF16), homo outputs for exact symmetry, and the two
kernels against each other.  Shapes cover odd numbers of 128-row tiles (the
odd CTA of the last pair has no rows), ragged tails, a single tile and the
diagonal items of mirrored problems.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split": 1e-5, "bf16": 1e-2}


def _ctx(kind, **env):
    import paper_1808_00685_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    saved = {k: os.environ.get(k) for k in list(env) + ["CORR2D_XSPEC"]}
    os.environ["CORR2D_XSPEC"] = kind
    os.environ.update(env)
    return pkg.Context(0), saved


def _restore(saved):
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


@pytest.fixture(scope="module")
def pair_ctx():
    c, saved = _ctx("pair")
    _, npairs = c.kernel_info()
    if npairs == 0:
        c.close()
        _restore(saved)
        pytest.fail("the CTA-pair kernel is unavailable on this device")
    yield c, saved
    c.close()
    _restore(saved)


@pytest.fixture(scope="module")
def single_ctx():
    import paper_1808_00685_gb300 as pkg
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


def run_pair(ctx, y1, y2=None, **kw):
    import paper_1808_00685_gb300 as pkg
    os.environ["CORR2D_XSPEC"] = "pair"
    phi, psi = ctx.compute(dev(y1), None if y2 is None else dev(y2), **kw)
    ctx.synchronize()
    assert ctx.kernel_info()[0] == pkg.XSPEC_TC_PAIR
    return host(phi), host(psi)


def run_single(ctx, y1, y2=None, **kw):
    import paper_1808_00685_gb300 as pkg
    saved = os.environ.get("CORR2D_XSPEC")
    os.environ["CORR2D_XSPEC"] = "single"
    try:
        phi, psi = ctx.compute(dev(y1), None if y2 is None else dev(y2), **kw)
        ctx.synchronize()
        assert ctx.kernel_info()[0] == pkg.XSPEC_TC
    finally:
        if saved is None:
            os.environ.pop("CORR2D_XSPEC", None)
        else:
            os.environ["CORR2D_XSPEC"] = saved
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


@pytest.mark.parametrize("m,n", [(11, 100), (64, 128), (33, 256), (64, 300), (200, 384),
                                 (257, 513), (16, 1000), (128, 1280)])
@pytest.mark.parametrize("prec", ["split", "bf16"])
def test_pair_homo_matches_oracle_and_is_exactly_symmetric(pair_ctx, m, n, prec):
    ctx, _ = pair_ctx
    y = workloads.random_stack(m, n, seed=1000 + m + n)
    # the tuner may pick full (non-mirrored) tiles for homo problems unless
    # exact symmetry is requested: check both
    phi, psi = run_pair(ctx, y, precision=prec)
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(phi, psi, ophi, opsi, TOL[prec], f"pair homo m={m} n={n} {prec}")
    phi, psi = run_pair(ctx, y, precision=prec, exact_symmetry=True)
    check(phi, psi, ophi, opsi, TOL[prec], f"pair homo mirrored m={m} n={n} {prec}")
    assert np.array_equal(phi, phi.T)
    assert np.array_equal(psi, -psi.T)
    assert np.all(np.diag(psi) == 0.0)


@pytest.mark.parametrize("m,n1,n2", [(11, 300, 200), (64, 129, 700), (128, 1000, 1000),
                                     (40, 384, 64), (200, 700, 130), (9, 1, 1)])
@pytest.mark.parametrize("prec", ["split", "bf16"])
def test_pair_hetero_matches_oracle(pair_ctx, m, n1, n2, prec):
    ctx, _ = pair_ctx
    y1 = workloads.random_stack(m, n1, seed=2000 + n1)
    y2 = workloads.random_stack(m, n2, seed=3000 + n2)
    phi, psi = run_pair(ctx, y1, y2, precision=prec)
    ophi, opsi, _, _ = oracle.corr2d(y1, y2)
    check(phi, psi, ophi, opsi, TOL[prec], f"pair hetero m={m} n1={n1} n2={n2} {prec}")


def test_pair_and_single_kernels_agree(pair_ctx, single_ctx):
    y = workloads.random_stack(96, 700, seed=77)
    y2 = workloads.random_stack(96, 450, seed=78)
    for a, b in ((y, None), (y, y2)):
        p1, q1 = run_pair(pair_ctx[0], a, b, precision="split", alpha=0.5)
        p2, q2 = run_single(single_ctx, a, b, precision="split", alpha=0.5)
        scale = max(np.abs(p2).max(), np.abs(q2).max())
        assert np.abs(p1 - p2).max() <= 1e-6 * scale
        assert np.abs(q1 - q2).max() <= 1e-6 * scale


def test_pair_c2_offset_baseline_and_scaling(pair_ctx):
    ctx, _ = pair_ctx
    y = workloads.c2()
    phi, psi = run_pair(ctx, y, precision="split", alpha=1.0)
    ophi, opsi, _, _ = oracle.corr2d(y, alpha=1.0)
    check(phi, psi, ophi, opsi, 1e-5, "pair c2 Pearson")


def test_pair_upper_triangle_output(pair_ctx):
    ctx, _ = pair_ctx
    import paper_1808_00685_gb300 as pkg
    y = workloads.random_stack(50, 450, seed=91)
    n = y.shape[1]
    phi_t, psi_t, ldo = pkg.Context.alloc_out(n, n, torch.device("cuda"))
    phi_t.fill_(7.0)
    psi_t.fill_(7.0)
    os.environ["CORR2D_XSPEC"] = "pair"
    ctx.compute(dev(y), precision="split", upper_triangle=True, out=(phi_t, psi_t))
    ctx.synchronize()
    assert ctx.kernel_info()[0] == pkg.XSPEC_TC_PAIR
    phi, psi = host(phi_t)[:, :n], host(psi_t)[:, :n]
    ophi, opsi, _, _ = oracle.corr2d(y)
    iu = np.triu_indices(n)
    check(phi[iu], psi[iu], ophi[iu], opsi[iu], 1e-5, "pair upper triangle")
    # below the diagonal 32 x 32 boxes nothing is written
    il = np.tril_indices(n, -32)
    assert np.all(phi[il] == 7.0) and np.all(psi[il] == 7.0)


def test_pair_stalled_producer_times_out_and_context_survives():
    import paper_1808_00685_gb300 as pkg
    y = torch.from_numpy(workloads.random_stack(16, 300, seed=3)).cuda()
    ctx, saved = _ctx("pair", CORR2D_FAULT="stall", CORR2D_WAIT_LIMIT_MS="200")
    try:
        if ctx.kernel_info()[1] == 0:
            pytest.fail("the CTA-pair kernel is unavailable on this device")
        ctx.compute(y, precision="split")
        with pytest.raises(pkg.Corr2dError) as ei:
            ctx.synchronize()
        assert ei.value.status == pkg.ETIMEOUT
        assert ctx.kernel_info()[0] == pkg.XSPEC_TC_PAIR
        ctx.synchronize()
    finally:
        ctx.close()
        _restore(saved)
    with pkg.Context(0) as ok:
        os.environ["CORR2D_XSPEC"] = "pair"
        try:
            phi, psi = ok.compute(y, precision="split")
            ok.synchronize()
        finally:
            os.environ.pop("CORR2D_XSPEC", None)
        ophi, opsi, _, _ = oracle.corr2d(y.cpu().numpy())
        check(host(phi), host(psi), ophi, opsi, 1e-5, "after time-out")
