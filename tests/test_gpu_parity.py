"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (relative Frobenius error of Phi and of Psi separately, on the same
seeded FP32 inputs): 1e-5 for FP32 and the FP16 hi/lo split, 1e-2 for plain
BF16 operands.  Beside the norm, every element is bounded: the max-abs error
of Phi and of Psi must stay within MAXABS_K x tol x the largest oracle
magnitude of that map, so that a localised error (one wrong 32 x 32 box of a
large map) cannot hide inside the norm.  The measured max-abs errors are
2e-6 .. 4e-6 of the largest magnitude (split), 1e-6 (FP32) and 6e-3 (BF16).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split": 1e-5, "bf16": 1e-2}


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


MAXABS_K = 4.0


def check(phi, psi, ophi, opsi, tol, what=""):
    ep, eq = rel(phi, ophi), rel(psi, opsi)
    mp, mq = np.abs(phi - ophi).max(), np.abs(psi - opsi).max()
    # the largest magnitude of the pair sets the scale of both (Psi can vanish
    # where Phi does not, e.g. in-phase bands)
    big = max(np.abs(ophi).max(), np.abs(opsi).max())
    msg = (f"{what}: rel Phi {ep:.3e} Psi {eq:.3e}; max-abs Phi {mp:.3e} Psi {mq:.3e} "
           f"(largest magnitude {big:.3e})")
    assert ep <= tol and eq <= tol, msg
    assert mp <= MAXABS_K * tol * big and mq <= MAXABS_K * tol * big, msg
    return ep, eq


def run(ctx, y1, y2=None, **kw):
    phi, psi = ctx.compute(dev(y1), None if y2 is None else dev(y2), **kw)
    ctx.synchronize()
    return host(phi), host(psi)


# -------------------------------------------------------------- paper configs

@pytest.mark.parametrize("prec", ["split", "bf16", "fp32"])
def test_c1_small_homo(ctx, prec):
    y = workloads.c1()
    phi, psi = run(ctx, y, precision=prec)
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(phi, psi, ophi, opsi, TOL[prec], f"c1 {prec}")


@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_c2_homo_offset_baseline(ctx, prec):
    """m=64, n=4096, baseline offset 10: centering cancels the baseline."""
    y = workloads.c2()
    phi, psi = run(ctx, y, precision=prec)
    ophi, opsi, _, _ = oracle.corr2d(y, nthreads=oracle.max_threads())
    check(phi, psi, ophi, opsi, TOL[prec], f"c2 {prec}")
    # the tuner may pick full tiles: symmetric to rounding
    assert rel(phi, phi.T) < 1e-6 and rel(psi, -psi.T) < 1e-6
    # mirrored tiles: exactly symmetric / antisymmetric, zero diagonal of Psi
    phi, psi = run(ctx, y, precision=prec, exact_symmetry=True)
    check(phi, psi, ophi, opsi, TOL[prec], f"c2 {prec} exact symmetry")
    assert np.array_equal(phi, phi.T) and np.array_equal(psi, -psi.T)
    assert np.all(np.diag(psi) == 0)


@pytest.mark.parametrize("m", [384, 512])
@pytest.mark.parametrize("kind", ["smooth", "noise"])
def test_split_error_bar_at_the_largest_m(ctx, m, kind):
    """The split path's error grows with the number of tensor-core additions
    (FP32 accumulation truncates); at the largest accepted m it must still be
    within 1e-5, for smooth (sigmoid-profile bands, baseline 10) and for
    noise-like spectra."""
    n = 1024
    y = (workloads.sigmoid_bands(m, n, 40, seed=m, baseline=10.0) if kind == "smooth"
         else workloads.random_stack(m, n, seed=m, offset=10.0))
    phi, psi = run(ctx, y, precision="split", exact_symmetry=True)
    ophi, opsi, _, _ = oracle.corr2d(y, nthreads=oracle.max_threads())
    check(phi, psi, ophi, opsi, 1e-5, f"split {kind} m={m}")


@pytest.mark.parametrize("m", [512, 257])
def test_large_baseline_small_dynamic_part(ctx, m):
    """Baseline 1000 (stack 2: -3000) under a dynamic part of 0.01: the mean
    must hold ~20 significant bits below the baseline's ulp for the centred
    spectra to keep theirs; sigma and sigma^-alpha at alpha = 0.5, 1, 3."""
    import paper_1808_00685_gb300 as pkg
    n1, n2 = 700, 333
    y1 = workloads.random_stack(m, n1, seed=m + 1, offset=1000.0, scale=0.01)
    y2 = workloads.random_stack(m, n2, seed=m + 2, offset=-3000.0, scale=0.01)
    phi, psi = run(ctx, y1, precision="split")
    ophi, opsi, os1, _ = oracle.corr2d(y1, nthreads=oracle.max_threads())
    check(phi, psi, ophi, opsi, 1e-5, f"m={m} homo")
    for alpha in (0.5, 1.0, 3.0):
        d1, d2 = dev(y1), dev(y2)
        p, q, lo = pkg.Context.alloc_out(n1, n2, d1.device)
        ph, ps, s1, s2 = ctx.compute(d1, d2, out=(p, q), precision="split", alpha=alpha,
                                     want_sigma=True)
        ctx.synchronize()
        ophi, opsi, os1, os2 = oracle.corr2d(y1, y2, alpha=alpha, nthreads=oracle.max_threads())
        check(host(ph)[:, :n2], host(ps)[:, :n2], ophi, opsi, 1e-5, f"m={m} alpha={alpha}")
        assert np.allclose(s1.cpu().numpy(), os1, rtol=1e-6)
        assert np.allclose(s2.cpu().numpy(), os2, rtol=1e-6)


@pytest.mark.parametrize("m", [512, 257])
@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_baseline_a_million_times_the_dynamic_part(ctx, m, alpha):
    """Baseline 1e4 (stack 2: -1e4) under a dynamic part of 0.01, a ratio of 1e6:
    the double-float mean and centering must still give the centred FP32 values the
    FP64 oracle forms from the same FP32 inputs.  (A mean error delta is the same
    at every step, so it reaches only the DC term, m delta, of the DFT; the centred
    values themselves are rounded once.)  Phi and Psi within 1e-5 homo and
    hetero, sigma within 1e-6."""
    import paper_1808_00685_gb300 as pkg
    n1, n2 = 400, 250
    y1 = workloads.random_stack(m, n1, seed=m + 11, offset=1.0e4, scale=0.01)
    y2 = workloads.random_stack(m, n2, seed=m + 12, offset=-1.0e4, scale=0.01)
    d1, d2 = dev(y1), dev(y2)
    ph, ps, s1, _ = ctx.compute(d1, precision="split", alpha=alpha, want_sigma=True,
                                exact_symmetry=True)
    ctx.synchronize()
    ophi, opsi, os1, _ = oracle.corr2d(y1, alpha=alpha, nthreads=oracle.max_threads())
    check(host(ph), host(ps), ophi, opsi, 1e-5, f"homo m={m} alpha={alpha}")
    assert np.allclose(s1.cpu().numpy(), os1, rtol=1e-6, atol=0)
    p, q, _ = pkg.Context.alloc_out(n1, n2, d1.device)
    ph, ps, s1, s2 = ctx.compute(d1, d2, out=(p, q), precision="split", alpha=alpha,
                                 want_sigma=True)
    ctx.synchronize()
    ophi, opsi, os1, os2 = oracle.corr2d(y1, y2, alpha=alpha, nthreads=oracle.max_threads())
    check(host(ph)[:, :n2], host(ps)[:, :n2], ophi, opsi, 1e-5, f"hetero m={m} alpha={alpha}")
    assert np.allclose(s1.cpu().numpy(), os1, rtol=1e-6, atol=0)
    assert np.allclose(s2.cpu().numpy(), os2, rtol=1e-6, atol=0)


def test_c3_hetero_with_preprocessing(ctx):
    """Raw spectra on non-uniform axes -> uniform grids -> hetero, alpha = 0.5."""
    raw = workloads.c3()
    y1g, _ = ctx.preprocess(dev(raw.x1), dev(raw.y1), raw.n1_out)
    y2g, _ = ctx.preprocess(dev(raw.x2), dev(raw.y2), raw.n2_out)
    ctx.synchronize()
    o1, _ = oracle.interp_linear(raw.x1, raw.y1, raw.n1_out)
    o2, _ = oracle.interp_linear(raw.x2, raw.y2, raw.n2_out)
    # interpolation: the correctly rounded FP32 value of the FP64 blend, bit for bit
    assert np.array_equal(y1g.cpu().numpy(), o1.astype(np.float32))
    assert np.array_equal(y2g.cpu().numpy(), o2.astype(np.float32))
    rows = workloads.sample_rows(raw.n1_out, 512, seed=31)
    phi, psi = ctx.compute(y1g, y2g, precision="split", alpha=raw.alpha)
    ctx.synchronize()
    ophi, opsi, _, _ = oracle.corr2d(o1.astype(np.float32), o2.astype(np.float32),
                                     alpha=raw.alpha, rows=rows, nthreads=oracle.max_threads())
    check(host(phi)[rows], host(psi)[rows], ophi, opsi, 1e-5, "c3 split sampled rows")


def test_c4_full_size_sampled_rows(ctx):
    """m=256, n=32768 (8.6 GB of output) in split precision; 256 sampled rows."""
    y = workloads.c4()
    yd = dev(y)
    phi, psi = ctx.compute(yd, precision="split")
    ctx.synchronize()
    rows = workloads.sample_rows(y.shape[1], 256, seed=41)
    rt = torch.from_numpy(rows.astype(np.int64)).cuda()
    gphi = host(phi.index_select(0, rt))
    gpsi = host(psi.index_select(0, rt))
    del phi, psi
    torch.cuda.empty_cache()
    ophi, opsi, _, _ = oracle.corr2d(y, rows=rows, nthreads=oracle.max_threads())
    check(gphi, gpsi, ophi, opsi, 1e-5, "c4 split sampled rows")
    # mirrored columns: Phi(j, i) = Phi(i, j) at sampled rows i
    assert np.all(np.isfinite(gphi))


# ----------------------------------------------------------------- edge cases

@pytest.mark.parametrize("m,n", [(2, 1), (2, 7), (3, 33), (4, 129), (5, 128), (16, 257),
                                 (65, 300), (130, 131), (257, 140), (512, 64)])
@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_ragged_and_extreme_shapes(ctx, m, n, prec):
    y = workloads.random_stack(m, n, seed=m * 1000 + n, offset=3.0)
    phi, psi = run(ctx, y, precision=prec)
    ophi, opsi, _, _ = oracle.corr2d(y)
    if np.linalg.norm(ophi) == 0:  # m = 2: only the DC term, zero after centering
        assert np.abs(phi).max() < 1e-6 and np.abs(psi).max() < 1e-6
        return
    check(phi, psi, ophi, opsi, TOL[prec], f"m={m} n={n} {prec}")


@pytest.mark.parametrize("prec", ["split", "bf16", "fp32"])
def test_hetero_uneven(ctx, prec):
    y1 = workloads.random_stack(37, 300, seed=1, offset=-2.0)
    y2 = workloads.random_stack(37, 170, seed=2, offset=5.0)
    phi, psi = run(ctx, y1, y2, precision=prec)
    ophi, opsi, _, _ = oracle.corr2d(y1, y2)
    check(phi, psi, ophi, opsi, TOL[prec], f"hetero {prec}")


@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_user_reference_norm_and_scaling(ctx, prec):
    y1 = workloads.random_stack(20, 200, seed=3)
    y2 = workloads.random_stack(20, 150, seed=4)
    r1, r2 = y1[0].copy(), y2[-1].copy()
    phi, psi = run(ctx, y1, y2, precision=prec, ref1=dev(r1), ref2=dev(r2), norm=0.5, alpha=1.0)
    ophi, opsi, _, _ = oracle.corr2d(y1, y2, ref1=r1, ref2=r2, norm=0.5, alpha=1.0)
    check(phi, psi, ophi, opsi, TOL[prec], f"user ref {prec}")


def test_constant_variable_gives_zero_rows(ctx):
    y = workloads.random_stack(9, 140, seed=5)
    y[:, 17] = 2.5
    for prec in ("split", "fp32"):
        phi, psi = run(ctx, y, precision=prec, alpha=0.5)
        assert np.all(phi[17] == 0) and np.all(phi[:, 17] == 0) and np.all(psi[17] == 0)
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(psi))
        ophi, opsi, _, _ = oracle.corr2d(y, alpha=0.5)
        check(phi, psi, ophi, opsi, TOL[prec], f"sigma=0 {prec}")


def test_sigma_outputs_and_padded_leading_dimensions(ctx):
    import paper_1808_00685_gb300 as pkg
    m, n = 24, 150
    y = workloads.random_stack(m, n, seed=6, offset=1.0)
    ypad = np.zeros((m, 160), np.float32)
    ypad[:, :n] = y
    yd = dev(ypad)[:, :n]  # leading dimension 160
    phi, psi, ldo = pkg.Context.alloc_out(n, n, yd.device, ld=164)
    ph, ps, s1, s2 = ctx.compute(yd, out=(phi, psi), want_sigma=True)
    ctx.synchronize()
    ophi, opsi, os1, _ = oracle.corr2d(y)
    check(host(ph)[:, :n], host(ps)[:, :n], ophi, opsi, 1e-5, "padded ld")
    assert np.allclose(s1.cpu().numpy(), os1, rtol=1e-6)


def test_mirror_and_full_tiles_agree(ctx):
    y = workloads.random_stack(40, 400, seed=7)
    a = run(ctx, y, precision="split")
    b = run(ctx, y, precision="split", no_mirror=True)
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(*a, ophi, opsi, 1e-5, "mirror")
    check(*b, ophi, opsi, 1e-5, "no mirror")


def test_repeated_calls_reuse_descriptors_correctly(ctx):
    """Identical calls launch from cached device descriptors; another shape in
    between must not leave a stale cache, and new input data must be used."""
    import paper_1808_00685_gb300 as pkg
    ya = workloads.random_stack(20, 300, seed=31)
    yb = workloads.random_stack(33, 170, seed=32)
    da, db = dev(ya), dev(yb)
    oa, ob = pkg.Context.alloc_out(300, 300, da.device), pkg.Context.alloc_out(170, 170, db.device)
    for step in range(3):
        for y, d, o in ((ya, da, oa), (yb, db, ob)):
            n = y.shape[1]
            phi, psi = ctx.compute(d, out=o[:2])
            ctx.synchronize()
            ophi, opsi, _, _ = oracle.corr2d(y)
            check(host(phi)[:, :n], host(psi)[:, :n], ophi, opsi, 1e-5, f"step {step} n={n}")
        ya *= np.float32(1.5)  # new data in the same buffer
        da.copy_(torch.from_numpy(ya))


def test_plan_cache_cycles_through_more_buffer_sets_than_slots(ctx):
    """Recent launches keep their descriptors (a few slots, least recently used
    replaced): cycling through six buffer sets of two shapes, hetero and homo,
    must give every call the result of its own inputs."""
    import paper_1808_00685_gb300 as pkg
    sets = []
    for i in range(6):
        n1 = 200 if i % 2 else 260
        y1 = workloads.random_stack(24, n1, seed=400 + i)
        y2 = None if i % 3 == 0 else workloads.random_stack(24, 150, seed=500 + i)
        n2 = n1 if y2 is None else 150
        o = pkg.Context.alloc_out(n1, n2, torch.device("cuda"))
        sets.append((y1, y2, dev(y1), None if y2 is None else dev(y2), o, n2))
    for rnd in range(3):
        order = list(range(6)) if rnd != 1 else [0, 1, 0, 1, 2, 0, 3, 4, 5, 1]
        for i in order:
            y1, y2, d1, d2, o, n2 = sets[i]
            phi, psi = ctx.compute(d1, d2, out=o[:2])
            ctx.synchronize()
            ophi, opsi, _, _ = oracle.corr2d(y1, y2)
            check(host(phi)[:, :n2], host(psi)[:, :n2], ophi, opsi, 1e-5, f"round {rnd} set {i}")


@pytest.mark.parametrize("tiles", ["128:1:0:1", "128:1:8:1", "128:1:12:1", "128:1:16:1",
                                   "128:1:24:1", "128:1:32:1", "128:1:64:1", "128:1:96:1",
                                   "128:1:8:4", "128:0:0:1", "128:0:12:1", "64:0:0:1",
                                   "128:0:0:1:0:5", "128:0:12:1:0:5", "128:1:64:1:0:5",
                                   "128:1:8:4:0:5"])
def test_every_tile_order_gives_the_oracle_result(ctx, tiles):
    """Each tile choice the tuner may pick (width, mirror, order: row-major or
    G x G super-blocks; run length per CTA), forced through CORR2D_TILES, on
    ragged homo and hetero problems."""
    import os
    y1 = workloads.random_stack(40, 2100, seed=71)  # 17 tile rows: partial super-blocks
    y2 = workloads.random_stack(40, 530, seed=72)
    os.environ["CORR2D_TILES"] = tiles
    try:
        phi, psi = run(ctx, y1, precision="split")
        hphi, hpsi = run(ctx, y1, y2, precision="split")
    finally:
        del os.environ["CORR2D_TILES"]
    ophi, opsi, _, _ = oracle.corr2d(y1)
    check(phi, psi, ophi, opsi, 1e-5, f"homo tiles {tiles}")
    if tiles.split(":")[1] == "1" and tiles.startswith("128"):  # mirrored: exact symmetry
        assert np.array_equal(phi, phi.T) and np.array_equal(psi, -psi.T)
    ophi, opsi, _, _ = oracle.corr2d(y1, y2)
    check(hphi, hpsi, ophi, opsi, 1e-5, f"hetero tiles {tiles}")


def test_self_hetero_matches_homo(ctx):
    """Hetero correlation of a stack with a copy of itself is the homo correlation
    (oracle), and agrees with the homo GPU call to rounding."""
    y = workloads.random_stack(30, 260, seed=8)
    a = run(ctx, y, precision="split", no_mirror=True)
    b = run(ctx, y, y.copy(), precision="split")
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(*a, ophi, opsi, 1e-5, "homo, all tiles")
    check(*b, ophi, opsi, 1e-5, "hetero with itself")
    assert rel(a[0], b[0]) < 1e-6 and rel(a[1], b[1]) < 1e-6


# ------------------------------------------------------------ preprocessing

def test_preprocess_reference_subtraction_bit_exact(ctx):
    rng = np.random.default_rng(9)
    x = workloads.jittered_axis(777, 0.0, 500.0, rng)
    y = workloads.random_stack(13, 777, seed=10)
    ref = workloads.random_stack(1, 600, seed=11)[0]
    out, dyn = ctx.preprocess(dev(x), dev(y), 600, ref=dev(ref))
    ctx.synchronize()
    o, od = oracle.interp_linear(x, y, 600, ref=ref)
    assert np.array_equal(out.cpu().numpy(), o.astype(np.float32))
    assert np.array_equal(dyn.cpu().numpy(), od.astype(np.float32))


@pytest.mark.parametrize("kind,m,n_raw,n_out", [("exponential", 7, 900, 640),
                                                 ("clustered", 33, 2000, 3000),
                                                 ("two points", 1, 2, 17),
                                                 ("one row", 1, 500, 123)])
def test_preprocess_on_non_uniform_axes_bit_exact(ctx, kind, m, n_raw, n_out):
    """The segment search starts from the equally spaced estimate and gallops: axes
    far from equal spacing (exponential, clustered) and the smallest shapes must
    give the oracle's values bit for bit."""
    rng = np.random.default_rng(n_raw)
    if kind == "exponential":
        x = np.exp(np.linspace(0.0, 9.0, n_raw))
    elif kind == "clustered":
        x = np.cumsum(rng.exponential(1.0, n_raw) ** 3 + 1e-6)
    else:
        x = np.sort(rng.uniform(-5.0, 5.0, n_raw))
    x = np.unique(x)
    assert len(x) == n_raw
    y = workloads.random_stack(m, n_raw, seed=n_out, offset=1.0)
    ref = workloads.random_stack(1, n_out, seed=n_out + 1)[0]
    out, dyn = ctx.preprocess(dev(x), dev(y), n_out, ref=dev(ref))
    ctx.synchronize()
    o, od = oracle.interp_linear(x, y, n_out, ref=ref)
    assert np.array_equal(out.cpu().numpy(), o.astype(np.float32))
    assert np.array_equal(dyn.cpu().numpy(), od.astype(np.float32))


def test_preprocess_rejects_non_increasing_axis(ctx):
    import paper_1808_00685_gb300 as pkg
    x = np.linspace(0, 1, 50)
    x[20] = x[19]
    y = workloads.random_stack(3, 50, seed=1)
    ctx.preprocess(dev(x), dev(y), 40)
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.synchronize()
    assert ei.value.status == pkg.EINVAL
    ctx.synchronize()  # the error word was cleared


# --------------------------------------------------------------- ABI errors

def test_invalid_arguments_return_status(ctx):
    import paper_1808_00685_gb300 as pkg
    y = dev(workloads.random_stack(8, 64, seed=1))
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.compute(y[:1])  # m = 1
    assert ei.value.status == pkg.EINVAL
    phi = torch.empty((64, 66), device="cuda")
    with pytest.raises(pkg.Corr2dError) as ei:  # ldo % 4 != 0 for TMA stores
        ctx.compute(y, out=(phi, phi.clone()))
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.Corr2dError) as ei:  # host stack
        hy = workloads.random_stack(8, 64, seed=1)
        p = pkg.make_params()
        out = torch.empty((64, 64), device="cuda")
        pkg.corr2d_compute(ctx.handle, 8, 64, hy.ctypes.data, 64, 0, None, 0, p, out.data_ptr(),
                           out.data_ptr(), 64)
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.Corr2dError) as ei:  # m beyond the tensor-core limit
        ctx.compute(dev(workloads.random_stack(513, 16, seed=2)))
    assert ei.value.status == pkg.EUNSUPPORTED
    ctx.synchronize()


def test_fp32_path_accepts_large_m(ctx):
    y = workloads.random_stack(600, 70, seed=12)
    phi, psi = run(ctx, y, precision="fp32")
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(phi, psi, ophi, opsi, 1e-5, "fp32 m=600")


# -------------------------------------------------------------------- batch

def test_batch_matches_oracle_and_single_calls(ctx):
    import paper_1808_00685_gb300 as pkg
    spec = workloads.c5_spec(count=10, seed=5, m_lo=8, m_hi=200, n_lo=40, n_hi=700)
    inputs = workloads.batch_inputs(spec, nbands=5)
    probs, outs = [], []
    for (y1, y2), p in zip(inputs, spec.problems):
        d1 = dev(y1)
        d2 = None if y2 is None else dev(y2)
        phi, psi, ldo = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
        probs.append((d1, d2, phi, psi))
        outs.append((phi, psi))
    for rep in range(2):  # second call replays the captured graph
        ctx.batch(probs, precision="split")
        ctx.synchronize()
        for (y1, y2), p, (phi, psi) in zip(inputs, spec.problems, outs):
            ophi, opsi, _, _ = oracle.corr2d(y1, y2)
            check(host(phi)[:, :p.n2], host(psi)[:, :p.n2], ophi, opsi, 1e-5,
                  f"batch m={p.m} n1={p.n1} n2={p.n2} homo={p.homo}")


def test_c5_full_batch_sampled_outputs(ctx):
    """The full batch of 512 problems in the benchmark's launch configuration
    (one corr2d_batch call: tuned tile widths and run lengths, graph replay),
    checked on sampled outputs.  Every step before the cross product acts on
    one spectral variable at a time (mean, centering, sigma, DFT), so the
    oracle run on the sampled columns of the stacks gives exactly those
    entries of Phi and Psi: 4 rows x 48 columns per problem, edges included."""
    import paper_1808_00685_gb300 as pkg
    spec = workloads.c5_spec()
    ins = workloads.batch_inputs(spec)
    probs = []
    for (y1, y2), p in zip(ins, spec.problems):
        d1 = dev(y1)
        d2 = None if y2 is None else dev(y2)
        phi, psi, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
        probs.append((d1, d2, phi, psi))
    plan = ctx.batch_plan(probs, precision="split")
    for rep in range(2):  # the second call replays the recorded graphs
        if rep == 1:
            for _, _, phi, psi in probs:
                phi.fill_(float("nan"))
                psi.fill_(float("nan"))
        plan.run()
        ctx.synchronize()
    worst = 0.0
    for i, ((y1, y2), p, (_, _, phi, psi)) in enumerate(zip(ins, spec.problems, probs)):
        rows = workloads.sample_rows(p.n1, 4, seed=9000 + i)
        cols = workloads.sample_rows(p.n2, 48, seed=19000 + i)
        rt = torch.from_numpy(rows.astype(np.int64)).cuda()
        ct = torch.from_numpy(cols.astype(np.int64)).cuda()
        gphi = host(phi.index_select(0, rt).index_select(1, ct))
        gpsi = host(psi.index_select(0, rt).index_select(1, ct))
        ys2 = (y1 if y2 is None else y2)[:, cols]
        ophi, opsi, _, _ = oracle.corr2d(np.ascontiguousarray(y1[:, rows]),
                                         np.ascontiguousarray(ys2))
        ep, eq = check(gphi, gpsi, ophi, opsi, 1e-5,
                       f"batch problem {i} m={p.m} n1={p.n1} n2={p.n2} homo={p.homo}")
        worst = max(worst, ep, eq)
    print(f"c5 full batch: worst relative error over 512 problems {worst:.2e}")


def test_batch_plan_replay_reads_current_inputs_and_new_lists_are_checked(ctx):
    """A replayed batch (same list: the recorded graph, no pointer queries) reads
    the inputs as they are at the time of the call; a changed list is validated."""
    import paper_1808_00685_gb300 as pkg
    spec = workloads.c5_spec(count=6, seed=8, m_lo=8, m_hi=90, n_lo=40, n_hi=400)
    inputs = workloads.batch_inputs(spec, nbands=4)
    probs = []
    for (y1, y2), p in zip(inputs, spec.problems):
        d1 = dev(y1)
        d2 = None if y2 is None else dev(y2)
        phi, psi, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
        probs.append((d1, d2, phi, psi))
    plan = ctx.batch_plan(probs, precision="split")
    for rep in range(3):
        scale = 1.0 + rep  # new values in the same buffers before each replay
        for (y1, y2), (d1, d2, _, _) in zip(inputs, probs):
            d1.copy_(dev(y1 * np.float32(scale)))
            if d2 is not None:
                d2.copy_(dev(y2 * np.float32(scale)))
        plan.run()
        ctx.synchronize()
        for (y1, y2), p, (_, _, phi, psi) in zip(inputs, spec.problems, probs):
            ys1 = (y1 * np.float32(scale)).astype(np.float32)
            ys2 = None if y2 is None else (y2 * np.float32(scale)).astype(np.float32)
            ophi, opsi, _, _ = oracle.corr2d(ys1, ys2)
            check(host(phi)[:, :p.n2], host(psi)[:, :p.n2], ophi, opsi, 1e-5,
                  f"replay {rep} m={p.m} n1={p.n1} n2={p.n2}")
    # the same shapes with one output in host memory: a new list, so it is checked
    d1, d2, phi, psi = probs[0]
    bad = [(d1, d2, phi.cpu(), psi)] + probs[1:]
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.batch(bad, precision="split")
    assert ei.value.status == pkg.EINVAL
    plan.run()  # the valid list still runs afterwards
    ctx.synchronize()


def test_host_buffer_entry_point(ctx):
    y1 = workloads.random_stack(33, 300, seed=13)
    y2 = workloads.random_stack(33, 260, seed=14)
    phi, psi = ctx.compute_host(torch.from_numpy(y1), torch.from_numpy(y2))
    ophi, opsi, _, _ = oracle.corr2d(y1, y2)
    check(phi.double().numpy(), psi.double().numpy(), ophi, opsi, 1e-5, "host buffers")
    phi, psi = ctx.compute_host(torch.from_numpy(y1))
    ophi, opsi, _, _ = oracle.corr2d(y1)
    check(phi.double().numpy(), psi.double().numpy(), ophi, opsi, 1e-5, "host buffers homo")


def test_host_buffer_entry_point_over_several_slabs(ctx):
    """The host path streams the output through two device slab buffers of up to 256 MB
    (here 8 tile rows of 32768 columns each), each slab's copies running while the next
    slab is computed into the other buffer: three slabs, the last one partial, held to the
    oracle on rows at the slab edges, then a second call into the same pinned buffers gives
    the same bits."""
    m, n1, n2 = 24, 2500, 32768
    y1 = workloads.random_stack(m, n1, seed=31)
    y2 = workloads.random_stack(m, n2, seed=32, offset=-1.0)
    t1, t2 = torch.from_numpy(y1).pin_memory(), torch.from_numpy(y2).pin_memory()
    phi = torch.empty((n1, n2), dtype=torch.float32, pin_memory=True)
    psi = torch.empty((n1, n2), dtype=torch.float32, pin_memory=True)
    ctx.compute_host(t1, t2, out=(phi, psi))
    rows = np.array([0, 1, 1023, 1024, 1025, 2047, 2048, 2049, 2498, 2499])
    ophi, opsi, _, _ = oracle.corr2d(y1, y2, rows=rows, nthreads=oracle.max_threads())
    a, b = phi.numpy()[rows].astype(np.float64), psi.numpy()[rows].astype(np.float64)
    check(a, b, ophi, opsi, 1e-5, "host buffers, three slabs")
    first = (phi.clone(), psi.clone())
    phi.fill_(float("nan"))
    psi.fill_(float("nan"))
    ctx.compute_host(t1, t2, out=(phi, psi))
    assert torch.equal(phi, first[0]) and torch.equal(psi, first[1])


def test_preprocess_perturbation_bit_exact_and_feeds_compute(ctx):
    """Sec. 4.2 perturbation-axis interpolation: uneven Time -> N equidistant steps,
    bit-exact against the oracle, then the correlation of the resampled stack."""
    rng = np.random.default_rng(12)
    m, n, N = 100, 777, 128
    time = np.sort(rng.uniform(0.0, 10.0, m))
    time[0], time[-1] = 0.0, 10.0
    y = workloads.sigmoid_bands(m, n, 15, seed=13)
    out = ctx.preprocess_perturbation(dev(time), dev(y), N)
    ctx.synchronize()
    o = oracle.interp_perturbation(time, y, N)
    assert np.array_equal(out.cpu().numpy(), o.astype(np.float32))
    phi, psi = ctx.compute(out, precision="split", alpha=0.5)
    ctx.synchronize()
    ophi, opsi, _, _ = oracle.corr2d(o.astype(np.float32), alpha=0.5)
    check(host(phi)[:, :n], host(psi)[:, :n], ophi, opsi, 1e-5, "interpolated along t")
    bad = time.copy()
    bad[5] = bad[4]
    ctx.preprocess_perturbation(dev(bad), dev(y), N)
    import paper_1808_00685_gb300 as pkg
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.synchronize()
    assert ei.value.status == pkg.EINVAL


@pytest.mark.parametrize("m,n,N", [(2, 5, 7), (3, 300, 2), (4, 33, 64), (5, 777, 9),
                                   (100, 777, 128), (257, 1000, 300)])
def test_perturbation_spline_matches_oracle(ctx, m, n, N):
    """splinefun (fmm) along the perturbation axis: the GPU rounds the same FP64
    spline to FP32, so every output is within one FP32 ulp of the oracle."""
    rng = np.random.default_rng(m * 7 + N)
    time = np.sort(rng.uniform(0.0, 5.0, m))
    time[0], time[-1] = 0.0, 5.0
    if m > 2:
        time = np.unique(time)
        assert len(time) == m
    y = workloads.sigmoid_bands(m, n, 9, seed=m + n, baseline=1.0)
    out = ctx.preprocess_perturbation(dev(time), dev(y), N, method="spline")
    ctx.synchronize()
    o = oracle.interp_perturbation(time, y, N, method="spline")
    got = out.cpu().numpy().astype(np.float64)
    tol = np.spacing(np.abs(o).astype(np.float32)).astype(np.float64) + 1e-12 * np.abs(y).max()
    assert np.all(np.abs(got - o) <= tol), np.abs(got - o).max()
    if m >= 4:  # the spline is not the line
        lin = ctx.preprocess_perturbation(dev(time), dev(y), N)
        ctx.synchronize()
        assert not np.array_equal(lin.cpu().numpy(), out.cpu().numpy())


def test_perturbation_spline_feeds_compute_and_checks_arguments(ctx):
    import paper_1808_00685_gb300 as pkg
    rng = np.random.default_rng(21)
    m, n, N = 60, 500, 64
    time = np.cumsum(rng.uniform(0.05, 0.3, m))
    y = workloads.sigmoid_bands(m, n, 12, seed=22)
    out = ctx.preprocess_perturbation(dev(time), dev(y), N, method="spline")
    phi, psi = ctx.compute(out, precision="split")
    ctx.synchronize()
    o = oracle.interp_perturbation(time, y, N, method="spline").astype(np.float32)
    ophi, opsi, _, _ = oracle.corr2d(o)
    check(host(phi)[:, :n], host(psi)[:, :n], ophi, opsi, 1e-5, "spline along t")
    bad = time.copy()
    bad[7] = bad[6]
    ctx.preprocess_perturbation(dev(bad), dev(y), N, method="spline")
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.synchronize()
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_interpolate_perturbation(ctx.handle, 7, m, n, dev(time).data_ptr(),
                                            dev(y).data_ptr(), n, N, out.data_ptr())
    assert ei.value.status == pkg.EINVAL


def test_row_slabs_assemble_the_full_result(ctx):
    """Multi-GPU layout on one GPU: the rows split into 128-aligned slabs (one per
    would-be GPU), each computed independently, equal one full call bit for bit."""
    import paper_1808_00685_gb300 as pkg
    y1 = workloads.random_stack(50, 700, seed=21)
    y2 = workloads.random_stack(50, 333, seed=22)
    d1, d2 = dev(y1), dev(y2)
    full = run(ctx, y1, y2, precision="split")
    for world in (2, 3):
        parts_phi, parts_psi = [], []
        for rank in range(world):
            r0, cnt = pkg.shard_rows(700, world, rank)
            ph, ps = ctx.compute_rows(d1, d2, r0, cnt)
            ctx.synchronize()
            parts_phi.append(host(ph))
            parts_psi.append(host(ps))
        phi = np.concatenate(parts_phi)
        psi = np.concatenate(parts_psi)
        # same arithmetic per element; the full call's tuned tile width may differ
        assert rel(phi, full[0]) < 1e-6 and rel(psi, full[1]) < 1e-6
        ophi, opsi, _, _ = oracle.corr2d(y1, y2)
        check(phi, psi, ophi, opsi, 1e-5, f"{world} row slabs")
    with pytest.raises(pkg.Corr2dError):
        ctx.compute_rows(d1, d2, 100, 10)  # not a multiple of 128


@pytest.mark.parametrize("homo", [True, False])
def test_tile_parts_assemble_the_full_result(ctx, homo):
    """Multi-GPU split of one problem on one GPU: each part (one per would-be GPU)
    written into its own NaN-filled buffers; every element is written by exactly one
    part, and the parts together equal the oracle (homo: exactly (anti)symmetric,
    since the parts keep the mirror)."""
    import paper_1808_00685_gb300 as pkg
    n1 = 900
    y1 = workloads.random_stack(40, n1, seed=81, offset=1.0)
    y2 = None if homo else workloads.random_stack(40, 333, seed=82, offset=-2.0)
    n2 = n1 if homo else 333
    d1 = dev(y1)
    d2 = None if homo else dev(y2)
    ophi, opsi, _, _ = oracle.corr2d(y1, y2)
    for nparts in (1, 2, 3, 5):
        got_phi, got_psi = [], []
        for part in range(nparts):
            phi, psi, _ = pkg.Context.alloc_out(n1, n2, d1.device)
            phi.fill_(float("nan"))
            psi.fill_(float("nan"))
            ph, ps = ctx.compute_part(d1, d2, part, nparts, out=(phi, psi))
            ctx.synchronize()
            got_phi.append(host(ph))
            got_psi.append(host(ps))
        wp = np.stack([~np.isnan(a) for a in got_phi])
        wq = np.stack([~np.isnan(a) for a in got_psi])
        assert np.all(wp.sum(0) == 1) and np.all(wq.sum(0) == 1), f"{nparts} parts overlap or leave gaps"
        phi = np.where(wp, np.stack(got_phi), 0.0).sum(0)
        psi = np.where(wq, np.stack(got_psi), 0.0).sum(0)
        check(phi, psi, ophi, opsi, 1e-5, f"{nparts} tile parts homo={homo}")
        if homo:
            assert np.array_equal(phi, phi.T) and np.array_equal(psi, -psi.T)
    with pytest.raises(pkg.Corr2dError):
        ctx.compute_part(d1, d2, 3, 3)


@pytest.mark.parametrize("n,m,prec,opts,nparts", [
    (129, 7, "split", {}, 4),                       # 2 tile rows: more parts than tiles
    (1000, 33, "bf16", {}, 3),
    (700, 65, "split", {"no_mirror": True}, 4),
    (700, 65, "split", {"upper_triangle": True}, 3),
    (520, 256, "split", {}, 2),
])
def test_tile_parts_edge_cases(ctx, n, m, prec, opts, nparts):
    """Ragged tile edges, BF16, NO_MIRROR (every tile, no mirrored blocks), the upper
    triangle (no mirrored blocks: nu2 >= nu1 and the diagonal tiles' mirrored lower
    halves), and more parts than tiles (empty parts write nothing)."""
    import paper_1808_00685_gb300 as pkg
    y = workloads.random_stack(m, n, seed=n + m, offset=-1.5)
    d = dev(y)
    ophi, opsi, _, _ = oracle.corr2d(y)
    upper = opts.get("upper_triangle", False)
    got = []
    for part in range(nparts):
        phi, psi, _ = pkg.Context.alloc_out(n, n, d.device)
        phi.fill_(float("nan"))
        psi.fill_(float("nan"))
        ph, ps = ctx.compute_part(d, None, part, nparts, precision=prec, out=(phi, psi), **opts)
        ctx.synchronize()
        got.append((host(ph), host(ps)))
        tiles = pkg.corr2d_plan_part(n, n, True, pkg.FLAG_NO_MIRROR if opts.get("no_mirror") else 0,
                                     part, nparts)
        if not tiles:
            assert np.all(np.isnan(got[-1][0])) and np.all(np.isnan(got[-1][1]))
    wp = np.stack([~np.isnan(a) for a, _ in got])
    phi = np.where(wp, np.stack([a for a, _ in got]), 0.0).sum(0)
    psi = np.where(wp, np.stack([b for _, b in got]), 0.0).sum(0)
    if upper:
        iu = np.triu_indices(n)
        assert np.all(wp.sum(0)[iu] == 1)
        check(phi[iu], psi[iu], ophi[iu], opsi[iu], TOL[prec], f"upper triangle in {nparts} parts")
    else:
        assert np.all(wp.sum(0) == 1)
        check(phi, psi, ophi, opsi, TOL[prec], f"{nparts} parts {prec} {opts}")


def test_upper_triangle_output(ctx):
    """CORR2D_FLAG_UPPER_TRIANGLE: nu2 >= nu1 equals the full result; lower boxes
    away from the diagonal are not written (sentinel NaNs stay)."""
    import paper_1808_00685_gb300 as pkg
    n = 700
    y = workloads.random_stack(40, n, seed=23)
    d = dev(y)
    full = run(ctx, y, precision="split", exact_symmetry=True)
    phi, psi, ldo = pkg.Context.alloc_out(n, n, d.device)
    phi.fill_(float("nan"))
    psi.fill_(float("nan"))
    ph, ps = ctx.compute(d, out=(phi, psi), upper_triangle=True)
    ctx.synchronize()
    ph, ps = host(ph)[:, :n], host(ps)[:, :n]
    iu = np.triu_indices(n)
    assert np.array_equal(ph[iu], full[0][iu]) and np.array_equal(ps[iu], full[1][iu])
    ophi, opsi, _, _ = oracle.corr2d(y)
    check(ph[iu], ps[iu], ophi[iu], opsi[iu], 1e-5, "upper triangle")
    r, c = np.indices((n, n))
    far_lower = (r // 32) > (c // 32)
    assert np.all(np.isnan(ph[far_lower])) and np.all(np.isnan(ps[far_lower]))


@pytest.mark.parametrize("reduce", [2, 5, 32])
def test_reduced_map_matches_the_full_map(ctx, reduce):
    """Sec. 4.3 `reduce`: only every reduce-th variable is correlated; equals the
    decimated full result (oracle) including the per-variable reference and scaling."""
    y1 = workloads.random_stack(30, 640, seed=24, offset=2.0)
    y2 = workloads.random_stack(30, 300, seed=25, offset=-1.0)
    for a, b in ((y1, None), (y1, y2)):
        phr, psr = ctx.compute_reduced(dev(a), None if b is None else dev(b), reduce, alpha=0.5)
        ctx.synchronize()
        ophi, opsi, _, _ = oracle.corr2d(a, b, alpha=0.5)
        check(host(phr), host(psr), oracle.reduce_map(ophi, reduce),
              oracle.reduce_map(opsi, reduce), 1e-5, f"reduce={reduce}")
    r1 = y1[0].copy()
    phr, psr = ctx.compute_reduced(dev(y1), None, reduce, ref1=dev(r1))
    ctx.synchronize()
    ophi, opsi, _, _ = oracle.corr2d(y1, ref1=r1)
    check(host(phr), host(psr), oracle.reduce_map(ophi, reduce), oracle.reduce_map(opsi, reduce),
          1e-5, f"reduce={reduce} user ref")
