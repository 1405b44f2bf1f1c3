"""BF16 output (CORR2D_FLAG_OUTPUT_BF16): Phi and Psi stored as bfloat16.

The kernel computes the same FP32 values as with FP32 output and rounds each to
the nearest BF16 (ties to even) before staging it, so every BF16 output here must
equal the FP32 output of the same call rounded by torch, bit for bit, on every
entry point that stores through the tensor-core kernel (single calls on mirrored
and full tiles, hetero, BF16 operands, the Hilbert variant, the upper triangle,
row slabs, tile parts, the reduced map and the batch).  Against the FP64 oracle
that leaves the rounding: BF16's unit roundoff 2^-8 plus the FP32 path's 1e-5,
checked at the 1e-2 tolerance of the BF16 forms (relative Frobenius error and,
element-wise, 2^-8 |oracle| + 4e-5 x the largest magnitude).  The entry points
that cannot store BF16 refuse the flag.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module", autouse=True)
def one_tile_choice():
    """Both calls of a comparison take the same tile layout (the tuner's first
    candidate): full and mirrored tiles may differ in the last FP32 bit of the
    mirrored half, and the tuner times FP32 and BF16 outputs separately."""
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


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def _same_bits(b16, f32):
    """b16 (BF16 tensor) equals f32 (FP32 tensor) rounded to nearest BF16."""
    want = f32.to(torch.bfloat16)
    return torch.equal(b16.contiguous().view(torch.int16), want.contiguous().view(torch.int16))


def _near_oracle(b16, o):
    g = b16.double().cpu().numpy()
    big = np.abs(o).max()
    assert np.linalg.norm(g - o) / np.linalg.norm(o) <= 1e-2
    assert np.all(np.abs(g - o) <= U_BF16 * np.abs(o) + 4e-5 * big)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    ("homo m=64 n=4096", (64, 4096, None), {}),
    ("homo m=64 n=4096 mirrored", (64, 4096, None), {"exact_symmetry": True}),
    ("hetero m=100 1000 x 517 alpha 0.5", (100, 1000, 517), {"alpha": 0.5}),
    ("homo m=33 n=700 bf16 operands", (33, 700, None), {"precision": "bf16"}),
    ("homo m=40 n=600 Hilbert", (40, 600, None), {"hilbert": True}),
]


@pytest.mark.parametrize("name,shape,kw", CASES, ids=[c[0] for c in CASES])
def test_bf16_output_is_the_fp32_output_rounded(ctx, name, shape, kw):
    m, n1, n2 = shape
    if name.startswith("homo m=64"):
        y1, y2 = workloads.c2()[:, :n1], None
    else:
        y1 = workloads.random_stack(m, n1, seed=m + n1, offset=2.0)
        y2 = None if n2 is None else workloads.random_stack(m, n2, seed=n2, offset=-1.0)
    d1, d2 = _dev(y1), None if y2 is None else _dev(y2)
    p32, q32 = ctx.compute(d1, d2, **kw)
    p16, q16 = ctx.compute(d1, d2, output_bf16=True, **kw)
    ctx.synchronize()
    assert p16.dtype == torch.bfloat16 and q16.dtype == torch.bfloat16
    assert _same_bits(p16, p32) and _same_bits(q16, q32), name
    if kw.get("exact_symmetry"):
        assert torch.equal(p16, p16.T) and torch.equal(q16, -q16.T)
    if kw.get("hilbert"):
        return  # the Hilbert oracle comparison lives with the FP32 output
    alpha = kw.get("alpha", 0.0)
    prec = kw.get("precision", "split")
    ophi, opsi, _, _ = oracle.corr2d(y1, y2, alpha=alpha, nthreads=oracle.max_threads())
    if prec == "split":
        _near_oracle(p16, ophi)
        _near_oracle(q16, opsi)


def test_bf16_output_on_slabs_parts_reduced_and_upper_triangle(ctx):
    n = 1100
    y = workloads.random_stack(48, n, seed=71, offset=1.0)
    d = _dev(y)
    # upper triangle: only nu2 >= nu1 is specified
    p32, q32 = ctx.compute(d, upper_triangle=True)
    p16, q16 = ctx.compute(d, upper_triangle=True, output_bf16=True)
    ctx.synchronize()
    iu = np.triu_indices(n)
    assert _same_bits(p16.cpu()[iu], p32.cpu()[iu]) and _same_bits(q16.cpu()[iu], q32.cpu()[iu])
    # row slab [256, 640)
    a32, b32 = ctx.compute_rows(d, None, 256, 384)
    a16, b16 = ctx.compute_rows(d, None, 256, 384, output_bf16=True)
    ctx.synchronize()
    assert _same_bits(a16, a32) and _same_bits(b16, b32)
    # tile parts of the mirrored list, assembled
    full16 = [t.fill_(float("nan")) for t in ctx.alloc_out(n, n, d.device, bf16=True)[:2]]
    full32 = [t.fill_(float("nan")) for t in ctx.alloc_out(n, n, d.device)[:2]]
    for part in range(3):
        ctx.compute_part(d, None, part, 3, out=tuple(full32))
        ctx.compute_part(d, None, part, 3, out=tuple(full16), output_bf16=True)
    ctx.synchronize()
    for x16, x32 in zip(full16, full32):
        assert not torch.isnan(x32[:, :n]).any()
        assert _same_bits(x16[:, :n], x32[:, :n])
    # reduced map, every 3rd variable
    r32, s32 = ctx.compute_reduced(d, None, 3)
    r16, s16 = ctx.compute_reduced(d, None, 3, output_bf16=True)
    ctx.synchronize()
    assert _same_bits(r16, r32) and _same_bits(s16, s32)


def test_bf16_output_batch(pkg, ctx):
    spec = workloads.c5_spec(count=10, seed=33, m_lo=8, m_hi=200, n_lo=100, n_hi=1500)
    ins = workloads.batch_inputs(spec, nbands=6)
    p32, p16 = [], []
    for (y1, y2), p in zip(ins, spec.problems):
        d1, d2 = _dev(y1), None if y2 is None else _dev(y2)
        a, b, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
        c, e, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device, bf16=True)
        p32.append((d1, d2, a, b))
        p16.append((d1, d2, c, e))
    ctx.batch(p32)
    ctx.batch(p16, output_bf16=True)
    ctx.synchronize()
    for (_, _, a, b), (_, _, c, e), p in zip(p32, p16, spec.problems):
        assert _same_bits(c[:, :p.n2], a[:, :p.n2]) and _same_bits(e[:, :p.n2], b[:, :p.n2])
    (y1, y2), p = ins[1], spec.problems[1]
    ophi, opsi, _, _ = oracle.corr2d(y1, y2, nthreads=oracle.max_threads())
    _near_oracle(p16[1][2][:, :p.n2], ophi)
    _near_oracle(p16[1][3][:, :p.n2], opsi)


def test_bf16_output_takes_the_single_cta_kernel_when_others_are_asked_for(pkg, ctx):
    y = workloads.random_stack(64, 900, seed=5, offset=0.5)
    d = _dev(y)
    p32, q32 = ctx.compute(d)  # the single-CTA kernel, FP32 output
    ctx.synchronize()
    old = os.environ.get("CORR2D_XSPEC")
    os.environ["CORR2D_XSPEC"] = "any"  # read by every call's tile choice
    c = pkg.Context(0)
    try:
        p16, q16 = c.compute(d, output_bf16=True)
        c.synchronize()
        assert c.kernel_info()[0] == pkg.XSPEC_TC
        assert _same_bits(p16, p32) and _same_bits(q16, q32)
    finally:
        c.close()
        if old is None:
            del os.environ["CORR2D_XSPEC"]
        else:
            os.environ["CORR2D_XSPEC"] = old


def test_bf16_output_is_refused_where_it_cannot_be_stored(pkg, ctx):
    y = workloads.random_stack(16, 200, seed=2)
    d = _dev(y)
    with pytest.raises(pkg.Corr2dError) as ei:
        ctx.compute(d, precision="fp32", output_bf16=True)
    assert ei.value.status == pkg.EUNSUPPORTED
    # ldo must be a multiple of 8 BF16 elements
    phi = torch.empty((200, 204), dtype=torch.bfloat16, device="cuda")
    psi = torch.empty((200, 204), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_compute(ctx.handle, 16, 200, d.data_ptr(), 200, 0, None, 0,
                           pkg.make_params(output_bf16=True), phi.data_ptr(), psi.data_ptr(), 204)
    assert ei.value.status == pkg.EINVAL
    # host buffers: FP32 slabs only
    yh = torch.from_numpy(y)
    ph = torch.empty((200, 256), dtype=torch.bfloat16)
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_compute_host(ctx.handle, 16, 200, yh.data_ptr(), 0, None,
                                pkg.make_params(output_bf16=True), ph.data_ptr(), ph.data_ptr(),
                                256)
    assert ei.value.status == pkg.EUNSUPPORTED
    # an unknown flag bit
    p = pkg.make_params()
    p.flags |= 1 << 10
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_compute(ctx.handle, 16, 200, d.data_ptr(), 200, 0, None, 0, p,
                           phi.data_ptr(), psi.data_ptr(), 200)
    assert ei.value.status == pkg.EINVAL


@pytest.mark.parametrize("m,n1,n2", [(2, 1, None), (2, 7, None), (3, 33, None), (4, 129, None),
                                     (5, 128, None), (16, 257, None), (130, 131, None),
                                     (257, 140, None), (512, 64, None), (9, 1, 40), (33, 70, 1),
                                     (65, 300, 77)])
def test_bf16_output_on_ragged_and_extreme_shapes(ctx, m, n1, n2):
    """Single variables, one step past a tile, the largest m: every BF16 element is
    the FP32 element rounded (boxes cut at ragged edges, the m = 2 zero map)."""
    y1 = workloads.random_stack(m, n1, seed=m * 1000 + n1, offset=3.0)
    y2 = None if n2 is None else workloads.random_stack(m, n2, seed=m * 77 + n2, offset=-1.0)
    d1, d2 = _dev(y1), None if y2 is None else _dev(y2)
    p32, q32 = ctx.compute(d1, d2)
    p16, q16 = ctx.compute(d1, d2, output_bf16=True)
    ctx.synchronize()
    assert _same_bits(p16, p32) and _same_bits(q16, q32), (m, n1, n2)
