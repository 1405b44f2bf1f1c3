"""Error of Phi and Psi against the FP64 oracle for every workload and precision.

For each configuration (the paper-shaped synthetic workloads at their full
sizes) and precision the test prints one row: relative Frobenius error and
max-abs error of Phi and of Psi, with the largest oracle magnitude for scale,
and asserts the bars (1e-5 relative for FP32 and the FP16 hi/lo split, 1e-2
for plain BF16).  Maps too large for the oracle are compared on sampled
entries: seeded rows (all columns) for the single problems, 4 rows x 48
columns per problem for the batch.  Run with -s to see the table.
"""
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


def report(name, prec, phi, psi, ophi, opsi):
    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    ep, eq = rel(phi, ophi), rel(psi, opsi)
    mp, mq = np.abs(phi - ophi).max(), np.abs(psi - opsi).max()
    print(f"| {name} | {prec} | {ep:.2e} | {mp:.2e} (of {np.abs(ophi).max():.2e}) | "
          f"{eq:.2e} | {mq:.2e} (of {np.abs(opsi).max():.2e}) |")
    assert ep <= TOL[prec] and eq <= TOL[prec], f"{name} {prec}: {ep:.3e} {eq:.3e}"


_ORACLE = {}


def oracle_once(key, fn):
    """The oracle's result for a configuration, computed once for all precisions."""
    if key not in _ORACLE:
        _ORACLE[key] = fn()
    return _ORACLE[key]


def rows_of(phi, psi, rows):
    rt = torch.from_numpy(rows.astype(np.int64)).cuda()
    return host(phi.index_select(0, rt)), host(psi.index_select(0, rt))


@pytest.mark.parametrize("prec", ["split", "bf16", "fp32"])
def test_c1_c2_full_maps(ctx, prec):
    for name, y in (("c1 homo m=11 n=500", workloads.c1()),
                    ("c2 homo m=64 n=4096 (baseline 10)", workloads.c2())):
        phi, psi = ctx.compute(dev(y), precision=prec)
        ctx.synchronize()
        ophi, opsi, _, _ = oracle_once(name, lambda: oracle.corr2d(y, nthreads=oracle.max_threads()))
        n = y.shape[1]
        report(name, prec, host(phi)[:, :n], host(psi)[:, :n], ophi, opsi)


@pytest.mark.parametrize("prec", ["split", "bf16", "fp32"])
def test_c3_preprocessed_hetero_sampled_rows(ctx, prec):
    raw = workloads.c3()
    y1, _ = ctx.preprocess(dev(raw.x1), dev(raw.y1), raw.n1_out)
    y2, _ = ctx.preprocess(dev(raw.x2), dev(raw.y2), raw.n2_out)
    phi, psi = ctx.compute(y1, y2, precision=prec, alpha=raw.alpha)
    ctx.synchronize()
    rows = workloads.sample_rows(raw.n1_out, 512, seed=31)
    gphi, gpsi = rows_of(phi, psi, rows)
    def ref():
        o1, _ = oracle.interp_linear(raw.x1, raw.y1, raw.n1_out)
        o2, _ = oracle.interp_linear(raw.x2, raw.y2, raw.n2_out)
        return oracle.corr2d(o1.astype(np.float32), o2.astype(np.float32), alpha=raw.alpha,
                             rows=rows, nthreads=oracle.max_threads())
    ophi, opsi, _, _ = oracle_once("c3", ref)
    report("c3 hetero m=128 8192 x 2048, alpha 0.5, 512 rows", prec, gphi, gpsi, ophi, opsi)


@pytest.mark.parametrize("prec", ["split", "bf16", "fp32"])
def test_c4_sampled_rows(ctx, prec):
    y = workloads.c4()
    phi, psi = ctx.compute(dev(y), precision=prec)
    ctx.synchronize()
    rows = workloads.sample_rows(y.shape[1], 256, seed=41)
    gphi, gpsi = rows_of(phi, psi, rows)
    del phi, psi
    torch.cuda.empty_cache()
    ophi, opsi, _, _ = oracle_once("c4", lambda: oracle.corr2d(y, rows=rows,
                                                               nthreads=oracle.max_threads()))
    report("c4 homo m=256 n=32768, 256 rows", prec, gphi, gpsi, ophi, opsi)


@pytest.mark.parametrize("prec", ["split", "bf16"])
def test_c5_batch_sampled_entries(ctx, prec):
    import paper_1808_00685_gb300 as pkg
    spec = workloads.c5_spec()
    ins = workloads.batch_inputs(spec)
    probs = []
    for (y1, y2), p in zip(ins, spec.problems):
        d1 = dev(y1)
        d2 = None if y2 is None else dev(y2)
        phi, psi, _ = pkg.Context.alloc_out(p.n1, p.n2, d1.device)
        probs.append((d1, d2, phi, psi))
    ctx.batch(probs, precision=prec)
    ctx.synchronize()
    g_p, g_q, o_p, o_q = [], [], [], []
    for i, ((y1, y2), p, (_, _, phi, psi)) in enumerate(zip(ins, spec.problems, probs)):
        rows = workloads.sample_rows(p.n1, 4, seed=9000 + i)
        cols = workloads.sample_rows(p.n2, 48, seed=19000 + i)
        rt = torch.from_numpy(rows.astype(np.int64)).cuda()
        ct = torch.from_numpy(cols.astype(np.int64)).cuda()
        g_p.append(host(phi.index_select(0, rt).index_select(1, ct)).ravel())
        g_q.append(host(psi.index_select(0, rt).index_select(1, ct)).ravel())
        ys2 = (y1 if y2 is None else y2)[:, cols]
        ophi, opsi, _, _ = oracle.corr2d(np.ascontiguousarray(y1[:, rows]), np.ascontiguousarray(ys2))
        # each problem's entries relative to its own scale, so that no problem dominates
        scale = max(np.linalg.norm(ophi), 1e-300)
        g_p[-1] /= scale
        g_q[-1] /= scale
        o_p.append(ophi.ravel() / scale)
        o_q.append(opsi.ravel() / scale)
    report("c5 batch of 512, 4 x 48 entries per problem (normalised per problem)", prec,
           np.concatenate(g_p), np.concatenate(g_q), np.concatenate(o_p), np.concatenate(o_q))
