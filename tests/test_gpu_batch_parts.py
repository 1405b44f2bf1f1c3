"""One batch split by problem (corr2d_plan_batch_part), each part one corr2d_batch
call, as several GPUs would run it (here one after the other on one GPU).

Every problem is computed by exactly one part, and with the tile tuner held to
its first candidate (CORR2D_NO_TUNE=1: each problem's tile choice then depends on
the problem alone, not on the batch around it) the parts give bit for bit what
one batch over the whole list gives.  Two problems are also held to the FP64
oracle at the parity tolerance (1e-5 relative Frobenius error).
"""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1808_00685_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load()
    return p


@pytest.mark.parametrize("nparts", [2, 3])
def test_batch_parts_give_the_whole_batch(pkg, nparts):
    spec = workloads.c5_spec(count=14, seed=44, m_lo=8, m_hi=200, n_lo=100, n_hi=1200)
    ins = workloads.batch_inputs(spec, nbands=6)
    shapes = [(p.m, p.n1, p.n2, p.homo) for p in spec.problems]
    parts = [pkg.plan_batch_part(shapes, r, nparts) for r in range(nparts)]
    assert sorted(i for part in parts for i in part) == list(range(len(shapes)))
    old = os.environ.get("CORR2D_NO_TUNE")
    os.environ["CORR2D_NO_TUNE"] = "1"
    ctx = pkg.Context(0)
    try:
        dev = []
        for (y1, y2) in ins:
            dev.append((torch.from_numpy(y1).cuda(),
                        None if y2 is None else torch.from_numpy(y2).cuda()))

        def outs():
            return [pkg.Context.alloc_out(p.n1, p.n2, "cuda")[:2] for p in spec.problems]

        whole = outs()
        ctx.batch([(d1, d2, a, b) for (d1, d2), (a, b) in zip(dev, whole)])
        split = outs()
        for t in split:
            t[0].fill_(float("nan"))
            t[1].fill_(float("nan"))
        for part in parts:  # one corr2d_batch call per part, as one per GPU
            ctx.batch([(dev[i][0], dev[i][1], split[i][0], split[i][1]) for i in part])
        ctx.synchronize()
    finally:
        ctx.close()
        if old is None:
            del os.environ["CORR2D_NO_TUNE"]
        else:
            os.environ["CORR2D_NO_TUNE"] = old
    for p, (a, b), (c, e) in zip(spec.problems, whole, split):
        assert torch.equal(a[:, :p.n2], c[:, :p.n2]) and torch.equal(b[:, :p.n2], e[:, :p.n2])
    for i in (0, 1):
        y1, y2 = ins[i]
        ophi, opsi, _, _ = oracle.corr2d(y1, y2, nthreads=oracle.max_threads())
        gp = split[i][0][:, :spec.problems[i].n2].double().cpu().numpy()
        gq = split[i][1][:, :spec.problems[i].n2].double().cpu().numpy()
        assert np.linalg.norm(gp - ophi) / np.linalg.norm(ophi) <= 1e-5
        assert np.linalg.norm(gq - opsi) / np.linalg.norm(opsi) <= 1e-5
