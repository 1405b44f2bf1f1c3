"""Failure detection without a GPU fault.

* CORR2D_FAULT=stall makes the cross-spectrum producer issue nothing: the MMA
  and epilogue warps' bounded waits must run out (CORR2D_WAIT_LIMIT_MS), the
  kernel must return on its own, and corr2d_synchronize must report
  CORR2D_ETIMEOUT; the GPU context stays usable afterwards.
* CORR2D_FAULT=alloc refuses the workspace allocation on the host: ENOMEM.
No test here traps, faults or hangs the GPU.
"""
import os
import time

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


def _context_with_env(pkg, **env):
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return pkg.Context(0)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_stalled_producer_times_out_and_context_survives(pkg):
    y = torch.from_numpy(workloads.random_stack(16, 300, seed=3)).cuda()
    ctx = _context_with_env(pkg, CORR2D_FAULT="stall", CORR2D_WAIT_LIMIT_MS="200")
    try:
        t0 = time.time()
        ctx.compute(y, precision="split", no_mirror=True)
        with pytest.raises(pkg.Corr2dError) as ei:
            ctx.synchronize()
        dt = time.time() - t0
        assert ei.value.status == pkg.ETIMEOUT
        assert 0.15 < dt < 30.0
        ctx.synchronize()  # the error word was cleared
    finally:
        ctx.close()
    # a normal context on the same GPU still computes correct results
    with pkg.Context(0) as ok:
        phi, psi = ok.compute(y, precision="split")
        ok.synchronize()
        ophi, _, _, _ = oracle.corr2d(y.cpu().numpy())
        err = np.linalg.norm(phi.double().cpu().numpy() - ophi) / np.linalg.norm(ophi)
        assert err < 1e-5


def test_refused_allocation_reports_enomem(pkg):
    y = torch.from_numpy(workloads.random_stack(8, 64, seed=4)).cuda()
    ctx = _context_with_env(pkg, CORR2D_FAULT="alloc")
    try:
        with pytest.raises(pkg.Corr2dError) as ei:
            ctx.compute(y)
        assert ei.value.status == pkg.ENOMEM
        assert "injected" in str(ei.value)
    finally:
        ctx.close()
