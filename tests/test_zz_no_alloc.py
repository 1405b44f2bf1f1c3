"""The allocation-free entry point against the ordinary one.

corr2d_compute_noalloc serves callers that must not allocate GPU memory (no
library context, no cudaMalloc/cudaFree): its intermediates live in a static
device array.  Here it is called through the C ABI twice in a row (the second
call reuses the array the first one left behind) and each result is compared
with corr2d_compute on the same inputs, within the parity tolerance of the
other GPU tests.  Requests larger than the static array must be refused up
front.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def pkg():
    import paper_1808_00685_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load()
    return p


def _noalloc(pkg, y1, y2, params, n1, n2):
    """Run the allocation-free entry point; outputs are allocated by the test."""
    phi, psi, ldo = pkg.Context.alloc_out(n1, n2, y1.device)
    stream = torch.cuda.current_stream().cuda_stream
    m = y1.shape[0]
    pkg.corr2d_compute_noalloc(0, stream, m, n1, y1.data_ptr(), y1.stride(0), n2,
                               None if y2 is None else y2.data_ptr(),
                               0 if y2 is None else y2.stride(0), params, phi.data_ptr(),
                               psi.data_ptr(), ldo)
    return phi[:, :n2].double().cpu().numpy(), psi[:, :n2].double().cpu().numpy()


@pytest.mark.parametrize("case", ["homo", "hetero"])
def test_noalloc_matches_compute_twice(pkg, case):
    if case == "homo":
        y1 = workloads.sigmoid_bands(64, 1000, 20, seed=21)
        y2 = None
    else:
        y1 = workloads.random_stack(100, 700, seed=22, offset=2.0)
        y2 = workloads.random_stack(100, 500, seed=23, offset=-1.0)
    d1 = torch.from_numpy(y1).cuda()
    d2 = None if y2 is None else torch.from_numpy(y2).cuda()
    n1 = y1.shape[1]
    n2 = n1 if y2 is None else y2.shape[1]
    with pkg.Context(0) as ctx:
        ref_phi, ref_psi = ctx.compute(d1, d2, precision="split", alpha=0.5)
        ctx.synchronize()
        ref_phi = ref_phi.double().cpu().numpy()
        ref_psi = ref_psi.double().cpu().numpy()
    params = pkg.make_params("split", alpha=0.5)
    for call in range(2):
        phi, psi = _noalloc(pkg, d1, d2, params, n1, n2)
        assert _rel(phi, ref_phi) <= TOL, f"call {call}: Phi {_rel(phi, ref_phi):.3e}"
        assert _rel(psi, ref_psi) <= TOL, f"call {call}: Psi {_rel(psi, ref_psi):.3e}"


def test_noalloc_refuses_problems_beyond_its_scratch(pkg):
    y = torch.zeros((256, 20000), dtype=torch.float32, device="cuda")
    phi = torch.empty((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.Corr2dError) as ei:
        pkg.corr2d_compute_noalloc(0, torch.cuda.current_stream().cuda_stream, 256, 20000,
                                   y.data_ptr(), 20000, 0, None, 0, pkg.make_params("split"),
                                   phi.data_ptr(), phi.data_ptr(), 20000)
    assert ei.value.status == pkg.EUNSUPPORTED
    assert "scratch" in str(ei.value)
