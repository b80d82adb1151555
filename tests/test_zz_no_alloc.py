"""rbsog_rho_noalloc: the structure factor for callers that cannot allocate device memory.

Its partial sums live in a fixed static device array instead of memory from cudaMalloc.
Checked through the C ABI against the structure factor of the regular context path
(rbsog_forces + rbsog_get_rho) on the same particles and modes, on two calls in a row
(the second call reuses the array the first one left behind).  This file is collected
last so that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, Ctx, modes_for, require_gpu, workload
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


# (12000, 1724): 152 blocks x 1724 modes = 262048 of the 262144 slots, four modes per lane
@pytest.mark.parametrize("N,L,P", [(20000, 27.0, 200), (3000, 14.0, 700), (500, 8.0, 40), (12000, 24.0, 1724)])
def test_rho_noalloc_matches_the_context_structure_factor(N, L, P):
    torch = require_gpu()
    w = workload(N, L, P=P, seed=N)
    r = W.positions(w)
    q = W.charges(w)
    modes = modes_for(w, P, 3)
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, r)
        R.rbsog_set_ksample(c.h, modes)
        R.rbsog_forces(c.h)
        ref = R.rbsog_get_rho(c.h, P)
    rd = torch.tensor(r, device="cuda", dtype=torch.float64)
    qd = torch.tensor(q, device="cuda", dtype=torch.float64)
    md = torch.tensor(modes, device="cuda", dtype=torch.int32)
    scale = float(np.max(np.abs(ref)))
    for call in range(2):
        out = torch.full((P, 2), float("nan"), device="cuda", dtype=torch.float64)
        R.rbsog_rho_noalloc(rd, qd, N, w.box, md, P, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.max(np.abs(got - ref)) <= FP32_TOL * scale, (call, np.max(np.abs(got - ref)) / scale)


@pytest.mark.parametrize("N,P", [(20000, 4096), (12000, 1725)])
def test_rho_noalloc_rejects_requests_beyond_its_scratch(N, P):
    """P = 1725 at 152 blocks needs 262200 slots, one mode more than the array holds."""
    torch = require_gpu()
    rd = torch.zeros((N, 3), device="cuda", dtype=torch.float64)
    qd = torch.ones(N, device="cuda", dtype=torch.float64)
    md = torch.ones((P, 3), device="cuda", dtype=torch.int32)
    out = torch.zeros((P, 2), device="cuda", dtype=torch.float64)
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_rho_noalloc(rd, qd, N, (10.0, 10.0, 10.0), md, P, out)
    assert "scratch" in R.rbsog_last_error(None)
