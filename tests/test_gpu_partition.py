"""Partition invariance of the structure factor on the GPU: rho(k_l) of a system equals the
sum of the rho of its spatial slabs (the partial sums one GPU per slab would all-reduce),
computed by the FP32 structure-factor kernel through rbsog_rho_noalloc, and the oracle's."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, modes_for, require_gpu, workload
from oracle import core
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("slabs", [2, 3, 8])
def test_rho_of_slabs_sums_to_rho_of_the_system(slabs):
    torch = require_gpu()
    w = workload(30000, 30.0, P=300, seed=77)
    r = W.positions(w)
    q = np.where(np.arange(w.N) % 3 == 0, -1.0, 1.0)
    modes = modes_for(w, w.P, 78)
    md = torch.tensor(modes, device="cuda", dtype=torch.int32)

    def rho_gpu(sel):
        rd = torch.tensor(r[sel], device="cuda", dtype=torch.float64)
        qd = torch.tensor(q[sel], device="cuda", dtype=torch.float64)
        out = torch.zeros((w.P, 2), device="cuda", dtype=torch.float64)
        R.rbsog_rho_noalloc(rd, qd, int(sel.size), w.box, md, w.P, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    whole = rho_gpu(np.arange(w.N))
    edges = np.linspace(0.0, w.box[0], slabs + 1)
    parts = [np.nonzero((r[:, 0] >= edges[k]) & (r[:, 0] < edges[k + 1]))[0] for k in range(slabs)]
    assert sum(p.size for p in parts) == w.N
    summed = sum(rho_gpu(p) for p in parts)
    ref = core.rho(r, q, w.box, modes)
    scale = float(np.max(np.abs(ref)))
    assert np.max(np.abs(summed - whole)) <= FP32_TOL * scale
    assert np.max(np.abs(summed - ref)) <= FP32_TOL * scale
    assert np.max(np.abs(whole - ref)) <= FP32_TOL * scale
