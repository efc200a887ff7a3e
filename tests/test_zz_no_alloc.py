"""The allocation-free residual entry point.

spai_true_residual_noalloc serves callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or they cannot pay
for cudaMalloc/cudaFree in a latency-critical loop).  It keeps its
workspace in a fixed array inside the library, so these checks run it twice
in a row (the second call finds the first call's leftovers in that array)
and compare it, through the C ABI, with the residual that pcg_solve reports.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _device_problem(n, rp, ci, v, b, x):
    import torch
    dev = "cuda"
    return (torch.tensor(rp, dtype=torch.int32, device=dev),
            torch.tensor(ci, dtype=torch.int32, device=dev),
            torch.tensor(v, dtype=torch.float64, device=dev),
            torch.tensor(b, dtype=torch.float64, device=dev),
            torch.tensor(x, dtype=torch.float64, device=dev))


# n = 1,024 and 8,000 fit in one group of 64 CTAs; n = 40,000 takes three
# groups (the cross-group hand-off) and n = 592,704 thirty-seven (the top
# level of the tree over more than 32 group sums)
@pytest.mark.parametrize("make", [lambda: I.laplacian_2d_5pt(32),
                                  lambda: I.varcoef_3d_7pt(20, seed=2),
                                  lambda: I.laplacian_2d_5pt(200),
                                  lambda: I.varcoef_3d_7pt(84, seed=4)],
                         ids=["lap32", "varcoef20", "lap200", "varcoef84"])
def test_noalloc_residual_matches_pcg_relres_twice(make):
    import torch
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = make()
    g = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
    g.mr(6)
    b = I.rhs_uniform(n, 0)
    res = g.pcg(b, rtol=1e-6, maxit=500, precond=spai.PREC_SPAI_SYM)
    x = res["x"]
    drp, dci, dv, db, dx = _device_problem(n, rp, ci, v, b, x)
    for _ in range(2):  # two calls in a row share the library's workspace
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = spai.true_residual_noalloc(n, drp, dci, dv, db, dx, out)
        assert rc == 0
        torch.cuda.synchronize()
        rnorm, bnorm = out.cpu().numpy()
        assert rnorm / bnorm == res["relres"]
        assert abs(bnorm - np.linalg.norm(b)) <= 1e-14 * bnorm


def test_noalloc_rejects_oversized_problem():
    import torch
    from paper_2511_09753_gb300 import spai
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = spai.true_residual_noalloc((1 << 24) + 1, i, i, t, t, t, t)
    assert rc == -9  # SPAI_ERR_UNSUPPORTED: above the fixed workspace's limit
    assert spai.true_residual_noalloc(0, i, i, t, t, t, t) == -1
