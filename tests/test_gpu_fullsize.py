"""Parity at the full size of the benchmark workload: the 64^3 variable-
coefficient operator (n = 262,144, 1,810,432 entries), mixed arithmetic,
cap 3 nnz(A[:,j]), with the launch shapes the autotuner picks (as
bench.py does).  Three iterations of each method against the oracle, bit for
bit: histories, coefficients and all 5.4 M entries of M; then 30 iterations
of the mixed PCG with the symmetric part of M, x bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATUS = {0: 0, 1: 3, 2: 4}


@pytest.fixture(scope="module")
def workload():
    return I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_bench_workload_matches_oracle(workload, method):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = workload
    g = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=3.0)
    g.set_pcg_prec("mixed")
    g.autotune(method, 2)
    r = g.run(method, 3)
    o = O.Oracle(n, rp, ci, v, mixed=True, cap_factor=3.0)
    ro = o.run(method, 3)
    assert r["done"] == ro["done"] == 3
    np.testing.assert_array_equal(r["resnorm"], ro["resnorm"])
    np.testing.assert_array_equal(r["coef"][:3], ro["coef"][:3])
    gm, om = g.get_M(), o.get_M()
    assert all(np.array_equal(a, b) for a, b in zip(gm, om))
    b = I.rhs_uniform(n, 0)
    p = g.pcg(b.copy(), rtol=1e-8, maxit=30, precond=spai.PREC_SPAI_SYM)
    po = O.pcg(n, rp, ci, v, b, rtol=1e-8, maxit=30, precond=3, M=om, mixed=True)
    assert p["iters"] == po["iters"] == 30
    assert p["status"] == STATUS[po["status"]]
    assert np.array_equal(p["x"], po["x"])
