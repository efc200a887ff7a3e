"""MR and MR_SPD with the paper's global dropping inside every iteration
(direction hard-thresholded over the whole matrix, Appendix A heuristic on
M) on the GPU against the oracle's flow, bit for bit."""
import numpy as np
import pytest

from oracle import dropping as D
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("method", ["mr", "mr_pi"])
def test_run_global_matches_oracle(prec, method):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((9, 11), seed=5)
    nnzA = len(v)
    iters, m_dir, m_M = 4, 2 * nnzA, int(1.5 * nnzA)
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=12.0)
    r = g.run_global(method, iters, m_dir, m_M)
    o = D.run_global_mr(n, rp, ci, v, iters, m_dir, m_M, mixed=(prec == "mixed"),
                        use_pi=(method == "mr_pi"))
    assert r["done"] == o["done"] == iters
    np.testing.assert_array_equal(r["resnorm"], o["resnorm"])
    np.testing.assert_array_equal(r["coef"][:iters, 0], o["coef"])
    got = g.get_M()
    assert all(np.array_equal(a, b) for a, b in zip(got, o["M"]))
    assert len(got[2]) <= m_M
