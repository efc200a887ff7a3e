"""MR, LOMR and CG (and their Pi forms) with the paper's global dropping
inside every iteration (directions hard-thresholded over the whole matrix,
Appendix A heuristic on M) on the GPU against the oracle's flows, bit for
bit."""
import numpy as np
import pytest

from oracle import dropping as D
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FLOWS = {"mr": D.run_global_mr, "lomr": D.run_global_lomr, "cg": D.run_global_cg}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("method", ["mr", "mr_pi", "lomr", "lomr_pi", "cg", "cg_pi"])
def test_run_global_matches_oracle(prec, method):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((9, 11), seed=5)
    nnzA = len(v)
    iters, m_dir, m_M = 4, 2 * nnzA, int(1.5 * nnzA)
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=12.0)
    r = g.run_global(method, iters, m_dir, m_M)
    base = method.split("_")[0]
    o = FLOWS[base](n, rp, ci, v, iters, m_dir, m_M, mixed=(prec == "mixed"),
                    use_pi=method.endswith("_pi"))
    assert r["done"] == o["done"] == iters
    np.testing.assert_array_equal(r["resnorm"], o["resnorm"])
    if base == "mr":
        np.testing.assert_array_equal(r["coef"][:iters, 0], o["coef"])
    else:
        np.testing.assert_array_equal(r["coef"][:iters], o["coef"])
    if base == "lomr":
        assert bool(r["flags"] & 2) == o["fallback"]
    got = g.get_M()
    assert all(np.array_equal(a, b) for a, b in zip(got, o["M"]))
    assert len(got[2]) <= m_M


def test_run_global_then_plain_run_continues_from_the_dropped_m():
    """After a global-dropping call, spai_run starts a fresh recurrence from
    the M it left (the same as the oracle's method run from that M)."""
    import oracle as O
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((9, 11), seed=5)
    g = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=12.0)
    g.run_global("lomr", 2, 2 * len(v), int(1.5 * len(v)))
    o = O.Oracle(n, rp, ci, v, mixed=True, cap_factor=12.0)
    o.set_M(*g.get_M())
    rg, ro = g.run("cg", 3), o.run("cg", 3)
    np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
    assert all(np.array_equal(a, b) for a, b in zip(g.get_M(), o.get_M()))


@pytest.mark.parametrize("method", ["mr", "lomr", "cg_pi"])
def test_run_global_zero_iterations_records_the_initial_residual(method):
    import oracle as O
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((9, 11), seed=5)
    g = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=12.0)
    r = g.run_global(method, 0, 2 * len(v), int(1.5 * len(v)))
    o = O.Oracle(n, rp, ci, v, cap_factor=12.0)
    assert r["done"] == 0
    assert r["resnorm"][0] == o.run("mr", 0)["resnorm"][0]  # ||I - A M_0||_F
    assert all(np.array_equal(a, b) for a, b in zip(g.get_M(), o.get_M()))
