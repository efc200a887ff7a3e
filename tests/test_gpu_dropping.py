"""The paper's global dropping operators on the GPU against the oracle, bit
for bit: hard thresholding with a global density cap (Sec. 6.1) and the
Appendix A heuristic (symmetrise, round-off drop, Eq. 435 scores)."""
import numpy as np
import pytest

import oracle as O
from oracle import dropping as D
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_global_hard_threshold_matches_oracle(prec):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.laplacian_2d_5pt(24)   # many exact ties in |m|
    for frac in (0.35, 0.6, 0.9):
        g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=3.0)
        o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=3.0)
        g.run("mr", 4)
        o.run("mr", 4)
        M = o.get_M()
        assert _same(g.get_M(), M)
        m = int(frac * len(M[2]))
        g.drop_global(m)
        want = D.hard_threshold(n, M, m)
        got = g.get_M()
        assert len(got[2]) == m
        assert _same(got, want)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_appendix_heuristic_matches_oracle(prec):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((11, 13), seed=7)
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=6.0)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=6.0)
    g.run("lomr", 3)
    o.run("lomr", 3)
    M = o.get_M()
    assert _same(g.get_M(), M)
    for m in (10 ** 9, 4 * n, 2 * n):
        gg = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=6.0)
        gg.set_M(*M)
        gg.drop_heuristic(m)
        want = D.heuristic(n, rp, ci, v, M, m, mixed=(prec == "mixed"))
        got = gg.get_M()
        assert _same(got, want), m
