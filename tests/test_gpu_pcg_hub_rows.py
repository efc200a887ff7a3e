"""PCG (Sec. 7's assessment) with hub rows in the symmetric part S of M:
rows longer than the sliced ELL takes (64 entries) are multiplied by a
thread each, and the other rows then sit in the sliced ELL longest first.
Every row's product is still the fma chain over ascending column, so x, the
iteration count, the status and relres equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATUS = {0: 0, 1: 3, 2: 4}


def _hub_matrix(n, rp, ci, v, hubs, width, seed):
    """diag(A)^-1 plus, in each hub row h, `width` small entries m_hj at
    random columns j (each column then holds at most a few entries), so row
    h of S has about `width` entries."""
    rng = np.random.default_rng(seed)
    d = np.zeros(n)
    for i in range(n):
        row = ci[rp[i]:rp[i + 1]]
        d[i] = v[rp[i]:rp[i + 1]][np.nonzero(row == i)[0][0]]
    cols = [{j: 1.0 / d[j]} for j in range(n)]
    for h in sorted(hubs):
        for j in rng.choice(n, size=width, replace=False):
            if int(j) != h:
                cols[int(j)][h] = 1e-3 * rng.uniform(-1.0, 1.0) / d[int(j)]
    colptr, rowind, vals = [0], [], []
    for j in range(n):
        for r in sorted(cols[j]):
            rowind.append(r)
            vals.append(cols[j][r])
        colptr.append(len(rowind))
    return (np.array(colptr, np.int32), np.array(rowind, np.int32), np.array(vals, np.float64))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("hubs", [(5,), (5, 700, 2222, 4095), tuple(range(0, 4096, 97))])
def test_pcg_with_hub_rows_matches_oracle(prec, hubs):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(16, seed=3)
    M = _hub_matrix(n, rp, ci, v, hubs=set(hubs), width=200, seed=9)
    g = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
    g.set_M(*M)
    g.set_pcg_prec(prec)
    b = I.rhs_uniform(n, 2)
    for maxit in (3, 2000):
        r = g.pcg(b.copy(), rtol=1e-9, maxit=maxit, precond=spai.PREC_SPAI_SYM)
        ro = O.pcg(n, rp, ci, v, b, rtol=1e-9, maxit=maxit, precond=3, M=M, mixed=prec == "mixed")
        assert r["iters"] == ro["iters"]
        assert r["status"] == STATUS[ro["status"]]
        assert np.array_equal(r["x"], ro["x"])
        assert r["relres"] == ro["relres"]
    g.close()
