"""Mixed-arithmetic PCG (FP32-values products, FP64 recurrences): the GPU's
vector and block solves against the oracle's mixed PCG, bit for bit, and the
mixed solve against the FP64 one within the stated tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATUS = {0: 0, 1: 3, 2: 4}

OPS = {
    "lap2d_32": lambda: I.laplacian_2d_5pt(32),
    "varcoef_17x19": lambda: I.varcoef_grid((17, 19), seed=4),
    "aniso9_30": lambda: I.aniso_2d_9pt(30),          # 9 entries per row: the wide-row path
}


@pytest.mark.parametrize("name", sorted(OPS))
@pytest.mark.parametrize("precond", [0, 1, 2, 3])
def test_vector_pcg_mixed_matches_oracle(name, precond):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = OPS[name]()
    s = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=2.0)
    s.run("lomr", 8)
    s.set_pcg_prec("mixed")
    o = O.Oracle(n, rp, ci, v, mixed=True, cap_factor=2.0)
    o.run("lomr", 8)
    b = I.rhs_uniform(n, 1)
    r = s.pcg(b.copy(), rtol=1e-8, maxit=600, precond=precond)
    ro = O.pcg(n, rp, ci, v, b, rtol=1e-8, maxit=600, precond=precond,
               M=o.get_M() if precond in (2, 3) else None, mixed=True)
    assert r["iters"] == ro["iters"]
    assert r["status"] == STATUS[ro["status"]]
    assert np.array_equal(r["x"], ro["x"])
    assert r["relres"] == ro["relres"]


@pytest.mark.parametrize("precond", [1, 3])
def test_block_pcg_mixed_matches_oracle(precond):
    from paper_2511_09753_gb300 import spai
    mats = [I.varcoef_grid((10, 12), seed=11), I.aniso_2d_9pt(18), I.varcoef_grid((5, 6, 7), seed=12)]
    g = spai.SpaiBatch(mats, prec="mixed", cap_factor=2.0)
    g.run("lomr", 6)
    g.set_pcg_prec("mixed")
    rng = np.random.default_rng(5)
    B = [rng.uniform(-1.0, 1.0, size=(8, m[0])) for m in mats]
    out = g.pcg_block(B, rtol=1e-8, maxit=800, precond=precond)
    for m, (n, rp, ci, v) in enumerate(mats):
        o = O.Oracle(n, rp, ci, v, mixed=True, cap_factor=2.0)
        o.run("lomr", 6)
        for j in range(8):
            ro = O.pcg(n, rp, ci, v, B[m][j], rtol=1e-8, maxit=800, precond=precond,
                       M=o.get_M(), mixed=True)
            assert out["iters"][m, j] == ro["iters"], (m, j)
            assert out["statuses"][m, j] == STATUS[ro["status"]], (m, j)
            assert np.array_equal(out["x"][m][j], ro["x"]), (m, j)
            assert out["relres"][m, j] == ro["relres"], (m, j)


def test_mixed_pcg_close_to_fp64_pcg_on_the_gpu():
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(24, seed=3)
    s = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=3.0)
    s.run("lomr", 20)
    b = I.rhs_uniform(n, 0)
    f = s.pcg(b.copy(), rtol=1e-8, maxit=2000, precond=3)
    s.set_pcg_prec("mixed")
    m = s.pcg(b.copy(), rtol=1e-8, maxit=2000, precond=3)
    assert f["status"] == m["status"] == 0
    assert abs(m["iters"] - f["iters"]) <= max(1, 0.02 * f["iters"])
    assert m["relres"] < 1e-5
    assert np.linalg.norm(m["x"] - f["x"]) <= 1e-5 * np.linalg.norm(f["x"])
