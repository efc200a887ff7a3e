"""Parity of the Pi-preconditioned forms (Section 5: MR_SPD Algorithm 5,
LOMR_SPD Algorithm 8, CG Algorithm 7, with Pi = diag(A)^{-1}) with the CPU
oracle: histories, coefficients, every entry of M and the FP64 residual,
bit for bit, for single and batched handles."""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "lap2d_32": lambda: I.laplacian_2d_5pt(32),           # constant diagonal
    "varcoef3d_16": lambda: I.varcoef_3d_7pt(16, seed=3),  # n = 4096
    "aniso9_45": lambda: I.aniso_2d_9pt(45),              # 9 diagonals, ragged tail
    "banded_60": lambda: I.random_spd_banded(60, 20, 7),  # > 32 diagonals: row-list SpGEMM
}


def _same(g, o):
    return all(np.array_equal(a, b) for a, b in zip(g, o))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("method", ["mr_pi", "lomr_pi", "cg_pi"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pi_method_parity(case, method, prec):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = CASES[case]()
    capf = 3.0 if case.startswith("varcoef3d") else (1.0 if case.startswith("banded") else 2.0)
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=capf)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
    rg = g.run(method, 10)
    ro = o.run(method, 10)
    assert rg["done"] == ro["done"]
    np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
    np.testing.assert_array_equal(rg["coef"][:ro["done"]], ro["coef"][:ro["done"]])
    assert _same(g.get_M(), o.get_M())
    assert g.residual_norm() == o.residual_norm()


@pytest.mark.parametrize("method", ["mr_pi", "lomr_pi", "cg_pi"])
def test_pi_continuation_equals_one_call(method):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_2d_5pt(30, seed=2)
    a = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=2.0)
    b = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=2.0)
    a.run(method, 7)
    b.run(method, 3)
    b.run(method, 4)
    assert _same(a.get_M(), b.get_M())
    assert a.residual_norm() == b.residual_norm()


@pytest.mark.parametrize("method", ["mr_pi", "lomr_pi", "cg_pi"])
def test_pi_batched_matches_single_oracle_runs(method):
    from paper_2511_09753_gb300 import spai
    mats = [I.varcoef_grid((10, 12), seed=11), I.varcoef_grid((5, 6, 7), seed=12),
            I.laplacian_2d_5pt(20), I.varcoef_grid((33, 11), seed=14)]
    g = spai.SpaiBatch(mats, prec="mixed", cap_factor=2.5)
    r = g.run(method, 8)
    res = g.residual_norms()
    for m, (n, rp, ci, v) in enumerate(mats):
        o = O.Oracle(n, rp, ci, v, mixed=True, cap_factor=2.5)
        ro = o.run(method, 8)
        assert r["done_each"][m] == ro["done"]
        np.testing.assert_array_equal(r["resnorm_each"][m][:ro["done"] + 1],
                                      ro["resnorm"][:ro["done"] + 1])
        assert _same(g.get_M_of(m), o.get_M())
        assert res[m] == o.residual_norm()


def test_pi_forms_equal_plain_forms_on_the_laplacian_gpu():
    """diag(A) = 4I: the Pi forms are the plain forms exactly (on the GPU too)."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.laplacian_2d_5pt(40)
    for m in ("mr", "lomr", "cg"):
        a = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=2.0)
        b = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=2.0)
        ra, rb = a.run(m, 9), b.run(m + "_pi", 9)
        np.testing.assert_array_equal(ra["resnorm"], rb["resnorm"])
        assert _same(a.get_M(), b.get_M())
