"""Batched SPAIs: many matrices of uneven size in one handle.

Every matrix of a batched handle must produce exactly what a single-matrix
run of the oracle produces (M, residual history, FP64 residual norm), even
when one matrix of the batch converges at step 0 and stops early.
"""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mats():
    mats = [I.varcoef_grid((10, 12), seed=11), I.varcoef_grid((5, 6, 7), seed=12),
            I.laplacian_2d_5pt(20), I.varcoef_grid((4, 5, 9), seed=13),
            I.dense_to_csr(np.diag(np.arange(1.0, 31.0))), I.varcoef_grid((33, 11), seed=14),
            I.varcoef_grid((6, 6, 6), seed=15)]
    return mats


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_matches_single_oracle_runs(method, prec):
    from paper_2511_09753_gb300 import spai
    mats = _mats()
    capf = 2.5
    iters = 8
    g = spai.SpaiBatch(mats, prec=prec, cap_factor=capf)
    r = g.run(method, iters)
    res = g.residual_norms()
    for m, (n, rp, ci, v) in enumerate(mats):
        o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
        ro = o.run(method, iters)
        assert r["done_each"][m] == ro["done"], (m, r["done_each"][m], ro["done"])
        k = ro["done"] + 1
        np.testing.assert_array_equal(r["resnorm_each"][m][:k], ro["resnorm"][:k])
        for a, b in zip(g.get_M_of(m), o.get_M()):
            assert np.array_equal(a, b), m
        assert res[m] == o.residual_norm()


def _check_against_oracle(g, r, mats, method, iters, prec, capf, res=None):
    for m, (n, rp, ci, v) in enumerate(mats):
        o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
        ro = o.run(method, iters)
        assert r["done_each"][m] == ro["done"], (m, r["done_each"][m], ro["done"])
        k = ro["done"] + 1
        np.testing.assert_array_equal(r["resnorm_each"][m][:k], ro["resnorm"][:k])
        for a, b in zip(g.get_M_of(m), o.get_M()):
            assert np.array_equal(a, b), m
        if res is not None:
            assert res[m] == o.residual_norm()


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_batched_general_sparsity_path(method):
    """Matrices with more than 32 distinct diagonals take the row-list SpGEMM."""
    from paper_2511_09753_gb300 import spai
    mats = [I.random_spd_banded(60, 20, 7), I.varcoef_grid((9, 13), seed=21),
            I.random_spd_banded(300, 17, 8)]
    g = spai.SpaiBatch(mats, prec="fp64", cap_factor=1.0)
    r = g.run(method, 6)
    _check_against_oracle(g, r, mats, method, 6, "fp64", 1.0, g.residual_norms())


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_batched_continuation_equals_one_call(method):
    from paper_2511_09753_gb300 import spai
    mats = [I.varcoef_grid((10, 12), seed=11), I.varcoef_grid((5, 6, 7), seed=12),
            I.laplacian_2d_5pt(20)]
    g1 = spai.SpaiBatch(mats, prec="mixed", cap_factor=3.0)
    g1.run(method, 8)
    g2 = spai.SpaiBatch(mats, prec="mixed", cap_factor=3.0)
    g2.run(method, 3)
    g2.run(method, 5)
    for m in range(len(mats)):
        for a, b in zip(g1.get_M_of(m), g2.get_M_of(m)):
            assert np.array_equal(a, b), m
    assert np.array_equal(g1.residual_norms(), g2.residual_norms())


def test_batched_single_matrix_equals_single_handle():
    from paper_2511_09753_gb300 import spai
    a = I.varcoef_grid((17, 19), seed=3)
    g = spai.SpaiBatch([a], prec="mixed", cap_factor=2.0)
    s = spai.Spai(*a, prec="mixed", cap_factor=2.0)
    rg = g.run("lomr", 7)
    rs = s.run("lomr", 7)
    np.testing.assert_array_equal(rg["resnorm_each"][0], rs["resnorm"])
    for x, y in zip(g.get_M_of(0), s.get_M()):
        assert np.array_equal(x, y)
    assert g.residual_norms()[0] == s.residual_norm()
    assert g.batch_info() == [a[0]]
