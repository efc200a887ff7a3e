"""The OpenMP build of the oracle (columns and PCG rows shared among
threads) gives the serial build's results bit for bit: each column is
computed by one thread with the serial arithmetic and every sum over
columns or rows is the same pairwise tree, taken after its loop.  No GPU."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I


@pytest.fixture(autouse=True)
def _threads(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("method", ["mr", "lomr", "cg", "mr_pi", "lomr_pi", "cg_pi"])
@pytest.mark.parametrize("mixed", [False, True])
def test_openmp_oracle_equals_serial(method, mixed):
    n, rp, ci, v = I.varcoef_3d_7pt(12, seed=3)
    runs = []
    for omp in (False, True):
        o = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=2.0, omp=omp)
        r1 = o.run(method, 4)
        r2 = o.run(method, 3)  # continuation
        runs.append((r1, r2, o.get(0), o.get(1), o.get(2), o.residual_norm(), o.spgemm_count()))
    (a1, a2, *ra), (b1, b2, *rb) = runs
    for x, y in ((a1, b1), (a2, b2)):
        assert x["done"] == y["done"] and x["flags"] == y["flags"]
        assert np.array_equal(x["resnorm"], y["resnorm"], equal_nan=True)
        assert np.array_equal(x["coef"], y["coef"], equal_nan=True)
    for x, y in zip(ra[:3], rb[:3]):
        _same(x, y)
    assert ra[3] == rb[3] and ra[4] == rb[4]


@pytest.mark.parametrize("mixed", [False, True])
def test_openmp_pcg_equals_serial(mixed):
    n, rp, ci, v = I.varcoef_3d_7pt(14, seed=2)
    o = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=2.0)
    o.run("lomr", 5)
    M = o.get_M()
    b = I.rhs_uniform(n, 0)
    for precond in (0, 1, 3):
        a = O.pcg(n, rp, ci, v, b, precond=precond, M=M, mixed=mixed)
        c = O.pcg(n, rp, ci, v, b, precond=precond, M=M, mixed=mixed, omp=True)
        assert a["iters"] == c["iters"] and a["status"] == c["status"]
        assert a["relres"] == c["relres"] and np.array_equal(a["x"], c["x"])
