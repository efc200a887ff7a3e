"""Definiteness diagnostics on the GPU: Lanczos on the symmetric part of M
against the oracle's Lanczos (coefficients bit for bit, extremal Ritz values
against scipy's tridiagonal eigensolver)."""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("method", ["mr", "lomr"])
def test_lanczos_matches_oracle(prec, method):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((23, 29), seed=6)      # 667 rows: ragged CTAs
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=2.0)
    g.run(method, 8)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=2.0)
    o.run(method, 8)
    v0 = np.random.default_rng(1).standard_normal(n)
    r = g.sym_spectrum(steps=60, v0=v0)
    ro = O.lanczos(n, o.get_M(), v0, 60)
    assert r["steps"] == ro["steps"] == 60
    np.testing.assert_array_equal(r["alpha"], ro["alpha"])
    np.testing.assert_array_equal(r["beta"], ro["beta"])
    scale = max(abs(ro["lmin"]), abs(ro["lmax"]))
    assert abs(r["lmin"] - ro["lmin"]) <= 1e-13 * scale
    assert abs(r["lmax"] - ro["lmax"]) <= 1e-13 * scale


def test_lanczos_sees_an_indefinite_symmetric_part():
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.laplacian_2d_5pt(10)
    g = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
    d = np.linspace(-0.5, 2.0, n)
    cp = np.arange(n + 1, dtype=np.int32)
    ri = np.arange(n, dtype=np.int32)
    g.set_M(cp, ri, d)
    r = g.sym_spectrum(steps=n, v0=np.ones(n))
    assert abs(r["lmin"] + 0.5) < 1e-12 and abs(r["lmax"] - 2.0) < 1e-12
    with pytest.raises(spai.SpaiError):
        g.sym_spectrum(steps=5, v0=np.zeros(n))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_fixed_pattern_spai_matches_oracle(prec, k):
    from paper_2511_09753_gb300 import spai
    for n, rp, ci, v in (I.varcoef_grid((13, 17), seed=8), I.varcoef_grid((5, 6, 7), seed=9)):
        g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=10.0)
        g.fixed_pattern(k)
        cp, ri, va = g.get_M()
        ocp, ori, ova = O.fixed_pattern_spai(n, rp, ci, v, k)
        assert np.array_equal(cp, ocp) and np.array_equal(ri, ori)
        tol = 1e-10 if prec == "fp64" else 2e-7
        np.testing.assert_allclose(va, ova, rtol=tol, atol=tol * np.abs(ova).max())
        # the FP64 residual of the stored M agrees with the oracle's M
        res = float(np.linalg.norm(np.eye(n) - I.csr_to_dense(n, rp, ci, v) @ _dense(n, ocp, ori, va)))
        assert abs(g.residual_norm() - res) <= 1e-9 * res


def _dense(n, cp, ri, va):
    M = np.zeros((n, n))
    for j in range(n):
        M[ri[cp[j]:cp[j + 1]], j] = va[cp[j]:cp[j + 1]]
    return M


def test_fixed_pattern_then_lanczos_extremes():
    """Exp. 09's question, answered by the GPU diagnostics: the extremal
    eigenvalues of the symmetric part of the best SPAI on supp(A^k) agree
    with dense eigenvalues of the oracle's M."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.aniso_2d_9pt(20)
    for k in (1, 2, 3):
        g = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=8.0)
        g.fixed_pattern(k)
        r = g.sym_spectrum(steps=n, v0=np.random.default_rng(k).standard_normal(n))
        M = _dense(n, *O.fixed_pattern_spai(n, rp, ci, v, k))
        ev = np.linalg.eigvalsh(0.5 * (M + M.T))
        scale = np.abs(ev).max()
        assert abs(r["lmin"] - ev[0]) <= 1e-8 * scale
        assert abs(r["lmax"] - ev[-1]) <= 1e-8 * scale
