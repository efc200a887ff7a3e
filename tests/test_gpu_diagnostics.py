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
