"""Seeded generators: sizes from the stencils, exact symmetry, definiteness."""
import numpy as np
import scipy.sparse as sp

from paper_2511_09753_gb300 import inputs as I


def _check(n, rp, ci, v):
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    assert (A != A.T).nnz == 0                       # exactly symmetric
    for i in range(0, n, max(1, n // 257)):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)  # rows column-sorted
    assert np.all(A.diagonal() > 0)
    return A


def test_nnz_match_stencil_formulas():
    n, rp, ci, v = I.laplacian_2d_5pt(32)
    assert (n, len(v)) == (1024, 4992)
    n, rp, ci, v = I.varcoef_3d_7pt(64)
    assert (n, len(v)) == (262144, 1810432)
    _check(n, rp, ci, v)
    n, rp, ci, v = I.aniso_2d_9pt(32)
    assert len(v) == 9 * 32 * 32 - 12 * 32 + 4


def test_small_operators_are_spd_and_deterministic():
    for f, args in ((I.laplacian_2d_5pt, (9,)), (I.varcoef_3d_7pt, (7,)),
                    (I.varcoef_2d_5pt, (11,)), (I.aniso_2d_9pt, (10,))):
        n, rp, ci, v = f(*args)
        A = _check(n, rp, ci, v).toarray()
        assert np.linalg.eigvalsh(A)[0] > 0
        n2, rp2, ci2, v2 = f(*args)
        assert np.array_equal(v, v2) and np.array_equal(ci, ci2)


def test_gaussian_field_statistics():
    g = I.gaussian_field((40, 40, 40), 1.5, 8.0, 0)
    assert abs(g.std() - 1.5) < 1e-12 and abs(g.mean()) < 1e-12
    # neighbouring nodes strongly correlated (correlation length 8 cells)
    c = np.corrcoef(g[:, :, :-1].ravel(), g[:, :, 1:].ravel())[0, 1]
    assert c > 0.95


def test_rhs_seed():
    assert np.array_equal(I.rhs_uniform(10, 0), np.random.default_rng(0).uniform(-1, 1, 10))


def test_batch_uneven_generator_shapes():
    mats = I.batch_uneven(count=64)
    ns = np.array([m[0] for m in mats])
    assert ns.min() >= 900 and ns.max() <= 70000
    assert abs(ns.sum() - 953176) < 1  # seeded: fixed
    # every matrix passes the library's host validation (SPD structure)
    for n, rp, ci, v in mats[:4]:
        assert np.all(np.diff(rp) >= 1)
