"""Differentiation of fixed-pattern MR and LOMR on the GPU: loss and gradient against
the oracle's hand-written adjoint, against central differences of the GPU
forward itself (h = 1e-6 on 50 entries, the 32^3 configuration), and
through torch.autograd."""
import numpy as np
import pytest

from oracle import fpmr as OF
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [0, 1, 3, 10])
def test_fpmr_matches_oracle(K):
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(8, seed=5)
    f = spai.FixedPatternMR(n, rp, ci, K)
    loss = f.forward(v)
    g = f.backward()
    lo, go = OF.gradient(n, rp, ci, v, K)
    assert abs(loss - lo) <= 1e-12 * lo
    np.testing.assert_allclose(g, go, rtol=1e-9, atol=1e-12 * np.abs(go).max())
    f.close()


def test_fpmr_central_differences_32cubed():
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(32, seed=0)
    K = 10
    f = spai.FixedPatternMR(n, rp, ci, K)
    L = f.forward(v)
    g = f.backward()
    rng = np.random.default_rng(0)
    scale = np.abs(g).max()
    eps = np.finfo(float).eps
    for e in rng.choice(len(v), 50, replace=False):
        h = 1e-6 * abs(v[e])
        vp, vm = v.copy(), v.copy()
        vp[e] += h
        vm[e] -= h
        fd = (f.forward(vp) - f.forward(vm)) / (2 * h)
        # truncation O(h^2) plus the rounding of L (a sum of ~1e6 terms)
        # amplified by 1/h
        tol = 1e-6 * scale + 100 * eps * L / h
        assert abs(fd - g[e]) <= tol, (e, fd, g[e], tol)
    f.close()


def test_fpmr_through_torch_autograd():
    torch = pytest.importorskip("torch")
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_2d_5pt(20, seed=3)
    f = spai.FixedPatternMR(n, rp, ci, 5)
    x = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = spai.fpmr_loss(x, f)
    (3.0 * loss).backward()
    ref = f.backward(3.0)
    np.testing.assert_array_equal(x.grad.cpu().numpy(), ref)
    lo, go = OF.gradient(n, rp, ci, v, 5)
    np.testing.assert_allclose(x.grad.cpu().numpy(), 3.0 * go, rtol=1e-9, atol=1e-12 * np.abs(go).max())
    f.close()


def test_fpmr_mixed_tracks_fp64():
    """FP32 values and products with FP64 inner products and scalars: loss
    and gradient within FP32 accuracy of the FP64 oracle."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(12, seed=6)
    f = spai.FixedPatternMR(n, rp, ci, 10, prec="mixed")
    loss = f.forward(v)
    g = f.backward()
    lo, go = OF.gradient(n, rp, ci, v, 10)
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.max(np.abs(g - go)) <= 1e-4 * np.abs(go).max()
    assert not np.array_equal(g, go)
    f.close()


# ---------------------------------------------- fixed-pattern LOMR steps

@pytest.mark.parametrize("K", [0, 1, 3, 10])
def test_fplomr_matches_oracle(K):
    """K fixed-pattern LOMR steps (Algorithm 4 / Theorem 3 on supp(A)): loss
    and gradient against the oracle's hand-written adjoint at 8^3."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(8, seed=5)
    f = spai.FixedPatternMR(n, rp, ci, K, method="lomr")
    loss = f.forward(v)
    g = f.backward()
    lo, go = OF.gradient_lomr(n, rp, ci, v, K)
    assert abs(loss - lo) <= 1e-12 * lo
    np.testing.assert_allclose(g, go, rtol=1e-9, atol=1e-11 * np.abs(go).max())
    f.close()


def test_fplomr_central_differences_32cubed():
    """The 32^3 configuration with 10 LOMR steps: central differences of the
    GPU forward (h = 1e-6 relative) on 50 entries."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(32, seed=0)
    K = 10
    f = spai.FixedPatternMR(n, rp, ci, K, method="lomr")
    L = f.forward(v)
    g = f.backward()
    rng = np.random.default_rng(1)
    scale = np.abs(g).max()
    eps = np.finfo(float).eps
    for e in rng.choice(len(v), 50, replace=False):
        h = 1e-6 * abs(v[e])
        vp, vm = v.copy(), v.copy()
        vp[e] += h
        vm[e] -= h
        fd = (f.forward(vp) - f.forward(vm)) / (2 * h)
        tol = 1e-6 * scale + 100 * eps * L / h
        assert abs(fd - g[e]) <= tol, (e, fd, g[e], tol)
    f.close()


def test_fplomr_method_switch_and_mixed():
    """The method can be switched on one handle (MR, LOMR, MR again give the
    oracle's gradients); the mixed LOMR gradient tracks the FP64 oracle."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_3d_7pt(10, seed=7)
    f = spai.FixedPatternMR(n, rp, ci, 6)
    for method in ("mr", "lomr", "mr"):
        assert f.lib.spai_fpmr_set_method(f.h, spai.METHODS[method]) == 0
        loss = f.forward(v)
        g = f.backward()
        lo, go = (OF.gradient if method == "mr" else OF.gradient_lomr)(n, rp, ci, v, 6)
        assert abs(loss - lo) <= 1e-12 * lo
        np.testing.assert_allclose(g, go, rtol=1e-9, atol=1e-11 * np.abs(go).max())
    assert f.lib.spai_fpmr_set_method(f.h, spai.METHODS["cg"]) == -1
    f.close()
    fm = spai.FixedPatternMR(n, rp, ci, 6, prec="mixed", method="lomr")
    loss = fm.forward(v)
    g = fm.backward()
    lo, go = OF.gradient_lomr(n, rp, ci, v, 6)
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.max(np.abs(g - go)) <= 1e-4 * np.abs(go).max()
    fm.close()


# ------------------------------------------------ device set-up

@pytest.mark.parametrize("make", [lambda: I.varcoef_3d_7pt(12, seed=2),
                                  lambda: I.aniso_2d_9pt(40),
                                  lambda: I.random_spd_banded(60, 4, seed=3)],
                         ids=["varcoef3d_12", "aniso9_40", "random_spd_60"])
@pytest.mark.parametrize("method", ["mr", "lomr"])
def test_device_setup_equals_host_setup(make, method, monkeypatch):
    """The patterns and product lists built on the GPU equal the host
    construction's (SPAI_FPMR_HOST_SETUP=1 forces that one): the same list
    lengths, and the same loss and gradient bit for bit."""
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = make()
    out = []
    for host in ("0", "1"):
        monkeypatch.setenv("SPAI_FPMR_HOST_SETUP", host)
        f = spai.FixedPatternMR(n, rp, ci, 4, method=method)
        loss = f.forward(v)
        out.append((f.info()["nnz_t"], f.info()["list_entries"], loss, f.backward().copy()))
        f.close()
    (t0, l0, a0, g0), (t1, l1, a1, g1) = out
    assert t0 == t1 and l0 == l1 and a0 == a1
    assert np.array_equal(g0, g1)


def test_device_setup_rejects_bad_patterns():
    """The GPU validation returns the host's codes: an unsorted row (CSR),
    a missing diagonal (NOT_SPD_DIAG), a missing mirror (NOT_SYMMETRIC)."""
    import ctypes as C
    from paper_2511_09753_gb300 import spai
    lib = spai.load()
    n, rp, ci, v = I.laplacian_2d_5pt(6)
    rp = np.array(rp, dtype=np.int32)

    def create(ci2):
        h = C.c_void_p()
        ci2 = np.ascontiguousarray(ci2, dtype=np.int32)
        rc = lib.spai_fpmr_create(C.byref(h), n, len(ci2), rp.ctypes.data, ci2.ctypes.data, 2,
                                  spai.SPAI_FP64, None)
        if rc == 0:
            lib.spai_fpmr_destroy(h)
        return rc

    assert create(ci) == 0
    bad = np.array(ci)
    bad[rp[7]], bad[rp[7] + 1] = bad[rp[7] + 1], bad[rp[7]]  # row 7 out of order
    assert create(bad) == -2
    nodiag = np.array(ci)
    e = rp[9] + list(ci[rp[9]:rp[10]]).index(9)
    nodiag[e] = 9 + 2 if 9 + 2 not in ci[rp[9]:rp[10]] else 9 - 2  # diagonal of row 9 moved away
    row = sorted(nodiag[rp[9]:rp[10]])
    nodiag[rp[9]:rp[10]] = row
    assert create(nodiag) in (-3,)
    asym = np.array(ci)
    e = rp[20] + 0  # first entry of row 20 points elsewhere (its mirror is missing)
    cand = [c for c in range(n) if c not in ci[rp[20]:rp[21]] and c < ci[rp[20] + 1]]
    asym[e] = cand[-1]
    asym[rp[20]:rp[21]] = sorted(asym[rp[20]:rp[21]])
    assert create(asym) == -4
