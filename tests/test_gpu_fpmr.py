"""Differentiation of fixed-pattern MR on the GPU: loss and gradient against
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
