"""Block PCG: every (matrix, right-hand side) recurrence of pcg_solve_block
must equal the oracle's one-vector PCG on that matrix and vector, with the
oracle's own SPAI as preconditioner: x bitwise, iteration count, stop reason
and true relative residual."""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATUS = {0: 0, 1: 3, 2: 4}  # oracle stop reason -> library status code


def _mats():
    return [I.varcoef_grid((10, 12), seed=11), I.varcoef_grid((5, 6, 7), seed=12),
            I.laplacian_2d_5pt(20), I.varcoef_grid((33, 11), seed=14),
            I.varcoef_grid((4, 5, 9), seed=13)]


def _rhs(mats, R, seed):
    rng = np.random.default_rng(seed)
    B = [rng.uniform(-1.0, 1.0, size=(R, m[0])) for m in mats]
    B[0][1] = 0.0  # a zero right-hand side stops at once with x = 0
    return B


def _oracle_check(mats, B, out, prec, precond, method, iters, capf, rtol, maxit):
    for m, (n, rp, ci, v) in enumerate(mats):
        Mo = None
        if precond in (2, 3):
            o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
            o.run(method, iters)
            Mo = o.get_M()
        for j in range(B[m].shape[0]):
            ro = O.pcg(n, rp, ci, v, B[m][j], rtol=rtol, maxit=maxit, precond=precond, M=Mo)
            assert out["iters"][m, j] == ro["iters"], (m, j)
            assert out["statuses"][m, j] == STATUS[ro["status"]], (m, j)
            assert np.array_equal(out["x"][m][j], ro["x"]), (m, j)
            assert out["relres"][m, j] == ro["relres"], (m, j)


@pytest.mark.parametrize("precond", [0, 1, 2, 3])
def test_block_pcg_batched_matches_oracle(precond):
    from paper_2511_09753_gb300 import spai
    mats = _mats()
    g = spai.SpaiBatch(mats, prec="mixed", cap_factor=3.0)
    g.run("lomr", 10)
    B = _rhs(mats, 32, seed=7)
    out = g.pcg_block(B, rtol=1e-8, maxit=500, precond=precond)
    if precond != 2:  # PCG with the nonsymmetric M itself may stall (Sec. 7)
        assert out["status"] == 0
    _oracle_check(mats, B, out, "mixed", precond, "lomr", 10, 3.0, 1e-8, 500)


def test_block_pcg_few_rhs_and_iteration_limit():
    from paper_2511_09753_gb300 import spai
    mats = _mats()[:3]
    g = spai.SpaiBatch(mats, prec="fp64", cap_factor=2.0)
    g.run("mr", 5)
    B = _rhs(mats, 5, seed=8)
    out = g.pcg_block(B, rtol=1e-10, maxit=7, precond=3)
    assert out["status"] == 3  # some recurrence hit the limit
    _oracle_check(mats, B, out, "fp64", 3, "mr", 5, 2.0, 1e-10, 7)


def test_block_pcg_single_handle_equals_vector_pcg():
    from paper_2511_09753_gb300 import spai
    n, rp, ci, v = I.varcoef_grid((40, 30), seed=5)  # 1200 rows: a ragged last CTA
    s = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=2.0)
    s.run("cg", 6)
    rng = np.random.default_rng(3)
    B = rng.uniform(-1.0, 1.0, size=(3, n))
    out = s.pcg_block([B], rtol=1e-8, maxit=1000, precond=3)
    for j in range(3):
        r1 = s.pcg(B[j].copy(), rtol=1e-8, maxit=1000, precond=3)
        assert out["iters"][0, j] == r1["iters"]
        assert np.array_equal(out["x"][0][j], r1["x"])
        assert out["relres"][0, j] == r1["relres"]


def test_block_pcg_device_buffers_equal_host_buffers():
    torch = pytest.importorskip("torch")
    from paper_2511_09753_gb300 import spai
    mats = _mats()[:2]
    g = spai.SpaiBatch(mats, prec="mixed", cap_factor=2.0)
    g.run("lomr", 4)
    B = _rhs(mats, 4, seed=9)
    host = g.pcg_block(B, precond=2)
    flat = torch.tensor(np.concatenate([b.ravel() for b in B]), dtype=torch.float64,
                        device="cuda")
    dev = g.pcg_block(flat, precond=2, nrhs=4)
    xs = np.concatenate([x.ravel() for x in host["x"]])
    assert np.array_equal(dev["x"].cpu().numpy(), xs)
    assert np.array_equal(dev["iters"], host["iters"])
    # a second solve on the same handle reuses the captured graph
    again = g.pcg_block(B, precond=2)
    assert np.array_equal(again["iters"], host["iters"])
    for a, b in zip(again["x"], host["x"]):
        assert np.array_equal(a, b)
