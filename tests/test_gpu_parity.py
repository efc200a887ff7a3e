"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The FP64 path and the mixed FP32-value path are compared with the oracle's
FP64 and exact mixed emulation, element by element: residual histories,
step coefficients and every entry of M must be identical (the arithmetic
order is fixed on both sides).  The mixed path is also held to the FP64
oracle within the stated tolerance (||I - A M||_F within 1e-5 relative).
"""
import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _spai():
    from paper_2511_09753_gb300 import spai
    return spai


CASES = {
    "lap2d_32": lambda: I.laplacian_2d_5pt(32),           # n = 1024
    "varcoef3d_16": lambda: I.varcoef_3d_7pt(16, seed=3),  # n = 4096
    "aniso9_45": lambda: I.aniso_2d_9pt(45),              # n = 2025 (ragged tail)
    "varcoef2d_37": lambda: I.varcoef_2d_5pt(37, seed=1), # n = 1369
}


def _same(g, o):
    return all(np.array_equal(a, b) for a, b in zip(g, o))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_method_parity(case, method, prec):
    spai = _spai()
    n, rp, ci, v = CASES[case]()
    capf = 3.0 if case.startswith("varcoef3d") else 2.0
    iters = 12
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=capf)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
    rg = g.run(method, iters)
    ro = o.run(method, iters)
    assert rg["done"] == ro["done"]
    np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
    np.testing.assert_array_equal(rg["coef"][:ro["done"]], ro["coef"][:ro["done"]])
    np.testing.assert_array_equal(rg["nnz"], ro["nnz"])  # nnz(M_i) history
    assert _same(g.get_M(), o.get_M())
    assert g.residual_norm() == o.residual_norm()


WIDE = {  # columns longer than 32 entries: the general diagonal-slot SpGEMM
    "varcoef3d_12_cap6": (lambda: I.varcoef_3d_7pt(12, seed=7), 6.0),  # 7 slots, cap 42
    "aniso9_30_cap4": (lambda: I.aniso_2d_9pt(30), 4.0),               # 9 slots, cap 36
}


@pytest.mark.parametrize("case", list(WIDE))
@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wide_columns_parity(case, method, prec):
    spai = _spai()
    make, capf = WIDE[case]
    n, rp, ci, v = make()
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=capf)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
    rg, ro = g.run(method, 10), o.run(method, 10)
    assert rg["done"] == ro["done"]
    np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
    np.testing.assert_array_equal(rg["coef"][:ro["done"]], ro["coef"][:ro["done"]])
    gm = g.get_M()
    assert _same(gm, o.get_M())
    assert np.diff(gm[0]).max() > 32  # the wide path was taken


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_mixed_within_tolerance_of_fp64_oracle(method):
    spai = _spai()
    n, rp, ci, v = I.varcoef_3d_7pt(16, seed=3)
    g = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=3.0)
    g.run(method, 10)
    o = O.Oracle(n, rp, ci, v, cap_factor=3.0)
    o.run(method, 10)
    a, b = g.residual_norm(), o.residual_norm()
    assert abs(a - b) <= 1e-5 * b, (a, b)


def test_laplacian32_mr_then_pcg_matches_oracle():
    """Plain MR, FP64, 32x32 Laplacian, 20 iterations, cap 2 nnz, then PCG to 1e-8."""
    spai = _spai()
    n, rp, ci, v = I.laplacian_2d_5pt(32)
    g = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
    o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    np.testing.assert_array_equal(g.mr(20)["resnorm"], o.run("mr", 20)["resnorm"])
    M = o.get_M()
    assert _same(g.get_M(), M)
    b = I.rhs_uniform(n, 0)
    for pre, opre in ((spai.PREC_SPAI_SYM, 3), (spai.PREC_JACOBI, 1), (spai.PREC_NONE, 0)):
        pg = g.pcg(b, rtol=1e-8, precond=pre)
        po = O.pcg(n, rp, ci, v, b, rtol=1e-8, precond=opre, M=M)
        assert pg["iters"] == po["iters"] and pg["status"] == po["status"] == 0
        np.testing.assert_array_equal(pg["x"], po["x"])
        assert pg["relres"] == po["relres"] and pg["relres"] < 1e-8
    # z = M r with the unsymmetrised M: same outcome as the oracle (capped run)
    pg = g.pcg(b, rtol=1e-8, maxit=300, precond=spai.PREC_SPAI)
    po = O.pcg(n, rp, ci, v, b, rtol=1e-8, maxit=300, precond=2, M=M)
    gpu_to_oracle = {spai.OK: 0, spai.PCG_MAXIT: 1, spai.PCG_BREAKDOWN: 2}
    assert (pg["iters"], gpu_to_oracle[pg["status"]]) == (po["iters"], po["status"])
    np.testing.assert_array_equal(pg["x"], po["x"])


def test_apply_matches_oracle_matrix():
    import torch
    spai = _spai()
    n, rp, ci, v = I.aniso_2d_9pt(20)
    g = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=4.0)
    g.lomr(6)
    cp, ri, va = g.get_M()
    x = torch.randn(3, n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    g.apply(x, y)
    M = np.zeros((n, n))
    for j in range(n):
        M[ri[cp[j]:cp[j + 1]], j] = va[cp[j]:cp[j + 1]]
    ref = (M @ x.cpu().numpy().T).T
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-14)


def test_continuation_and_checkpoint():
    spai = _spai()
    n, rp, ci, v = I.varcoef_2d_5pt(30, seed=4)
    for method in ("mr", "lomr", "cg"):
        a = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
        a.run(method, 6)
        state = a.save_state()
        a.run(method, 5)
        b = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
        b.run(method, 11)
        assert _same(a.get_M(), b.get_M())
        c = spai.Spai(n, rp, ci, v, prec="fp64", cap_factor=2.0)
        c.load_state(state)
        c.run(method, 5)
        assert _same(c.get_M(), b.get_M())


def test_diagonal_matrix_converges_immediately():
    spai = _spai()
    n, rp, ci, v = I.dense_to_csr(np.diag(np.arange(1.0, 41.0)))
    for method in ("mr", "lomr", "cg"):
        g = spai.Spai(n, rp, ci, v, cap_factor=2.0)
        r = g.run(method, 5)
        assert r["status"] == spai.CONVERGED_EARLY and r["done"] == 0
        assert r["resnorm"][0] == 0.0
        cp, ri, va = g.get_M()
        assert np.array_equal(va, 1.0 / np.arange(1.0, 41.0))


def test_tiny_sizes_and_no_drop():
    spai = _spai()
    for N in (1, 2, 3):
        n, rp, ci, v = I.laplacian_1d(N)
        g = spai.Spai(n, rp, ci, v, cap_factor=2.0)
        o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
        for m in ("mr", "lomr", "cg"):
            rg, ro = g.run(m, 4), o.run(m, 4)
            assert rg["done"] == ro["done"]
            np.testing.assert_array_equal(rg["resnorm"][:ro["done"] + 1], ro["resnorm"][:ro["done"] + 1])
            assert _same(g.get_M(), o.get_M())
    n, rp, ci, v = I.random_spd_banded(24, 2, 9)
    for m in ("mr", "lomr", "cg"):
        g = spai.Spai(n, rp, ci, v, cap_factor=1e9)
        o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
        rg, ro = g.run(m, 10, drop=False), o.run(m, 10, drop=O.DROP_NONE)
        np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
        assert _same(g.get_M(), o.get_M())


def test_capacity_overflow_is_reported():
    spai = _spai()
    n, rp, ci, v = I.laplacian_2d_5pt(12)
    g = spai.Spai(n, rp, ci, v, cap_factor=1.0)
    with pytest.raises(spai.SpaiError) as e:
        g.run("mr", 3, drop=False)
    assert e.value.code == spai.ERR_CAPACITY


def test_table2_spgemm_counts_on_gpu():
    spai = _spai()
    n, rp, ci, v = I.laplacian_2d_5pt(16)
    K = 5
    # column SpGEMMs per iteration: MR 2, LOMR 3, CG 2 (Table 2), plus the
    # final (MR, LOMR) or initial (CG) residual; CG's pass B reads the R that
    # the previous pass A computed
    for m, per, extra in (("mr", 2, 1), ("lomr", 3, 1), ("cg", 2, 1)):
        g = spai.Spai(n, rp, ci, v, cap_factor=2.0)
        s0 = g.stats()["spgemm_columns"]
        g.run(m, K)
        used = g.stats()["spgemm_columns"] - s0
        assert used == n * (per * K + extra), (m, used)


@pytest.mark.parametrize("method", ["mr", "lomr", "cg", "lomr_pi"])
def test_autotune_keeps_results_bitwise(method):
    """Any launch shape the autotuner picks gives the same iterates."""
    spai = _spai()
    n, rp, ci, v = I.varcoef_3d_7pt(16, seed=3)
    a = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=3.0)
    ra = a.run(method, 6)
    b = spai.Spai(n, rp, ci, v, prec="mixed", cap_factor=3.0)
    ms = b.autotune(method, 2)
    assert ms > 0
    rb = b.run(method, 6)
    np.testing.assert_array_equal(ra["resnorm"], rb["resnorm"])
    assert _same(a.get_M(), b.get_M())


@pytest.mark.parametrize("case", ["varcoef3d_16", "aniso9_45"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cg_without_the_r_slab_matches_oracle(case, prec, monkeypatch):
    """CG's pass B recomputing R (the path taken when the R slab cannot be
    allocated, forced here with SPAI_CG_NO_R_SLAB=1) gives the oracle's
    results bit for bit, over several calls that continue the recurrence."""
    spai = _spai()
    monkeypatch.setenv("SPAI_CG_NO_R_SLAB", "1")
    n, rp, ci, v = CASES[case]()
    capf = 3.0 if case.startswith("varcoef3d") else 2.0
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=capf)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
    for iters in (5, 4):
        rg = g.run("cg", iters)
        ro = o.run("cg", iters)
        assert rg["done"] == ro["done"] == iters
        np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
        np.testing.assert_array_equal(rg["coef"][:iters], ro["coef"][:iters])
        assert _same(g.get_M(), o.get_M())
    g.close()


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_steady_and_general_kernels_match_oracle(method, prec, monkeypatch):
    """Mid-run passes on an operator whose column products all take the short
    DIA form (7-point stencil, cap 21) run the kernels compiled for
    steady-state flags; with SPAI_GENERAL_KERNELS=1 the same passes run the
    general kernels.  Both give the oracle's results bit for bit, and the
    launch counts show which kernels ran (6 iterations: MR and LOMR have 5
    mid-run passes, CG 5 passes B reading R and 5 passes A storing it)."""
    spai = _spai()
    n, rp, ci, v = CASES["varcoef3d_16"]()
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=3.0)
    ro = o.run(method, 6)
    Mo = o.get_M()
    for general in (False, True):
        if general:
            monkeypatch.setenv("SPAI_GENERAL_KERNELS", "1")
        g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=3.0)
        rg = g.run(method, 6)
        assert rg["done"] == ro["done"] == 6
        np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
        np.testing.assert_array_equal(rg["coef"][:6], ro["coef"][:6])
        assert _same(g.get_M(), Mo)
        steady = g.stats()["colpass_steady_launches"]
        assert steady == (0 if general else (10 if method == "cg" else 5))
        g.close()


@pytest.mark.parametrize("case", ["lap2d_32", "varcoef3d_16", "aniso9_45"])
@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_keep_diag_parity(case, method, prec):
    """The drop that always keeps the column's diagonal (Appendix A's rule,
    SPAI_DROP_TOPK_COL_DIAG) against the oracle's, bit for bit, with a cap
    small enough that it decides (0.6 nnz(A[:,j])); every column of M keeps
    its diagonal.  Also the nnz(M_i) history over two continued calls."""
    spai = _spai()
    n, rp, ci, v = CASES[case]()
    capf = 0.6
    g = spai.Spai(n, rp, ci, v, prec=prec, cap_factor=capf)
    o = O.Oracle(n, rp, ci, v, mixed=(prec == "mixed"), cap_factor=capf)
    o.set_keep_diag(True)
    for iters in (6, 4):
        rg = g.run(method, iters, keep_diag=True)
        ro = o.run(method, iters)
        assert rg["done"] == ro["done"]
        np.testing.assert_array_equal(rg["resnorm"], ro["resnorm"])
        np.testing.assert_array_equal(rg["coef"][:ro["done"]], ro["coef"][:ro["done"]])
        np.testing.assert_array_equal(rg["nnz"], ro["nnz"])
        gm = g.get_M()
        assert _same(gm, o.get_M())
    cp, ri, _ = gm
    assert all(j in ri[cp[j]:cp[j + 1]] for j in range(n))
    g.close()
