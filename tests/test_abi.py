"""The C-ABI library loads, exports every symbol of include/spai.h, and its
host-only entry points (CSR validation, status strings) behave; no GPU."""
import os
import re

import numpy as np
import pytest

from paper_2511_09753_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spai.h")


def _lib():
    from paper_2511_09753_gb300 import build, spai
    if not os.path.exists(spai.LIB_PATH):
        build.build()
    return spai


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_library_exports_every_declared_function():
    spai = _lib()
    import ctypes
    lib = ctypes.CDLL(spai.LIB_PATH)
    decl = header_functions()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(decl) == sorted(spai.EXPORTED)


def test_status_strings():
    spai = _lib()
    for code in (0, 1, 2, 3, 4, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10):
        s = spai.status_string(code)
        assert s and s != "unknown status"
    assert spai.status_string(12345) == "unknown status"


def test_validate_csr_accepts_generators():
    spai = _lib()
    for f, a in ((I.laplacian_2d_5pt, (8,)), (I.varcoef_3d_7pt, (5,)), (I.aniso_2d_9pt, (7,))):
        n, rp, ci, v = f(*a)
        assert spai.validate_csr(n, rp, ci, v) == 0


def test_validate_csr_symmetry_is_a_equals_a_transpose():
    """The symmetry check agrees with A == A^T (scipy) on random perturbations
    of values and of the pattern (an entry moved to another column)."""
    sp = pytest.importorskip("scipy.sparse")
    spai = _lib()
    rng = np.random.default_rng(5)
    n, rp, ci, v = I.varcoef_grid((9, 7), seed=3)
    for t in range(200):
        ci2, v2 = ci.copy(), v.copy()
        e = int(rng.integers(len(v)))
        i = int(np.searchsorted(rp, e, side="right") - 1)
        if t % 3 == 0:
            v2[e] = v2[e] * (1.0 + 1e-12)
        elif t % 3 == 1:  # move an off-diagonal entry to a free column of its row
            free = sorted(set(range(n)) - set(ci[rp[i]:rp[i + 1]].tolist()))
            if ci[e] == i or not free:
                continue
            row = sorted(set(ci[rp[i]:rp[i + 1]].tolist()) - {int(ci[e])} | {free[t % len(free)]})
            ci2[rp[i]:rp[i + 1]] = row
            v2[rp[i]:rp[i + 1]] = [v[rp[i] + ci[rp[i]:rp[i + 1]].tolist().index(c)]
                                   if c in ci[rp[i]:rp[i + 1]] else v[e] for c in row]
        A = sp.csr_matrix((v2, ci2, rp), shape=(n, n))
        sym = (A != A.T).nnz == 0
        code = spai.validate_csr(n, rp, ci2, v2)
        assert code == (0 if sym else -4), (t, code, sym)


def test_validate_csr_rejects_bad_input():
    spai = _lib()
    n, rp, ci, v = I.laplacian_2d_5pt(4)
    bad = v.copy(); bad[0] = np.nan
    assert spai.validate_csr(n, rp, ci, bad) == -5            # non-finite
    nd = v.copy(); nd[rp[3]:rp[4]][ci[rp[3]:rp[4]] == 3] = -1.0
    assert spai.validate_csr(n, rp, ci, nd) == -3             # non-positive diagonal
    asym = v.copy(); asym[1] = -0.5
    assert spai.validate_csr(n, rp, ci, asym) == -4           # not symmetric
    assert spai.validate_csr(n, rp, ci, asym, check_symmetry=False) == 0
    unsorted = ci.copy(); unsorted[0], unsorted[1] = unsorted[1], unsorted[0]
    assert spai.validate_csr(n, rp, unsorted, v) == -2        # unsorted row
    oob = ci.copy(); oob[-1] = n
    assert spai.validate_csr(n, rp, oob, v) == -2             # column out of range
    rp2 = rp.copy(); rp2[-1] += 1
    assert spai.validate_csr(n, rp2, ci, v) == -2             # rowptr[n] != nnz


def test_handle_calls_reject_null():
    spai = _lib()
    import ctypes
    lib = spai.load()
    assert lib.spai_destroy(None) == -1
    assert lib.spai_run(None, 0, 1, 1, None) == -1
    out = ctypes.c_void_p()
    opts = spai._Opts(0, 2.0)
    assert lib.spai_create(ctypes.byref(out), 0, 1, None, None, None, 0, ctypes.byref(opts), None) == -1


def test_create_batched_rejects_bad_input_before_any_device_call():
    spai = _lib()
    good = I.laplacian_2d_5pt(8)
    with pytest.raises(spai.SpaiError) as e:
        spai.SpaiBatch([], prec="fp64")
    assert e.value.code == -1
    n, rp, ci, v = I.laplacian_2d_5pt(8)
    v = v.copy()
    v[1] += 0.5  # breaks symmetry of one off-diagonal pair
    with pytest.raises(spai.SpaiError) as e:
        spai.SpaiBatch([good, (n, rp, ci, v)], prec="fp64")
    assert e.value.code == -4
    with pytest.raises(spai.SpaiError) as e:
        spai.SpaiBatch([good], prec="fp64", cap_factor=0.0)
    assert e.value.code == -1


def test_validate_csr_large_matrix_reports_the_first_failing_row():
    """A matrix large enough for the row ranges to be checked on several host
    threads (64^3, 1.8 M entries): of several faults, the one in the
    smallest row decides the code, as a scan in row order would; a row
    pointer that runs backwards or past nnz is a CSR error at its row."""
    spai = _lib()
    n, rp, ci, v = I.varcoef_3d_7pt(64)
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci, np.int32)
    v = np.ascontiguousarray(v, np.float64)
    assert spai.validate_csr(n, rp, ci, v) == 0
    a = v.copy(); a[1000] = np.nan
    b = ci.copy(); b[1_500_000] = -5
    assert spai.validate_csr(n, rp, b, a) == -5               # non-finite first
    a = v.copy(); a[1_700_000] = np.inf
    b = ci.copy(); b[100] = n + 3
    assert spai.validate_csr(n, rp, b, a) == -2               # column out of range first
    for e in (4, 900_001, len(v) - 2):                        # off-diagonal entries
        assert ci[e] != np.searchsorted(rp, e, side="right") - 1
        a = v.copy(); a[e] *= 1.0000001
        assert spai.validate_csr(n, rp, ci, a) == -4
        assert spai.validate_csr(n, rp, ci, a, check_symmetry=False) == 0
    r = rp.copy(); r[200_000] = r[200_001] + 3                # backwards at row 199,999
    a = v.copy(); a[10] = np.nan
    assert spai.validate_csr(n, r, ci, a) == -5
    assert spai.validate_csr(n, r, ci, v) == -2
    d = v.copy()
    last = n - 1
    d[rp[last]:rp[last + 1]][ci[rp[last]:rp[last + 1]] == last] = 0.0
    assert spai.validate_csr(n, rp, ci, d) == -3              # diagonal of the last row
