"""The Python binding of the allocation-free entry point checks every
argument before the C call: the C entry point trusts its device pointers,
so a host tensor, a wrong dtype or a short array must raise here instead of
reaching the GPU.  No GPU: stand-in tensors carry the attributes checked,
and the library is never loaded."""
import types

import pytest
import torch

from paper_2511_09753_gb300 import spai


class FakeCuda:
    def __init__(self, numel, dtype, cuda=True, contiguous=True, index=None):
        self.is_cuda = cuda
        self.device = types.SimpleNamespace(index=index)
        self.dtype = dtype
        self._n = numel
        self._c = contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("no pointer may be taken before the checks pass")


def _good(n=10, nnz=28):
    return dict(rowptr=FakeCuda(n + 1, torch.int32), colind=FakeCuda(nnz, torch.int32),
                vals=FakeCuda(nnz, torch.float64), b=FakeCuda(n, torch.float64),
                x=FakeCuda(n, torch.float64), out=FakeCuda(2, torch.float64))


BAD = {
    "host_vals": ("vals", dict(cuda=False), "CUDA tensor"),
    "int64_rowptr": ("rowptr", dict(dtype=torch.int64), "torch.int32"),
    "int64_colind": ("colind", dict(dtype=torch.int64), "torch.int32"),
    "float32_vals": ("vals", dict(dtype=torch.float32), "torch.float64"),
    "float32_b": ("b", dict(dtype=torch.float32), "torch.float64"),
    "short_out": ("out", dict(numel=1), "out needs 2"),
    "short_rowptr": ("rowptr", dict(numel=10), "rowptr needs"),
    "short_x": ("x", dict(numel=9), "b and x need"),
    "colind_vs_vals": ("colind", dict(numel=27), "differ in length"),
    "strided_b": ("b", dict(contiguous=False), "contiguous"),
    "other_device": ("x", dict(index=3), "not the current device"),
}


@pytest.fixture(autouse=True)
def _no_library(monkeypatch):
    def boom():
        raise AssertionError("the library must not be called")
    monkeypatch.setattr(spai, "load", boom)


@pytest.mark.parametrize("case", list(BAD))
def test_bad_argument_raises_before_the_call(case):
    name, change, msg = BAD[case]
    args = _good()
    t = args[name]
    kw = dict(numel=t.numel(), dtype=t.dtype, cuda=True, contiguous=True, index=None)
    kw.update(change)
    args[name] = FakeCuda(**kw)
    with pytest.raises(ValueError, match=msg):
        spai.true_residual_noalloc(10, **args)


def test_good_arguments_reach_the_call():
    with pytest.raises(AssertionError, match="no pointer|library must not"):
        spai.true_residual_noalloc(10, **_good())
