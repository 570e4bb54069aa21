"""Host-side argument checks of the allocation-free RMSE entry point's
binding (no GPU): every malformed argument raises ValueError before anything
reaches the library, so no kernel can be launched on a bad pointer."""
import pytest

from paper_2012_03550_gb300 import binding as B


class FakeDevice:
    def __init__(self, index, cuda=True):
        self.index = index
        self.type = "cuda" if cuda else "cpu"

    def __str__(self):
        return f"{self.type}:{self.index}"


class FakeTensor:
    """Stands in for a torch tensor: only the attributes the checks read."""

    def __init__(self, shape, dtype, cuda=True, device=0, contiguous=True):
        self.shape = tuple(shape)
        self.dtype = f"torch.{dtype}"
        self.is_cuda = cuda
        self.device = FakeDevice(device if cuda else None, cuda)
        self._contig = contiguous

    def dim(self):
        return len(self.shape)

    def numel(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return 0x1000


SHAPE, RANKS, R, K = (50, 40, 30), (3, 4, 5), 2, 100


def _good():
    A = [FakeTensor((I, J), "float32") for I, J in zip(SHAPE, RANKS)]
    Bm = [FakeTensor((J, R), "float32") for J in RANKS]
    return dict(A=A, B=Bm, coords=FakeTensor((K, 3), "int32"), values=FakeTensor((K,), "float32"),
                out=FakeTensor((2,), "float64"))


def test_good_arguments_pass():
    a = _good()
    B.check_static_args(3, SHAPE, RANKS, R, a["A"], a["B"], K, a["coords"], a["values"], a["out"],
                        current_device=0)


@pytest.fixture(autouse=True)
def no_library(monkeypatch):
    # a call that got past the checks would reach the library: make that fail loudly
    def boom(*a, **k):
        raise AssertionError("the library was called")
    monkeypatch.setattr(B, "lib", boom)


def _bad(**over):
    a = _good()
    k = over.pop("k", K)
    a.update(over)
    with pytest.raises(ValueError):
        B.std_rmse_static(3, SHAPE, RANKS, R, a["A"], a["B"], k, a["coords"], a["values"], a["out"])


def test_rejects_host_arrays(monkeypatch):
    import numpy as np
    import torch
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    _bad(values=np.zeros(K, np.float32))


def test_rejects_everything_without_a_device(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    _bad()


def test_rejects_cpu_tensor_and_other_device(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    _bad(coords=FakeTensor((K, 3), "int32", cuda=False))
    _bad(out=FakeTensor((2,), "float64", device=1))


def test_rejects_wrong_dtypes(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    _bad(coords=FakeTensor((K, 3), "int64"))
    _bad(values=FakeTensor((K,), "float64"))
    _bad(out=FakeTensor((2,), "float32"))
    a = _good()["A"]
    a[1] = FakeTensor((40, 4), "bfloat16")
    _bad(A=a)


def test_rejects_wrong_shapes_and_short_buffers(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    a = _good()["A"]
    a[2] = FakeTensor((30, 4), "float32")          # J_3 is 5
    _bad(A=a)
    b = _good()["B"]
    b[0] = FakeTensor((3, R + 1), "float32")
    _bad(B=b)
    _bad(A=_good()["A"][:2])                        # one matrix short
    _bad(coords=FakeTensor((K - 1, 3), "int32"))    # fewer rows than k
    _bad(coords=FakeTensor((K, 4), "int32"))        # wrong order
    _bad(values=FakeTensor((K - 1,), "float32"))
    _bad(out=FakeTensor((1,), "float64"))
    _bad(out=FakeTensor((2,), "float64", contiguous=False))
    _bad(k=-1)
