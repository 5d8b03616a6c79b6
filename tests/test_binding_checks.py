"""The Python binding refuses tensors that the C library would read or write
through a raw device pointer unless they are contiguous CUDA tensors of the
right type and size: a host pointer or a short buffer would otherwise reach
the kernels.  CPU only (a tensor subclass stands in for a CUDA tensor)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2305_17111_gb300 import _require_cuda  # noqa: E402


class _FakeCuda(torch.Tensor):
    @property
    def is_cuda(self):
        return True


def _fake(t):
    return torch.Tensor._make_subclass(_FakeCuda, t)


def test_host_tensors_and_arrays_are_refused():
    with pytest.raises(TypeError, match="CUDA"):
        _require_cuda(torch.zeros(4), "out", torch.float32, numel=4)
    with pytest.raises(TypeError, match="CUDA"):
        _require_cuda(np.zeros(4, np.float32), "out", torch.float32, numel=4)


def test_dtype_size_and_layout_are_checked():
    ok = _fake(torch.zeros(6))
    assert _require_cuda(ok, "out", torch.float32, numel=6) is ok
    assert _require_cuda(ok, "out", torch.float32, min_numel=5) is ok
    with pytest.raises(TypeError, match="dtype"):
        _require_cuda(_fake(torch.zeros(6, dtype=torch.float64)), "out", torch.float32)
    with pytest.raises(ValueError, match="6 elements"):
        _require_cuda(_fake(torch.zeros(5)), "out", torch.float32, numel=6)
    with pytest.raises(ValueError, match="at least 7"):
        _require_cuda(ok, "loglik", torch.float32, min_numel=7)
    with pytest.raises(TypeError, match="contiguous"):
        _require_cuda(_fake(torch.zeros(4, 4)).t(), "x", torch.float32)
