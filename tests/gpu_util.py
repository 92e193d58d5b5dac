"""Helpers for the GPU tests: build/load the library, move arrays to and from
the device.  The library is always reached through its C ABI."""
import numpy as np
import pytest

import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300 import build as _build


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    ntt._lib.load()
    return torch


def to_dev(a: np.ndarray, torch):
    """numpy uint32/uint64 array -> device tensor holding the same bytes."""
    a = np.ascontiguousarray(a)
    view = a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int64)
    return torch.from_numpy(view.copy()).cuda()


def from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)
