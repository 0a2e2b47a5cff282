"""Helpers shared by the GPU parity tests (device tensors, error norms)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device())


def rel_err(a, ref):
    """Norm-wise relative error |a - ref| / |ref|."""
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))


def max_err(a, ref):
    """Element-wise max |a - ref| / max |ref|."""
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.abs(a - ref).max() / np.abs(ref).max())
