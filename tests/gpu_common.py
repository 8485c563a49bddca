"""Helpers shared by the GPU parity tests (device buffers via torch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    torch.cuda.synchronize()
    return t


def host(t, ctx=None):
    if ctx is not None:
        ctx.synchronize()
    torch.cuda.synchronize()
    return t.cpu().numpy()


def elem(a, b):
    """Largest element-wise deviation against the output scale: max |a - b| / max |b|
    (a wrong block at a ragged edge shows here even when the norm barely moves)."""
    a, b = np.ravel(a), np.ravel(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if b.size else 0.0


def rel(a, b):
    """The larger of the norm-wise relative error and the element-wise one (elem)."""
    nr = float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))
    return max(nr, elem(a, b))
