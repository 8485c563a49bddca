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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))
