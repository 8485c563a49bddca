"""Failure detection on the device without a GPU fault: a bounded mbarrier wait of the
tcgen05 GEMM kernel is made to run out (its producer role issues no copies, the wait limit
is 2^14 iterations), and the call reports A2_ETIMEOUT with the device error word; the
context then runs ordinary work correctly.  C-ABI calls."""
import numpy as np
import pytest

from oracle.env import heff_apply as oracle_heff
from synthetic import heisenberg_mpo

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402
from gpu_common import dev, host, rel  # noqa: E402

A2_ETIMEOUT = -6


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    c.close()


def test_bounded_wait_runs_out_and_reports_timeout(ctx):
    assert a2.device_error(ctx) == 0
    st, code = a2.selftest_timeout(ctx)
    assert st == A2_ETIMEOUT
    assert code == 3                         # the MMA role's wait for a full stage
    assert "gave up" in a2.last_error(ctx)
    assert a2.device_error(ctx) == 0         # the word was read and cleared
    # the context and the tensor-core path still work
    m = heisenberg_mpo(8)
    mpo = a2.MPO(ctx, m)
    rng = np.random.default_rng(3)
    k, D = 3, 16
    Lh = rng.standard_normal((D, m[k].shape[0], D))
    Rh = rng.standard_normal((D, m[k + 1].shape[3], D))
    x = rng.standard_normal((D, 2, 2, D))
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec="f32emu")
    assert rel(host(y, ctx), oracle_heff(Lh, m[k], m[k + 1], Rh, x)) < 5e-6
    assert a2.device_error(ctx) == 0


def test_selftest_repeats(ctx):
    """Each run clears the word it raised, so a second run behaves like the first."""
    for _ in range(2):
        st, code = a2.selftest_timeout(ctx)
        assert st == A2_ETIMEOUT and code == 3
        assert a2.device_error(ctx) == 0
