"""The allocation-free H_eff entry point (a2_heff_apply_noalloc), called through the
C ABI, must give the same y as the regular FP64 entry point (a2_heff_apply) on two
calls in a row, and must refuse sizes above its fixed scratch.  It is meant for
callers that cannot allocate device memory while they run.  This file sorts last
so that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402
from paper_2505_23429_gb300.a2dmrg import heff_apply_noalloc  # noqa: E402
from gpu_common import dev, host, rel  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    c.close()


def _case(cores, k, Dl, Dr, n, seed):
    rng = np.random.default_rng(seed)
    Lh = rng.standard_normal((Dl, cores[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, cores[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, n, n, Dr))
    return dev(Lh), dev(Rh), dev(x)


@pytest.mark.parametrize("which,k,Dl,Dr", [("heis", 5, 32, 32), ("heis", 0, 1, 32),
                                           ("chem", 2, 16, 64), ("chem", 4, 64, 1)])
def test_noalloc_matches_regular_entry_point_twice(ctx, which, k, Dl, Dr):
    if which == "heis":
        cores, n = heisenberg_mpo(12), 2
    else:
        h, eri = chemistry_integrals(6, 2505)
        cores, n = chemistry_mpo(h, eri), 4
    mpo = a2.MPO(ctx, cores)
    L, R, x = _case(cores, k, Dl, Dr, n, k + Dl)
    y_ref = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, L, R, x, y_ref, prec="fp64")
    ref = host(y_ref, ctx)
    for _ in range(2):                       # the scratch keeps the previous call's data
        y = torch.full(x.shape, float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        heff_apply_noalloc(ctx, mpo, k, L, R, x, y)
        assert rel(host(y, ctx), ref) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    h, eri = chemistry_integrals(6, 2505)
    cores = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, cores)
    L, R, x = _case(cores, 2, 64, 64, 4, 1)      # needs far more than 4 Mi doubles
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(a2.A2Error, match="fixed scratch"):
        heff_apply_noalloc(ctx, mpo, 2, L, R, x, y)
