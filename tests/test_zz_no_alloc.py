"""The allocation-free H_eff entry point (a2_heff_apply_noalloc), called through the
C ABI, must give the same y as the regular FP64 entry point (a2_heff_apply) on two
calls in a row, agree with the oracle's H_eff contraction, overwrite whatever an earlier
call of a different shape left in its scratch, and refuse sizes above its fixed scratch.
It is meant for callers that cannot allocate device memory while they run (their GPU
memory belongs to their own pool or budget).  This file sorts last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from oracle.env import heff_apply as oracle_heff
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


def _host_case(cores, k, Dl, Dr, n, seed):
    rng = np.random.default_rng(seed)
    Lh = rng.standard_normal((Dl, cores[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, cores[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, n, n, Dr))
    return Lh, Rh, x


def _case(cores, k, Dl, Dr, n, seed):
    return tuple(dev(a) for a in _host_case(cores, k, Dl, Dr, n, seed))


def _mpo(which):
    if which == "heis":
        return heisenberg_mpo(12), 2
    h, eri = chemistry_integrals(6, 2505)
    return chemistry_mpo(h, eri), 4


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


@pytest.mark.parametrize("which,k,Dl,Dr", [("heis", 5, 8, 8), ("chem", 2, 9, 13)])
def test_noalloc_matches_oracle(ctx, which, k, Dl, Dr):
    cores, n = _mpo(which)
    mpo = a2.MPO(ctx, cores)
    Lh, Rh, xh = _host_case(cores, k, Dl, Dr, n, 7 + k)
    ref = oracle_heff(Lh, cores[k], cores[k + 1], Rh, xh)
    y = torch.full(xh.shape, float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    heff_apply_noalloc(ctx, mpo, k, dev(Lh), dev(Rh), dev(xh), y)
    assert rel(host(y, ctx), ref) < 1e-12


def test_noalloc_after_a_larger_call_of_another_layout(ctx):
    """A large chemistry call fills much of the scratch with its own T1/T2/T3 layout;
    the smaller Heisenberg call that follows reads only what it wrote itself."""
    chem, _ = _mpo("chem")
    heis, _ = _mpo("heis")
    m_chem, m_heis = a2.MPO(ctx, chem), a2.MPO(ctx, heis)
    Lc, Rc, xc = _host_case(chem, 2, 16, 64, 4, 11)
    yc = torch.full(xc.shape, float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    heff_apply_noalloc(ctx, m_chem, 2, dev(Lc), dev(Rc), dev(xc), yc)
    assert rel(host(yc, ctx), oracle_heff(Lc, chem[2], chem[3], Rc, xc)) < 1e-12
    Lh, Rh, xh = _host_case(heis, 5, 32, 32, 2, 12)
    yh = torch.full(xh.shape, float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    heff_apply_noalloc(ctx, m_heis, 5, dev(Lh), dev(Rh), dev(xh), yh)
    assert rel(host(yh, ctx), oracle_heff(Lh, heis[5], heis[6], Rh, xh)) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    h, eri = chemistry_integrals(6, 2505)
    cores = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, cores)
    L, R, x = _case(cores, 2, 64, 64, 4, 1)      # needs far more than 4 Mi doubles
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(a2.A2Error, match="fixed scratch"):
        heff_apply_noalloc(ctx, mpo, 2, L, R, x, y)
