"""Checkpoint / resume of the state between global iterations (the left-orthogonal TT
that Alg. 2 keeps): a2_tt_save / a2_tt_load round trip the cores bit for bit, resuming
repeats the next iteration, and damaged files are rejected.  C-ABI calls."""
import numpy as np
import pytest

from synthetic import chemistry_integrals, chemistry_mpo, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402

KW = dict(svd_tol=1e-10, eig_tol=1e-10, coarse_eps=1e-10)


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    c.close()


def test_round_trip_bitwise(ctx, tmp_path):
    raw = random_tt_cores([4, 2, 3, 4, 2], 5, 99)
    t = a2.TT.from_cores(ctx, raw)
    t.left_orthogonalize()
    path = tmp_path / "tt.a2ckp"
    t.save(path)
    u = a2.TT.load(ctx, path)
    assert u.phys == [4, 2, 3, 4, 2]
    for a, b in zip(t.cores(), u.cores()):
        assert a.shape == b.shape and np.array_equal(a, b)
    size = 8 + 4 + 4 * 5 + 4 * 6 + 8 * sum(c.size for c in t.cores())
    assert path.stat().st_size == size


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16", 2e-6)])
def test_resume_repeats_the_next_iteration(ctx, tmp_path, prec, tol):
    h, eri = chemistry_integrals(8, 2505)
    mpo = a2.MPO(ctx, chemistry_mpo(h, eri))
    t = a2.TT.from_cores(ctx, random_tt_cores([4] * 8, 8, 5))
    t.left_orthogonalize()
    kw = dict(partition=[3, 2, 2], D_max=16, prec=prec, sequential=True, **KW)
    a2.additive_sweep(ctx, t, mpo, 3, **kw)
    path = tmp_path / "it1.a2ckp"
    t.save(path)
    r_cont = a2.additive_sweep(ctx, t, mpo, 3, **kw)
    E_cont = a2.energy(ctx, t, mpo)[0]
    u = a2.TT.load(ctx, path)
    r_res = a2.additive_sweep(ctx, u, mpo, 3, **kw)
    E_res = a2.energy(ctx, u, mpo)[0]
    assert abs(r_cont["energy_in"] - r_res["energy_in"]) < 1e-13 * abs(E_cont)
    assert abs(r_cont["lambda_coarse"] - r_res["lambda_coarse"]) < tol * abs(E_cont)
    assert np.allclose(r_cont["S_hat"], r_res["S_hat"], atol=tol)
    assert abs(E_cont - E_res) < tol * abs(E_cont)


def test_damaged_files_rejected(ctx, tmp_path):
    t = a2.TT.from_cores(ctx, random_tt_cores([2] * 4, 2, 1))
    good = tmp_path / "good.a2ckp"
    t.save(good)
    data = good.read_bytes()
    cases = {"magic": b"XXXXXXXX" + data[8:], "truncated": data[:-8],
             "trailing": data + b"\0", "bonds": data[:12 + 16] + (7).to_bytes(4, "little")
             + data[12 + 20:]}
    for name, blob in cases.items():
        p = tmp_path / (name + ".a2ckp")
        p.write_bytes(blob)
        with pytest.raises(a2.A2Error):
            a2.TT.load(ctx, p)
    with pytest.raises(a2.A2Error):
        a2.TT.load(ctx, tmp_path / "missing.a2ckp")
