"""Gradient configuration (random chemistry integrals, L = 16, D = 256, P = 4): dE with
respect to the one- and two-body coefficients through the adjoint of the energy
sandwich (a2_energy_gradient), against the oracle's reduced density matrices of the
full state (tiny chains), central finite differences of FP64 energies, and single
entries at full size through one-term operators (oracle.env.sandwich)."""
import numpy as np
import pytest

from oracle.env import sandwich
from oracle.rdm import hamiltonian_gradient
from oracle.tt import tt_full
from synthetic import chemistry_integrals, chemistry_mpo, get_config, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    assert a2.device_error(c) == 0
    c.close()


def _split(g, L):
    return g[: L * L].reshape(L, L), g[L * L:].reshape(L, L, L, L)


def test_gradient_matches_rdms_small(ctx):
    L = 4
    h, eri = chemistry_integrals(L, 2505)
    W, cm = chemistry_mpo(h, eri, coeff_map=True)
    mpo = a2.MPO(ctx, W)
    cores = random_tt_cores([4] * L, 16, 5)          # not orthogonal, not normalised
    tt = a2.TT.from_cores(ctx, cores)
    E, g = a2.energy_gradient(ctx, tt, mpo, cm)
    gh, geri = _split(g, L)
    rh, reri = hamiltonian_gradient(tt_full(cores).ravel(), L)
    assert np.abs(gh - rh).max() < 1e-12
    assert np.abs(geri - reri).max() < 1e-12
    assert abs(np.sum(h * gh) + np.sum(eri * geri) - E) < 1e-12 * abs(E)


def test_gradient_central_differences(ctx):
    L, step = 5, 1e-5
    h, eri = chemistry_integrals(L, 99)
    W, cm = chemistry_mpo(h, eri, coeff_map=True)
    mpo = a2.MPO(ctx, W)
    tt = a2.TT.from_cores(ctx, random_tt_cores([4] * L, 12, 6))
    tt.left_orthogonalize()
    _, g = a2.energy_gradient(ctx, tt, mpo, cm)
    gh, geri = _split(g, L)

    def energy(hh, ee):
        m = a2.MPO(ctx, chemistry_mpo(hh, ee))
        e, _ = a2.energy(ctx, tt, m, "fp64")
        m.close()
        return e

    for (i, j) in [(0, 0), (1, 4), (3, 2)]:
        dh = np.zeros_like(h)
        dh[i, j] = step
        fd = (energy(h + dh, eri) - energy(h - dh, eri)) / (2 * step)
        assert abs(fd - gh[i, j]) < 1e-8 * max(1.0, abs(gh[i, j]))
    for idx in [(0, 1, 2, 3), (4, 4, 4, 4), (2, 0, 3, 1)]:
        de = np.zeros_like(eri)
        de[idx] = step
        fd = (energy(h, eri + de) - energy(h, eri - de)) / (2 * step)
        assert abs(fd - geri[idx]) < 1e-8 * max(1.0, abs(geri[idx]))


def test_energy_autograd(ctx):
    L = 4
    h, eri = chemistry_integrals(L, 31)
    W, cm = chemistry_mpo(h, eri, coeff_map=True)
    mpo = a2.MPO(ctx, W)
    tt = a2.TT.from_cores(ctx, random_tt_cores([4] * L, 16, 8))
    ht = torch.tensor(h, requires_grad=True)
    et = torch.tensor(eri, requires_grad=True)
    E = a2.energy_autograd(ht, et, ctx, tt, mpo, cm)
    (2.0 * E).backward()
    _, g = a2.energy_gradient(ctx, tt, mpo, cm)
    gh, geri = _split(g, L)
    assert np.allclose(ht.grad.numpy(), 2.0 * gh, rtol=1e-13, atol=1e-14)
    assert np.allclose(et.grad.numpy(), 2.0 * geri, rtol=1e-13, atol=1e-14)
    e = float(E.detach())
    assert abs(e - a2.energy(ctx, tt, mpo, "fp64")[0]) < 1e-12 * abs(e)


def test_gradient_full_size_sampled(ctx):
    """L = 16, D = 256 (the gradient configuration's sizes), random left-orthogonal TT."""
    cfg = get_config("chem_grad_L16_D256")
    L, D = cfg["L"], cfg["D"]
    h, eri = chemistry_integrals(L, cfg["seed_int"])
    W, cm = chemistry_mpo(h, eri, coeff_map=True)
    mpo = a2.MPO(ctx, W)
    tt = a2.TT.from_cores(ctx, random_tt_cores([4] * L, D, 17))
    tt.left_orthogonalize()
    E, g = a2.energy_gradient(ctx, tt, mpo, cm)
    gh, geri = _split(g, L)
    cores = tt.cores()
    assert abs(np.sum(h * gh) + np.sum(eri * geri) - E) < 1e-10 * abs(E)
    for (i, j) in [(0, 0), (3, 12), (15, 7)]:
        h1 = np.zeros((L, L))
        h1[i, j] = 1.0
        ref = sandwich(cores, chemistry_mpo(h1, np.zeros((L, L, L, L))), cores)
        assert abs(gh[i, j] - ref) < 1e-10 * max(1.0, abs(ref))
    for idx in [(0, 1, 2, 3), (8, 8, 7, 7), (15, 0, 3, 12)]:
        e1 = np.zeros((L, L, L, L))
        e1[idx] = 1.0
        ref = sandwich(cores, chemistry_mpo(np.zeros((L, L)), e1), cores)
        assert abs(geri[idx] - ref) < 1e-10 * max(1.0, abs(ref))


def _converge_fp64(ctx, tt, mpo, L, max_iter=12):
    """FP64 global iterations at full rank until the energy stops moving (|dE| < 1e-13)."""
    E_prev = None
    for _ in range(max_iter):
        rep = a2.additive_sweep(ctx, tt, mpo, L - 1, D_max=64, prec="fp64", svd_tol=1e-13,
                                eig_tol=1e-12, coarse_eps=1e-10)
        E = rep["energy_in"]
        if E_prev is not None and abs(E - E_prev) < 1e-13:
            break
        E_prev = E
    return a2.energy(ctx, tt, mpo, "fp64")[0]


def _images(i, j, k, l):
    """The distinct index quadruples related by the 8-fold symmetry of real (ij|kl)."""
    return sorted({(i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                   (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)})


def test_hellmann_feynman_at_converged_ground_state(ctx):
    """L = 4 orbitals, full rank (no truncation): at the converged A2DMRG ground state the
    gradient of a2_energy_gradient is the total derivative of the ground energy.  Checked
    against central differences (step 1e-5) of ground energies re-converged to 1e-13 with
    the perturbed integrals (symmetric perturbations, so that H stays symmetric), and
    against the oracle's RDMs of the exact-diagonalisation ground vector."""
    from oracle.ed import fermion_sparse
    L, step = 4, 1e-5
    h, eri = chemistry_integrals(L, 2505)
    W, cm = chemistry_mpo(h, eri, coeff_map=True)
    mpo = a2.MPO(ctx, W)
    tt = a2.TT.from_cores(ctx, random_tt_cores([4] * L, 16, 23429))
    tt.left_orthogonalize()
    E0 = _converge_fp64(ctx, tt, mpo, L)
    E, g = a2.energy_gradient(ctx, tt, mpo, cm)
    gh, geri = _split(g, L)
    w, V = np.linalg.eigh(fermion_sparse(h, eri).toarray())
    assert abs(E0 - w[0]) < 1e-11 * abs(w[0])
    rh, reri = hamiltonian_gradient(V[:, 0], L)
    assert np.abs(gh - rh).max() < 1e-8
    assert np.abs(geri - reri).max() < 1e-8
    base = tt.cores()

    def ground(hh, ee):
        m = a2.MPO(ctx, chemistry_mpo(hh, ee))
        t = a2.TT.from_cores(ctx, base)
        e = _converge_fp64(ctx, t, m, L)
        t.close()
        m.close()
        return e

    for (i, j) in [(0, 0), (1, 3), (2, 2)]:
        dh = np.zeros_like(h)
        dh[i, j] = dh[j, i] = step
        fd = (ground(h + dh, eri) - ground(h - dh, eri)) / (2 * step)
        want = gh[i, j] + (gh[j, i] if i != j else 0.0)
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want))
    for q in [(0, 1, 2, 3), (1, 1, 0, 0), (3, 2, 3, 2)]:
        de = np.zeros_like(eri)
        for im in _images(*q):
            de[im] = step
        fd = (ground(h, eri + de) - ground(h, eri - de)) / (2 * step)
        want = sum(geri[im] for im in _images(*q))
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want))


def test_gradient_at_converged_gradient_config_iterate(ctx):
    """The gradient configuration itself (L = 16, D = 256, P = 4): the BF16 default path
    takes the seeded TT through 10 global iterations (near its converged energy), then the
    gradient at that iterate is checked on sampled entries against the oracle's sandwich
    of the iterate with one-term operators, and against E = sum theta dE/dtheta."""
    cfg = get_config("chem_grad_L16_D256")
    L, D = cfg["L"], cfg["D"]
    h, eri = chemistry_integrals(L, cfg["seed_int"])
    W, cm = chemistry_mpo(h, eri, coeff_map=True)
    mpo = a2.MPO(ctx, W)
    tt = a2.TT.from_cores(ctx, random_tt_cores([4] * L, cfg["r0"], cfg["seed_tt"]))
    tt.left_orthogonalize()
    for _ in range(10):
        a2.additive_sweep(ctx, tt, mpo, cfg["P"], partition=cfg["partition"], D_max=D,
                          prec="bf16", svd_tol=1e-6, eig_tol=1e-6, coarse_eps=1e-10,
                          max_restarts=50, sequential=True)
    E, g = a2.energy_gradient(ctx, tt, mpo, cm)
    gh, geri = _split(g, L)
    cores = tt.cores()
    assert max(c.shape[2] for c in cores) == D
    assert abs(np.sum(h * gh) + np.sum(eri * geri) - E) < 1e-10 * abs(E)
    for (i, j) in [(0, 0), (7, 8), (12, 3)]:
        h1 = np.zeros((L, L))
        h1[i, j] = 1.0
        ref = sandwich(cores, chemistry_mpo(h1, np.zeros((L, L, L, L))), cores)
        assert abs(gh[i, j] - ref) < 1e-10 * max(1.0, abs(ref))
    for idx in [(0, 0, 1, 1), (8, 7, 7, 8), (15, 2, 3, 14)]:
        e1 = np.zeros((L, L, L, L))
        e1[idx] = 1.0
        ref = sandwich(cores, chemistry_mpo(np.zeros((L, L)), e1), cores)
        assert abs(geri[idx] - ref) < 1e-10 * max(1.0, abs(ref))
