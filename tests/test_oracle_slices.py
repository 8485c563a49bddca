"""CPU: the one-slice oracle contractions used by the full-size GPU parity tests agree
with the full oracle contractions (which are themselves pinned to P*AP and to exact
diagonalisation in test_oracle_dmrg.py)."""
import numpy as np

from oracle.env import (env_left_update, env_left_update_entry, heff_apply,
                        heff_apply_entry)
from synthetic import chemistry_integrals, chemistry_mpo


def test_heff_entry_matches_full_contraction():
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    rng = np.random.default_rng(0)
    k, Dl, Dr = 2, 7, 9
    HL = rng.standard_normal((Dl, m[k].shape[0], Dl))
    HR = rng.standard_normal((Dr, m[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, 4, 4, Dr))
    y = heff_apply(HL, m[k], m[k + 1], HR, x)
    for a in range(Dl):
        for b in range(Dr):
            e = heff_apply_entry(HL, m[k], m[k + 1], HR, x, a, b)
            assert np.allclose(e, y[a, :, :, b], rtol=1e-13, atol=1e-13 * np.abs(y).max())


def test_env_entry_matches_full_update():
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    rng = np.random.default_rng(1)
    j, Dlb, Drb, Dlk, Drk = 3, 5, 6, 4, 7
    HL = rng.standard_normal((Dlb, m[j].shape[0], Dlk))
    bra = rng.standard_normal((Dlb, 4, Drb))
    ket = rng.standard_normal((Dlk, 4, Drk))
    out = env_left_update(HL, bra, m[j], ket)
    for b in range(Drb):
        for bp in range(Drk):
            e = env_left_update_entry(HL, bra, m[j], ket, b, bp)
            assert np.allclose(e, out[b, :, bp], rtol=1e-13, atol=1e-13 * np.abs(out).max())
