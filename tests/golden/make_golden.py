"""Writes tests/golden/golden_values.json from the oracle's exact
diagonalisation routines and closed forms only (no GPU code involved).

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle.ed import fermion_sparse, ground_energy, heisenberg_sparse  # noqa: E402
from synthetic import chemistry_integrals  # noqa: E402


def main():
    out = {}
    out["heisenberg_L12_obc_J1_ed"] = dict(
        value=ground_energy(heisenberg_sparse(12)),
        source="ED of the 4096x4096 Heisenberg chain (oracle.ed); config heisenberg_L12_D32")
    h, eri = chemistry_integrals(6, 2505)
    out["chemistry_L6_seed2505_ed"] = dict(
        value=ground_energy(fermion_sparse(h, eri)),
        source="ED of the Fock-space Hamiltonian of Sec. 3.2, L=6 spatial orbitals, seed 2505")
    h8, _ = chemistry_integrals(8, 2505)
    e = np.linalg.eigvalsh(h8)
    out["free_fermion_L8_seed2505_closed_form"] = dict(
        value=float(2.0 * e[e < 0].sum()),
        source="one-body only: 2 * sum of negative eigenvalues of h (whole Fock space)")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
