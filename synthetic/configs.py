"""The five benchmark workloads (sizes, seeds, partitions), as plain data."""

CONFIGS = {
    "heisenberg_L12_D32": dict(
        kind="heisenberg", L=12, n=2, J=1.0, D=32, P=2, partition=[6, 5],
        seed_tt=23429, r0=4),
    "chem_L16_D256": dict(
        kind="chemistry", L=16, n=4, seed_int=2505, D=256, P=4,
        partition=[4, 4, 4, 3], seed_tt=23429, r0=4),
    "chem_L32_D512": dict(
        kind="chemistry", L=32, n=4, seed_int=2506, D=512, P=8,
        partition=[2, 3, 4, 5, 5, 4, 4, 4], seed_tt=23429, r0=4),
    "chem_grad_L16_D256": dict(
        kind="chemistry", L=16, n=4, seed_int=2505, D=256, P=4,
        partition=[4, 4, 4, 3], seed_tt=23429, r0=4),
    "hubbard_L64_D1024": dict(
        kind="hubbard", L=64, n=4, t=1.0, U=4.0, D=1024, P=16,
        partition=[2, 3, 4, 5, 5, 4, 4, 4, 2, 3, 4, 5, 5, 4, 4, 5],
        seed_tt=23429, r0=4),
}


def get_config(name):
    return dict(CONFIGS[name])
