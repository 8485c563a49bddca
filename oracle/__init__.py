"""Plain FP64 CPU oracle of two-site DMRG (Alg. 1) and two-site A2DMRG (Alg. 2).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  It shares
no code with the CUDA path; the two meet only in the seeded input generators
of the `synthetic` package.

Every routine is a direct, slow, NumPy/SciPy restatement of the paper's
definitions (Sec. 2-3.1, App. A): TT contraction (Def. TT contraction mapping),
orthogonal decompositions (Def. orthogonal TT), environments (eqs. env_L /
env_R), the two-site micro-iteration as the lowest eigenpair of the projected
operator (Lemma DMRG micro-iterations), the truncated SVD step (Alg. 1 step 2),
the LQ sweep of Alg. 2 step 1, the coarse problem of Sec. 3.1 (eq. A_reduced,
eq. aux_eig_final_sym) and TT rounding for the compression step; `blocksparse` adds the
particle-number preserving variants of Sec. 3.2 (bond charges, block-wise truncation).

Parity status per function is listed in each module's header.
"""
