"""Second-level (coarse) minimisation of Sec. 3.1 (oracle; test only).

Given A_hat, S_hat (m x m, eq. A_reduced): eigendecompose S_hat = V diag(sig) V^T,
keep the p eigenvalues sig_k > eps * max(sig) (the rank-deficient branch of
Sec. 3.1 with the tolerance eps), form the reduced symmetric problem
    Sig+^{-1/2} V+^T A_hat V+ Sig+^{-1/2} z = lambda z      (eq. aux_eig_final_sym)
and return lambda_min and c = V+ Sig+^{-1/2} z (so c^T S_hat c = 1).  Sign
convention: c_0 >= 0, or if c_0 = 0 the entry of largest magnitude is positive.
Pinned by tests/test_oracle_dmrg.py (the coarse-solve test against
scipy.linalg.eigh(A, S), including a rank-deficient S).
"""
import numpy as np


def coarse_solve(A_hat, S_hat, eps=1e-10):
    A = 0.5 * (A_hat + A_hat.T)
    S = 0.5 * (S_hat + S_hat.T)
    sig, V = np.linalg.eigh(S)
    keep = sig > eps * sig.max()
    Vp, sp = V[:, keep], sig[keep]
    Ms = (Vp / np.sqrt(sp)).T @ A @ (Vp / np.sqrt(sp))
    lam, Z = np.linalg.eigh(0.5 * (Ms + Ms.T))
    c = (Vp / np.sqrt(sp)) @ Z[:, 0]
    ref = c[0] if abs(c[0]) > 1e-14 * np.abs(c).max() else c[np.argmax(np.abs(c))]
    if ref < 0:
        c = -c
    return c, float(lam[0]), int(keep.sum())
