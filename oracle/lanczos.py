"""Restarted Lanczos for the lowest eigenpair (oracle; test only).

Used for the local two-site problems (Lemma DMRG micro-iterations; the
experiments use Lanczos warm-started from the previous iterate).  Full
re-orthogonalisation (twice) against the current Krylov basis; the basis is
restarted from the current Ritz vector after max_krylov vectors.  Stop when
the Lanczos residual estimate |beta_j e_j^T s| <= tol * max(1, |theta|) for the
unit Ritz vector, or on Krylov breakdown.  Returned vector has <x, x0> >= 0.
Pinned by tests/test_oracle_dmrg.py against numpy.linalg.eigh on dense H_eff.
"""
import numpy as np


def lanczos_lowest(matvec, x0, tol=1e-10, max_krylov=40, max_cycles=200):
    x0 = np.asarray(x0, dtype=np.float64)
    shape = x0.shape
    v = x0.ravel().copy()
    nv = np.linalg.norm(v)
    if nv == 0.0:
        v = np.ones_like(v)
        nv = np.linalg.norm(v)
    v /= nv
    N = v.size
    m_max = min(max_krylov, N)
    n_mv = 0
    theta = None
    for cycle in range(1, max_cycles + 1):
        V = [v]
        alphas, betas = [], []
        converged = False
        for j in range(m_max):
            w = matvec(V[j].reshape(shape)).ravel()
            n_mv += 1
            a = float(V[j] @ w)
            alphas.append(a)
            Vm = np.array(V)
            w = w - Vm.T @ (Vm @ w)
            w = w - Vm.T @ (Vm @ w)
            b = float(np.linalg.norm(w))
            T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
            ev, evec = np.linalg.eigh(T)
            theta, s = ev[0], evec[:, 0]
            resid = abs(b * s[-1])
            breakdown = b <= 1e-14 * max(1.0, abs(theta))
            if resid <= tol * max(1.0, abs(theta)) or breakdown or len(V) == N:
                converged = True
                break
            if j == m_max - 1:
                break
            betas.append(b)
            V.append(w / b)
        x = np.array(V[:len(s)]).T @ s
        x /= np.linalg.norm(x)
        v = x
        if converged:
            break
    if float(x @ x0.ravel()) < 0:
        x = -x
    return float(theta), x.reshape(shape), n_mv, cycle
