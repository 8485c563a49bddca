"""Environments and the two-site effective Hamiltonian (oracle; test only).

Left environment after sites 0..j-1, eq. env_L (App. A):
    HL[a, w, a'] = sum U*(bra) A U(ket) over those sites, bra index first.
Right environment of sites j..L-1, eq. env_R, same index order [bra, w, ket].
Two-site H_eff at bond k (sites k, k+1), Lemma (DMRG micro-iterations) and
the contraction of App. A with the two-site modification:
    y[a,s1,s2,b] = sum L[a,w,a'] A_k[w,s1,t1,w1] A_{k+1}[w1,s2,t2,w2]
                        R[b,w2,b'] x[a',t1,t2,b'].
Pinned by tests/test_oracle_dmrg.py (H_eff equals P* A P built from the dense
operator and the retraction of Def. retraction on tiny chains; symmetry).
"""
import numpy as np


def env_left_update(HL, U_bra, W, U_ket):
    T = np.tensordot(HL, U_ket, axes=(2, 0))              # a w t b'
    T = np.tensordot(T, W, axes=([1, 2], [0, 2]))         # a b' s w'
    T = np.tensordot(U_bra, T, axes=([0, 1], [0, 2]))     # b b' w'
    return np.ascontiguousarray(T.transpose(0, 2, 1))     # b w' b'


def env_right_update(HR, V_bra, W, V_ket):
    T = np.tensordot(V_ket, HR, axes=(2, 2))              # a' t b w'
    T = np.tensordot(W, T, axes=([2, 3], [1, 3]))         # w s a' b
    T = np.tensordot(V_bra, T, axes=([1, 2], [1, 3]))     # a w a'
    return np.ascontiguousarray(T)


def left_envs(U, mpo, upto=None):
    """HL[j] = environment of sites < j for j = 0..upto (default L-1)."""
    L = len(U)
    upto = L - 1 if upto is None else upto
    out = [np.ones((1, 1, 1))]
    for j in range(upto):
        out.append(env_left_update(out[-1], U[j], mpo[j], U[j]))
    return out


def right_envs(V, mpo, downto=1):
    """HR[j] = environment of sites >= j for j = downto..L (dict)."""
    L = len(V)
    out = {L: np.ones((1, 1, 1))}
    for j in range(L - 1, downto - 1, -1):
        out[j] = env_right_update(out[j + 1], V[j], mpo[j], V[j])
    return out


def heff_apply(HL, W1, W2, HR, x):
    T = np.tensordot(HL, x, axes=(2, 0))                  # a w t1 t2 b'
    T = np.tensordot(T, W1, axes=([1, 2], [0, 2]))        # a t2 b' s1 w1
    T = np.tensordot(T, W2, axes=([1, 4], [2, 0]))        # a b' s1 s2 w2
    T = np.tensordot(T, HR, axes=([1, 4], [2, 1]))        # a s1 s2 b
    return T


def heff1_apply(HL, W, HR, x):
    """One-site H_eff of the j-th one-site micro-iteration (Def. of the micro-iterations,
    one-site case): y[a,s,b] = sum HL[a,w,a'] W[w,s,t,w'] HR[b,w',b'] x[a',t,b']."""
    T = np.tensordot(HL, x, axes=(2, 0))                  # a w t b'
    T = np.tensordot(T, W, axes=([1, 2], [0, 2]))         # a b' s w'
    T = np.tensordot(T, HR, axes=([1, 3], [2, 1]))        # a s b
    return T


def heff_apply_entry(HL, W1, W2, HR, x, a, b):
    """The slice y[a, :, :, b] of heff_apply, contracted for that one pair of outer bond
    indices only (the same sum as above with a and b fixed), so that single outputs of a
    full-size application can be checked without forming the whole product."""
    T = np.tensordot(HL[a], x, axes=(1, 0))                      # w t1 t2 b'
    T = np.tensordot(T, HR[b], axes=(3, 1))                      # w t1 t2 w2
    T = np.tensordot(W1, T, axes=([0, 2], [0, 1]))               # s1 w1 t2 w2
    return np.tensordot(T, W2, axes=([1, 2, 3], [0, 2, 3]))      # s1 s2


def env_left_update_entry(HL, U_bra, W, U_ket, b, bp):
    """The slice out[b, :, bp] of env_left_update (eq. env_L update with bra index b and
    ket index bp fixed)."""
    X = np.tensordot(HL, U_ket[:, :, bp], axes=(2, 0))           # a w t
    Z = np.tensordot(U_bra[:, :, b], X, axes=(0, 0))             # s w t
    return np.tensordot(Z, W, axes=([0, 1, 2], [1, 0, 2]))       # w'


def heff_dense(HL, W1, W2, HR):
    Dl, n1, n2, Dr = HL.shape[0], W1.shape[1], W2.shape[1], HR.shape[0]
    N = Dl * n1 * n2 * Dr
    M = np.empty((N, N))
    e = np.zeros(N)
    for i in range(N):
        e[:] = 0.0
        e[i] = 1.0
        M[:, i] = heff_apply(HL, W1, W2, HR, e.reshape(Dl, n1, n2, Dr)).ravel()
    return M


def sandwich(bra, mpo, ket):
    """<tau(bra), A tau(ket)> over the whole chain."""
    H = np.ones((1, 1, 1))
    for b, W, k in zip(bra, mpo, ket):
        H = env_left_update(H, b, W, k)
    return float(H[0, 0, 0])
