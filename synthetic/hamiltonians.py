"""Synthetic Hamiltonians in matrix-product-operator form (eq. MPO, App. A).

MPO core convention (shared by every consumer): core j is a dense float64
array W[w_left, s, t, w_right] of shape (R_{j-1}, n, n, R_j) with R_0 = R_L = 1,
where s is the output (bra) physical index and t the input (ket) index, so that
(A x)(s_1..s_L) = sum_t W_1[.,s_1,t_1,.] ... W_L[.,s_L,t_L,.] x(t_1..t_L).

Two families are built here:

* the spin-1/2 Heisenberg chain with open boundaries (exact 5-state MPO);
* the second-quantised electronic Hamiltonian of Sec. 3.2 over spatial orbitals
  with spin (local basis |0>, |up>, |dn>, |up dn>, index n_up + 2 n_dn;
  Jordan-Wigner mode order 1up, 1dn, 2up, 2dn, ...),
      H = sum_{ij,s} h_ij a+_{is} a_{js}
        + 1/2 sum_{ijkl,s,t} (ij|kl) a+_{is} a+_{kt} a_{lt} a_{js},
  (chemists' notation, so the paper's V_{ijkl} equals (ik|jl)), assembled by an
  exact operator-string automaton: every term is split at one site, left of it
  the automaton state records the operator prefix (unweighted), right of it the
  remaining operators (weighted), so that sums over the far indices collapse
  onto shared states (complementary operators).  No truncation is applied.
"""
import bisect
import functools
import itertools

import numpy as np

from .rng import SplitMix64

# ---------------------------------------------------------------- spin chain

def heisenberg_mpo(L, J=1.0):
    """H = J sum_i S_i . S_{i+1} (open chain).  Local basis |up>=0, |dn>=1."""
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])   # S+ |dn> = |up>
    sm = sp.T.copy()
    sz = np.diag([0.5, -0.5])
    eye = np.eye(2)
    W = np.zeros((5, 2, 2, 5))
    W[0, :, :, 0] = eye
    W[0, :, :, 1] = sp
    W[0, :, :, 2] = sm
    W[0, :, :, 3] = sz
    W[1, :, :, 4] = 0.5 * J * sm
    W[2, :, :, 4] = 0.5 * J * sp
    W[3, :, :, 4] = J * sz
    W[4, :, :, 4] = eye
    cores = []
    for j in range(L):
        c = W
        if j == 0:
            c = c[0:1]
        if j == L - 1:
            c = c[..., 4:5]
        cores.append(np.ascontiguousarray(c))
    return cores


# ---------------------------------------------------------------- integrals

def chemistry_integrals(L, seed):
    """Random chemistry-like integrals.

    h: upper triangle (i <= j) drawn N(0,1)/sqrt(L) in row-major order, mirrored,
    then h_ii += eps_i with eps_i = -2 + 4 i/(L-1) (diagonal dominance).
    (ij|kl): one draw 0.1 N(0,1)/L per canonical quadruple (i>=j, k>=l,
    ij>=kl in compound index) in lexicographic order, expanded with the
    8-fold permutational symmetry.
    """
    g = SplitMix64(seed)
    h = np.zeros((L, L))
    iu = [(i, j) for i in range(L) for j in range(i, L)]
    vals = g.standard_normal(len(iu)) / np.sqrt(L)
    for (i, j), v in zip(iu, vals):
        h[i, j] = h[j, i] = v
    eps = -2.0 + 4.0 * np.arange(L) / max(L - 1, 1)
    h[np.diag_indices(L)] += eps
    pairs = [(i, j) for i in range(L) for j in range(i + 1)]
    quads = [(p, q) for a, p in enumerate(pairs) for q in pairs[:a + 1]]
    vals = 0.1 * g.standard_normal(len(quads)) / L
    eri = np.zeros((L, L, L, L))
    for ((i, j), (k, l)), v in zip(quads, vals):
        for (a, b) in ((i, j), (j, i)):
            for (c, d) in ((k, l), (l, k)):
                eri[a, b, c, d] = v
                eri[c, d, a, b] = v
    return h, eri


def hubbard_integrals(L, t=1.0, U=4.0):
    """1D Hubbard chain as integrals: h_{i,i+1} = -t, (ii|ii) = U."""
    h = np.zeros((L, L))
    for i in range(L - 1):
        h[i, i + 1] = h[i + 1, i] = -t
    eri = np.zeros((L, L, L, L))
    for i in range(L):
        eri[i, i, i, i] = U
    return h, eri


# ---------------------------------------------------------------- automaton

_I2 = np.eye(2)
_Z2 = np.diag([1.0, -1.0])
_CD = np.array([[0.0, 0.0], [1.0, 0.0]])   # creation: |1><0|
_C = _CD.T.copy()                           # annihilation: |0><1|
_PAR = np.kron(_Z2, _Z2)                    # site parity (-1)^(n_up+n_dn)
_I4 = np.eye(4)


def _own_factor(spin, dagger):
    op = _CD if dagger else _C
    if spin == 0:            # up mode is first in Jordan-Wigner order
        return np.kron(_I2, op)
    return np.kron(op, _Z2)  # dn mode: the up mode of the same site carries Z


@functools.lru_cache(maxsize=None)
def _local_op(pattern):
    """Ordered product of per-operator factors at one site.

    pattern: tuple over the term's operators in product order of
    ('o', spin, dagger) for an operator on this site, 'P' for one on a site to
    the right (Jordan-Wigner string) and 'I' for one on a site to the left.
    Returns (key, sign, matrix) with the sign normalised away, or None if zero.
    """
    m = _I4
    for f in pattern:
        if f == "P":
            m = m @ _PAR
        elif f == "I":
            continue
        else:
            m = m @ _own_factor(f[1], f[2])
    if not np.any(m):
        return None
    flat = m.ravel()
    first = flat[np.nonzero(flat)[0][0]]
    sign = 1.0 if first > 0 else -1.0
    m = m * sign
    key = tuple(np.rint(m).astype(np.int8).ravel())
    return key, sign, m


def _term_sites(ops):
    return sorted(set(p // 2 for p, _ in ops))


def _place_term(coef, ops, L, split_site, table):
    """Split one fermionic operator string into per-site local operators."""
    sites = _term_sites(ops)
    local = {}
    sign = 1.0
    nops = {}
    for k in sites:
        pat = []
        for p, d in ops:
            s = p // 2
            if s == k:
                pat.append(("o", p % 2, d))
            elif s > k:
                pat.append("P")
            else:
                pat.append("I")
        r = _local_op(tuple(pat))
        if r is None:
            return
        key, sg, m = r
        if key not in table:          # local operators are interned as small ints
            table[key] = (len(table), m)
        local[k] = table[key][0]
        sign *= sg
        nops[k] = sum(1 for p, _ in ops if p // 2 == k)
    # split site tau: at every cut left of tau the prefix holds at most two
    # operators, right of it the suffix holds at most two; within that window
    # tau is clamped to split_site so that two-operator prefixes live on the
    # left half of the chain and two-operator suffixes on the right half.
    nleft = 0
    lo, hi = sites[0], sites[-1]
    total = len(ops)
    for k in sites:
        if nleft <= 2:
            hi = k
        nleft += nops[k]
    nright = total
    for k in sites:
        nright -= nops[k]
        if nright <= 2:
            lo = k
            break
    if len(sites) == 2 and total == 2:
        lo, hi = sites[0], sites[1]
    tau = min(max(split_site, lo), hi)
    return sites, local, nops, sign * coef, tau


def chemistry_mpo(h, eri, split_site=None, tol=0.0, coeff_map=False):
    """Exact MPO (list of (R_l, 4, 4, R_r) cores) of the spin-orbital
    Hamiltonian built from spatial integrals h (L,L) and eri (L,L,L,L).

    Terms whose coefficient magnitude is <= tol are skipped (tol=0 keeps every
    nonzero term).  split_site (default L//2) is the site where two-operator
    prefixes hand over to two-operator suffixes.

    coeff_map=True also returns the linear map from the parameters to the cores:
    every core entry is an affine function of the parameters theta = (h.ravel(),
    eri.ravel()) (parameter p = i*L + j for h[i, j], L*L + ((i*L + j)*L + k)*L + l for
    eri[i, j, k, l]), W(theta) = W(0) + sum_p theta_p M_p.  The map lists the nonzero
    entries of every M_p as arrays param, site, index (flat index into the core),
    factor.  Parameters skipped by tol have no entries.
    """
    L = h.shape[0]
    if split_site is None:
        split_site = L // 2
    table = {}
    placed = []
    params = []      # (parameter index, d coefficient / d parameter) per placed term
    for i, j in itertools.product(range(L), repeat=2):
        if abs(h[i, j]) <= tol:
            continue
        for s in (0, 1):
            r = _place_term(h[i, j], [(2 * i + s, 1), (2 * j + s, 0)], L,
                            split_site, table)
            if r is not None:
                placed.append(r)
                params.append((i * L + j, r[3] / h[i, j]))
    for i, j, k, l in itertools.product(range(L), repeat=4):
        v = eri[i, j, k, l]
        if abs(v) <= tol:
            continue
        for s, t in itertools.product((0, 1), repeat=2):
            ops = [(2 * i + s, 1), (2 * k + t, 1), (2 * l + t, 0), (2 * j + s, 0)]
            r = _place_term(0.5 * v, ops, L, split_site, table)
            if r is not None:
                placed.append(r)
                params.append((L * L + ((i * L + j) * L + k) * L + l, r[3] / v))
    mats = [m for _, m in sorted(table.values(), key=lambda t: t[0])]
    return _assemble(placed, L, mats, 4, params if coeff_map else None)


def _assemble(placed, L, mats, n, params=None):
    """Build MPO cores from placed terms (sites, local keys, nops, coef, tau)."""
    # state identity at cut c (between site c-1 and site c):
    #   ('I',)  nothing placed; ('F',) term complete;
    #   ('p', content) prefix of (site, key, nops) for sites < c, unweighted;
    #   ('s', content) suffix of (site, key, nops) for sites >= c, weighted.
    states = [dict() for _ in range(L + 1)]

    def sid(c, st):
        d = states[c]
        if st not in d:
            d[st] = len(d)
        return d[st]

    # the identity channels exist at every cut they can be used on
    for c in range(L):
        sid(c, ("I",))
    for c in range(1, L + 1):
        sid(c, ("F",))
    trans = [dict() for _ in range(L)]   # site -> {(a, b): matrix}

    cmap = []        # (param, site, a, b, op, factor) of the coefficient-bearing blocks
    for ti, (sites, local, nops, coef, tau) in enumerate(placed):
        items = [(k, local[k], nops[k]) for k in sites]
        # cuts left of both the first operator and tau stay on the shared identity
        # channel I -> I, cuts right of both on F -> F: only [k0, k1] gets transitions
        k0, k1 = min(sites[0], tau), max(sites[-1], tau)

        def state_at(c):
            cnt = bisect.bisect_left(sites, c)     # operators on sites < c
            if c <= tau:
                return ("p", tuple(items[:cnt])) if cnt else ("I",)
            return ("s", tuple(items[cnt:])) if cnt < len(items) else ("F",)

        b = state_at(k0)
        for k in range(k0, k1 + 1):
            a, b = b, state_at(k + 1)
            ia, ib = sid(k, a), sid(k + 1, b)
            if k in local:
                op = mats[local[k]]
            else:   # operator-free site: identity or the Jordan-Wigner parity
                op = _PAR if sum(x[2] for x in a[1]) % 2 else _I4
            if k == tau:
                t = trans[k]
                if (ia, ib) in t:
                    t[(ia, ib)] = t[(ia, ib)] + coef * op
                else:
                    t[(ia, ib)] = coef * op
                if params is not None:
                    cmap.append((params[ti][0], k, ia, ib, op, params[ti][1]))
            else:
                trans[k][(ia, ib)] = op
    cores = []
    for k in range(L):
        Rl, Rr = len(states[k]), len(states[k + 1])
        W = np.zeros((Rl, n, n, Rr))
        if k < L and ("I",) in states[k] and ("I",) in states[k + 1]:
            W[states[k][("I",)], :, :, states[k + 1][("I",)]] = np.eye(n)
        if ("F",) in states[k] and ("F",) in states[k + 1]:
            W[states[k][("F",)], :, :, states[k + 1][("F",)]] = np.eye(n)
        for (ia, ib), m in trans[k].items():
            W[ia, :, :, ib] += m
        cores.append(W)
    # boundary: keep only the I state on the left and the F state on the right
    i0, fL = states[0][("I",)], states[L][("F",)]
    cores[0] = cores[0][i0:i0 + 1]
    cores[-1] = cores[-1][..., fL:fL + 1]
    cores = [np.ascontiguousarray(c) for c in cores]
    if params is None:
        return cores
    ps, st, ix, fa = [], [], [], []
    for p, k, ia, ib, op, d in cmap:
        if k == 0:
            assert ia == i0
            ia = 0
        if k == L - 1:
            assert ib == fL
            ib = 0
        Rr = cores[k].shape[3]
        for s_, t_ in zip(*np.nonzero(op)):
            ps.append(p)
            st.append(k)
            ix.append(((ia * n + s_) * n + t_) * Rr + ib)
            fa.append(d * op[s_, t_])
    cm = dict(param=np.array(ps, dtype=np.int64), site=np.array(st, dtype=np.int32),
              index=np.array(ix, dtype=np.int64), factor=np.array(fa, dtype=np.float64),
              nparam=L * L + L ** 4)
    return cores, cm
