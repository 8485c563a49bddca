"""Thin ctypes binding of the C ABI in include/a2dmrg.h (argument marshalling only).

Every computation runs in liba2dmrg.so (CUDA kernels for sm_103a).  Loading
fails loudly when the library is missing: there is no CPU fallback.  PyTorch
is used only for device buffers (kernel-level entry points take CUDA tensors)
and for the current CUDA stream.
"""
import ctypes
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liba2dmrg.so")

PRECISION = {"fp64": 0, "bf16": 1, "tf32": 2, "fp32": 3, "f32emu": 4, "f64emu": 5}
STATUS = {0: "A2_OK", -1: "A2_EINVAL", -2: "A2_ENOMEM", -3: "A2_ECUDA", -4: "A2_ENOCONV",
          -5: "A2_ENUMERIC", -6: "A2_ETIMEOUT", -7: "A2_EUNSUPPORTED"}


class A2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SweepOpts(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("bond_partition", ctypes.POINTER(ctypes.c_int)),
                ("D_max", ctypes.c_int), ("svd_tol", ctypes.c_double),
                ("eig_tol", ctypes.c_double), ("coarse_eps", ctypes.c_double),
                ("max_krylov", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("prec", ctypes.c_int), ("refine_f64", ctypes.c_int), ("solver", ctypes.c_int),
                ("group_streams", ctypes.c_int), ("one_site", ctypes.c_int),
                ("n_eig", ctypes.c_int), ("env_mode", ctypes.c_int),
                ("graphs", ctypes.c_int)]


class SweepReport(ctypes.Structure):
    _fields_ = [("energy_in", ctypes.c_double), ("lambda_coarse", ctypes.c_double),
                ("energy_local", ctypes.POINTER(ctypes.c_double)),
                ("coeffs", ctypes.POINTER(ctypes.c_double)),
                ("S_hat", ctypes.POINTER(ctypes.c_double)),
                ("A_hat", ctypes.POINTER(ctypes.c_double)),
                ("coarse_rank", ctypes.c_int),
                ("krylov_iters", ctypes.POINTER(ctypes.c_int)),
                ("max_discarded_weight", ctypes.c_double), ("seconds", ctypes.c_double),
                ("alg_flops", ctypes.c_double), ("matvecs", ctypes.c_longlong),
                ("coarse_dim", ctypes.c_int), ("unconverged", ctypes.c_int),
                ("matvecs_f64", ctypes.c_longlong)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run `python -m paper_2505_23429_gb300.build` "
                          "(needs nvcc; there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "a2_ctx_create": [ctypes.c_int, _P, ctypes.POINTER(_P)],
        "a2_ctx_destroy": [_P],
        "a2_ctx_synchronize": [_P],
        "a2_tt_create": [_P, ctypes.c_int, _I, _I, ctypes.c_uint64, ctypes.POINTER(_P)],
        "a2_tt_set_core": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D],
        "a2_tt_get_core": [_P, ctypes.c_int, _I, _I, _I, _D],
        "a2_tt_left_orthogonalize": [_P, _D],
        "a2_tt_destroy": [_P],
        "a2_tt_save": [_P, ctypes.c_char_p],
        "a2_tt_load": [_P, ctypes.c_char_p, ctypes.POINTER(_P)],
        "a2_mpo_load": [_P, ctypes.c_int, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_P)],
        "a2_mpo_nnz": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)],
        "a2_mpo_destroy": [_P],
        "a2_mpo_fold_split": [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D,
                              ctypes.POINTER(ctypes.c_longlong), _I],
        "a2_mpo_fold_info": [_P, ctypes.c_int, _I, ctypes.POINTER(ctypes.c_longlong)],
        "a2_mpo_set_fold": [_P, ctypes.c_int],
        "a2_heff_create": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                           _P, ctypes.POINTER(_P)],
        "a2_heff_apply_op": [_P, _P, _P],
        "a2_heff_destroy": [_P],
        "a2_set_autotune": [ctypes.c_int],
        "a2_energy_gradient": [_P, _P, _P, ctypes.c_longlong, ctypes.c_longlong,
                               ctypes.POINTER(ctypes.c_longlong), _I,
                               ctypes.POINTER(ctypes.c_longlong), _D, _D, _D],
        "a2_additive_sweep": [_P, _P, _P, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepReport)],
        "a2_classical_sweep": [_P, _P, _P, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepReport)],
        "a2_coarse_solve": [_P, ctypes.c_int, _D, _D, ctypes.c_double, _D, _D, _I],
        "a2_energy": [_P, _P, _P, ctypes.c_int, _D, _D],
        "a2_heff_apply": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          _P, _P, _P, _P],
        "a2_env_update": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P],
        "a2_svd_split": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                         ctypes.c_int, ctypes.c_double, _P, _P, _I, _D],
        "a2_gemm_bf16": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_longlong,
                         _P, ctypes.c_longlong, _P, ctypes.c_longlong, ctypes.c_int],
        "a2_device_error": [_P, ctypes.c_int, _I],
        "a2_selftest_timeout": [_P, _I],
        "a2_lq": [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P],
        "a2_profile": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _D, _D,
                       _D],
        "a2_heff_apply_noalloc": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                  _P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.a2_last_error.argtypes = [_P]
    L.a2_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points the binding expects from the library."""
    lib()
    return ["a2_ctx_create", "a2_ctx_destroy", "a2_last_error", "a2_ctx_synchronize",
            "a2_tt_create", "a2_tt_set_core", "a2_tt_get_core", "a2_tt_left_orthogonalize",
            "a2_tt_destroy", "a2_mpo_load", "a2_mpo_nnz", "a2_mpo_destroy",
            "a2_additive_sweep", "a2_classical_sweep", "a2_coarse_solve", "a2_energy",
            "a2_heff_apply", "a2_env_update", "a2_svd_split", "a2_gemm_bf16",
            "a2_device_error", "a2_profile", "a2_heff_apply_noalloc", "a2_mpo_fold_split",
            "a2_mpo_fold_info", "a2_mpo_set_fold", "a2_heff_create", "a2_heff_apply_op",
            "a2_heff_destroy", "a2_energy_gradient", "a2_set_autotune", "a2_tt_save",
            "a2_tt_load", "a2_selftest_timeout", "a2_lq"]


def _dp(a):
    return a.ctypes.data_as(_D)


def _ptr(t):
    """Device pointer of a CUDA tensor (torch) or an integer address."""
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


class Context:
    def __init__(self, device=0, stream=None):
        self._h = _P()
        self._children = []     # weak references to TT / MPO / HeffOp handles, in creation order
        st = lib().a2_ctx_create(device, _P(stream) if stream else None, ctypes.byref(self._h))
        if st != 0:
            raise A2Error(st, "a2_ctx_create failed")

    def _adopt(self, child):
        self._children.append(weakref.ref(child))

    def check(self, st):
        if st != 0:
            raise A2Error(st, lib().a2_last_error(self._h).decode())

    def synchronize(self):
        self.check(lib().a2_ctx_synchronize(self._h))

    def close(self):
        """Destroy every handle made on this context (newest first), then the context."""
        if self._h:
            for ref in reversed(self._children):
                ch = ref()
                if ch is not None:
                    ch.close()
            self._children = []
            lib().a2_ctx_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TT:
    def __init__(self, ctx, handle, phys):
        self.ctx, self._h, self.phys = ctx, handle, list(phys)
        ctx._adopt(self)

    @classmethod
    def random(cls, ctx, phys, bonds, seed):
        h = _P()
        ph = np.ascontiguousarray(phys, dtype=np.int32)
        bd = np.ascontiguousarray(bonds, dtype=np.int32)
        ctx.check(lib().a2_tt_create(ctx._h, len(ph), ph.ctypes.data_as(_I),
                                     bd.ctypes.data_as(_I), ctypes.c_uint64(seed),
                                     ctypes.byref(h)))
        return cls(ctx, h, ph)

    @classmethod
    def from_cores(cls, ctx, cores):
        phys = [c.shape[1] for c in cores]
        t = cls.random(ctx, phys, [1] * (len(cores) - 1), 1)
        for j, c in enumerate(cores):
            t.set_core(j, c)
        return t

    def set_core(self, j, core):
        a = np.ascontiguousarray(core, dtype=np.float64)
        self.ctx.check(lib().a2_tt_set_core(self._h, j, a.shape[0], a.shape[1], a.shape[2], _dp(a)))

    def core(self, j):
        dl, n, dr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.ctx.check(lib().a2_tt_get_core(self._h, j, ctypes.byref(dl), ctypes.byref(n),
                                            ctypes.byref(dr), None))
        out = np.empty((dl.value, n.value, dr.value))
        self.ctx.check(lib().a2_tt_get_core(self._h, j, None, None, None, _dp(out)))
        return out

    def cores(self):
        return [self.core(j) for j in range(len(self.phys))]

    def save(self, path):
        """Checkpoint (a2_tt_save): the TT's cores and dims to the host file `path`."""
        self.ctx.check(lib().a2_tt_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, ctx, path):
        """A new TT from a checkpoint written by save (a2_tt_load)."""
        h = _P()
        ctx.check(lib().a2_tt_load(ctx._h, os.fsencode(path), ctypes.byref(h)))
        with open(path, "rb") as f:   # the site count and physical dims of the header
            f.read(8)
            L = int(np.frombuffer(f.read(4), dtype="<i4")[0])
            phys = np.frombuffer(f.read(4 * L), dtype="<i4").tolist()
        return cls(ctx, h, phys)

    def left_orthogonalize(self):
        nrm = ctypes.c_double()
        self.ctx.check(lib().a2_tt_left_orthogonalize(self._h, ctypes.byref(nrm)))
        return nrm.value

    def close(self):
        if self._h:
            lib().a2_tt_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPO:
    def __init__(self, ctx, cores):
        self.ctx = ctx
        self.cores = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
        L = len(cores)
        phys = np.array([c.shape[1] for c in cores], dtype=np.int32)
        R = np.array([1] + [c.shape[3] for c in cores], dtype=np.int32)
        ptrs = (_D * L)(*[_dp(c) for c in self.cores])
        self._h = _P()
        ctx.check(lib().a2_mpo_load(ctx._h, L, phys.ctypes.data_as(_I), R.ctypes.data_as(_I),
                                    ptrs, ctypes.byref(self._h)))
        ctx._adopt(self)
        self.L, self.phys, self.R = L, phys, R

    def nnz(self, j):
        v = ctypes.c_longlong()
        self.ctx.check(lib().a2_mpo_nnz(self._h, j, ctypes.byref(v)))
        return v.value

    def fold_info(self, j):
        """(folded, nnz(G)) of core j (identity-on-physical block, see fold_split)."""
        f, v = ctypes.c_int(), ctypes.c_longlong()
        self.ctx.check(lib().a2_mpo_fold_info(self._h, j, ctypes.byref(f), ctypes.byref(v)))
        return bool(f.value), v.value

    def set_fold(self, enable):
        self.ctx.check(lib().a2_mpo_set_fold(self._h, 1 if enable else 0))

    def close(self):
        if self._h:
            lib().a2_mpo_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(L, P, partition, D_max, svd_tol, eig_tol, coarse_eps, max_krylov, max_restarts, prec,
          refine, solver="lanczos", sequential=False, one_site=False, n_eig=1,
          low_memory=False, graphs=False):
    o = SweepOpts()
    o.P = P
    part = None
    if partition is not None:
        part = np.ascontiguousarray(partition, dtype=np.int32)
        o.bond_partition = part.ctypes.data_as(_I)
    o.D_max, o.svd_tol, o.eig_tol, o.coarse_eps = D_max, svd_tol, eig_tol, coarse_eps
    o.max_krylov, o.max_restarts = max_krylov, max_restarts
    o.prec = PRECISION[prec]
    o.refine_f64 = refine
    o.solver = {"lanczos": 0, "davidson": 1}[solver]
    o.group_streams = 1 if sequential else 0
    o.one_site = 1 if one_site else 0
    o.n_eig = n_eig
    o.env_mode = 1 if low_memory else 0
    o.graphs = 1 if graphs else 0
    return o, part


def _sweep(fn, ctx, tt, mpo, P, partition=None, D_max=64, svd_tol=1e-10, eig_tol=1e-10,
           coarse_eps=1e-10, max_krylov=40, max_restarts=200, prec="fp64", refine=1,
           solver="lanczos", sequential=False, one_site=False, n_eig=1, low_memory=False,
           graphs=False):
    """one_site=True: the one-site case of Alg. 2 (partition over the L cores);
    n_eig = K > 1: Extension One (K eigenvectors of each group's last local problem);
    low_memory=True: the memory-limited environment mode (environments rebuilt on
    demand, none kept); graphs=True: H_eff applications replayed from CUDA graphs."""
    L = len(tt.phys)
    o, part = _opts(L, P, partition, D_max, svd_tol, eig_tol, coarse_eps, max_krylov,
                    max_restarts, prec, refine, solver, sequential, one_site, n_eig,
                    low_memory, graphs)
    m = P * max(1, n_eig) + 1
    bufs = dict(energy_local=np.zeros(m - 1), coeffs=np.zeros(m), S_hat=np.zeros(m * m),
                A_hat=np.zeros(m * m))
    kry = np.zeros(L if one_site else L - 1, dtype=np.int32)
    r = SweepReport()
    for k, v in bufs.items():
        setattr(r, k, _dp(v))
    r.krylov_iters = kry.ctypes.data_as(_I)
    ctx.check(fn(ctx._h, tt._h, mpo._h, ctypes.byref(o), ctypes.byref(r)))
    out = dict(energy_in=r.energy_in, lambda_coarse=r.lambda_coarse, coarse_rank=r.coarse_rank,
               max_discarded=r.max_discarded_weight, seconds=r.seconds, alg_flops=r.alg_flops,
               matvecs=r.matvecs, krylov=kry.tolist())
    m = r.coarse_dim
    out["coarse_dim"] = m
    out["unconverged"] = r.unconverged
    out["matvecs_f64"] = r.matvecs_f64
    out["energy_local"] = bufs["energy_local"][:m - 1]
    out["coeffs"] = bufs["coeffs"][:m]
    out["S_hat"] = bufs["S_hat"][:m * m].reshape(m, m)
    out["A_hat"] = bufs["A_hat"][:m * m].reshape(m, m)
    return out


def additive_sweep(ctx, tt, mpo, P, **kw):
    return _sweep(lib().a2_additive_sweep, ctx, tt, mpo, P, **kw)


def classical_sweep(ctx, tt, mpo, **kw):
    kw.pop("partition", None)
    return _sweep(lib().a2_classical_sweep, ctx, tt, mpo, 1, **kw)


def coarse_solve(ctx, A, S, eps=1e-10):
    A = np.ascontiguousarray(A, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    m = A.shape[0]
    c = np.zeros(m)
    lam, p = ctypes.c_double(), ctypes.c_int()
    ctx.check(lib().a2_coarse_solve(ctx._h, m, _dp(A), _dp(S), eps, _dp(c), ctypes.byref(lam),
                                    ctypes.byref(p)))
    return c, lam.value, p.value


def energy(ctx, tt, mpo, prec="fp64"):
    E, nrm = ctypes.c_double(), ctypes.c_double()
    ctx.check(lib().a2_energy(ctx._h, tt._h, mpo._h, PRECISION[prec], ctypes.byref(E),
                              ctypes.byref(nrm)))
    return E.value, nrm.value


def heff_apply(ctx, mpo, k, Lenv, Renv, x, y, prec="fp64"):
    """y = H_eff x at bond k; CUDA float64 tensors Lenv [Dl,R,Dl], Renv [Dr,R,Dr], x, y."""
    Dl, Dr = Lenv.shape[0], Renv.shape[0]
    ctx.check(lib().a2_heff_apply(ctx._h, mpo._h, k, PRECISION[prec], Dl, Dr, _ptr(Lenv),
                                  _ptr(Renv), _ptr(x), _ptr(y)))


class HeffOp:
    """H_eff at bond k with its environments converted once (a2_heff_create); apply(x, y)
    enqueues y = H_eff x on the context's stream."""
    def __init__(self, ctx, mpo, k, Lenv, Renv, prec="fp64"):
        Dl, Dr = Lenv.shape[0], Renv.shape[0]
        self.ctx, self.mpo = ctx, mpo
        self._h = _P()
        ctx.check(lib().a2_heff_create(ctx._h, mpo._h, k, PRECISION[prec], Dl, Dr,
                                       _ptr(Lenv), _ptr(Renv), ctypes.byref(self._h)))
        ctx._adopt(self)

    def apply(self, x, y):
        self.ctx.check(lib().a2_heff_apply_op(self._h, _ptr(x), _ptr(y)))

    def close(self):
        if self._h:
            lib().a2_heff_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def env_update(ctx, mpo, j, side, Hin, bra, ket, out, prec="fp64"):
    Dlb, _, Drb = bra.shape
    Dlk, _, Drk = ket.shape
    ctx.check(lib().a2_env_update(ctx._h, mpo._h, j, side, PRECISION[prec], Dlb, Drb, Dlk, Drk,
                                  _ptr(Hin), _ptr(bra), _ptr(ket), _ptr(out)))


def lq(ctx, M, L_out, Q_out):
    """M = L Q on the device (a2_lq): CUDA float64 M (rows x cols), L_out (rows x k),
    Q_out (k x cols), k = min(rows, cols)."""
    rows, cols = M.shape
    ctx.check(lib().a2_lq(ctx._h, rows, cols, _ptr(M), _ptr(L_out), _ptr(Q_out)))


def svd_split(ctx, x, D_max, tol, P_out, SQ_out):
    Dl, n1, n2, Dr = x.shape
    r, disc = ctypes.c_int(), ctypes.c_double()
    ctx.check(lib().a2_svd_split(ctx._h, Dl, n1, n2, Dr, _ptr(x), D_max, tol, _ptr(P_out),
                                 _ptr(SQ_out), ctypes.byref(r), ctypes.byref(disc)))
    return r.value, disc.value


def gemm_bf16(ctx, A, B, C, K=None, splitk=1):
    """C[m][n] = sum_k A[m][k] B[n][k] on tcgen05; A (M x lda), B (N x ldb) bf16 CUDA
    tensors whose first K columns are used; C (M x ldc) float32 CUDA tensor."""
    M, lda = A.shape
    N, ldb = B.shape
    K = lda if K is None else K
    ctx.check(lib().a2_gemm_bf16(ctx._h, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C),
                                 C.shape[1], splitk))


def last_error(ctx):
    """Message of the last failure on the context (a2_last_error)."""
    return lib().a2_last_error(ctx._h).decode()


def device_error(ctx, reset=True):
    v = ctypes.c_int()
    ctx.check(lib().a2_device_error(ctx._h, int(reset), ctypes.byref(v)))
    return v.value


def selftest_timeout(ctx):
    """Failure-path self-test of the bounded device waits (a2_selftest_timeout): returns
    (status, error code); the status is A2_ETIMEOUT (-6) when the wait ran out."""
    code = ctypes.c_int(0)
    st = lib().a2_selftest_timeout(ctx._h, ctypes.byref(code))
    return st, code.value


PROFILE_KINDS = ["tc_s1", "sparse_s2", "sparse_s3", "tc_s4", "heff_simt", "env", "lanczos",
                 "svd", "lq", "emu_s1", "emu_s2", "emu_s3", "emu_s4", "f64e_s1", "f64e_sparse",
                 "f64e_s4", "f64e_split", "heff_graph"]


def profile(ctx, op, kind=0):
    """op: 'off', 'on', 'reset' or 'read' (returns dict for `kind`)."""
    code = {"off": 0, "on": 1, "reset": 2, "read": 3, "launches": 4}[op]
    n, ms, fl, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ctx.check(lib().a2_profile(ctx._h, code, kind, ctypes.byref(n), ctypes.byref(ms),
                               ctypes.byref(fl), ctypes.byref(by)))
    if code == 3:
        return dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)
    if code == 4:
        return n.value
    return None


def heff_apply_noalloc(ctx, mpo, k, Lenv, Renv, x, y):
    """Same as heff_apply(..., prec="fp64") but with no device allocation: the
    intermediates live in a fixed 32 MiB array inside the library (for callers
    that cannot allocate while they run).  Larger problems raise A2Error."""
    Dl, Dr = Lenv.shape[0], Renv.shape[0]
    ctx.check(lib().a2_heff_apply_noalloc(ctx._h, mpo._h, k, Dl, Dr, _ptr(Lenv), _ptr(Renv),
                                          _ptr(x), _ptr(y)))


def fold_split(W):
    """Identity-on-physical split of a core W[wl][s][t][wr] (host only): returns
    (G, nnz(G), foldable) with W = delta_st G + W_rest."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    Rl, n, _, Rr = W.shape
    G = np.zeros((Rl, Rr))
    nz, f = ctypes.c_longlong(), ctypes.c_int()
    st = lib().a2_mpo_fold_split(_dp(W), Rl, n, Rr, _dp(G), ctypes.byref(nz), ctypes.byref(f))
    if st != 0:
        raise A2Error(st, "a2_mpo_fold_split failed")
    return G, nz.value, bool(f.value)


def energy_gradient(ctx, tt, mpo, cmap):
    """(E, dE/dtheta) at the fixed TT for an MPO built with a coefficient map
    (synthetic.chemistry_mpo(..., coeff_map=True)): cmap holds param, site, index,
    factor arrays and nparam."""
    p = np.ascontiguousarray(cmap["param"], dtype=np.int64)
    st = np.ascontiguousarray(cmap["site"], dtype=np.int32)
    ix = np.ascontiguousarray(cmap["index"], dtype=np.int64)
    fa = np.ascontiguousarray(cmap["factor"], dtype=np.float64)
    nparam = int(cmap["nparam"])
    grad = np.zeros(nparam)
    E = ctypes.c_double()
    LL = ctypes.POINTER(ctypes.c_longlong)
    ctx.check(lib().a2_energy_gradient(ctx._h, tt._h, mpo._h, nparam, len(p),
                                       p.ctypes.data_as(LL), st.ctypes.data_as(_I),
                                       ix.ctypes.data_as(LL), _dp(fa), _dp(grad),
                                       ctypes.byref(E)))
    return E.value, grad


def energy_autograd(h, eri, ctx, tt, mpo, cmap):
    """Energy of the fixed TT as a differentiable function of the one- and two-body
    coefficients (torch tensors h [L, L], eri [L, L, L, L]); the MPO must have been built
    from the same values.  Backward returns dE/dh, dE/deri (Hellmann-Feynman at the TT)."""
    import torch

    class _Energy(torch.autograd.Function):
        @staticmethod
        def forward(fctx, h_, eri_):
            E, g = energy_gradient(ctx, tt, mpo, cmap)
            L = h_.shape[0]
            fctx.save_for_backward(torch.from_numpy(g[: L * L].reshape(L, L)).to(h_),
                                   torch.from_numpy(g[L * L:].reshape(L, L, L, L)).to(eri_))
            return torch.tensor(E, dtype=torch.float64, device=h_.device)

        @staticmethod
        def backward(fctx, gE):
            gh, geri = fctx.saved_tensors
            return gE * gh, gE * geri

    return _Energy.apply(h, eri)


def set_autotune(enable, sparse=False):
    """Enable / disable the tcgen05 GEMM autotuner (on by default) and, with sparse=True,
    the sparse-stage autotuner (off by default); library-wide."""
    lib().a2_set_autotune((1 if enable else 0) | (2 if sparse else 0))
