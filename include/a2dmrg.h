/* a2dmrg.h -- C ABI of the GB300 (sm_103a) two-site A2DMRG library.
 *
 * The library computes the lowest eigenpair of a symmetric operator A given as
 * a matrix product operator (eq. MPO, App. A) over tensor trains (Def. TT
 * parameter space, Sec. 2.1), by the additive two-level DMRG iteration
 * (Alg. 2) with the coarse-space correction of Sec. 3.1.
 *
 * Conventions (all functions):
 *  - Every function returns a2_status: A2_OK (0) or a negative error code; no
 *    exception crosses the ABI.  a2_last_error() returns the message of the
 *    last failure on a context (valid until the next call on that context).
 *  - Handles (a2_ctx, a2_tt, a2_mpo, a2_heff) are opaque and owned by the library;
 *    create/destroy them with the functions below.  A context is used by one
 *    host thread at a time; all its work is ordered on its CUDA stream.
 *    a2_ctx_destroy also destroys the TT / MPO / H_eff handles still made on that
 *    context; a destroy call on a handle that is no longer live returns A2_EINVAL and
 *    does nothing.
 *  - "host" pointers are read or written synchronously and may be freed after
 *    the call returns.  "device" pointers are CUDA device addresses on the
 *    context's device; the call enqueues work on the context stream and the
 *    caller must keep the buffers alive until that stream has completed the
 *    work (a2_ctx_synchronize).
 *  - Arrays are row-major.  TT core j: [D_{j}][n_j][D_{j+1}] float64 with
 *    D_0 = D_L = 1.  MPO core j: [R_j][n_j][n_j][R_{j+1}] float64, index order
 *    (left bond, bra/output s, ket/input t, right bond), R_0 = R_L = 1.
 *    Environments: [bra bond][MPO bond][ket bond] (eqs. env_L / env_R).
 *  - On error the TT handed to a sweep is left unchanged (the iterate of
 *    Alg. 2 is kept until the global iteration succeeds).
 */
#ifndef A2DMRG_H
#define A2DMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  A2_OK = 0,
  A2_EINVAL = -1,       /* invalid argument (sizes, null pointers, mismatched dims) */
  A2_ENOMEM = -2,       /* device allocation failed */
  A2_ECUDA = -3,        /* CUDA runtime error (or a factorisation kernel's bounded grid
                           barrier gave up) */
  A2_ENOCONV = -4,      /* an iterative solve did not reach its tolerance */
  A2_ENUMERIC = -5,     /* non-finite value detected */
  A2_ETIMEOUT = -6,     /* a bounded device-side wait gave up */
  A2_EUNSUPPORTED = -7  /* option not supported by this build */
} a2_status;

typedef enum {
  A2_FP64 = 0, /* every contraction in FP64 */
  A2_BF16 = 1, /* Lanczos on tcgen05 tensor cores with BF16 operands to a residual of
                  3e-3, then continued with the A2_F32EMU products to eig_tol, then (with
                  refine_f64) the FP64 refinement of the Ritz pair; environments FP64,
                  computed to FP64-class accuracy on the tensor cores as in A2_F64EMU;
                  coarse matrices, vectors, SVD and coarse eigensolve in FP64 */
  A2_TF32 = 2, /* reserved */
  A2_FP32 = 3, /* every contraction in FP32 (SIMT), vectors / SVD / coarse in FP64 */
  A2_F32EMU = 4, /* H_eff on tcgen05 with FP32-accurate products: operands split into
                   three BF16 slices, six slice pairs accumulated in FP32; environments,
                   refinement and coarse problem as in A2_BF16 */
  A2_F64EMU = 5  /* H_eff to FP64-class accuracy (~2^-48) on tcgen05 (Ozaki scheme): FP64
                   operands split row-wise into eight 7-bit BF16 slices, the 36 slice
                   pairs of level <= 9 accumulated exactly in FP32 per level and K chunk,
                   the partial tiles summed by error-free two-sums into FP32 pairs; the
                   sparse MPO stages in double-float (FP32 pairs); environments FP64,
                   their updates emulated the same way (two Ozaki GEMMs and a double-float
                   sparse stage) above a small size, plain FP64 below; vectors, SVD and
                   coarse problem in FP64 */
} a2_precision;

typedef struct a2_ctx a2_ctx;
typedef struct a2_tt a2_tt;
typedef struct a2_mpo a2_mpo;

/* Context on CUDA device `device`.  cuda_stream: a cudaStream_t to run on, or
 * NULL to create a private non-blocking stream. */
a2_status a2_ctx_create(int device, void* cuda_stream, a2_ctx** out);
a2_status a2_ctx_destroy(a2_ctx* ctx);
const char* a2_last_error(const a2_ctx* ctx);
a2_status a2_ctx_synchronize(a2_ctx* ctx);

/* ---- tensor trains (Def. TT parameter space; Def. orthogonal TT) ---------- */

/* New TT with L sites, physical dims phys[L] and bond dims bonds[L-1] (each
 * clipped to the exact maximal rank min(prod n_<=k, prod n_>k)).  Cores are
 * filled with SplitMix64 uniforms on [-1,1) (53-bit mantissa, site by site in
 * row-major order, one stream from `seed`); then the TT is left-orthogonalised
 * (QR, diag(R) >= 0) and normalised to norm 1. */
a2_status a2_tt_create(a2_ctx* ctx, int L, const int* phys, const int* bonds, uint64_t seed,
                       a2_tt** out);
/* Copy a host core into site `site`; its bond dims must match the neighbours'
 * after all cores are set (checked when the TT is used). */
a2_status a2_tt_set_core(a2_tt* tt, int site, int Dl, int n, int Dr, const double* host_core);
/* Query dims (host_out NULL) or copy core `site` to host. */
a2_status a2_tt_get_core(const a2_tt* tt, int site, int* Dl, int* n, int* Dr, double* host_out);
/* QR sweep left to right (diag(R) >= 0), then scale to norm 1; *norm_out
 * (host, may be NULL) receives the norm before scaling. */
a2_status a2_tt_left_orthogonalize(a2_tt* tt, double* norm_out);
a2_status a2_tt_destroy(a2_tt* tt);

/* Checkpoint of the state between global iterations (Alg. 2 keeps exactly the
 * left-orthogonal TT U^(n),d): a2_tt_save writes the TT to the file `path` (host path,
 * replaced if it exists) as little-endian raw data: the 8 bytes "A2TTCKP1", int32 L,
 * int32 phys[L], int32 bonds[L+1] (bonds[0] = bonds[L] = 1), then every core as FP64
 * [Dl][n][Dr] row-major, site 0 first.  a2_tt_load reads such a file into a new TT of
 * the context (the caller owns it; a2_tt_destroy).  Errors: A2_EINVAL (NULL arguments,
 * unreadable / unwritable file, wrong magic, inconsistent or truncated contents, bond
 * dims that do not chain), A2_ECUDA.  Resuming from the file repeats the iteration that
 * follows the save, to the reproducibility of the precision (split-K tiles are added
 * with atomics, so bitwise equality is not promised). */
a2_status a2_tt_save(const a2_tt* tt, const char* path);
a2_status a2_tt_load(a2_ctx* ctx, const char* path, a2_tt** out);

/* ---- matrix product operator (eq. MPO) ------------------------------------ */

/* Load L cores (host pointers) with MPO bond dims mpo_bonds[L+1] (first and
 * last are 1).  The dense cores are scanned once into sparse row lists for
 * the left-to-right and right-to-left actions (exact zeros are skipped). */
a2_status a2_mpo_load(a2_ctx* ctx, int L, const int* phys, const int* mpo_bonds,
                      const double* const* cores, a2_mpo** out);
/* Number of nonzeros of core `site` (for flop accounting). */
a2_status a2_mpo_nnz(const a2_mpo* mpo, int site, long long* nnz_out);
a2_status a2_mpo_destroy(a2_mpo* mpo);

/* Identity-on-physical split of a core (a regrouping of the App. A contraction, not a
 * step of the paper): W[wl][s][t][wr] = delta_st G[wl][wr] + W_rest[wl][s][t][wr] with
 * G[wl][wr] = W[wl][s][s][wr] where all n diagonal entries are equal and nonzero, else
 * 0.  Host only (no device, no context): W is a host array [Rl][n][n][Rr], G_out
 * (host, Rl*Rr, may be NULL) receives G row-major, *nnz_g its nonzero count,
 * *foldable whether a2_mpo_load marks such a core for folding (the H_eff
 * applications of the BF16 / split-precision paths then contract G into the
 * environments once per local problem and keep only W_rest sparse).  A2_EINVAL on
 * NULL W / outputs or non-positive sizes. */
a2_status a2_mpo_fold_split(const double* W, int Rl, int n, int Rr, double* G_out,
                            long long* nnz_g, int* foldable);
/* Whether core `site` of a loaded MPO is folded (*foldable) and nnz(G) (*nnz_g). */
a2_status a2_mpo_fold_info(const a2_mpo* mpo, int site, int* foldable, long long* nnz_g);
/* Enable (1, default) or disable (0) folding for every foldable core of the MPO; the
 * results agree up to rounding either way.  Not thread-safe against running sweeps. */
a2_status a2_mpo_set_fold(a2_mpo* mpo, int enable);

/* ---- one global iteration -------------------------------------------------- */

typedef struct {
  int P;                       /* number of groups of bonds (subdomains), 1..L-1 (groups
                                  of cores, 1..L, with one_site) */
  const int* bond_partition;   /* P group sizes summing to L-1 (L with one_site) (host), or
                                  NULL = even split */
  int D_max;                   /* rank cap of the truncated SVD steps and the compression */
  double svd_tol;              /* keep smallest r with discarded 2-norm <= svd_tol*||sigma|| */
  double eig_tol;              /* Lanczos: ||H x - theta x|| <= eig_tol*max(1,|theta|) */
  double coarse_eps;           /* drop S_hat eigenvalues <= coarse_eps * max (Sec. 3.1) */
  int max_krylov;              /* Krylov basis size before a restart (<= 64) */
  int max_restarts;            /* restart cycles per local solve */
  a2_precision prec;
  int refine_f64;              /* A2_BF16 / A2_F32EMU, two-site local problems: 1 = FP64
                                  refinement of every local Ritz pair after the tensor-core
                                  phases (the spec precision split): Lanczos continued
                                  from the Ritz vector on the FP64-class (A2_F64EMU)
                                  operator, whose first application gives the FP64 Rayleigh
                                  quotient and residual, until that residual meets eig_tol;
                                  the reported local energies are then FP64 Rayleigh
                                  quotients.  0 = none.  Ignored by the other precisions,
                                  the one-site case and Extension One's further
                                  eigenvectors. */
  int solver;                  /* local eigensolver: 0 = restarted Lanczos (as in the
                                  paper's experiments), 1 = Davidson with the diagonal
                                  preconditioner (same stopping rule, fewer matvecs) */
  int group_streams;           /* 0 = the P groups run concurrently (one host thread and
                                  CUDA stream each), 1 = one after another */
  int one_site;                /* 0 = two-site A2DMRG (groups of bonds, partition sums to
                                  L-1); 1 = the one-site case of Alg. 2: P groups of cores
                                  (partition sums to L), one-site micro-steps with QR between
                                  the cores of a group, no rank change in the local steps,
                                  compression of the rank-2r structured sum; the local
                                  contractions run on the SIMT path for A2_FP64 / A2_FP32
                                  and on the tensor cores with FP32-accurate products for
                                  A2_BF16 / A2_F32EMU; krylov_iters then has L entries */
  int n_eig;                   /* K: 0 or 1 = one eigenvector per local problem; K > 1 =
                                  Extension One (extension remark after Alg. 2): the last
                                  local problem of every group keeps its K lowest
                                  eigenvectors (the lowest by the usual solve, the others by
                                  Lanczos on the operator deflated by those found), each
                                  giving one updated TT (two-site: its own truncated SVD),
                                  so the coarse space has up to K*P + 1 <= 63 vectors and
                                  the compression rounds their block-diagonal sum.  Not
                                  allowed in a2_classical_sweep. */
  int env_mode;                /* 0 = every environment built once per iteration and kept
                                  (storage O(d r^2 R)); 1 = memory-limited mode (the
                                  paper's cost discussion of the micro-iterations): no
                                  environment is kept, each local problem and each coarse
                                  entry rebuilds the two it needs from the chain ends
                                  (storage O(r^2 R), O(d) more environment updates);
                                  results agree to the rounding of the precision */
  int graphs;                  /* 1: every local operator's H_eff application is captured
                                  once into a CUDA graph (after one eager application) and
                                  replayed by the eigensolver, one launch per application;
                                  results are those of the eager path.  The profiler then
                                  books replayed applications as a whole (kind 17). */
} a2_sweep_opts;

typedef struct {
  double energy_in;            /* Rayleigh quotient of the input iterate (A_hat_00/S_hat_00) */
  double lambda_coarse;        /* lowest eigenvalue of the coarse problem */
  double* energy_local;        /* [m-1] caller-owned or NULL: last Ritz value of each group
                                  (with n_eig > 1: the group's eigenvalues, ascending, group
                                  after group) */
  double* coeffs;              /* [m] caller-owned or NULL: coarse coefficients c */
  double* S_hat;               /* [m*m] caller-owned or NULL */
  double* A_hat;               /* [m*m] caller-owned or NULL; m = P + 1, or up to
                                  n_eig*P + 1 with n_eig > 1 (size the arrays for that) */
  int coarse_rank;             /* p, numerical rank of S_hat */
  int* krylov_iters;           /* [L-1] ([L] one-site) caller-owned or NULL: matvecs per
                                  bond (per core) */
  double max_discarded_weight; /* largest discarded 2-norm over the SVD steps */
  double seconds;              /* wall time of the call */
  double alg_flops;            /* algorithmic flops of the contractions performed */
  long long matvecs;           /* H_eff applications in the call */
  int coarse_dim;              /* m, the number of coarse basis vectors used */
  int unconverged;             /* local eigensolves that stopped with the residual still
                                  above eig_tol -- after max_restarts cycles, or (Davidson)
                                  when the preconditioned residual adds no new direction to
                                  the search space: their last Ritz pair is accepted (the
                                  coarse step and the compression use it) and counted here.
                                  A Lanczos breakdown (invariant Krylov space: the Ritz
                                  pair is exact) counts as converged. */
  long long matvecs_f64;       /* of `matvecs`: the FP64-class (Ozaki-emulated) H_eff
                                  applications, e.g. those of the refine_f64 step */
} a2_sweep_report;

/* One global iteration of two-site A2DMRG (Alg. 2, with P groups of adjoining
 * bonds swept as in Alg. 1 inside each group; the one-site case, Extension One and the
 * memory-limited mode through the options).  In: left-orthogonal TT of norm 1
 * (U^(n),d).  Out (in place): the compressed left-orthogonal TT of norm 1 (U^(n+1),d);
 * on any error the input TT is restored.  report may be NULL. */
a2_status a2_additive_sweep(a2_ctx* ctx, a2_tt* tt, const a2_mpo* mpo, const a2_sweep_opts* opts,
                            a2_sweep_report* report);

/* One left-to-right half-sweep of classical two-site DMRG (Alg. 1 step 1-2 for
 * i = 1..d-1) on the same kernels, preceded by the right-to-left LQ sweep that
 * supplies the right-orthogonal input.  Output: left-orthogonal TT, norm 1. */
a2_status a2_classical_sweep(a2_ctx* ctx, a2_tt* tt, const a2_mpo* mpo,
                             const a2_sweep_opts* opts, a2_sweep_report* report);

/* Coarse problem of Sec. 3.1 alone (eq. aux_eig_final_sym) on the device:
 * host A_hat, S_hat (m x m symmetric, m <= 63), eps; outputs (host) c[m]
 * with c^T S c = 1 and c_0 >= 0, lambda, and the kept rank p. */
a2_status a2_coarse_solve(a2_ctx* ctx, int m, const double* A_hat, const double* S_hat,
                          double eps, double* c_out, double* lambda_out, int* rank_out);

/* Rayleigh quotient E = <x, A x>/<x, x> (eq. energy_eig) of the TT, contracted
 * with precision prec; norm_out = ||x|| (both host, norm_out may be NULL). */
a2_status a2_energy(a2_ctx* ctx, const a2_tt* tt, const a2_mpo* mpo, a2_precision prec,
                    double* E_out, double* norm_out);

/* ---- gradients with respect to the Hamiltonian's parameters --------------- */

/* dE/dtheta of E(theta) = <x, A(theta) x>/<x, x> at the fixed TT x (Hellmann-Feynman:
 * at a converged iterate this is the total derivative of the ground energy), for an MPO
 * whose cores are affine in the parameters, W_j(theta) = W_j(0) + sum_p theta_p M_p,j.
 * The map lists the nonzero entries of every M_p,j: entry e says that core
 * map_site[e] (flat index map_index[e] into its [R_l][n][n][R_r] array) has
 * dW/dtheta_{map_param[e]} = map_factor[e] (host arrays of length nmap, copied).
 * The adjoint of the sandwich, G_j = dE/dW_j (App. A contraction with core j taken out:
 * left environment, core j as bra and ket, right environment), is formed for every
 * core that the map touches, in FP64 on the device, and contracted with the map;
 * grad_out (host, nparam) receives dE/dtheta, E_out (host, may be NULL) the energy.
 * Not a step of the paper's method (the gradient configuration of the benchmark).
 * Errors: A2_EINVAL on NULL / out-of-range map entries or mismatched handles. */
a2_status a2_energy_gradient(a2_ctx* ctx, const a2_tt* tt, const a2_mpo* mpo, long long nparam,
                             long long nmap, const long long* map_param, const int* map_site,
                             const long long* map_index, const double* map_factor,
                             double* grad_out, double* E_out);

/* Library-wide autotuners, `enable` a bit set: bit 0 (1) the tcgen05 GEMM autotuner (on
 * by default), bit 1 (2) the sparse-stage autotuner (off by default).  When on, the first
 * GEMM of every shape class times the candidate kernel variants / K splits, and the
 * first sparse launch of every shape the candidate rows per thread block, on the caller's
 * stream (synchronising it once), and keeps the fastest; switching one off forgets its
 * choices and uses the built-in heuristics.  (The sparse classes are per bond, so their
 * trials cost more than they gain within a few iterations.)  Always A2_OK. */
a2_status a2_set_autotune(int enable);

/* ---- kernel-level entry points (device pointers, FP64 in/out) ------------- */

/* y = H_eff x for the two-site problem at bond k (sites k, k+1), the
 * contraction of App. A with the two-site modification:
 *   y[a,s1,s2,b] = sum L[a,w,a'] A_k[w,s1,t1,w1] A_k+1[w1,s2,t2,w2] R[b,w2,b'] x[a',t1,t2,b']
 * L: [Dl][R_k][Dl], R: [Dr][R_{k+2}][Dr], x, y: [Dl][n_k][n_k+1][Dr] (device). */
a2_status a2_heff_apply(a2_ctx* ctx, const a2_mpo* mpo, int k, a2_precision prec, int Dl, int Dr,
                        const double* L, const double* R, const double* x, double* y);

/* The same operator as a handle whose environments are copied / converted once (as
 * inside a local solve of Alg. 2 step 2, where H^L and H^R stay fixed while Lanczos
 * applies H_eff many times): a2_heff_create copies L, R (device, FP64, layouts as
 * above; the caller may free them afterwards) into the precision's working form
 * (FP64, FP32, BF16 or split BF16 planes, with the identity-block fold of
 * a2_mpo_fold_split); a2_heff_apply_op(x, y) then enqueues y = H_eff x on the
 * context's stream (device x, y as above; asynchronous: a2_synchronize before y is
 * read elsewhere).  The handle references the context and the MPO (both must
 * outlive it) and uses the context's scratch: one application at a time per context.
 * Errors: A2_EINVAL on bad sizes / NULLs, A2_ECUDA on CUDA failure. */
typedef struct a2_heff a2_heff;
a2_status a2_heff_create(a2_ctx* ctx, const a2_mpo* mpo, int k, a2_precision prec, int Dl,
                         int Dr, const double* L, const double* R, a2_heff** out);
a2_status a2_heff_apply_op(a2_heff* op, const double* x, double* y);
a2_status a2_heff_destroy(a2_heff* op);

/* Environment update at site j (eqs. env_L / env_R and the update of App. A):
 * side 0 (left):  out[b,w',b'] = sum bra[a,s,b] in[a,w,a'] A_j[w,s,t,w'] ket[a',t,b'],
 *                 in [Dlb][R_j][Dlk], out [Drb][R_j+1][Drk];
 * side 1 (right): out[a,w,a'] = sum bra[a,s,b] A_j[w,s,t,w'] in[b,w',b'] ket[a',t,b'],
 *                 in [Drb][R_j+1][Drk], out [Dlb][R_j][Dlk].
 * bra: [Dlb][n][Drb], ket: [Dlk][n][Drk] (device). */
a2_status a2_env_update(a2_ctx* ctx, const a2_mpo* mpo, int j, int side, a2_precision prec,
                        int Dlb, int Drb, int Dlk, int Drk, const double* in, const double* bra,
                        const double* ket, double* out);

/* Truncated SVD step of Alg. 1 (two-site): x [Dl][n1][n2][Dr] (device) viewed as
 * a (Dl n1) x (n2 Dr) matrix = P Sigma Q; keeps the smallest rank r <= D_max
 * with discarded 2-norm <= tol*||sigma||.  P_out [Dl][n1][r] (left-orthonormal),
 * SQ_out [r][n2][Dr] (device, capacity min(Dl n1, n2 Dr) columns/rows);
 * rank_out, discarded_out (host).  Computed by this library's FP64 kernels: Householder
 * bidiagonalisation, all singular values by bisection of the Golub-Kahan tridiagonal
 * (FP32 brackets refined in FP64 to a relative width 2^-40; no Gram matrix, so small
 * singular values keep their relative accuracy), the kept left vectors by inverse
 * iteration, re-orthonormalised (block Gram-Schmidt with CholeskyQR2 panels) and
 * transformed back; SQ = P^T x.  Within an exactly degenerate multiplet any orthonormal
 * basis may be returned; FP64 atomic sums in the bidiagonalisation may change the last
 * bits of the result from run to run.  Errors: A2_EINVAL on bad sizes / NULLs (more than
 * 12800 rows Dl n1 or, for the smaller of the two dimensions, more than 2400), A2_ECUDA
 * on CUDA failure (including a bounded grid barrier that gave up). */
a2_status a2_svd_split(a2_ctx* ctx, int Dl, int n1, int n2, int Dr, const double* x, int D_max,
                       double tol, double* P_out, double* SQ_out, int* rank_out,
                       double* discarded_out);

/* LQ factorisation of Alg. 2 step 1 (W_i = L_i Q_i, and of the TT rounding) alone:
 * M (device, rows x cols row-major, not modified) = L Q with Q (device, k x cols,
 * k = min(rows, cols)) orthonormal rows and L (device, rows x k) lower trapezoidal with
 * diag(L) >= 0; Householder reflections in FP64 on the device (this library's kernel:
 * the owner of row i + 1 publishes reflection i + 1 on a ready flag that the other blocks
 * wait for).  Synchronous.  Errors: A2_EINVAL on bad sizes / NULLs (rows of more than
 * 25600 entries), A2_ECUDA if a bounded wait of the kernel gave up. */
a2_status a2_lq(a2_ctx* ctx, int rows, int cols, const double* M, double* L, double* Q);

/* Stages S1 and S4 of the H_eff chain alone: the tcgen05 tensor-core GEMM
 *   C[m][n] = sum_k A[m][k] B[n][k],  A: M x K (row stride lda), B: N x K (row
 *   stride ldb), BF16 (device, 16-byte aligned, strides multiples of 8 elements),
 *   C: M x N FP32 (device, row stride ldc).  splitk > 1 splits K across CTAs and
 *   accumulates atomically (C is zeroed first).  Synchronous. */
a2_status a2_gemm_bf16(a2_ctx* ctx, int M, int N, int K, const void* A, long long lda,
                       const void* B, long long ldb, float* C, long long ldc, int splitk);

/* Device-side error code of the bounded waits (0 = none): the tensor-core kernels' mbarrier
 * waits (codes 1-16), or 101 when a bounded wait of a factorisation kernel (grid barrier
 * or ready flag) gave up; reset != 0
 * clears it.  Synchronizes the context stream. */
a2_status a2_device_error(a2_ctx* ctx, int reset, int* code_out);

/* Failure-path self-test of the bounded device waits (not paper content): runs one tile
 * of the tcgen05 GEMM kernel whose producer role issues no copies, with a wait limit of
 * 2^14 iterations, on the context stream, and waits for it.  The MMA role's first wait
 * can never complete; it gives up, raises the device error word and the abort flag, the
 * other roles leave, no copy or MMA is in flight and tensor memory is freed.  Returns
 * A2_ETIMEOUT with *code_out (host) = the error code that was raised, after clearing the
 * error word, and the context stays usable.  A2_EINVAL when the error word is already set
 * before the call (read it with a2_device_error first), A2_ECUDA if the wait did not run
 * out. */
a2_status a2_selftest_timeout(a2_ctx* ctx, int* code_out);

/* Live kernel timing with CUDA events on the context stream (not paper content;
 * used to report achieved throughput per kernel class).  op: 0 = disable,
 * 1 = enable, 2 = reset totals, 3 = read the totals of `kind` (0 tcgen05 S1,
 * 1 sparse S2, 2 sparse S3, 3 tcgen05 S4, 4 SIMT H_eff, 5 environment update,
 * 6 Lanczos vector work, 7 truncated SVD, 8 LQ/QR, 9-12 the four stages of the
 * FP32-accurate split-product H_eff, 13-16 the FP64-emulated H_eff: S1, the sparse
 * stages, S4, the operand slicing, 17 H_eff applications replayed from CUDA graphs)
 * into the host outputs
 * (launches, milliseconds, algorithmic flops, algorithmic bytes; any may be NULL).
 * op 4 returns in *launches the number of kernel launches this library has made
 * since the process started (all of its own kernels, library calls excluded). */
a2_status a2_profile(a2_ctx* ctx, int op, int kind, long long* launches, double* ms,
                     double* flops, double* bytes);

/* Allocation-free variant of a2_heff_apply (FP64 contraction only).  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate device
 * memory while they run -- for example applications whose GPU memory belongs to
 * their own pool or fixed budget, or loops that must not stall on an allocator.
 * It takes the same arguments as a2_heff_apply (minus the precision) and computes
 * the same y, but all of its intermediate tensors live in one fixed device array
 * built into the library (4 Mi doubles = 32 MiB, reserved on every GPU that loads
 * the library until the process exits).  It never calls cudaMalloc or cudaFree.
 *  - Size limit: the intermediates need max(s1, s3) + s2 doubles with
 *    s1 = Dl*R_k*n_k*n_k+1*Dr, s2 = Dl*R_k+1*n_k*n_k+1*Dr, s3 = Dl*n_k*n_k+1*R_k+2*Dr
 *    (R_j = MPO bond j); anything above 4 Mi doubles is rejected with A2_EINVAL and
 *    a message naming both numbers.
 *  - The first call on a device looks up the device address of the array (this can
 *    load the library's device code); make that first call before any CUDA stream
 *    capture.
 *  - Every call shares the one array and leaves its contents behind; each call
 *    overwrites everything it reads.  Calls whose work overlaps on the GPU (other
 *    streams, other contexts on the same device) race on the array: order them.
 *  - y is overwritten (zeroed first when the last stage splits its reduction).
 *  - The device address of the array is looked up once per device and kept for the life
 *    of the library: do not reset a device (cudaDeviceReset) while the library is loaded
 *    and still in use on it. */
a2_status a2_heff_apply_noalloc(a2_ctx* ctx, const a2_mpo* mpo, int k, int Dl, int Dr,
                                const double* L, const double* R, const double* x, double* y);

#ifdef __cplusplus
}
#endif

#endif /* A2DMRG_H */
