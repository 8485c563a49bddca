// Device kernels of the A2DMRG hot path (declarations).
#pragma once
#include "common.cuh"

namespace a2 {

// C(m,n) {=, +=, atomic +=} alpha * sum_k A(m,k) B(n,k), general strides:
//   A(m,k) = A[m*sam + k*sak], B(n,k) = B[n*sbn + k*sbk], C(m,n) = C[m*scm + n*scn]
// batched over `batch` with element strides abs/bbs/cbs, optional split-K
// (splitk > 1 requires mode == GEMM_ATOMIC and a zeroed C).
enum GemmMode { GEMM_STORE = 0, GEMM_ADD = 1, GEMM_ATOMIC = 2 };

template <typename T, typename OutT>
struct SimtGemm {
  int M = 0, N = 0, K = 0;
  const T* A = nullptr; long long sam = 0, sak = 1;
  const T* B = nullptr; long long sbn = 0, sbk = 1;
  OutT* C = nullptr; long long scm = 0, scn = 1;
  int batch = 1; long long abs = 0, bbs = 0, cbs = 0;
  int splitk = 1;
  T alpha = T(1);
  int mode = GEMM_STORE;
};

template <typename T, typename OutT>
void simt_gemm(const SimtGemm<T, OutT>& g, cudaStream_t s);

// Sparse action of one MPO core on rows of a dense tensor:
//   out[ob + ro(r)][v] = sum_{nz in row r} val[nz] * in[ib + ci(nz)][v],  v < veclen
// row r carries two indices (rw, rs): ro = rw*out_sw + rs*out_ss;
// nonzero carries (cw, ct):           ci = cw*in_sw + ct*in_st;
// batch (b1 < B1, b2 < B2): ib = b1*in_b1 + b2*in_b2, ob = b1*out_b1 + b2*out_b2.
template <typename V>
struct SparseRows {
  int nrows = 0;
  const int* row_ptr = nullptr;     // nrows + 1
  const int* row_w = nullptr;       // nrows
  const int* row_s = nullptr;       // nrows
  const int* nz_w = nullptr;        // nnz
  const int* nz_t = nullptr;        // nnz
  const V* nz_val = nullptr;        // nnz
  long long nnz_total = 0;
  const float* nz_lo = nullptr;     // nnz: FP64 value - (float)value (double-float kernels)
};

struct SparseGeom {
  int veclen = 0;
  int accumulate = 0;               // 1: out += result (read in the output's type)
  long long out_sw = 0, out_ss = 0, in_sw = 0, in_st = 0;
  int B1 = 1, B2 = 1;
  long long in_b1 = 0, in_b2 = 0, out_b1 = 0, out_b2 = 0;
};

template <typename TI, typename TO, typename V>
void sparse_rows_apply(const SparseRows<V>& sp, const SparseGeom& g, const TI* in, TO* out,
                       cudaStream_t s);

// Same action with the FP32 result written as three BF16 planes (hi, mid, lo) at
// out, out + plane, out + 2*plane.  in_plane > 0 (BF16 input only): the input is itself
// three planes in, in + in_plane, in + 2*in_plane and each value is their sum.  add
// (optional, FP32, laid out like one output plane) is added to the result before the
// split.  g.accumulate is ignored.
template <typename TI, typename V>
void sparse_rows_apply_split3(const SparseRows<V>& sp, const SparseGeom& g, const TI* in,
                              long long in_plane, const float* add, __nv_bfloat16* out,
                              long long plane, cudaStream_t s);
// out planes [p][r*ld + c] = BF16 slice p of in[r*cols + c]  (x = hi + mid + lo)
template <typename TI>
void split3_ld(const TI* in, long long rows, long long cols, __nv_bfloat16* out, long long ld,
               long long plane, cudaStream_t s);
// out planes [p][c*ld + r] = BF16 slice p of in[r*cols + c]  (transpose and split)
template <typename TI>
void transpose_split3(const TI* in, int rows, int cols, __nv_bfloat16* out, long long ld,
                      long long plane, cudaStream_t s);

// ---- permutes and conversions
// out[(i*d1 + j)*d2 + k] = in[(j*d0 + i)*d2 + k]   (swap the two outer dims, k contiguous)
template <typename TI, typename TO>
void permute_swap01(const TI* in, TO* out, int d0, int d1, int d2, cudaStream_t s);
template <typename TI, typename TO>
void convert(const TI* in, TO* out, long long n, cudaStream_t s);
// 2D transpose of a (rows x cols) row-major matrix: out (cols x rows)
template <typename TI, typename TO>
void transpose2d(const TI* in, TO* out, int rows, int cols, cudaStream_t s);
// same with an output row stride ld_out >= rows (padding untouched)
template <typename TI, typename TO>
void transpose2d_ld(const TI* in, TO* out, int rows, int cols, long long ld_out, cudaStream_t s);
// out[r*ld_out + c] = in[r*cols + c]  (copy/convert into a row-padded matrix)
template <typename TI, typename TO>
void convert_ld(const TI* in, TO* out, long long rows, long long cols, long long ld_out,
                cudaStream_t s);

// ---- FP64 vector kernels (deterministic two-pass reductions)
// partial buffer must hold at least kReduceBlocks * k doubles.
constexpr int kReduceBlocks = 304;
void dot_multi(const double* V, long long ldv, int k, const double* w, long long n,
               double* partial, double* out, cudaStream_t s);          // out[j] = <V_j, w>
void gemv_sub(const double* V, long long ldv, int k, const double* h, double* w, long long n,
              cudaStream_t s);                                         // w -= sum_j h[j] V_j
void gemv_set(const double* V, long long ldv, int k, const double* h, double* out, long long n,
              cudaStream_t s);                                         // out = sum_j h[j] V_j
void axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s);
void scale_dev(double* x, const double* num, const double* den_sqrt, long long n, cudaStream_t s);
void lanczos_update(double* w, const double* v, const double* vprev, const double* alpha,
                    double beta_prev, long long n, cudaStream_t s);    // w -= a v + b vprev
void normalize_into(const double* w, const double* nrm2, double* out, long long n, cudaStream_t s);

// ---- small symmetric eigensolver (one CTA, cyclic Jacobi, m <= 64)
// A (m x m, row-major, symmetric) is overwritten; evals ascending, evecs column-major
// (evecs[j*m + i] = component i of eigenvector j).  status[0] = sweeps used (or -1).
void jacobi_eig(double* A, int m, double* evals, double* evecs, int* status, cudaStream_t s);

// Lowest eigenpair of a symmetric tridiagonal matrix passed by value (k <= 64):
// out[0] = eigenvalue, out[1..k] = unit eigenvector (sign arbitrary).
struct TridiagIn {
  int k;
  double a[64];
  double b[64];
};
void tridiag_lowest(const TridiagIn& in, double* out, cudaStream_t s);

// Coarse problem of Sec. 3.1 (m <= 63) in one CTA; outputs on the device.
void coarse_solve_dev(const double* A, const double* S, int m, double eps, double* c,
                      double* lam, int* rank, int* status, cudaStream_t s);

// ---- diagonal of H_eff (Davidson preconditioner)
template <typename T>
void env_diag(const T* E, int D, int R, double* out, cudaStream_t s);     // out[b][w] = E[b][w][b]
void diag_action(const SparseRows<double>& sp, int Rrow, int n, const double* Ed, int Rin, int B,
                 double* out, cudaStream_t s);
void precondition(const double* r, const double* diag, const double* theta, double* t,
                  long long n, cudaStream_t s);

// ---- assorted
// P[i][c] = G[(col_first - c) * ld + i] for i < rows, c < r (P row-major rows x r): the
// columns col_first, col_first - 1, ... of a column-major matrix, as rows of P.
void cols_rev_to_rows(const double* G, long long ld, int rows, int col_first, int r, double* P,
                      cudaStream_t s);
void fill_zero(void* p, size_t bytes, cudaStream_t s);
// Enable / disable (default) the rows-per-CTA autotuner of the sparse stages (disabling
// also forgets its choices).
void sparse_autotune(bool on);
// FP64-class sparse action in double-float arithmetic: input and weights as FP32 pairs
// (in_hi + in_lo, nz_val + nz_lo; in_lo = in_hi + in_plane), output as FP32 pairs
// (out_hi, out_hi + out_plane) or, with out64 set, in FP64.  Geometry as for
// sparse_rows_apply (float4 rows when every stride is a multiple of 4 and the bases are
// 16-byte aligned, scalar otherwise).
void sparse_rows_apply_df(const SparseRows<float>& sp, const SparseGeom& g, const float* in_hi,
                          long long in_plane, float* out_hi, long long out_plane, double* out64,
                          cudaStream_t s);
// grad[param[e]] += factor[e] * G[index[e]] for e < n (FP64 atomics)
void gather_axpy_atomic(const double* G, const long long* index, const long long* param,
                        const double* factor, long long n, double* grad, cudaStream_t s);
void sign_fix_qr(double* Q, int ldq, int rows, double* R, int ldr, int k, cudaStream_t s);
void scale_rows(double* M, int rows, int cols, const double* svals, cudaStream_t s); // M[r,:]*=s[r]
// TT-sum block copy: dst[(o0 + i)*dst_s0 + j*dst_s1 + o2 + k] = alpha * src[i][j][k]
// (added to dst when add is set)
void copy_block3(const double* src, int d0, int d1, int d2, double* dst, long long dst_s0,
                 long long dst_s1, int o0, int o2, double alpha, cudaStream_t s, bool add = false);

}  // namespace a2
