// Dense FP64 factorisations of the sweep, written for this library (no vendor solver):
// the Householder LQ of Alg. 2 step 1 and of the TT rounding.
#pragma once
#include <vector>

#include "common.cuh"

namespace a2 {

// Scratch of the factorisations (grown on demand, owned by a context).
struct FactorWork {
  DevBuf a, v, s, bar;
};

// LQ of a row-major (rows x cols) matrix M: M = L Q with Q (k x cols) orthonormal rows and
// L (rows x k) lower trapezoidal with diag(L) >= 0, k = min(rows, cols).  Householder
// reflections from the right, one per row of M (Golub & Van Loan, Matrix Computations,
// Sec. 5.1-5.2), in FP64.  M is not modified.  Returns k.
int hh_lq(const double* M, int rows, int cols, double* L, double* Q, FactorWork& w,
          cudaStream_t s);

// Truncated SVD step of Alg. 1 (step 2) for a row-major (rows x cols) matrix M, in FP64:
// Golub-Kahan bidiagonalisation of M (or of M^T when rows < cols) by Householder
// reflections, all singular values by bisection of the Golub-Kahan tridiagonal (no Gram
// matrix; FP32 brackets refined in FP64 to a relative width 2^-40, so small singular
// values keep their relative accuracy), the kept left singular vectors by inverse
// iteration on the same tridiagonal, re-orthonormalised (block Gram-Schmidt, CholeskyQR2
// panels) and transformed back.  Keeps the smallest r <= D_max with discarded 2-norm
// <= tol * ||sigma|| (r >= 1); P (rows x r, row-major) receives the left singular
// vectors, *discarded the discarded 2-norm, sv_out (optional) all singular values in
// descending order.  rows <= 12800, min(rows, cols) <= 2400.  Returns r.
int svd_trunc(const double* M, int rows, int cols, int D_max, double tol, double* P,
              double* discarded, std::vector<double>* sv_out, FactorWork& w, cudaStream_t s);

// Device error word of the factorisation kernels (nonzero: a bounded grid barrier gave
// up); reset != 0 clears it.
int factor_error_flag(bool reset);

}  // namespace a2
