// Dense FP64 factorisations used by the sweep: this library's own kernels (factor.cu) --
// the Householder LQ and the bidiagonalisation SVD; no vendor solver is linked.
#pragma once
#include <vector>
#include "common.cuh"
#include "factor.cuh"

namespace a2 {

struct Solver {
  FactorWork fw;
  void init(cudaStream_t s) { (void)s; }
  void destroy() {
    fw.a.release();
    fw.v.release();
    fw.s.release();
    fw.bar.release();
  }
  void set_stream(cudaStream_t s) { (void)s; }
  // LQ of a row-major (rows x cols) matrix M: M = L Q, Q (k x cols) orthonormal rows,
  // L (rows x k) lower-trapezoidal with diag >= 0, k = min(rows, cols).
  // Q is written row-major (k x cols), L row-major (rows x k).  M is not modified.
  int lq(const double* M, int rows, int cols, double* L, double* Q, cudaStream_t s) {
    return hh_lq(M, rows, cols, L, Q, fw, s);
  }
};

}  // namespace a2
