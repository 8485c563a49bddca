// Dense FP64 factorizations used by the sweep (cuSOLVER for geqrf/orgqr/syevd).
#pragma once
#include <cusolverDn.h>
#include <vector>
#include "common.cuh"

namespace a2 {

struct Solver {
  cusolverDnHandle_t h = nullptr;
  DevBuf work, info, tmp;
  void init(cudaStream_t s);
  void destroy();
  void set_stream(cudaStream_t s);
  // LQ of a row-major (rows x cols) matrix M: M = L Q, Q (k x cols) orthonormal rows,
  // L (rows x k) lower-trapezoidal with diag >= 0, k = min(rows, cols).
  // Q is written row-major (k x cols), L row-major (rows x k).  M is not modified.
  int lq(const double* M, int rows, int cols, double* L, double* Q, cudaStream_t s);
  // Symmetric eigendecomposition of a (m x m) matrix in place: on exit A holds the
  // eigenvectors column-major (column j <-> eigenvalue w[j], ascending).
  void syevd(double* A, int m, double* w, cudaStream_t s);
  // The `nev` largest eigenpairs only (ascending order in w[0..nev-1], eigenvectors in
  // the first nev columns of A, column-major).
  void syevd_top(double* A, int m, int nev, double* w, cudaStream_t s);
};

}  // namespace a2
