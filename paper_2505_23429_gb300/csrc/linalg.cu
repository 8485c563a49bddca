#include "kernels.cuh"
#include "linalg.cuh"

namespace a2 {

#define A2_SOLVER(expr)                                                                  \
  do {                                                                                   \
    cusolverStatus_t st__ = (expr);                                                      \
    if (st__ != CUSOLVER_STATUS_SUCCESS)                                                 \
      throw ::a2::CudaError(std::string(#expr) + " failed with status " +                \
                            std::to_string((int)st__));                                  \
  } while (0)

void Solver::init(cudaStream_t s) {
  A2_SOLVER(cusolverDnCreate(&h));
  A2_SOLVER(cusolverDnSetStream(h, s));
  info.ensure(sizeof(int) * 4, s);
}

void Solver::set_stream(cudaStream_t s) { A2_SOLVER(cusolverDnSetStream(h, s)); }

void Solver::destroy() {
  if (h) cusolverDnDestroy(h);
  h = nullptr;
  work.release();
  info.release();
  tmp.release();
}

// Extract L (rows x k, row-major) from the geqrf factor of M^T (column-major, ld = cols):
// L[i][j] = R'[j][i] for j <= i, R' stored in the upper triangle of buf.
__global__ void extract_l_kernel(const double* buf, int ld, int rows, int k, double* L) {
  const long long n = (long long)rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    L[e] = (j <= i) ? buf[(long long)i * ld + j] : 0.0;
  }
}
// diag(L) >= 0: flip column j of L and row j of Q where L_jj < 0.
__global__ void lq_sign_kernel(double* L, int rows, int k, double* Q, int cols) {
  const int j = blockIdx.x;
  if (L[(long long)j * k + j] >= 0.0) return;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) L[(long long)i * k + j] *= -1.0;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) Q[(long long)j * cols + c] *= -1.0;
}

int Solver::lq(const double* M, int rows, int cols, double* L, double* Q, cudaStream_t s) {
  const int k = rows < cols ? rows : cols;
  ProfScope ps(PK_LQ, s, 4.0 * (double)rows * rows * cols, 8.0 * 3.0 * rows * (double)cols);
  // M row-major (rows x cols) == M^T column-major (cols x rows), ld = cols
  tmp.ensure(sizeof(double) * ((size_t)rows * cols + (size_t)k), s);
  double* A = tmp.as<double>();
  double* tau = A + (size_t)rows * cols;
  A2_CUDA(cudaMemcpyAsync(A, M, sizeof(double) * (size_t)rows * cols, cudaMemcpyDeviceToDevice, s));
  int lw1 = 0, lw2 = 0;
  A2_SOLVER(cusolverDnDgeqrf_bufferSize(h, cols, rows, A, cols, &lw1));
  A2_SOLVER(cusolverDnDorgqr_bufferSize(h, cols, k, k, A, cols, tau, &lw2));
  const int lw = lw1 > lw2 ? lw1 : lw2;
  work.ensure(sizeof(double) * (size_t)(lw > 0 ? lw : 1), s);
  A2_SOLVER(cusolverDnDgeqrf(h, cols, rows, A, cols, tau, work.as<double>(), lw, info.as<int>()));
  {
    long long n = (long long)rows * k;
    int g = (int)((n + 255) / 256);
    extract_l_kernel<<<g > 4096 ? 4096 : (g ? g : 1), 256, 0, s>>>(A, cols, rows, k, L);
    A2_CHECK_LAUNCH();
  }
  A2_SOLVER(cusolverDnDorgqr(h, cols, k, k, A, cols, tau, work.as<double>(), lw, info.as<int>()));
  // Q' is column-major (cols x k) with ld = cols  ==  row-major (k x cols): the Q we want.
  A2_CUDA(cudaMemcpyAsync(Q, A, sizeof(double) * (size_t)k * cols, cudaMemcpyDeviceToDevice, s));
  lq_sign_kernel<<<k, 128, 0, s>>>(L, rows, k, Q, cols);
  A2_CHECK_LAUNCH();
  return k;
}

void Solver::syevd(double* A, int m, double* w, cudaStream_t s) {
  int lw = 0;
  A2_SOLVER(cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, A,
                                        m, w, &lw));
  work.ensure(sizeof(double) * (size_t)(lw > 0 ? lw : 1), s);
  A2_SOLVER(cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, A, m, w,
                             work.as<double>(), lw, info.as<int>()));
}

}  // namespace a2

namespace a2 {
void Solver::syevd_top(double* A, int m, int nev, double* w, cudaStream_t s) {
  int lw = 0, meig = 0;
  const int il = m - nev + 1, iu = m;
  A2_SOLVER(cusolverDnDsyevdx_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                         CUBLAS_FILL_MODE_LOWER, m, A, m, 0.0, 0.0, il, iu,
                                         &meig, w, &lw));
  work.ensure(sizeof(double) * (size_t)(lw > 0 ? lw : 1), s);
  A2_SOLVER(cusolverDnDsyevdx(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                              CUBLAS_FILL_MODE_LOWER, m, A, m, 0.0, 0.0, il, iu, &meig, w,
                              work.as<double>(), lw, info.as<int>()));
  if (meig != nev) throw CudaError("syevdx returned " + std::to_string(meig) + " of " +
                                   std::to_string(nev) + " eigenpairs");
}
}  // namespace a2
