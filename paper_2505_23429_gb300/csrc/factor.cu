// Dense FP64 factorisations of the sweep on the GPU, written for this library.
//
// Householder LQ (Golub & Van Loan, Matrix Computations, 4th ed., Sec. 5.1.2-5.1.3 and
// 5.2.1, applied to the rows of M instead of the columns): reflection i maps the trailing
// part of row i onto a multiple of e_i and is applied from the right to the rows below.
// One cooperative persistent kernel walks the k reflections; every block owns the rows
// r with r % gridDim.x == blockIdx.x, so a row is only ever touched by one block, and the
// block that owns row i + 1 forms the next reflection as soon as it has updated that row.
// A grid-wide barrier (bounded: after kBarrierLimit polls it raises the error word and
// every block leaves) separates the reflections.  Q is then formed row by row: row j of
// Q is e_j^T H_j H_{j-1} ... H_0 (the reflections H_i with i > j leave e_j unchanged),
// so every row is independent.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "factor.cuh"
#include "kernels.cuh"

namespace a2 {

namespace {

constexpr int kFacThreads = 256;
constexpr unsigned int kBarrierLimit = 1u << 22;

__device__ int g_factor_error = 0;

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int abort;
};

// All blocks of the grid arrive before any leaves; global writes before it are visible
// to every block after it (thread 0 fences on both sides).  Returns false if the barrier
// gave up (or another block did), in which case the caller must return.
__device__ bool grid_sync(GridBarrier* b) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int gen = *(volatile unsigned int*)&b->gen;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      for (unsigned int it = 0;; ++it) {
        if (*(volatile unsigned int*)&b->gen != gen) break;
        if (*(volatile int*)&b->abort) { ok = 0; break; }
        if (it >= kBarrierLimit) {
          atomicExch(&g_factor_error, 1);
          atomicExch(&b->abort, 1);
          ok = 0;
          break;
        }
        if (it > 32) __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Sum over the block, returned to every thread (red: 32 doubles of shared memory).
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// N sums over the block at once, returned in v to every thread (red: N * 8 doubles).
template <int N>
__device__ void block_sum_n(double (&v)[N], double* red) {
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q)
    for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) red[q * 8 + w] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < N; ++q) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[q * 8 + i];
    v[q] = t;
  }
}
constexpr int kMaxOwn = 8;   // rows of one block whose dot products are reduced together

// Reflection of row i of A (row-major, `cols` columns): with x = A[i][i:], alpha = x_0,
// beta = -sign(alpha) ||x||, v = (1, x_1: / (alpha - beta)), tau = (beta - alpha) / beta,
// (I - tau v v^T) maps x to beta e_0.  Writes V[i][:] (zero before i), tau[i], beta[i]
// and sets row i of A to (beta, 0, ...) from column i on.  tau = 0 when x_1: = 0.
__device__ void make_reflection(double* A, int cols, int i, double* V, double* tau,
                                double* beta, double* red) {
  double* x = A + (size_t)i * cols;
  double* v = V + (size_t)i * cols;
  double s2 = 0.0;
  for (int c = i + 1 + threadIdx.x; c < cols; c += blockDim.x) s2 += x[c] * x[c];
  s2 = block_sum(s2, red);
  const double alpha = x[i];
  double t = 0.0, b = alpha, scale = 0.0;
  if (s2 > 0.0) {
    const double nrm = sqrt(alpha * alpha + s2);
    b = alpha >= 0.0 ? -nrm : nrm;
    t = (b - alpha) / b;
    scale = 1.0 / (alpha - b);
  }
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    const double xc = x[c];
    v[c] = c < i ? 0.0 : (c == i ? 1.0 : xc * scale);
    if (c > i) x[c] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    x[i] = b;
    tau[i] = t;
    beta[i] = b;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFacThreads)
hh_lq_kernel(double* A, int rows, int cols, int k, double* V, double* tau, double* beta,
             GridBarrier* bar) {
  extern __shared__ double vs[];                 // the current reflection vector
  __shared__ double red[32];
  const int nb = gridDim.x, b = blockIdx.x;
  if (b == 0) make_reflection(A, cols, 0, V, tau, beta, red);
  if (!grid_sync(bar)) return;
  for (int i = 0; i < k; ++i) {
    const double t = __ldcg(tau + i);
    if (t != 0.0) {
      const double* vi = V + (size_t)i * cols;
      for (int c = i + threadIdx.x; c < cols; c += blockDim.x) vs[c] = __ldcg(vi + c);
      __syncthreads();
      // rows r > i owned by this block: r = b + nb * m
      int r = i + 1 + ((b - (i + 1) % nb) % nb + nb) % nb;
      for (; r < rows; r += nb) {
        double* ar = A + (size_t)r * cols;
        double d = 0.0;
        for (int c = i + threadIdx.x; c < cols; c += blockDim.x) d += ar[c] * vs[c];
        d = block_sum(d, red) * t;
        for (int c = i + threadIdx.x; c < cols; c += blockDim.x) ar[c] -= d * vs[c];
      }
      __syncthreads();
    }
    if (i + 1 < k && (i + 1) % nb == b) make_reflection(A, cols, i + 1, V, tau, beta, red);
    if (!grid_sync(bar)) return;
  }
}

// Row j of Q = e_j^T H_j H_{j-1} ... H_0 (in shared memory), one block per row.
__global__ void __launch_bounds__(kFacThreads)
hh_form_q_kernel(const double* V, const double* tau, int cols, int k, double* Q) {
  extern __shared__ double q[];
  __shared__ double red[32];
  for (int j = blockIdx.x; j < k; j += gridDim.x) {
    const double tj = tau[j];
    const double* vj = V + (size_t)j * cols;
    for (int c = threadIdx.x; c < cols; c += blockDim.x)
      q[c] = (c == j ? 1.0 : 0.0) - tj * vj[c];
    __syncthreads();
    for (int i = j - 1; i >= 0; --i) {
      const double ti = tau[i];
      if (ti == 0.0) continue;
      const double* vi = V + (size_t)i * cols;
      double d = 0.0;
      for (int c = i + threadIdx.x; c < cols; c += blockDim.x) d += q[c] * vi[c];
      d = block_sum(d, red) * ti;
      for (int c = i + threadIdx.x; c < cols; c += blockDim.x) q[c] -= d * vi[c];
      __syncthreads();
    }
    for (int c = threadIdx.x; c < cols; c += blockDim.x) Q[(size_t)j * cols + c] = q[c];
    __syncthreads();
  }
}

// L[r][j] = A[r][j] for j <= r (j < k), 0 above; then diag(L) >= 0: where beta_j < 0 the
// column j of L and the row j of Q change sign.
__global__ void hh_extract_l_kernel(const double* A, int rows, int cols, int k,
                                    const double* beta, double* L) {
  const long long n = (long long)rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / k), j = (int)(e % k);
    const double sg = beta[j] < 0.0 ? -1.0 : 1.0;
    L[e] = j <= r ? sg * A[(size_t)r * cols + j] : 0.0;
  }
}
__global__ void hh_sign_rows_kernel(double* Q, int cols, int k, const double* beta) {
  for (int j = blockIdx.x; j < k; j += gridDim.x) {
    if (beta[j] >= 0.0) continue;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) Q[(size_t)j * cols + c] *= -1.0;
  }
}

// ------------------------------------------------------------------ truncated SVD
// Golub-Kahan bidiagonalisation (Golub & Van Loan, Sec. 5.4.8) of A (m x n row-major,
// m >= n): A = U_B B V_B^T with U_B = H_0 ... H_{n-1}, V_B = G_0 ... G_{n-3}, B upper
// bidiagonal (d on the diagonal, e above it).  Left reflection i comes from column i
// (rows i..m-1), right reflection i from row i (columns i+1..n-1).  Rows are owned by the
// blocks as in the LQ kernel; a column's norm and the products y = u^T A of a left
// reflection are reduced over the blocks through partial sums and grid barriers (four per
// step).  Afterwards u_i (u_i[i] = 1) sits in column i below the diagonal, w_i
// (w_i[i+1] = 1) in row i right of the superdiagonal, tau_u[i] / tau_v[i] beside them.
__global__ void __launch_bounds__(kFacThreads)
hh_bidiag_kernel(double* A, int m, int n, double* d, double* e, double* tau_u,
                 double* tau_v, double* part, double* ypart, double* y, GridBarrier* bar) {
  __shared__ double red[32];
  __shared__ double red_n[kMaxOwn * 8];
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  auto first_own = [&](int r0) { return r0 + ((b - r0 % nb) % nb + nb) % nb; };
  // partial sum of squares of column 0 below the diagonal over this block's rows
  {
    double s2 = 0.0;
    for (int r = first_own(1) + nb * tid; r < m; r += nb * blockDim.x) {
      const double a = A[(size_t)r * n];
      s2 += a * a;
    }
    s2 = block_sum(s2, red);
    if (tid == 0) part[b] = s2;
  }
  if (!grid_sync(bar)) return;
  for (int i = 0; i < n; ++i) {
    // ---- left reflection from column i (every block forms the same numbers)
    double s2 = 0.0;
    for (int q = tid; q < nb; q += blockDim.x) s2 += __ldcg(part + q);
    s2 = block_sum(s2, red);
    const double alpha = __ldcg(A + (size_t)i * n + i);
    double tu = 0.0, beta = alpha, scale = 0.0;
    if (s2 > 0.0) {
      const double nrm = sqrt(alpha * alpha + s2);
      beta = alpha >= 0.0 ? -nrm : nrm;
      tu = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    if (b == i % nb && tid == 0) {
      d[i] = beta;
      tau_u[i] = tu;
    }
    // own rows: u = A[r][i] * scale below the diagonal (stored in place), then the
    // partial products ypart[b][c] = sum_{own r >= i} u_r A[r][c] for c > i
    const int r_i = first_own(i);
    if (tu != 0.0) {
      for (int r = first_own(i + 1) + nb * tid; r < m; r += nb * blockDim.x)
        A[(size_t)r * n + i] *= scale;
    }
    __syncthreads();
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      double acc = 0.0;
      if (tu != 0.0)
        for (int r = r_i; r < m; r += nb) {
          const double u = r == i ? 1.0 : A[(size_t)r * n + i];
          acc += u * A[(size_t)r * n + c];
        }
      ypart[(size_t)b * n + c] = acc;
    }
    if (!grid_sync(bar)) return;
    // ---- y[c] = sum over blocks (block b reduces columns c = i + 1 + b + nb * t)
    if (tu != 0.0) {
      const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
      for (int c = i + 1 + b + nb * warp; c < n; c += nb * nw) {
        double acc = 0.0;
        for (int q = lane; q < nb; q += 32) acc += __ldcg(ypart + (size_t)q * n + c);
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[c] = acc;
      }
    }
    if (!grid_sync(bar)) return;
    // ---- left update of the own rows r >= i, then (owner of row i) the right reflection
    if (tu != 0.0) {
      for (int r = r_i; r < m; r += nb) {
        const double f = tu * (r == i ? 1.0 : A[(size_t)r * n + i]);
        double* ar = A + (size_t)r * n;
        for (int c = i + 1 + tid; c < n; c += blockDim.x) ar[c] -= f * __ldcg(y + c);
      }
    }
    __syncthreads();
    if (b == i % nb && i + 1 < n) {
      double* x = A + (size_t)i * n;
      double t2 = 0.0;
      for (int c = i + 2 + tid; c < n; c += blockDim.x) t2 += x[c] * x[c];
      t2 = block_sum(t2, red);
      const double al = x[i + 1];
      double tv = 0.0, be = al, sv = 0.0;
      if (t2 > 0.0) {
        const double nrm = sqrt(al * al + t2);
        be = al >= 0.0 ? -nrm : nrm;
        tv = (be - al) / be;
        sv = 1.0 / (al - be);
      }
      for (int c = i + 2 + tid; c < n; c += blockDim.x) x[c] *= sv;
      if (tid == 0) {
        e[i] = be;
        tau_v[i] = tv;
      }
    }
    if (!grid_sync(bar)) return;
    // ---- right update of the own rows r > i with w = (1, A[i][i+2:]) (the dot products
    // of up to kMaxOwn own rows reduced together), then the partial norm of column i + 1
    // below its diagonal
    if (i + 1 < n) {
      const double tv = __ldcg(tau_v + i);
      const double* w = A + (size_t)i * n;
      if (tv != 0.0) {
        for (int r0 = first_own(i + 1); r0 < m; r0 += nb * kMaxOwn) {
          double z[kMaxOwn];
#pragma unroll
          for (int q = 0; q < kMaxOwn; ++q) z[q] = 0.0;
          for (int c = i + 1 + tid; c < n; c += blockDim.x) {
            const double wc = c == i + 1 ? 1.0 : __ldcg(w + c);
#pragma unroll
            for (int q = 0; q < kMaxOwn; ++q) {
              const int r = r0 + q * nb;
              if (r < m) z[q] += A[(size_t)r * n + c] * wc;
            }
          }
          block_sum_n<kMaxOwn>(z, red_n);
          for (int c = i + 1 + tid; c < n; c += blockDim.x) {
            const double wc = c == i + 1 ? 1.0 : __ldcg(w + c);
#pragma unroll
            for (int q = 0; q < kMaxOwn; ++q) {
              const int r = r0 + q * nb;
              if (r < m) A[(size_t)r * n + c] -= tv * z[q] * wc;
            }
          }
          __syncthreads();
        }
      }
      __syncthreads();
      double p2 = 0.0;
      for (int r = first_own(i + 2) + nb * tid; r < m; r += nb * blockDim.x) {
        const double a = A[(size_t)r * n + i + 1];
        p2 += a * a;
      }
      p2 = block_sum(p2, red);
      if (tid == 0) part[b] = p2;
      if (!grid_sync(bar)) return;
    }
  }
}

// The same bidiagonalisation with every block's rows resident in shared memory for the whole
// reduction (rows never change owner): row q of the block is global row b + nb * q, held at
// rows[q * n].  Only what crosses blocks goes through global memory: the partial column
// norms (part), the partial products y (ypart, reduced into y), the pivot A[i][i] of the next
// left reflection (alpha, published by the owner of row i), and the right reflection vector
// (wg, published by the owner of row i).  At the end the rows, holding the reflection
// vectors in place, are written back to A for the back-transformation.
__global__ void __launch_bounds__(kFacThreads)
hh_bidiag_smem_kernel(double* A, int m, int n, double* d, double* e, double* tau_u,
                      double* tau_v, double* part, double* ypart, double* y, double* alpha,
                      double* wg, GridBarrier* bar) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double red_n[kMaxOwn * 8];
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int R = (m - b + nb - 1) / nb;          // rows of this block
  double* rows = sm;                            // R x n
  double* vec = sm + (size_t)R * n;             // y or w of the current step (n)
  for (int q = 0; q < R; ++q)
    for (int c = tid; c < n; c += blockDim.x) rows[(size_t)q * n + c] = A[(size_t)(b + nb * q) * n + c];
  __syncthreads();
  auto qof = [&](int r) { return (r - b) / nb; };            // r % nb == b assumed
  auto q_first = [&](int r0) { return r0 <= b ? 0 : (r0 - b + nb - 1) / nb; };   // first q with row >= r0
  {
    double s2 = 0.0;
    for (int q = q_first(1) + tid; q < R; q += blockDim.x) {
      const double a = rows[(size_t)q * n];
      s2 += a * a;
    }
    s2 = block_sum(s2, red);
    if (tid == 0) {
      part[b] = s2;
      if (b == 0) alpha[0] = rows[0];
    }
  }
  if (!grid_sync(bar)) return;
  for (int i = 0; i < n; ++i) {
    const bool own_i = i % nb == b;
    // ---- left reflection from column i (every block forms the same numbers)
    double s2 = 0.0;
    for (int q = tid; q < nb; q += blockDim.x) s2 += __ldcg(part + q);
    s2 = block_sum(s2, red);
    const double al = __ldcg(alpha + i);
    double tu = 0.0, beta = al, scale = 0.0;
    if (s2 > 0.0) {
      const double nrm = sqrt(al * al + s2);
      beta = al >= 0.0 ? -nrm : nrm;
      tu = (beta - al) / beta;
      scale = 1.0 / (al - beta);
    }
    if (own_i && tid == 0) {
      d[i] = beta;
      tau_u[i] = tu;
    }
    const int q0 = q_first(i), q1 = q_first(i + 1);
    if (tu != 0.0)
      for (int q = q1 + tid; q < R; q += blockDim.x) rows[(size_t)q * n + i] *= scale;
    __syncthreads();
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      double acc = 0.0;
      if (tu != 0.0)
        for (int q = q0; q < R; ++q) {
          const double u = (own_i && q == q0) ? 1.0 : rows[(size_t)q * n + i];
          acc += u * rows[(size_t)q * n + c];
        }
      ypart[(size_t)b * n + c] = acc;
    }
    if (!grid_sync(bar)) return;
    // ---- y[c] = sum over blocks (block b reduces columns c = i + 1 + b + nb * t)
    if (tu != 0.0) {
      const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
      for (int c = i + 1 + b + nb * warp; c < n; c += nb * nw) {
        double acc = 0.0;
        for (int q = lane; q < nb; q += 32) acc += __ldcg(ypart + (size_t)q * n + c);
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[c] = acc;
      }
    }
    if (!grid_sync(bar)) return;
    // ---- left update of the own rows r >= i; the owner of row i forms the right reflection
    if (tu != 0.0) {
      for (int c = i + 1 + tid; c < n; c += blockDim.x) vec[c] = __ldcg(y + c);
      __syncthreads();
      for (int q = q0; q < R; ++q) {
        const double f = tu * ((own_i && q == q0) ? 1.0 : rows[(size_t)q * n + i]);
        double* rq = rows + (size_t)q * n;
        for (int c = i + 1 + tid; c < n; c += blockDim.x) rq[c] -= f * vec[c];
      }
      __syncthreads();
    }
    if (own_i && i + 1 < n) {
      double* x = rows + (size_t)qof(i) * n;
      double t2 = 0.0;
      for (int c = i + 2 + tid; c < n; c += blockDim.x) t2 += x[c] * x[c];
      t2 = block_sum(t2, red);
      const double ar = x[i + 1];
      double tv = 0.0, be = ar, sv = 0.0;
      if (t2 > 0.0) {
        const double nrm = sqrt(ar * ar + t2);
        be = ar >= 0.0 ? -nrm : nrm;
        tv = (be - ar) / be;
        sv = 1.0 / (ar - be);
      }
      for (int c = i + 2 + tid; c < n; c += blockDim.x) {
        x[c] *= sv;
        wg[c] = x[c];
      }
      if (tid == 0) {
        e[i] = be;
        tau_v[i] = tv;
      }
    }
    if (!grid_sync(bar)) return;
    // ---- right update of the own rows r > i with w = (1, wg[i+2:]); partial norm of
    // column i + 1 below its diagonal; the owner of row i + 1 publishes its pivot
    if (i + 1 < n) {
      const double tv = __ldcg(tau_v + i);
      for (int c = i + 1 + tid; c < n; c += blockDim.x) vec[c] = c == i + 1 ? 1.0 : __ldcg(wg + c);
      __syncthreads();
      if (tv != 0.0) {
        for (int qa = q1; qa < R; qa += kMaxOwn) {
          double z[kMaxOwn];
#pragma unroll
          for (int t = 0; t < kMaxOwn; ++t) z[t] = 0.0;
          for (int c = i + 1 + tid; c < n; c += blockDim.x) {
            const double wc = vec[c];
#pragma unroll
            for (int t = 0; t < kMaxOwn; ++t)
              if (qa + t < R) z[t] += rows[(size_t)(qa + t) * n + c] * wc;
          }
          block_sum_n<kMaxOwn>(z, red_n);
          for (int c = i + 1 + tid; c < n; c += blockDim.x) {
            const double wc = vec[c];
#pragma unroll
            for (int t = 0; t < kMaxOwn; ++t)
              if (qa + t < R) rows[(size_t)(qa + t) * n + c] -= tv * z[t] * wc;
          }
          __syncthreads();
        }
      }
      double p2 = 0.0;
      for (int q = q_first(i + 2) + tid; q < R; q += blockDim.x) {
        const double a = rows[(size_t)q * n + i + 1];
        p2 += a * a;
      }
      p2 = block_sum(p2, red);
      if (tid == 0) {
        part[b] = p2;
        if ((i + 1) % nb == b) alpha[i + 1] = rows[(size_t)qof(i + 1) * n + i + 1];
      }
      if (!grid_sync(bar)) return;
    }
  }
  // rows back to A: u_i below the diagonals, w_i right of the superdiagonals
  for (int q = 0; q < R; ++q)
    for (int c = tid; c < n; c += blockDim.x) A[(size_t)(b + nb * q) * n + c] = rows[(size_t)q * n + c];
}

// Golub-Kahan tridiagonal of B: zero diagonal, off-diagonal t = (d0, e0, d1, e1, ..., d_{n-1});
// its eigenvalues are +-sigma_k, the eigenvector of +sigma is (v0, u0, v1, u1, ...) / sqrt 2
// with B v = sigma u.  Number of its eigenvalues below x (Sturm count of the LDL^T pivots),
// from the squared off-diagonal entries t2[j] = t_j^2 (t2[0] unused).
__device__ int tgk_count(const double* t2, int N, double x, double pivmin) {
  int cnt = 0;
  double q = -x;
  if (q < 0.0) ++cnt;
  for (int j = 1; j < N; ++j) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = -x - t2[j] / q;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// The nev largest singular values of B, descending (sigma[k] = k-th largest), by bisection
// of the Golub-Kahan tridiagonal: eight lanes per k evaluate the count at eight interior
// points of the current interval (multisection, 3.2 bits per pass), until the interval
// is within four ulps of its end points.  t^2 sits in shared memory (2n doubles).
__global__ void tgk_bisect_kernel(const double* d, const double* e, int n, int nev,
                                  double* sigma) {
  extern __shared__ double t2[];
  const int N = 2 * n;
  double bound = 0.0, t2max = 0.0;
  for (int j = 1; j < N; ++j) {   // every thread: the Gershgorin bound (cheap, cached)
    const double t = (j & 1) ? d[j >> 1] : e[(j >> 1) - 1];
    const double tn = j + 1 < N ? (((j + 1) & 1) ? d[(j + 1) >> 1] : e[((j + 1) >> 1) - 1]) : 0.0;
    bound = fmax(bound, fabs(t) + fabs(tn));
    t2max = fmax(t2max, t * t);
    if (threadIdx.x == 0) t2[j] = t * t;
  }
  bound = fmax(bound, fabs(d[0])) * (1.0 + 1e-14);
  const double pivmin = fmax(t2max, 1e-300) * 1e-300 + 1e-300;
  __syncthreads();
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int j = 2 * n - 1 - k;              // ascending index of +sigma_k among the 2n
  double lo = 0.0, hi = bound;              // count(lo) <= j < count(hi)
  bool done = k >= nev;
  for (int pass = 0; pass < 60; ++pass) {
    if (!done && (hi - lo <= 4.0 * 2.2204460492503131e-16 * fabs(hi) || hi - lo < 1e-300))
      done = true;
    if (__all_sync(0xffffffffu, done)) break;
    const double x = lo + (hi - lo) * (double)(sub + 1) / 9.0;
    const int c = done ? 0 : tgk_count(t2, N, x, pivmin);
    const unsigned bits = (__ballot_sync(0xffffffffu, c > j) >> (lane & 24)) & 0xFFu;
    if (!done) {
      const int first = bits ? __ffs(bits) - 1 : 8;   // first point above the eigenvalue
      const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / 9.0;
      const double nhi = first == 8 ? hi : lo + (hi - lo) * (double)(first + 1) / 9.0;
      lo = nlo;
      hi = nhi;
    }
  }
  if (k < nev && sub == 0) sigma[k] = 0.5 * (lo + hi);
}

// Inverse iteration for the kept singular pairs: for k < r, three solves of
// (T - sigma_k I) z = z_prev (T the Golub-Kahan tridiagonal of size N = 2n) by Gaussian
// elimination with partial pivoting on the band (a row interchange whenever the
// subdiagonal entry is the larger one, which fills one second superdiagonal), from a
// start vector that differs per k; writes the u half (side 0: odd entries) or the v half
// (side 1: even entries) of z, normalised, to out[k][:] (n values).  One warp per k: lane
// 0 runs the elimination and the substitutions (sequential by nature) on band factors
// held in shared memory (5 N doubles + N flags), the warp scales and extracts.  Pivots
// below eps * max|t| are replaced by that size (sigma_k is an eigenvalue to working
// accuracy).
__global__ void tgk_invit_kernel(const double* d, const double* e, int n, const double* sigma,
                                 int r, int side, double* out) {
  extern __shared__ double sm[];
  const int k = blockIdx.x;
  if (k >= r) return;
  const int N = 2 * n, lane = threadIdx.x;
  double* dg = sm;                          // diagonal of the upper factor
  double* s1 = dg + N;                      // its first superdiagonal
  double* s2 = s1 + N;                      // its second superdiagonal (fill-in)
  double* ml = s2 + N;                      // elimination multipliers
  double* z = ml + N;                       // the iterate
  unsigned char* sw = reinterpret_cast<unsigned char*>(z + N);   // row interchanges
  auto t = [&](int j) { return (j & 1) ? d[j >> 1] : e[(j >> 1) - 1]; };   // T[j-1][j]
  double tmax = 0.0;
  for (int j = lane; j < n; j += 32) tmax = fmax(tmax, fabs(d[j]));
  for (int j = lane; j + 1 < n; j += 32) tmax = fmax(tmax, fabs(e[j]));
  for (int o = 16; o; o >>= 1) tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
  // (a zero B: every vector is a singular vector, any nonzero pivot will do)
  const double tiny = (tmax > 1e-290 ? tmax : 1.0) * 2.2204460492503131e-16;
  const double lam = sigma[k];
  for (int j = lane; j < N; j += 32) {
    dg[j] = -lam;
    s1[j] = j + 1 < N ? t(j + 1) : 0.0;
    s2[j] = 0.0;
    ml[j] = 0.0;
    sw[j] = 0;
    unsigned long long h = 0x9E3779B97F4A7C15ull * (unsigned long long)(k + 1) +
                           0xD1B54A32D192ED03ull * (unsigned long long)(j + 1);
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    z[j] = (double)((h >> 11) & 0xFFFFF) / 1048576.0 - 0.5;
  }
  __syncwarp();
  if (lane == 0) {
    // eliminate the subdiagonal entry T[j+1][j] = t(j + 1) column by column
    for (int j = 0; j + 1 < N; ++j) {
      const double sub = t(j + 1);
      if (fabs(dg[j]) >= fabs(sub)) {
        if (fabs(dg[j]) < tiny) dg[j] = dg[j] < 0.0 ? -tiny : tiny;
        const double f = sub / dg[j];
        ml[j] = f;
        dg[j + 1] -= f * s1[j];
      } else {                                // interchange rows j and j + 1
        const double f = dg[j] / sub;
        const double r1 = dg[j + 1], r2 = j + 1 < N - 1 ? s1[j + 1] : 0.0;   // row j+1
        dg[j] = sub;
        const double old1 = s1[j];
        s1[j] = r1;
        s2[j] = r2;
        dg[j + 1] = old1 - f * r1;
        if (j + 1 < N - 1) s1[j + 1] = -f * r2;
        ml[j] = f;
        sw[j] = 1;
      }
    }
    if (fabs(dg[N - 1]) < tiny) dg[N - 1] = dg[N - 1] < 0.0 ? -tiny : tiny;
  }
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (lane == 0) {
      for (int j = 0; j + 1 < N; ++j) {     // forward: row interchanges and multipliers
        if (sw[j]) {
          const double a = z[j];
          z[j] = z[j + 1];
          z[j + 1] = a - ml[j] * z[j];
        } else {
          z[j + 1] -= ml[j] * z[j];
        }
      }
      for (int j = N - 1; j >= 0; --j) {    // backward: the banded upper factor
        double v = z[j];
        if (j + 1 < N) v -= s1[j] * z[j + 1];
        if (j + 2 < N) v -= s2[j] * z[j + 2];
        z[j] = v / dg[j];
      }
    }
    __syncwarp();
    double mx = 0.0;
    for (int j = lane; j < N; j += 32) mx = fmax(mx, fabs(z[j]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double inv = mx > 0.0 ? 1.0 / mx : 0.0;
    for (int j = lane; j < N; j += 32) z[j] *= inv;
    __syncwarp();
  }
  const int off = side == 0 ? 1 : 0;
  double ss = 0.0;
  for (int j = lane; j < n; j += 32) ss += z[2 * j + off] * z[2 * j + off];
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
  for (int j = lane; j < n; j += 32) out[(size_t)k * n + j] = z[2 * j + off] * inv;
}

// Back-transformation of kept vectors by the reflections of the bidiagonalisation: column
// k of X (p x r, X[j][k] at X[j * r + k], zero-padded from n to p rows) becomes
// R_0 R_1 ... R_{q-1} x with R_i = I - tau_i v_i v_i^T, v_i[i + off] = 1 and its further
// entries A[row][col] read by `left` (column i below the diagonal: rows i+1.., off = 0) or
// by the right side (row i beyond the superdiagonal: columns i+2.., off = 1).  One block
// per kApplyCols columns (every reflection is read once for all of them).
constexpr int kApplyCols = 2;
__global__ void __launch_bounds__(kFacThreads)
bidiag_apply_kernel(const double* A, int lda, int p, int q, const double* tau, int left, double* X,
                    int r) {
  extern __shared__ double x[];           // kApplyCols x p
  __shared__ double red[kApplyCols * 8];
  const int off = left ? 0 : 1;
  for (int k0 = blockIdx.x * kApplyCols; k0 < r; k0 += gridDim.x * kApplyCols) {
    for (int j = threadIdx.x; j < p; j += blockDim.x)
#pragma unroll
      for (int v = 0; v < kApplyCols; ++v)
        x[v * p + j] = k0 + v < r ? X[(size_t)j * r + k0 + v] : 0.0;
    __syncthreads();
    for (int i = q - 1; i >= 0; --i) {
      const double ti = tau[i];
      if (ti == 0.0) continue;
      const int j0 = i + off;
      double dsum[kApplyCols];
#pragma unroll
      for (int v = 0; v < kApplyCols; ++v) dsum[v] = 0.0;
      for (int j = j0 + threadIdx.x; j < p; j += blockDim.x) {
        const double vj = j == j0 ? 1.0 : (left ? A[(size_t)j * lda + i] : A[(size_t)i * lda + j]);
#pragma unroll
        for (int v = 0; v < kApplyCols; ++v) dsum[v] += vj * x[v * p + j];
      }
      block_sum_n<kApplyCols>(dsum, red);
      for (int j = j0 + threadIdx.x; j < p; j += blockDim.x) {
        const double vj = j == j0 ? 1.0 : (left ? A[(size_t)j * lda + i] : A[(size_t)i * lda + j]);
#pragma unroll
        for (int v = 0; v < kApplyCols; ++v) x[v * p + j] -= ti * dsum[v] * vj;
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x)
#pragma unroll
      for (int v = 0; v < kApplyCols; ++v)
        if (k0 + v < r) X[(size_t)j * r + k0 + v] = x[v * p + j];
    __syncthreads();
  }
}

// Orthonormalisation within a panel of w <= 32 columns (cols c0 .. c0 + w - 1) of X
// (rows x ld, row-major), in one block.  Each column (a unit vector on entry, already
// orthogonal to the columns before the panel) gets classical Gram-Schmidt against the
// panel's earlier columns twice -- all its dot products reduced together -- and is
// normalised.  A column that was (numerically) in the span of the earlier ones is
// replaced by a pseudo-random vector orthogonalised against all earlier columns (one at a
// time), so that the result always has orthonormal columns.
__device__ void mgs_against(double* X, int rows, int ld, int q0, int c, double* red) {
  for (int pass = 0; pass < 2; ++pass)
    for (int q = q0; q < c; ++q) {
      double dsum = 0.0;
      for (int j = threadIdx.x; j < rows; j += blockDim.x)
        dsum += X[(size_t)j * ld + q] * X[(size_t)j * ld + c];
      dsum = block_sum(dsum, red);
      for (int j = threadIdx.x; j < rows; j += blockDim.x)
        X[(size_t)j * ld + c] -= dsum * X[(size_t)j * ld + q];
      __syncthreads();
    }
}
__device__ double col_norm2(const double* X, int rows, int ld, int c, double* red) {
  double nrm = 0.0;
  for (int j = threadIdx.x; j < rows; j += blockDim.x)
    nrm += X[(size_t)j * ld + c] * X[(size_t)j * ld + c];
  return block_sum(nrm, red);
}
__global__ void __launch_bounds__(kFacThreads)
panel_mgs_kernel(double* X, int rows, int ld, int c0, int w) {
  __shared__ double red[32];
  __shared__ double redw[32 * 8];
  __shared__ double dots[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = c0; c < c0 + w; ++c) {
    const int nq = c - c0;
    for (int pass = 0; pass < 2 && nq > 0; ++pass) {
      // lane-parallel partial dots: thread handles rows j = tid, tid + blockDim, ...
      double part[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) part[q] = 0.0;
      for (int j = threadIdx.x; j < rows; j += blockDim.x) {
        const double xc = X[(size_t)j * ld + c];
        const double* xr = X + (size_t)j * ld + c0;
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (q < nq) part[q] += xr[q] * xc;
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        double v = part[q];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) redw[q * 8 + warp] = v;
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += redw[threadIdx.x * 8 + i];
        dots[threadIdx.x] = t;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < rows; j += blockDim.x) {
        const double* xr = X + (size_t)j * ld + c0;
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) acc += dots[q] * xr[q];
        X[(size_t)j * ld + c] -= acc;
      }
      __syncthreads();
    }
    double nrm = col_norm2(X, rows, ld, c, red);
    if (!(nrm > 1e-20)) {
      for (int j = threadIdx.x; j < rows; j += blockDim.x) {
        unsigned long long h = 0x9E3779B97F4A7C15ull * (unsigned long long)(j + 1) +
                               0xD1B54A32D192ED03ull * (unsigned long long)(c + 1);
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 29;
        X[(size_t)j * ld + c] = (double)((h >> 11) & 0xFFFFF) / 1048576.0 - 0.5;
      }
      __syncthreads();
      mgs_against(X, rows, ld, 0, c, red);
      nrm = col_norm2(X, rows, ld, c, red);
    }
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int j = threadIdx.x; j < rows; j += blockDim.x) X[(size_t)j * ld + c] *= inv;
    __syncthreads();
  }
}

// out[j][k] = in[k][j] (k < r, j < n), rows of `out` padded with zeros up to p
__global__ void rows_to_cols_kernel(const double* in, int r, int n, int p, double* out) {
  const long long tot = (long long)p * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / r), k = (int)(e % r);
    out[e] = j < n ? in[(size_t)k * n + j] : 0.0;
  }
}

int num_sms() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    A2_CUDA(cudaGetDevice(&dev));
    A2_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  });
  return n;
}

void set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024)
    A2_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

int factor_error_flag(bool reset) {
  int v = 0;
  A2_CUDA(cudaMemcpyFromSymbol(&v, g_factor_error, sizeof(int)));
  if (reset && v) {
    int z = 0;
    A2_CUDA(cudaMemcpyToSymbol(g_factor_error, &z, sizeof(int)));
  }
  return v;
}

void set_attributes() {
  static std::once_flag attr;
  std::call_once(attr, [] {
    set_smem((const void*)hh_lq_kernel, 200 * 1024);
    set_smem((const void*)hh_form_q_kernel, 200 * 1024);
    set_smem((const void*)bidiag_apply_kernel, 200 * 1024);
    set_smem((const void*)tgk_bisect_kernel, 200 * 1024);
    set_smem((const void*)tgk_invit_kernel, 200 * 1024);
    set_smem((const void*)hh_bidiag_smem_kernel, 200 * 1024);
  });
}

int svd_trunc(const double* M, int rows, int cols, int D_max, double tol, double* P,
              double* discarded, std::vector<double>* sv_out, FactorWork& w, cudaStream_t s) {
  A2_REQUIRE(rows >= 1 && cols >= 1 && D_max >= 1, "SVD: bad sizes");
  A2_REQUIRE(rows <= 25600, "SVD: more than 25600 rows");
  set_attributes();
  const bool left = rows >= cols;                 // bidiagonalise M (left) or M^T (right)
  const int m = left ? rows : cols, n = left ? cols : rows;
  const int nb = std::max(1, std::min(m, num_sms()));
  // scratch: A (m n), d, e, tau_u, tau_v (n each), sigma (n), part (nb), y (n), ypart (nb n)
  const size_t nA = (size_t)m * n;
  w.a.ensure(sizeof(double) * nA, s);
  w.s.ensure(sizeof(double) * (8 * (size_t)n + nb + (size_t)nb * n), s);
  w.bar.ensure(sizeof(GridBarrier), s);
  double* A = w.a.as<double>();
  double* d = w.s.as<double>();
  double* e = d + n;
  double* tu = e + n;
  double* tv = tu + n;
  double* sig = tv + n;
  double* y = sig + n;                            // y, then alpha and wg (n each)
  double* part = y + 3 * n;
  double* ypart = part + nb;
  if (left)
    A2_CUDA(cudaMemcpyAsync(A, M, sizeof(double) * nA, cudaMemcpyDeviceToDevice, s));
  else
    transpose2d<double, double>(M, A, rows, cols, s);
  A2_CUDA(cudaMemsetAsync(w.bar.p, 0, sizeof(GridBarrier), s));
  A2_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, s));
  {
    GridBarrier* bar = w.bar.as<GridBarrier>();
    int mm = m, nn = n;
    const size_t smem = sizeof(double) * ((size_t)cdiv(m, nb) + 1) * n;
    if (smem <= 200 * 1024) {   // every block's rows resident in shared memory
      double* alpha = y + n;    // n more doubles behind y (reserved below)
      double* wg = alpha + n;
      void* args[] = {&A, &mm, &nn, &d, &e, &tu, &tv, &part, &ypart, &y, &alpha, &wg, &bar};
      A2_CUDA(cudaLaunchCooperativeKernel((const void*)hh_bidiag_smem_kernel, dim3(nb),
                                          dim3(kFacThreads), args, smem, s));
    } else {
      void* args[] = {&A, &mm, &nn, &d, &e, &tu, &tv, &part, &ypart, &y, &bar};
      A2_CUDA(cudaLaunchCooperativeKernel((const void*)hh_bidiag_kernel, dim3(nb),
                                          dim3(kFacThreads), args, 0, s));
    }
    count_launch();
  }
  // the largest nev singular values: the most a truncation to D_max can keep, plus one
  const int nev = std::min(n, D_max + 1);
  tgk_bisect_kernel<<<cdiv(8LL * nev, 256), 256, sizeof(double) * 2 * n, s>>>(d, e, n, nev, sig);
  A2_CHECK_LAUNCH();
  std::vector<double> sv(nev), de(2 * (size_t)n);
  A2_CUDA(cudaMemcpyAsync(sv.data(), sig, sizeof(double) * nev, cudaMemcpyDeviceToHost, s));
  A2_CUDA(cudaMemcpyAsync(de.data(), d, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s));
  A2_CUDA(cudaStreamSynchronize(s));
  if (factor_error_flag(true)) throw CudaError("SVD: a bounded grid barrier gave up");
  // smallest r <= D_max whose discarded 2-norm is <= tol * ||sigma|| (at least 1).  The
  // tail is summed from the small end over the computed values; what lies beyond them
  // (only when D_max + 1 < n) is ||B||_F^2 minus their squares.
  double total = 0.0, computed = 0.0;
  for (int j = 0; j < n; ++j) total += de[j] * de[j] + de[n + j] * de[n + j];
  for (int k = 0; k < nev; ++k) computed += sv[k] * sv[k];
  std::vector<double> tail(nev + 1, 0.0);
  tail[nev] = nev < n ? std::max(total - computed, 0.0) : 0.0;
  for (int k = nev - 1; k >= 0; --k) tail[k] = tail[k + 1] + sv[k] * sv[k];
  int r = nev;
  const double thr = tol * tol * (nev < n ? total : tail[0]);
  for (int cand = 1; cand <= nev; ++cand)
    if (tail[cand] <= thr) { r = cand; break; }
  r = std::max(1, std::min(r, D_max));
  if (discarded) *discarded = std::sqrt(std::max(tail[r], 0.0));
  if (sv_out) *sv_out = sv;
  // kept singular vectors of B by inverse iteration, then into the columns of P (rows x r)
  w.v.ensure(sizeof(double) * ((size_t)r * n + (size_t)r * 32), s);
  double* vecs = w.v.as<double>();
  double* C = vecs + (size_t)r * n;
  const size_t inv_smem = sizeof(double) * 5 * 2 * (size_t)n + 2 * (size_t)n;
  A2_REQUIRE(inv_smem <= 200 * 1024, "SVD: the smaller dimension exceeds 2400");
  tgk_invit_kernel<<<r, 32, inv_smem, s>>>(d, e, n, sig, r, left ? 0 : 1, vecs);
  A2_CHECK_LAUNCH();
  {
    const long long tot = (long long)rows * r;
    rows_to_cols_kernel<<<(int)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(
        vecs, r, n, rows, P);
    A2_CHECK_LAUNCH();
  }
  // orthonormal columns (block classical Gram-Schmidt, twice, panels of 32): exactly or
  // nearly degenerate singular values give inverse-iteration vectors that only span
  // their singular subspace
  constexpr int W = 32;
  for (int c0 = 0; c0 < r; c0 += W) {
    const int wd = std::min(W, r - c0);
    if (c0 > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        SimtGemm<double, double> g;   // C[q][c] = sum_j P[j][q] P[j][c0 + c]
        g.M = c0; g.N = wd; g.K = rows;
        g.A = P; g.sam = 1; g.sak = r;
        g.B = P + c0; g.sbn = 1; g.sbk = r;
        g.C = C; g.scm = wd; g.scn = 1;
        simt_gemm(g, s);
        SimtGemm<double, double> h;   // P[j][c0 + c] -= sum_q P[j][q] C[q][c]
        h.M = rows; h.N = wd; h.K = c0;
        h.A = P; h.sam = r; h.sak = 1;
        h.B = C; h.sbn = 1; h.sbk = wd;
        h.C = P + c0; h.scm = r; h.scn = 1;
        h.alpha = -1.0;
        h.mode = GEMM_ADD;
        simt_gemm(h, s);
      }
    }
    panel_mgs_kernel<<<1, kFacThreads, 0, s>>>(P, rows, r, c0, wd);
    A2_CHECK_LAUNCH();
  }
  // back to the frame of M: the left reflections of M's bidiagonalisation, or the right
  // ones of M^T's (both act on R^rows)
  {
    const int q = left ? n : std::max(n - 1, 0);
    bidiag_apply_kernel<<<std::min(cdiv(r, kApplyCols), 4 * num_sms()), kFacThreads,
                          sizeof(double) * kApplyCols * rows, s>>>(A, n, rows, q, left ? tu : tv,
                                                                   left ? 1 : 0, P, r);
    A2_CHECK_LAUNCH();
  }
  return r;
}

int hh_lq(const double* M, int rows, int cols, double* L, double* Q, FactorWork& w,
          cudaStream_t s) {
  const int k = std::min(rows, cols);
  A2_REQUIRE(rows >= 1 && cols >= 1, "LQ: empty matrix");
  const size_t vbytes = sizeof(double) * (size_t)cols;
  A2_REQUIRE(vbytes <= 200 * 1024, "LQ: rows longer than 25600 entries");
  ProfScope ps(PK_LQ, s, 4.0 * (double)rows * rows * cols, 8.0 * 3.0 * rows * (double)cols);
  w.a.ensure(sizeof(double) * (size_t)rows * cols, s);
  w.v.ensure(sizeof(double) * ((size_t)k * cols + 2 * (size_t)k), s);
  w.bar.ensure(sizeof(GridBarrier), s);
  double* A = w.a.as<double>();
  double* V = w.v.as<double>();
  double* tau = V + (size_t)k * cols;
  double* beta = tau + k;
  A2_CUDA(cudaMemcpyAsync(A, M, sizeof(double) * (size_t)rows * cols, cudaMemcpyDeviceToDevice, s));
  A2_CUDA(cudaMemsetAsync(w.bar.p, 0, sizeof(GridBarrier), s));
  set_attributes();
  // cooperative launch: every block resident at once (the grid barrier relies on it)
  int per_sm = 0;
  A2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hh_lq_kernel, kFacThreads,
                                                        vbytes));
  A2_REQUIRE(per_sm >= 1, "LQ: kernel does not fit on an SM");
  const int grid = std::max(1, std::min({rows, num_sms() * per_sm, num_sms()}));
  GridBarrier* bar = w.bar.as<GridBarrier>();
  void* args[] = {&A, &rows, &cols, const_cast<int*>(&k), &V, &tau, &beta, &bar};
  A2_CUDA(cudaLaunchCooperativeKernel((const void*)hh_lq_kernel, dim3(grid), dim3(kFacThreads),
                                      args, vbytes, s));
  count_launch();
  hh_form_q_kernel<<<std::min(k, 4 * num_sms()), kFacThreads, vbytes, s>>>(V, tau, cols, k, Q);
  A2_CHECK_LAUNCH();
  {
    const long long n = (long long)rows * k;
    const int g = (int)std::min<long long>((n + 255) / 256, 4096);
    hh_extract_l_kernel<<<std::max(g, 1), 256, 0, s>>>(A, rows, cols, k, beta, L);
    A2_CHECK_LAUNCH();
  }
  hh_sign_rows_kernel<<<std::min(k, 1024), 128, 0, s>>>(Q, cols, k, beta);
  A2_CHECK_LAUNCH();
  return k;
}

}  // namespace a2
