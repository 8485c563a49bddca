// Dense FP64 factorisations of the sweep on the GPU, written for this library.
//
// Householder LQ (Golub & Van Loan, Matrix Computations, 4th ed., Sec. 5.1.2-5.1.3 and
// 5.2.1, applied to the rows of M instead of the columns): reflection i maps the trailing
// part of row i onto a multiple of e_i and is applied from the right to the rows below.
// One cooperative persistent kernel walks the k reflections; every block owns the rows
// r with r % gridDim.x == blockIdx.x, so a row is only ever touched by one block, and the
// block that owns row i + 1 forms and publishes the next reflection as soon as it has
// updated that row.  The blocks synchronise on those publications alone (one flag per
// reflection, bounded waits: after kBarrierLimit polls a wait raises the error word and
// every block leaves), so they pipeline behind the owners instead of meeting at a
// grid-wide barrier per reflection.  Q is then formed row by row: row j of
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
  unsigned int count;   // arrivals since the launch (monotonic)
  int abort;
};

// All blocks of the grid arrive before any leaves; global writes before it are visible
// to every block after it (thread 0 fences on both sides).  epoch counts the caller's
// barriers (every block passes the same number), so barrier e waits for e * gridDim.x
// arrivals on one monotonic counter: an arrival is a single reduction, no reset.  Returns
// false if the barrier gave up after kBarrierLimit polls (or another block did), in which
// case the caller must return.
__device__ bool grid_sync(GridBarrier* b, unsigned& epoch) {
  __shared__ int ok;
  ++epoch;
  const unsigned target = epoch * gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(&b->count, 1u);
    for (unsigned int it = 0;; ++it) {
      if (*(volatile unsigned int*)&b->count >= target) break;
      if (*(volatile int*)&b->abort) { ok = 0; break; }
      if (it >= kBarrierLimit) {
        atomicExch(&g_factor_error, 1);
        atomicExch(&b->abort, 1);
        ok = 0;
        break;
      }
      if (it > 64) __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Sum over the block, returned to every thread (red: 32 doubles of shared memory).  The
// warps' partial sums are combined by one warp only: an FP64 instruction occupies a
// sub-partition's FP64 pipe for many cycles on this part, so redundant adds are not free.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
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
  // the scalars in one thread, broadcast through shared memory (an FP64 instruction holds
  // a sub-partition's FP64 pipe for many cycles on this part)
  if (threadIdx.x == 0) {
    const double alpha = x[i];
    double t = 0.0, b = alpha, scale = 0.0;
    if (s2 > 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, s2));
      b = alpha >= 0.0 ? -nrm : nrm;
      t = (b - alpha) / b;
      scale = 1.0 / (alpha - b);
    }
    red[1] = t;
    red[2] = b;
    red[3] = scale;
  }
  __syncthreads();
  const double t = red[1], b = red[2], scale = red[3];
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

// Point-to-point publication of reflection j: every thread's writes of it are ordered
// before the flag (the block's barrier, then thread 0 fences and sets ready[j]).
__device__ void publish_ready(int* ready, int j) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(ready + j, 1);
  }
}
// Bounded wait of the block for ready[j] (thread 0 polls, then fences); false if it gave
// up after kBarrierLimit polls (raising the error word) or another block did.
__device__ bool wait_ready(const int* ready, int j, GridBarrier* b) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    for (unsigned int it = 0;; ++it) {
      if (*(volatile const int*)(ready + j)) break;
      if (*(volatile int*)&b->abort) { ok = 0; break; }
      if (it >= kBarrierLimit) {
        atomicExch(&g_factor_error, 1);
        atomicExch(&b->abort, 1);
        ok = 0;
        break;
      }
      if (it > 64) __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Applies reflection i (vector in vs, factor t) to row r of A, the whole block on the row.
__device__ void lq_update_row_block(double* A, int cols, int i, int r, const double* vs,
                                    double t, double* red) {
  double* ar = A + (size_t)r * cols;
  double d = 0.0;
  for (int c = i + threadIdx.x; c < cols; c += blockDim.x) d = fma(ar[c], vs[c], d);
  d = block_sum(d, red) * t;
  for (int c = i + threadIdx.x; c < cols; c += blockDim.x) ar[c] = fma(-d, vs[c], ar[c]);
  __syncthreads();
}

// The reflections need no grid-wide barrier: a row only ever changes in the block that
// owns it, so the one dependency between blocks is reflection i itself, which its row's
// owner publishes (ready[i]) as soon as that row has received reflections 0..i-1.  The
// owner of row i + 1 therefore applies reflection i to that row first, forms and
// publishes reflection i + 1, and only then updates its other rows, while the other
// blocks run behind it.  ready (k ints) must be zero on entry.
__global__ void __launch_bounds__(kFacThreads)
hh_lq_kernel(double* A, int rows, int cols, int k, double* V, double* tau, double* beta,
             GridBarrier* bar, int* ready) {
  extern __shared__ double vs[];                 // the current reflection vector
  __shared__ double red[32];
  const int nb = gridDim.x, b = blockIdx.x;
  if (b == 0) {
    make_reflection(A, cols, 0, V, tau, beta, red);
    publish_ready(ready, 0);
  }
  for (int i = 0; i < k; ++i) {
    if (!wait_ready(ready, i, bar)) return;
    const double t = __ldcg(tau + i);
    const int nxt = i + 1;
    const bool own_next = nxt < k && nxt % nb == b;
    if (t != 0.0) {
      const double* vi = V + (size_t)i * cols;
      for (int c = i + threadIdx.x; c < cols; c += blockDim.x) vs[c] = __ldcg(vi + c);
      __syncthreads();
      if (own_next) lq_update_row_block(A, cols, i, nxt, vs, t, red);
    }
    if (own_next) {
      make_reflection(A, cols, nxt, V, tau, beta, red);
      publish_ready(ready, nxt);
    }
    if (t != 0.0) {
      // the other rows r > i owned by this block (r = b + nb * m): one warp per row (a
      // lane keeps its columns, the dot product needs only the warp's shuffles) when the
      // block owns at least four of them, else the whole block on each row (the FP64
      // work of a row spread over the four sub-partitions)
      int r0 = i + 1 + ((b - (i + 1) % nb) % nb + nb) % nb;
      if (own_next) r0 += nb;                      // row i + 1 is done
      const int nown = r0 < rows ? (rows - 1 - r0) / nb + 1 : 0;
      if (nown >= 4) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r = r0 + nb * warp; r < rows; r += nb * nw) {
          double* ar = A + (size_t)r * cols;
          double d0 = 0.0, d1 = 0.0;
          for (int c = i + lane; c < cols; c += 64) {
            d0 = fma(ar[c], vs[c], d0);
            if (c + 32 < cols) d1 = fma(ar[c + 32], vs[c + 32], d1);
          }
          double d = d0 + d1;
          for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          d *= t;
          for (int c = i + lane; c < cols; c += 32) ar[c] = fma(-d, vs[c], ar[c]);
        }
      } else {
        for (int r = r0; r < rows; r += nb) lq_update_row_block(A, cols, i, r, vs, t, red);
      }
    }
    __syncthreads();   // vs is reloaded for the next reflection
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
  unsigned epoch = 0;
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
  if (!grid_sync(bar, epoch)) return;
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
    if (!grid_sync(bar, epoch)) return;
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
    if (!grid_sync(bar, epoch)) return;
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
    if (!grid_sync(bar, epoch)) return;
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
      if (!grid_sync(bar, epoch)) return;
    }
  }
}

// The same bidiagonalisation with every block's rows resident in shared memory for the
// whole reduction (rows never change owner: row q of the block is global row b + nb * q,
// held at rows[q * n]), in one grid barrier per step.  What crosses blocks goes through
// global memory, published in step i - 1 for step i:
//   the partial squared norms of column i below the diagonal (part, by step parity), the
//   pivot A[i][i] (alpha) and row i itself (rowg, by step parity) from the owner of row i,
//   and Z_i[c] = sum_{r > i} A[r][i] A[r][c], the unscaled products of the left reflection
//   (FP64 atomics into one of three buffers, so Z may differ in its last bits from run to
//   run).
// Step i then runs in every block without further exchange: the left reflection
// (beta, tau_u, scale) from the norm and the pivot, y = u^T A = row_i + scale Z_i (u_i = 1,
// u_r = scale A[r][i]), the left update of its rows, the right reflection from row i after
// the left update (x = row_i - tau_u y, formed by one warp while the others update the
// rows; each row's left update also accumulates its dot product with x, so the right
// update is one more pass over the row), the right update of its rows (one warp per row),
// and the publications for step i + 1.  The scalar work of a reflection runs in one warp and
// is broadcast through shared memory: an FP64 instruction holds a sub-partition's FP64
// pipe for many cycles on this part, so the other warps must not repeat it.  At the end
// the rows, holding the reflection vectors in place, are written back to A for the
// back-transformation.  zbuf (3 n) must be zero on entry.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// (beta, tau, scale) of the reflection mapping (al, x_1..) with sum x_k^2 = s2 onto
// beta e_0: beta = -sign(al) sqrt(al^2 + s2), tau = (beta - al) / beta,
// scale = 1 / (al - beta); tau = 0 (and beta = al) when s2 = 0.
__device__ __forceinline__ void reflection_scalars(double al, double s2, double& beta,
                                                   double& tau, double& scale) {
  beta = al;
  tau = 0.0;
  scale = 0.0;
  if (s2 > 0.0) {
    const double nrm = sqrt(fma(al, al, s2));
    beta = al >= 0.0 ? -nrm : nrm;
    tau = (beta - al) / beta;
    scale = 1.0 / (al - beta);
  }
}
__global__ void __launch_bounds__(kFacThreads)
hh_bidiag_smem_kernel(double* A, int m, int n, double* d, double* e, double* tau_u,
                      double* tau_v, double* part, double* zbuf, double* alpha, double* rowg,
                      GridBarrier* bar) {
  unsigned epoch = 0;
  extern __shared__ double sm[];
  __shared__ double sc[4];                      // tau_u, scale_u, tau_v, scale_v
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int R = (m - b + nb - 1) / nb;          // rows of this block
  double* rows = sm;                            // R x n
  double* yv = sm + (size_t)R * n;              // y of the current step (n)
  double* wv = yv + n;                          // row i after the left update, x (n)
  double* zr = wv + n;                          // x . row_r beyond the superdiagonal (R)
  for (int q = 0; q < R; ++q)
    for (int c = tid; c < n; c += blockDim.x) rows[(size_t)q * n + c] = A[(size_t)(b + nb * q) * n + c];
  __syncthreads();
  auto qof = [&](int r) { return (r - b) / nb; };            // r % nb == b assumed
  auto q_first = [&](int r0) { return r0 <= b ? 0 : (r0 - b + nb - 1) / nb; };   // first q with row >= r0
  // publications for step j (column j, row j) from this block's rows, which are final
  // for step j: partial norm, unscaled products Z_j, and (owner of row j) row j and pivot
  auto publish = [&](int j) {
    const int qa = q_first(j + 1);
    if (warp == 0) {
      double p2 = 0.0;
      for (int q = qa + lane; q < R; q += 32)
        p2 = fma(rows[(size_t)q * n + j], rows[(size_t)q * n + j], p2);
      p2 = warp_sum(p2);
      if (lane == 0) part[(size_t)(j & 1) * nb + b] = p2;
    }
    if (qa < R) {
      double* zj = zbuf + (size_t)(j % 3) * n;
      for (int c = j + 1 + tid; c < n; c += blockDim.x) {
        double acc = 0.0;
        for (int q = qa; q < R; ++q) acc = fma(rows[(size_t)q * n + j], rows[(size_t)q * n + c], acc);
        atomicAdd(zj + c, acc);
      }
    }
    if (j % nb == b) {
      const double* rj = rows + (size_t)qof(j) * n;
      double* rn = rowg + (size_t)(j & 1) * n;
      for (int c = j + 1 + tid; c < n; c += blockDim.x) rn[c] = rj[c];
      if (tid == 0) alpha[j] = rj[j];
    }
  };
  publish(0);
  if (!grid_sync(bar, epoch)) return;
  for (int i = 0; i < n; ++i) {
    const bool own_i = i % nb == b;
    const int q0 = q_first(i), q1 = q_first(i + 1);
    const double* zi = zbuf + (size_t)(i % 3) * n;
    const double* rg = rowg + (size_t)(i & 1) * n;
    // ---- left reflection from column i (one warp per block forms it)
    if (warp == 0) {
      const double al = __ldcg(alpha + i);
      double s2 = 0.0;
      for (int q = lane; q < nb; q += 32) s2 += __ldcg(part + (size_t)(i & 1) * nb + q);
      s2 = warp_sum(s2);
      double beta, tu, scale;
      reflection_scalars(al, s2, beta, tu, scale);
      if (lane == 0) {
        sc[0] = tu;
        sc[1] = scale;
        if (own_i) {
          d[i] = beta;
          tau_u[i] = tu;
        }
      }
    }
    // meanwhile: row i and Z_i into shared memory
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      wv[c] = __ldcg(rg + c);
      yv[c] = __ldcg(zi + c);
    }
    __syncthreads();
    const double tu = sc[0], scale = sc[1];
    // u below the diagonal (kept in place for the back-transformation)
    if (tu != 0.0)
      for (int q = q1 + tid; q < R; q += blockDim.x) rows[(size_t)q * n + i] *= scale;
    if (i + 1 >= n) break;
    // y = row_i + scale Z_i; row i after the left update
    for (int c = i + 1 + tid; c < n; c += blockDim.x) {
      const double yc = fma(scale, yv[c], wv[c]);
      yv[c] = yc;
      wv[c] = fma(-tu, yc, wv[c]);
    }
    __syncthreads();
    // warp 0 forms the right reflection from x = row i after the left update (in wv)
    // while warps 1.. apply the left update to the block's rows, one warp per row; a row
    // r > i also accumulates its dot product with x beyond the superdiagonal, z_r, so that
    // the right update needs no second pass over it: with w = (1, sv x_{i+2:}),
    // w . row_r = row_r[i+1] + sv z_r
    if (warp == 0) {
      double t2 = 0.0;
      for (int c = i + 2 + lane; c < n; c += 32) t2 = fma(wv[c], wv[c], t2);
      t2 = warp_sum(t2);
      double be, tv, sv;
      reflection_scalars(wv[i + 1], t2, be, tv, sv);
      if (lane == 0) {
        sc[2] = tv;
        sc[3] = sv;
        if (own_i) {
          e[i] = be;
          tau_v[i] = tv;
        }
      }
    } else {
      const int cb = (i + 1) & ~31;
      for (int q = q0 + warp - 1; q < R; q += nw - 1) {
        const bool row_i = own_i && q == q0;
        const double f = tu * (row_i ? 1.0 : rows[(size_t)q * n + i]);
        double* rq = rows + (size_t)q * n;
        double z0 = 0.0, z1 = 0.0;
        for (int c = cb + lane; c < n; c += 64) {
          if (c > i) {
            const double v = tu != 0.0 ? fma(-f, yv[c], rq[c]) : rq[c];
            rq[c] = v;
            if (c > i + 1) z0 = fma(v, wv[c], z0);
          }
          if (c + 32 < n) {
            const double v = tu != 0.0 ? fma(-f, yv[c + 32], rq[c + 32]) : rq[c + 32];
            rq[c + 32] = v;
            if (c + 32 > i + 1) z1 = fma(v, wv[c + 32], z1);
          }
        }
        const double z = warp_sum(z0 + z1);
        if (lane == 0) zr[q] = z;
      }
    }
    __syncthreads();
    const double tv = sc[2], sv = sc[3];
    // right update of the own rows r > i: row_r -= tv (w . row_r) w, each warp on the rows
    // whose dot product it formed; the owner of row i stores w_i right of the superdiagonal
    if (warp > 0) {
      const int cb = (i + 1) & ~31;
      for (int q = q0 + warp - 1; q < R; q += nw - 1) {
        double* rq = rows + (size_t)q * n;
        if (own_i && q == q0) {
          for (int c = cb + lane; c < n; c += 32)
            if (c > i + 1) rq[c] = sv * wv[c];
          continue;
        }
        if (tv == 0.0) continue;
        const double f = tv * fma(sv, zr[q], rq[i + 1]);
        const double fs = f * sv;
        __syncwarp();   // every lane has read rq[i + 1] before its owner changes it
        for (int c = cb + lane; c < n; c += 32) {
          if (c == i + 1) rq[c] -= f;
          else if (c > i + 1) rq[c] = fma(-fs, wv[c], rq[c]);
        }
      }
    }
    __syncthreads();
    publish(i + 1);
    // the buffer read in step i - 1 is cleared for step i + 2
    double* zc = zbuf + (size_t)((i + 2) % 3) * n;
    for (int c = b + nb * tid; c < n; c += nb * blockDim.x) zc[c] = 0.0;
    if (!grid_sync(bar, epoch)) return;
  }
  // rows back to A: u_i below the diagonals, w_i right of the superdiagonals
  __syncthreads();
  for (int q = 0; q < R; ++q)
    for (int c = tid; c < n; c += blockDim.x) A[(size_t)(b + nb * q) * n + c] = rows[(size_t)q * n + c];
}

// Golub-Kahan tridiagonal of B: zero diagonal, off-diagonal t = (d0, e0, d1, e1, ..., d_{n-1});
// its eigenvalues are +-sigma_k, the eigenvector of +sigma is (v0, u0, v1, u1, ...) / sqrt 2
// with B v = sigma u.  Number of its eigenvalues below x: the sign changes of the leading
// principal minors p_j of T - x I (Sturm sequence; Wilkinson, The Algebraic Eigenvalue
// Problem, Ch. 5), by the three-term recurrence p_j = -x p_{j-1} - t_j^2 p_{j-2} on
// T scaled by a power of two to entries <= 1 (nt2[j] = -t_j^2, nt2[0] unused).  Each step
// is one multiply and one fused multiply-add (no division on the dependent chain); signs,
// zero tests and exponents are read from the bits.  The pair (p_{j-1}, p_j) is rescaled by
// a power of two through the exponent fields whenever its larger entry leaves
// [2^-E, 2^E] (exact; an entry pushed below the normal range becomes zero).  With the fused
// multiply-add the computed signs are those of the exact minors of T + F, F a diagonal of
// size <= eps |x| and a relative change <= eps of each t_j^2 (the rounding factors of the
// steps cancel from the signs), as for the pivot recurrence.  A ratio p_j / p_{j-1} below
// 2^-G in magnitude (p_j = 0 included) counts as -2^-G for the next step.  The FP32 form
// (E = 32, G = 40) brackets the values to ~1e-6 at a small fraction of the FP64 cost; the
// FP64 form (E = 256, G = 300) refines them.
__device__ __forceinline__ int expo(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}
__device__ __forceinline__ int expo(float v) { return (__float_as_int(v) >> 23) & 0xff; }
__device__ __forceinline__ bool sign_change(double a, double b) {   // a != 0, sign(a) != sign(b)
  const long long ba = __double_as_longlong(a);
  return ((ba ^ __double_as_longlong(b)) < 0) & ((ba << 1) != 0);
}
__device__ __forceinline__ bool sign_change(float a, float b) {
  const int ba = __float_as_int(a);
  return ((ba ^ __float_as_int(b)) < 0) & ((ba << 1) != 0);
}
// v * 2^s by the exponent field (no floating-point instruction: on this part an FP64
// instruction, even a predicated-off one, costs a slot of the narrow FP64 pipe); a result
// below the normal range (or a zero / subnormal v) becomes a signed zero.
__device__ __forceinline__ double scale_exp(double v, int s) {
  const long long b = __double_as_longlong(v);
  const int ev = (int)((b >> 52) & 0x7ff), en = ev + s;
  return __longlong_as_double((ev == 0 || en <= 0) ? (b & (long long)0x8000000000000000ull)
                                                   : b + ((long long)s << 52));
}
__device__ __forceinline__ double flip_sign(double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
}
template <typename R, int K>
__device__ void tgk_count(const R* nt2, int N, const R (&xs)[K], int (&cnt)[K]) {
  constexpr int bias = sizeof(R) == 8 ? 1023 : 127;
  constexpr int E = sizeof(R) == 8 ? 256 : 32;
  constexpr int G = sizeof(R) == 8 ? 300 : 40;
  R nxs[K], pm[K], p[K];
#pragma unroll
  for (int u = 0; u < K; ++u) {   // K independent counts interleaved (their chains overlap)
    nxs[u] = -xs[u];
    pm[u] = 1;
    p[u] = nxs[u];
    cnt[u] = xs[u] > 0;
  }
  for (int j = 1; j < N; ++j) {
    const R t = nt2[j];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      // guard: p / pm below 2^-G in magnitude counts as -2^-G, i.e. p = -pm 2^-G; the
      // larger entry of the pair is kept near 1.  FP64: by the exponent fields (integer
      // instructions); FP32: by multiplications (the FP32 pipe is wide, integer work is
      // what the FP32 count is bound by)
      if constexpr (sizeof(R) == 8) {
        if (expo(p[u]) + G < expo(pm[u])) p[u] = flip_sign(scale_exp(pm[u], -G));
      } else {
        if (expo(p[u]) + G < expo(pm[u])) p[u] = -pm[u] * 0x1p-40f;
      }
      R pn = fma(t, pm[u], nxs[u] * p[u]);
      cnt[u] += sign_change(pn, p[u]);
      const int emax = max(expo(pn), expo(p[u]));
      if (emax > bias + E || emax < bias - E) {
        if constexpr (sizeof(R) == 8) {
          pn = scale_exp(pn, bias - emax);
          p[u] = scale_exp(p[u], bias - emax);
        } else {
          const float sc = __int_as_float((254 - emax) << 23);   // 2^(127 - emax)
          pn *= sc;
          p[u] *= sc;
        }
      }
      pm[u] = p[u];
      p[u] = pn;
    }
  }
}

// Scale of the Golub-Kahan tridiagonal: 2^ex > max_j |t_j| + |t_{j+1}| (every warp forms
// the same value).
__device__ int tgk_scale_exponent(const double* d, const double* e, int n) {
  const int N = 2 * n, lane = threadIdx.x & 31;
  double bound = 0.0;
  for (int j = 1 + lane; j < N; j += 32) {
    const double t = (j & 1) ? d[j >> 1] : e[(j >> 1) - 1];
    const double tn = j + 1 < N ? (((j + 1) & 1) ? d[(j + 1) >> 1] : e[((j + 1) >> 1) - 1]) : 0.0;
    bound = fmax(bound, fabs(t) + fabs(tn));
  }
  for (int o = 16; o; o >>= 1) bound = fmax(bound, __shfl_xor_sync(0xffffffffu, bound, o));
  bound = fmax(bound, fabs(d[0]));
  int ex = 0;
  frexp(bound > 0.0 ? bound : 1.0, &ex);
  return bound > 0.0 ? ex : 0x7fffffff;   // a zero matrix is flagged
}

// Multisection step shared by both phases: L lanes per value k evaluate the count at
// K points each, L K interior points of [lo, hi] in all, and keep the sub-interval holding
// the eigenvalue of ascending index j (the count crosses j there).
template <int L, int K, typename R>
__device__ void multisect(const R* nt2, int N, int j, bool done, double& lo, double& hi) {
  const int lane = threadIdx.x & 31, sub = lane & (L - 1), base = lane & (32 - L);
  const unsigned mask = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
  constexpr int P = L * K;
  R xs[K];
  int c[K];
#pragma unroll
  for (int u = 0; u < K; ++u)
    xs[u] = (R)(lo + (hi - lo) * (double)(sub * K + u + 1) / (double)(P + 1));
  if (!done) tgk_count<R, K>(nt2, N, xs, c);
  unsigned mine = 0;
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (!done && c[u] > j) mine |= 1u << u;
  const unsigned any = (__ballot_sync(0xffffffffu, mine != 0) >> base) & mask;
  const int fl = any ? __ffs(any) - 1 : 0;
  const unsigned fb = __shfl_sync(0xffffffffu, mine, base + fl);
  if (!done) {
    const int first = any ? fl * K + __ffs(fb) - 1 : P;   // first point above the eigenvalue
    const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / (double)(P + 1);
    const double nhi = first == P ? hi : lo + (hi - lo) * (double)(first + 1) / (double)(P + 1);
    lo = nlo;
    hi = nhi;
  }
}

// Phase 1, FP32: brackets [lo_k, hi_k] (scaled by 2^-ex) of the nev largest singular values,
// descending, to a relative width 2^-20, by multisection of the FP32 count.  Four
// warps per block (one per sub-partition), 32 / L values per warp; -t^2 in shared memory.
template <int L>
__global__ void __launch_bounds__(128)
tgk_bisect32_kernel(const double* d, const double* e, int n, int nev, double* blo, double* bhi) {
  extern __shared__ float nt2f[];
  const int N = 2 * n;
  const int ex = tgk_scale_exponent(d, e, n);
  const bool zero = ex == 0x7fffffff;
  for (int j = 1 + threadIdx.x; j < N; j += blockDim.x) {
    const double t = zero ? 0.0 : ldexp((j & 1) ? d[j >> 1] : e[(j >> 1) - 1], -ex);
    nt2f[j] = (float)(-(t * t));
  }
  __syncthreads();
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) / L;
  const int j = 2 * n - 1 - k;              // ascending index of +sigma_k among the 2n
  double lo = 0.0, hi = zero ? 0.0 : 1.0;   // count(lo) <= j < count(hi), scaled
  bool done = k >= nev;
  for (int pass = 0; pass < 48; ++pass) {
    if (!done && (hi - lo <= 0x1p-20 * hi || hi < 0x1p-120)) done = true;
    if (__all_sync(0xffffffffu, done)) break;
    multisect<L, 1, float>(nt2f, N, j, done, lo, hi);
  }
  if (k < nev && (threadIdx.x & (L - 1)) == 0) {
    blo[k] = lo;
    bhi[k] = hi;
  }
}

// Phase 2, FP64: sigma_k to a relative width 2^-40.  The FP32 bracket is first widened and
// checked with FP64 counts: half of the lanes test lower ends lo (1 - w_c), the other half
// upper ends hi (1 + w_c), w_c from 2^-24 up to ~2^-9 (beyond the worst-case relative error
// of the FP32 phase), and the tightest ends that hold are kept (0 or the bound when none
// does); then L-lane multisection.  sigma[k] = midpoint, unscaled.
template <int L>
__global__ void __launch_bounds__(128)
tgk_refine64_kernel(const double* d, const double* e, int n, int nev, const double* blo,
                    const double* bhi, double* sigma) {
  extern __shared__ double nt2[];
  const int N = 2 * n, lane = threadIdx.x & 31, sub = lane & (L - 1);
  const int ex = tgk_scale_exponent(d, e, n);
  const bool zero = ex == 0x7fffffff;
  for (int j = 1 + threadIdx.x; j < N; j += blockDim.x) {
    const double t = zero ? 0.0 : ldexp((j & 1) ? d[j >> 1] : e[(j >> 1) - 1], -ex);
    nt2[j] = -(t * t);
  }
  __syncthreads();
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) / L;
  const int j = 2 * n - 1 - k;
  bool done = k >= nev || zero;
  double lo = 0.0, hi = zero ? 0.0 : 1.0;
  {
    constexpr int H = L / 2, step = 16 / H;            // candidates per side, log2 spacing
    const double l0 = done ? 0.0 : blo[k], h0 = done ? 0.0 : bhi[k];
    const int c = sub < H ? sub : sub - H;
    const double w = ldexp(1.0, -24 + step * c);
    const double x[1] = {sub < H ? l0 * (1.0 - w) : fmin(h0 * (1.0 + w), 1.0)};
    int cnt[1] = {0};
    if (!done) tgk_count<double, 1>(nt2, N, x, cnt);
    const bool ok = sub < H ? cnt[0] <= j : cnt[0] > j;
    const unsigned grp = (__ballot_sync(0xffffffffu, ok) >> (lane & (32 - L))) &
                         (L == 32 ? 0xffffffffu : ((1u << L) - 1u));
    const unsigned lo_ok = grp & ((1u << H) - 1u), hi_ok = grp >> H;
    if (!done) {
      if (lo_ok) lo = l0 * (1.0 - ldexp(1.0, -24 + step * (__ffs(lo_ok) - 1)));
      if (hi_ok) hi = fmin(h0 * (1.0 + ldexp(1.0, -24 + step * (__ffs(hi_ok) - 1))), 1.0);
    }
  }
  for (int pass = 0; pass < 64; ++pass) {
    if (!done && (hi - lo <= 0x1p-40 * hi || hi < 0x1p-600)) done = true;
    if (__all_sync(0xffffffffu, done)) break;
    multisect<L, 2, double>(nt2, N, j, done, lo, hi);
  }
  if (k < nev && sub == 0) sigma[k] = zero ? 0.0 : ldexp(0.5 * (lo + hi), ex);
}

// Inverse iteration for the kept singular pairs: for k < r, three solves of
// (T - sigma_k I) z = z_prev (T the Golub-Kahan tridiagonal of size N = 2n) by Gaussian
// elimination with partial pivoting on the band (a row interchange whenever the
// subdiagonal entry is the larger one, which fills one second superdiagonal), from a
// start vector that differs per k; writes the u half (side 0: odd entries) or the v half
// (side 1: even entries) of z, normalised, to out[k][:] (n values).  One warp per k: lane
// 0 runs the elimination and the substitutions (sequential by nature) on band factors
// held in shared memory (5 N doubles + N flags; the pivots kept as reciprocals), the warp
// scales and extracts.  Pivots below eps * max|t| are replaced by that size (sigma_k is
// an eigenvalue to working accuracy).
__global__ void tgk_invit_kernel(const double* d, const double* e, int n, const double* sigma,
                                 int r, int side, double* out) {
  extern __shared__ double smem_all[];
  const int N = 2 * n, lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int k = blockIdx.x * (blockDim.x >> 5) + wib;      // one warp per k
  if (k >= r) return;
  // this warp's slice: 5 N doubles + N flag bytes, rounded up to whole doubles
  double* sm = smem_all + (size_t)wib * (5 * (size_t)N + (N + 7) / 8);
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
    // eliminate the subdiagonal entry T[j+1][j] = t(j + 1) column by column; the final
    // pivots are kept as their reciprocals for the substitutions
    for (int j = 0; j + 1 < N; ++j) {
      const double sub = t(j + 1);
      if (fabs(dg[j]) >= fabs(sub)) {
        if (fabs(dg[j]) < tiny) dg[j] = dg[j] < 0.0 ? -tiny : tiny;
        const double inv = 1.0 / dg[j];
        const double f = sub * inv;
        ml[j] = f;
        dg[j + 1] -= f * s1[j];
        dg[j] = inv;
      } else {                                // interchange rows j and j + 1
        const double inv = 1.0 / sub;
        const double f = dg[j] * inv;
        const double r1 = dg[j + 1], r2 = j + 1 < N - 1 ? s1[j + 1] : 0.0;   // row j+1
        dg[j] = inv;
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
    dg[N - 1] = 1.0 / dg[N - 1];
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
        z[j] = v * dg[j];
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
// by the right side (row i beyond the superdiagonal: columns i+2.., off = 1).  One warp per
// column (kApplyCols per block): a lane always owns the entries j = lane mod 32, so a
// reflection needs only the warp's shuffles.  The reflections are staged in shared memory
// g at a time (g >= 1, rows padded to p + 1 against bank conflicts), read from global
// memory once per block, coalesced; g = 0 reads them from global memory directly.  With
// xsm the block's columns are held in shared memory, otherwise they are updated in place.
constexpr int kApplyCols = 4;
__global__ void __launch_bounds__(32 * kApplyCols)
bidiag_apply_kernel(const double* A, int lda, int p, int q, const double* tau, int left, double* X,
                    int r, int g, int xsm) {
  extern __shared__ double x[];           // [kApplyCols x p if xsm], then g x (p + 1)
  __shared__ double taus[16];             // tau of the staged reflections (g <= 16)
  double* vs = x + (xsm ? (size_t)kApplyCols * p : 0);
  const int off = left ? 0 : 1;
  const int ps = p + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto vglob = [&](int i, int j) {        // entry j of v_i, j >= i + off
    return j == i + off ? 1.0 : (left ? A[(size_t)j * lda + i] : A[(size_t)i * lda + j]);
  };
  for (int k0 = blockIdx.x * kApplyCols; k0 < r; k0 += gridDim.x * kApplyCols) {
    const bool active = k0 + warp < r;
    double* xk = xsm ? x + (size_t)warp * p : X + k0 + warp;   // entry j at xk[j * xs]
    const long long xs = xsm ? 1 : r;
    if (xsm)
      for (int j = threadIdx.x; j < p; j += blockDim.x)
#pragma unroll
        for (int v = 0; v < kApplyCols; ++v)
          x[v * p + j] = k0 + v < r ? X[(size_t)j * r + k0 + v] : 0.0;
    __syncthreads();
    const int gs = g > 0 ? g : 1;
    for (int ihi = q; ihi > 0; ihi -= gs) {
      const int ilo = max(0, ihi - gs), cnt = ihi - ilo;
      if (g > 0) {   // stage v_ilo .. v_{ihi-1} (entries from row ilo + off on) and tau
        const int j0 = ilo + off;
        if (threadIdx.x < cnt) taus[threadIdx.x] = tau[ilo + threadIdx.x];
        // eight loads in flight per thread (the copy is latency-bound otherwise)
        const int tot = (p - j0) * cnt;
        for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * blockDim.x) {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            int j = 0, t = 0;
            if (left) { j = j0 + e / cnt; t = e % cnt; }          // row-major: v_i's across
            else { t = e / (p - j0); j = j0 + e % (p - j0); }     // one reflection per row
            v[u] = (e < tot && j >= ilo + t + off) ? vglob(ilo + t, j) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) {
              const int j = left ? j0 + e / cnt : j0 + e % (p - j0);
              const int t = left ? e % cnt : e / (p - j0);
              vs[t * ps + j] = v[u];
            }
          }
        }
        __syncthreads();
      }
      if (active)
        for (int i = ihi - 1; i >= ilo; --i) {
          const double ti = g > 0 ? taus[i - ilo] : tau[i];
          if (ti == 0.0) continue;
          const int j0 = i + off, jb = j0 & ~31;
          const double* vi = vs + (size_t)(i - ilo) * ps;
          double s0 = 0.0, s1 = 0.0;
          for (int j = jb + lane; j < p; j += 64) {
            if (j >= j0) s0 = fma(g > 0 ? vi[j] : vglob(i, j), xk[j * xs], s0);
            if (j + 32 < p) s1 = fma(g > 0 ? vi[j + 32] : vglob(i, j + 32), xk[(j + 32) * xs], s1);
          }
          double sum = s0 + s1;
          for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          const double f = ti * sum;
          for (int j = jb + lane; j < p; j += 32)
            if (j >= j0) xk[j * xs] = fma(-f, g > 0 ? vi[j] : vglob(i, j), xk[j * xs]);
        }
      __syncthreads();
    }
    if (xsm)
      for (int j = threadIdx.x; j < p; j += blockDim.x)
#pragma unroll
        for (int v = 0; v < kApplyCols; ++v)
          if (k0 + v < r) X[(size_t)j * r + k0 + v] = x[v * p + j];
    __syncthreads();
  }
}

// ---- block Gram-Schmidt with CholeskyQR2 panels (all FP64, deterministic reductions)
// Partial inner products of two column blocks over row chunks:
// W[ch][q][c] = sum_{j in chunk ch} X[j][q] Y[j][c] for q < a, c < b <= 32 (chunk: rows
// per chunk, a multiple of 32).  Block (blockIdx.x, ch) covers q in [32 blockIdx.x, +32);
// rows are staged 32 at a time.
__global__ void __launch_bounds__(256)
tsgram_partial_kernel(const double* X, int ldx, int a, const double* Y, int ldy, int b, int rows,
                      int chunk, double* W) {
  __shared__ double xs[32][33];
  __shared__ double ys[32][33];
  const int q0 = blockIdx.x * 32, ch = blockIdx.y, tid = threadIdx.x;
  const int j0 = ch * chunk, j1 = min(rows, j0 + chunk);
  const int qq = tid >> 3, cc = tid & 7;     // outputs (qq, cc + 8 t), t < 4
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int js = j0; js < j1; js += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int jj = e >> 5, col = e & 31, j = js + jj;
      xs[jj][col] = (j < j1 && q0 + col < a) ? X[(size_t)j * ldx + q0 + col] : 0.0;
      ys[jj][col] = (j < j1 && col < b) ? Y[(size_t)j * ldy + col] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const double xv = xs[jj][qq];
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] = fma(xv, ys[jj][cc + 8 * t], acc[t]);
    }
    __syncthreads();
  }
  const int q = q0 + qq;
  if (q < a)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (cc + 8 * t < b) W[((size_t)ch * a + q) * b + cc + 8 * t] = acc[t];
}

// C[q][c] = sum over the nch chunks of W[ch][q][c], in chunk order (a x b, row stride b).
__global__ void tsgram_reduce_kernel(const double* W, int nch, int a, int b, double* C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a * b) return;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += W[(size_t)ch * a * b + e];
  C[e] = s;
}

// Cholesky factor of the w x w (w <= 32) Gram matrix G of a panel, G = R^T R with R upper
// triangular, and Rinv = R^{-1} (row stride w); one warp.  A pivot below kCholFloor (the
// squared norm left of a column, which entered with norm ~1, once its components along
// the panel's earlier columns are removed) marks the panel as numerically dependent:
// *flag is set and Rinv = I, so that the panel is left unchanged for the fallback.
constexpr double kCholFloor = 1e-12;
__global__ void __launch_bounds__(32) chol_inv_kernel(const double* G, int w, double* Rinv,
                                                      int* flag) {
  __shared__ double R[32][33];
  __shared__ double X[32][33];
  __shared__ int bad;
  const int lane = threadIdx.x;
  double dev = 0.0;                         // max |G - I|
  for (int i = 0; i < w; ++i) {
    const double gv = lane < w ? G[i * w + lane] : 0.0;
    R[i][lane] = gv;
    if (lane < w) dev = fmax(dev, fabs(gv - (i == lane ? 1.0 : 0.0)));
  }
  for (int o = 16; o; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
  if (lane == 0) bad = *flag;
  __syncwarp();
  if (dev <= 64 * 2.2204460492503131e-16 || bad) {   // orthonormal already, or given up
    for (int i = 0; i < w; ++i)
      if (lane < w) Rinv[i * w + lane] = i == lane ? 1.0 : 0.0;
    return;
  }
  for (int j = 0; j < w; ++j) {             // right-looking, upper triangle
    const double piv = R[j][j];
    if (!(piv > kCholFloor)) {
      if (lane == 0) bad = 1;
      break;
    }
    const double rjj = sqrt(piv);
    __syncwarp();
    if (lane > j && lane < w) R[j][lane] /= rjj;
    __syncwarp();
    if (lane == 0) R[j][j] = rjj;
    if (lane > j && lane < w) {
      const double rjl = R[j][lane];
      for (int i = j + 1; i <= lane; ++i) R[i][lane] -= R[j][i] * rjl;
    }
    __syncwarp();
  }
  __syncwarp();
  if (bad) {
    if (lane == 0) *flag = 1;
    for (int i = 0; i < w; ++i)
      if (lane < w) Rinv[i * w + lane] = i == lane ? 1.0 : 0.0;
    return;
  }
  // column `lane` of R^{-1} by back substitution: R x = e_lane
  if (lane < w) {
    for (int i = w - 1; i >= 0; --i) {
      double v = i == lane ? 1.0 : 0.0;
      for (int k = i + 1; k <= lane; ++k) v -= R[i][k] * X[k][lane];
      X[i][lane] = i > lane ? 0.0 : v / R[i][i];
    }
  }
  __syncwarp();
  for (int i = 0; i < w; ++i)
    if (lane < w) Rinv[i * w + lane] = X[i][lane];
}

// Y[j][c] = alpha sum_{q < a} X[j][q] C[q][c] + beta Y[j][c] for every row j < rows and
// c < b <= 32 (C: a x b, row stride b).  One warp per row (eight rows per block); C is
// staged in shared memory kMixRows rows at a time.  X may alias Y when a <= 32: the warp
// reads its whole row before it writes.
constexpr int kMixRows = 128;
__global__ void __launch_bounds__(256)
rowmix_kernel(const double* X, int ldx, int a, const double* C, int b, double* Y, int ldy,
              int rows, double alpha, double beta) {
  __shared__ double cs[kMixRows][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + warp;
  double acc = 0.0;
  for (int qc = 0; qc < a; qc += kMixRows) {
    const int qn = min(kMixRows, a - qc);
    __syncthreads();
    for (int e = threadIdx.x; e < kMixRows * 32; e += blockDim.x) {
      const int qq = e >> 5, c = e & 31;
      cs[qq][c] = (qq < qn && c < b) ? C[(size_t)(qc + qq) * b + c] : 0.0;
    }
    __syncthreads();
    if (j < rows)
      for (int q0 = 0; q0 < qn; q0 += 32) {
        const double xv = q0 + lane < qn ? X[(size_t)j * ldx + qc + q0 + lane] : 0.0;
        const int m = min(32, qn - q0);
        for (int qq = 0; qq < m; ++qq)
          acc = fma(__shfl_sync(0xffffffffu, xv, qq), cs[q0 + qq][lane], acc);
      }
  }
  __syncwarp();
  if (j < rows && lane < b) {
    double* yp = Y + (size_t)j * ldy + lane;
    *yp = alpha * acc + (beta != 0.0 ? beta * *yp : 0.0);
  }
}

// Fallback orthonormalisation within a panel of w <= 32 columns (cols c0 .. c0 + w - 1)
// of X (rows x ld, row-major), in one block, run when the panel's CholeskyQR2 found it
// numerically dependent (*flag != 0).  Each column (a unit vector on entry, already
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
panel_mgs_kernel(double* X, int rows, int ld, int c0, int w, const int* flag) {
  if (*(volatile const int*)flag == 0) return;    // the panel's CholeskyQR2 held
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
    set_smem((const void*)tgk_bisect32_kernel<32>, 200 * 1024);
    set_smem((const void*)tgk_refine64_kernel<8>, 200 * 1024);
    set_smem((const void*)tgk_refine64_kernel<16>, 200 * 1024);
    set_smem((const void*)tgk_refine64_kernel<32>, 200 * 1024);
    set_smem((const void*)tgk_invit_kernel, 200 * 1024);
    set_smem((const void*)hh_bidiag_smem_kernel, 200 * 1024);
  });
}

int svd_trunc(const double* M, int rows, int cols, int D_max, double tol, double* P,
              double* discarded, std::vector<double>* sv_out, FactorWork& w, cudaStream_t s) {
  A2_REQUIRE(rows >= 1 && cols >= 1 && D_max >= 1, "SVD: bad sizes");
  A2_REQUIRE(rows <= 12800, "SVD: more than 12800 rows");
  A2_REQUIRE(std::min(rows, cols) <= 2400, "SVD: the smaller dimension exceeds 2400");
  set_attributes();
  const bool left = rows >= cols;                 // bidiagonalise M (left) or M^T (right)
  const int m = left ? rows : cols, n = left ? cols : rows;
  const int nb = std::max(1, std::min(m, num_sms()));
  // scratch: A (m n); d, e, tau_u, tau_v (n each); sigma and its brackets (3n); y (n);
  // Z by step modulo 3 (3n); pivots (n); published rows by step parity (2n); part by step
  // parity (2 nb); ypart (nb n)
  const size_t nA = (size_t)m * n;
  w.a.ensure(sizeof(double) * nA, s);
  w.s.ensure(sizeof(double) * (14 * (size_t)n + 2 * nb + (size_t)nb * n), s);
  w.bar.ensure(sizeof(GridBarrier), s);
  double* A = w.a.as<double>();
  double* d = w.s.as<double>();
  double* e = d + n;
  double* tu = e + n;
  double* tv = tu + n;
  double* sig = tv + n;
  double* y = sig + 3 * n;
  double* zbuf = y + n;
  double* alpha = zbuf + 3 * n;
  double* rowg = alpha + n;
  double* part = rowg + 2 * n;
  double* ypart = part + 2 * nb;
  if (left)
    A2_CUDA(cudaMemcpyAsync(A, M, sizeof(double) * nA, cudaMemcpyDeviceToDevice, s));
  else
    transpose2d<double, double>(M, A, rows, cols, s);
  A2_CUDA(cudaMemsetAsync(w.bar.p, 0, sizeof(GridBarrier), s));
  A2_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, s));
  {
    GridBarrier* bar = w.bar.as<GridBarrier>();
    int mm = m, nn = n;
    const size_t smem = sizeof(double) * (((size_t)cdiv(m, nb) + 2) * n + cdiv(m, nb));
    if (smem <= 200 * 1024) {   // every block's rows resident in shared memory
      A2_CUDA(cudaMemsetAsync(zbuf, 0, sizeof(double) * 3 * (size_t)n, s));
      void* args[] = {&A, &mm, &nn, &d, &e, &tu, &tv, &part, &zbuf, &alpha, &rowg, &bar};
      A2_CUDA(cudaLaunchCooperativeKernel((const void*)hh_bidiag_smem_kernel, dim3(nb),
                                          dim3(kFacThreads), args, smem, s));
    } else {
      void* args[] = {&A, &mm, &nn, &d, &e, &tu, &tv, &part, &ypart, &y, &bar};
      A2_CUDA(cudaLaunchCooperativeKernel((const void*)hh_bidiag_kernel, dim3(nb),
                                          dim3(kFacThreads), args, 0, s));
    }
    count_launch();
  }
  // all n singular values: the discarded weight is summed from the small end (a remainder
  // ||B||_F^2 - sum of the kept sigma^2 would lose the tail to cancellation).  FP32
  // multisection brackets them, FP64 multisection refines the brackets.
  const int nev = n;
  {
    double* blo = sig + n;
    double* bhi = blo + n;
    tgk_bisect32_kernel<32><<<cdiv(nev * 32, 128), 128, sizeof(float) * 2 * (size_t)n, s>>>(
        d, e, n, nev, blo, bhi);
    A2_CHECK_LAUNCH();
    // lanes per value L of the FP64 phase: fewest passes (one to check the bracket, then
    // ~21 bits / log2(2 L + 1)) times the warps that share a sub-partition's FP64 pipe
    const size_t sm2 = sizeof(double) * 2 * (size_t)n;
    int best = 8;
    double best_cost = 1e300;
    for (int L : {8, 16, 32}) {
      const double share = std::ceil((double)cdiv(nev * L, 32) / (4.0 * num_sms()));
      const double cost = (1.0 + std::ceil(21.0 / std::log2(2.0 * L + 1.0))) * std::max(1.0, share);
      if (cost <= best_cost) { best_cost = cost; best = L; }
    }
    const int grid = cdiv(nev * best, 128);
    if (best == 32)
      tgk_refine64_kernel<32><<<grid, 128, sm2, s>>>(d, e, n, nev, blo, bhi, sig);
    else if (best == 16)
      tgk_refine64_kernel<16><<<grid, 128, sm2, s>>>(d, e, n, nev, blo, bhi, sig);
    else
      tgk_refine64_kernel<8><<<grid, 128, sm2, s>>>(d, e, n, nev, blo, bhi, sig);
    A2_CHECK_LAUNCH();
  }
  std::vector<double> sv(nev);
  A2_CUDA(cudaMemcpyAsync(sv.data(), sig, sizeof(double) * nev, cudaMemcpyDeviceToHost, s));
  A2_CUDA(cudaStreamSynchronize(s));
  if (factor_error_flag(true)) throw CudaError("SVD: a bounded grid barrier gave up");
  // smallest r <= D_max whose discarded 2-norm is <= tol * ||sigma|| (at least 1), the
  // tail summed from the small end
  std::vector<double> tail(nev + 1, 0.0);
  for (int k = nev - 1; k >= 0; --k) tail[k] = tail[k + 1] + sv[k] * sv[k];
  int r = nev;
  const double thr = tol * tol * tail[0];
  for (int cand = 1; cand <= nev; ++cand)
    if (tail[cand] <= thr) { r = cand; break; }
  r = std::max(1, std::min(r, D_max));
  if (discarded) *discarded = std::sqrt(std::max(tail[r], 0.0));
  if (sv_out) *sv_out = sv;
  // kept singular vectors of B by inverse iteration, then into the columns of P (rows x r)
  constexpr int W = 32;
  const int npan = cdiv(r, W);
  const int sms = num_sms();
  // Gram chunk: rows per partial sum, so that the widest Gram has about 2 blocks per SM
  auto gram_chunk = [&](int a) {
    const long long want = (long long)rows * cdiv(a, 32) / (2LL * sms);
    return (int)std::max<long long>(32, (want + 31) / 32 * 32);
  };
  const size_t wmax = (size_t)cdiv(rows, 32) * r * W;      // partial sums of any Gram
  w.v.ensure(sizeof(double) * ((size_t)r * n + (size_t)r * W + W * W + wmax) +
                 sizeof(int) * npan, s);
  double* vecs = w.v.as<double>();
  double* C = vecs + (size_t)r * n;
  double* Rinv = C + (size_t)r * W;
  double* Wp = Rinv + W * W;
  int* flags = reinterpret_cast<int*>(Wp + wmax);
  // one warp per kept vector, two per block when both slices fit (their warps then sit on
  // different sub-partitions)
  const size_t inv_slice = sizeof(double) * (5 * 2 * (size_t)n + (2 * (size_t)n + 7) / 8);
  const int ipb = 2 * inv_slice <= 200 * 1024 ? 2 : 1;
  tgk_invit_kernel<<<cdiv(r, ipb), 32 * ipb, ipb * inv_slice, s>>>(d, e, n, sig, r,
                                                                  left ? 0 : 1, vecs);
  A2_CHECK_LAUNCH();
  {
    const long long tot = (long long)rows * r;
    rows_to_cols_kernel<<<(int)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(
        vecs, r, n, rows, P);
    A2_CHECK_LAUNCH();
  }
  A2_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * npan, s));
  // G = X^T Y over the rows of P (X: columns x0 .. x0 + a - 1, Y: y0 .. y0 + b - 1)
  auto gram = [&](int x0, int a, int y0, int b, double* G) {
    const int chunk = gram_chunk(a), nch = cdiv(rows, chunk);
    tsgram_partial_kernel<<<dim3(cdiv(a, 32), nch), 256, 0, s>>>(P + x0, r, a, P + y0, r, b,
                                                                 rows, chunk, Wp);
    A2_CHECK_LAUNCH();
    tsgram_reduce_kernel<<<cdiv(a * b, 256), 256, 0, s>>>(Wp, nch, a, b, G);
    A2_CHECK_LAUNCH();
  };
  // orthonormal columns, panel by panel: classical Gram-Schmidt against the earlier panels
  // (twice), then CholeskyQR2 within the panel (twice: X <- X R^{-1}, G = X^T X = R^T R).
  // Exactly or nearly degenerate singular values give inverse-iteration vectors that only
  // span their singular subspace; a panel found numerically dependent by its Cholesky
  // factorisation is redone by the one-block Gram-Schmidt fallback.
  for (int pi = 0; pi < npan; ++pi) {
    const int c0 = pi * W, wd = std::min(W, r - c0);
    if (c0 > 0)
      for (int pass = 0; pass < 2; ++pass) {
        gram(0, c0, c0, wd, C);              // C[q][c] = sum_j P[j][q] P[j][c0 + c]
        rowmix_kernel<<<cdiv(rows, 8), 256, 0, s>>>(P, r, c0, C, wd, P + c0, r, rows, -1.0, 1.0);
        A2_CHECK_LAUNCH();
      }
    for (int pass = 0; pass < 2; ++pass) {
      gram(c0, wd, c0, wd, C);
      chol_inv_kernel<<<1, 32, 0, s>>>(C, wd, Rinv, flags + pi);
      A2_CHECK_LAUNCH();
      rowmix_kernel<<<cdiv(rows, 8), 256, 0, s>>>(P + c0, r, wd, Rinv, wd, P + c0, r, rows, 1.0,
                                                  0.0);
      A2_CHECK_LAUNCH();
    }
    panel_mgs_kernel<<<1, kFacThreads, 0, s>>>(P, rows, r, c0, wd, flags + pi);
    A2_CHECK_LAUNCH();
  }
  // back to the frame of M: the left reflections of M's bidiagonalisation, or the right
  // ones of M^T's (both act on R^rows)
  {
    const int q = left ? n : std::max(n - 1, 0);
    // the block's columns in shared memory when they fit; reflections staged per pass: as
    // many as fit beside them (at most 16)
    const long long cap = 200LL * 1024 / 8;
    const int xsm = (long long)kApplyCols * rows <= cap / 2 ? 1 : 0;
    const long long room = cap - (xsm ? (long long)kApplyCols * rows : 0);
    const int g = (int)std::max<long long>(0, std::min<long long>(16, room / (rows + 1)));
    const size_t smem =
        sizeof(double) * ((xsm ? (size_t)kApplyCols * rows : 0) + (size_t)g * (rows + 1));
    bidiag_apply_kernel<<<std::min(cdiv(r, kApplyCols), 4 * num_sms()), 32 * kApplyCols, smem,
                          s>>>(A, n, rows, q, left ? tu : tv, left ? 1 : 0, P, r, g, xsm);
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
  w.bar.ensure(sizeof(GridBarrier) + sizeof(int) * (size_t)k, s);
  double* A = w.a.as<double>();
  double* V = w.v.as<double>();
  double* tau = V + (size_t)k * cols;
  double* beta = tau + k;
  A2_CUDA(cudaMemcpyAsync(A, M, sizeof(double) * (size_t)rows * cols, cudaMemcpyDeviceToDevice, s));
  A2_CUDA(cudaMemsetAsync(w.bar.p, 0, sizeof(GridBarrier) + sizeof(int) * (size_t)k, s));
  set_attributes();
  // cooperative launch: every block resident at once (the ready flags rely on it)
  int per_sm = 0;
  A2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hh_lq_kernel, kFacThreads,
                                                        vbytes));
  A2_REQUIRE(per_sm >= 1, "LQ: kernel does not fit on an SM");
  const int grid = std::max(1, std::min({rows, num_sms() * per_sm, num_sms()}));
  GridBarrier* bar = w.bar.as<GridBarrier>();
  int* ready = reinterpret_cast<int*>(bar + 1);
  void* args[] = {&A, &rows, &cols, const_cast<int*>(&k), &V, &tau, &beta, &bar, &ready};
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
