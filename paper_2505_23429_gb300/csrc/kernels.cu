// SIMT GEMM, sparse MPO action, vector and small dense kernels (sm_103a).
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace a2 {

// ----------------------------------------------------------------------------- memory pool
cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  A2_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    A2_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = ~0ull;
    A2_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    int no = 0;
    A2_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no));
    pools[dev] = pool;
  }
  return pools[dev];
}

// ----------------------------------------------------------------------------- launch count
namespace {
std::atomic<long long> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Set while this thread captures a stream into a CUDA graph: the profiler's event pairs
// are then skipped (a replayed graph does not re-record them).
thread_local bool t_capturing = false;
void set_capturing(bool on) { t_capturing = on; }

// ----------------------------------------------------------------------------- profiler
namespace {
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double flops, bytes;
};
struct ProfState {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  long long n[PK_COUNT] = {};
  double ms[PK_COUNT] = {}, fl[PK_COUNT] = {}, by[PK_COUNT] = {};
  std::mutex mu;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    A2_CUDA(cudaEventCreate(&e));
    return e;
  }
  void drain() {
    for (auto& r : recs) {
      A2_CUDA(cudaEventSynchronize(r.b));
      float t = 0.f;
      A2_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      n[r.kind] += 1;
      ms[r.kind] += t;
      fl[r.kind] += r.flops;
      by[r.kind] += r.bytes;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
};
ProfState& P() {
  static ProfState st;
  return st;
}
}  // namespace

void prof_enable(bool on) { P().on = on; }
bool prof_enabled() { return P().on; }

ProfScope::ProfScope(int kind, cudaStream_t stream, double flops, double bytes) : s(stream) {
  ProfState& st = P();
  if (!st.on || t_capturing) return;
  std::lock_guard<std::mutex> g(st.mu);
  ProfRec r{kind, st.get(), st.get(), flops, bytes};
  A2_CUDA(cudaEventRecord(r.a, stream));
  st.recs.push_back(r);
  idx = (int)st.recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx < 0) return;
  ProfState& st = P();
  std::lock_guard<std::mutex> g(st.mu);
  if (idx < (int)st.recs.size()) cudaEventRecord(st.recs[idx].b, s);
}

void prof_read(int kind, long long* launches, double* ms, double* flops, double* bytes) {
  ProfState& st = P();
  std::lock_guard<std::mutex> g(st.mu);
  st.drain();
  if (kind < 0 || kind >= PK_COUNT) throw ArgError("bad profile kind");
  if (launches) *launches = st.n[kind];
  if (ms) *ms = st.ms[kind];
  if (flops) *flops = st.fl[kind];
  if (bytes) *bytes = st.by[kind];
}

void prof_reset() {
  ProfState& st = P();
  std::lock_guard<std::mutex> g(st.mu);
  st.drain();
  for (int k = 0; k < PK_COUNT; ++k) st.n[k] = 0, st.ms[k] = st.fl[k] = st.by[k] = 0.0;
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// ----------------------------------------------------------------------------- SIMT GEMM
template <typename T, typename OutT, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
simt_gemm_kernel(SimtGemm<T, OutT> g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int GX = BN / TN;            // threads along n
  constexpr int GY = BM / TM;            // threads along m
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % GX, ty = tid / GX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  const int b = z / g.splitk, sk = z % g.splitk;
  const T* A = g.A + (long long)b * g.abs;
  const T* B = g.B + (long long)b * g.bbs;
  OutT* C = g.C + (long long)b * g.cbs;
  const int kchunk = ((g.K + g.splitk - 1) / g.splitk + BK - 1) / BK * BK;
  const int kbeg = sk * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  const bool a_kfast = (g.sak == 1);
  const bool b_kfast = (g.sbk == 1);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (a_kfast) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < kend) ? A[(long long)m * g.sam + (long long)k * g.sak] : T(0);
    }
#pragma unroll
    for (int e = tid; e < BN * BK; e += NT) {
      int nn, kk;
      if (b_kfast) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < kend) ? B[(long long)n * g.sbn + (long long)k * g.sbk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * GY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * GX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + i * GY;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + j * GX;
      if (n >= g.N) continue;
      OutT* p = C + (long long)m * g.scm + (long long)n * g.scn;
      const OutT v = (OutT)(g.alpha * acc[i][j]);
      if (g.mode == GEMM_STORE) *p = v;
      else if (g.mode == GEMM_ADD) *p += v;
      else atomicAdd(p, v);
    }
  }
}

template <typename T, typename OutT>
void simt_gemm(const SimtGemm<T, OutT>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  A2_REQUIRE(g.splitk == 1 || g.mode == GEMM_ATOMIC, "split-K needs atomic mode");
  if constexpr (sizeof(T) == 8) {
    constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
    dim3 grid(cdiv(g.N, BN), cdiv(g.M, BM), g.batch * g.splitk);
    A2_REQUIRE(grid.y < 65536 && grid.z < 65536, "GEMM grid too large");
    simt_gemm_kernel<T, OutT, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(g);
  } else {
    constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
    dim3 grid(cdiv(g.N, BN), cdiv(g.M, BM), g.batch * g.splitk);
    A2_REQUIRE(grid.y < 65536 && grid.z < 65536, "GEMM grid too large");
    simt_gemm_kernel<T, OutT, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(g);
  }
  A2_CHECK_LAUNCH();
}

template void simt_gemm<double, double>(const SimtGemm<double, double>&, cudaStream_t);
template void simt_gemm<float, float>(const SimtGemm<float, float>&, cudaStream_t);
template void simt_gemm<float, double>(const SimtGemm<float, double>&, cudaStream_t);

// ----------------------------------------------------------------------------- sparse MPO action
template <typename T> __device__ __forceinline__ float to_f(T x) { return (float)x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <typename T> struct AccT { using type = float; };
template <> struct AccT<double> { using type = double; };

template <typename TO, typename A> __device__ __forceinline__ TO from_acc(A x) { return (TO)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}
template <typename A, typename TI> __device__ __forceinline__ A load_as(const TI* p) {
  return (A)(*p);
}
template <> __device__ __forceinline__ float load_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <typename TI, typename TO, typename V>
__global__ void sparse_rows_kernel(SparseRows<V> sp, SparseGeom g, const TI* __restrict__ in,
                                   TO* __restrict__ out, int rows_per_cta) {
  using Acc = typename AccT<TO>::type;
  const int r0 = blockIdx.x * rows_per_cta;
  const int bz = blockIdx.y;
  const int b1 = bz / g.B2, b2 = bz % g.B2;
  const long long ib = b1 * g.in_b1 + b2 * g.in_b2;
  const long long ob = b1 * g.out_b1 + b2 * g.out_b2;
  const int nr = min(rows_per_cta, sp.nrows - r0);
  const int items = nr * g.veclen;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int r = r0 + it / g.veclen;
    const int v = it % g.veclen;
    Acc acc = Acc(0);
    const int e1 = sp.row_ptr[r + 1];
    for (int e = sp.row_ptr[r]; e < e1; ++e) {
      const long long ci = sp.nz_w[e] * g.in_sw + sp.nz_t[e] * g.in_st;
      acc += (Acc)sp.nz_val[e] * load_as<Acc, TI>(in + ib + ci + v);
    }
    const long long ro = sp.row_w[r] * g.out_sw + sp.row_s[r] * g.out_ss;
    if (g.accumulate) acc += load_as<Acc, TO>(out + ob + ro + v);
    out[ob + ro + v] = from_acc<TO, Acc>(acc);
  }
}

// Output rows per CTA of the vectorised kernels: the CTAs resident at one time then span
// few batches, so the input rows they gather from stay in L2 between their uses.
constexpr int kSparseRowsPerCta = 16;

// Autotuner of the rows per CTA of the vectorised sparse launches (off by default: every
// bond of a sweep is a new shape class, and the trials cost more than the few per cent
// they gain in a single global iteration).  The first launch of a
// shape class (kernel variant, rows, vector length, batches, nonzeros) times 4, 8, 16, 32
// and 64 rows per CTA with CUDA events on the caller's stream and keeps the fastest.  Only
// launches whose output does not depend on its previous contents are tuned (re-running
// them is harmless); the others use kSparseRowsPerCta.
namespace {
struct SparseTuneKey {
  int kid, nrows, veclen, batches;
  long long nnz;
  bool operator<(const SparseTuneKey& o) const {
    if (kid != o.kid) return kid < o.kid;
    if (nrows != o.nrows) return nrows < o.nrows;
    if (veclen != o.veclen) return veclen < o.veclen;
    if (batches != o.batches) return batches < o.batches;
    return nnz < o.nnz;
  }
};
std::mutex g_sp_mu;
std::map<SparseTuneKey, int> g_sp_tune;
std::atomic<bool> g_sp_on{false};   // opt-in (a2_set_autotune bit 1)

template <class Launch>
int sparse_rows_tuned(const SparseTuneKey& key, bool tunable, Launch&& launch, cudaStream_t s) {
  if (!tunable || !g_sp_on.load()) return kSparseRowsPerCta;
  {
    std::lock_guard<std::mutex> g(g_sp_mu);
    auto it = g_sp_tune.find(key);
    if (it != g_sp_tune.end()) return it->second;
  }
  static const int cand[5] = {4, 8, 16, 32, 64};
  cudaEvent_t e0, e1;
  A2_CUDA(cudaEventCreate(&e0));
  A2_CUDA(cudaEventCreate(&e1));
  int best = kSparseRowsPerCta;
  float best_ms = 1e30f;
  for (int c : cand) {
    launch(c);                         // warm-up of this configuration
    A2_CUDA(cudaEventRecord(e0, s));
    launch(c);
    A2_CUDA(cudaEventRecord(e1, s));
    A2_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    A2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> g(g_sp_mu);
  g_sp_tune[key] = best;
  return best;
}
}  // namespace

// Vectorised variant: each lane owns VEC consecutive vector elements (16-byte loads),
// `lpr` lanes cover one row chunk of lpr*VEC elements, a warp serves 32/lpr rows at a
// time.  Grid: x = row blocks, y = vector chunks, z = batch; consecutive CTAs share the
// batch and chunk, so the input rows they re-read stay in L2.
template <typename T> struct Vec16 { static constexpr int N = 16 / sizeof(T); };

template <typename TI, typename A>
__device__ __forceinline__ void load_vec(const TI* p, A (&x)[Vec16<TI>::N]) {
  const uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
  const TI* e = reinterpret_cast<const TI*>(&raw);
#pragma unroll
  for (int i = 0; i < Vec16<TI>::N; ++i) x[i] = load_as<A, TI>(e + i);
}

template <typename TO, typename A, int NV>
__device__ __forceinline__ void store_vec(TO* p, const A (&x)[NV]) {
  if constexpr (sizeof(TO) * NV == 16) {
    __align__(16) TO t[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) t[i] = from_acc<TO, A>(x[i]);
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(t);
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) p[i] = from_acc<TO, A>(x[i]);
  }
}

// U consecutive nonzeros e .. e + U - 1 of one row: their index loads, then their row
// loads, are issued together; the FMAs into acc keep the nonzero order.
template <int U, typename TI, typename V, typename Acc, int NV>
__device__ __forceinline__ void nz_batch(const SparseRows<V>& sp, const SparseGeom& g,
                                         const TI* __restrict__ in, long long ib, int e,
                                         Acc (&acc)[NV]) {
  long long ci[U];
  Acc w[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    ci[u] = __ldg(sp.nz_w + e + u) * g.in_sw + __ldg(sp.nz_t + e + u) * g.in_st;
    w[u] = (Acc)__ldg(sp.nz_val + e + u);
  }
  Acc x[U][NV];
#pragma unroll
  for (int u = 0; u < U; ++u) load_vec<TI, Acc>(in + ib + ci[u], x[u]);
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = fma(w[u], x[u][i], acc[i]);
}

template <typename TI, typename TO, typename V, bool ACC>
__global__ void __launch_bounds__(256)
sparse_rows_vec_kernel(SparseRows<V> sp, SparseGeom g, const TI* __restrict__ in,
                       TO* __restrict__ out, int lpr, int rows_per_cta) {
  using Acc = typename AccT<TO>::type;
  constexpr int NV = Vec16<TI>::N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpw = 32 / lpr;                           // rows served by a warp at once
  const int slot = lane / lpr, l = lane % lpr;
  const int v0 = blockIdx.y * (lpr * NV) + l * NV;
  const int bz = blockIdx.z;
  const int b1 = bz / g.B2, b2 = bz % g.B2;
  const long long ib = b1 * g.in_b1 + b2 * g.in_b2 + v0;
  const long long ob = b1 * g.out_b1 + b2 * g.out_b2 + v0;
  const int r_beg = blockIdx.x * rows_per_cta;
  const int r_end = min(sp.nrows, r_beg + rows_per_cta);
  const int step = (blockDim.x >> 5) * rpw;
  if (v0 >= g.veclen) return;
  for (int r = r_beg + warp * rpw + slot; r < r_end; r += step) {
    Acc acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = Acc(0);
    const int e1 = __ldg(sp.row_ptr + r + 1);
    int e = __ldg(sp.row_ptr + r);
    // four nonzeros at a time: their index loads, then their row loads, are issued
    // together (more loads in flight; eight at a time cost more in occupancy than they
    // gained); the FMAs keep the nonzero order
    for (; e + 4 <= e1; e += 4) nz_batch<4, TI, V, Acc, NV>(sp, g, in, ib, e, acc);
    for (; e < e1; ++e) {
      const long long ci = __ldg(sp.nz_w + e) * g.in_sw + __ldg(sp.nz_t + e) * g.in_st;
      const Acc w = (Acc)__ldg(sp.nz_val + e);
      Acc x[NV];
      load_vec<TI, Acc>(in + ib + ci, x);
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = fma(w, x[i], acc[i]);
    }
    const long long ro = __ldg(sp.row_w + r) * g.out_sw + __ldg(sp.row_s + r) * g.out_ss;
    if constexpr (ACC) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += load_as<Acc, TO>(out + ob + ro + i);
    }
    store_vec<TO, Acc, NV>(out + ob + ro, acc);
  }
}

// x = hi + mid + lo with each part rounded to BF16 (three 8-bit mantissa slices)
template <typename A>
__device__ __forceinline__ void split3(A x, __nv_bfloat16& h, __nv_bfloat16& m,
                                       __nv_bfloat16& l) {
  h = __float2bfloat16_rn((float)x);
  const A r1 = x - (A)__bfloat162float(h);
  m = __float2bfloat16_rn((float)r1);
  const A r2 = r1 - (A)__bfloat162float(m);
  l = __float2bfloat16_rn((float)r2);
}

// Same as sparse_rows_vec_kernel with the output split into three BF16 planes.
template <typename TI, typename V, bool PLANES, bool ADD>
__global__ void __launch_bounds__(256)
sparse_rows_split3_kernel(SparseRows<V> sp, SparseGeom g, const TI* __restrict__ in,
                          long long in_plane, const float* __restrict__ add,
                          __nv_bfloat16* __restrict__ out, long long plane, int lpr,
                          int rows_per_cta) {
  using Acc = float;
  constexpr int NV = Vec16<TI>::N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpw = 32 / lpr;
  const int slot = lane / lpr, l = lane % lpr;
  const int v0 = blockIdx.y * (lpr * NV) + l * NV;
  const int bz = blockIdx.z;
  const int b1 = bz / g.B2, b2 = bz % g.B2;
  const long long ib = b1 * g.in_b1 + b2 * g.in_b2 + v0;
  const long long ob = b1 * g.out_b1 + b2 * g.out_b2 + v0;
  const int r_beg = blockIdx.x * rows_per_cta;
  const int r_end = min(sp.nrows, r_beg + rows_per_cta);
  const int step = (blockDim.x >> 5) * rpw;
  if (v0 >= g.veclen) return;
  for (int r = r_beg + warp * rpw + slot; r < r_end; r += step) {
    Acc acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = Acc(0);
    const int e1 = __ldg(sp.row_ptr + r + 1);
    int e = __ldg(sp.row_ptr + r);
    if constexpr (!PLANES) {   // four nonzeros at a time, as in sparse_rows_vec_kernel
      for (; e + 4 <= e1; e += 4) nz_batch<4, TI, V, Acc, NV>(sp, g, in, ib, e, acc);
    }
    for (; e < e1; ++e) {
      const long long ci = __ldg(sp.nz_w + e) * g.in_sw + __ldg(sp.nz_t + e) * g.in_st;
      const Acc w = (Acc)__ldg(sp.nz_val + e);
      Acc x[NV];
      load_vec<TI, Acc>(in + ib + ci, x);
      if constexpr (PLANES) {
        Acc x1[NV], x2[NV];
        load_vec<TI, Acc>(in + ib + ci + in_plane, x1);
        load_vec<TI, Acc>(in + ib + ci + 2 * in_plane, x2);
#pragma unroll
        for (int i = 0; i < NV; ++i) x[i] += x1[i] + x2[i];
      }
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = fma(w, x[i], acc[i]);
    }
    const long long ro = __ldg(sp.row_w + r) * g.out_sw + __ldg(sp.row_s + r) * g.out_ss;
    if constexpr (ADD) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += add[ob + ro + i];
    }
    __nv_bfloat16* o = out + ob + ro;
    // NV consecutive values per plane in one vector store (8 or 16 bytes)
    __align__(16) __nv_bfloat16 h[NV], m[NV], lo[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) split3<Acc>(acc[i], h[i], m[i], lo[i]);
    if constexpr (NV == 8) {
      *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(h);
      *reinterpret_cast<uint4*>(o + plane) = *reinterpret_cast<const uint4*>(m);
      *reinterpret_cast<uint4*>(o + 2 * plane) = *reinterpret_cast<const uint4*>(lo);
    } else {
      static_assert(NV == 4, "split3 stores: 4 or 8 values per lane");
      *reinterpret_cast<uint2*>(o) = *reinterpret_cast<const uint2*>(h);
      *reinterpret_cast<uint2*>(o + plane) = *reinterpret_cast<const uint2*>(m);
      *reinterpret_cast<uint2*>(o + 2 * plane) = *reinterpret_cast<const uint2*>(lo);
    }
  }
}

// scalar fallback of the split3 stage (rows not 16-byte aligned)
template <typename TI, typename V>
__global__ void sparse_rows_split3_scalar(SparseRows<V> sp, SparseGeom g, const TI* __restrict__ in,
                                          long long in_plane, const float* __restrict__ add,
                                          __nv_bfloat16* __restrict__ out, long long plane,
                                          int rows_per_cta) {
  const int r0 = blockIdx.x * rows_per_cta;
  const int b1 = blockIdx.y / g.B2, b2 = blockIdx.y % g.B2;
  const long long ib = b1 * g.in_b1 + b2 * g.in_b2;
  const long long ob = b1 * g.out_b1 + b2 * g.out_b2;
  const int nr = min(rows_per_cta, sp.nrows - r0);
  for (int it = threadIdx.x; it < nr * g.veclen; it += blockDim.x) {
    const int r = r0 + it / g.veclen, v = it % g.veclen;
    float acc = 0.f;
    for (int e = sp.row_ptr[r]; e < sp.row_ptr[r + 1]; ++e) {
      const TI* p = in + ib + sp.nz_w[e] * g.in_sw + sp.nz_t[e] * g.in_st + v;
      float x = load_as<float, TI>(p);
      if (in_plane) x += load_as<float, TI>(p + in_plane) + load_as<float, TI>(p + 2 * in_plane);
      acc += (float)sp.nz_val[e] * x;
    }
    const long long o = ob + sp.row_w[r] * g.out_sw + sp.row_s[r] * g.out_ss + v;
    if (add) acc += add[o];
    __nv_bfloat16 h, m, l;
    split3<float>(acc, h, m, l);
    out[o] = h;
    out[plane + o] = m;
    out[2 * plane + o] = l;
  }
}

template <typename TI, typename V>
void sparse_rows_apply_split3(const SparseRows<V>& sp, const SparseGeom& g, const TI* in,
                              long long in_plane, const float* add, __nv_bfloat16* out,
                              long long plane, cudaStream_t s) {
  if (sp.nrows == 0 || g.veclen == 0) return;
  constexpr int NV = Vec16<TI>::N;
  if constexpr (sizeof(TI) != 2) A2_REQUIRE(in_plane == 0, "input planes need BF16 input");
  auto al = [](long long x) { return x % NV == 0; };
  if (!(al(g.veclen) && al(g.in_sw) && al(g.in_st) && al(g.in_b1) && al(g.in_b2) &&
        al(in_plane) && reinterpret_cast<uintptr_t>(in) % 16 == 0 && al(g.out_sw) &&
        al(g.out_ss) && al(g.out_b1) && al(g.out_b2) && al(plane) &&
        reinterpret_cast<uintptr_t>(out) % (2 * NV) == 0)) {
    const int rows = std::min(64, std::max(1, 2048 / g.veclen));
    dim3 grid(cdiv(sp.nrows, rows), g.B1 * g.B2);
    A2_REQUIRE(grid.y < 65536, "sparse grid too large");
    sparse_rows_split3_scalar<TI, V><<<grid, 256, 0, s>>>(sp, g, in, in_plane, add, out, plane,
                                                         rows);
    A2_CHECK_LAUNCH();
    return;
  }
  int lpr = 1;
  while (lpr < 32 && lpr * NV < g.veclen) lpr *= 2;
  const int chunks = cdiv(g.veclen, lpr * NV);
  A2_REQUIRE(chunks < 65536 && g.B1 * g.B2 < 65536, "sparse grid too large");
  auto kern = in_plane ? (add ? sparse_rows_split3_kernel<TI, V, true, true>
                               : sparse_rows_split3_kernel<TI, V, true, false>)
                      : (add ? sparse_rows_split3_kernel<TI, V, false, true>
                             : sparse_rows_split3_kernel<TI, V, false, false>);
  auto launch = [&](int rows) {
    dim3 grid(cdiv(sp.nrows, rows), chunks, g.B1 * g.B2);
    kern<<<grid, 256, 0, s>>>(sp, g, in, in_plane, add, out, plane, lpr, rows);
    A2_CHECK_LAUNCH();
  };
  const SparseTuneKey key{100 + (int)sizeof(TI) * 4 + (in_plane ? 2 : 0) + (add ? 1 : 0),
                          sp.nrows, g.veclen, g.B1 * g.B2, sp.nnz_total};
  launch(sparse_rows_tuned(key, true, launch, s));
}
template void sparse_rows_apply_split3<float, float>(const SparseRows<float>&, const SparseGeom&,
                                                     const float*, long long, const float*,
                                                     __nv_bfloat16*, long long, cudaStream_t);
template void sparse_rows_apply_split3<__nv_bfloat16, float>(const SparseRows<float>&,
                                                             const SparseGeom&,
                                                             const __nv_bfloat16*, long long,
                                                             const float*, __nv_bfloat16*,
                                                             long long, cudaStream_t);

template <typename TI>
__global__ void split3_ld_kernel(const TI* in, long long rows, long long cols,
                                 __nv_bfloat16* out, long long ld, long long plane) {
  const long long n = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    __nv_bfloat16 h, m, l;
    split3<double>((double)in[e], h, m, l);
    const long long o = r * ld + c;
    out[o] = h;
    out[plane + o] = m;
    out[2 * plane + o] = l;
  }
}
template <typename TI>
void split3_ld(const TI* in, long long rows, long long cols, __nv_bfloat16* out, long long ld,
               long long plane, cudaStream_t s) {
  if (!rows || !cols) return;
  split3_ld_kernel<TI><<<grid_for(rows * cols), 256, 0, s>>>(in, rows, cols, out, ld, plane);
  A2_CHECK_LAUNCH();
}
template void split3_ld<float>(const float*, long long, long long, __nv_bfloat16*, long long,
                               long long, cudaStream_t);
template void split3_ld<double>(const double*, long long, long long, __nv_bfloat16*, long long,
                                long long, cudaStream_t);

// out planes (cols x ld) = split3 of in^T, in: rows x cols row-major (FP64 or FP32)
template <typename TI>
__global__ void transpose_split3_kernel(const TI* in, int rows, int cols, __nv_bfloat16* out,
                                        long long ld, long long plane) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = (double)in[(long long)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int c = bx + j, r = by + threadIdx.x;
    if (r < rows && c < cols) {
      __nv_bfloat16 h, m, l;
      split3<double>(tile[threadIdx.x][j], h, m, l);
      const long long o = (long long)c * ld + r;
      out[o] = h;
      out[plane + o] = m;
      out[2 * plane + o] = l;
    }
  }
}
template <typename TI>
void transpose_split3(const TI* in, int rows, int cols, __nv_bfloat16* out, long long ld,
                      long long plane, cudaStream_t s) {
  if (!rows || !cols) return;
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32));
  A2_REQUIRE(grid.y < 65536, "transpose grid too large");
  transpose_split3_kernel<TI><<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, out, ld, plane);
  A2_CHECK_LAUNCH();
}
template void transpose_split3<double>(const double*, int, int, __nv_bfloat16*, long long,
                                       long long, cudaStream_t);
template void transpose_split3<float>(const float*, int, int, __nv_bfloat16*, long long,
                                      long long, cudaStream_t);

template <typename TI, typename TO, typename V>
void sparse_rows_apply(const SparseRows<V>& sp, const SparseGeom& g, const TI* in, TO* out,
                       cudaStream_t s) {
  if (sp.nrows == 0 || g.veclen == 0) return;
  constexpr int NV = Vec16<TI>::N;
  auto al = [](long long x) { return x % NV == 0; };
  const bool vec_ok = al(g.veclen) && al(g.in_sw) && al(g.in_st) && al(g.out_sw) &&
                      al(g.out_ss) && al(g.in_b1) && al(g.in_b2) && al(g.out_b1) &&
                      al(g.out_b2) && (reinterpret_cast<uintptr_t>(in) % 16 == 0) &&
                      (reinterpret_cast<uintptr_t>(out) % (sizeof(TO) * NV) == 0);
  if (vec_ok) {
    int lpr = 1;
    while (lpr < 32 && lpr * NV < g.veclen) lpr *= 2;
    const int chunks = cdiv(g.veclen, lpr * NV);
    A2_REQUIRE(chunks < 65536 && g.B1 * g.B2 < 65536, "sparse grid too large");
    auto launch = [&](int rows) {
      dim3 grid(cdiv(sp.nrows, rows), chunks, g.B1 * g.B2);
      if (g.accumulate)
        sparse_rows_vec_kernel<TI, TO, V, true><<<grid, 256, 0, s>>>(sp, g, in, out, lpr, rows);
      else
        sparse_rows_vec_kernel<TI, TO, V, false><<<grid, 256, 0, s>>>(sp, g, in, out, lpr, rows);
      A2_CHECK_LAUNCH();
    };
    const SparseTuneKey key{(int)(sizeof(TI) * 16 + sizeof(TO)), sp.nrows, g.veclen,
                            g.B1 * g.B2, sp.nnz_total};
    launch(sparse_rows_tuned(key, !g.accumulate && (const void*)in != (const void*)out,
                             launch, s));
    return;
  }
  int rows = max(1, 2048 / g.veclen);
  rows = min(rows, 64);
  dim3 grid(cdiv(sp.nrows, rows), g.B1 * g.B2);
  A2_REQUIRE(grid.y < 65536, "sparse grid too large");
  sparse_rows_kernel<TI, TO, V><<<grid, 256, 0, s>>>(sp, g, in, out, rows);
  A2_CHECK_LAUNCH();
}

// Double-float multiply-add (Dekker's exact product via FMA, Knuth's two-sum; the
// product of the two low parts, below 2^-48 of the result, is dropped).
__device__ __forceinline__ void df_fma(float& ah, float& al, float wh, float wl, float xh,
                                       float xl) {
  const float p = __fmul_rn(wh, xh);
  const float pe = __fmaf_rn(wh, xh, -p);
  const float q = __fmaf_rn(wh, xl, __fmaf_rn(wl, xh, pe));
  const float s = __fadd_rn(ah, p);
  const float bp = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  ah = s;
  al = __fadd_rn(al, __fadd_rn(err, q));
}

// NV = 4: float4 rows (16-byte aligned); NV = 1: any alignment.
template <bool OUT64, int NV>
__global__ void __launch_bounds__(256)
sparse_rows_df_kernel(SparseRows<float> sp, SparseGeom g, const float* __restrict__ ih,
                      long long in_plane, float* __restrict__ oh, long long out_plane,
                      double* __restrict__ o64, int lpr, int rows_per_cta) {
  const float* il = ih + in_plane;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpw = 32 / lpr;
  const int slot = lane / lpr, l = lane % lpr;
  const int v0 = blockIdx.y * (lpr * NV) + l * NV;
  const int bz = blockIdx.z;
  const int b1 = bz / g.B2, b2 = bz % g.B2;
  const long long ib = b1 * g.in_b1 + b2 * g.in_b2 + v0;
  const long long ob = b1 * g.out_b1 + b2 * g.out_b2 + v0;
  const int r_beg = blockIdx.x * rows_per_cta;
  const int r_end = min(sp.nrows, r_beg + rows_per_cta);
  const int step = (blockDim.x >> 5) * rpw;
  if (v0 >= g.veclen) return;
  for (int r = r_beg + warp * rpw + slot; r < r_end; r += step) {
    float ah[NV], al[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) ah[i] = al[i] = 0.f;
    const int e1 = __ldg(sp.row_ptr + r + 1);
    for (int e = __ldg(sp.row_ptr + r); e < e1; ++e) {
      const long long ci = __ldg(sp.nz_w + e) * g.in_sw + __ldg(sp.nz_t + e) * g.in_st;
      const float wh = __ldg(sp.nz_val + e), wl = __ldg(sp.nz_lo + e);
      if constexpr (NV == 4) {
        const float4 xh = __ldg(reinterpret_cast<const float4*>(ih + ib + ci));
        const float4 xl = __ldg(reinterpret_cast<const float4*>(il + ib + ci));
        df_fma(ah[0], al[0], wh, wl, xh.x, xl.x);
        df_fma(ah[1], al[1], wh, wl, xh.y, xl.y);
        df_fma(ah[2], al[2], wh, wl, xh.z, xl.z);
        df_fma(ah[3], al[3], wh, wl, xh.w, xl.w);
      } else {
        df_fma(ah[0], al[0], wh, wl, __ldg(ih + ib + ci), __ldg(il + ib + ci));
      }
    }
    const long long ro = __ldg(sp.row_w + r) * g.out_sw + __ldg(sp.row_s + r) * g.out_ss;
    if constexpr (OUT64) {
#pragma unroll
      for (int i = 0; i < NV; ++i) o64[ob + ro + i] = (double)ah[i] + (double)al[i];
    } else {
      float h[NV], lo[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) {   // renormalise: |lo| <= ulp(hi) / 2
        const float s = __fadd_rn(ah[i], al[i]);
        h[i] = s;
        lo[i] = __fsub_rn(al[i], __fsub_rn(s, ah[i]));
      }
      if constexpr (NV == 4) {
        *reinterpret_cast<float4*>(oh + ob + ro) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(oh + out_plane + ob + ro) =
            make_float4(lo[0], lo[1], lo[2], lo[3]);
      } else {
        oh[ob + ro] = h[0];
        oh[out_plane + ob + ro] = lo[0];
      }
    }
  }
}

void sparse_rows_apply_df(const SparseRows<float>& sp, const SparseGeom& g, const float* in_hi,
                          long long in_plane, float* out_hi, long long out_plane, double* out64,
                          cudaStream_t s) {
  if (sp.nrows == 0 || g.veclen == 0) return;
  A2_REQUIRE(sp.nz_lo && !g.accumulate, "double-float sparse action: bad arguments");
  auto al = [](long long x) { return x % 4 == 0; };
  const bool vec = al(g.veclen) && al(g.in_sw) && al(g.in_st) && al(g.out_sw) &&
                   al(g.out_ss) && al(g.in_b1) && al(g.in_b2) && al(g.out_b1) &&
                   al(g.out_b2) && al(in_plane) && al(out_plane) &&
                   reinterpret_cast<uintptr_t>(in_hi) % 16 == 0 &&
                   (out64 || reinterpret_cast<uintptr_t>(out_hi) % 16 == 0);
  const int nv = vec ? 4 : 1;
  int lpr = 1;
  while (lpr < 32 && lpr * nv < g.veclen) lpr *= 2;
  const int chunks = cdiv(g.veclen, lpr * nv);
  A2_REQUIRE(chunks < 65536 && g.B1 * g.B2 < 65536, "sparse grid too large");
  auto launch = [&](int rows) {
    dim3 grid(cdiv(sp.nrows, rows), chunks, g.B1 * g.B2);
    if (vec && out64)
      sparse_rows_df_kernel<true, 4><<<grid, 256, 0, s>>>(sp, g, in_hi, in_plane, nullptr, 0,
                                                          out64, lpr, rows);
    else if (vec)
      sparse_rows_df_kernel<false, 4><<<grid, 256, 0, s>>>(sp, g, in_hi, in_plane, out_hi,
                                                           out_plane, nullptr, lpr, rows);
    else if (out64)
      sparse_rows_df_kernel<true, 1><<<grid, 256, 0, s>>>(sp, g, in_hi, in_plane, nullptr, 0,
                                                          out64, lpr, rows);
    else
      sparse_rows_df_kernel<false, 1><<<grid, 256, 0, s>>>(sp, g, in_hi, in_plane, out_hi,
                                                           out_plane, nullptr, lpr, rows);
    A2_CHECK_LAUNCH();
  };
  const SparseTuneKey key{200 + (vec ? 2 : 0) + (out64 ? 1 : 0), sp.nrows, g.veclen,
                          g.B1 * g.B2, sp.nnz_total};
  launch(sparse_rows_tuned(key, true, launch, s));
}

template void sparse_rows_apply<double, double, double>(const SparseRows<double>&,
                                                        const SparseGeom&, const double*,
                                                        double*, cudaStream_t);
template void sparse_rows_apply<float, float, float>(const SparseRows<float>&, const SparseGeom&,
                                                     const float*, float*, cudaStream_t);
template void sparse_rows_apply<__nv_bfloat16, __nv_bfloat16, float>(
    const SparseRows<float>&, const SparseGeom&, const __nv_bfloat16*, __nv_bfloat16*,
    cudaStream_t);
template void sparse_rows_apply<__nv_bfloat16, float, float>(const SparseRows<float>&,
                                                             const SparseGeom&,
                                                             const __nv_bfloat16*, float*,
                                                             cudaStream_t);
template void sparse_rows_apply<float, __nv_bfloat16, float>(const SparseRows<float>&,
                                                             const SparseGeom&, const float*,
                                                             __nv_bfloat16*, cudaStream_t);

// ----------------------------------------------------------------------------- permutes
template <typename TI, typename TO>
__global__ void permute_swap01_kernel(const TI* in, TO* out, int d0, int d1, int d2) {
  const long long n = (long long)d0 * d1 * d2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % d2);
    const long long ij = e / d2;
    const int j = (int)(ij % d1);
    const int i = (int)(ij / d1);
    out[e] = (TO)in[((long long)j * d0 + i) * d2 + k];
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* in, TO* out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (TO)in[e];
}
template <>
__global__ void convert_kernel<double, __nv_bfloat16>(const double* in, __nv_bfloat16* out,
                                                      long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = __double2bfloat16(in[e]);
}
template <>
__global__ void convert_kernel<float, __nv_bfloat16>(const float* in, __nv_bfloat16* out,
                                                     long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(in[e]);
}

template <typename TO> __device__ __forceinline__ TO cvt_out(double v) { return (TO)v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}

template <typename TI, typename TO>
__global__ void transpose_kernel(const TI* in, TO* out, int rows, int cols, long long ld) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = (double)in[(long long)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int c = bx + j, r = by + threadIdx.x;
    if (r < rows && c < cols) out[(long long)c * ld + r] = cvt_out<TO>(tile[threadIdx.x][j]);
  }
}

template <typename TI, typename TO>
__global__ void convert_ld_kernel(const TI* in, TO* out, long long rows, long long cols,
                                  long long ld) {
  const long long n = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    out[r * ld + c] = cvt_out<TO>((double)in[e]);
  }
}


template <typename TI, typename TO>
void permute_swap01(const TI* in, TO* out, int d0, int d1, int d2, cudaStream_t s) {
  long long n = (long long)d0 * d1 * d2;
  if (!n) return;
  permute_swap01_kernel<TI, TO><<<grid_for(n), 256, 0, s>>>(in, out, d0, d1, d2);
  A2_CHECK_LAUNCH();
}
template <typename TI, typename TO>
void convert(const TI* in, TO* out, long long n, cudaStream_t s) {
  if (!n) return;
  convert_kernel<TI, TO><<<grid_for(n), 256, 0, s>>>(in, out, n);
  A2_CHECK_LAUNCH();
}
template <typename TI, typename TO>
void transpose2d_ld(const TI* in, TO* out, int rows, int cols, long long ld, cudaStream_t s) {
  if (!rows || !cols) return;
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32));
  A2_REQUIRE(grid.y < 65536, "transpose grid too large");
  transpose_kernel<TI, TO><<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols, ld);
  A2_CHECK_LAUNCH();
}
template <typename TI, typename TO>
void transpose2d(const TI* in, TO* out, int rows, int cols, cudaStream_t s) {
  transpose2d_ld<TI, TO>(in, out, rows, cols, rows, s);
}
template <typename TI, typename TO>
void convert_ld(const TI* in, TO* out, long long rows, long long cols, long long ld,
                cudaStream_t s) {
  if (!rows || !cols) return;
  convert_ld_kernel<TI, TO><<<grid_for(rows * cols), 256, 0, s>>>(in, out, rows, cols, ld);
  A2_CHECK_LAUNCH();
}
template void permute_swap01<double, double>(const double*, double*, int, int, int, cudaStream_t);
template void permute_swap01<float, float>(const float*, float*, int, int, int, cudaStream_t);
template void permute_swap01<double, float>(const double*, float*, int, int, int, cudaStream_t);
template void convert<double, float>(const double*, float*, long long, cudaStream_t);
template void convert<float, double>(const float*, double*, long long, cudaStream_t);
template void convert<double, __nv_bfloat16>(const double*, __nv_bfloat16*, long long, cudaStream_t);
template void convert<float, __nv_bfloat16>(const float*, __nv_bfloat16*, long long, cudaStream_t);
template void transpose2d<double, double>(const double*, double*, int, int, cudaStream_t);
template void transpose2d<double, float>(const double*, float*, int, int, cudaStream_t);
template void transpose2d<double, __nv_bfloat16>(const double*, __nv_bfloat16*, int, int,
                                                 cudaStream_t);
template void transpose2d_ld<double, __nv_bfloat16>(const double*, __nv_bfloat16*, int, int,
                                                    long long, cudaStream_t);
template void convert_ld<double, __nv_bfloat16>(const double*, __nv_bfloat16*, long long,
                                                long long, long long, cudaStream_t);
template void convert_ld<float, __nv_bfloat16>(const float*, __nv_bfloat16*, long long,
                                               long long, long long, cudaStream_t);

// ----------------------------------------------------------------------------- vector kernels
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[j * kReduceBlocks + block] = sum over the block's grid-stride slice of V_j . w
__global__ void dot_multi_partial(const double* __restrict__ V, long long ldv, int k,
                                  const double* __restrict__ w, long long n,
                                  double* __restrict__ partial) {
  __shared__ double red[8][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j0 = 0; j0 < k; j0 += 8) {
    const int jn = min(8, k - j0);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < jn) acc[q] = fma(V[(long long)(j0 + q) * ldv + i], wi, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double v = warp_sum(acc[q]);
      if (lane == 0) red[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < jn) {
      double t = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[threadIdx.x][ww];
      partial[(long long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void reduce_partials(const double* __restrict__ partial, int nb, int k,
                                double* __restrict__ out) {
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[(long long)j * nb + b];
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[j] = t;
  }
}

void dot_multi(const double* V, long long ldv, int k, const double* w, long long n,
               double* partial, double* out, cudaStream_t s) {
  if (k <= 0) return;
  dot_multi_partial<<<kReduceBlocks, 256, 0, s>>>(V, ldv, k, w, n, partial);
  A2_CHECK_LAUNCH();
  reduce_partials<<<k, 256, 0, s>>>(partial, kReduceBlocks, k, out);
  A2_CHECK_LAUNCH();
}

__global__ void gemv_sub_kernel(const double* __restrict__ V, long long ldv, int k,
                                const double* __restrict__ h, double* __restrict__ w,
                                long long n, int set_mode) {
  __shared__ double hs[64];
  if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(hs[j], V[(long long)j * ldv + i], acc);
    if (set_mode) w[i] = acc; else w[i] -= acc;
  }
}

void gemv_sub(const double* V, long long ldv, int k, const double* h, double* w, long long n,
              cudaStream_t s) {
  if (k <= 0) return;
  A2_REQUIRE(k <= 64, "at most 64 basis vectors");
  gemv_sub_kernel<<<grid_for(n), 256, 0, s>>>(V, ldv, k, h, w, n, 0);
  A2_CHECK_LAUNCH();
}
void gemv_set(const double* V, long long ldv, int k, const double* h, double* out, long long n,
              cudaStream_t s) {
  A2_REQUIRE(k >= 1 && k <= 64, "1..64 basis vectors");
  gemv_sub_kernel<<<grid_for(n), 256, 0, s>>>(V, ldv, k, h, out, n, 1);
  A2_CHECK_LAUNCH();
}

__global__ void axpby_kernel(double a, const double* x, double b, double* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
void axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s) {
  if (!n) return;
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(a, x, b, y, n);
  A2_CHECK_LAUNCH();
}

__global__ void lanczos_update_kernel(double* w, const double* v, const double* vprev,
                                      const double* alpha, double beta, long long n) {
  const double a = *alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double t = w[i] - a * v[i];
    if (vprev) t -= beta * vprev[i];
    w[i] = t;
  }
}
void lanczos_update(double* w, const double* v, const double* vprev, const double* alpha,
                    double beta_prev, long long n, cudaStream_t s) {
  lanczos_update_kernel<<<grid_for(n), 256, 0, s>>>(w, v, vprev, alpha, beta_prev, n);
  A2_CHECK_LAUNCH();
}

__global__ void normalize_kernel(const double* w, const double* nrm2, double* out, long long n) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = w[i] * inv;
}
void normalize_into(const double* w, const double* nrm2, double* out, long long n,
                    cudaStream_t s) {
  normalize_kernel<<<grid_for(n), 256, 0, s>>>(w, nrm2, out, n);
  A2_CHECK_LAUNCH();
}

__global__ void scale_dev_kernel(double* x, const double* num, const double* den_sqrt,
                                 long long n) {
  const double f = (num ? *num : 1.0) / (den_sqrt ? sqrt(*den_sqrt) : 1.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= f;
}
void scale_dev(double* x, const double* num, const double* den_sqrt, long long n,
               cudaStream_t s) {
  scale_dev_kernel<<<grid_for(n), 256, 0, s>>>(x, num, den_sqrt, n);
  A2_CHECK_LAUNCH();
}

// ----------------------------------------------------------------------------- Jacobi eigensolver
// Cyclic Jacobi with the round-robin parallel ordering (Golub & Van Loan, Sec. 8.5).
// Works in shared memory on a (me x me) padded matrix; all threads of the CTA call it.
// On return a is (numerically) diagonal, v holds the rotations (columns = eigvecs),
// perm[0..m-1] sorts the first m diagonal entries ascending.
struct JacobiShared {
  double a[64][65];
  double v[64][65];
  double cs[32], sn[32];
  int pp[32], qq[32];
  int perm[64];
  double off, tot;
};

__device__ int jacobi_shared(JacobiShared& J, int m) {
  const int me = (m + 1) & ~1;
  for (int e = threadIdx.x; e < me * me; e += blockDim.x) {
    const int i = e / me, j = e % me;
    J.v[i][j] = (i == j) ? 1.0 : 0.0;
    if (i >= m || j >= m) J.a[i][j] = 0.0;
  }
  __syncthreads();
  int sweep = 0;
  const int max_sweeps = 60;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < me; ++i)
        for (int j = 0; j < me; ++j) {
          tot += J.a[i][j] * J.a[i][j];
          if (i != j) off += J.a[i][j] * J.a[i][j];
        }
      J.off = off;
      J.tot = tot;
    }
    __syncthreads();
    if (J.off <= 1e-30 * J.tot || J.off == 0.0) break;
    for (int step = 0; step < me - 1; ++step) {
      if (threadIdx.x < me / 2) {
        const int t = threadIdx.x;
        const int p0 = (t == 0) ? 0 : 1 + (t - 1 + step) % (me - 1);
        const int tq = me - 1 - t;
        const int q0 = (tq == 0) ? 0 : 1 + (tq - 1 + step) % (me - 1);
        const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
        J.pp[t] = p;
        J.qq[t] = q;
        const double apq = J.a[p][q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double tau = (J.a[q][q] - J.a[p][p]) / (2.0 * apq);
          const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
        }
        J.cs[t] = c;
        J.sn[t] = s;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < (me / 2) * me; e += blockDim.x) {
        const int t = e / me, j = e % me;
        const int p = J.pp[t], q = J.qq[t];
        const double c = J.cs[t], s = J.sn[t];
        const double ap = J.a[p][j], aq = J.a[q][j];
        J.a[p][j] = c * ap - s * aq;
        J.a[q][j] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < (me / 2) * me; e += blockDim.x) {
        const int t = e / me, i = e % me;
        const int p = J.pp[t], q = J.qq[t];
        const double c = J.cs[t], s = J.sn[t];
        const double ap = J.a[i][p], aq = J.a[i][q];
        J.a[i][p] = c * ap - s * aq;
        J.a[i][q] = s * ap + c * aq;
        const double vp = J.v[i][p], vq = J.v[i][q];
        J.v[i][p] = c * vp - s * vq;
        J.v[i][q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    // the padding index (odd m) never rotates: its column stays e_m; skip it
    for (int i = 0; i < m; ++i) J.perm[i] = i;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j)
        if (J.a[J.perm[j]][J.perm[j]] < J.a[J.perm[i]][J.perm[i]]) {
          int x = J.perm[i]; J.perm[i] = J.perm[j]; J.perm[j] = x;
        }
  }
  __syncthreads();
  return sweep < max_sweeps ? sweep : -1;
}

__global__ void jacobi_kernel(double* A, int m, double* evals, double* evecs, int* status) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  JacobiShared& J = *reinterpret_cast<JacobiShared*>(dyn_smem);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    J.a[i][j] = 0.5 * (A[i * m + j] + A[j * m + i]);
  }
  __syncthreads();
  const int sw = jacobi_shared(J, m);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int j = e / m, i = e % m;
    evecs[j * m + i] = J.v[i][J.perm[j]];
  }
  if (threadIdx.x < m) evals[threadIdx.x] = J.a[J.perm[threadIdx.x]][J.perm[threadIdx.x]];
  if (threadIdx.x == 0) status[0] = sw;
}

void jacobi_eig(double* A, int m, double* evals, double* evecs, int* status, cudaStream_t s) {
  A2_REQUIRE(m >= 1 && m <= 63, "jacobi_eig: 1 <= m <= 63");
  static std::once_flag once;
  std::call_once(once, [] {
    A2_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(JacobiShared)));
  });
  jacobi_kernel<<<1, 256, sizeof(JacobiShared), s>>>(A, m, evals, evecs, status);
  A2_CHECK_LAUNCH();
}

// Coarse problem of Sec. 3.1 in one CTA:  S = V diag(sig) V^T, keep sig > eps*max,
// M = Sig+^{-1/2} V+^T A V+ Sig+^{-1/2}, lowest eigpair (lam, z), c = V+ Sig+^{-1/2} z,
// sign: c_0 >= 0 (else the largest |c_j| positive).
struct CoarseShared {
  JacobiShared J;
  double Ws[64][65];   // V+ Sig+^{-1/2}  (m x p)
  double As[64][65];
  int keep[64];
  int p;
};

__global__ void coarse_kernel(const double* A, const double* S, int m, double eps, double* c,
                              double* lam, int* rank, int* status) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  CoarseShared& C = *reinterpret_cast<CoarseShared*>(dyn_smem);
  JacobiShared& J = C.J;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    J.a[i][j] = 0.5 * (S[i * m + j] + S[j * m + i]);
    C.As[i][j] = 0.5 * (A[i * m + j] + A[j * m + i]);
  }
  __syncthreads();
  const int sw1 = jacobi_shared(J, m);
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int i = 0; i < m; ++i) smax = fmax(smax, J.a[i][i]);
    int p = 0;
    for (int j = 0; j < m; ++j) {       // ascending order of eigenvalues
      const int col = J.perm[j];
      if (J.a[col][col] > eps * smax) C.keep[p++] = col;
    }
    C.p = p;
  }
  __syncthreads();
  const int p = C.p;
  for (int e = threadIdx.x; e < m * p; e += blockDim.x) {
    const int i = e / p, k = e % p;
    const int col = C.keep[k];
    C.Ws[i][k] = J.v[i][col] / sqrt(J.a[col][col]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * p; e += blockDim.x) {   // T = A Ws (m x p) into J.v
    const int i = e / p, k = e % p;
    double t = 0.0;
    for (int l = 0; l < m; ++l) t += C.As[i][l] * C.Ws[l][k];
    J.v[i][k] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {   // M = Ws^T T (p x p) into As
    const int k = e / p, l = e % p;
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += C.Ws[i][k] * J.v[i][l];
    C.As[k][l] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int k = e / p, l = e % p;
    J.a[k][l] = 0.5 * (C.As[k][l] + C.As[l][k]);
  }
  __syncthreads();
  const int sw2 = jacobi_shared(J, p);
  if (threadIdx.x == 0) {
    const int col = J.perm[0];
    double amax = 0.0;
    int imax = 0;
    for (int i = 0; i < m; ++i) {
      double t = 0.0;
      for (int k = 0; k < p; ++k) t += C.Ws[i][k] * J.v[k][col];
      C.As[0][i] = t;
      if (fabs(t) > amax) { amax = fabs(t); imax = i; }
    }
    const double ref = (fabs(C.As[0][0]) > 1e-14 * amax) ? C.As[0][0] : C.As[0][imax];
    const double sg = ref < 0 ? -1.0 : 1.0;
    for (int i = 0; i < m; ++i) c[i] = sg * C.As[0][i];
    lam[0] = J.a[col][col];
    rank[0] = p;
    status[0] = (sw1 < 0 || sw2 < 0) ? -1 : 0;
  }
}

void coarse_solve_dev(const double* A, const double* S, int m, double eps, double* c,
                      double* lam, int* rank, int* status, cudaStream_t s) {
  A2_REQUIRE(m >= 1 && m <= 63, "coarse problem: 1 <= m <= 63");
  static std::once_flag once;
  std::call_once(once, [] {
    A2_CUDA(cudaFuncSetAttribute(coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(CoarseShared)));
  });
  coarse_kernel<<<1, 256, sizeof(CoarseShared), s>>>(A, S, m, eps, c, lam, rank, status);
  A2_CHECK_LAUNCH();
}

// ----------------------------------------------------------------------------- tridiagonal
// Lowest eigenpair of the symmetric tridiagonal T (diag a[0..k-1], off-diag b[0..k-2]):
// bisection on the Sturm count of T - x I (Golub & Van Loan, Sec. 8.4; here 32-way
// multisection by one warp), then inverse iteration with a partially pivoted tridiagonal
// solve (one thread, shared-memory arrays).  k <= 64.
__device__ int sturm_below(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double d = a[0] - x;
  if (d < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    const double dd = (d == 0.0) ? 1e-300 : d;
    d = a[i] - x - b[i - 1] * b[i - 1] / dd;
    if (d < 0) ++cnt;
  }
  return cnt;
}

__global__ void tridiag_lowest_kernel(TridiagIn in, double* out) {
  // multisection: the 32 lanes evaluate the Sturm count at 32 interior points of the
  // bracket at once, so that every round shrinks it 33-fold
  const int lane = threadIdx.x & 31;
  const int k = in.k;
  const double* a = in.a;
  const double* b = in.b;
  double lo = 1e300, hi = -1e300, scale = 0.0;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
    scale = fmax(scale, fabs(a[i]) + r);
  }
  for (int it = 0; it < 40 && hi - lo > 4e-16 * fmax(scale, 1e-300); ++it) {
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const bool above = sturm_below(a, b, k, x) >= 1;     // lowest eigenvalue <= x
    const unsigned m = __ballot_sync(0xffffffffu, above);
    const int j = m ? __ffs(m) - 1 : 32;                 // first point above the eigenvalue
    const double nlo = j == 0 ? lo : lo + (hi - lo) * (double)j / 33.0;
    const double nhi = j == 32 ? hi : lo + (hi - lo) * (double)(j + 1) / 33.0;
    if (!(nlo >= lo && nhi <= hi && nlo < nhi)) break;  // no further progress in FP64
    lo = nlo;
    hi = nhi;
  }
  const double theta = 0.5 * (lo + hi);
  if (lane != 0) return;
  // inverse iteration: (T - theta I) y = v, partially pivoted tridiagonal elimination
  __shared__ double y[64], v[64], dl[64], d[64], du[64], du2[64], rhs[64];
  for (int i = 0; i < k; ++i) v[i] = 1.0 / sqrt((double)k) * (1.0 + 0.01 * i);
  const double eps = 1e-14 * fmax(scale, 1e-300);
  for (int rep = 0; rep < 3; ++rep) {
    for (int i = 0; i < k; ++i) {
      d[i] = a[i] - theta;
      du[i] = (i + 1 < k) ? b[i] : 0.0;
      dl[i] = (i + 1 < k) ? b[i] : 0.0;
      du2[i] = 0.0;
      rhs[i] = v[i];
    }
    for (int i = 0; i + 1 < k; ++i) {
      if (fabs(d[i]) >= fabs(dl[i])) {
        const double piv = (d[i] == 0.0) ? eps : d[i];
        d[i] = piv;
        const double f = dl[i] / piv;
        d[i + 1] -= f * du[i];
        rhs[i + 1] -= f * rhs[i];
        dl[i] = 0.0;
      } else {
        const double f = d[i] / dl[i];
        d[i] = dl[i];
        double t = d[i + 1];
        d[i + 1] = du[i] - f * t;
        if (i + 2 < k) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du2[i];
        }
        du[i] = t;
        t = rhs[i];
        rhs[i] = rhs[i + 1];
        rhs[i + 1] = t - f * rhs[i + 1];
      }
    }
    if (d[k - 1] == 0.0) d[k - 1] = eps;
    y[k - 1] = rhs[k - 1] / d[k - 1];
    if (k > 1) y[k - 2] = (rhs[k - 2] - du[k - 2] * y[k - 1]) / d[k - 2];
    for (int i = k - 3; i >= 0; --i) y[i] = (rhs[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / d[i];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += y[i] * y[i];
    const double inv = 1.0 / sqrt(nrm);
    for (int i = 0; i < k; ++i) v[i] = y[i] * inv;
  }
  out[0] = theta;
  for (int i = 0; i < k; ++i) out[1 + i] = v[i];
}

void tridiag_lowest(const TridiagIn& in, double* out, cudaStream_t s) {
  A2_REQUIRE(in.k >= 1 && in.k <= 64, "tridiagonal size 1..64");
  tridiag_lowest_kernel<<<1, 32, 0, s>>>(in, out);
  A2_CHECK_LAUNCH();
}

// ----------------------------------------------------------------------------- H_eff diagonal
// Ed[b][w] = E[b][w][b] for an environment E [D][R][D] (any float type) -> double
template <typename T>
__global__ void env_diag_kernel(const T* E, int D, int R, double* out) {
  const long long n = (long long)D * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / R, w = e % R;
    out[e] = (double)E[(b * R + w) * D + b];
  }
}
template <typename T>
void env_diag(const T* E, int D, int R, double* out, cudaStream_t s) {
  env_diag_kernel<T><<<grid_for((long long)D * R), 256, 0, s>>>(E, D, R, out);
  A2_CHECK_LAUNCH();
}
template void env_diag<double>(const double*, int, int, double*, cudaStream_t);
template void env_diag<float>(const float*, int, int, double*, cudaStream_t);

// out[b][rs][rw] = sum over entries (w, t) of row (rw, rs) with t == rs of val * Ed[b][w]
// (the diagonal s = t part of one MPO core, acting on a diagonal environment)
__global__ void diag_action_kernel(SparseRows<double> sp, int Rrow, int n, const double* Ed,
                                   int Rin, int B, double* out) {
  const int r = blockIdx.x;
  const int rw = sp.row_w[r], rs = sp.row_s[r];
  for (int b = threadIdx.x + blockIdx.y * blockDim.x; b < B; b += blockDim.x * gridDim.y) {
    double acc = 0.0;
    for (int e = sp.row_ptr[r]; e < sp.row_ptr[r + 1]; ++e)
      if (sp.nz_t[e] == rs) acc += sp.nz_val[e] * Ed[(long long)b * Rin + sp.nz_w[e]];
    out[((long long)b * n + rs) * Rrow + rw] = acc;
  }
}
void diag_action(const SparseRows<double>& sp, int Rrow, int n, const double* Ed, int Rin, int B,
                 double* out, cudaStream_t s) {
  if (!sp.nrows || !B) return;
  dim3 grid(sp.nrows, std::max(1, std::min(8, cdiv(B, 256))));
  diag_action_kernel<<<grid, 256, 0, s>>>(sp, Rrow, n, Ed, Rin, B, out);
  A2_CHECK_LAUNCH();
}

// Davidson correction t_i = r_i / (diag_i - theta), guarded away from zero
__global__ void precond_kernel(const double* r, const double* diag, const double* theta,
                               double* t, long long n) {
  const double th = *theta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double d = diag[i] - th;
    if (fabs(d) < 1e-4) d = d < 0 ? -1e-4 : 1e-4;
    t[i] = r[i] / d;
  }
}
void precondition(const double* r, const double* diag, const double* theta, double* t,
                  long long n, cudaStream_t s) {
  precond_kernel<<<grid_for(n), 256, 0, s>>>(r, diag, theta, t, n);
  A2_CHECK_LAUNCH();
}

// ----------------------------------------------------------------------------- assorted
__global__ void cols_rev_to_rows_kernel(const double* __restrict__ G, long long ld, int rows,
                                        int col_first, int r, double* __restrict__ P) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {           // read columns (contiguous in i)
    const int c = c0 + j, i = i0 + threadIdx.x;
    if (c < r && i < rows) tile[j][threadIdx.x] = G[(long long)(col_first - c) * ld + i];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {           // write rows of P (contiguous in c)
    const int i = i0 + j, c = c0 + threadIdx.x;
    if (c < r && i < rows) P[(long long)i * r + c] = tile[threadIdx.x][j];
  }
}
void cols_rev_to_rows(const double* G, long long ld, int rows, int col_first, int r, double* P,
                      cudaStream_t s) {
  if (rows <= 0 || r <= 0) return;
  A2_REQUIRE(col_first - (r - 1) >= 0, "cols_rev_to_rows: column range");
  dim3 grid(cdiv(rows, 32), cdiv(r, 32));
  A2_REQUIRE(grid.y < 65536, "cols_rev_to_rows: grid too large");
  cols_rev_to_rows_kernel<<<grid, dim3(32, 8), 0, s>>>(G, ld, rows, col_first, r, P);
  A2_CHECK_LAUNCH();
}

__global__ void gather_axpy_atomic_kernel(const double* __restrict__ G,
                                          const long long* __restrict__ index,
                                          const long long* __restrict__ param,
                                          const double* __restrict__ factor, long long n,
                                          double* grad) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    atomicAdd(grad + param[e], factor[e] * G[index[e]]);
}
void gather_axpy_atomic(const double* G, const long long* index, const long long* param,
                        const double* factor, long long n, double* grad, cudaStream_t s) {
  if (n <= 0) return;
  gather_axpy_atomic_kernel<<<grid_for(n), 256, 0, s>>>(G, index, param, factor, n, grad);
  A2_CHECK_LAUNCH();
}

void fill_zero(void* p, size_t bytes, cudaStream_t s) {
  if (bytes) A2_CUDA(cudaMemsetAsync(p, 0, bytes, s));
}

// Q: rows x k column-major (ld ldq) from orgqr; R: k x k upper (col-major, ld ldr) from geqrf.
// Flip signs so that diag(R) >= 0: column j of Q and row j of R change sign if R_jj < 0.
__global__ void sign_fix_kernel(double* Q, int ldq, int rows, double* R, int ldr, int k) {
  const int j = blockIdx.x;
  const double d = R[(long long)j * ldr + j];
  if (d >= 0.0) return;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) Q[(long long)j * ldq + i] *= -1.0;
  for (int c = j + threadIdx.x; c < k; c += blockDim.x) R[(long long)c * ldr + j] *= -1.0;
}
void sign_fix_qr(double* Q, int ldq, int rows, double* R, int ldr, int k, cudaStream_t s) {
  if (!k) return;
  sign_fix_kernel<<<k, 128, 0, s>>>(Q, ldq, rows, R, ldr, k);
  A2_CHECK_LAUNCH();
}

__global__ void scale_rows_kernel(double* M, int rows, int cols, const double* sv) {
  const long long n = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    M[e] *= sv[e / cols];
}
void scale_rows(double* M, int rows, int cols, const double* svals, cudaStream_t s) {
  long long n = (long long)rows * cols;
  if (!n) return;
  scale_rows_kernel<<<grid_for(n), 256, 0, s>>>(M, rows, cols, svals);
  A2_CHECK_LAUNCH();
}

// dst[(o0 + i)*dst_s0 + j*dst_s1 + (o2 + k)] = alpha * src[(i*d1 + j)*d2 + k]
__global__ void copy_block3_kernel(const double* src, int d0, int d1, int d2, double* dst,
                                   long long s0, long long s1, int o0, int o2, double alpha,
                                   bool add) {
  const long long n = (long long)d0 * d1 * d2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % d2);
    const long long ij = e / d2;
    const int j = (int)(ij % d1), i = (int)(ij / d1);
    double* d = dst + (long long)(o0 + i) * s0 + (long long)j * s1 + (o2 + k);
    *d = add ? *d + alpha * src[e] : alpha * src[e];
  }
}
void copy_block3(const double* src, int d0, int d1, int d2, double* dst, long long dst_s0,
                 long long dst_s1, int o0, int o2, double alpha, cudaStream_t s, bool add) {
  long long n = (long long)d0 * d1 * d2;
  if (!n) return;
  copy_block3_kernel<<<grid_for(n), 256, 0, s>>>(src, d0, d1, d2, dst, dst_s0, dst_s1, o0, o2,
                                                 alpha, add);
  A2_CHECK_LAUNCH();
}

void sparse_autotune(bool on) {
  std::lock_guard<std::mutex> g(g_sp_mu);
  g_sp_on.store(on);
  if (!on) g_sp_tune.clear();
}

}  // namespace a2
