// Host driver of the two-site A2DMRG iteration (Alg. 2) and the C ABI (a2dmrg.h).
//
// Data layout on the device (row-major):
//   TT core j        [D_j][n_j][D_j+1]            float64 master copy
//   environments     [bra][MPO bond][ket]          float64 or float32 (precision mode)
//   MPO core j       sparse row lists, left-to-right action (rows (w_r,s), entries (w_l,t))
//                    and right-to-left action (rows (w_l,s), entries (w_r,t)).
// The H_eff application is the chain of App. A (two-site form):
//   S1 T1[a,w,t1,t2,b'] = sum_a' L[a,w,a'] x[a',t1,t2,b']           dense GEMM
//   S2 T2[a,w1,s1,t2,b'] = sum_{w,t1} A_k[w,s1,t1,w1] T1[...]       sparse MPO action
//   S3 T3[a,s1,s2,w2,b'] = sum_{w1,t2} A_k+1[w1,s2,t2,w2] T2[...]   sparse MPO action
//   S4 y[a,s1,s2,b]      = sum_{w2,b'} T3[...] R[b,w2,b']            dense GEMM (split K)
#include <cstdio>
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <atomic>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/a2dmrg.h"
#include "kernels.cuh"
#include "linalg.cuh"
#include "tc_gemm.cuh"

using namespace a2;

// ============================================================================= handles
struct a2_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Solver solver;
  std::string err;
  DevBuf scal, partial;         // device scalars, reduction partials
  double* h_scal = nullptr;     // pinned host mirror
  DevBuf t1, t2, t3, xa, ya, cb, ck, gram, wv, tmp1, tmp2, tf;   // scratch
  std::vector<a2_ctx*> lanes;   // per-group contexts (own stream, scratch, solver)
  const a2_ctx* parent = nullptr;   // group lanes: the context they belong to
  // the FP64 products of the sweep's folds, overlaps and SVD splits may run on the
  // tensor cores by the Ozaki scheme (set while a mixed or FP64-emulated sweep runs)
  bool gemm_tc = false;
  std::mutex lane_mu;
  // group lanes only: a high-priority stream for the latency-bound factorisations, so
  // that their many small kernels are not queued behind the other groups' matvecs
  cudaStream_t hi = nullptr;
  cudaEvent_t ev_to_hi = nullptr, ev_from_hi = nullptr;
};

struct a2_tt {
  a2_ctx* ctx = nullptr;
  int L = 0;
  std::vector<int> phys;
  std::vector<int> dims;        // L + 1 bond dims (left bond of core j = dims[j])
  std::vector<DevBuf> cores;
};

namespace {

// NVTX range for the steps of a global iteration (visible to nsys / ncu --nvtx; free
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* name, int i) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), "%s %d", name, i);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct SiteOps {
  int Rl = 0, n = 0, Rr = 0;
  long long nnz = 0;
  // W = I (x) G + W_rest (G[wl][wr] = the common value of the n diagonal entries
  // W[wl][s][s][wr]); when G is large (the hand-over core of the operator automaton)
  // the H_eff chains fold G into the environments and keep only W_rest sparse.
  int foldable = 0, fold_on = 1;
  long long nnz_g = 0;
  struct Part {
    int nrows = 0, nnz = 0;
    DevBuf ptr, rw, rs, nw, nt, v64, v32, v32lo;
    template <typename V> SparseRows<V> rows() const {
      SparseRows<V> r;
      r.nrows = nrows;
      r.row_ptr = ptr.as<int>();
      r.row_w = rw.as<int>();
      r.row_s = rs.as<int>();
      r.nz_w = nw.as<int>();
      r.nz_t = nt.as<int>();
      r.nnz_total = nnz;
      if constexpr (sizeof(V) == 8) r.nz_val = v64.as<double>();
      else r.nz_val = v32.as<float>();
      r.nz_lo = v32lo.as<float>();
      return r;
    }
  } lr, rl;
  Part lr_rest;            // left-to-right action of W_rest (foldable cores only)
  Part g_lr;               // G by columns: rows wr, entries (wl, 0, G[wl][wr])
  Part g_rl;               // G by rows:    rows wl, entries (wr, 0, G[wl][wr])
  bool fold() const { return foldable && fold_on; }
};

}  // namespace

struct a2_mpo {
  a2_ctx* ctx = nullptr;
  int L = 0;
  std::vector<int> phys, R;
  std::vector<SiteOps> site;
};

// ============================================================================= helpers
namespace {

// I (x) G split of an MPO core W[wl][s][t][wr]: G[wl][wr] = W[wl][s][s][wr] where all n
// diagonal entries are equal and nonzero, else 0 (G: Rl x Rr, written in full).  Returns
// the number of nonzeros of G.
long long identity_block_split(const double* W, int Rl, int n, int Rr, double* G) {
  long long nnz = 0;
  for (int wl = 0; wl < Rl; ++wl)
    for (int wr = 0; wr < Rr; ++wr) {
      const double v = W[(((size_t)wl * n + 0) * n + 0) * Rr + wr];
      bool same = v != 0.0;
      for (int sx = 1; sx < n && same; ++sx)
        same = W[(((size_t)wl * n + sx) * n + sx) * Rr + wr] == v;
      G[(size_t)wl * Rr + wr] = same ? v : 0.0;
      nnz += same ? 1 : 0;
    }
  return nnz;
}

// Folding G into an environment costs a dense contraction over the whole (Rl x Rr)
// block; it pays when G holds at least ~1/64 of that block and is not tiny.
bool fold_worthwhile(long long nnz_g, int Rl, int Rr) {
  return nnz_g >= 1024 && nnz_g * 64 >= (long long)Rl * Rr;
}

void upload(DevBuf& b, const void* h, size_t bytes, cudaStream_t s) {
  b.ensure(bytes, s);
  if (bytes) A2_CUDA(cudaMemcpyAsync(b.p, h, bytes, cudaMemcpyHostToDevice, s));
}

void build_part(SiteOps::Part& part, const std::vector<std::vector<std::array<double, 3>>>& rows,
                const std::vector<std::pair<int, int>>& rowid, cudaStream_t s) {
  part.nrows = (int)rows.size();
  std::vector<int> ptr(rows.size() + 1, 0), rw, rs, nw, nt;
  std::vector<double> v64;
  std::vector<float> v32, v32lo;
  for (size_t r = 0; r < rows.size(); ++r) {
    rw.push_back(rowid[r].first);
    rs.push_back(rowid[r].second);
    for (auto& e : rows[r]) {
      nw.push_back((int)e[0]);
      nt.push_back((int)e[1]);
      v64.push_back(e[2]);
      v32.push_back((float)e[2]);
      v32lo.push_back((float)(e[2] - (double)(float)e[2]));
    }
    ptr[r + 1] = (int)nw.size();
  }
  part.nnz = (int)nw.size();
  upload(part.ptr, ptr.data(), ptr.size() * sizeof(int), s);
  upload(part.rw, rw.data(), rw.size() * sizeof(int), s);
  upload(part.rs, rs.data(), rs.size() * sizeof(int), s);
  upload(part.nw, nw.data(), nw.size() * sizeof(int), s);
  upload(part.nt, nt.data(), nt.size() * sizeof(int), s);
  upload(part.v64, v64.data(), v64.size() * sizeof(double), s);
  upload(part.v32, v32.data(), v32.size() * sizeof(float), s);
  upload(part.v32lo, v32lo.data(), v32lo.size() * sizeof(float), s);
}

// Scan a dense core W[wl][s][t][wr] (minus `sub` = I (x) G when given) into the two
// sparse actions; returns the number of nonzeros.
long long scan_actions(const double* W, const double* G, int Rl, int n, int Rr,
                       SiteOps::Part& plr, SiteOps::Part* prl, cudaStream_t s) {
  std::vector<std::vector<std::array<double, 3>>> lr((size_t)Rr * n), rl((size_t)Rl * n);
  std::vector<std::pair<int, int>> lrid((size_t)Rr * n), rlid((size_t)Rl * n);
  for (int wr = 0; wr < Rr; ++wr)
    for (int sx = 0; sx < n; ++sx) lrid[(size_t)wr * n + sx] = {wr, sx};
  for (int wl = 0; wl < Rl; ++wl)
    for (int sx = 0; sx < n; ++sx) rlid[(size_t)wl * n + sx] = {wl, sx};
  long long nnz = 0;
  for (int wl = 0; wl < Rl; ++wl)
    for (int sx = 0; sx < n; ++sx)
      for (int t = 0; t < n; ++t)
        for (int wr = 0; wr < Rr; ++wr) {
          double v = W[(((size_t)wl * n + sx) * n + t) * Rr + wr];
          if (G && sx == t) v -= G[(size_t)wl * Rr + wr];
          if (v == 0.0) continue;
          ++nnz;
          lr[(size_t)wr * n + sx].push_back({(double)wl, (double)t, v});
          rl[(size_t)wl * n + sx].push_back({(double)wr, (double)t, v});
        }
  build_part(plr, lr, lrid, s);
  if (prl) build_part(*prl, rl, rlid, s);
  return nnz;
}

void build_site(SiteOps& so, const double* W, int Rl, int n, int Rr, cudaStream_t s) {
  so.Rl = Rl; so.n = n; so.Rr = Rr;
  so.nnz = scan_actions(W, nullptr, Rl, n, Rr, so.lr, &so.rl, s);
  std::vector<double> G((size_t)Rl * Rr, 0.0);
  so.nnz_g = identity_block_split(W, Rl, n, Rr, G.data());
  so.foldable = fold_worthwhile(so.nnz_g, Rl, Rr) ? 1 : 0;
  if (!so.foldable) return;
  scan_actions(W, G.data(), Rl, n, Rr, so.lr_rest, nullptr, s);
  std::vector<std::vector<std::array<double, 3>>> gc((size_t)Rr), gr((size_t)Rl);
  std::vector<std::pair<int, int>> gcid((size_t)Rr), grid((size_t)Rl);
  for (int wr = 0; wr < Rr; ++wr) gcid[wr] = {wr, 0};
  for (int wl = 0; wl < Rl; ++wl) grid[wl] = {wl, 0};
  for (int wl = 0; wl < Rl; ++wl)
    for (int wr = 0; wr < Rr; ++wr) {
      const double v = G[(size_t)wl * Rr + wr];
      if (v == 0.0) continue;
      gc[wr].push_back({(double)wl, 0.0, v});
      gr[wl].push_back({(double)wr, 0.0, v});
    }
  build_part(so.g_lr, gc, gcid, s);
  build_part(so.g_rl, gr, grid, s);
}

double* scal(a2_ctx* c, int i) { return c->scal.as<double>() + i; }

// Stream, scratch and solver of one concurrent group (created on first use, kept).
a2_ctx* lane(a2_ctx* c, int i) {
  std::lock_guard<std::mutex> g(c->lane_mu);
  while ((int)c->lanes.size() <= i) {
    auto* l = new a2_ctx();
    l->device = c->device;
    l->parent = c;
    A2_CUDA(cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking));
    l->own_stream = true;
    int least = 0, greatest = 0;
    A2_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    A2_CUDA(cudaStreamCreateWithPriority(&l->hi, cudaStreamNonBlocking, greatest));
    A2_CUDA(cudaEventCreateWithFlags(&l->ev_to_hi, cudaEventDisableTiming));
    A2_CUDA(cudaEventCreateWithFlags(&l->ev_from_hi, cudaEventDisableTiming));
    l->solver.init(l->stream);
    l->scal.ensure(sizeof(double) * 16384, l->stream);
    l->partial.ensure(sizeof(double) * kReduceBlocks * 64, l->stream);
    A2_CUDA(cudaMallocHost(&l->h_scal, sizeof(double) * 64));
    A2_CUDA(cudaStreamSynchronize(l->stream));
    c->lanes.push_back(l);
  }
  return c->lanes[i];
}

// Runs the enclosed work of a group lane on its high-priority stream (ordered after and
// before the lane's normal stream by events); a no-op for contexts without one.
struct HiScope {
  a2_ctx* c;
  cudaStream_t saved = nullptr;
  explicit HiScope(a2_ctx* ctx) : c(ctx) {
    if (!c->hi) return;
    A2_CUDA(cudaEventRecord(c->ev_to_hi, c->stream));
    A2_CUDA(cudaStreamWaitEvent(c->hi, c->ev_to_hi, 0));
    saved = c->stream;
    c->stream = c->hi;
    c->solver.set_stream(c->hi);
  }
  ~HiScope() {
    if (!saved) return;
    cudaEventRecord(c->ev_from_hi, c->hi);
    cudaStreamWaitEvent(saved, c->ev_from_hi, 0);
    c->stream = saved;
    try {
      c->solver.set_stream(saved);
    } catch (...) {
    }
  }
};

void destroy_ctx_resources(a2_ctx* c) {
  cudaStreamSynchronize(c->stream);
  c->solver.destroy();
  for (DevBuf* b : {&c->scal, &c->partial, &c->t1, &c->t2, &c->t3, &c->xa, &c->ya, &c->cb, &c->ck,
                    &c->gram, &c->wv, &c->tmp1, &c->tmp2, &c->tf})
    b->release();
  cudaStreamSynchronize(c->stream);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  c->h_scal = nullptr;
}

// copy `count` doubles from the device scalar area to the pinned host mirror and wait
void fetch_scalars(a2_ctx* c, int first, int count) {
  A2_CUDA(cudaMemcpyAsync(c->h_scal + first, scal(c, first), sizeof(double) * count,
                          cudaMemcpyDeviceToHost, c->stream));
  A2_CUDA(cudaStreamSynchronize(c->stream));
}

double dot_dev(a2_ctx* c, const double* x, const double* y, long long n, int slot) {
  dot_multi(x, 0, 1, y, n, c->partial.as<double>(), scal(c, slot), c->stream);
  fetch_scalars(c, slot, 1);
  return c->h_scal[slot];
}

void check_finite(double v, const char* what) {
  if (!std::isfinite(v)) throw NumericError(std::string("non-finite value in ") + what);
}

// ============================================================================= contractions
double heff_flops(const SiteOps& A1, const SiteOps& A2, int Dl, int Dr);
double env_flops(const SiteOps& so, int Dl, int Dr);
// A TT core viewed in compute type T (converted copy for float).
template <typename T>
const T* as_compute(a2_ctx* c, const double* core, long long n, DevBuf& buf) {
  if constexpr (sizeof(T) == 8) {
    (void)c; (void)n; (void)buf;
    return core;
  } else {
    buf.ensure(sizeof(float) * (size_t)n, c->stream);
    convert<double, float>(core, buf.as<float>(), n, c->stream);
    return buf.as<float>();
  }
}

// Left environment update (eq. env_L update): Hin [Dlb][Rl][Dlk] -> Hout [Drb][Rr][Drk].
template <typename T>
void env_left(a2_ctx* c, const SiteOps& so, const T* Hin, const T* bra, int Dlb, int Drb,
              const T* ket, int Dlk, int Drk, T* Hout) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_ENV, s, env_flops(so, std::max(Dlb, Dlk), std::max(Drb, Drk)),
               sizeof(T) * ((double)Dlb * Rl * Dlk + (double)Drb * Rr * Drk +
                            2.0 * Dlb * Rl * n * Drk + 2.0 * Dlb * n * Rr * Drk));
  c->tmp1.ensure(sizeof(T) * (size_t)Dlb * Rl * n * Drk, s);
  c->tmp2.ensure(sizeof(T) * (size_t)Dlb * n * Rr * Drk, s);
  T* T1 = c->tmp1.as<T>();
  T* T2 = c->tmp2.as<T>();
  {  // E1: T1[(a w)][(t b')] = sum_a' Hin[(a w)][a'] ket[a'][(t b')]
    SimtGemm<T, T> g;
    g.M = Dlb * Rl; g.N = n * Drk; g.K = Dlk;
    g.A = Hin; g.sam = Dlk; g.sak = 1;
    g.B = ket; g.sbn = 1; g.sbk = (long long)n * Drk;
    g.C = T1; g.scm = (long long)n * Drk; g.scn = 1;
    simt_gemm(g, s);
  }
  {  // E2: T2[(a s)][(w' b')] = sum_{w,t} A[w,s,t,w'] T1[(a w)][(t b')]
    SparseGeom gm;
    gm.veclen = Drk;
    gm.in_sw = (long long)n * Drk; gm.in_st = Drk;
    gm.out_sw = Drk; gm.out_ss = (long long)Rr * Drk;
    gm.B1 = Dlb; gm.in_b1 = (long long)Rl * n * Drk; gm.out_b1 = (long long)n * Rr * Drk;
    sparse_rows_apply<T, T, T>(so.lr.rows<T>(), gm, T1, T2, s);
  }
  {  // E3: Hout[b][(w' b')] = sum_{(a s)} bra[(a s)][b] T2[(a s)][(w' b')]
    SimtGemm<T, T> g;
    g.M = Drb; g.N = Rr * Drk; g.K = Dlb * n;
    g.A = bra; g.sam = 1; g.sak = Drb;
    g.B = T2; g.sbn = 1; g.sbk = (long long)Rr * Drk;
    g.C = Hout; g.scm = (long long)Rr * Drk; g.scn = 1;
    simt_gemm(g, s);
  }
}

// Right environment update (eq. env_R update): Hin [Drb][Rr][Drk] -> Hout [Dlb][Rl][Dlk].
template <typename T>
void env_right(a2_ctx* c, const SiteOps& so, const T* Hin, const T* bra, int Dlb, int Drb,
               const T* ket, int Dlk, int Drk, T* Hout) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_ENV, s, env_flops(so, std::max(Dlb, Dlk), std::max(Drb, Drk)),
               sizeof(T) * ((double)Dlb * Rl * Dlk + (double)Drb * Rr * Drk +
                            2.0 * Drb * Rr * n * Dlk + 2.0 * n * Drb * Rl * Dlk));
  c->tmp1.ensure(sizeof(T) * ((size_t)Drb * Rr * n * Dlk + (size_t)n * Dlk * Drk), s);
  c->tmp2.ensure(sizeof(T) * (size_t)n * Drb * Rl * Dlk, s);
  T* T1 = c->tmp1.as<T>();
  T* Vt = T1 + (size_t)Drb * Rr * n * Dlk;
  T* T2 = c->tmp2.as<T>();
  permute_swap01<T, T>(ket, Vt, n, Dlk, Drk, s);      // Vt[t][a'][b'] = ket[a'][t][b']
  {  // F1: T1[(b w')][(t a')] = sum_b' Hin[(b w')][b'] Vt[(t a')][b']
    SimtGemm<T, T> g;
    g.M = Drb * Rr; g.N = n * Dlk; g.K = Drk;
    g.A = Hin; g.sam = Drk; g.sak = 1;
    g.B = Vt; g.sbn = Drk; g.sbk = 1;
    g.C = T1; g.scm = (long long)n * Dlk; g.scn = 1;
    simt_gemm(g, s);
  }
  {  // F2: T2[(s b)][(w a')] = sum_{w',t} A[w,s,t,w'] T1[(b w')][(t a')]
    SparseGeom gm;
    gm.veclen = Dlk;
    gm.in_sw = (long long)n * Dlk; gm.in_st = Dlk;
    gm.out_sw = Dlk; gm.out_ss = (long long)Drb * Rl * Dlk;
    gm.B1 = Drb; gm.in_b1 = (long long)Rr * n * Dlk; gm.out_b1 = (long long)Rl * Dlk;
    sparse_rows_apply<T, T, T>(so.rl.rows<T>(), gm, T1, T2, s);
  }
  {  // F3: Hout[a][(w a')] = sum_{(s b)} bra[a][(s b)] T2[(s b)][(w a')]
    SimtGemm<T, T> g;
    g.M = Dlb; g.N = Rl * Dlk; g.K = n * Drb;
    g.A = bra; g.sam = (long long)n * Drb; g.sak = 1;
    g.B = T2; g.sbn = 1; g.sbk = (long long)Rl * Dlk;
    g.C = Hout; g.scm = (long long)Rl * Dlk; g.scn = 1;
    simt_gemm(g, s);
  }
}

// ---- environment updates with FP32-accurate split products on tcgen05 (FP32 envs)
inline long long round64(long long x) { return (x + 63) / 64 * 64; }
static const int kPairA[6] = {0, 0, 1, 0, 1, 2};
static const int kPairB[6] = {0, 1, 0, 2, 1, 0};

struct Planes {   // three BF16 slices of a (rows x K) operand, row stride ld
  const __nv_bfloat16* p[3];
  long long ld;
};
Planes planes_at(__nv_bfloat16* base, long long ld, long long plane) {
  return Planes{{base, base + plane, base + 2 * plane}, ld};
}

void env_left_emu(a2_ctx* c, const SiteOps& so, const float* Hin, const double* bra, int Dlb,
                  int Drb, const double* ket, int Dlk, int Drk, float* Hout) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_ENV, s, env_flops(so, std::max(Dlb, Dlk), std::max(Drb, Drk)),
               4.0 * ((double)Dlb * Rl * Dlk + (double)Drb * Rr * Drk +
                      2.0 * Dlb * Rl * n * Drk + 2.0 * Dlb * n * Rr * Drk));
  const long long ldH = pad8(Dlk), pH = round64((long long)Dlb * Rl * ldH);
  const long long ldK = pad8(Dlk), pK = round64((long long)n * Drk * ldK);
  const long long ldB = pad8((long long)Dlb * n), pB = round64((long long)Drb * ldB);
  const long long pT = round64((long long)Rr * Drk * ldB);
  c->cb.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * (pH + pK + pB)), s);
  __nv_bfloat16* Hp = c->cb.as<__nv_bfloat16>();
  __nv_bfloat16* Kp = Hp + 3 * pH;
  __nv_bfloat16* Bp = Kp + 3 * pK;
  c->tmp1.ensure(sizeof(float) * (size_t)Dlb * Rl * n * Drk, s);
  c->tmp2.ensure(sizeof(float) * (size_t)Dlb * n * Rr * Drk, s);
  c->t3.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * pT), s);
  float* T1 = c->tmp1.as<float>();
  float* T2 = c->tmp2.as<float>();
  __nv_bfloat16* T2p = c->t3.as<__nv_bfloat16>();
  split3_ld<float>(Hin, (long long)Dlb * Rl, Dlk, Hp, ldH, pH, s);
  transpose_split3<double>(ket, Dlk, n * Drk, Kp, ldK, pK, s);
  {  // E1: T1[(a w)][(t b')] = sum_a' Hin[(a w)][a'] ket[a'][(t b')]
    Planes A = planes_at(Hp, ldH, pH), B = planes_at(Kp, ldK, pK);
    tc_gemm_bf16_pairs(A.p, A.ld, B.p, B.ld, Dlb * Rl, n * Drk, Dlk, 6, kPairA, kPairB, T1,
                       (long long)n * Drk, 1, 1, s);
  }
  {  // E2 (FP32)
    SparseGeom gm;
    gm.veclen = Drk;
    gm.in_sw = (long long)n * Drk; gm.in_st = Drk;
    gm.out_sw = Drk; gm.out_ss = (long long)Rr * Drk;
    gm.B1 = Dlb; gm.in_b1 = (long long)Rl * n * Drk; gm.out_b1 = (long long)n * Rr * Drk;
    sparse_rows_apply<float, float, float>(so.lr.rows<float>(), gm, T1, T2, s);
  }
  transpose_split3<double>(bra, Dlb * n, Drb, Bp, ldB, pB, s);
  transpose_split3<float>(T2, Dlb * n, Rr * Drk, T2p, ldB, pT, s);
  {  // E3: Hout[b][(w' b')] = sum_{(a s)} bra[(a s)][b] T2[(a s)][(w' b')]
    Planes A = planes_at(Bp, ldB, pB), B = planes_at(T2p, ldB, pT);
    tc_gemm_bf16_pairs(A.p, A.ld, B.p, B.ld, Drb, Rr * Drk, Dlb * n, 6, kPairA, kPairB, Hout,
                       (long long)Rr * Drk, 1, 1, s);
  }
}

void env_right_emu(a2_ctx* c, const SiteOps& so, const float* Hin, const double* bra, int Dlb,
                   int Drb, const double* ket, int Dlk, int Drk, float* Hout) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_ENV, s, env_flops(so, std::max(Dlb, Dlk), std::max(Drb, Drk)),
               4.0 * ((double)Dlb * Rl * Dlk + (double)Drb * Rr * Drk +
                      2.0 * Drb * Rr * n * Dlk + 2.0 * n * Drb * Rl * Dlk));
  const long long ldH = pad8(Drk), pH = round64((long long)Drb * Rr * ldH);
  const long long ldV = pad8(Drk), pV = round64((long long)n * Dlk * ldV);
  const long long ldB = pad8((long long)n * Drb), pB = round64((long long)Dlb * ldB);
  const long long pT = round64((long long)Rl * Dlk * ldB);
  c->cb.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * (pH + pV + pB)) +
                   sizeof(double) * (size_t)n * Dlk * Drk, s);
  __nv_bfloat16* Hp = c->cb.as<__nv_bfloat16>();
  __nv_bfloat16* Vp = Hp + 3 * pH;
  __nv_bfloat16* Bp = Vp + 3 * pV;
  double* Vt = reinterpret_cast<double*>(Bp + 3 * pB);
  c->tmp1.ensure(sizeof(float) * (size_t)Drb * Rr * n * Dlk, s);
  c->tmp2.ensure(sizeof(float) * (size_t)n * Drb * Rl * Dlk, s);
  c->t3.ensure(sizeof(__nv_bfloat16) * (size_t)(3 * pT), s);
  float* T1 = c->tmp1.as<float>();
  float* T2 = c->tmp2.as<float>();
  __nv_bfloat16* T2p = c->t3.as<__nv_bfloat16>();
  split3_ld<float>(Hin, (long long)Drb * Rr, Drk, Hp, ldH, pH, s);
  permute_swap01<double, double>(ket, Vt, n, Dlk, Drk, s);          // Vt[t][a'][b']
  split3_ld<double>(Vt, (long long)n * Dlk, Drk, Vp, ldV, pV, s);
  {  // F1: T1[(b w')][(t a')] = sum_b' Hin[(b w')][b'] Vt[(t a')][b']
    Planes A = planes_at(Hp, ldH, pH), B = planes_at(Vp, ldV, pV);
    tc_gemm_bf16_pairs(A.p, A.ld, B.p, B.ld, Drb * Rr, n * Dlk, Drk, 6, kPairA, kPairB, T1,
                       (long long)n * Dlk, 1, 1, s);
  }
  {  // F2 (FP32)
    SparseGeom gm;
    gm.veclen = Dlk;
    gm.in_sw = (long long)n * Dlk; gm.in_st = Dlk;
    gm.out_sw = Dlk; gm.out_ss = (long long)Drb * Rl * Dlk;
    gm.B1 = Drb; gm.in_b1 = (long long)Rr * n * Dlk; gm.out_b1 = (long long)Rl * Dlk;
    sparse_rows_apply<float, float, float>(so.rl.rows<float>(), gm, T1, T2, s);
  }
  split3_ld<double>(bra, Dlb, (long long)n * Drb, Bp, ldB, pB, s);
  transpose_split3<float>(T2, n * Drb, Rl * Dlk, T2p, ldB, pT, s);
  {  // F3: Hout[a][(w a')] = sum_{(s b)} bra[a][(s b)] T2[(s b)][(w a')]
    Planes A = planes_at(Bp, ldB, pB), B = planes_at(T2p, ldB, pT);
    tc_gemm_bf16_pairs(A.p, A.ld, B.p, B.ld, Dlb, Rl * Dlk, n * Drb, 6, kPairA, kPairB, Hout,
                       (long long)Rl * Dlk, 1, 1, s);
  }
}

// ---- environment updates to FP64-class accuracy on tcgen05 (FP64 envs): the two GEMMs
// emulated by the Ozaki scheme (tc_gemm_f64emu), the sparse MPO stage in double-float
// arithmetic.  Same contraction and intermediate layouts as env_left / env_right.
void env_left_f64e(a2_ctx* c, const SiteOps& so, const double* Hin, const double* bra, int Dlb,
                   int Drb, const double* ket, int Dlk, int Drk, double* Hout) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_ENV, s, env_flops(so, std::max(Dlb, Dlk), std::max(Drb, Drk)),
               8.0 * ((double)Dlb * Rl * Dlk + (double)Drb * Rr * Drk +
                      2.0 * Dlb * Rl * n * Drk + 2.0 * Dlb * n * Rr * Drk));
  const long long M1 = (long long)Dlb * Rl, N1 = (long long)n * Drk;
  const long long N3 = (long long)Rr * Drk, K3 = (long long)Dlb * n;
  const long long ldH = pad8(Dlk), pH = round64(M1 * ldH);
  const long long ldK = pad8(Dlk), pK = round64(N1 * ldK);
  const long long ldB = pad8(K3), pB = round64((long long)Drb * ldB);
  const long long pT = round64(N3 * ldB);
  const long long s1 = M1 * N1, p1 = (s1 + 3) / 4 * 4, s2 = K3 * N3;
  c->cb.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * (pH + pK + pB)), s);
  __nv_bfloat16* Hp = c->cb.as<__nv_bfloat16>();
  __nv_bfloat16* Kp = Hp + kOzSlices * pH;
  __nv_bfloat16* Bp = Kp + kOzSlices * pK;
  c->tmp1.ensure(std::max(sizeof(float) * 2 * (size_t)p1, sizeof(double) * (size_t)s2), s);
  c->tmp2.ensure(sizeof(double) * (size_t)s2, s);
  c->t3.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * pT), s);
  float* T1 = c->tmp1.as<float>();
  double* T2 = c->tmp2.as<double>();
  __nv_bfloat16* T2p = c->t3.as<__nv_bfloat16>();
  ozaki_split(Hin, Dlk, 1, (int)M1, Dlk, Hp, ldH, pH, s);            // rows (a w), K = a'
  ozaki_split(ket, 1, N1, (int)N1, Dlk, Kp, ldK, pK, s);             // rows (t b'), K = a'
  // E1: T1[(a w)][(t b')] = sum_a' Hin[(a w)][a'] ket[a'][(t b')]   (FP32 pair out)
  tc_gemm_f64emu(Hp, ldH, pH, Kp, ldK, pK, (int)M1, (int)N1, Dlk, nullptr, N1, c->tf, s, T1, p1);
  {  // E2: T2[(a s)][(w' b')] = sum_{w,t} A[w,s,t,w'] T1[(a w)][(t b')]   (FP64 out)
    SparseGeom gm;
    gm.veclen = Drk;
    gm.in_sw = N1; gm.in_st = Drk;
    gm.out_sw = Drk; gm.out_ss = N3;
    gm.B1 = Dlb; gm.in_b1 = (long long)Rl * N1; gm.out_b1 = (long long)n * N3;
    sparse_rows_apply_df(so.lr.rows<float>(), gm, T1, p1, nullptr, 0, T2, s);
  }
  // E3: Hout[b][(w' b')] = sum_{(a s)} bra[(a s)][b] T2[(a s)][(w' b')]
  ozaki_split(bra, 1, Drb, Drb, (int)K3, Bp, ldB, pB, s);            // rows b, K = (a s)
  ozaki_split_cols(T2, N3, (int)N3, (int)K3, T2p, ldB, pT, s);      // rows (w' b'), K = (a s)
  tc_gemm_f64emu(Bp, ldB, pB, T2p, ldB, pT, Drb, (int)N3, (int)K3, Hout, N3, c->tf, s);
}

void env_right_f64e(a2_ctx* c, const SiteOps& so, const double* Hin, const double* bra, int Dlb,
                    int Drb, const double* ket, int Dlk, int Drk, double* Hout) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_ENV, s, env_flops(so, std::max(Dlb, Dlk), std::max(Drb, Drk)),
               8.0 * ((double)Dlb * Rl * Dlk + (double)Drb * Rr * Drk +
                      2.0 * Drb * Rr * n * Dlk + 2.0 * n * Drb * Rl * Dlk));
  const long long M1 = (long long)Drb * Rr, N1 = (long long)n * Dlk;
  const long long N3 = (long long)Rl * Dlk, K3 = (long long)n * Drb;
  const long long ldH = pad8(Drk), pH = round64(M1 * ldH);
  const long long ldV = pad8(Drk), pV = round64(N1 * ldV);
  const long long ldB = pad8(K3), pB = round64((long long)Dlb * ldB);
  const long long pT = round64(N3 * ldB);
  const long long s1 = M1 * N1, p1 = (s1 + 3) / 4 * 4, s2 = K3 * N3;
  c->cb.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * (pH + pV + pB)) +
                   sizeof(double) * (size_t)n * Dlk * Drk, s);
  __nv_bfloat16* Hp = c->cb.as<__nv_bfloat16>();
  __nv_bfloat16* Vp = Hp + kOzSlices * pH;
  __nv_bfloat16* Bp = Vp + kOzSlices * pV;
  double* Vt = reinterpret_cast<double*>(Bp + kOzSlices * pB);
  c->tmp1.ensure(std::max(sizeof(float) * 2 * (size_t)p1, sizeof(double) * (size_t)s2), s);
  c->tmp2.ensure(sizeof(double) * (size_t)s2, s);
  c->t3.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * pT), s);
  float* T1 = c->tmp1.as<float>();
  double* T2 = c->tmp2.as<double>();
  __nv_bfloat16* T2p = c->t3.as<__nv_bfloat16>();
  permute_swap01<double, double>(ket, Vt, n, Dlk, Drk, s);            // Vt[t][a'][b']
  ozaki_split(Hin, Drk, 1, (int)M1, Drk, Hp, ldH, pH, s);             // rows (b w'), K = b'
  ozaki_split(Vt, Drk, 1, (int)N1, Drk, Vp, ldV, pV, s);              // rows (t a'), K = b'
  // F1: T1[(b w')][(t a')] = sum_b' Hin[(b w')][b'] Vt[(t a')][b']   (FP32 pair out)
  tc_gemm_f64emu(Hp, ldH, pH, Vp, ldV, pV, (int)M1, (int)N1, Drk, nullptr, N1, c->tf, s, T1, p1);
  {  // F2: T2[(s b)][(w a')] = sum_{w',t} A[w,s,t,w'] T1[(b w')][(t a')]   (FP64 out)
    SparseGeom gm;
    gm.veclen = Dlk;
    gm.in_sw = N1; gm.in_st = Dlk;
    gm.out_sw = Dlk; gm.out_ss = (long long)Drb * N3;
    gm.B1 = Drb; gm.in_b1 = (long long)Rr * N1; gm.out_b1 = N3;
    sparse_rows_apply_df(so.rl.rows<float>(), gm, T1, p1, nullptr, 0, T2, s);
  }
  // F3: Hout[a][(w a')] = sum_{(s b)} bra[a][(s b)] T2[(s b)][(w a')]
  ozaki_split(bra, K3, 1, Dlb, (int)K3, Bp, ldB, pB, s);             // rows a, K = (s b)
  ozaki_split_cols(T2, N3, (int)N3, (int)K3, T2p, ldB, pT, s);      // rows (w a'), K = (s b)
  tc_gemm_f64emu(Bp, ldB, pB, T2p, ldB, pT, Dlb, (int)N3, (int)K3, Hout, N3, c->tf, s);
}

// Environment updates this small stay on the FP64 SIMT kernels (the Ozaki path costs a
// dozen launches and 36 tensor-core products per FP64 product).
constexpr double kF64eEnvMinFlops = 2e8;

// Split-K factor so that the skinny S4 GEMM fills the GPU.
int pick_splitk(int M, int N, int K, int tile) {
  const long long tiles = (long long)cdiv(M, tile) * cdiv(N, tile);
  int sk = (int)std::max<long long>(1, 608 / std::max<long long>(1, tiles));
  sk = std::min(sk, std::max(1, K / 256));
  return std::max(1, std::min(sk, 64));
}

// y = H_eff x (two-site, App. A) in compute type T; x, y in T.
template <typename T>
void heff_T(a2_ctx* c, const SiteOps& A1, const SiteOps& A2, const T* HL, const T* HR, int Dl,
            int Dr, const T* x, T* y) {
  const int n1 = A1.n, n2 = A2.n, Rl = A1.Rl, R1 = A1.Rr, Rr = A2.Rr;
  cudaStream_t s = c->stream;
  const size_t s1 = (size_t)Dl * Rl * n1 * n2 * Dr;
  const size_t s2 = (size_t)Dl * R1 * n1 * n2 * Dr;
  const size_t s3 = (size_t)Dl * n1 * n2 * Rr * Dr;
  ProfScope ps(PK_HEFF_SIMT, s, heff_flops(A1, A2, Dl, Dr),
               sizeof(T) * (2.0 * (s1 + s2 + s3) + (double)Dl * Rl * Dl + (double)Dr * Rr * Dr));
  c->t1.ensure(sizeof(T) * std::max(s1, s3), s);
  c->t2.ensure(sizeof(T) * s2, s);
  T* T1 = c->t1.as<T>();
  T* T2 = c->t2.as<T>();
  T* T3 = c->t1.as<T>();
  const long long N1 = (long long)n1 * n2 * Dr;
  {  // S1
    SimtGemm<T, T> g;
    g.M = Dl * Rl; g.N = (int)N1; g.K = Dl;
    g.A = HL; g.sam = Dl; g.sak = 1;
    g.B = x; g.sbn = 1; g.sbk = N1;
    g.C = T1; g.scm = N1; g.scn = 1;
    simt_gemm(g, s);
  }
  {  // S2: rows (w1, s1), entries (w, t1); vector (t2, b')
    SparseGeom gm;
    gm.veclen = n2 * Dr;
    gm.in_sw = (long long)n1 * n2 * Dr; gm.in_st = (long long)n2 * Dr;
    gm.out_sw = (long long)n1 * n2 * Dr; gm.out_ss = (long long)n2 * Dr;
    gm.B1 = Dl; gm.in_b1 = (long long)Rl * n1 * n2 * Dr; gm.out_b1 = (long long)R1 * n1 * n2 * Dr;
    sparse_rows_apply<T, T, T>(A1.lr.rows<T>(), gm, T1, T2, s);
  }
  {  // S3: batch (a, s1); rows (w2, s2), entries (w1, t2); vector b'
    SparseGeom gm;
    gm.veclen = Dr;
    gm.in_sw = (long long)n1 * n2 * Dr; gm.in_st = Dr;
    gm.out_sw = Dr; gm.out_ss = (long long)Rr * Dr;
    gm.B1 = Dl; gm.B2 = n1;
    gm.in_b1 = (long long)R1 * n1 * n2 * Dr; gm.in_b2 = (long long)n2 * Dr;
    gm.out_b1 = (long long)n1 * n2 * Rr * Dr; gm.out_b2 = (long long)n2 * Rr * Dr;
    sparse_rows_apply<T, T, T>(A2.lr.rows<T>(), gm, T2, T3, s);
  }
  {  // S4: y[(a s1 s2)][b] = sum_{(w2 b')} T3[(a s1 s2)][(w2 b')] HR[b][(w2 b')]
    SimtGemm<T, T> g;
    g.M = Dl * n1 * n2; g.N = Dr; g.K = Rr * Dr;
    g.A = T3; g.sam = g.K; g.sak = 1;
    g.B = HR; g.sbn = g.K; g.sbk = 1;
    g.C = y; g.scm = Dr; g.scn = 1;
    g.splitk = pick_splitk(g.M, g.N, g.K, sizeof(T) == 8 ? 64 : 128);
    if (g.splitk > 1) {
      g.mode = GEMM_ATOMIC;
      fill_zero(y, sizeof(T) * (size_t)g.M * g.N, s);
    }
    simt_gemm(g, s);
  }
}

// y = H_eff x for the one-site micro-step at core j (one-site case of Alg. 1 / Alg. 2):
//   y[a,s,b] = sum HL[a,w,a'] A_j[w,s,t,w'] HR[b,w',b'] x[a',t,b']
// as T1 = HL x (GEMM over a'), the MPO core on the rows (sparse), and the contraction
// with HR over (w', b') (GEMM); compute type T.
template <typename T>
void heff1_T(a2_ctx* c, const SiteOps& so, const T* HL, const T* HR, int Dl, int Dr, const T* x,
             T* y) {
  const int n = so.n, Rl = so.Rl, Rr = so.Rr;
  cudaStream_t s = c->stream;
  ProfScope ps(PK_HEFF_SIMT, s, env_flops(so, Dl, Dr),
               sizeof(T) * ((double)Dl * Rl * Dl + (double)Dr * Rr * Dr +
                            2.0 * Dl * Rl * n * Dr + 2.0 * Dl * n * Rr * Dr));
  c->t1.ensure(sizeof(T) * (size_t)Dl * Rl * n * Dr, s);
  c->t2.ensure(sizeof(T) * (size_t)Dl * n * Rr * Dr, s);
  T* T1 = c->t1.as<T>();
  T* T2 = c->t2.as<T>();
  {  // T1[(a w)][(t b')] = sum_a' HL[(a w)][a'] x[a'][(t b')]
    SimtGemm<T, T> g;
    g.M = Dl * Rl; g.N = n * Dr; g.K = Dl;
    g.A = HL; g.sam = Dl; g.sak = 1;
    g.B = x; g.sbn = 1; g.sbk = (long long)n * Dr;
    g.C = T1; g.scm = (long long)n * Dr; g.scn = 1;
    simt_gemm(g, s);
  }
  {  // T2[(a s)][(w' b')] = sum_{w,t} A[w,s,t,w'] T1[(a w)][(t b')]
    SparseGeom gm;
    gm.veclen = Dr;
    gm.in_sw = (long long)n * Dr; gm.in_st = Dr;
    gm.out_sw = Dr; gm.out_ss = (long long)Rr * Dr;
    gm.B1 = Dl; gm.in_b1 = (long long)Rl * n * Dr; gm.out_b1 = (long long)n * Rr * Dr;
    sparse_rows_apply<T, T, T>(so.lr.rows<T>(), gm, T1, T2, s);
  }
  {  // y[(a s)][b] = sum_{(w' b')} T2[(a s)][(w' b')] HR[b][(w' b')]
    SimtGemm<T, T> g;
    g.M = Dl * n; g.N = Dr; g.K = Rr * Dr;
    g.A = T2; g.sam = g.K; g.sak = 1;
    g.B = HR; g.sbn = g.K; g.sbk = 1;
    g.C = y; g.scm = Dr; g.scn = 1;
    g.splitk = pick_splitk(g.M, g.N, g.K, sizeof(T) == 8 ? 64 : 128);
    if (g.splitk > 1) {
      g.mode = GEMM_ATOMIC;
      fill_zero(y, sizeof(T) * (size_t)g.M * g.N, s);
    }
    simt_gemm(g, s);
  }
}

double heff_flops(const SiteOps& A1, const SiteOps& A2, int Dl, int Dr) {
  const double n1 = A1.n, n2 = A2.n;
  return 2.0 * n1 * n2 * Dl * Dr * (A1.Rl * (double)Dl + A2.Rr * (double)Dr) +
         2.0 * n2 * Dl * Dr * (double)A1.nnz + 2.0 * n1 * Dl * Dr * (double)A2.nnz;
}
double env_flops(const SiteOps& so, int Dl, int Dr) {
  return 2.0 * so.n * (double)Dl * Dr * (so.Rl * (double)Dl + so.Rr * (double)Dr) +
         2.0 * (double)Dl * Dr * (double)so.nnz;
}

// BF16 environments with padded rows for TMA: L [(a w)][a'] -> ld pad8(Dl); R [b][(w2 b')].
// With three planes each value is split into BF16 hi + mid + lo slices (plane 0 alone
// is the plain BF16 rounding used by the BF16 matvec).
// Fold of an identity-on-physical block W = I (x) G + W_rest (App. A contraction regrouped):
//   A_k = I (x) G:     sum_w L[a,w,a'] G[w,w1] = Lt[a,w1,a'], so stage S2's G part is the
//                      GEMM Lt x (written straight into T2);
//   A_{k+1} = I (x) G: sum_w2 G[w1,w2] R[b,w2,b'] = Rt[b,w1,b'], so stage S3's G part
//                      becomes a second K segment of S4 over T2: sum_{w1,b'} T2 Rt.
// Lt / Rt are built once per local problem (the environments are fixed during it).
struct Bf16Envs {
  DevBuf buf, fbuf, ftmp;
  const __nv_bfloat16* L = nullptr;
  const __nv_bfloat16* R = nullptr;
  const __nv_bfloat16* Lt = nullptr;    // [(a w1)][a'], row stride ldl, plane ltplane
  const __nv_bfloat16* Rt = nullptr;    // [b][w1][b'] dense, plane rtplane
  long long ldl = 0, ldr = 0, lplane = 0, rplane = 0, ltplane = 0, rtplane = 0;
  int planes = 0;
  template <typename T>
  void set(a2_ctx* c, const T* Lf, int Dl, int Rl, const T* Rf, int Dr, int Rr, int np,
           const SiteOps* A1 = nullptr, const SiteOps* A2 = nullptr) {
    cudaStream_t s = c->stream;
    ldl = pad8(Dl);
    ldr = pad8((long long)Rr * Dr);
    lplane = ((long long)Dl * Rl * ldl + 63) / 64 * 64;   // keep planes 128-byte aligned
    rplane = ((long long)Dr * ldr + 63) / 64 * 64;
    planes = np;
    buf.ensure(sizeof(__nv_bfloat16) * (size_t)(np * (lplane + rplane)), s);
    __nv_bfloat16* lb = buf.as<__nv_bfloat16>();
    __nv_bfloat16* rb = lb + np * lplane;
    if (np == 1) {
      convert_ld<T, __nv_bfloat16>(Lf, lb, (long long)Dl * Rl, Dl, ldl, s);
      convert_ld<T, __nv_bfloat16>(Rf, rb, Dr, (long long)Rr * Dr, ldr, s);
    } else {
      split3_ld<T>(Lf, (long long)Dl * Rl, Dl, lb, ldl, lplane, s);
      split3_ld<T>(Rf, Dr, (long long)Rr * Dr, rb, ldr, rplane, s);
    }
    L = lb;
    R = rb;
    Lt = Rt = nullptr;
    if (!A1 || !A2) return;
    const bool fl = A1->fold();
    const bool fr = A2->fold() && Dr % 8 == 0 && 128 % (A1->n * A2->n) == 0;
    if (!fl && !fr) return;
    const int R1 = A1->Rr;
    ltplane = fl ? ((long long)Dl * R1 * ldl + 63) / 64 * 64 : 0;
    rtplane = fr ? ((long long)Dr * R1 * Dr + 63) / 64 * 64 : 0;
    fbuf.ensure(sizeof(__nv_bfloat16) * (size_t)(np * (ltplane + rtplane)), s);
    ftmp.ensure(sizeof(T) * (size_t)std::max(fl ? (long long)Dl * R1 * Dl : 0,
                                             fr ? (long long)Dr * R1 * Dr : 0), s);
    T* tmp = ftmp.as<T>();
    __nv_bfloat16* ltb = fbuf.as<__nv_bfloat16>();
    __nv_bfloat16* rtb = ltb + np * ltplane;
    if (fl) {   // Lt[a][w1][a'] = sum_w G[w][w1] L[a][w][a']
      SparseGeom gm;
      gm.veclen = Dl;
      gm.in_sw = Dl; gm.out_sw = Dl;
      gm.B1 = Dl; gm.in_b1 = (long long)Rl * Dl; gm.out_b1 = (long long)R1 * Dl;
      sparse_rows_apply<T, T, T>(A1->g_lr.rows<T>(), gm, Lf, tmp, s);
      if (np == 1) convert_ld<T, __nv_bfloat16>(tmp, ltb, (long long)Dl * R1, Dl, ldl, s);
      else split3_ld<T>(tmp, (long long)Dl * R1, Dl, ltb, ldl, ltplane, s);
      Lt = ltb;
    }
    if (fr) {   // Rt[b][w1][b'] = sum_w2 G[w1][w2] R[b][w2][b']
      SparseGeom gm;
      gm.veclen = Dr;
      gm.in_sw = Dr; gm.out_sw = Dr;
      gm.B1 = Dr; gm.in_b1 = (long long)Rr * Dr; gm.out_b1 = (long long)R1 * Dr;
      sparse_rows_apply<T, T, T>(A2->g_rl.rows<T>(), gm, Rf, tmp, s);
      const long long cols = (long long)R1 * Dr;
      if (np == 1) convert_ld<T, __nv_bfloat16>(tmp, rtb, Dr, cols, cols, s);
      else split3_ld<T>(tmp, Dr, cols, rtb, cols, rtplane, s);
      Rt = rtb;
    }
  }
  HeffFold fold() const {
    HeffFold f;
    f.Lt = Lt; f.ltplane = ltplane;
    f.Rt = Rt; f.rtplane = rtplane;
    return f;
  }
};

void heff_bf16(a2_ctx* c, const SiteOps& A1, const SiteOps& A2, const Bf16Envs& E, int Dl, int Dr,
               const double* x, double* y) {
  const long long N = (long long)Dl * A1.n * A2.n * Dr;
  c->ya.ensure(sizeof(float) * N, c->stream);
  const auto& W1 = E.Lt ? A1.lr_rest : A1.lr;
  const auto& W2 = E.Rt ? A2.lr_rest : A2.lr;
  tc_heff_bf16(c->stream, A1.n, A2.n, A1.Rl, A1.Rr, A2.Rr, Dl, Dr, E.L, E.ldl, E.R, E.ldr, x,
               c->ya.as<float>(), W1.rows<float>(), W2.rows<float>(), E.fold(), c->t1, c->t2,
               c->t3, c->tf);
  convert<float, double>(c->ya.as<float>(), y, N, c->stream);
}

void heff_emu(a2_ctx* c, const SiteOps& A1, const SiteOps& A2, const Bf16Envs& E, int Dl, int Dr,
              const double* x, double* y) {
  A2_REQUIRE(E.planes == 3, "split environments required");
  const long long N = (long long)Dl * A1.n * A2.n * Dr;
  c->ya.ensure(sizeof(float) * N, c->stream);
  const auto& W1 = E.Lt ? A1.lr_rest : A1.lr;
  const auto& W2 = E.Rt ? A2.lr_rest : A2.lr;
  tc_heff_f32emu(c->stream, A1.n, A2.n, A1.Rl, A1.Rr, A2.Rr, Dl, Dr, E.L, E.ldl, E.lplane, E.R,
                 E.ldr, E.rplane, x, c->ya.as<float>(), W1.rows<float>(), W2.rows<float>(),
                 E.fold(), c->t1, c->t2, c->t3, c->tf);
  convert<float, double>(c->ya.as<float>(), y, N, c->stream);
}

// FP64 environments as Ozaki slices (kOzSlices BF16 planes each) for the FP64-emulated
// H_eff: L [(a w)][a'] (rows Dl*Rl, K = Dl), R [b][(w2 b')] (rows Dr, K = Rr*Dr).
struct OzEnvs {
  DevBuf buf;
  const __nv_bfloat16* L = nullptr;
  const __nv_bfloat16* R = nullptr;
  long long ldl = 0, ldr = 0, lplane = 0, rplane = 0;
  void set(a2_ctx* c, const double* Lf, int Dl, int Rl, const double* Rf, int Dr, int Rr) {
    cudaStream_t s = c->stream;
    ProfScope ps(PK_F64E_SPLIT, s, 0.0,
                 10.0 * ((double)Dl * Rl * Dl + (double)Dr * Rr * Dr) * 2.0);
    ldl = pad8(Dl);
    ldr = pad8((long long)Rr * Dr);
    lplane = ((long long)Dl * Rl * ldl + 63) / 64 * 64;
    rplane = ((long long)Dr * ldr + 63) / 64 * 64;
    buf.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * (lplane + rplane)), s);
    __nv_bfloat16* lb = buf.as<__nv_bfloat16>();
    __nv_bfloat16* rb = lb + kOzSlices * lplane;
    ozaki_split(Lf, Dl, 1, Dl * Rl, Dl, lb, ldl, lplane, s);
    ozaki_split(Rf, (long long)Rr * Dr, 1, Dr, Rr * Dr, rb, ldr, rplane, s);
    L = lb;
    R = rb;
  }
};

// y = H_eff x to FP64-class accuracy: the tensor-core stages S1 and S4 emulated by the
// Ozaki scheme (tc_gemm_f64emu), the sparse MPO stages S2, S3 in double-float arithmetic
// (FP32 pairs, ~2^-48; the FP64 pipe of this GPU is ~60x slower than its FP32 pipe);
// the full MPO cores are used (no identity-block fold).
void heff_f64emu(a2_ctx* c, const SiteOps& A1, const SiteOps& A2, const OzEnvs& E, int Dl,
                 int Dr, const double* x, double* y) {
  A2_REQUIRE(E.L && E.R, "FP64-emulation environments not set");
  const int n1 = A1.n, n2 = A2.n, Rl = A1.Rl, R1 = A1.Rr, Rr = A2.Rr;
  cudaStream_t s = c->stream;
  const long long NX = (long long)n1 * n2 * Dr;
  const long long ldx = pad8(Dl);
  const long long xplane = (NX * ldx + 63) / 64 * 64;
  const long long s1 = (long long)Dl * Rl * NX, s2 = (long long)Dl * R1 * NX;
  const long long M4 = (long long)Dl * n1 * n2, K4 = (long long)Rr * Dr;
  const long long s3 = M4 * K4;
  const long long ld3 = pad8(K4);
  const long long plane3 = (M4 * ld3 + 63) / 64 * 64;
  // T1 and T2 as FP32 pairs (hi plane, lo plane), T3 in FP64 (the slicing input)
  const long long p1 = (s1 + 3) / 4 * 4, p2 = (s2 + 3) / 4 * 4;
  c->xa.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * xplane), s);
  c->t1.ensure(std::max(sizeof(float) * 2 * (size_t)p1, sizeof(double) * (size_t)s3), s);
  c->t2.ensure(sizeof(float) * 2 * (size_t)p2, s);
  c->t3.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * plane3), s);
  __nv_bfloat16* XT = c->xa.as<__nv_bfloat16>();
  float* T1 = c->t1.as<float>();
  float* T2 = c->t2.as<float>();
  double* T3 = c->t1.as<double>();
  __nv_bfloat16* T3p = c->t3.as<__nv_bfloat16>();
  {  // slices of x^T: row n = column n of x [a'][(s1 s2 b')]
    ProfScope ps(PK_F64E_SPLIT, s, 0.0, (8.0 + 2.0 * kOzSlices) * (double)NX * Dl);
    ozaki_split(x, 1, NX, (int)NX, Dl, XT, ldx, xplane, s);
  }
  {  // S1: T1[(a w)][(s1 s2 b')] = sum_a' L[(a w)][a'] x[a'][(s1 s2 b')]
    const double M = (double)Dl * Rl, N = (double)NX, K = Dl;
    ProfScope ps(PK_F64E_S1, s, 2.0 * M * N * K,
                 2.0 * kOzSlices * (M * K + N * K) + 8.0 * M * N);
    tc_gemm_f64emu(E.L, E.ldl, E.lplane, XT, ldx, xplane, Dl * Rl, (int)NX, Dl, nullptr, NX,
                   c->tf, s, T1, p1);
  }
  {  // S2 / S3 in double-float arithmetic (FP32 pairs) on the full MPO cores
    ProfScope ps(PK_F64E_SPARSE, s,
                 2.0 * A1.lr.nnz * (double)n2 * Dr * Dl +
                     2.0 * A2.lr.nnz * (double)Dr * Dl * n1,
                 8.0 * (double)(s1 + 2 * s2 + s3));
    SparseGeom g2;
    g2.veclen = n2 * Dr;
    g2.in_sw = NX; g2.in_st = (long long)n2 * Dr;
    g2.out_sw = NX; g2.out_ss = (long long)n2 * Dr;
    g2.B1 = Dl; g2.in_b1 = (long long)Rl * NX; g2.out_b1 = (long long)R1 * NX;
    sparse_rows_apply_df(A1.lr.rows<float>(), g2, T1, p1, T2, p2, nullptr, s);
    SparseGeom g3;
    g3.veclen = Dr;
    g3.in_sw = NX; g3.in_st = Dr;
    g3.out_sw = Dr; g3.out_ss = K4;
    g3.B1 = Dl; g3.B2 = n1;
    g3.in_b1 = (long long)R1 * NX; g3.in_b2 = (long long)n2 * Dr;
    g3.out_b1 = (long long)n1 * n2 * K4; g3.out_b2 = (long long)n2 * K4;
    sparse_rows_apply_df(A2.lr.rows<float>(), g3, T2, p2, nullptr, 0, T3, s);
  }
  {
    ProfScope ps(PK_F64E_SPLIT, s, 0.0, (8.0 + 2.0 * kOzSlices) * (double)s3);
    ozaki_split(T3, K4, 1, (int)M4, (int)K4, T3p, ld3, plane3, s);
  }
  {  // S4: y[(a s1 s2)][b] = sum_{(w2 b')} T3[(a s1 s2)][(w2 b')] R[b][(w2 b')]
    const double M = (double)M4, N = Dr, K = (double)K4;
    ProfScope ps(PK_F64E_S4, s, 2.0 * M * N * K,
                 2.0 * kOzSlices * (M * K + N * K) + 8.0 * M * N);
    tc_gemm_f64emu(T3p, ld3, plane3, E.R, E.ldr, E.rplane, (int)M4, Dr, (int)K4, y, Dr, c->tf,
                   s);
  }
}

// ============================================================================= engine
struct View {   // a TT as per-site device pointers and bond dims
  std::vector<const double*> core;
  std::vector<int> Dl, Dr;
  int n(int j, const a2_mpo* m) const { return m->phys[j]; }
};

template <typename T>
struct Engine {
  a2_ctx* c;
  const a2_mpo* mpo;
  int L;
  a2_precision prec;
  std::vector<DevBuf> HL, HR;            // envs in T
  std::vector<int> HLd, HRd;             // bond dims of the stored envs
  double flops = 0.0;
  long long matvecs = 0, matvecs_bf16 = 0, matvecs_f64 = 0;
  DevBuf cvt_bra, cvt_ket;
  Bf16Envs bfe;
  OzEnvs oze;   // FP64-emulation slices of the current local problem's environments

  Engine(a2_ctx* c_, const a2_mpo* m, a2_precision p) : c(c_), mpo(m), L(m->L), prec(p) {
    HL.resize(L + 1);
    HR.resize(L + 1);
    HLd.assign(L + 1, 0);
    HRd.assign(L + 1, 0);
  }

  void set_unit(DevBuf& b) {
    b.ensure(sizeof(T), c->stream);
    const T one = T(1);
    A2_CUDA(cudaMemcpyAsync(b.p, &one, sizeof(T), cudaMemcpyHostToDevice, c->stream));
    A2_CUDA(cudaStreamSynchronize(c->stream));   // `one` lives on the host stack
  }

  // FP64-class environments on the tensor cores (Ozaki scheme) for the FP64-emulated and
  // the mixed modes, once an update is large enough to pay for the slicing
  bool f64e_env(int j, int Dl, int Dr) const {
    return (prec == A2_F64EMU || prec == A2_BF16 || prec == A2_F32EMU) &&
           env_flops(mpo->site[j], Dl, Dr) >= kF64eEnvMinFlops;
  }

  // env update with FP64 cores converted to T
  void left_update(const T* Hin, int j, const double* bra, int Dlb, int Drb, const double* ket,
                   int Dlk, int Drk, T* Hout) {
    const int n = mpo->phys[j];
    if constexpr (sizeof(T) == 8) {
      if (f64e_env(j, std::max(Dlb, Dlk), std::max(Drb, Drk))) {
        env_left_f64e(c, mpo->site[j], Hin, bra, Dlb, Drb, ket, Dlk, Drk, Hout);
        flops += env_flops(mpo->site[j], std::max(Dlb, Dlk), std::max(Drb, Drk));
        return;
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (prec == A2_BF16 || prec == A2_F32EMU) {
        env_left_emu(c, mpo->site[j], Hin, bra, Dlb, Drb, ket, Dlk, Drk, Hout);
        flops += env_flops(mpo->site[j], std::max(Dlb, Dlk), std::max(Drb, Drk));
        return;
      }
    }
    const T* b = as_compute<T>(c, bra, (long long)Dlb * n * Drb, cvt_bra);
    const T* k = (ket == bra) ? b : as_compute<T>(c, ket, (long long)Dlk * n * Drk, cvt_ket);
    env_left<T>(c, mpo->site[j], Hin, b, Dlb, Drb, k, Dlk, Drk, Hout);
    flops += env_flops(mpo->site[j], std::max(Dlb, Dlk), std::max(Drb, Drk));
  }
  void right_update(const T* Hin, int j, const double* bra, int Dlb, int Drb,
                    const double* ket, int Dlk, int Drk, T* Hout) {
    const int n = mpo->phys[j];
    if constexpr (sizeof(T) == 8) {
      if (f64e_env(j, std::max(Dlb, Dlk), std::max(Drb, Drk))) {
        env_right_f64e(c, mpo->site[j], Hin, bra, Dlb, Drb, ket, Dlk, Drk, Hout);
        flops += env_flops(mpo->site[j], std::max(Dlb, Dlk), std::max(Drb, Drk));
        return;
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (prec == A2_BF16 || prec == A2_F32EMU) {
        env_right_emu(c, mpo->site[j], Hin, bra, Dlb, Drb, ket, Dlk, Drk, Hout);
        flops += env_flops(mpo->site[j], std::max(Dlb, Dlk), std::max(Drb, Drk));
        return;
      }
    }
    const T* b = as_compute<T>(c, bra, (long long)Dlb * n * Drb, cvt_bra);
    const T* k = (ket == bra) ? b : as_compute<T>(c, ket, (long long)Dlk * n * Drk, cvt_ket);
    env_right<T>(c, mpo->site[j], Hin, b, Dlb, Drb, k, Dlk, Drk, Hout);
    flops += env_flops(mpo->site[j], std::max(Dlb, Dlk), std::max(Drb, Drk));
  }

  // y = H_eff x at bond k with FP64 vectors and envs HL_ (T) / HR_ (T)
  void matvec(int k, const T* HL_, const T* HR_, int Dl, int Dr, const double* x, double* y) {
    const SiteOps& A1 = mpo->site[k];
    const SiteOps& A2 = mpo->site[k + 1];
    const long long N = (long long)Dl * A1.n * A2.n * Dr;
    if constexpr (sizeof(T) == 8) {
      heff_T<double>(c, A1, A2, HL_, HR_, Dl, Dr, x, y);
    } else {
      c->xa.ensure(sizeof(float) * N, c->stream);
      c->ya.ensure(sizeof(float) * N, c->stream);
      convert<double, float>(x, c->xa.as<float>(), N, c->stream);
      heff_T<float>(c, A1, A2, HL_, HR_, Dl, Dr, c->xa.as<float>(), c->ya.as<float>());
      convert<float, double>(c->ya.as<float>(), y, N, c->stream);
    }
    flops += heff_flops(A1, A2, Dl, Dr);
    ++matvecs;
  }
  void matvec_bf16(int k, int Dl, int Dr, const double* x, double* y) {
    heff_bf16(c, mpo->site[k], mpo->site[k + 1], bfe, Dl, Dr, x, y);
    flops += heff_flops(mpo->site[k], mpo->site[k + 1], Dl, Dr);
    ++matvecs;
    ++matvecs_bf16;
  }
  void matvec_emu(int k, int Dl, int Dr, const double* x, double* y) {
    heff_emu(c, mpo->site[k], mpo->site[k + 1], bfe, Dl, Dr, x, y);
    flops += heff_flops(mpo->site[k], mpo->site[k + 1], Dl, Dr);
    ++matvecs;
  }
  // FP64-emulated H_eff at bond k with the environments set in oze
  void matvec_f64e(int k, int Dl, int Dr, const double* x, double* y) {
    heff_f64emu(c, mpo->site[k], mpo->site[k + 1], oze, Dl, Dr, x, y);
    flops += heff_flops(mpo->site[k], mpo->site[k + 1], Dl, Dr);
    ++matvecs;
    ++matvecs_f64;
  }
  // one-site H_eff on the tensor cores with FP32-accurate products (environments in bfe)
  void matvec1_emu(int j, int Dl, int Dr, const double* x, double* y) {
    const SiteOps& A = mpo->site[j];
    const long long N = (long long)Dl * A.n * Dr;
    c->ya.ensure(sizeof(float) * N, c->stream);
    tc_heff1_f32emu(c->stream, A.n, A.Rl, A.Rr, Dl, Dr, bfe.L, bfe.ldl, bfe.lplane, bfe.R,
                    bfe.ldr, bfe.rplane, x, c->ya.as<float>(), A.lr.rows<float>(), c->t1, c->t2,
                    c->xa);
    convert<float, double>(c->ya.as<float>(), y, N, c->stream);
    flops += env_flops(A, Dl, Dr);
    ++matvecs;
  }
  // one-site H_eff at core j with FP64 vectors and envs HL_ / HR_ (T)
  void matvec1(int j, const T* HL_, const T* HR_, int Dl, int Dr, const double* x, double* y) {
    const SiteOps& A = mpo->site[j];
    const long long N = (long long)Dl * A.n * Dr;
    if constexpr (sizeof(T) == 8) {
      heff1_T<double>(c, A, HL_, HR_, Dl, Dr, x, y);
    } else {
      c->xa.ensure(sizeof(float) * N, c->stream);
      c->ya.ensure(sizeof(float) * N, c->stream);
      convert<double, float>(x, c->xa.as<float>(), N, c->stream);
      heff1_T<float>(c, A, HL_, HR_, Dl, Dr, c->xa.as<float>(), c->ya.as<float>());
      convert<float, double>(c->ya.as<float>(), y, N, c->stream);
    }
    flops += env_flops(A, Dl, Dr);
    ++matvecs;
  }
};

// ============================================================================= Lanczos
// residual tolerance of the BF16 tensor-core Lanczos phase (BF16 operator accuracy)
constexpr double kBf16Tol = 3e-3;
// tightest residual asked of the FP32-accurate split-product phase when the FP64
// refinement follows (its products carry ~1e-6 relative error, and the rounding order of
// its split-K sums varies from run to run, so tighter targets would stall)
constexpr double kSplitTol = 1e-6;

struct LanczosResult {
  double theta = 0.0;
  int matvecs = 0, cycles = 0;
  bool converged = false;
};

// Restarted Lanczos with full re-orthogonalisation (twice) for the lowest eigenpair of
// the operator `mv`, started from x0 (device, overwritten by the unit Ritz vector with
// <x, x0> >= 0).  Scalars are reduced on the device and read back once per step.
template <typename MV>
LanczosResult lanczos(a2_ctx* c, MV&& mv, double* x, long long N, double tol, int max_krylov,
                      int max_cycles) {
  cudaStream_t s = c->stream;
  const int m = (int)std::min<long long>(std::min(max_krylov, 63), N);
  c->wv.ensure(sizeof(double) * (size_t)(m + 3) * N, s);
  double* V = c->wv.as<double>();
  double* w = V + (size_t)m * N;
  double* x0 = w + N;
  double* tmp = x0 + N;
  A2_CUDA(cudaMemcpyAsync(x0, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  double nrm2 = dot_dev(c, x, x, N, 0);
  check_finite(nrm2, "Lanczos start vector");
  if (!(nrm2 > 0.0)) {   // zero start vector: use the constant vector
    std::vector<double> ones((size_t)N, 1.0);
    A2_CUDA(cudaMemcpyAsync(x, ones.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    A2_CUDA(cudaMemcpyAsync(x0, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    nrm2 = dot_dev(c, x, x, N, 0);
  }
  A2_CUDA(cudaMemcpyAsync(V, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  A2_CUDA(cudaMemcpyAsync(tmp, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  normalize_into(tmp, scal(c, 0), V, N, s);
  LanczosResult res;
  std::vector<double> alpha, beta;
  std::vector<double> ev(65);
  double* dev_ev = scal(c, 128);
  for (int cyc = 1; cyc <= max_cycles; ++cyc) {
    res.cycles = cyc;
    alpha.clear();
    beta.clear();
    int j = 0;
    bool conv = false;
    double theta = 0.0;
    std::vector<double> svec;
    for (j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * N;
      mv(vj, w);
      ++res.matvecs;
      // alpha_j = <v_j, w>; w -= alpha v_j + beta v_{j-1}
      ProfScope ps(PK_LANCZOS, s, 2.0 * N * (2.0 * (j + 1) * 2 + 6), 8.0 * N * (4.0 * (j + 1) + 6));
      dot_multi(vj, 0, 1, w, N, c->partial.as<double>(), scal(c, 1), s);
      lanczos_update(w, vj, j > 0 ? V + (size_t)(j - 1) * N : nullptr, scal(c, 1),
                     j > 0 ? beta.back() : 0.0, N, s);
      for (int pass = 0; pass < 2; ++pass) {   // full re-orthogonalisation
        dot_multi(V, N, j + 1, w, N, c->partial.as<double>(), scal(c, 8), s);
        gemv_sub(V, N, j + 1, scal(c, 8), w, N, s);
      }
      dot_multi(w, 0, 1, w, N, c->partial.as<double>(), scal(c, 2), s);
      fetch_scalars(c, 1, 2);
      const double a = c->h_scal[1];
      const double b2 = c->h_scal[2];
      check_finite(a, "Lanczos alpha");
      check_finite(b2, "Lanczos beta");
      const double b = std::sqrt(std::max(b2, 0.0));
      alpha.push_back(a);
      // lowest eigenpair of the tridiagonal T_j (device bisection + inverse iteration)
      const int k = j + 1;
      TridiagIn tin;
      tin.k = k;
      for (int i = 0; i < k; ++i) tin.a[i] = alpha[i];
      for (int i = 0; i + 1 < k; ++i) tin.b[i] = beta[i];
      tridiag_lowest(tin, dev_ev, s);
      A2_CUDA(cudaMemcpyAsync(ev.data(), dev_ev, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
      A2_CUDA(cudaStreamSynchronize(s));
      theta = ev[0];
      svec.assign(ev.begin() + 1, ev.begin() + 1 + k);
      const double resid = std::fabs(b * svec[k - 1]);
      const bool breakdown = b <= 1e-14 * std::max(1.0, std::fabs(theta));
      if (resid <= tol * std::max(1.0, std::fabs(theta)) || breakdown || k == N) {
        conv = true;
        ++j;
        break;
      }
      if (j == m - 1) { ++j; break; }
      beta.push_back(b);
      // v_{j+1} = w / b
      A2_CUDA(cudaMemcpyAsync(scal(c, 3), &b2, sizeof(double), cudaMemcpyHostToDevice, s));
      normalize_into(w, scal(c, 3), V + (size_t)(j + 1) * N, N, s);
      A2_CUDA(cudaStreamSynchronize(s));   // b2 is a host stack value
    }
    // Ritz vector x = V s (unit), becomes the restart vector
    A2_CUDA(cudaMemcpyAsync(scal(c, 8), svec.data(), sizeof(double) * svec.size(),
                            cudaMemcpyHostToDevice, s));
    gemv_set(V, N, (int)svec.size(), scal(c, 8), x, N, s);
    double xn = dot_dev(c, x, x, N, 4);
    A2_CUDA(cudaMemcpyAsync(V, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    normalize_into(x, scal(c, 4), V, N, s);
    A2_CUDA(cudaMemcpyAsync(x, V, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    (void)xn;
    res.theta = theta;
    if (conv) { res.converged = true; break; }
  }
  // sign convention <x, x0> >= 0
  const double sgn = dot_dev(c, x, x0, N, 5);
  if (sgn < 0) axpby(0.0, x, -1.0, x, N, s);
  return res;
}

// Extension One (extension remark after Alg. 2): the eigenpairs above the lowest of a
// local operator, one at a time, by Lanczos on the deflated operator
// (I - Q Q^T) H (I - Q Q^T) with Q the eigenvectors found so far, each started from
// `start` with those directions removed.  On return Q (K x N, row-major) holds the
// lowest eigenvector `x1` (normalised) in row 0 and the others below; the eigenvalues
// of rows 1..K-1 are returned.  K is capped at N.
template <class MV>
std::vector<double> deflated_eigs(a2_ctx* c, MV&& mv, const double* start, const double* x1,
                                  long long N, int K, double tol, int max_krylov,
                                  int max_cycles, DevBuf& Q, int* matvecs,
                                  std::atomic<int>* unconverged = nullptr) {
  cudaStream_t s = c->stream;
  K = (int)std::min<long long>(K, N);
  A2_REQUIRE(K >= 1 && K <= 64, "n_eig: at most 64 eigenvectors per local problem");
  Q.ensure(sizeof(double) * (size_t)K * N, s);
  double* Qp = Q.as<double>();
  DevBuf tmp;
  tmp.ensure(sizeof(double) * (size_t)N, s);
  double* coef = scal(c, 4200);
  auto project = [&](double* v, int k) {   // v -= Q_k Q_k^T v, twice
    for (int pass = 0; pass < 2; ++pass) {
      dot_multi(Qp, N, k, v, N, c->partial.as<double>(), coef, s);
      gemv_sub(Qp, N, k, coef, v, N, s);
    }
  };
  auto normalise = [&](double* v) {
    dot_multi(v, 0, 1, v, N, c->partial.as<double>(), scal(c, 4290), s);
    scale_dev(v, nullptr, scal(c, 4290), N, s);
  };
  A2_CUDA(cudaMemcpyAsync(Qp, x1, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  normalise(Qp);
  const double s2 = dot_dev(c, start, start, N, 6);
  std::vector<double> th;
  for (int e = 1; e < K; ++e) {
    double* v = Qp + (size_t)e * N;
    A2_CUDA(cudaMemcpyAsync(v, start, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    project(v, e);
    if (!(dot_dev(c, v, v, N, 6) > 1e-16 * s2)) {   // start inside span(Q): a fixed vector
      std::vector<double> h((size_t)N);
      for (long long i = 0; i < N; ++i) h[i] = std::sin(0.7 * (double)i + 0.3 * e);
      A2_CUDA(cudaMemcpyAsync(v, h.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
      A2_CUDA(cudaStreamSynchronize(s));
      project(v, e);
    }
    auto mvd = [&](const double* in, double* out) {
      A2_CUDA(cudaMemcpyAsync(tmp.p, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      project(tmp.as<double>(), e);
      mv(tmp.as<double>(), out);
      project(out, e);
    };
    LanczosResult lr = lanczos(c, mvd, v, N, tol, max_krylov, max_cycles);
    check_finite(lr.theta, "local eigenvalue (deflated)");
    if (!lr.converged && unconverged) unconverged->fetch_add(1);
    project(v, e);
    normalise(v);
    th.push_back(lr.theta);
    *matvecs += lr.matvecs;
  }
  return th;
}

// H_eff applications of one local problem replayed from a CUDA graph (one launch per
// application instead of one per stage kernel): the first call runs eagerly (it sizes
// the scratch buffers and lets the autotuners settle), the second is captured on the
// caller's stream and instantiated, later calls launch the graph.  The graph's pointers
// are fixed, so the vectors pass through two device buffers of its own.  Whatever cannot
// be captured (a synchronisation, an allocation) ends the capture and the applications
// stay eager.  Replays add the eager application's launch and flop counts to the
// counters, and their time to the profiler class PK_HEFF_GRAPH.
struct GraphedMV {
  a2_ctx* c;
  long long N;
  int state = 0;            // 0 eager next, 1 capture next, 2 replay, 3 eager for good
  DevBuf xg, yg;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0, mvs = 0, mvs16 = 0;
  double flops = 0.0;
  GraphedMV(a2_ctx* c_, long long n) : c(c_), N(n) {}
  GraphedMV(const GraphedMV&) = delete;
  GraphedMV& operator=(const GraphedMV&) = delete;
  ~GraphedMV() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  template <class MV, class Eng>
  void operator()(MV&& mv, Eng& eng, const double* in, double* out) {
    cudaStream_t s = c->stream;
    if (state == 3) {
      mv(in, out);
      return;
    }
    xg.ensure(sizeof(double) * N, s);
    yg.ensure(sizeof(double) * N, s);
    A2_CUDA(cudaMemcpyAsync(xg.p, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    if (state == 0) {
      const long long l0 = launch_count(), m0 = eng.matvecs, b0 = eng.matvecs_bf16;
      const double f0 = eng.flops;
      mv(xg.as<double>(), yg.as<double>());
      launches = launch_count() - l0;
      mvs = eng.matvecs - m0;
      mvs16 = eng.matvecs_bf16 - b0;
      flops = eng.flops - f0;
      state = 1;
    } else {
      if (state == 1) {
        cudaGraph_t g = nullptr;
        const long long l0 = launch_count(), m0 = eng.matvecs, b0 = eng.matvecs_bf16;
        const double f0 = eng.flops;
        bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          set_capturing(true);
          try {
            mv(xg.as<double>(), yg.as<double>());
          } catch (...) {
            ok = false;
          }
          set_capturing(false);
          // captured launches did not run: take back what the capture counted
          count_launches(l0 - launch_count());
          eng.matvecs = m0;
          eng.matvecs_bf16 = b0;
          eng.flops = f0;
          ok = (cudaStreamEndCapture(s, &g) == cudaSuccess) && ok && g;
          if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
          if (g) cudaGraphDestroy(g);
        }
        if (!ok) {
          (void)cudaGetLastError();   // capture errors are not sticky
          if (exec) cudaGraphExecDestroy(exec);
          exec = nullptr;
          state = 3;
          A2_CUDA(cudaMemcpyAsync(xg.p, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
          mv(xg.as<double>(), yg.as<double>());
          A2_CUDA(cudaMemcpyAsync(out, yg.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
          return;
        }
        state = 2;
      }
      {
        ProfScope ps(PK_HEFF_GRAPH, s, flops, 0.0);
        A2_CUDA(cudaGraphLaunch(exec, s));
      }
      count_launches(launches);
      eng.matvecs += mvs;
      eng.matvecs_bf16 += mvs16;
      eng.flops += flops;
    }
    A2_CUDA(cudaMemcpyAsync(out, yg.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  }
};

// Diagonal of H_eff at bond k (FP64): diag[a,s1,s2,b] = sum_{w,w1,w2} L[a,w,a]
// A_k[w,s1,s1,w1] A_k+1[w1,s2,s2,w2] R[b,w2,b] (preconditioner of the Davidson solver).
template <typename T>
void heff_diag(a2_ctx* c, const SiteOps& A1, const SiteOps& A2, const T* HL, const T* HR, int Dl,
               int Dr, double* diag) {
  cudaStream_t s = c->stream;
  const int n1 = A1.n, n2 = A2.n, Rl = A1.Rl, R1 = A1.Rr, Rr = A2.Rr;
  c->ck.ensure(sizeof(double) * ((size_t)Dl * Rl + (size_t)Dr * Rr + (size_t)Dl * n1 * R1 +
                                 (size_t)Dr * n2 * R1), s);
  double* Ld = c->ck.as<double>();
  double* Rd = Ld + (size_t)Dl * Rl;
  double* P1 = Rd + (size_t)Dr * Rr;
  double* Q = P1 + (size_t)Dl * n1 * R1;
  env_diag<T>(HL, Dl, Rl, Ld, s);
  env_diag<T>(HR, Dr, Rr, Rd, s);
  diag_action(A1.lr.rows<double>(), R1, n1, Ld, Rl, Dl, P1, s);   // P1[a][s1][w1]
  diag_action(A2.rl.rows<double>(), R1, n2, Rd, Rr, Dr, Q, s);    // Q[b][s2][w1]
  for (int s1 = 0; s1 < n1; ++s1)
    for (int s2 = 0; s2 < n2; ++s2) {
      SimtGemm<double, double> g;
      g.M = Dl; g.N = Dr; g.K = R1;
      g.A = P1 + (size_t)s1 * R1; g.sam = (long long)n1 * R1; g.sak = 1;
      g.B = Q + (size_t)s2 * R1; g.sbn = (long long)n2 * R1; g.sbk = 1;
      g.C = diag + (size_t)(s1 * n2 + s2) * Dr; g.scm = (long long)n1 * n2 * Dr; g.scn = 1;
      simt_gemm(g, s);
    }
}

// Davidson iteration with the diagonal preconditioner for the lowest eigenpair of `mv`
// (same stopping rule and sign convention as `lanczos`); x: start in, unit Ritz vector out.
template <typename MV>
LanczosResult davidson(a2_ctx* c, MV&& mv, const double* diag, double* x, long long N, double tol,
                       int max_sub, int max_iter) {
  cudaStream_t s = c->stream;
  const int m = (int)std::min<long long>(std::min(max_sub, 63), N);
  c->wv.ensure(sizeof(double) * ((size_t)2 * m + 4) * N, s);
  double* V = c->wv.as<double>();
  double* AV = V + (size_t)m * N;
  double* r = AV + (size_t)m * N;
  double* t = r + N;
  double* x0 = t + N;
  double* ax = x0 + N;
  A2_CUDA(cudaMemcpyAsync(x0, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  double nrm2 = dot_dev(c, x, x, N, 0);
  check_finite(nrm2, "Davidson start vector");
  if (!(nrm2 > 0.0)) {
    std::vector<double> ones((size_t)N, 1.0);
    A2_CUDA(cudaMemcpyAsync(x, ones.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    A2_CUDA(cudaMemcpyAsync(x0, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    nrm2 = dot_dev(c, x, x, N, 0);
  }
  normalize_into(x, scal(c, 0), V, N, s);
  LanczosResult res;
  mv(V, AV);
  ++res.matvecs;
  std::vector<double> G(64 * 64, 0.0), Gs(64 * 64), ev(64), evec(64 * 64), h(64);
  G[0] = dot_dev(c, V, AV, N, 1);
  int nv = 1;
  double* dG = scal(c, 4300);
  double* dev_ev = scal(c, 8500);
  double* dev_evec = dev_ev + 64;
  int* dstat = reinterpret_cast<int*>(dev_evec + 64 * 64);
  double* dtheta = scal(c, 3);
  for (int it = 0; it < max_iter; ++it) {
    res.cycles = it + 1;
    // Rayleigh-Ritz in span(V)
    for (int i = 0; i < nv; ++i)
      for (int j = 0; j < nv; ++j) Gs[i * nv + j] = G[i * 64 + j];
    A2_CUDA(cudaMemcpyAsync(dG, Gs.data(), sizeof(double) * nv * nv, cudaMemcpyHostToDevice, s));
    jacobi_eig(dG, nv, dev_ev, dev_evec, dstat, s);
    A2_CUDA(cudaMemcpyAsync(ev.data(), dev_ev, sizeof(double), cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaMemcpyAsync(evec.data(), dev_evec, sizeof(double) * nv, cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaStreamSynchronize(s));
    const double theta = ev[0];
    check_finite(theta, "Davidson Ritz value");
    res.theta = theta;
    A2_CUDA(cudaMemcpyAsync(scal(c, 8), evec.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, s));
    gemv_set(V, N, nv, scal(c, 8), x, N, s);
    gemv_set(AV, N, nv, scal(c, 8), ax, N, s);
    A2_CUDA(cudaMemcpyAsync(r, ax, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    axpby(-theta, x, 1.0, r, N, s);                          // r = A x - theta x
    const double rn = std::sqrt(std::max(dot_dev(c, r, r, N, 2), 0.0));
    check_finite(rn, "Davidson residual");
    if (rn <= tol * std::max(1.0, std::fabs(theta))) { res.converged = true; break; }
    if (nv == m) {                                           // restart from the Ritz pair
      A2_CUDA(cudaMemcpyAsync(V, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      A2_CUDA(cudaMemcpyAsync(AV, ax, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      nv = 1;
      G[0] = theta;
    }
    A2_CUDA(cudaMemcpyAsync(dtheta, &theta, sizeof(double), cudaMemcpyHostToDevice, s));
    precondition(r, diag, dtheta, t, N, s);
    A2_CUDA(cudaStreamSynchronize(s));                       // theta is a host stack value
    for (int pass = 0; pass < 2; ++pass) {
      dot_multi(V, N, nv, t, N, c->partial.as<double>(), scal(c, 8), s);
      gemv_sub(V, N, nv, scal(c, 8), t, N, s);
    }
    const double tn2 = dot_dev(c, t, t, N, 4);
    if (!(tn2 > 1e-28)) break;                               // no new direction
    normalize_into(t, scal(c, 4), V + (size_t)nv * N, N, s);
    mv(V + (size_t)nv * N, AV + (size_t)nv * N);
    ++res.matvecs;
    dot_multi(V, N, nv + 1, AV + (size_t)nv * N, N, c->partial.as<double>(), scal(c, 8), s);
    A2_CUDA(cudaMemcpyAsync(h.data(), scal(c, 8), sizeof(double) * (nv + 1), cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i <= nv; ++i) G[i * 64 + nv] = G[nv * 64 + i] = h[i];
    ++nv;
  }
  const double sgn = dot_dev(c, x, x0, N, 5);
  if (sgn < 0) axpby(0.0, x, -1.0, x, N, s);
  return res;
}

// ============================================================================= SVD step
// M (rows x cols, row-major) = P Sigma Q truncated (Alg. 1 step 2): P = the kept left
// singular vectors (left-orthonormal, this library's bidiagonalisation SVD, factor.cu),
// SQ = P^T M.  Returns the rank r and the discarded 2-norm.  P (rows x r) and SQ
// (r x cols) row-major.
void gemm_f64(a2_ctx* c, int M, int N, int K, const double* A, long long sam, long long sak,
              const double* B, long long sbn, long long sbk, double* C, long long ldc);

int svd_split_dev(a2_ctx* c, const double* M, int rows, int cols, int D_max, double tol,
                  double* P, double* SQ, double* discarded, std::vector<double>* sv_out = nullptr) {
  cudaStream_t s = c->stream;
  const double mm = std::max(rows, cols), nn = std::min(rows, cols);
  // algorithmic flops: bidiagonalisation, the back-transformation of the kept vectors
  // (bounded by nn of them), the product P^T M
  ProfScope ps(PK_SVD, s,
               4.0 * mm * nn * nn - 4.0 / 3.0 * nn * nn * nn + 4.0 * (double)rows * nn * nn +
                   2.0 * nn * (double)rows * cols,
               8.0 * (2.0 * rows * cols + 2.0 * rows * nn));
  const int r = svd_trunc(M, rows, cols, D_max, tol, P, discarded, sv_out, c->solver.fw, s);
  // SQ = P^T M : (r x cols)
  gemm_f64(c, r, cols, rows, P, 1, r, M, 1, cols, SQ, cols);
  return r;
}

// C = A (ra x k) * B (k x cb), all row-major FP64
// C[m][n] (row stride ldc) = sum_k A(m, k) B(n, k) in FP64, A(m, k) at A[m sam + k sak],
// B(n, k) at B[n sbn + k sbk]: on the tensor cores by the Ozaki scheme (FP64-class) when
// the context allows it (a mixed or FP64-emulated sweep) and the product is large enough
// to pay for the slicing, else on the FP64 SIMT kernel.
struct GemmTcScope {   // allows the Ozaki path for the lifetime of the scope
  a2_ctx* c;
  bool saved;
  GemmTcScope(a2_ctx* ctx, bool on) : c(ctx), saved(ctx->gemm_tc) { c->gemm_tc = on; }
  ~GemmTcScope() { c->gemm_tc = saved; }
};
constexpr double kF64eGemmMinFlops = 5e7;
void gemm_f64(a2_ctx* c, int M, int N, int K, const double* A, long long sam, long long sak,
              const double* B, long long sbn, long long sbk, double* C, long long ldc) {
  cudaStream_t s = c->stream;
  const bool tc_ok = (c->parent ? c->parent->gemm_tc : c->gemm_tc) && tc_available();
  if (tc_ok && M >= 16 && N >= 16 && K >= 16 && 2.0 * M * (double)N * K >= kF64eGemmMinFlops) {
    const long long ld = pad8(K), pA = round64((long long)M * ld), pB = round64((long long)N * ld);
    c->cb.ensure(sizeof(__nv_bfloat16) * (size_t)(kOzSlices * (pA + pB)), s);
    __nv_bfloat16* Ap = c->cb.as<__nv_bfloat16>();
    __nv_bfloat16* Bp = Ap + kOzSlices * pA;
    ozaki_split(A, sam, sak, M, K, Ap, ld, pA, s);
    ozaki_split(B, sbn, sbk, N, K, Bp, ld, pB, s);
    tc_gemm_f64emu(Ap, ld, pA, Bp, ld, pB, M, N, K, C, ldc, c->tf, s);
    return;
  }
  SimtGemm<double, double> g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.sam = sam; g.sak = sak;
  g.B = B; g.sbn = sbn; g.sbk = sbk;
  g.C = C; g.scm = ldc; g.scn = 1;
  simt_gemm(g, s);
}

void matmul_dev(a2_ctx* c, const double* A, int ra, int k, const double* B, int cb, double* C) {
  gemm_f64(c, ra, cb, k, A, k, 1, B, 1, cb, C, cb);
}

// ============================================================================= TT helpers
void tt_check(const a2_tt* tt) {
  A2_REQUIRE(tt && tt->L >= 2, "TT with at least two sites required");
  for (int j = 0; j < tt->L; ++j) A2_REQUIRE(tt->cores[j].p, "TT core not set");
  A2_REQUIRE(tt->dims[0] == 1 && tt->dims[tt->L] == 1, "TT boundary bonds must be 1");
}

// Thin QR of M (rows x cols, row-major, FP64): M = Q R with Q (rows x k) orthonormal
// columns and R (k x cols), k = min(rows, cols), computed as the LQ factorisation of M^T.
// Q and R are allocated here; returns k.
int qr_split_dev(a2_ctx* c, const double* M, int rows, int cols, DevBuf& Q, DevBuf& R) {
  cudaStream_t s = c->stream;
  const int kk = std::min(rows, cols);
  c->tmp2.ensure(sizeof(double) * ((size_t)rows * cols * 2 + (size_t)cols * kk), s);
  double* Mt = c->tmp2.as<double>();
  double* Lf = Mt + (size_t)rows * cols;
  double* Qf = Lf + (size_t)cols * kk;
  transpose2d<double, double>(M, Mt, rows, cols, s);
  const int k = c->solver.lq(Mt, cols, rows, Lf, Qf, s);   // Mt = Lf (cols x k) Qf (k x rows)
  Q.ensure(sizeof(double) * (size_t)rows * k, s);
  transpose2d<double, double>(Qf, Q.as<double>(), k, rows, s);
  R.ensure(sizeof(double) * (size_t)k * cols, s);
  transpose2d<double, double>(Lf, R.as<double>(), cols, k, s);
  return k;
}

void left_orthogonalize(a2_tt* tt, double* norm_out) {
  a2_ctx* c = tt->ctx;
  cudaStream_t s = c->stream;
  for (int j = 0; j + 1 < tt->L; ++j) {
    const int Dl = tt->dims[j], n = tt->phys[j], Dr = tt->dims[j + 1];
    const int rows = Dl * n;
    // core j = Q (rows x k);  core j+1 <- R core_{j+1}
    DevBuf nc, Rm;
    const int k = qr_split_dev(c, tt->cores[j].as<double>(), rows, Dr, nc, Rm);
    const int n2 = tt->phys[j + 1], Dr2 = tt->dims[j + 2];
    DevBuf nxt;
    nxt.ensure(sizeof(double) * (size_t)k * n2 * Dr2, s);
    matmul_dev(c, Rm.as<double>(), k, Dr, tt->cores[j + 1].as<double>(), n2 * Dr2,
               nxt.as<double>());
    tt->cores[j] = std::move(nc);
    tt->cores[j + 1] = std::move(nxt);
    tt->dims[j + 1] = k;
  }
  const int last = tt->L - 1;
  const long long nl = (long long)tt->dims[last] * tt->phys[last] * tt->dims[last + 1];
  double nrm2 = dot_dev(c, tt->cores[last].as<double>(), tt->cores[last].as<double>(), nl, 6);
  check_finite(nrm2, "TT norm");
  A2_REQUIRE(nrm2 > 0.0, "TT has zero norm");
  if (norm_out) *norm_out = std::sqrt(nrm2);
  scale_dev(tt->cores[last].as<double>(), nullptr, scal(c, 6), nl, s);
}

// ============================================================================= global iteration
template <typename T>
struct Sweeper {
  a2_ctx* c;
  a2_tt* tt;
  const a2_mpo* mpo;
  a2_sweep_opts o;
  Engine<T> eng;
  int L;
  std::vector<DevBuf> Vc, Cc;         // right-orth cores V_i, centres C_i
  std::vector<int> kd;                // bond dims of the right-orthogonal part
  std::vector<int> kry;
  std::atomic<int> unconv{0};   // local eigensolves stopped at max_restarts above eig_tol
  double max_disc = 0.0;

  Sweeper(a2_ctx* c_, a2_tt* t, const a2_mpo* m, const a2_sweep_opts& op)
      : c(c_), tt(t), mpo(m), o(op), eng(c_, m, op.prec), L(t->L) {}

  const T* hl(int j) { return eng.HL[j].template as<T>(); }
  const T* hr(int j) { return eng.HR[j].template as<T>(); }

  // Memory-limited environment mode (storage O(r^2 R) instead of O(d r^2 R), Sec. on
  // the cost of the micro-iterations): no environment is kept between uses; the left
  // environment of site j is rebuilt from the left end through U_0..U_{j-1}, the right
  // one from the right end through V_{L-1}..V_j, on the engine (stream) of the caller.
  // In the stored mode these return the environments built once by build_envs.
  bool lazy() const { return o.env_mode == 1; }
  const T* hl_at(int j, Engine<T>& e, DevBuf& buf) {
    if (!lazy()) return hl(j);
    cudaStream_t s = e.c->stream;
    DevBuf a, b;
    e.set_unit(a);
    for (int i = 0; i < j; ++i) {
      const int Dl = tt->dims[i], Dr = tt->dims[i + 1];
      b.ensure(sizeof(T) * (size_t)Dr * mpo->R[i + 1] * Dr, s);
      e.left_update(a.template as<T>(), i, tt->cores[i].as<double>(), Dl, Dr,
                    tt->cores[i].as<double>(), Dl, Dr, b.template as<T>());
      std::swap(a, b);
    }
    buf = std::move(a);
    return buf.template as<T>();
  }
  const T* hr_at(int j, Engine<T>& e, DevBuf& buf) {
    if (!lazy()) return hr(j);
    cudaStream_t s = e.c->stream;
    DevBuf a, b;
    e.set_unit(a);
    for (int i = L - 1; i >= j; --i) {
      const int Dl = kd[i], Dr = kd[i + 1];
      b.ensure(sizeof(T) * (size_t)Dl * mpo->R[i] * Dl, s);
      e.right_update(a.template as<T>(), i, Vc[i].as<double>(), Dl, Dr, Vc[i].as<double>(), Dl,
                     Dr, b.template as<T>());
      std::swap(a, b);
    }
    buf = std::move(a);
    return buf.template as<T>();
  }

  // Step 1 of Alg. 2: right-to-left LQ sweep, every i-orthogonal copy.
  void step1() {
    cudaStream_t s = c->stream;
    Vc.clear(); Vc.resize(L);
    Cc.clear(); Cc.resize(L);
    kd.assign(L + 1, 1);
    const size_t nlast = (size_t)tt->dims[L - 1] * tt->phys[L - 1];
    Cc[L - 1].ensure(sizeof(double) * nlast, s);
    A2_CUDA(cudaMemcpyAsync(Cc[L - 1].p, tt->cores[L - 1].p, sizeof(double) * nlast,
                            cudaMemcpyDeviceToDevice, s));
    kd[L] = 1;
    for (int i = L - 1; i >= 1; --i) {
      const int Dl = tt->dims[i], n = tt->phys[i], Dr = kd[i + 1];
      const int cols = n * Dr;
      const int k = std::min(Dl, cols);
      DevBuf Lf;
      Lf.ensure(sizeof(double) * (size_t)Dl * k, s);
      Vc[i].ensure(sizeof(double) * (size_t)k * cols, s);
      c->solver.lq(Cc[i].as<double>(), Dl, cols, Lf.as<double>(), Vc[i].as<double>(), s);
      kd[i] = k;
      const int Dl0 = tt->dims[i - 1], n0 = tt->phys[i - 1];
      Cc[i - 1].ensure(sizeof(double) * (size_t)Dl0 * n0 * k, s);
      matmul_dev(c, tt->cores[i - 1].as<double>(), Dl0 * n0, Dl, Lf.as<double>(), k,
                 Cc[i - 1].as<double>());
    }
    kd[0] = 1;
  }

  // Step 2 (first part): left envs from U, right envs from V.
  void build_envs() {
    cudaStream_t s = c->stream;
    if (lazy()) return;   // memory-limited mode: built on demand (hl_at / hr_at)
    eng.set_unit(eng.HL[0]);
    eng.HLd[0] = 1;
    for (int j = 0; j + 1 < L; ++j) {
      const int Dl = tt->dims[j], Dr = tt->dims[j + 1];
      eng.HL[j + 1].ensure(sizeof(T) * (size_t)Dr * mpo->R[j + 1] * Dr, s);
      eng.left_update(hl(j), j, tt->cores[j].as<double>(), Dl, Dr, tt->cores[j].as<double>(),
                      Dl, Dr, eng.HL[j + 1].template as<T>());
      eng.HLd[j + 1] = Dr;
    }
    eng.set_unit(eng.HR[L]);
    eng.HRd[L] = 1;
    for (int j = L - 1; j >= 1; --j) {
      const int Dl = kd[j], Dr = kd[j + 1];
      eng.HR[j].ensure(sizeof(T) * (size_t)Dl * mpo->R[j] * Dl, s);
      eng.right_update(hr(j + 1), j, Vc[j].as<double>(), Dl, Dr, Vc[j].as<double>(), Dl, Dr,
                       eng.HR[j].template as<T>());
      eng.HRd[j] = Dl;
    }
  }

  // the last cores of a further updated TT of a group (Extension One): they replace the
  // group's final cores mg+2-cores.size() .. mg+1
  struct Tail {
    std::vector<DevBuf> cores;
    std::vector<int> dl, dr;
    double theta = 0.0;
  };
  struct Group {
    int kg, mg;
    std::vector<DevBuf> cores;   // new cores kg..mg+1 (mg - kg + 2 of them)
    std::vector<int> dl, dr;     // their bond dims
    double theta = 0.0;
    double disc = 0.0;           // largest discarded weight of the group's SVD steps
    std::vector<Tail> extra;     // eigenvectors 2..K of the last local problem
  };

  // Step 2 (second part): the group's left-to-right two-site micro-steps, on the lane
  // context `c` (own stream and scratch) with its own engine; environments are shared.
  void solve_group(Group& G, a2_ctx* c, Engine<T>& eng) {
    cudaStream_t s = c->stream;
    DevBuf Hloc;
    int Dl = tt->dims[G.kg];
    // centre C_kg
    DevBuf centre;
    {
      const size_t nb = (size_t)Dl * tt->phys[G.kg] * kd[G.kg + 1];
      centre.ensure(sizeof(double) * nb, s);
      A2_CUDA(cudaMemcpyAsync(centre.p, Cc[G.kg].p, sizeof(double) * nb,
                              cudaMemcpyDeviceToDevice, s));
    }
    int cdim = kd[G.kg + 1];           // right bond of the centre
    DevBuf HLbuf, HRbuf;
    const T* HLcur = hl_at(G.kg, eng, HLbuf);
    for (int k = G.kg; k <= G.mg; ++k) {
      NvtxRange r_local("a2: local solve at bond", k);
      const int n1 = tt->phys[k], n2 = tt->phys[k + 1];
      const int Dr = kd[k + 2];
      const long long N = (long long)Dl * n1 * n2 * Dr;
      DevBuf x;
      x.ensure(sizeof(double) * N, s);
      matmul_dev(c, centre.as<double>(), Dl * n1, cdim, Vc[k + 1].as<double>(), n2 * Dr,
                 x.as<double>());
      const T* HRk = hr_at(k + 2, eng, HRbuf);
      if constexpr (sizeof(T) == 8) {   // FP64 emulation: slice the environments once
        if (o.prec == A2_F64EMU)
          eng.oze.set(c, HLcur, Dl, mpo->R[k], HRk, Dr, mpo->R[k + 2]);
      }
      auto mv_raw = [&](const double* in, double* out) {
        if constexpr (sizeof(T) == 8) {
          if (o.prec == A2_F64EMU) {
            eng.matvec_f64e(k, Dl, Dr, in, out);
            return;
          }
        }
        eng.matvec(k, HLcur, HRk, Dl, Dr, in, out);
      };
      // with o.graphs, every operator of this local problem is replayed from a CUDA graph
      GraphedMV g_mv(c, N), g_b(c, N), g_e(c, N);
      auto graphed = [&](GraphedMV& g, auto& f) {
        return [&g, &f, &eng, this](const double* in, double* out) {
          if (o.graphs) g(f, eng, in, out);
          else f(in, out);
        };
      };
      auto mv = graphed(g_mv, mv_raw);
      const bool ext = o.n_eig > 1 && k == G.mg;
      DevBuf xstart;   // Extension One: start vector of the further eigenvectors
      if (ext) {
        xstart.ensure(sizeof(double) * N, s);
        A2_CUDA(cudaMemcpyAsync(xstart.p, x.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      }
      int nmv = 0;
      LanczosResult lr;
      bool done = false;
      const bool mixed = o.prec == A2_BF16 || o.prec == A2_F32EMU;
      if (o.solver == 1) {
        // Davidson with the diagonal preconditioner on the accurate operator
        DevBuf dg;
        dg.ensure(sizeof(double) * (size_t)N, c->stream);
        heff_diag<T>(c, mpo->site[k], mpo->site[k + 1], HLcur, HRk, Dl, Dr, dg.as<double>());
        if (mixed) {
          eng.bfe.set(c, HLcur, Dl, mpo->R[k], HRk, Dr, mpo->R[k + 2], 3, &mpo->site[k],
                       &mpo->site[k + 1]);
          auto mve_raw = [&](const double* in, double* out) {
            eng.matvec_emu(k, Dl, Dr, in, out);
          };
          auto mve = graphed(g_e, mve_raw);
          lr = davidson(c, mve, dg.as<double>(), x.as<double>(), N, o.eig_tol, o.max_krylov,
                        o.max_krylov * o.max_restarts);
          done = true;
        }
        if (!done)
          lr = davidson(c, mv, dg.as<double>(), x.as<double>(), N, o.eig_tol, o.max_krylov,
                        o.max_krylov * o.max_restarts);
        done = true;
      }
      {
        if (!done && mixed) {
          eng.bfe.set(c, HLcur, Dl, mpo->R[k], HRk, Dr, mpo->R[k + 2], 3, &mpo->site[k],
                         &mpo->site[k + 1]);
          if (o.prec == A2_BF16) {
            // tensor-core Lanczos on the BF16 operator to a loose tolerance ...
            auto mvb_raw = [&](const double* in, double* out) {
              eng.matvec_bf16(k, Dl, Dr, in, out);
            };
            auto mvb = graphed(g_b, mvb_raw);
            LanczosResult lb = lanczos(c, mvb, x.as<double>(), N, std::max(o.eig_tol, kBf16Tol),
                                       o.max_krylov, o.max_restarts);
            nmv += lb.matvecs;
          }
          // ... then FP32-accurate tensor-core products from that vector to eig_tol (or
          // to kSplitTol when the FP64 refinement takes it further)
          auto mve_raw = [&](const double* in, double* out) {
            eng.matvec_emu(k, Dl, Dr, in, out);
          };
          auto mve = graphed(g_e, mve_raw);
          const double tol_split =
              (sizeof(T) == 8 && o.refine_f64) ? std::max(o.eig_tol, kSplitTol) : o.eig_tol;
          lr = lanczos(c, mve, x.as<double>(), N, tol_split, o.max_krylov, o.max_restarts);
          done = true;
        }
      }
      if (!done)
        lr = lanczos(c, mv, x.as<double>(), N, o.eig_tol, o.max_krylov, o.max_restarts);
      if constexpr (sizeof(T) == 8) {
        if (mixed && o.refine_f64) {
          // FP64 refinement of the Ritz pair: Lanczos continued from x on the FP64-class
          // (Ozaki-emulated) operator.  Its first application gives the FP64 Rayleigh
          // quotient and the FP64 residual; it stops as soon as that residual meets
          // eig_tol, so an x the tensor-core phases left accurate enough costs one
          // application.
          nmv += lr.matvecs;
          eng.oze.set(c, HLcur, Dl, mpo->R[k], HRk, Dr, mpo->R[k + 2]);
          auto mvf = [&](const double* in, double* out) { eng.matvec_f64e(k, Dl, Dr, in, out); };
          lr = lanczos(c, mvf, x.as<double>(), N, o.eig_tol, o.max_krylov, o.max_restarts);
        }
      }
      check_finite(lr.theta, "local eigenvalue");
      kry[k] = nmv + lr.matvecs;
      if (!lr.converged) unconv.fetch_add(1);
      G.theta = lr.theta;
      const int rows = Dl * n1, cols = n2 * Dr;
      if (ext) {
        // the further eigenvectors on the accurate operator (FP32-accurate tensor-core
        // products in the mixed modes), each truncated by its own SVD
        auto mvx = [&](const double* in, double* out) {
          if (mixed) {
            eng.matvec_emu(k, Dl, Dr, in, out);
            return;
          }
          mv(in, out);
        };
        DevBuf Qx;
        int nx = 0;
        std::vector<double> th = deflated_eigs(c, mvx, xstart.as<double>(), x.as<double>(), N,
                                               o.n_eig, o.eig_tol, o.max_krylov, o.max_restarts,
                                               Qx, &nx, &unconv);
        kry[k] += nx;
        for (size_t e = 0; e < th.size(); ++e) {
          Tail t;
          t.theta = th[e];
          DevBuf Pe, SQe;
          Pe.ensure(sizeof(double) * (size_t)rows * std::min(rows, cols), s);
          SQe.ensure(sizeof(double) * (size_t)std::min(rows, cols) * cols, s);
          double de = 0.0;
          int re = 0;
          {
            HiScope hs(c);
            re = svd_split_dev(c, Qx.as<double>() + (size_t)(e + 1) * N, rows, cols, o.D_max,
                               o.svd_tol, Pe.as<double>(), SQe.as<double>(), &de);
          }
          G.disc = std::max(G.disc, de);
          t.cores.push_back(std::move(Pe));
          t.dl.push_back(Dl);
          t.dr.push_back(re);
          t.cores.push_back(std::move(SQe));
          t.dl.push_back(re);
          t.dr.push_back(Dr);
          G.extra.push_back(std::move(t));
        }
      }
      const int kmax = std::min(rows, cols);
      DevBuf P, SQ;
      P.ensure(sizeof(double) * (size_t)rows * kmax, s);
      SQ.ensure(sizeof(double) * (size_t)kmax * cols, s);
      double disc = 0.0;
      int r = 0;
      {
        HiScope hs(c);
        r = svd_split_dev(c, x.as<double>(), rows, cols, o.D_max, o.svd_tol, P.as<double>(),
                          SQ.as<double>(), &disc);
      }
      G.disc = std::max(G.disc, disc);
      // group-local left environment with the new left-orthogonal core
      DevBuf Hn;
      Hn.ensure(sizeof(T) * (size_t)r * mpo->R[k + 1] * r, s);
      eng.left_update(HLcur, k, P.as<double>(), Dl, r, P.as<double>(), Dl, r, Hn.template as<T>());
      Hloc = std::move(Hn);
      HLcur = Hloc.template as<T>();
      G.cores.push_back(std::move(P));
      G.dl.push_back(Dl);
      G.dr.push_back(r);
      centre = std::move(SQ);
      cdim = Dr;
      Dl = r;
    }
    G.cores.push_back(std::move(centre));
    G.dl.push_back(Dl);
    G.dr.push_back(kd[G.mg + 2]);
  }

  // per-site view of basis element j (0 = iterate, in its kg-orthogonal form for `form_k`)
  View base_view(int form_k) {
    View v;
    v.core.resize(L); v.Dl.resize(L); v.Dr.resize(L);
    for (int j = 0; j < L; ++j) {
      if (j < form_k) {
        v.core[j] = tt->cores[j].as<double>(); v.Dl[j] = tt->dims[j]; v.Dr[j] = tt->dims[j + 1];
      } else if (j == form_k) {
        v.core[j] = Cc[j].as<double>(); v.Dl[j] = tt->dims[j]; v.Dr[j] = kd[j + 1];
      } else {
        v.core[j] = Vc[j].as<double>(); v.Dl[j] = kd[j]; v.Dr[j] = kd[j + 1];
      }
    }
    return v;
  }
  // Step 2, one-site case: the group's cores first..last (G.kg .. G.mg + 1) in order; each
  // local problem is the one-site H_eff of the current orthogonal TT, warm-started from its
  // centre core; between the cores of the group the new core is orthogonalised (thin QR,
  // ranks unchanged) and the triangular factor moves into the next core, with the
  // group-local left environment updated (Alg. 1, one-site, step 2).
  void solve_group1(Group& G, a2_ctx* c, Engine<T>& eng) {
    cudaStream_t s = c->stream;
    const int first = G.kg, last = G.mg + 1;
    DevBuf Hloc, centre;
    int Dl = tt->dims[first];
    {
      const size_t nb = (size_t)Dl * tt->phys[first] * kd[first + 1];
      centre.ensure(sizeof(double) * nb, s);
      A2_CUDA(cudaMemcpyAsync(centre.p, Cc[first].p, sizeof(double) * nb,
                              cudaMemcpyDeviceToDevice, s));
    }
    DevBuf HLbuf, HRbuf;
    const T* HLcur = hl_at(first, eng, HLbuf);
    for (int j = first; j <= last; ++j) {
      NvtxRange r_local("a2: one-site local solve at core", j);
      const int n = tt->phys[j], Dr = kd[j + 1];
      const long long N = (long long)Dl * n * Dr;
      const T* HRj = hr_at(j + 1, eng, HRbuf);
      // mixed modes: FP32-accurate tensor-core products (environments split once)
      bool tc1 = false;
      if (o.prec == A2_BF16 || o.prec == A2_F32EMU) {
        eng.bfe.set(c, HLcur, Dl, mpo->R[j], HRj, Dr, mpo->R[j + 1], 3);
        tc1 = true;
      }
      auto mv_raw = [&](const double* in, double* out) {
        if (tc1) eng.matvec1_emu(j, Dl, Dr, in, out);
        else eng.matvec1(j, HLcur, HRj, Dl, Dr, in, out);
      };
      GraphedMV g_mv(c, N);   // with o.graphs, replayed from a CUDA graph
      auto mv = [&](const double* in, double* out) {
        if (o.graphs) g_mv(mv_raw, eng, in, out);
        else mv_raw(in, out);
      };
      const bool ext = o.n_eig > 1 && j == last;
      DevBuf xstart;
      if (ext) {
        xstart.ensure(sizeof(double) * N, s);
        A2_CUDA(cudaMemcpyAsync(xstart.p, centre.p, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                s));
      }
      LanczosResult lr = lanczos(c, mv, centre.as<double>(), N, o.eig_tol, o.max_krylov,
                                 o.max_restarts);
      check_finite(lr.theta, "local eigenvalue");
      kry[j] = lr.matvecs;
      if (!lr.converged) unconv.fetch_add(1);
      G.theta = lr.theta;
      if (ext) {   // Extension One: each further eigenvector replaces the last core
        DevBuf Qx;
        int nx = 0;
        std::vector<double> th = deflated_eigs(c, mv, xstart.as<double>(), centre.as<double>(),
                                               N, o.n_eig, o.eig_tol, o.max_krylov,
                                               o.max_restarts, Qx, &nx, &unconv);
        kry[j] += nx;
        for (size_t e = 0; e < th.size(); ++e) {
          Tail t;
          t.theta = th[e];
          DevBuf xe;
          xe.ensure(sizeof(double) * N, s);
          A2_CUDA(cudaMemcpyAsync(xe.p, Qx.as<double>() + (size_t)(e + 1) * N,
                                  sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
          t.cores.push_back(std::move(xe));
          t.dl.push_back(Dl);
          t.dr.push_back(Dr);
          G.extra.push_back(std::move(t));
        }
      }
      if (j == last) {
        G.cores.push_back(std::move(centre));
        G.dl.push_back(Dl);
        G.dr.push_back(Dr);
        break;
      }
      DevBuf P, SQ;   // x = P SQ: P left-orthonormal, SQ moves into the next core
      const int r = qr_split_dev(c, centre.as<double>(), Dl * n, Dr, P, SQ);
      DevBuf Hn;
      Hn.ensure(sizeof(T) * (size_t)r * mpo->R[j + 1] * r, s);
      eng.left_update(HLcur, j, P.as<double>(), Dl, r, P.as<double>(), Dl, r, Hn.template as<T>());
      Hloc = std::move(Hn);
      HLcur = Hloc.template as<T>();
      G.cores.push_back(std::move(P));
      G.dl.push_back(Dl);
      G.dr.push_back(r);
      // next centre: (S Q) V_{j+1}
      const int n2 = tt->phys[j + 1], Dr2 = kd[j + 2];
      DevBuf next;
      next.ensure(sizeof(double) * (size_t)r * n2 * Dr2, s);
      matmul_dev(c, SQ.as<double>(), r, Dr, Vc[j + 1].as<double>(), n2 * Dr2, next.as<double>());
      centre = std::move(next);
      Dl = r;
    }
  }

  // updated TT e of group G (0: the lowest eigenvector; e >= 1: Extension One's tails)
  View group_view(const Group& G, int e = 0) {
    View v;
    v.core.resize(L); v.Dl.resize(L); v.Dr.resize(L);
    for (int j = 0; j < L; ++j) {
      if (j < G.kg) {
        v.core[j] = tt->cores[j].as<double>(); v.Dl[j] = tt->dims[j]; v.Dr[j] = tt->dims[j + 1];
      } else if (j <= G.mg + 1) {
        const int q = j - G.kg;
        v.core[j] = G.cores[q].template as<double>(); v.Dl[j] = G.dl[q]; v.Dr[j] = G.dr[q];
      } else {
        v.core[j] = Vc[j].as<double>(); v.Dl[j] = kd[j]; v.Dr[j] = kd[j + 1];
      }
    }
    if (e > 0) {
      const Tail& t = G.extra[e - 1];
      const int first = G.mg + 2 - (int)t.cores.size();
      for (size_t q = 0; q < t.cores.size(); ++q) {
        v.core[first + q] = t.cores[q].template as<double>();
        v.Dl[first + q] = t.dl[q];
        v.Dr[first + q] = t.dr[q];
      }
    }
    return v;
  }

  // <bra, ket> over sites lo..hi with identity outside (shared orthogonal prefix/suffix)
  double overlap_span(const View& bra, const View& ket, int lo, int hi) {
    cudaStream_t s = c->stream;
    A2_REQUIRE(bra.Dl[lo] == ket.Dl[lo], "overlap: mismatched left bond");
    const int D0 = bra.Dl[lo];
    DevBuf E, En, Tm;
    E.ensure(sizeof(double) * (size_t)D0 * D0, s);
    {
      std::vector<double> I((size_t)D0 * D0, 0.0);
      for (int i = 0; i < D0; ++i) I[(size_t)i * D0 + i] = 1.0;
      A2_CUDA(cudaMemcpyAsync(E.p, I.data(), sizeof(double) * I.size(), cudaMemcpyHostToDevice, s));
      A2_CUDA(cudaStreamSynchronize(s));
    }
    for (int j = lo; j <= hi; ++j) {
      const int n = tt->phys[j];
      const int bl = bra.Dl[j], br = bra.Dr[j], kl = ket.Dl[j], kr = ket.Dr[j];
      Tm.ensure(sizeof(double) * (size_t)bl * n * kr, s);
      matmul_dev(c, E.as<double>(), bl, kl, ket.core[j], n * kr, Tm.as<double>());  // [a][(s b')]
      En.ensure(sizeof(double) * (size_t)br * kr, s);
      // En[b][b'] = sum_{(a s)} bra[(a s)][b] Tm[(a s)][b']
      gemm_f64(c, br, kr, bl * n, bra.core[j], 1, br, Tm.as<double>(), 1, kr, En.as<double>(), kr);
      std::swap(E, En);
    }
    const int Df = bra.Dr[hi];
    A2_REQUIRE(Df == ket.Dr[hi], "overlap: mismatched right bond");
    // trace(E)
    std::vector<double> h((size_t)Df * Df);
    A2_CUDA(cudaMemcpyAsync(h.data(), E.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaStreamSynchronize(s));
    double tr = 0.0;
    for (int i = 0; i < Df; ++i) tr += h[(size_t)i * Df + i];
    return tr;
  }

  // <bra, A ket> over sites lo..hi, closed by the iterate's envs HL[lo] and HR[hi+1]
  double sandwich_span(const View& bra, const View& ket, int lo, int hi) {
    DevBuf Hb;
    return sandwich_from(hl_at(lo, eng, Hb), lo, bra, ket, hi);
  }
  // Mixed left environment E of (bra, ket) at site p (sites before p contracted) advanced
  // to site q: the left updates of sites p..q-1 (E is replaced).
  void advance_left(DevBuf& E, int p, int q, const View& bra, const View& ket) {
    cudaStream_t s = c->stream;
    DevBuf En;
    for (int j = p; j < q; ++j) {
      En.ensure(sizeof(T) * (size_t)bra.Dr[j] * mpo->R[j + 1] * ket.Dr[j], s);
      eng.left_update(E.template as<T>(), j, bra.core[j], bra.Dl[j], bra.Dr[j], ket.core[j],
                      ket.Dl[j], ket.Dr[j], En.template as<T>());
      std::swap(E, En);
    }
  }
  // <bra, A ket> from the mixed left environment E0 at site p (not modified) over sites
  // p..hi, closed by the iterate's HR[hi+1]
  double sandwich_from(const T* E0, int p, const View& bra, const View& ket, int hi) {
    cudaStream_t s = c->stream;
    DevBuf E, En;
    const T* Ecur = E0;
    for (int j = p; j <= hi; ++j) {
      En.ensure(sizeof(T) * (size_t)bra.Dr[j] * mpo->R[j + 1] * ket.Dr[j], s);
      eng.left_update(Ecur, j, bra.core[j], bra.Dl[j], bra.Dr[j], ket.core[j], ket.Dl[j],
                      ket.Dr[j], En.template as<T>());
      std::swap(E, En);
      Ecur = E.template as<T>();
    }
    const long long ne = (long long)bra.Dr[hi] * mpo->R[hi + 1] * ket.Dr[hi];
    A2_REQUIRE(kd[hi + 1] == bra.Dr[hi] && kd[hi + 1] == ket.Dr[hi], "sandwich: right env dims");
    DevBuf Rb;
    const T* Rcur = hr_at(hi + 1, eng, Rb);
    // full contraction <E, HR[hi+1]> in FP64
    c->xa.ensure(sizeof(double) * ne * 2, s);
    double* e64 = c->xa.as<double>();
    double* r64 = e64 + ne;
    if constexpr (sizeof(T) == 8) {
      A2_CUDA(cudaMemcpyAsync(e64, Ecur, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
      A2_CUDA(cudaMemcpyAsync(r64, Rcur, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
    } else {
      convert<float, double>(Ecur, e64, ne, s);
      convert<float, double>(Rcur, r64, ne, s);
    }
    return dot_dev(c, e64, r64, ne, 7);
  }

  // Device bytes one group lane needs at its largest local problem (bond dims capped by
  // D_max): the H_eff intermediates of the tensor-core chain (or of the SIMT chain), the
  // converted environments, the Lanczos basis and the environment-update scratch.
  double lane_bytes() const {
    // exact-rank caps of the bond dims: prod of the physical dims on either side
    std::vector<double> lcap(L + 1, 1.0), rcap(L + 1, 1.0);
    for (int j = 0; j < L; ++j) lcap[j + 1] = std::min<double>(o.D_max, lcap[j] * tt->phys[j]);
    for (int j = L - 1; j >= 0; --j) rcap[j] = std::min<double>(o.D_max, rcap[j + 1] * tt->phys[j]);
    double worst = 0.0;
    const double m = std::min(o.max_krylov, 63) + 3;
    const double es = sizeof(T);
    for (int k = 0; k + 1 < L; ++k) {
      const double n1 = tt->phys[k], n2 = tt->phys[k + 1];
      const double Dl = lcap[k], Dr = rcap[k + 2];
      const double Rl = mpo->R[k], R1 = mpo->R[k + 1], Rr = mpo->R[k + 2];
      const double N = Dl * n1 * n2 * Dr;
      double heff;
      if (o.prec == A2_BF16 || o.prec == A2_F32EMU)  // tensor-core chains (split planes)
        heff = std::max(4.0 * Dl * Rl, 6.0 * Dl * Rr) * n1 * n2 * Dr + 6.0 * Dl * R1 * n1 * n2 * Dr +
               12.0 * (Dl * Rl * Dl + Dr * Rr * Dr + 2.0 * Dl * R1 * Dl);
      else                                           // SIMT chain: t1 = max(T1, T3), t2 = T2
        heff = es * (std::max(Rl, Rr) + R1) * Dl * n1 * n2 * Dr;
      const double env = 2.0 * es * Dl * std::max(Rl, Rr) * n1 * Dr;
      worst = std::max(worst, heff + env + 8.0 * m * N + 16.0 * N);
    }
    return worst;
  }

  // Number of group lanes that fit in the free device memory next to what is resident.
  int concurrent_lanes(int P) const {
    size_t free_b = 0, total_b = 0;
    A2_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double need = std::max(1.0, lane_bytes());
    const int fit = (int)std::floor(0.8 * (double)free_b / need);
    return std::max(1, std::min(P, fit));
  }

  void run(a2_sweep_report* rep, bool classical) {
    cudaStream_t s = c->stream;
    auto t0 = std::chrono::steady_clock::now();
    tt_check(tt);
    A2_REQUIRE(tt->phys == mpo->phys, "TT and MPO physical dims differ");
    A2_REQUIRE(o.n_eig >= 0 && o.n_eig <= 64, "n_eig must be in 0..64");
    A2_REQUIRE(o.env_mode == 0 || o.env_mode == 1, "env_mode must be 0 or 1");
    A2_REQUIRE(!(classical && o.n_eig > 1), "n_eig > 1 (Extension One) needs the coarse step");
    std::vector<int> sizes;
    const bool one = o.one_site != 0;
    const int units = one ? L : L - 1;               // cores (one-site) or bonds (two-site)
    int P = classical ? 1 : o.P;
    A2_REQUIRE(P >= 1 && P <= units, "P must be in 1..L-1 (1..L one-site)");
    if (!classical && o.bond_partition) {
      sizes.assign(o.bond_partition, o.bond_partition + P);
    } else {
      for (int g = 0; g < P; ++g) sizes.push_back(units / P + (g < units % P ? 1 : 0));
    }
    A2_REQUIRE(std::accumulate(sizes.begin(), sizes.end(), 0) == units,
               one ? "core partition must sum to L" : "bond partition must sum to L-1");
    for (int x : sizes) A2_REQUIRE(x >= 1, "empty group");
    A2_REQUIRE(o.D_max >= 1, "D_max >= 1");
    A2_REQUIRE(o.max_krylov >= 2 && o.max_krylov <= 63, "max_krylov in 2..63");
    kry.assign(units, 0);
    unconv.store(0);
    {
      NvtxRange r("a2: step 1 (LQ sweep)");
      step1();
    }
    {
      NvtxRange r("a2: environments");
      build_envs();
    }
    // groups as blocks of modified cores [kg, mg + 1]: two-site, bonds kg..mg; one-site,
    // cores kg..mg + 1
    std::vector<Group> groups(P);
    int k0 = 0;
    for (int g = 0; g < P; ++g) {
      groups[g].kg = k0;
      groups[g].mg = k0 + sizes[g] - 1 - (one ? 1 : 0);
      k0 += sizes[g];
    }
    auto solve = [&](Group& G, a2_ctx* lc, Engine<T>& e) {
      NvtxRange r("a2: group from site", G.kg);
      if (one) solve_group1(G, lc, e);
      else solve_group(G, lc, e);
    };
    const int nl = (P > 1 && o.group_streams != 1) ? concurrent_lanes(P) : 1;
    if (nl > 1) {
      // the groups are independent (Alg. 2 step 2): nl host threads, each with its own
      // stream, scratch and solver, take the groups one after another
      A2_CUDA(cudaStreamSynchronize(s));                 // environments are ready
      std::vector<std::unique_ptr<Engine<T>>> engs;
      for (int i = 0; i < nl; ++i) engs.emplace_back(new Engine<T>(lane(c, i), mpo, o.prec));
      std::vector<std::exception_ptr> errs(nl);
      std::atomic<int> next{0};
      std::vector<std::thread> th;
      for (int i = 0; i < nl; ++i)
        th.emplace_back([&, i] {
          try {
            A2_CUDA(cudaSetDevice(c->device));
            a2_ctx* lc = lane(c, i);
            for (int g = next.fetch_add(1); g < P; g = next.fetch_add(1))
              solve(groups[g], lc, *engs[i]);
            A2_CUDA(cudaStreamSynchronize(lc->stream));
          } catch (...) {
            errs[i] = std::current_exception();
            next.store(P);                         // the other lanes stop at their next group
          }
        });
      for (auto& t : th) t.join();
      for (auto& e : errs)
        if (e) std::rethrow_exception(e);
      for (auto& e : engs) {
        eng.flops += e->flops;
        eng.matvecs += e->matvecs;
        eng.matvecs_bf16 += e->matvecs_bf16;
        eng.matvecs_f64 += e->matvecs_f64;
      }
    } else {
      for (int g = 0; g < P; ++g) solve(groups[g], c, eng);
    }
    for (auto& G : groups) max_disc = std::max(max_disc, G.disc);
    // coarse basis: the iterate, then every group's updated TTs (Extension One: the
    // further eigenvectors follow the lowest one of their group)
    struct Item { int g, e; };
    std::vector<Item> items;
    for (int g = 0; g < P; ++g)
      for (int e = 0; e <= (int)groups[g].extra.size(); ++e) items.push_back({g, e});
    const int m = (int)items.size() + 1;
    A2_REQUIRE(m <= 63, "coarse dimension (P * n_eig + 1) above 63");
    std::vector<double> S((size_t)m * m, 0.0), A((size_t)m * m, 0.0);
    NvtxRange r_coarse("a2: coarse problem and compression");
    // iterate: its (L-1)-orthogonal form is the stored left-orthogonal TT
    {
      View b = base_view(L - 1);
      S[0] = overlap_span(b, b, L - 1, L - 1);
      A[0] = sandwich_span(b, b, L - 1, L - 1);
    }
    std::vector<View> gv(m - 1);
    for (int a = 0; a + 1 < m; ++a) gv[a] = group_view(groups[items[a].g], items[a].e);
    for (int a = 0; a + 1 < m; ++a) {
      const Group& Ga = groups[items[a].g];
      const int lo = Ga.kg, hi = Ga.mg + 1;
      View b = base_view(lo);
      S[(size_t)(a + 1)] = S[(size_t)(a + 1) * m] = overlap_span(b, gv[a], lo, hi);
      A[(size_t)(a + 1)] = A[(size_t)(a + 1) * m] = sandwich_span(b, gv[a], lo, hi);
      S[(size_t)(a + 1) * m + a + 1] = overlap_span(gv[a], gv[a], lo, hi);
      A[(size_t)(a + 1) * m + a + 1] = sandwich_span(gv[a], gv[a], lo, hi);
      // cross entries with the later items: left of item b2's first site its TT is the
      // iterate's left-orthogonal cores, so the mixed left environment of (gv[a], iterate)
      // from lo up to that site is shared by all b2 and advanced once
      DevBuf Pre;
      int pre_at = lo;
      {
        DevBuf Hb;
        const T* h0 = hl_at(lo, eng, Hb);
        const size_t nb0 = sizeof(T) * (size_t)gv[a].Dl[lo] * mpo->R[lo] * gv[a].Dl[lo];
        Pre.ensure(nb0, c->stream);
        A2_CUDA(cudaMemcpyAsync(Pre.p, h0, nb0, cudaMemcpyDeviceToDevice, c->stream));
      }
      for (int b2 = a + 1; b2 + 1 < m; ++b2) {
        const int lo2 = groups[items[b2].g].kg, hi2 = groups[items[b2].g].mg + 1;
        const double sv = overlap_span(gv[a], gv[b2], lo, hi2);
        if (lo2 > pre_at) {
          advance_left(Pre, pre_at, lo2, gv[a], gv[b2]);
          pre_at = lo2;
        }
        const double av = sandwich_from(Pre.template as<T>(), pre_at, gv[a], gv[b2], hi2);
        S[(size_t)(a + 1) * m + b2 + 1] = S[(size_t)(b2 + 1) * m + a + 1] = sv;
        A[(size_t)(a + 1) * m + b2 + 1] = A[(size_t)(b2 + 1) * m + a + 1] = av;
      }
    }
    for (double v : S) check_finite(v, "S_hat");
    for (double v : A) check_finite(v, "A_hat");
    std::vector<double> cvec(m, 0.0);
    double lam = 0.0;
    int prank = 0;
    if (classical) {   // Alg. 1: the half-sweep result is the new iterate
      cvec[1] = 1.0 / std::sqrt(S[(size_t)1 * m + 1]);
      lam = A[(size_t)1 * m + 1] / S[(size_t)1 * m + 1];
      prank = 1;
    } else {
      double* dA = scal(c, 9000);
      double* dS = dA + m * m;
      double* dc = dS + m * m;
      double* dl = dc + m;
      int* drk = reinterpret_cast<int*>(dl + 1);
      A2_CUDA(cudaMemcpyAsync(dA, A.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, s));
      A2_CUDA(cudaMemcpyAsync(dS, S.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, s));
      coarse_solve_dev(dA, dS, m, o.coarse_eps, dc, dl, drk, drk + 1, s);
      A2_CUDA(cudaMemcpyAsync(cvec.data(), dc, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
      int rk[2];
      A2_CUDA(cudaMemcpyAsync(&lam, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
      A2_CUDA(cudaMemcpyAsync(rk, drk, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
      A2_CUDA(cudaStreamSynchronize(s));
      prank = rk[0];
      if (rk[1] != 0) throw NumericError("coarse Jacobi did not converge");
    }
    check_finite(lam, "coarse eigenvalue");
    // Step 4: compression of sum_j c_j tau(U~^j) from its three-channel TT form
    {
      NvtxRange r("a2: compression");
      std::vector<DevBuf> X;
      std::vector<int> xd;
      if (m == P + 1) {
        structured_sum(groups, cvec, X, xd);
      } else {   // Extension One: block-diagonal sum of all m terms
        std::vector<View> terms(1, base_view(L - 1));
        terms.insert(terms.end(), gv.begin(), gv.end());
        plain_sum(terms, cvec, X, xd);
      }
      round_into_tt(X, xd);
    }
    // round_into_tt ended with a stream synchronisation: the error word is current
    if (factor_error_flag(true)) throw CudaError("a factorisation kernel's bounded wait gave up");
    if (rep) {
      rep->energy_in = A[0] / S[0];
      rep->lambda_coarse = lam;
      rep->coarse_rank = prank;
      if (rep->energy_local)
        for (int a = 0; a + 1 < m; ++a) {
          const Group& Ga = groups[items[a].g];
          rep->energy_local[a] = items[a].e == 0 ? Ga.theta : Ga.extra[items[a].e - 1].theta;
        }
      rep->coarse_dim = m;
      if (rep->coeffs) std::copy(cvec.begin(), cvec.end(), rep->coeffs);
      if (rep->S_hat) std::copy(S.begin(), S.end(), rep->S_hat);
      if (rep->A_hat) std::copy(A.begin(), A.end(), rep->A_hat);
      if (rep->krylov_iters) std::copy(kry.begin(), kry.end(), rep->krylov_iters);
      rep->max_discarded_weight = max_disc;
      rep->alg_flops = eng.flops;
      rep->matvecs = eng.matvecs;
      rep->matvecs_f64 = eng.matvecs_f64;
      rep->unconverged = unconv.load();
      A2_CUDA(cudaStreamSynchronize(s));
      rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  }

  // Three-channel TT of sum_j c_j tau(U~^j) (j = 0: the iterate).  At bond l the
  // channels are: P, the left-orthogonal prefix U_0..U_{l-1} shared by the iterate and
  // by every group that has not started; A, the single group whose block contains
  // bond l (its new cores, weighted by c_g when the channel opens); S, the
  // right-orthogonal suffix V_l..V_{L-1} shared by every group whose block has ended.
  // Each core is block upper-triangular in (P, A, S); bond <= D_P + D_A + D_S.
  void structured_sum(const std::vector<Group>& groups, const std::vector<double>& cvec,
                      std::vector<DevBuf>& X, std::vector<int>& xd) {
    cudaStream_t s = c->stream;
    const int P = (int)groups.size();
    std::vector<int> act(L + 1, -1);   // active group at bond l
    for (int g = 0; g < P; ++g)
      for (int l = groups[g].kg + 1; l <= groups[g].mg + 1; ++l) act[l] = g;
    std::vector<int> dP(L + 1, 0), dA(L + 1, 0), dS(L + 1, 0);
    xd.assign(L + 1, 1);
    for (int l = 1; l < L; ++l) {
      // two-site blocks cover every bond; one-site blocks leave the bonds between groups
      // without an active channel
      dP[l] = tt->dims[l];
      dA[l] = act[l] >= 0 ? groups[act[l]].dl[l - groups[act[l]].kg] : 0;
      dS[l] = (l > groups[0].mg + 1) ? kd[l] : 0;
      xd[l] = dP[l] + dA[l] + dS[l];
    }
    X.clear();
    X.resize(L);
    for (int j = 0; j < L; ++j) {
      const int n = tt->phys[j];
      const int Dl = xd[j], Dr = xd[j + 1];
      X[j].ensure(sizeof(double) * (size_t)Dl * n * Dr, s);
      fill_zero(X[j].p, sizeof(double) * (size_t)Dl * n * Dr, s);
      double* dst = X[j].as<double>();
      const long long s0 = (long long)n * Dr, s1 = Dr;
      const bool last = (j == L - 1);
      // rows: P at 0, A at dP[j], S at dP[j] + dA[j]   (bond 0: P only)
      const int rP = 0, rA = (j > 0) ? dP[j] : 0, rS = (j > 0) ? dP[j] + dA[j] : 0;
      const int cP = 0, cA = last ? 0 : dP[j + 1], cS = last ? 0 : dP[j + 1] + dA[j + 1];
      // P -> P (or P -> end for the iterate, weighted by c_0)
      copy_block3(tt->cores[j].as<double>(), tt->dims[j], n, tt->dims[j + 1], dst, s0, s1, rP,
                  cP, last ? cvec[0] : 1.0, s);
      // P -> A: a group opens at site j (P -> S for a one-core group)
      for (int g = 0; g < P; ++g)
        if (groups[g].kg == j) {
          const Group& G = groups[g];
          const int col = (G.mg + 1 == j && !last) ? cS : cA;
          // at the last site this block shares rows and column with P -> end
          copy_block3(G.cores[0].template as<double>(), G.dl[0], n, G.dr[0], dst, s0, s1, rP, col,
                      cvec[g + 1], s, last);
        }
      // A -> A / A -> S / A -> end
      if (j > 0 && act[j] >= 0) {
        const Group& G = groups[act[j]];
        const int q = j - G.kg;
        const bool closes = (j == G.mg + 1);
        const int col = last ? 0 : (closes ? cS : cA);
        copy_block3(G.cores[q].template as<double>(), G.dl[q], n, G.dr[q], dst, s0, s1, rA, col,
                    1.0, s);
      }
      // S -> S / S -> end
      if (j > 0 && dS[j] > 0)
        copy_block3(Vc[j].as<double>(), kd[j], n, kd[j + 1], dst, s0, s1, rS, last ? 0 : cS, 1.0,
                    s);
    }
  }

  // TT-sum (block-diagonal cores) of the given views, for callers with explicit terms.
  void plain_sum(const std::vector<View>& terms, const std::vector<double>& coef,
                 std::vector<DevBuf>& X, std::vector<int>& xd) {
    cudaStream_t s = c->stream;
    const int nt = (int)terms.size();
    X.clear();
    X.resize(L);
    xd.assign(L + 1, 0);
    xd[0] = 1;
    xd[L] = 1;
    for (int j = 1; j < L; ++j) {
      int d = 0;
      for (auto& t : terms) d += t.Dl[j];
      xd[j] = d;
    }
    for (int j = 0; j < L; ++j) {
      const int n = tt->phys[j];
      X[j].ensure(sizeof(double) * (size_t)xd[j] * n * xd[j + 1], s);
      fill_zero(X[j].p, sizeof(double) * (size_t)xd[j] * n * xd[j + 1], s);
      int o0 = 0, o2 = 0;
      for (int q = 0; q < nt; ++q) {
        const View& t = terms[q];
        const double alpha = (j == 0) ? coef[q] : 1.0;
        copy_block3(t.core[j], t.Dl[j], n, t.Dr[j], X[j].as<double>(), (long long)n * xd[j + 1],
                    xd[j + 1], j == 0 ? 0 : o0, j == L - 1 ? 0 : o2, alpha, s);
        o0 += t.Dl[j];
        o2 += t.Dr[j];
      }
    }
  }

  // TT rounding of X (right-to-left LQ, left-to-right truncated SVD), normalised, into tt.
  void round_into_tt(std::vector<DevBuf>& X, std::vector<int>& xd) {
    cudaStream_t s = c->stream;
    // right-to-left LQ sweep
    for (int j = L - 1; j >= 1; --j) {
      const int Dl = xd[j], n = tt->phys[j], Dr = xd[j + 1];
      const int cols = n * Dr;
      const int k = std::min(Dl, cols);
      DevBuf Lf, Q;
      Lf.ensure(sizeof(double) * (size_t)Dl * k, s);
      Q.ensure(sizeof(double) * (size_t)k * cols, s);
      c->solver.lq(X[j].as<double>(), Dl, cols, Lf.as<double>(), Q.as<double>(), s);
      X[j] = std::move(Q);
      const int Dl0 = xd[j - 1], n0 = tt->phys[j - 1];
      DevBuf nx;
      nx.ensure(sizeof(double) * (size_t)Dl0 * n0 * k, s);
      matmul_dev(c, X[j - 1].as<double>(), Dl0 * n0, Dl, Lf.as<double>(), k, nx.as<double>());
      X[j - 1] = std::move(nx);
      xd[j] = k;
    }
    // left-to-right truncated SVD sweep
    for (int j = 0; j + 1 < L; ++j) {
      const int Dl = xd[j], n = tt->phys[j], Dr = xd[j + 1];
      const int rows = Dl * n;
      const int kmax = std::min(rows, Dr);
      DevBuf P, SQ;
      P.ensure(sizeof(double) * (size_t)rows * kmax, s);
      SQ.ensure(sizeof(double) * (size_t)kmax * Dr, s);
      double disc = 0.0;
      const int r = svd_split_dev(c, X[j].as<double>(), rows, Dr, o.D_max, o.svd_tol,
                                  P.as<double>(), SQ.as<double>(), &disc);
      X[j] = std::move(P);
      const int n1 = tt->phys[j + 1], Dr1 = xd[j + 2];
      DevBuf nx;
      nx.ensure(sizeof(double) * (size_t)r * n1 * Dr1, s);
      matmul_dev(c, SQ.as<double>(), r, Dr, X[j + 1].as<double>(), n1 * Dr1, nx.as<double>());
      X[j + 1] = std::move(nx);
      xd[j + 1] = r;
    }
    // normalise the last core
    const long long nl = (long long)xd[L - 1] * tt->phys[L - 1];
    const double nrm2 = dot_dev(c, X[L - 1].as<double>(), X[L - 1].as<double>(), nl, 6);
    check_finite(nrm2, "compressed norm");
    A2_REQUIRE(nrm2 > 0.0, "compressed iterate vanished");
    scale_dev(X[L - 1].as<double>(), nullptr, scal(c, 6), nl, s);
    A2_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < L; ++j) tt->cores[j] = std::move(X[j]);
    tt->dims = xd;
  }
};

template <typename T>
double energy_T(a2_ctx* c, const a2_tt* tt, const a2_mpo* mpo, double* norm_out,
                a2_precision prec = A2_FP64) {
  Engine<T> eng(c, mpo, prec);
  cudaStream_t s = c->stream;
  const int L = tt->L;
  DevBuf E, En;
  eng.set_unit(E);
  for (int j = 0; j < L; ++j) {
    const int Dl = tt->dims[j], Dr = tt->dims[j + 1];
    En.ensure(sizeof(T) * (size_t)Dr * mpo->R[j + 1] * Dr, s);
    eng.left_update(E.as<T>(), j, tt->cores[j].as<double>(), Dl, Dr, tt->cores[j].as<double>(),
                    Dl, Dr, En.as<T>());
    std::swap(E, En);
  }
  T e;
  A2_CUDA(cudaMemcpyAsync(&e, E.p, sizeof(T), cudaMemcpyDeviceToHost, s));
  A2_CUDA(cudaStreamSynchronize(s));
  // norm by transfer matrices in FP64
  DevBuf N, Nn, Tm;
  N.ensure(sizeof(double), s);
  const double one = 1.0;
  A2_CUDA(cudaMemcpyAsync(N.p, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  for (int j = 0; j < L; ++j) {
    const int Dl = tt->dims[j], n = tt->phys[j], Dr = tt->dims[j + 1];
    Tm.ensure(sizeof(double) * (size_t)Dl * n * Dr, s);
    matmul_dev(c, N.as<double>(), Dl, Dl, tt->cores[j].as<double>(), n * Dr, Tm.as<double>());
    Nn.ensure(sizeof(double) * (size_t)Dr * Dr, s);
    SimtGemm<double, double> g;
    g.M = Dr; g.N = Dr; g.K = Dl * n;
    g.A = tt->cores[j].as<double>(); g.sam = 1; g.sak = Dr;
    g.B = Tm.as<double>(); g.sbn = 1; g.sbk = Dr;
    g.C = Nn.as<double>(); g.scm = Dr; g.scn = 1;
    simt_gemm(g, s);
    std::swap(N, Nn);
  }
  double nn;
  A2_CUDA(cudaMemcpyAsync(&nn, N.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  A2_CUDA(cudaStreamSynchronize(s));
  check_finite(nn, "norm");
  if (norm_out) *norm_out = std::sqrt(std::max(nn, 0.0));
  return (double)e / nn;
}

a2_status fail(a2_ctx* c, a2_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

template <typename F>
a2_status guarded(a2_ctx* c, F&& f) {
  try {
    f();
    return A2_OK;
  } catch (const ArgError& e) {
    return fail(c, A2_EINVAL, e.what());
  } catch (const NumericError& e) {
    return fail(c, A2_ENUMERIC, e.what());
  } catch (const CudaError& e) {
    const std::string m = e.what();
    if (m.find("out of memory") != std::string::npos) return fail(c, A2_ENOMEM, m);
    return fail(c, A2_ECUDA, m);
  } catch (const std::bad_alloc& e) {
    return fail(c, A2_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, A2_ECUDA, e.what());
  }
}

// Registry of the live handles: a context owns the TT / MPO / H_eff handles made on it, so
// destroying it destroys what is left of them, and a destroy call on a handle that is no
// longer live is ignored (A2_EINVAL) instead of touching freed memory.
enum HandleKind { HK_CTX = 0, HK_TT = 1, HK_MPO = 2, HK_HEFF = 3 };
struct HandleInfo {
  int kind;
  a2_ctx* owner;
};
std::mutex g_handle_mu;
std::map<const void*, HandleInfo> g_handles;

void handle_add(const void* h, int kind, a2_ctx* owner) {
  std::lock_guard<std::mutex> g(g_handle_mu);
  g_handles[h] = HandleInfo{kind, owner};
}
// Removes h if it is live with the given kind; false otherwise.
bool handle_take(const void* h, int kind) {
  std::lock_guard<std::mutex> g(g_handle_mu);
  auto it = g_handles.find(h);
  if (it == g_handles.end() || it->second.kind != kind) return false;
  g_handles.erase(it);
  return true;
}
// Removes and returns every live handle owned by c (ctx itself excluded).
std::vector<std::pair<const void*, int>> handles_owned_by(a2_ctx* c) {
  std::lock_guard<std::mutex> g(g_handle_mu);
  std::vector<std::pair<const void*, int>> out;
  for (auto it = g_handles.begin(); it != g_handles.end();) {
    if (it->second.owner == c && it->second.kind != HK_CTX) {
      out.push_back({it->first, it->second.kind});
      it = g_handles.erase(it);
    } else {
      ++it;
    }
  }
  return out;
}

uint64_t splitmix_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Adjoint of the energy sandwich with respect to one MPO core (the Hellmann-Feynman
// derivative at a fixed TT): G[w,s,t,w'] = sum HL[a,w,a'] U[a,s,b] U[a',t,b'] HR[b,w',b']
// with HL the environment of the sites left of the core and HR of those right of it,
// both built from the same TT (any gauge).  FP64 SIMT contractions:
//   X[a,w,t,b'] = sum_a' HL U;  Z[(s b)][(w t b')] = sum_a U X;
//   G[w,s,t,w'] = sum_{b,b'} Z HR   (batched over b, one launch per (s, t)).
void core_gradient(a2_ctx* c, const double* HL, int Dl, int Rl, const double* U, int n, int Dr,
                   const double* HR, int Rr, double* G, DevBuf& bx, DevBuf& bz) {
  cudaStream_t s = c->stream;
  bx.ensure(sizeof(double) * (size_t)Dl * Rl * n * Dr, s);
  bz.ensure(sizeof(double) * (size_t)n * Dr * Rl * n * Dr, s);
  double* X = bx.as<double>();
  double* Z = bz.as<double>();
  const long long nD = (long long)n * Dr, RnD = (long long)Rl * n * Dr;
  {
    SimtGemm<double, double> g;
    g.M = Dl * Rl; g.N = (int)nD; g.K = Dl;
    g.A = HL; g.sam = Dl; g.sak = 1;
    g.B = U; g.sbn = 1; g.sbk = nD;
    g.C = X; g.scm = nD; g.scn = 1;
    simt_gemm(g, s);
  }
  {
    SimtGemm<double, double> g;
    g.M = (int)nD; g.N = (int)RnD; g.K = Dl;
    g.A = U; g.sam = 1; g.sak = nD;
    g.B = X; g.sbn = 1; g.sbk = RnD;
    g.C = Z; g.scm = RnD; g.scn = 1;
    simt_gemm(g, s);
  }
  fill_zero(G, sizeof(double) * (size_t)Rl * n * n * Rr, s);
  for (int sx = 0; sx < n; ++sx)
    for (int t = 0; t < n; ++t) {
      SimtGemm<double, double> g;
      g.M = Rl; g.N = Rr; g.K = Dr;
      g.A = Z + (long long)sx * Dr * RnD + (long long)t * Dr; g.sam = nD; g.sak = 1;
      g.B = HR; g.sbn = Dr; g.sbk = 1;
      g.C = G + ((long long)sx * n + t) * Rr; g.scm = (long long)n * n * Rr; g.scn = 1;
      g.batch = Dr; g.abs = RnD; g.bbs = (long long)Rr * Dr; g.cbs = 0;
      g.mode = GEMM_ATOMIC;
      simt_gemm(g, s);
    }
}

}  // namespace

// ============================================================================= C ABI
// Deletes the TT / MPO / H_eff handles still registered to c (defined after a2_heff).
void destroy_owned(a2_ctx* c);

extern "C" {

a2_status a2_ctx_create(int device, void* cuda_stream, a2_ctx** out) {
  if (!out) return A2_EINVAL;
  *out = nullptr;
  a2_ctx* c = new (std::nothrow) a2_ctx();
  if (!c) return A2_ENOMEM;
  a2_status st = guarded(c, [&] {
    A2_CUDA(cudaSetDevice(device));
    c->device = device;
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      A2_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    cudaMemPool_t pool;
    A2_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    A2_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    c->solver.init(c->stream);
    c->scal.ensure(sizeof(double) * 16384, c->stream);
    c->partial.ensure(sizeof(double) * kReduceBlocks * 64, c->stream);
    A2_CUDA(cudaMallocHost(&c->h_scal, sizeof(double) * 64));
    A2_CUDA(cudaStreamSynchronize(c->stream));
  });
  if (st != A2_OK) {
    fprintf(stderr, "a2_ctx_create: %s\n", c->err.c_str());
    delete c;
    return st;
  }
  handle_add(c, HK_CTX, c);
  *out = c;
  return A2_OK;
}

a2_status a2_ctx_destroy(a2_ctx* c) {
  if (!c || !handle_take(c, HK_CTX)) return A2_EINVAL;
  // handles still attached to the context go first (their buffers use its stream)
  cudaStreamSynchronize(c->stream);
  destroy_owned(c);
  for (a2_ctx* l : c->lanes) {
    destroy_ctx_resources(l);
    if (l->hi) {
      cudaStreamSynchronize(l->hi);
      cudaStreamDestroy(l->hi);
      cudaEventDestroy(l->ev_to_hi);
      cudaEventDestroy(l->ev_from_hi);
    }
    cudaStreamDestroy(l->stream);
    delete l;
  }
  c->lanes.clear();
  destroy_ctx_resources(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  // hand the pool's cached, now unused memory back (other contexts keep theirs)
  try {
    int prev = 0;
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(c->device) == cudaSuccess) {
      cudaMemPoolTrimTo(lib_pool(), 0);   // the context's streams were synchronised above
      cudaSetDevice(prev);
    }
  } catch (...) {
  }
  delete c;
  return A2_OK;
}

const char* a2_last_error(const a2_ctx* c) { return c ? c->err.c_str() : "null context"; }

a2_status a2_ctx_synchronize(a2_ctx* c) {
  if (!c) return A2_EINVAL;
  return guarded(c, [&] { A2_CUDA(cudaStreamSynchronize(c->stream)); });
}

a2_status a2_tt_create(a2_ctx* c, int L, const int* phys, const int* bonds, uint64_t seed,
                       a2_tt** out) {
  if (!c || !out || !phys || L < 2) return c ? fail(c, A2_EINVAL, "a2_tt_create: bad arguments") : A2_EINVAL;
  *out = nullptr;
  auto* t = new (std::nothrow) a2_tt();
  if (!t) return A2_ENOMEM;
  a2_status st = guarded(c, [&] {
    t->ctx = c;
    t->L = L;
    t->phys.assign(phys, phys + L);
    for (int n : t->phys) A2_REQUIRE(n >= 1, "physical dims must be >= 1");
    t->dims.assign(L + 1, 1);
    for (int k = 1; k < L; ++k) {
      double left = 1, right = 1;
      for (int j = 0; j < k; ++j) left *= phys[j];
      for (int j = k; j < L; ++j) right *= phys[j];
      double cap = std::min(left, right);
      const int want = bonds ? bonds[k - 1] : 1;
      A2_REQUIRE(want >= 1, "bond dims must be >= 1");
      t->dims[k] = (int)std::min<double>(want, cap);
    }
    t->cores.resize(L);
    uint64_t state = seed;
    for (int j = 0; j < L; ++j) {
      const size_t nel = (size_t)t->dims[j] * phys[j] * t->dims[j + 1];
      std::vector<double> h(nel);
      for (size_t e = 0; e < nel; ++e) {
        const uint64_t z = splitmix_next(state);
        h[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
      }
      upload(t->cores[j], h.data(), sizeof(double) * nel, c->stream);
      A2_CUDA(cudaStreamSynchronize(c->stream));
    }
    left_orthogonalize(t, nullptr);
    A2_CUDA(cudaStreamSynchronize(c->stream));
  });
  if (st != A2_OK) { delete t; return st; }
  handle_add(t, HK_TT, c);
  *out = t;
  return A2_OK;
}

a2_status a2_tt_set_core(a2_tt* t, int site, int Dl, int n, int Dr, const double* h) {
  if (!t) return A2_EINVAL;
  a2_ctx* c = t->ctx;
  return guarded(c, [&] {
    A2_REQUIRE(site >= 0 && site < t->L && h, "a2_tt_set_core: bad site or pointer");
    A2_REQUIRE(n == t->phys[site] && Dl >= 1 && Dr >= 1, "a2_tt_set_core: bad dims");
    A2_REQUIRE(site > 0 || Dl == 1, "first core must have Dl = 1");
    A2_REQUIRE(site < t->L - 1 || Dr == 1, "last core must have Dr = 1");
    const size_t nel = (size_t)Dl * n * Dr;
    t->cores[site].release();
    upload(t->cores[site], h, sizeof(double) * nel, c->stream);
    A2_CUDA(cudaStreamSynchronize(c->stream));
    t->dims[site] = Dl;
    t->dims[site + 1] = Dr;
  });
}

a2_status a2_tt_get_core(const a2_tt* t, int site, int* Dl, int* n, int* Dr, double* h) {
  if (!t) return A2_EINVAL;
  a2_ctx* c = t->ctx;
  return guarded(c, [&] {
    A2_REQUIRE(site >= 0 && site < t->L, "a2_tt_get_core: bad site");
    if (Dl) *Dl = t->dims[site];
    if (n) *n = t->phys[site];
    if (Dr) *Dr = t->dims[site + 1];
    if (h) {
      const size_t nel = (size_t)t->dims[site] * t->phys[site] * t->dims[site + 1];
      A2_CUDA(cudaMemcpyAsync(h, t->cores[site].p, sizeof(double) * nel, cudaMemcpyDeviceToHost,
                              c->stream));
      A2_CUDA(cudaStreamSynchronize(c->stream));
    }
  });
}

a2_status a2_tt_save(const a2_tt* t, const char* path) {
  if (!t) return A2_EINVAL;
  a2_ctx* c = t->ctx;
  return guarded(c, [&] {
    A2_REQUIRE(path, "a2_tt_save: null path");
    tt_check(t);
    std::FILE* f = std::fopen(path, "wb");
    A2_REQUIRE(f, "a2_tt_save: cannot open the file for writing");
    bool ok = std::fwrite("A2TTCKP1", 1, 8, f) == 8;
    const int32_t L = t->L;
    ok = ok && std::fwrite(&L, sizeof(L), 1, f) == 1;
    std::vector<int32_t> ph(t->phys.begin(), t->phys.end()), bd(t->dims.begin(), t->dims.end());
    ok = ok && std::fwrite(ph.data(), sizeof(int32_t), ph.size(), f) == ph.size();
    ok = ok && std::fwrite(bd.data(), sizeof(int32_t), bd.size(), f) == bd.size();
    std::vector<double> h;
    for (int j = 0; ok && j < t->L; ++j) {
      const size_t nel = (size_t)t->dims[j] * t->phys[j] * t->dims[j + 1];
      h.resize(nel);
      A2_CUDA(cudaMemcpyAsync(h.data(), t->cores[j].p, sizeof(double) * nel,
                              cudaMemcpyDeviceToHost, c->stream));
      A2_CUDA(cudaStreamSynchronize(c->stream));
      ok = std::fwrite(h.data(), sizeof(double), nel, f) == nel;
    }
    ok = (std::fclose(f) == 0) && ok;
    A2_REQUIRE(ok, "a2_tt_save: write failed");
  });
}

a2_status a2_tt_load(a2_ctx* c, const char* path, a2_tt** out) {
  if (!c || !out) return c ? fail(c, A2_EINVAL, "a2_tt_load: null argument") : A2_EINVAL;
  *out = nullptr;
  auto* t = new (std::nothrow) a2_tt();
  if (!t) return A2_ENOMEM;
  a2_status st = guarded(c, [&] {
    A2_REQUIRE(path, "a2_tt_load: null path");
    std::FILE* f = std::fopen(path, "rb");
    A2_REQUIRE(f, "a2_tt_load: cannot open the file");
    struct Closer {
      std::FILE* f;
      ~Closer() { std::fclose(f); }
    } closer{f};
    char magic[8];
    A2_REQUIRE(std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "A2TTCKP1", 8) == 0,
               "a2_tt_load: not a TT checkpoint");
    int32_t L = 0;
    A2_REQUIRE(std::fread(&L, sizeof(L), 1, f) == 1 && L >= 2 && L <= (1 << 20),
               "a2_tt_load: bad site count");
    std::vector<int32_t> ph(L), bd(L + 1);
    A2_REQUIRE(std::fread(ph.data(), sizeof(int32_t), L, f) == (size_t)L &&
                   std::fread(bd.data(), sizeof(int32_t), L + 1, f) == (size_t)(L + 1),
               "a2_tt_load: truncated header");
    A2_REQUIRE(bd[0] == 1 && bd[L] == 1, "a2_tt_load: boundary bonds must be 1");
    for (int j = 0; j < L; ++j)
      A2_REQUIRE(ph[j] >= 1 && bd[j] >= 1 && bd[j + 1] >= 1 &&
                     (double)bd[j] * ph[j] * bd[j + 1] < 4e9,
                 "a2_tt_load: bad dimensions");
    t->ctx = c;
    t->L = L;
    t->phys.assign(ph.begin(), ph.end());
    t->dims.assign(bd.begin(), bd.end());
    t->cores.resize(L);
    std::vector<double> h;
    for (int j = 0; j < L; ++j) {
      const size_t nel = (size_t)bd[j] * ph[j] * bd[j + 1];
      h.resize(nel);
      A2_REQUIRE(std::fread(h.data(), sizeof(double), nel, f) == nel, "a2_tt_load: truncated core");
      upload(t->cores[j], h.data(), sizeof(double) * nel, c->stream);
      A2_CUDA(cudaStreamSynchronize(c->stream));   // h is reused for the next core
    }
    char extra;
    A2_REQUIRE(std::fread(&extra, 1, 1, f) == 0, "a2_tt_load: trailing data");
  });
  if (st != A2_OK) {
    delete t;
    return st;
  }
  handle_add(t, HK_TT, c);
  *out = t;
  return A2_OK;
}

a2_status a2_tt_left_orthogonalize(a2_tt* t, double* norm_out) {
  if (!t) return A2_EINVAL;
  return guarded(t->ctx, [&] {
    for (int j = 0; j + 1 < t->L; ++j) {
      A2_REQUIRE(t->cores[j].bytes >= sizeof(double) * (size_t)t->dims[j] * t->phys[j] * t->dims[j + 1],
                 "inconsistent TT bond dims");
    }
    tt_check(t);
    left_orthogonalize(t, norm_out);
    A2_CUDA(cudaStreamSynchronize(t->ctx->stream));
  });
}

a2_status a2_tt_destroy(a2_tt* t) {
  if (!t || !handle_take(t, HK_TT)) return A2_EINVAL;
  cudaStreamSynchronize(t->ctx->stream);
  delete t;
  return A2_OK;
}

a2_status a2_mpo_load(a2_ctx* c, int L, const int* phys, const int* R, const double* const* cores,
                      a2_mpo** out) {
  if (!c || !out) return A2_EINVAL;
  *out = nullptr;
  auto* m = new (std::nothrow) a2_mpo();
  if (!m) return A2_ENOMEM;
  a2_status st = guarded(c, [&] {
    A2_REQUIRE(L >= 2 && phys && R && cores, "a2_mpo_load: bad arguments");
    A2_REQUIRE(R[0] == 1 && R[L] == 1, "MPO boundary bonds must be 1");
    m->ctx = c;
    m->L = L;
    m->phys.assign(phys, phys + L);
    m->R.assign(R, R + L + 1);
    m->site.resize(L);
    for (int j = 0; j < L; ++j) {
      A2_REQUIRE(cores[j] && R[j] >= 1 && R[j + 1] >= 1 && phys[j] >= 1, "a2_mpo_load: bad core");
      build_site(m->site[j], cores[j], R[j], phys[j], R[j + 1], c->stream);
    }
    A2_CUDA(cudaStreamSynchronize(c->stream));
  });
  if (st != A2_OK) { delete m; return st; }
  handle_add(m, HK_MPO, c);
  *out = m;
  return A2_OK;
}

a2_status a2_mpo_nnz(const a2_mpo* m, int site, long long* nnz) {
  if (!m || !nnz || site < 0 || site >= m->L) return A2_EINVAL;
  *nnz = m->site[site].nnz;
  return A2_OK;
}

a2_status a2_set_autotune(int enable) {
  tc_autotune((enable & 1) != 0);
  sparse_autotune((enable & 2) != 0);
  return A2_OK;
}

a2_status a2_mpo_fold_split(const double* W, int Rl, int n, int Rr, double* G_out,
                            long long* nnz_g, int* foldable) {
  if (!W || !nnz_g || !foldable || Rl < 1 || n < 1 || Rr < 1) return A2_EINVAL;
  try {
    std::vector<double> G((size_t)Rl * Rr, 0.0);
    *nnz_g = identity_block_split(W, Rl, n, Rr, G.data());
    *foldable = fold_worthwhile(*nnz_g, Rl, Rr) ? 1 : 0;
    if (G_out) std::copy(G.begin(), G.end(), G_out);
  } catch (...) {
    return A2_ENOMEM;
  }
  return A2_OK;
}

a2_status a2_mpo_fold_info(const a2_mpo* m, int site, int* foldable, long long* nnz_g) {
  if (!m || !foldable || !nnz_g || site < 0 || site >= m->L) return A2_EINVAL;
  *foldable = m->site[site].fold() ? 1 : 0;
  *nnz_g = m->site[site].nnz_g;
  return A2_OK;
}

a2_status a2_mpo_set_fold(a2_mpo* m, int enable) {
  if (!m) return A2_EINVAL;
  for (auto& so : m->site) so.fold_on = enable ? 1 : 0;
  return A2_OK;
}

a2_status a2_mpo_destroy(a2_mpo* m) {
  if (!m || !handle_take(m, HK_MPO)) return A2_EINVAL;
  cudaStreamSynchronize(m->ctx->stream);
  delete m;
  return A2_OK;
}

static a2_status run_sweep(a2_ctx* c, a2_tt* t, const a2_mpo* m, const a2_sweep_opts* o,
                           a2_sweep_report* rep, bool classical) {
  if (!c || !t || !m || !o) return c ? fail(c, A2_EINVAL, "null argument") : A2_EINVAL;
  // keep the iterate until the iteration succeeds (Alg. 2 saves U^(n),d)
  std::vector<DevBuf> saved;
  std::vector<int> saved_dims = t->dims;
  a2_status st = guarded(c, [&] {
    A2_REQUIRE(t->ctx == c && m->L == t->L, "handles from different contexts / sizes");
    saved.resize(t->L);
    for (int j = 0; j < t->L; ++j) {
      saved[j].ensure(t->cores[j].bytes, c->stream);
      A2_CUDA(cudaMemcpyAsync(saved[j].p, t->cores[j].p, t->cores[j].bytes,
                              cudaMemcpyDeviceToDevice, c->stream));
    }
    if (o->prec == A2_FP64 || o->prec == A2_F64EMU || o->prec == A2_BF16 ||
        o->prec == A2_F32EMU) {
      // FP64 environments; the tensor-core modes keep them to FP64-class accuracy
      if (o->prec != A2_FP64 && !tc_available())
        throw ArgError("this precision needs the tcgen05 path, which this build lacks");
      GemmTcScope gs(c, o->prec != A2_FP64);
      Sweeper<double> sw(c, t, m, *o);
      sw.run(rep, classical);
    } else if (o->prec == A2_FP32) {
      Sweeper<float> sw(c, t, m, *o);
      sw.run(rep, classical);
    } else {
      throw ArgError("unsupported precision");
    }
  });
  if (st != A2_OK) {
    for (int j = 0; j < t->L && j < (int)saved.size(); ++j)
      if (saved[j].p) t->cores[j] = std::move(saved[j]);
    t->dims = saved_dims;
    cudaStreamSynchronize(c->stream);
  }
  return st;
}

a2_status a2_additive_sweep(a2_ctx* c, a2_tt* t, const a2_mpo* m, const a2_sweep_opts* o,
                            a2_sweep_report* rep) {
  return run_sweep(c, t, m, o, rep, false);
}

a2_status a2_classical_sweep(a2_ctx* c, a2_tt* t, const a2_mpo* m, const a2_sweep_opts* o,
                             a2_sweep_report* rep) {
  return run_sweep(c, t, m, o, rep, true);
}

a2_status a2_coarse_solve(a2_ctx* c, int m, const double* A, const double* S, double eps,
                          double* c_out, double* lam_out, int* rank_out) {
  if (!c) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(m >= 1 && m <= 63 && A && S && c_out && lam_out, "a2_coarse_solve: bad arguments");
    cudaStream_t s = c->stream;
    double* dA = scal(c, 9000);
    double* dS = dA + m * m;
    double* dc = dS + m * m;
    double* dl = dc + m;
    int* drk = reinterpret_cast<int*>(dl + 1);
    A2_CUDA(cudaMemcpyAsync(dA, A, sizeof(double) * m * m, cudaMemcpyHostToDevice, s));
    A2_CUDA(cudaMemcpyAsync(dS, S, sizeof(double) * m * m, cudaMemcpyHostToDevice, s));
    coarse_solve_dev(dA, dS, m, eps, dc, dl, drk, drk + 1, s);
    int rk[2];
    A2_CUDA(cudaMemcpyAsync(c_out, dc, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaMemcpyAsync(lam_out, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaMemcpyAsync(rk, drk, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaStreamSynchronize(s));
    if (rank_out) *rank_out = rk[0];
    if (rk[1] != 0) throw NumericError("coarse Jacobi did not converge");
  });
}

a2_status a2_energy(a2_ctx* c, const a2_tt* t, const a2_mpo* m, a2_precision prec, double* E,
                    double* norm_out) {
  if (!c || !t || !m || !E) return c ? fail(c, A2_EINVAL, "null argument") : A2_EINVAL;
  return guarded(c, [&] {
    tt_check(t);
    A2_REQUIRE(t->phys == m->phys, "TT and MPO physical dims differ");
    if (prec == A2_FP64) *E = energy_T<double>(c, t, m, norm_out);
    else if (prec == A2_F64EMU) {
      GemmTcScope gs(c, true);
      *E = energy_T<double>(c, t, m, norm_out, A2_F64EMU);
    }
    else *E = energy_T<float>(c, t, m, norm_out);
  });
}

struct a2_heff {
  a2_ctx* ctx = nullptr;
  const a2_mpo* mpo = nullptr;
  int k = 0, Dl = 0, Dr = 0;
  a2_precision prec = A2_FP64;
  DevBuf env;          // FP64 / FP32 copies of L and R
  Bf16Envs bfe;        // BF16 / split planes (with folded blocks)
  OzEnvs oze;          // Ozaki slices (FP64 emulation)
};

a2_status a2_heff_create(a2_ctx* c, const a2_mpo* m, int k, a2_precision prec, int Dl, int Dr,
                         const double* L, const double* R, a2_heff** out) {
  if (!c || !m || !out) return c ? fail(c, A2_EINVAL, "null argument") : A2_EINVAL;
  *out = nullptr;
  auto* h = new (std::nothrow) a2_heff();
  if (!h) return A2_ENOMEM;
  a2_status st = guarded(c, [&] {
    A2_REQUIRE(k >= 0 && k + 1 < m->L && Dl >= 1 && Dr >= 1 && L && R,
               "a2_heff_create: bad arguments");
    const SiteOps& A1 = m->site[k];
    const SiteOps& A2 = m->site[k + 1];
    cudaStream_t s = c->stream;
    h->ctx = c; h->mpo = m; h->k = k; h->Dl = Dl; h->Dr = Dr; h->prec = prec;
    const long long nl = (long long)Dl * A1.Rl * Dl, nr = (long long)Dr * A2.Rr * Dr;
    if (prec == A2_FP64) {
      h->env.ensure(sizeof(double) * (size_t)(nl + nr), s);
      A2_CUDA(cudaMemcpyAsync(h->env.p, L, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
      A2_CUDA(cudaMemcpyAsync(h->env.as<double>() + nl, R, sizeof(double) * nr,
                              cudaMemcpyDeviceToDevice, s));
    } else if (prec == A2_FP32) {
      h->env.ensure(sizeof(float) * (size_t)(nl + nr), s);
      convert<double, float>(L, h->env.as<float>(), nl, s);
      convert<double, float>(R, h->env.as<float>() + nl, nr, s);
    } else if (prec == A2_BF16 || prec == A2_F32EMU) {
      A2_REQUIRE(tc_available(), "this precision needs the tcgen05 path");
      h->bfe.set<double>(c, L, Dl, A1.Rl, R, Dr, A2.Rr, prec == A2_BF16 ? 1 : 3, &A1, &A2);
    } else if (prec == A2_F64EMU) {
      A2_REQUIRE(tc_available(), "this precision needs the tcgen05 path");
      h->oze.set(c, L, Dl, A1.Rl, R, Dr, A2.Rr);
    } else {
      throw ArgError("unsupported precision");
    }
    A2_CUDA(cudaStreamSynchronize(s));
  });
  if (st != A2_OK) { delete h; return st; }
  handle_add(h, HK_HEFF, c);
  *out = h;
  return A2_OK;
}

a2_status a2_heff_apply_op(a2_heff* h, const double* x, double* y) {
  if (!h) return A2_EINVAL;
  a2_ctx* c = h->ctx;
  return guarded(c, [&] {
    A2_REQUIRE(x && y, "a2_heff_apply_op: null vector");
    const SiteOps& A1 = h->mpo->site[h->k];
    const SiteOps& A2 = h->mpo->site[h->k + 1];
    const int Dl = h->Dl, Dr = h->Dr;
    const long long nl = (long long)Dl * A1.Rl * Dl;
    cudaStream_t s = c->stream;
    if (h->prec == A2_FP64) {
      heff_T<double>(c, A1, A2, h->env.as<double>(), h->env.as<double>() + nl, Dl, Dr, x, y);
    } else if (h->prec == A2_FP32) {
      const long long N = (long long)Dl * A1.n * A2.n * Dr;
      c->xa.ensure(sizeof(float) * N, s);
      c->ya.ensure(sizeof(float) * N, s);
      convert<double, float>(x, c->xa.as<float>(), N, s);
      heff_T<float>(c, A1, A2, h->env.as<float>(), h->env.as<float>() + nl, Dl, Dr,
                    c->xa.as<float>(), c->ya.as<float>());
      convert<float, double>(c->ya.as<float>(), y, N, s);
    } else if (h->prec == A2_BF16) {
      heff_bf16(c, A1, A2, h->bfe, Dl, Dr, x, y);
    } else if (h->prec == A2_F64EMU) {
      heff_f64emu(c, A1, A2, h->oze, Dl, Dr, x, y);
    } else {
      heff_emu(c, A1, A2, h->bfe, Dl, Dr, x, y);
    }
  });
}

a2_status a2_heff_destroy(a2_heff* h) {
  if (!h || !handle_take(h, HK_HEFF)) return A2_EINVAL;
  cudaStreamSynchronize(h->ctx->stream);
  delete h;
  return A2_OK;
}

a2_status a2_energy_gradient(a2_ctx* c, const a2_tt* t, const a2_mpo* m, long long nparam,
                             long long nmap, const long long* map_param, const int* map_site,
                             const long long* map_index, const double* map_factor,
                             double* grad_out, double* E_out) {
  if (!c || !t || !m) return c ? fail(c, A2_EINVAL, "null argument") : A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(nparam >= 1 && nmap >= 0 && grad_out && (nmap == 0 || (map_param && map_site &&
               map_index && map_factor)), "a2_energy_gradient: bad arguments");
    tt_check(t);
    A2_REQUIRE(t->ctx == c && m->L == t->L && t->phys == m->phys, "TT / MPO mismatch");
    const int L = t->L;
    cudaStream_t s = c->stream;
    // map entries grouped by site, checked against the core sizes
    std::vector<std::vector<long long>> by_site(L);
    for (long long e = 0; e < nmap; ++e) {
      const int j = map_site[e];
      A2_REQUIRE(j >= 0 && j < L, "a2_energy_gradient: map site out of range");
      const long long size = (long long)m->R[j] * m->phys[j] * m->phys[j] * m->R[j + 1];
      A2_REQUIRE(map_index[e] >= 0 && map_index[e] < size && map_param[e] >= 0 &&
                 map_param[e] < nparam, "a2_energy_gradient: map entry out of range");
      by_site[j].push_back(e);
    }
    double nrm = 0.0;
    const double E = energy_T<double>(c, t, m, &nrm);
    const double n2 = nrm * nrm;
    A2_REQUIRE(n2 > 0.0, "a2_energy_gradient: zero TT");
    Engine<double> eng(c, m, A2_FP64);
    // right environments of every suffix
    std::vector<DevBuf> HR(L + 1);
    eng.set_unit(HR[L]);
    for (int j = L - 1; j >= 1; --j) {
      const int Dl = t->dims[j], Dr = t->dims[j + 1];
      HR[j].ensure(sizeof(double) * (size_t)Dl * m->R[j] * Dl, s);
      eng.right_update(HR[j + 1].as<double>(), j, t->cores[j].as<double>(), Dl, Dr,
                       t->cores[j].as<double>(), Dl, Dr, HR[j].as<double>());
    }
    DevBuf grad, HL, HLn, G, bx, bz, mp, mi, mf;
    grad.ensure(sizeof(double) * (size_t)nparam, s);
    fill_zero(grad.p, sizeof(double) * (size_t)nparam, s);
    eng.set_unit(HL);
    for (int j = 0; j < L; ++j) {
      const int Dl = t->dims[j], n = t->phys[j], Dr = t->dims[j + 1];
      const int Rl = m->R[j], Rr = m->R[j + 1];
      if (!by_site[j].empty()) {
        G.ensure(sizeof(double) * (size_t)Rl * n * n * Rr, s);
        core_gradient(c, HL.as<double>(), Dl, Rl, t->cores[j].as<double>(), n, Dr,
                      HR[j + 1].as<double>(), Rr, G.as<double>(), bx, bz);
        const auto& es = by_site[j];
        const size_t ne = es.size();
        std::vector<long long> hp(ne), hi(ne);
        std::vector<double> hf(ne);
        for (size_t q = 0; q < ne; ++q) {
          hp[q] = map_param[es[q]];
          hi[q] = map_index[es[q]];
          hf[q] = map_factor[es[q]] / n2;
        }
        upload(mp, hp.data(), sizeof(long long) * ne, s);
        upload(mi, hi.data(), sizeof(long long) * ne, s);
        upload(mf, hf.data(), sizeof(double) * ne, s);
        gather_axpy_atomic(G.as<double>(), mi.as<long long>(), mp.as<long long>(),
                           mf.as<double>(), (long long)ne, grad.as<double>(), s);
        A2_CUDA(cudaStreamSynchronize(s));     // the host staging vectors go out of scope
      }
      if (j + 1 < L) {
        HLn.ensure(sizeof(double) * (size_t)Dr * m->R[j + 1] * Dr, s);
        eng.left_update(HL.as<double>(), j, t->cores[j].as<double>(), Dl, Dr,
                        t->cores[j].as<double>(), Dl, Dr, HLn.as<double>());
        std::swap(HL, HLn);
        HR[j + 1].release();
      }
    }
    A2_CUDA(cudaMemcpyAsync(grad_out, grad.p, sizeof(double) * (size_t)nparam,
                            cudaMemcpyDeviceToHost, s));
    A2_CUDA(cudaStreamSynchronize(s));
    if (E_out) *E_out = E;
  });
}

a2_status a2_heff_apply(a2_ctx* c, const a2_mpo* m, int k, a2_precision prec, int Dl, int Dr,
                        const double* L, const double* R, const double* x, double* y) {
  if (!c || !m) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(k >= 0 && k + 1 < m->L && Dl >= 1 && Dr >= 1 && L && R && x && y,
               "a2_heff_apply: bad arguments");
    const SiteOps& A1 = m->site[k];
    const SiteOps& A2 = m->site[k + 1];
    cudaStream_t s = c->stream;
    if (prec == A2_FP64) {
      heff_T<double>(c, A1, A2, L, R, Dl, Dr, x, y);
    } else if (prec == A2_FP32) {
      const long long nl = (long long)Dl * A1.Rl * Dl, nr = (long long)Dr * A2.Rr * Dr;
      const long long N = (long long)Dl * A1.n * A2.n * Dr;
      c->cb.ensure(sizeof(float) * (nl + nr), s);
      float* Lf = c->cb.as<float>();
      float* Rf = Lf + nl;
      convert<double, float>(L, Lf, nl, s);
      convert<double, float>(R, Rf, nr, s);
      c->xa.ensure(sizeof(float) * N, s);
      c->ya.ensure(sizeof(float) * N, s);
      convert<double, float>(x, c->xa.as<float>(), N, s);
      heff_T<float>(c, A1, A2, Lf, Rf, Dl, Dr, c->xa.as<float>(), c->ya.as<float>());
      convert<float, double>(c->ya.as<float>(), y, N, s);
    } else if (prec == A2_BF16 || prec == A2_F32EMU) {
      A2_REQUIRE(tc_available(), "this precision needs the tcgen05 path");
      Bf16Envs E;
      E.set<double>(c, L, Dl, A1.Rl, R, Dr, A2.Rr, prec == A2_BF16 ? 1 : 3, &A1, &A2);
      if (prec == A2_BF16) heff_bf16(c, A1, A2, E, Dl, Dr, x, y);
      else heff_emu(c, A1, A2, E, Dl, Dr, x, y);
      A2_CUDA(cudaStreamSynchronize(s));
    } else if (prec == A2_F64EMU) {
      A2_REQUIRE(tc_available(), "this precision needs the tcgen05 path");
      OzEnvs E;
      E.set(c, L, Dl, A1.Rl, R, Dr, A2.Rr);
      heff_f64emu(c, A1, A2, E, Dl, Dr, x, y);
      A2_CUDA(cudaStreamSynchronize(s));
    } else {
      throw ArgError("unsupported precision");
    }
  });
}

a2_status a2_env_update(a2_ctx* c, const a2_mpo* m, int j, int side, a2_precision prec, int Dlb,
                        int Drb, int Dlk, int Drk, const double* in, const double* bra,
                        const double* ket, double* out) {
  if (!c || !m) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(j >= 0 && j < m->L && (side == 0 || side == 1) && in && bra && ket && out,
               "a2_env_update: bad arguments");
    const SiteOps& so = m->site[j];
    cudaStream_t s = c->stream;
    const int n = so.n;
    if (prec == A2_FP64) {
      if (side == 0) env_left<double>(c, so, in, bra, Dlb, Drb, ket, Dlk, Drk, out);
      else env_right<double>(c, so, in, bra, Dlb, Drb, ket, Dlk, Drk, out);
    } else if (prec == A2_F64EMU) {   // Ozaki-emulated GEMMs, double-float sparse stage
      A2_REQUIRE(tc_available(), "this precision needs the tcgen05 path");
      if (side == 0) env_left_f64e(c, so, in, bra, Dlb, Drb, ket, Dlk, Drk, out);
      else env_right_f64e(c, so, in, bra, Dlb, Drb, ket, Dlk, Drk, out);
    } else {
      const long long nin = side == 0 ? (long long)Dlb * so.Rl * Dlk : (long long)Drb * so.Rr * Drk;
      const long long nout = side == 0 ? (long long)Drb * so.Rr * Drk : (long long)Dlb * so.Rl * Dlk;
      const long long nb = (long long)Dlb * n * Drb, nk = (long long)Dlk * n * Drk;
      // own buffer: the update kernels use the context scratch (cb, tmp1, tmp2, t3)
      DevBuf fbuf;
      fbuf.ensure(sizeof(float) * (nin + nout + nb + nk), s);
      float* fi = fbuf.as<float>();
      float* fo = fi + nin;
      float* fb = fo + nout;
      float* fk = fb + nb;
      convert<double, float>(in, fi, nin, s);
      convert<double, float>(bra, fb, nb, s);
      convert<double, float>(ket, fk, nk, s);
      if (prec == A2_F32EMU || prec == A2_BF16) {
        A2_REQUIRE(tc_available(), "this precision needs the tcgen05 path");
        if (side == 0) env_left_emu(c, so, fi, bra, Dlb, Drb, ket, Dlk, Drk, fo);
        else env_right_emu(c, so, fi, bra, Dlb, Drb, ket, Dlk, Drk, fo);
      } else if (side == 0) {
        env_left<float>(c, so, fi, fb, Dlb, Drb, fk, Dlk, Drk, fo);
      } else {
        env_right<float>(c, so, fi, fb, Dlb, Drb, fk, Dlk, Drk, fo);
      }
      convert<float, double>(fo, out, nout, s);
    }
  });
}

a2_status a2_gemm_bf16(a2_ctx* c, int M, int N, int K, const void* A, long long lda,
                       const void* B, long long ldb, float* C, long long ldc, int splitk) {
  if (!c) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(M >= 1 && N >= 1 && K >= 1 && A && B && C && splitk >= 1, "a2_gemm_bf16: bad arguments");
    A2_REQUIRE(tc_available(), "tcgen05 path not built");
    if (splitk > 1) fill_zero(C, sizeof(float) * (size_t)M * ldc, c->stream);
    tc_gemm_bf16(static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B),
                 ldb, M, N, K, C, ldc, splitk > 1 ? 2 : 1, splitk, c->stream);
    A2_CUDA(cudaStreamSynchronize(c->stream));
  });
}

a2_status a2_device_error(a2_ctx* c, int reset, int* code_out) {
  if (!c || !code_out) return A2_EINVAL;
  return guarded(c, [&] {
    A2_CUDA(cudaStreamSynchronize(c->stream));
    const int f = factor_error_flag(reset != 0);
    *code_out = tc_error_flag(reset != 0);
    if (!*code_out && f) *code_out = 100 + f;
  });
}

a2_status a2_lq(a2_ctx* c, int rows, int cols, const double* M, double* L, double* Q) {
  if (!c) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(rows >= 1 && cols >= 1 && M && L && Q, "a2_lq: bad arguments");
    c->solver.lq(M, rows, cols, L, Q, c->stream);
    A2_CUDA(cudaStreamSynchronize(c->stream));
    if (factor_error_flag(true)) throw CudaError("a2_lq: a bounded wait of the LQ kernel gave up");
  });
}

a2_status a2_selftest_timeout(a2_ctx* c, int* code_out) {
  if (!c || !code_out) return A2_EINVAL;
  int code = 0;
  a2_status st = guarded(c, [&] {
    A2_REQUIRE(tc_available(), "the tcgen05 path is not built");
    A2_CUDA(cudaSetDevice(c->device));
    A2_CUDA(cudaStreamSynchronize(c->stream));
    A2_REQUIRE(tc_error_flag(false) == 0,
               "a2_selftest_timeout: the device error word is already set");
    code = tc_selftest_timeout(c->stream);
  });
  if (st != A2_OK) return st;
  *code_out = code;
  if (code == 0) return fail(c, A2_ECUDA, "a2_selftest_timeout: the wait did not run out");
  return fail(c, A2_ETIMEOUT, "a bounded device wait gave up (error code " +
                                  std::to_string(code) + ", self-test)");
}

a2_status a2_profile(a2_ctx* c, int op, int kind, long long* launches, double* ms,
                     double* flops, double* bytes) {
  if (!c) return A2_EINVAL;
  return guarded(c, [&] {
    A2_CUDA(cudaStreamSynchronize(c->stream));
    if (op == 0) prof_enable(false);
    else if (op == 1) prof_enable(true);
    else if (op == 2) prof_reset();
    else if (op == 3) prof_read(kind, launches, ms, flops, bytes);
    else if (op == 4) { if (launches) *launches = launch_count(); }
    else throw ArgError("a2_profile: op must be 0..4");
  });
}

a2_status a2_svd_split(a2_ctx* c, int Dl, int n1, int n2, int Dr, const double* x, int D_max,
                       double tol, double* P_out, double* SQ_out, int* rank_out,
                       double* discarded_out) {
  if (!c) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(Dl >= 1 && n1 >= 1 && n2 >= 1 && Dr >= 1 && x && P_out && SQ_out && rank_out &&
                   D_max >= 1,
               "a2_svd_split: bad arguments");
    double disc = 0.0;
    const int r = svd_split_dev(c, x, Dl * n1, n2 * Dr, D_max, tol, P_out, SQ_out, &disc);
    A2_CUDA(cudaStreamSynchronize(c->stream));
    *rank_out = r;
    if (discarded_out) *discarded_out = disc;
  });
}

}  // extern "C"

void destroy_owned(a2_ctx* c) {
  std::vector<a2_heff*> hs;
  std::vector<a2_tt*> ts;
  std::vector<a2_mpo*> ms;
  for (auto& hk : handles_owned_by(c)) {
    void* p = const_cast<void*>(hk.first);
    if (hk.second == HK_HEFF) hs.push_back(static_cast<a2_heff*>(p));
    else if (hk.second == HK_TT) ts.push_back(static_cast<a2_tt*>(p));
    else if (hk.second == HK_MPO) ms.push_back(static_cast<a2_mpo*>(p));
  }
  for (auto* h : hs) delete h;     // an H_eff handle refers to its MPO
  for (auto* t : ts) delete t;
  for (auto* m : ms) delete m;
}

// ============================================================================= allocation-free H_eff
// A second way to apply H_eff for callers that must not allocate device memory
// while they run: applications whose device memory is owned by their own pool or
// budget, code that replays fixed work inside latency-critical loops, or callers
// in a process where cudaMalloc is disallowed once set-up is over.  The regular
// entry point grows its intermediate buffers on demand; this one instead uses one
// fixed scratch array compiled into the library.
//
// The scratch array below is a file-scope device array, so every GPU that loads the
// library reserves it until the process exits.  In host code its name is only a
// host-side stand-in for the symbol, never a device address: the real device address
// is looked up with cudaGetSymbolAddress once per device and then passed to the
// kernels.
namespace {

constexpr long long kNoAllocScratchDoubles = 4LL << 20;   // 4 Mi doubles = 32 MiB
static __device__ __align__(256) double g_heff_scratch[kNoAllocScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {};

// Device address of g_heff_scratch on `device` (looked up on first use).
double* scratch_address(int device) {
  A2_REQUIRE(device >= 0 && device < 64, "device index out of range");
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    int cur = -1;
    A2_CUDA(cudaGetDevice(&cur));
    if (cur != device) A2_CUDA(cudaSetDevice(device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_heff_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess || !p)
      throw CudaError(std::string("cudaGetSymbolAddress(g_heff_scratch) failed: ") +
                      cudaGetErrorString(e));
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  return g_scratch_ptr[device];
}

}  // namespace

extern "C" a2_status a2_heff_apply_noalloc(a2_ctx* c, const a2_mpo* m, int k, int Dl, int Dr,
                                           const double* L, const double* R, const double* x,
                                           double* y) {
  if (!c || !m) return A2_EINVAL;
  return guarded(c, [&] {
    A2_REQUIRE(k >= 0 && k + 1 < m->L && Dl >= 1 && Dr >= 1 && L && R && x && y,
               "a2_heff_apply_noalloc: bad arguments");
    const SiteOps& A1 = m->site[k];
    const SiteOps& A2 = m->site[k + 1];
    const int n1 = A1.n, n2 = A2.n, Rl = A1.Rl, R1 = A1.Rr, Rr = A2.Rr;
    const long long s1 = (long long)Dl * Rl * n1 * n2 * Dr;
    const long long s2 = (long long)Dl * R1 * n1 * n2 * Dr;
    const long long s3 = (long long)Dl * n1 * n2 * Rr * Dr;
    const long long need = std::max(s1, s3) + s2;
    if (need > kNoAllocScratchDoubles)
      throw ArgError("a2_heff_apply_noalloc: intermediates need " + std::to_string(need) +
                     " doubles, the fixed scratch holds " +
                     std::to_string(kNoAllocScratchDoubles) +
                     " (use a2_heff_apply for this size)");
    double* T1 = scratch_address(c->device);
    double* T2 = T1 + std::max(s1, s3);
    double* T3 = T1;
    cudaStream_t s = c->stream;
    const long long N1 = (long long)n1 * n2 * Dr;
    {  // S1: T1[(a w)][(t1 t2 b')] = sum_a' L[(a w)][a'] x[a'][(t1 t2 b')]
      SimtGemm<double, double> g;
      g.M = Dl * Rl; g.N = (int)N1; g.K = Dl;
      g.A = L; g.sam = Dl; g.sak = 1;
      g.B = x; g.sbn = 1; g.sbk = N1;
      g.C = T1; g.scm = N1; g.scn = 1;
      simt_gemm(g, s);
    }
    {  // S2: MPO core k on rows (w, t1) -> (w1, s1)
      SparseGeom gm;
      gm.veclen = n2 * Dr;
      gm.in_sw = (long long)n1 * n2 * Dr; gm.in_st = (long long)n2 * Dr;
      gm.out_sw = (long long)n1 * n2 * Dr; gm.out_ss = (long long)n2 * Dr;
      gm.B1 = Dl; gm.in_b1 = (long long)Rl * n1 * n2 * Dr;
      gm.out_b1 = (long long)R1 * n1 * n2 * Dr;
      sparse_rows_apply<double, double, double>(A1.lr.rows<double>(), gm, T1, T2, s);
    }
    {  // S3: MPO core k+1 on rows (w1, t2) -> (w2, s2), batch (a, s1)
      SparseGeom gm;
      gm.veclen = Dr;
      gm.in_sw = (long long)n1 * n2 * Dr; gm.in_st = Dr;
      gm.out_sw = Dr; gm.out_ss = (long long)Rr * Dr;
      gm.B1 = Dl; gm.B2 = n1;
      gm.in_b1 = (long long)R1 * n1 * n2 * Dr; gm.in_b2 = (long long)n2 * Dr;
      gm.out_b1 = (long long)n1 * n2 * Rr * Dr; gm.out_b2 = (long long)n2 * Rr * Dr;
      sparse_rows_apply<double, double, double>(A2.lr.rows<double>(), gm, T2, T3, s);
    }
    {  // S4: y[(a s1 s2)][b] = sum_{(w2 b')} T3[(a s1 s2)][(w2 b')] R[b][(w2 b')]
      SimtGemm<double, double> g;
      g.M = Dl * n1 * n2; g.N = Dr; g.K = Rr * Dr;
      g.A = T3; g.sam = g.K; g.sak = 1;
      g.B = R; g.sbn = g.K; g.sbk = 1;
      g.C = y; g.scm = Dr; g.scn = 1;
      g.splitk = pick_splitk(g.M, g.N, g.K, 64);
      if (g.splitk > 1) {
        g.mode = GEMM_ATOMIC;
        fill_zero(y, sizeof(double) * (size_t)g.M * g.N, s);   // atomics accumulate into y
      }
      simt_gemm(g, s);
    }
  });
}
