// Shared device/host helpers for the A2DMRG library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <stdexcept>

namespace a2 {

struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};
struct ArgError : std::runtime_error {
  explicit ArgError(const std::string& s) : std::runtime_error(s) {}
};
struct NumericError : std::runtime_error {
  explicit NumericError(const std::string& s) : std::runtime_error(s) {}
};

#define A2_CUDA(expr)                                                              \
  do {                                                                             \
    cudaError_t e__ = (expr);                                                      \
    if (e__ != cudaSuccess)                                                        \
      throw ::a2::CudaError(std::string(#expr) + ": " + cudaGetErrorString(e__) +  \
                            " at " + __FILE__ + ":" + std::to_string(__LINE__));   \
  } while (0)

// Every kernel launch of this library goes through A2_CHECK_LAUNCH, which also counts it.
void count_launch();
long long launch_count();
void count_launches(long long n);     // n launches replayed from a CUDA graph
void set_capturing(bool on);          // this thread is capturing a CUDA graph
#define A2_CHECK_LAUNCH()            \
  do {                               \
    ::a2::count_launch();            \
    A2_CUDA(cudaGetLastError());     \
  } while (0)

#define A2_REQUIRE(cond, msg)                                                      \
  do {                                                                             \
    if (!(cond)) throw ::a2::ArgError(std::string(msg));                           \
  } while (0)

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// The library's stream-ordered memory pool of the current device: memory stays cached
// in the pool (no release at stream synchronisation) and is never handed to another
// stream with an implicit dependency on the freeing stream (the concurrent group
// streams must not serialise through their scratch).
cudaMemPool_t lib_pool();

// Stream-ordered device buffer (allocated from lib_pool()).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t nbytes, cudaStream_t stream) {
    if (nbytes <= bytes && p) return;
    release();
    s = stream;
    size_t nb = nbytes ? nbytes : 16;
    A2_CUDA(cudaMallocFromPoolAsync(&p, nb, lib_pool(), stream));
    bytes = nb;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// ---- live per-kernel-class timing with CUDA events (off unless enabled)
enum ProfKind {
  PK_TC_S1 = 0,      // tcgen05 GEMM, H_eff stage S1 (BF16)
  PK_SPARSE_S2,      // sparse MPO action, H_eff stage S2 (BF16 path)
  PK_SPARSE_S3,      // sparse MPO action, H_eff stage S3 (BF16 path)
  PK_TC_S4,          // tcgen05 GEMM, H_eff stage S4 (BF16)
  PK_HEFF_SIMT,      // whole H_eff application on the SIMT path (FP32/FP64)
  PK_ENV,            // environment update (whole)
  PK_LANCZOS,        // Lanczos vector work (dots, updates, re-orthogonalisation)
  PK_SVD,            // truncated SVD step (Gram + eigensolve + products)
  PK_LQ,             // LQ / QR factorisations
  PK_EMU_S1,         // tcgen05 S1 with FP32-accurate split products (6 BF16 pairs)
  PK_EMU_S2,         // sparse S2 in FP32 (accurate matvec)
  PK_EMU_S3,         // sparse S3 in FP32 with split BF16 output (accurate matvec)
  PK_EMU_S4,         // tcgen05 S4 with split products
  PK_F64E_S1,        // FP64-emulated S1 (Ozaki level products + combine)
  PK_F64E_SPARSE,    // FP64 sparse S2 + S3 of the emulated H_eff
  PK_F64E_S4,        // FP64-emulated S4
  PK_F64E_SPLIT,     // Ozaki slicing of operands
  PK_HEFF_GRAPH,     // H_eff applications replayed from a CUDA graph (all stages)
  PK_COUNT
};
void prof_enable(bool on);
bool prof_enabled();
// Records an event pair around the scope on stream s with algorithmic flops / bytes.
struct ProfScope {
  int idx = -1;
  cudaStream_t s = nullptr;
  ProfScope(int kind, cudaStream_t stream, double flops, double bytes);
  ~ProfScope();
};
// Accumulated totals since the last reset (synchronizes all recorded events).
void prof_read(int kind, long long* launches, double* ms, double* flops, double* bytes);
void prof_reset();

}  // namespace a2
