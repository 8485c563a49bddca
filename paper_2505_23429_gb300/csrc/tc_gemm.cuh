// tcgen05 (5th-generation tensor core) BF16 path of the H_eff contraction.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace a2 {

// True when this build carries the tcgen05 kernels (sm_103a).
bool tc_available();
// Device error flag of the tcgen05 kernels (nonzero: a bounded wait gave up).
int tc_error_flag(bool reset);
// Runs one GEMM unit whose producer issues no copies, so that a bounded wait runs out;
// returns the device error code it raised (and clears it).  Synchronous.
int tc_selftest_timeout(cudaStream_t s);

// C[m][n] (=|+=atomic) sum_k A[m][k] B[n][k]; A: M x K (row stride lda), B: N x K
// (row stride ldb), both BF16 with 16-byte aligned bases and row strides that are
// multiples of 8 elements.  out_kind: 0 = BF16 store, 1 = FP32 store, 2 = FP32 atomic
// add (required when splitk > 1; C must be zeroed by the caller — the autotuner
// re-zeroes it between its trials).  splitk is a hint the autotuner may change.
void tc_gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb,
                  int M, int N, int K, void* C, long long ldc, int out_kind, int splitk,
                  cudaStream_t s);

// Optional second K segment of a GEMM with M = Dl*n12 rows (a, s12) and N = Nb columns b:
//   C[(a s12)][b] += sum_{w1, b'} A2[a][w1][s12][b'] * B2[b][w1][b'],
// A2 dense [Dl][R1][n12][Dr], B2 dense [Nb][R1][Dr] (BF16 planes; Dr % 8 == 0,
// 128 % n12 == 0, 16-byte aligned bases).  It folds an identity-on-physical MPO block
// into the right environment (B2) of the last stage of H_eff.
struct TcSeg2 {
  const __nv_bfloat16* A[3] = {nullptr, nullptr, nullptr};
  const __nv_bfloat16* B[3] = {nullptr, nullptr, nullptr};
  int Dl = 0, n12 = 0, R1 = 0, Dr = 0, Nb = 0;
};

// Same GEMM accumulating npairs operand pairs (A[pa[p]], B[pb[p]]) into one FP32 tile:
// with A = A0 + A1 + A2 and B = B0 + B1 + B2 split into BF16 planes, the six pairs
// (0,0) (0,1) (1,0) (0,2) (1,1) (2,0) reproduce the FP32 product to ~2^-24.  With seg,
// the second K segment is accumulated into the same tile with the same pairs.
void tc_gemm_bf16_pairs(const __nv_bfloat16* const* A, long long lda,
                        const __nv_bfloat16* const* B, long long ldb, int M, int N, int K,
                        int npairs, const int* pa, const int* pb, void* C, long long ldc,
                        int out_kind, int splitk, cudaStream_t s, const TcSeg2* seg = nullptr);

// Identity-on-physical MPO blocks folded into the environments (W = I (x) G + W_rest):
// Lt [(a w1)][a'] (row stride = that of L) when A_k is folded, Rt [b][w1][b'] (dense)
// when A_{k+1} is folded; BF16 planes as for L / R.  The sparse stages then get W_rest.
struct HeffFold {
  const __nv_bfloat16* Lt = nullptr;
  const __nv_bfloat16* Rt = nullptr;
  long long ltplane = 0, rtplane = 0;
};

// y = H_eff x: BF16 environments Lb [(a w)][a'] (row stride ldl) and Rb [b][(w2 b')]
// (row stride ldr), FP64 x in, FP32 y out; intermediates T1..T3 in BF16 with FP32
// accumulation inside each stage.
void tc_heff_bf16(cudaStream_t s, int n1, int n2, int Rl, int R1, int Rr, int Dl, int Dr,
                  const __nv_bfloat16* Lb, long long ldl, const __nv_bfloat16* Rb, long long ldr,
                  const double* x, float* y, const SparseRows<float>& W1,
                  const SparseRows<float>& W2, const HeffFold& F, DevBuf& t1, DevBuf& t2,
                  DevBuf& xa, DevBuf& tf);

// y = H_eff x with FP32-accurate tensor-core products (three BF16 planes per operand,
// six plane pairs per GEMM); L / R given as three BF16 planes each.
void tc_heff_f32emu(cudaStream_t s, int n1, int n2, int Rl, int R1, int Rr, int Dl, int Dr,
                    const __nv_bfloat16* Lp, long long ldl, long long lplane,
                    const __nv_bfloat16* Rp, long long ldr, long long rplane, const double* x,
                    float* y, const SparseRows<float>& W1, const SparseRows<float>& W2,
                    const HeffFold& F, DevBuf& t1, DevBuf& t2, DevBuf& xa, DevBuf& tf);

// One-site H_eff y[a,s,b] = sum L[a,w,a'] W[w,s,t,w'] R[b,w',b'] x[a',t,b'] with
// FP32-accurate tensor-core products; L / R as three BF16 planes (layouts as for the
// two-site chain), W the left-to-right rows of the core, FP64 x in, FP32 y out.
void tc_heff1_f32emu(cudaStream_t s, int n, int Rl, int Rr, int Dl, int Dr,
                     const __nv_bfloat16* Lp, long long ldl, long long lplane,
                     const __nv_bfloat16* Rp, long long ldr, long long rplane, const double* x,
                     float* y, const SparseRows<float>& W, DevBuf& t1, DevBuf& t2, DevBuf& xa);

// FP64 emulation (Ozaki scheme with BF16 slices, see tc_gemm.cu).
constexpr int kOzSlices = 8;   // slices per FP64 operand
constexpr int kOzBits = 7;     // bits per slice
// Split the FP64 matrix X (element (r, k) at X[r*sr + k*sk], rows x K) into kOzSlices BF16
// planes P + i*plane, row r at P + i*plane + r*ldp (ldp % 8 == 0, 16-byte aligned P).
void ozaki_split(const double* X, long long sr, long long sk, int rows, int K, __nv_bfloat16* P,
                 long long ldp, long long plane, cudaStream_t s);
// The same slices for the rows of X^T, X a (K x N) row-major FP64 matrix with row stride
// ldx (output row n holds X[k][n]): no transposed copy of X is needed.
void ozaki_split_cols(const double* X, long long ldx, int N, int K, __nv_bfloat16* P,
                      long long ldp, long long plane, cudaStream_t s);
// C (FP64, M x N, row stride ldc) = sum_k A[m][k] B[n][k] to FP64 accuracy from the split
// planes of A (row stride lda, plane stride aplane) and B; slab is FP32 scratch for the
// double-float partial sums of the K splits, when the product is split (grown as
// needed).  With Cdf set the result is written as an FP32 pair instead (Cdf + r*ldc + c
// and the same at + df_plane), C unused.
void tc_gemm_f64emu(const __nv_bfloat16* A, long long lda, long long aplane,
                    const __nv_bfloat16* B, long long ldb, long long bplane, int M, int N, int K,
                    double* C, long long ldc, DevBuf& slab, cudaStream_t s,
                    float* Cdf = nullptr, long long df_plane = 0);

// Enable (default) or disable the GEMM autotuner (disabling also forgets its choices).
void tc_autotune(bool on);

inline long long pad8(long long x) { return (x + 7) / 8 * 8; }

}  // namespace a2
