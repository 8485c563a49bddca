// tcgen05 (5th-generation tensor core) BF16 path of the H_eff contraction.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace a2 {

// True when this build carries the tcgen05 kernels (sm_103a).
bool tc_available();

// y = H_eff x with BF16 operands and FP32 accumulation on tcgen05 (S1, S4) and the
// sparse MPO stages in FP32 (S2, S3).  FP64 L, R, x in; FP64 y out (device).
void tc_heff_apply(cudaStream_t s, int n1, int n2, int Rl, int R1, int Rr, int Dl, int Dr,
                   const double* L, const double* R, const double* x, double* y,
                   const SparseRows<float>& W1, const SparseRows<float>& W2, DevBuf& t1,
                   DevBuf& t2, DevBuf& t3, DevBuf& xa, DevBuf& ya, DevBuf& cb);

}  // namespace a2
