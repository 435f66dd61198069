// GEMM arguments shared by the contraction kernels of the layer library
// (mma.sync path in nn.cu, tcgen05 path in nn_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pointemray.h"

struct pe_gemm_args {
  int M, N;
  int64_t K;
  const __nv_bfloat16 *A;
  int64_t sam, sak;  // element (m, k) at A[m * sam + k * sak]
  const __nv_bfloat16 *B;
  int64_t sbk, sbn;  // element (k, n) at B[k * sbk + n * sbn]
  void *C;
  int64_t ldc;
  int c_f32;
  const float *bias;  // [N] or null
  const __nv_bfloat16 *R;      // residual [M][ldr] or null
  int64_t ldr;
  __nv_bfloat16 *Z;            // pre-activation copy (gelu) or null
  int64_t ldz;
  int gelu;
  float alpha, beta;  // beta applies to an FP32 C only
  float *part;        // split-K partials [split][M][N]
  int64_t k_per_split;
  int vec_a, vec_b;   // 16-byte operand copies are legal
  int vec_c;          // 16-byte epilogue accesses (C, R, Z) are legal
};

// True when both operands are K-contiguous with 16-byte aligned rows and the
// tensor-map encoder is available: the tcgen05 kernel can take the GEMM.
bool pe_gemm_tc_eligible(const pe_gemm_args &g);
// The GEMM on the tcgen05 tensor cores (no split-K).
pe_status pe_gemm_tc(const pe_gemm_args &g, cudaStream_t s);
