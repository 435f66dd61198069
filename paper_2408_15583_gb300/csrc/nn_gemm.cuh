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
  int gelu;           // 1: GELU (pre-activation to Z); 2: multiply by GELU'(Z)
  float alpha, beta;  // beta applies to an FP32 C only
  float *part;        // split-K partials [split][M][N]
  int64_t k_per_split;
  int vec_a, vec_b;   // 16-byte operand copies are legal
  int vec_c;          // 16-byte epilogue accesses (C, R, Z) are legal
};

// GELU (exact erf form) and its derivative, for the GEMM epilogues.
__device__ __forceinline__ float pe_gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float pe_gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// Epilogue of one output (m, n): bias, residual, beta * C (FP32 C), GELU
// (mode 1, with the pre-activation to Z) or GELU' (mode 2, Z read), store.
__device__ __forceinline__ void pe_gemm_store(const pe_gemm_args &g, int m, int n, float v) {
  if (m >= g.M || n >= g.N) return;
  if (g.bias) v += g.bias[n];
  if (g.R) v += __bfloat162float(g.R[(int64_t)m * g.ldr + n]);
  if (g.c_f32 && g.beta != 0.0f) v += g.beta * static_cast<float *>(g.C)[(int64_t)m * g.ldc + n];
  if (g.gelu == 1) {
    if (g.Z) g.Z[(int64_t)m * g.ldz + n] = __float2bfloat16_rn(v);
    v = pe_gelu(v);
  } else if (g.gelu == 2) {
    v *= pe_gelu_grad(__bfloat162float(g.Z[(int64_t)m * g.ldz + n]));
  }
  if (g.c_f32)
    static_cast<float *>(g.C)[(int64_t)m * g.ldc + n] = v;
  else
    static_cast<__nv_bfloat16 *>(g.C)[(int64_t)m * g.ldc + n] = __float2bfloat16_rn(v);
}

// Epilogue of the eight outputs (m, n .. n+7) of one row with 16-byte
// accesses when the row has them and the buffers allow it (g.vec_c).
__device__ __forceinline__ void pe_gemm_store8(const pe_gemm_args &g, int m, int n, float (&v)[8]) {
  typedef __nv_bfloat162 bf162;
  if (n + 8 > g.N || !g.vec_c) {
    for (int e = 0; e < 8 && n + e < g.N; ++e) pe_gemm_store(g, m, n + e, v[e]);
    return;
  }
  if (g.bias) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] += __ldg(g.bias + n + e);
  }
  if (g.R) {
    const uint4 rv = *reinterpret_cast<const uint4 *>(g.R + (int64_t)m * g.ldr + n);
    const bf162 *rp = reinterpret_cast<const bf162 *>(&rv);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(rp[e]);
      v[2 * e] += f.x;
      v[2 * e + 1] += f.y;
    }
  }
  if (g.c_f32 && g.beta != 0.0f) {
    const float *cp = static_cast<const float *>(g.C) + (int64_t)m * g.ldc + n;
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] += g.beta * cp[e];
  }
  if (g.gelu == 1) {
    if (g.Z) {
      uint4 zv;
      bf162 *zp = reinterpret_cast<bf162 *>(&zv);
#pragma unroll
      for (int e = 0; e < 4; ++e) zp[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      *reinterpret_cast<uint4 *>(g.Z + (int64_t)m * g.ldz + n) = zv;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = pe_gelu(v[e]);
  } else if (g.gelu == 2) {
    const uint4 zv = *reinterpret_cast<const uint4 *>(g.Z + (int64_t)m * g.ldz + n);
    const bf162 *zp = reinterpret_cast<const bf162 *>(&zv);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 z = __bfloat1622float2(zp[e]);
      v[2 * e] *= pe_gelu_grad(z.x);
      v[2 * e + 1] *= pe_gelu_grad(z.y);
    }
  }
  if (g.c_f32) {
    float4 *cp = reinterpret_cast<float4 *>(static_cast<float *>(g.C) + (int64_t)m * g.ldc + n);
    cp[0] = make_float4(v[0], v[1], v[2], v[3]);
    cp[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    uint4 ov;
    bf162 *op = reinterpret_cast<bf162 *>(&ov);
#pragma unroll
    for (int e = 0; e < 4; ++e) op[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(g.C) + (int64_t)m * g.ldc + n) = ov;
  }
}

// True when both operands are K-contiguous with 16-byte aligned rows and the
// tensor-map encoder is available: the tcgen05 kernel can take the GEMM.
bool pe_gemm_tc_eligible(const pe_gemm_args &g);
// The GEMM on the tcgen05 tensor cores (no split-K).
pe_status pe_gemm_tc(const pe_gemm_args &g, cudaStream_t s);
