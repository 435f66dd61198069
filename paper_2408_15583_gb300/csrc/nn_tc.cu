// Tensor-core GEMM on the fifth-generation tensor cores (tcgen05) for the
// U-Net's contractions whose operands are both K-contiguous:
//   C[m][n] = epilogue(alpha * sum_k A[m][k] * B[n][k])
// (A: activations [M][lda], B: weights [N][ldb], BF16, FP32 accumulation).
//
// One CTA computes a 128 x BN tile (BN = 32, 64, 128 or 256) with eight warps:
//   warp 0 (one lane)  streams 128 x 64 and BN x 64 operand tiles into a
//                      shared-memory ring of up to four stages with TMA
//                      (128-byte swizzle, zero fill outside the matrices);
//   warp 1 (one lane)  issues tcgen05.mma (kind::f16, M = 128, N = BN,
//                      K = 16 per instruction) accumulating in tensor memory
//                      and releases each stage with tcgen05.commit;
//   warp 2             allocates and frees the BN tensor-memory columns;
//   all eight warps    read the accumulator back (tcgen05.ld, 32 rows and
//                      half the columns per warp) into shared memory, then
//                      write coalesced rows through the epilogue (bias,
//                      residual, GELU with the pre-activation copy or GELU',
//                      FP32 or BF16 output).
// Every wait on an mbarrier has an iteration limit; on expiry the kernel sets
// the library's timeout flag, skips its stores, waits (again bounded) for its
// own copies and products still in flight and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstring>

#include "nn_gemm.cuh"
#include "pe_internal.cuh"

namespace {

typedef __nv_bfloat16 bf16;
typedef __nv_bfloat162 bf162;

constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 4, TC_THREADS = 256;
constexpr uint32_t kWaitLimit = 1u << 22;

template <int BN>
struct tc_cfg {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;  // 16 KB, 1024-byte multiple
  static constexpr int B_BYTES = BN * TC_BK * 2;     // 4/8/16/32 KB
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int C_LD = BN + 4;                        // FP32 staging row (floats)
  static constexpr int C_BYTES = TC_BM * C_LD * 4;
  // ring of `stages` operand stages, reused for the FP32 output tile; then
  // the barriers; plus slack to align the base to 1024 bytes
  static int smem(int stages) {
    const int ring = stages * STAGE > C_BYTES ? stages * STAGE : C_BYTES;
    return ((ring + 1023) / 1024) * 1024 + 1024 + 1024;
  }
  // instruction descriptor, kind::f16: D = F32 (bits 4-5), A = B = BF16
  // (bits 7-9, 10-12), both K-major (bits 15, 16 clear), N >> 3 (bits
  // 17-22), M >> 4 (bits 24-28)
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t sm_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte
// swizzle: start address >> 4 (bits 0-13), leading offset 16 B (unused for
// this layout), stride offset 1024 B between 8-row groups (bits 32-45),
// descriptor version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t kmajor_sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sm_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sm_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with the given parity to complete: at most
// `limit` polls (each mbarrier.try_wait may itself suspend the thread for a
// short, system-dependent time); false if the phase has not completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = kWaitLimit) {
  const uint32_t a = sm_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(sm_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sm_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every tcgen05 operation issued so far by this thread
// has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          sm_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 3)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const pe_gemm_args g, int stages, uint32_t wait_limit, unsigned int *err) {
  // wait_limit bounds the waits of the main loop and of the epilogue; the
  // clean-up after a failed wait always waits the full kWaitLimit for the
  // copies and products already issued (they complete in microseconds)
  using cfg = tc_cfg<BN>;
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int ring = stages * cfg::STAGE > cfg::C_BYTES ? stages * cfg::STAGE : cfg::C_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(base + ((ring + 1023) / 1024) * 1024);
  uint64_t *empty = full + TC_STAGES;
  uint64_t *accum = empty + TC_STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int nk = (int)((g.K + TC_BK - 1) / TC_BK);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     sm_u32(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // k-blocks whose loads were issued (producer lane)
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % stages;
      const uint32_t ph = (uint32_t)(kb / stages) & 1u;
      if (!mbar_wait(empty + s, ph ^ 1u, wait_limit)) {
        atomicOr(&s_fail, 1);
        break;
      }
      uint8_t *sa = base + s * cfg::STAGE;
      mbar_expect_tx(full + s, (uint32_t)cfg::STAGE);
      tma_load_2d(sa, &tmA, kb * TC_BK, m0, full + s);
      tma_load_2d(sa + cfg::A_BYTES, &tmB, kb * TC_BK, n0, full + s);
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    int kb = 0;
    for (; kb < nk; ++kb) {
      const int s = kb % stages;
      const uint32_t ph = (uint32_t)(kb / stages) & 1u;
      if (!mbar_wait(full + s, ph, wait_limit)) {
        atomicOr(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t sa = sm_u32(base + s * cfg::STAGE);
      const uint64_t ad = kmajor_sw128_desc(sa), bd = kmajor_sw128_desc(sa + cfg::A_BYTES);
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k)  // +32 bytes per K step inside the swizzled row
        tc_mma(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), cfg::IDESC,
               (kb > 0 || k > 0) ? 1u : 0u);
      tc_commit(empty + s);
    }
    tc_commit(accum);  // all products issued above are complete
  }
  // epilogue: the accumulator goes through shared memory (the operand ring
  // is free once every product has completed), then all threads write
  // coalesced rows.  Warp w reads tensor-memory lanes 32 (w % 4) .. + 31
  // (its rows) for half of the columns.
  const bool ready = mbar_wait(accum, 0u, wait_limit);
  if (!ready) atomicOr(&s_fail, 1);
  tc_fence_after();
  __syncwarp();
  // a warp-uniform decision: tcgen05.ld needs the whole warp
  const bool ok = __all_sync(0xffffffffu, ready && !s_fail);
  float *Cs = reinterpret_cast<float *>(base);
  if (ok) {
    const int quad = warp & 3, half = warp >> 2;
    const int r = quad * 32 + lane;
    const uint32_t row = tmem + ((uint32_t)(quad * 32) << 16);
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 16) {
      float v[16];
      tc_ld16(row + (uint32_t)c, v);
      float4 *dst = reinterpret_cast<float4 *>(Cs + r * cfg::C_LD + c);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        dst[q] = make_float4(v[4 * q] * g.alpha, v[4 * q + 1] * g.alpha, v[4 * q + 2] * g.alpha,
                             v[4 * q + 3] * g.alpha);
    }
  }
  __syncthreads();
  if (!s_fail) {
    for (int c = threadIdx.x; c < TC_BM * BN / 8; c += TC_THREADS) {
      const int r = c / (BN / 8), cc = (c % (BN / 8)) * 8;
      const int m = m0 + r, n = n0 + cc;
      if (m >= g.M || n >= g.N) continue;
      float v[8];
      const float4 a = *reinterpret_cast<const float4 *>(Cs + r * cfg::C_LD + cc);
      const float4 b = *reinterpret_cast<const float4 *>(Cs + r * cfg::C_LD + cc + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      pe_gemm_store8(g, m, n, v);
    }
  }
  __syncthreads();
  if (s_fail) {
    // Let the copies issued by the producer land before the shared memory is
    // released: each issued stage's full barrier completes when its bytes
    // have arrived (bounded wait), and the products were committed above.
    if (threadIdx.x == 0) {
      atomicOr(err, PE_ERR_TIMEOUT);
    }
    if (warp == 0 && lane == 0) {
      for (int kb = (issued > stages ? issued - stages : 0); kb < issued; ++kb)
        mbar_wait(full + kb % stages, (uint32_t)(kb / stages) & 1u);
    }
    if (warp == 1 && lane == 0) mbar_wait(accum, 0u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)BN)
                 : "memory");
  }
}

typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_tiled_fn encoder() {
  static encode_tiled_fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<encode_tiled_fn>(p);
  }
  return fn;
}

// Row-major [rows][ld] BF16 matrix, K = inner extent; box 64 x box_rows,
// 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t K, int64_t ld, int box_rows) {
  encode_tiled_fn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Polls of the kernel's main-loop waits (pe_nn_set_wait_limit).
std::atomic<uint32_t> g_wait_limit{kWaitLimit};

template <int BN>
pe_status launch_bn(const pe_gemm_args &g, cudaStream_t s) {
  using cfg = tc_cfg<BN>;
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, g.M, g.K, g.sam, TC_BM) || !make_map(&mb, g.B, g.N, g.K, g.sbn, BN))
    return PE_EUNSUPPORTED;  // the caller takes the other kernel
  // as many stages as K-blocks, up to four; the shared memory this takes
  // also caps the CTAs per SM so their tensor memory (BN columns each)
  // stays within the SM's 512 columns
  const int nk = (int)((g.K + TC_BK - 1) / TC_BK);
  const int stages = nk < TC_STAGES ? nk : TC_STAGES;
  const int smem = cfg::smem(stages);
  static bool attr = false;
  if (!attr) {
    PE_TRY_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     cfg::smem(TC_STAGES)));
    // the whole unified L1 as shared memory: up to three CTAs of the
    // narrow shapes side by side (registers are capped for three as well)
    PE_TRY_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<BN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    attr = true;
  }
  dim3 grid((unsigned)((g.M + TC_BM - 1) / TC_BM), (unsigned)((g.N + BN - 1) / BN));
  gemm_tc_kernel<BN><<<grid, TC_THREADS, smem, s>>>(ma, mb, g, stages, g_wait_limit.load(),
                                                     pe_err_word());
  PE_TRY_LAUNCH("gemm_tc_kernel");
  return PE_OK;
}

}  // namespace

bool pe_gemm_tc_eligible(const pe_gemm_args &g) {
  auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return g.sak == 1 && g.sbk == 1 && g.sam % 8 == 0 && g.sbn % 8 == 0 && al16(g.A) && al16(g.B) &&
         g.K >= 16 && g.M >= 1 && g.N >= 1 && (int64_t)g.M + TC_BM < (1ll << 31) && encoder();
}

pe_status pe_gemm_tc(const pe_gemm_args &g, cudaStream_t s) {
  if (g.N <= 32) return launch_bn<32>(g, s);
  if (g.N <= 64) return launch_bn<64>(g, s);
  if (g.N <= 128) return launch_bn<128>(g, s);
  return launch_bn<256>(g, s);
}

extern "C" pe_status pe_nn_set_wait_limit(int64_t polls) {
  if (polls > (int64_t)UINT32_MAX) return pe_fail(PE_EINVAL, "pe_nn_set_wait_limit: at most 2^32 - 1");
  g_wait_limit.store(polls < 0 ? kWaitLimit : (uint32_t)polls);
  return PE_OK;
}
