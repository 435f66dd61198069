// Unit-throughput probes: the rates that bound the ALU- and atomic-bound
// kernels of the path (the PO term's FMAs and sines, the splat's 64-bit
// atomicMin), plus FP64 and L2-read rates for reference, measured on the
// device in use.  No counterpart in the paper; every loop has a fixed trip
// count and every access stays inside the caller's scratch buffer.
#include "pe_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

// The chains converge to c / (1 - b) = 1 and stay normal; the sum is never
// -1, so the store only keeps the chains from being removed.
__global__ void __launch_bounds__(kProbeThreads) probe_fma32(int n_iter, float b, float c,
                                                             float *sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < n_iter; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) sink[0] = s;
}

// The same chains as probe_fma32, two per packed FP32x2 FMA (__ffma2_rn):
// the issue rate of the paired form the PO kernel's accumulations use.
__global__ void __launch_bounds__(kProbeThreads) probe_fma32x2(int n_iter, float b, float c,
                                                               float *sink) {
  float2 a[kChains];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x + k) * 2e-3f);
  for (int i = 0; i < n_iter; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == -1.0f) sink[0] = s;
}

// x <- sin(x) from x in [1, 1.8): positive, decreasing like sqrt(3 / i),
// far from the denormal range for any trip count used here.
__global__ void __launch_bounds__(kProbeThreads) probe_sin(int n_iter, float *sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 0.1f * (float)k + 1e-6f * (float)threadIdx.x;
  for (int i = 0; i < n_iter; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __sinf(a[k]);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_fma64(int n_iter, double b, double c,
                                                             double *sink) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < n_iter; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0) sink[0] = s;
}

// n_iter passes over nvec float4 (kept in L2, not L1: ld.global.cg); four
// independent sums.  The caller zeroes the buffer, so the sum is never -1.
__global__ void __launch_bounds__(kProbeThreads) probe_l2_read(const float4 *__restrict__ p,
                                                               int64_t nvec, int n_iter,
                                                               float *sink) {
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int it = 0; it < n_iter; ++it)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride) {
      const float4 v = __ldcg(p + i);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  if ((acc.x + acc.y) + (acc.z + acc.w) == -1.0f) sink[0] = acc.x;
}

// A 32-bit integer mixer (xor-shift / multiply rounds) spreading the
// atomics over the table.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// n_iter 64-bit atomicMin per thread into a power-of-two table, result
// unused (the fire-and-forget form the splat issues).
__global__ void __launch_bounds__(kProbeThreads) probe_atomic_min64(unsigned long long *w,
                                                                    uint32_t mask, int n_iter) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = 0; i < n_iter; ++i) {
    const uint32_t h = mix32(t * 0x9e3779b9u + (uint32_t)i);
    atomicMin(w + (h & mask), ((unsigned long long)h << 8) | (unsigned long long)(i & 0xff));
  }
}

}  // namespace

extern "C" int64_t pe_probe_units(int32_t kind, int32_t blocks, int32_t n_iter, void *scratch,
                                  size_t scratch_bytes, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (kind < 0 || kind > 5) {
    pe_fail(PE_EINVAL, "pe_probe_units: kind in [0, 5]");
    return -1;
  }
  if (blocks < 1 || blocks > (1 << 20) || n_iter < 1 || n_iter > (1 << 24)) {
    pe_fail(PE_EINVAL, "pe_probe_units: blocks in [1, 2^20], n_iter in [1, 2^24]");
    return -1;
  }
  if (!scratch || scratch_bytes < 4096 || !pe_aligned(scratch, 256)) {
    pe_fail(PE_EINVAL, "pe_probe_units: scratch of at least 4096 bytes, 256-byte aligned");
    return -1;
  }
  const int64_t threads = (int64_t)blocks * kProbeThreads;
  int64_t ops = 0;
  switch (kind) {
    case 0:
      probe_fma32<<<blocks, kProbeThreads, 0, s>>>(n_iter, 0.9999f, 1e-4f,
                                                   static_cast<float *>(scratch));
      ops = threads * n_iter * kChains * 2;  // flops (an FMA is 2)
      break;
    case 1:
      probe_sin<<<blocks, kProbeThreads, 0, s>>>(n_iter, static_cast<float *>(scratch));
      ops = threads * n_iter * kChains;  // sines
      break;
    case 2:
      probe_fma64<<<blocks, kProbeThreads, 0, s>>>(n_iter, 0.9999, 1e-4,
                                                   static_cast<double *>(scratch));
      ops = threads * n_iter * kChains * 2;  // flops
      break;
    case 3: {
      const int64_t nvec = (int64_t)(scratch_bytes / 16) - 1;  // the last 16 bytes: sink
      probe_l2_read<<<blocks, kProbeThreads, 0, s>>>(
          static_cast<const float4 *>(scratch), nvec, n_iter,
          reinterpret_cast<float *>(static_cast<char *>(scratch) + nvec * 16));
      ops = nvec * 16 * (int64_t)n_iter;  // bytes read
      break;
    }
    case 4: {
      uint64_t words = 1;
      while (words * 2 <= scratch_bytes / 8 && words * 2 <= (1ull << 31)) words *= 2;
      probe_atomic_min64<<<blocks, kProbeThreads, 0, s>>>(
          static_cast<unsigned long long *>(scratch), (uint32_t)(words - 1), n_iter);
      ops = threads * n_iter;  // atomics
      break;
    }
    case 5:
      probe_fma32x2<<<blocks, kProbeThreads, 0, s>>>(n_iter, 0.9999f, 1e-4f,
                                                     static_cast<float *>(scratch));
      ops = threads * n_iter * kChains * 4;  // flops (two FMAs per instruction)
      break;
  }
  cudaError_t e = cudaGetLastError();
  pe_count_launch();
  if (e != cudaSuccess) {
    pe_fail(PE_ECUDA, "pe_probe_units: %s", cudaGetErrorString(e));
    return -1;
  }
  return ops;
}
