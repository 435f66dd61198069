// Layer kernels of the learned GFB completion network (a8): BF16 activations
// in NHWC layout, FP32 accumulation, FP32 master weights.
//
//   GEMM (tensor cores, mma.sync m16n8k16 BF16 -> FP32) with fused bias,
//   residual, GELU epilogues and deterministic split-K; im2col / col2im for
//   3x3 convolutions; depthwise 7x7; LayerNorm over channels; max-pool 2x2;
//   pixel shuffle x2; channel copies for concatenation; bias / LayerNorm /
//   depthwise weight reductions in a fixed order; the losses of Eq. 17-21 with
//   their gradients; AdamW.
#include <cuda_bf16.h>

#include <cstring>

#include "pe_internal.cuh"
#include "nn_gemm.cuh"

typedef __nv_bfloat16 bf16;
typedef __nv_bfloat162 bf162;

namespace {

__device__ __forceinline__ float b2f(bf16 x) { return __bfloat162float(x); }
__device__ __forceinline__ bf16 f2b(float x) { return __float2bfloat16_rn(x); }

int n_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int grid1(int64_t n, int threads, int per_sm = 16) {
  int64_t b = (n + threads - 1) / threads;
  int64_t cap = (int64_t)n_sms() * per_sm;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// ---------------------------------------------------------------------------
// GEMM
// ---------------------------------------------------------------------------


// Block tile 128 (M) x 64 (N) x 32 (K), eight warps of 32 x 32, a
// three-stage cp.async pipeline; fragments by ldmatrix (transposed for the
// operands whose M or N index is the contiguous one, as in the weight
// gradients).  Shared-memory rows are padded by 16 bytes so the eight row
// addresses of an ldmatrix fall in distinct banks.
constexpr int TM = 128, TN = 64, TK = 32, STAGES = 3, GEMM_THREADS = 256;
constexpr int A_STAGE = TM * (TK + 8);  // >= TK * (TM + 8)
constexpr int B_STAGE = TN * (TK + 8);  // >= TK * (TN + 8)
static_assert(A_STAGE >= TK * (TM + 8) && B_STAGE >= TK * (TN + 8), "stage sizes");
constexpr int GEMM_SMEM = STAGES * (A_STAGE + B_STAGE) * 2;
constexpr int C_LD = TN + 4;  // FP32 staging of the output tile
static_assert(TM * C_LD * 4 <= GEMM_SMEM, "epilogue staging fits the pipeline buffers");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy; bytes < 16 zero-fills the rest (0: all zeros,
// the source is then not read).
__device__ __forceinline__ void cp16(void *dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// Stage one operand tile.  ROWS x TK with K contiguous (KC: S[row][k], row
// stride TK + 8) or TK x ROWS with the row index contiguous (S[k][row], row
// stride ROWS + 8).  X(row, k) = X[row * s_r + k * s_k]; rows >= n_rows and
// k >= k_end read as zero.  vec: 16-byte copies are legal (aligned base,
// contiguous stride 1 and the other stride a multiple of 8 elements).
template <bool KC, int ROWS>
__device__ __forceinline__ void stage_tile(bf16 *S, const bf16 *__restrict__ X, int64_t s_r,
                                           int64_t s_k, int row0, int64_t k0, int n_rows,
                                           int64_t k_end, bool vec) {
  const bf16 zero = f2b(0.0f);
  if (KC) {
    constexpr int CH = ROWS * TK / 8;
    for (int c = threadIdx.x; c < CH; c += GEMM_THREADS) {
      const int r = c >> 2, kc = (c & 3) * 8;
      const int gr = row0 + r;
      const int64_t gk = k0 + kc;
      bf16 *d = S + r * (TK + 8) + kc;
      if (vec) {
        int64_t left = k_end - gk;
        int bytes = (gr < n_rows && left > 0) ? (int)(left >= 8 ? 16 : 2 * left) : 0;
        cp16(d, bytes ? X + (int64_t)gr * s_r + gk : X, bytes);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          d[e] = (gr < n_rows && gk + e < k_end) ? X[(int64_t)gr * s_r + (gk + e) * s_k] : zero;
      }
    }
  } else {
    constexpr int CH = ROWS * TK / 8, PER_K = ROWS / 8;
    for (int c = threadIdx.x; c < CH; c += GEMM_THREADS) {
      const int k = c / PER_K, rc = (c % PER_K) * 8;
      const int64_t gk = k0 + k;
      const int gr = row0 + rc;
      bf16 *d = S + k * (ROWS + 8) + rc;
      if (vec) {
        int left = n_rows - gr;
        int bytes = (gk < k_end && left > 0) ? (left >= 8 ? 16 : 2 * left) : 0;
        cp16(d, bytes ? X + gk * s_k + gr : X, bytes);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          d[e] = (gk < k_end && gr + e < n_rows) ? X[(int64_t)(gr + e) * s_r + gk * s_k] : zero;
      }
    }
  }
}

// C = epilogue(alpha * A B) over one 128 x 64 tile and the K range of split
// blockIdx.z; with split-K the raw products go to part[z][M][N].
template <bool AK, bool BK>
__global__ void __launch_bounds__(GEMM_THREADS, 3) gemm_kernel(const pe_gemm_args g) {
  __shared__ __align__(128) bf16 smem[STAGES * (A_STAGE + B_STAGE)];
  bf16 *As = smem, *Bs = smem + STAGES * A_STAGE;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int64_t kb = (int64_t)blockIdx.z * g.k_per_split;
  int64_t ke = kb + g.k_per_split;
  if (ke > g.K) ke = g.K;
  const int nk = (int)((ke - kb + TK - 1) / TK);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp & 3) * 32, wn = (warp >> 2) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;

  auto load = [&](int st, int kt) {
    if (kt < nk) {
      const int64_t k0 = kb + (int64_t)kt * TK;
      stage_tile<AK, TM>(As + st * A_STAGE, g.A, g.sam, g.sak, m0, k0, g.M, ke, g.vec_a);
      stage_tile<BK, TN>(Bs + st * B_STAGE, g.B, g.sbn, g.sbk, n0, k0, g.N, ke, g.vec_b);
    }
    cp_commit();
  };
#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) load(st, st);
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<STAGES - 2>();
    __syncthreads();
    const bf16 *A = As + (kt % STAGES) * A_STAGE, *B = Bs + (kt % STAGES) * B_STAGE;
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (AK) {
          const int r = wm + 16 * i + (lane & 7) + ((lane >> 3) & 1) * 8;
          ldsm4(a[i], A + r * (TK + 8) + kk + (lane >> 4) * 8);
        } else {
          const int k = kk + (lane >> 4) * 8 + (lane & 7);
          ldsm4t(a[i], A + k * (TM + 8) + wm + 16 * i + ((lane >> 3) & 1) * 8);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        uint32_t r[4];
        if (BK) {
          const int n = wn + 8 * (j + (lane >> 4)) + (lane & 7);
          ldsm4(r, B + n * (TK + 8) + kk + ((lane >> 3) & 1) * 8);
        } else {
          const int q = lane >> 3;
          const int k = kk + (q & 1) * 8 + (lane & 7);
          ldsm4t(r, B + k * (TN + 8) + wn + 8 * (j + (q >> 1)));
        }
        b[j][0] = r[0];
        b[j][1] = r[1];
        b[j + 1][0] = r[2];
        b[j + 1][1] = r[3];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
              "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]),
                "r"(b[j][1]));
    }
    load((kt + STAGES - 1) % STAGES, kt + STAGES - 1);
  }
  cp_wait<0>();
  __syncthreads();
  // stage alpha * acc as FP32 in shared memory, then write rows of eight
  float *Cs = reinterpret_cast<float *>(smem);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = wm + 16 * i + gq + 8 * h, c = wn + 8 * j + 2 * tq;
        *reinterpret_cast<float2 *>(Cs + r * C_LD + c) =
            make_float2(acc[i][j][2 * h] * g.alpha, acc[i][j][2 * h + 1] * g.alpha);
      }
  __syncthreads();
  const bool split = g.part != nullptr;
  for (int c = threadIdx.x; c < TM * TN / 8; c += GEMM_THREADS) {
    const int r = c >> 3, cc = (c & 7) * 8;
    const int m = m0 + r, n = n0 + cc;
    if (m >= g.M || n >= g.N) continue;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = Cs[r * C_LD + cc + e];
    if (split) {
      float *dst = g.part + ((int64_t)blockIdx.z * g.M + m) * g.N + n;
      for (int e = 0; e < 8 && n + e < g.N; ++e) dst[e] = v[e];
      continue;
    }
    pe_gemm_store8(g, m, n, v);
  }
}

// Sum of the split-K partials in a fixed order (lane ty of a (32, 8) block
// takes splits ty, ty + 8, ...; the eight are added in order), then the
// epilogue.
__global__ void gemm_splitk_reduce(const pe_gemm_args g, int split) {
  __shared__ float red[8][33];
  const int64_t total = (int64_t)g.M * g.N;
  const int64_t t = (int64_t)blockIdx.x * 32 + threadIdx.x;
  float v = 0.0f;
  if (t < total)
    for (int z = threadIdx.y; z < split; z += 8) v += g.part[(int64_t)z * total + t];
  red[threadIdx.y][threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.y == 0 && t < total) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
    pe_gemm_store(g, (int)(t / g.N), (int)(t % g.N), s);
  }
}

// ---------------------------------------------------------------------------
// 3x3 convolution helpers (NHWC, zero padding 1): col[p][(ky*3+kx)*C + c]
// ---------------------------------------------------------------------------
// VEC channels per thread: 8 (one 16-byte load and store) when C is a
// multiple of 8 and the buffers are 16-byte aligned, else 1.  The index
// arithmetic runs once per VEC channels.
template <int VEC>
struct chunk_of;
template <>
struct chunk_of<1> {
  using T = bf16;
};
template <>
struct chunk_of<8> {
  using T = uint4;
};

template <int VEC>
__global__ void im2col3_kernel(const bf16 *__restrict__ X, int B, int H, int W, int C,
                               bf16 *__restrict__ col) {
  using T = typename chunk_of<VEC>::T;
  const int CV = C / VEC;
  const T *Xv = reinterpret_cast<const T *>(X);
  T *colv = reinterpret_cast<T *>(col);
  const int64_t total = (int64_t)B * H * W * 9 * CV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int cv = (int)(t % CV);
    const int64_t r = t / CV;
    const int tap = (int)(r % 9);
    const int64_t p = r / 9;
    const int x = (int)(p % W);
    const int64_t q = p / W;
    const int y = (int)(q % H), b = (int)(q / H);
    const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
    T v;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      v = Xv[(((int64_t)b * H + yy) * W + xx) * CV + cv];
    } else {
      memset(&v, 0, sizeof(T));  // bf16 zero is all-zero bits
    }
    colv[t] = v;
  }
}

// dX[b,y,x,c] = sum over taps of dcol at the pixel that read (y, x) through
// that tap (taps in order 0..8, FP32 sums).
template <int VEC>
__global__ void col2im3_kernel(const bf16 *__restrict__ dcol, int B, int H, int W, int C,
                               bf16 *__restrict__ dX) {
  const int CV = C / VEC;
  const int64_t total = (int64_t)B * H * W * CV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int cv = (int)(t % CV);
    const int64_t p = t / CV;
    const int x = (int)(p % W);
    const int64_t q = p / W;
    const int y = (int)(q % H), b = (int)(q / H);
    float s[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) s[k] = 0.0f;
    for (int tap = 0; tap < 9; ++tap) {
      const int py = y - (tap / 3 - 1), px = x - (tap % 3 - 1);
      if (py < 0 || py >= H || px < 0 || px >= W) continue;
      const bf16 *src = dcol + ((((int64_t)b * H + py) * W + px) * 9 + tap) * C + (int64_t)cv * VEC;
      if (VEC == 8) {
        const uint4 u = *reinterpret_cast<const uint4 *>(src);
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int k = 0; k < VEC; ++k) s[k] += b2f(e[k]);
      } else {
        s[0] += b2f(src[0]);
      }
    }
    bf16 *dst = dX + p * C + (int64_t)cv * VEC;
    if (VEC == 8) {
      uint4 u;
      bf16 *e = reinterpret_cast<bf16 *>(&u);
#pragma unroll
      for (int k = 0; k < VEC; ++k) e[k] = f2b(s[k]);
      *reinterpret_cast<uint4 *>(dst) = u;
    } else {
      dst[0] = f2b(s[0]);
    }
  }
}

// ---------------------------------------------------------------------------
// depthwise 7x7 (zero padding 3), weights w[ky][kx][c] FP32; C even, rows of
// channel pairs (bf16x2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 ld2(const bf162 *p) { return __bfloat1622float2(*p); }

// Y = bias + sum_taps w * X (FLIP = 0), or the data gradient dX = sum_taps
// w[6-ky][6-kx] * dY[y+ky-3][x+kx-3] (FLIP = 1, X = dY, no bias).  A thread
// owns one channel pair and eight consecutive pixels of one row; block row y
// = image row (b, y).
template <bool FLIP>
__global__ void __launch_bounds__(256, 4) dw7_kernel(const bf162 *__restrict__ X,
                                                  const float *__restrict__ w,
                                                  const float *__restrict__ bias, int B, int H,
                                                  int W, int C, bf162 *__restrict__ Y) {
  constexpr int NPX = 8;  // pixels per thread
  const int cp2 = C >> 1, groups = (W + NPX - 1) / NPX, per_row = groups * cp2, rows = B * H;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int b = r / H, y = r - b * H;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < per_row; t += gridDim.x * blockDim.x) {
      const int cp = t % cp2, x0 = (t / cp2) * NPX;
      float2 acc[NPX];
      const float2 b0 = bias ? make_float2(bias[2 * cp], bias[2 * cp + 1]) : make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NPX; ++i) acc[i] = b0;
#pragma unroll 1
      for (int ky = 0; ky < 7; ++ky) {
        const int yy = y + ky - 3;
        if (yy < 0 || yy >= H) continue;
        const bf162 *row = X + (size_t)(b * H + yy) * W * cp2 + cp;
        float2 in[NPX + 6];
#pragma unroll
        for (int k = 0; k < NPX + 6; ++k) {
          const int xx = x0 + k - 3;
          in[k] = (xx >= 0 && xx < W) ? ld2(row + (size_t)xx * cp2) : make_float2(0.f, 0.f);
        }
        const int wy = FLIP ? 6 - ky : ky;
#pragma unroll
        for (int kx = 0; kx < 7; ++kx) {
          const int wx = FLIP ? 6 - kx : kx;
          const float2 wv = __ldg(reinterpret_cast<const float2 *>(w + (wy * 7 + wx) * C) + cp);
#pragma unroll
          for (int i = 0; i < NPX; ++i) {
            acc[i].x = fmaf(wv.x, in[i + kx].x, acc[i].x);
            acc[i].y = fmaf(wv.y, in[i + kx].y, acc[i].y);
          }
        }
      }
      bf162 *out = Y + (size_t)r * W * cp2 + cp;
#pragma unroll
      for (int i = 0; i < NPX; ++i)
        if (x0 + i < W) out[(size_t)(x0 + i) * cp2] = __floats2bfloat162_rn(acc[i].x, acc[i].y);
    }
  }
}

// Partial weight/bias gradients: part[chunk][50][C] (tap 49 = bias) with
// chunk = blockIdx.x over image rows r = chunk, chunk + gridDim.x, ...  A
// thread owns channel pair cp and tap row ky and slides a 7-pixel window of X
// along each row, so every load is used by seven taps.
__global__ void dw7_wgrad_kernel(const bf162 *__restrict__ X, const bf162 *__restrict__ dY,
                                 int B, int H, int W, int C, float *__restrict__ part) {
  const int cp2 = C >> 1;
  const int cp = blockIdx.y * blockDim.x + threadIdx.x, ky = threadIdx.y;
  if (cp >= cp2) return;
  float2 acc[7], accb = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 7; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int r = blockIdx.x; r < B * H; r += gridDim.x) {
    const int b = r / H, y = r - b * H, yy = y + ky - 3;
    const bool rowok = yy >= 0 && yy < H;
    if (!rowok && ky != 3) continue;
    const bf162 *g = dY + (size_t)r * W * cp2 + cp;
    const bf162 *xr = X + (size_t)(b * H + (rowok ? yy : y)) * W * cp2 + cp;
    float2 win[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const int xx = k - 3;
      win[k] = (xx >= 0 && xx < W) ? ld2(xr + (size_t)xx * cp2) : make_float2(0.f, 0.f);
    }
    for (int x = 0; x < W; ++x) {
      const float2 gv = ld2(g + (size_t)x * cp2);
      accb.x += gv.x;
      accb.y += gv.y;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        acc[k].x = fmaf(gv.x, win[k].x, acc[k].x);
        acc[k].y = fmaf(gv.y, win[k].y, acc[k].y);
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) win[k] = win[k + 1];
      const int xn = x + 4;
      win[6] = xn < W ? ld2(xr + (size_t)xn * cp2) : make_float2(0.f, 0.f);
    }
  }
  float *pb = part + (size_t)blockIdx.x * 50 * C + 2 * cp;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    pb[(ky * 7 + k) * C] = acc[k].x;
    pb[(ky * 7 + k) * C + 1] = acc[k].y;
  }
  if (ky == 3) {
    pb[49 * C] = accb.x;
    pb[49 * C + 1] = accb.y;
  }
}

// out[i] = (accumulate ? out[i] : 0) + sum over chunks of part[chunk][i],
// i < n, in a fixed order: lane ty of the block sums chunks ty, ty + 8, ...
// and the eight partial sums are added in order.  Block (32, 8).
__global__ void __launch_bounds__(1024) sum_chunks_kernel(const float *part, int chunks,
                                                          int64_t n, float *out,
                                                          int accumulate) {
  // 32 outputs per block, 32 threads per output walking the chunks in a
  // fixed interleave, then their 32 sums in a fixed order (deterministic).
  // out may be part itself (chunk 0 overwritten): a block reads only its own
  // 32 columns, all of them before the barrier, and writes them after it
  // (hence no __restrict__ here).
  __shared__ float red[32][33];
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  float s = 0.0f;
  if (i < n)
    for (int k = threadIdx.y; k < chunks; k += 32) s += part[(int64_t)k * n + i];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && i < n) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) t += red[k][threadIdx.x];
    out[i] = accumulate ? out[i] + t : t;
  }
}

// ---------------------------------------------------------------------------
// LayerNorm over the C channels of each pixel (one warp per pixel)
// ---------------------------------------------------------------------------
__global__ void ln_fwd_kernel(const bf16 *__restrict__ X, const float *__restrict__ gam,
                              const float *__restrict__ bet, int64_t P, int C, float eps,
                              bf16 *__restrict__ Y, float *__restrict__ mean,
                              float *__restrict__ rstd) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
    const bf16 *x = X + p * C;
    float v[8];  // C <= 256: channel lane + 32 i
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = lane + 32 * i;
      v[i] = c < C ? b2f(x[c]) : 0.0f;
      s += v[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mu = s / C;
    float var = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float d = lane + 32 * i < C ? v[i] - mu : 0.0f;
      var += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) var += __shfl_xor_sync(0xffffffffu, var, o);
    const float rs = rsqrtf(var / C + eps);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = lane + 32 * i;
      if (c < C) Y[p * C + c] = f2b((v[i] - mu) * rs * gam[c] + bet[c]);
    }
    if (lane == 0) {
      mean[p] = mu;
      rstd[p] = rs;
    }
  }
}

// LayerNorm for narrow pixels (C a multiple of 8, used for C = 32): one thread per
// pixel, its C channels in registers through 16-byte loads and stores, the
// mean and variance summed in channel order (no shuffles).
template <int C>
__global__ void __launch_bounds__(256) ln_fwd_narrow_kernel(
    const bf16 *__restrict__ X, const float *__restrict__ gam, const float *__restrict__ bet,
    int64_t P, float eps, bf16 *__restrict__ Y, float *__restrict__ mean,
    float *__restrict__ rstd) {
  static_assert(C % 8 == 0 && C <= 64, "narrow LayerNorm: C a multiple of 8, at most 64");
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    float v[C];
    const uint4 *x = reinterpret_cast<const uint4 *>(X + p * C);
#pragma unroll
    for (int k = 0; k < C / 8; ++k) {
      const uint4 u = x[k];
      const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
      for (int m = 0; m < 8; ++m) v[8 * k + m] = b2f(e[m]);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) s += v[c];
    const float mu = s / C;
    float var = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float d = v[c] - mu;
      var += d * d;
    }
    const float rs = rsqrtf(var / C + eps);
    uint4 *y = reinterpret_cast<uint4 *>(Y + p * C);
#pragma unroll
    for (int k = 0; k < C / 8; ++k) {
      uint4 u;
      bf16 *e = reinterpret_cast<bf16 *>(&u);
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int c = 8 * k + m;
        e[m] = f2b((v[c] - mu) * rs * __ldg(gam + c) + __ldg(bet + c));
      }
      y[k] = u;
    }
    mean[p] = mu;
    rstd[p] = rs;
  }
}

// dX and per-warp partials of dgamma, dbeta: part[warp][2][C].
__global__ void __launch_bounds__(256, 4) ln_bwd_kernel(const bf16 *__restrict__ dY, const bf16 *__restrict__ X,
                              const float *__restrict__ gam, const float *__restrict__ mean,
                              const float *__restrict__ rstd, int64_t P, int C,
                              bf16 *__restrict__ dX, float *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  float dg[8], db[8];  // C <= 256
#pragma unroll
  for (int i = 0; i < 8; ++i) dg[i] = db[i] = 0.0f;
  for (int64_t p = gw; p < P; p += warps) {
    const float mu = mean[p], rs = rstd[p];
    float xh[8], gg[8];
    float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int c = lane + 32 * i;
      xh[i] = gg[i] = 0.0f;
      if (c >= C) continue;
      xh[i] = (b2f(X[p * C + c]) - mu) * rs;
      float gy = b2f(dY[p * C + c]);
      gg[i] = gy * gam[c];
      s1 += gg[i];
      s2 += gg[i] * xh[i];
      dg[i] += gy * xh[i];
      db[i] += gy;
    }
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    s1 /= C;
    s2 /= C;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int c = lane + 32 * i;
      if (c < C) dX[p * C + c] = f2b(rs * (gg[i] - s1 - xh[i] * s2));
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int c = lane + 32 * i;
    if (c >= C) break;
    part[(gw * 2 + 0) * C + c] = dg[i];
    part[(gw * 2 + 1) * C + c] = db[i];
  }
}

// Column sums of a [M][ld] BF16 matrix in a fixed order: block (32, 8) owns
// 32 columns (PAIR: 32 column pairs) of chunk blockIdx.y; lane ty sums rows
// r0 + ty, r0 + ty + 8, ...; the eight lanes are added in order into
// part[chunk][N].
template <bool PAIR>
__global__ void colsum_kernel(const bf16 *__restrict__ Xs, int64_t M, int N, int64_t ld,
                              int64_t rows_per_chunk, float *__restrict__ part) {
  __shared__ float2 red[8][33];
  const int c = (blockIdx.x * 32 + threadIdx.x) * (PAIR ? 2 : 1);
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk;
  if (r1 > M) r1 = M;
  float2 s = make_float2(0.f, 0.f);
  if (c < N) {
    for (int64_t r = r0 + threadIdx.y; r < r1; r += 8) {
      if (PAIR) {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const bf162 *>(Xs + r * ld + c));
        s.x += v.x;
        s.y += v.y;
      } else {
        s.x += b2f(Xs[r * ld + c]);
      }
    }
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < N) {
    float2 t = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      t.x += red[k][threadIdx.x].x;
      t.y += red[k][threadIdx.x].y;
    }
    part[(int64_t)blockIdx.y * N + c] = t.x;
    if (PAIR) part[(int64_t)blockIdx.y * N + c + 1] = t.y;
  }
}

// ---------------------------------------------------------------------------
// elementwise
// ---------------------------------------------------------------------------
__global__ void gelu_bwd_kernel(const bf16 *__restrict__ dA, const bf16 *__restrict__ Z, int64_t n,
                                bf16 *__restrict__ dZ) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    dZ[i] = f2b(b2f(dA[i]) * pe_gelu_grad(b2f(Z[i])));
  }
}

__global__ void maxpool2_fwd_kernel(const bf16 *__restrict__ X, int B, int H, int W, int C,
                                    bf16 *__restrict__ Y, uint8_t *__restrict__ arg) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t total = (int64_t)B * Ho * Wo * C;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    int64_t p = t / C;
    int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((int64_t)Wo * Ho));
    float best = -INFINITY;
    int bi = 0;
    for (int k = 0; k < 4; ++k) {
      float v = b2f(X[(((int64_t)b * H + 2 * y + (k >> 1)) * W + 2 * x + (k & 1)) * C + c]);
      if (v > best) {
        best = v;
        bi = k;
      }
    }
    Y[t] = f2b(best);
    arg[t] = (uint8_t)bi;
  }
}

__global__ void maxpool2_bwd_kernel(const bf16 *__restrict__ dY, const uint8_t *__restrict__ arg,
                                    int B, int H, int W, int C, bf16 *__restrict__ dX) {
  const int64_t total = (int64_t)B * H * W * C;
  const int Ho = H / 2, Wo = W / 2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    int64_t p = t / C;
    int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    int64_t q = (((int64_t)b * Ho + y / 2) * Wo + x / 2) * C + c;
    dX[t] = (arg[q] == (uint8_t)(((y & 1) << 1) | (x & 1))) ? dY[q] : f2b(0.0f);
  }
}

// out[b, 2y+i, 2x+j, off + c] = in[b, y, x, 4c + 2i + j]; dir 1: the reverse.
// One thread per pixel (Y, X) of the 2H x 2W image and VEC consecutive
// channels c: the small image's element [b, Y/2, X/2][4c + 2(Y&1) + (X&1)]
// moves to / from the large image's [b, Y, X][off + c] (VEC = 8: the large
// side as one 16-byte access).
template <int VEC>
__global__ void pixel_shuffle2_kernel(const bf16 *__restrict__ src, int B, int H, int W, int C,
                                      bf16 *__restrict__ dst, int64_t ld_big, int off, int dir) {
  const int CV = C / VEC;
  const int W2 = 2 * W, H2 = 2 * H;
  const int64_t total = (int64_t)B * H2 * W2 * CV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c0 = (int)(t % CV) * VEC;
    const int64_t P = t / CV;                 // large-image pixel
    const int X = (int)(P % W2);
    const int64_t q = P / W2;
    const int Y = (int)(q % H2), b = (int)(q / H2);
    const int sub = 2 * (Y & 1) + (X & 1);
    const int64_t small = ((int64_t)b * H + (Y >> 1)) * W + (X >> 1);
    const int64_t sbase = small * 4 * C + 4 * (int64_t)c0 + sub;   // stride 4 over c
    const int64_t bbase = P * ld_big + off + c0;
    if (VEC == 8) {
      if (dir == 0) {
        uint4 u;
        bf16 *e = reinterpret_cast<bf16 *>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) e[k] = src[sbase + 4 * k];
        *reinterpret_cast<uint4 *>(dst + bbase) = u;
      } else {
        const uint4 u = *reinterpret_cast<const uint4 *>(src + bbase);
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) dst[sbase + 4 * k] = e[k];
      }
    } else {
      if (dir == 0)
        dst[bbase] = src[sbase];
      else
        dst[sbase] = src[bbase];
    }
  }
}

// dst[p][doff + c] (=|+=) src[p][soff + c] for c < C; VEC = 8: 16-byte
// chunks (sums per element in FP32, as for VEC = 1).
template <int VEC>
__global__ void copy_channels_kernel(const bf16 *__restrict__ src, int64_t lds, int soff,
                                     bf16 *__restrict__ dst, int64_t ldd, int doff, int64_t P,
                                     int C, int accumulate) {
  const int CV = C / VEC;
  const int64_t total = P * CV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % CV) * VEC;
    const int64_t p = t / CV;
    const bf16 *sp = src + p * lds + soff + c;
    bf16 *d = dst + p * ldd + doff + c;
    if (VEC == 8) {
      uint4 u = *reinterpret_cast<const uint4 *>(sp);
      if (accumulate) {
        const uint4 w = *reinterpret_cast<const uint4 *>(d);
        bf16 *e = reinterpret_cast<bf16 *>(&u);
        const bf16 *f = reinterpret_cast<const bf16 *>(&w);
#pragma unroll
        for (int k = 0; k < 8; ++k) e[k] = f2b(b2f(f[k]) + b2f(e[k]));
      }
      *reinterpret_cast<uint4 *>(d) = u;
    } else {
      const float v = b2f(*sp);
      *d = f2b(accumulate ? b2f(*d) + v : v);
    }
  }
}

// dst[c][r] = src[r][c] (BF16), 32 x 32 tiles through shared memory.
__global__ void transpose_kernel(const bf16 *__restrict__ src, int R, int Cc,
                                 bf16 *__restrict__ dst) {
  __shared__ bf16 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cc) t[i][threadIdx.x] = src[(int64_t)r * Cc + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cc && r < R) dst[(int64_t)c * R + r] = t[threadIdx.x][i];
  }
}

__global__ void f32_to_bf16_kernel(const float *__restrict__ x, int64_t n, bf16 *__restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = f2b(x[i]);
}

__global__ void adamw_kernel(float *__restrict__ p, const float *__restrict__ g,
                             float *__restrict__ m, float *__restrict__ v, bf16 *__restrict__ pb,
                             int64_t n, float lr, float b1, float b2, float eps, float wd,
                             float bc1, float bc2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] * (1.0f - lr * wd) - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    if (pb) pb[i] = f2b(pi);
  }
}

// ---------------------------------------------------------------------------
// Losses of Eq. 17-21 and their gradients.  Outputs are FP32 head outputs:
// depth [P], normal [P][3], mask logit [P].  Ground truth: d_gt [P],
// n_gt [P][3], m_gt [P] (0/1).  counts[0] = hit pixels, [1] = L4 pixels,
// [2] = all pixels (set by loss_count_kernel).
// ---------------------------------------------------------------------------
struct loss_args {
  const float *d, *n, *z, *d_gt, *n_gt, *m_gt;
  int B, H, W;
  float alpha, gamma, w1, w2, w3, w4;
  const float *counts;
  float *g_d, *g_n, *g_z;  // gradients of the total loss
  float *c4u, *c4v;        // per pixel dL4/d(gu), dL4/d(gv) (scratch)
  float *part;             // [blocks][4] loss partial sums
};

__device__ __forceinline__ bool hit_at(const loss_args &a, int b, int y, int x) {
  return a.m_gt[((int64_t)b * a.H + y) * a.W + x] > 0.5f;
}

__device__ __forceinline__ bool l4_valid(const loss_args &a, int b, int y, int x) {
  if (x < 1 || y < 1 || x > a.W - 2 || y > a.H - 2) return false;
  return hit_at(a, b, y, x) && hit_at(a, b, y, x - 1) && hit_at(a, b, y, x + 1) &&
         hit_at(a, b, y - 1, x) && hit_at(a, b, y + 1, x);
}

// f = |a x b| / (|a| |b| + e) with |a x b| = sqrt(|a x b|^2 + 1e-12); returns f
// and df/da.
__device__ __forceinline__ float cross_ratio(const float a[3], const float b[3], float ga[3]) {
  float c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  float cn = sqrtf(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + 1e-12f);
  float na = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  float nb = sqrtf(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  float den = na * nb + 1e-8f;
  float bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
  for (int k = 0; k < 3; ++k)
    ga[k] = (bxc[k] / cn) / den - cn * nb * (na > 0.0f ? a[k] / na : 0.0f) / (den * den);
  return cn / den;
}

// Hit pixels and valid L4 centres, as exact integer counts (cnt zeroed first).
__global__ void loss_count_kernel(const loss_args a, unsigned long long *cnt) {
  const int64_t P = (int64_t)a.B * a.H * a.W;
  unsigned c0 = 0, c1 = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(p % a.W), y = (int)((p / a.W) % a.H), b = (int)(p / ((int64_t)a.W * a.H));
    c0 += hit_at(a, b, y, x) ? 1u : 0u;
    c1 += l4_valid(a, b, y, x) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c0 += __shfl_xor_sync(0xffffffffu, c0, o);
    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd(cnt, (unsigned long long)c0);
    if (c1) atomicAdd(cnt + 1, (unsigned long long)c1);
  }
}

__global__ void loss_count_finish(const unsigned long long *cnt, int64_t P, float *counts) {
  counts[0] = fmaxf((float)cnt[0], 1.0f);
  counts[1] = fmaxf((float)cnt[1], 1.0f);
  counts[2] = (float)P;
}

__device__ __forceinline__ void grads_at(const loss_args &a, const float *d, int b, int y, int x,
                                         float g[3]) {
  const int64_t row = ((int64_t)b * a.H + y) * a.W;
  g[0] = 0.5f * (d[row + x + 1] - d[row + x - 1]);
  g[1] = 0.5f * (d[row + a.W + x] - d[row - a.W + x]);
  g[2] = 1.0f;
}

// Pass 1: per-pixel terms of L1, L2, L3 with their gradients, and the L4
// partials with respect to the centre's (gu, gv).
__global__ void __launch_bounds__(256) loss_pass1_kernel(const loss_args a) {
  __shared__ float red[4][256];
  const int64_t P = (int64_t)a.B * a.H * a.W;
  const float nh = a.counts[0], n4 = a.counts[1], na = a.counts[2];
  float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(p % a.W), y = (int)((p / a.W) % a.H), b = (int)(p / ((int64_t)a.W * a.H));
    const bool hit = a.m_gt[p] > 0.5f;
    // L1
    float gd = 0.0f;
    if (hit) {
      float e = a.d[p] - a.d_gt[p];
      s[0] += e * e / nh;
      gd = a.w1 * 2.0f * e / nh;
    }
    a.g_d[p] = gd;
    // L2
    float gn[3] = {0.0f, 0.0f, 0.0f};
    if (hit) {
      float np_[3] = {a.n[3 * p], a.n[3 * p + 1], a.n[3 * p + 2]};
      float ng[3] = {a.n_gt[3 * p], a.n_gt[3 * p + 1], a.n_gt[3 * p + 2]};
      float ga[3];
      s[1] += cross_ratio(np_, ng, ga) / nh;
      for (int k = 0; k < 3; ++k) gn[k] = a.w2 * ga[k] / nh;
    }
    for (int k = 0; k < 3; ++k) a.g_n[3 * p + k] = gn[k];
    // L3 (focal, alpha-balanced)
    {
      float z = a.z[p];
      float pr = 1.0f / (1.0f + expf(-z));
      float lp = -(fmaxf(-z, 0.0f) + log1pf(expf(-fabsf(z))));   // log p
      float l1p = -(fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))));   // log (1 - p)
      float l, dl;
      if (hit) {
        float q = powf(1.0f - pr, a.gamma);
        l = -a.alpha * q * lp;
        dl = -a.alpha * q * (-a.gamma * pr * lp + (1.0f - pr));
      } else {
        float q = powf(pr, a.gamma);
        l = -(1.0f - a.alpha) * q * l1p;
        dl = -(1.0f - a.alpha) * q * (a.gamma * (1.0f - pr) * l1p - pr);
      }
      s[2] += l / na;
      a.g_z[p] = a.w3 * dl / na;
    }
    // L4 partials at valid centres
    float cu = 0.0f, cv = 0.0f;
    if (l4_valid(a, b, y, x)) {
      float gp[3], gg[3], ga[3];
      grads_at(a, a.d, b, y, x, gp);
      grads_at(a, a.d_gt, b, y, x, gg);
      s[3] += cross_ratio(gp, gg, ga) / n4;
      cu = a.w4 * ga[0] / n4;
      cv = a.w4 * ga[1] / n4;
    }
    a.c4u[p] = cu;
    a.c4v[p] = cv;
  }
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      float t = 0.0f;
      for (int i = 0; i < (int)blockDim.x; ++i) t += red[k][i];
      a.part[blockIdx.x * 4 + k] = t;
    }
  }
}

// Pass 2: scatter the L4 centre partials to the depths they were made of
// (gather form): d(x+1) gets +0.5 cu(x), d(x-1) gets -0.5 cu(x), likewise v.
__global__ void loss_pass2_kernel(const loss_args a) {
  const int64_t P = (int64_t)a.B * a.H * a.W;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(p % a.W), y = (int)((p / a.W) % a.H);
    float g = 0.0f;
    if (x >= 1) g += 0.5f * a.c4u[p - 1];
    if (x <= a.W - 2) g -= 0.5f * a.c4u[p + 1];
    if (y >= 1) g += 0.5f * a.c4v[p - a.W];
    if (y <= a.H - 2) g -= 0.5f * a.c4v[p + a.W];
    a.g_d[p] += g;
  }
}

__global__ void loss_total_kernel(const float *part, int blocks, float w1, float w2, float w3,
                                  float w4, float *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float s[4] = {0, 0, 0, 0};
  for (int b = 0; b < blocks; ++b)
    for (int k = 0; k < 4; ++k) s[k] += part[b * 4 + k];
  out[0] = w1 * s[0] + w2 * s[1] + w3 * s[2] + w4 * s[3];
  for (int k = 0; k < 4; ++k) out[1 + k] = s[k];
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
#define NN_CHECK_STREAM cudaStream_t s = static_cast<cudaStream_t>(stream)

// 0: tcgen05 kernel where it applies (K-contiguous operands, no split-K),
// else the mma.sync kernel; 1: the mma.sync kernel only.
static int g_gemm_path = 0;

extern "C" int32_t pe_nn_gemm_path(int32_t path) {
  const int prev = g_gemm_path;
  if (path == 0 || path == 1) g_gemm_path = path;
  return prev;
}

// Split-K factor: enough blocks for the whole GPU (about 1024, fixed so the
// summation order does not depend on the device), at least 8 K-steps each.
static int64_t gemm_split(int32_t M, int32_t N, int64_t K, int64_t *kps_out) {
  const int64_t tiles = (int64_t)((N + TN - 1) / TN) * ((M + TM - 1) / TM);
  int64_t split = tiles >= 1024 ? 1 : (1024 + tiles - 1) / tiles;
  const int64_t max_split = (K + 8 * TK - 1) / (8 * TK);
  if (split > max_split) split = max_split;
  if (split > 4096) split = 4096;
  if (split < 1) split = 1;
  int64_t kps = (K + split - 1) / split;
  kps = (kps + TK - 1) / TK * TK;
  split = (K + kps - 1) / kps;
  if (kps_out) *kps_out = kps;
  return split;
}

extern "C" size_t pe_nn_gemm_workspace(int32_t M, int32_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  const int64_t split = gemm_split(M, N, K, nullptr);
  if (split <= 1) return 256;
  return (size_t)split * M * N * sizeof(float) + 256;
}

extern "C" pe_status pe_nn_gemm(int32_t M, int32_t N, int64_t K, const void *A, int64_t sam,
                                int64_t sak, const void *B, int64_t sbk, int64_t sbn, void *C,
                                int64_t ldc, int32_t c_f32, const float *bias, const void *R,
                                int64_t ldr, void *Z, int64_t ldz, int32_t gelu, float alpha,
                                float beta, void *ws, size_t ws_bytes, void *stream) {
  NN_CHECK_STREAM;
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || gelu < 0 || gelu > 2 || (gelu == 2 && !Z))
    return pe_fail(PE_EINVAL, "pe_nn_gemm: bad sizes, null operands or gelu mode");
  pe_gemm_args g;
  memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = static_cast<const bf16 *>(A);
  g.sam = sam;
  g.sak = sak;
  g.B = static_cast<const bf16 *>(B);
  g.sbk = sbk;
  g.sbn = sbn;
  g.C = C;
  g.ldc = ldc;
  g.c_f32 = c_f32;
  g.bias = bias;
  g.R = static_cast<const bf16 *>(R);
  g.ldr = ldr;
  g.Z = static_cast<bf16 *>(Z);
  g.ldz = ldz;
  g.gelu = gelu;
  g.alpha = alpha;
  g.beta = beta;
  const bool ak = sak == 1, bk = sbk == 1;
  // 16-byte copies need aligned bases and rows along the contiguous dimension
  auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  g.vec_a = al(A) && (ak ? (sam % 8 == 0) : (sam == 1 && sak % 8 == 0));
  g.vec_b = al(B) && (bk ? (sbn % 8 == 0) : (sbn == 1 && sbk % 8 == 0));
  g.vec_c = al(C) && (c_f32 ? ldc % 4 == 0 : ldc % 8 == 0) && (!R || (al(R) && ldr % 8 == 0)) &&
            (!Z || (al(Z) && ldz % 8 == 0)) && (!bias || (reinterpret_cast<uintptr_t>(bias) & 3) == 0);
  int64_t kps = 0;
  const int64_t split = gemm_split(M, N, K, &kps);
  g.k_per_split = kps;
  if (split > 1) {
    size_t need = (size_t)split * M * N * sizeof(float);
    if (!ws || ws_bytes < need) return pe_fail(PE_ENOMEM, "pe_nn_gemm: workspace needs %zu", need);
    g.part = static_cast<float *>(ws);
  }
  if ((N + TN - 1) / TN > 65535) return pe_fail(PE_EINVAL, "pe_nn_gemm: N too large");
  if (split == 1 && g_gemm_path == 0 && pe_gemm_tc_eligible(g)) {
    const pe_status st = pe_gemm_tc(g, s);
    if (st != PE_EUNSUPPORTED) return st;
  }
  dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN, (unsigned)split);
  if (ak && bk) gemm_kernel<true, true><<<grid, GEMM_THREADS, 0, s>>>(g);
  else if (ak && !bk) gemm_kernel<true, false><<<grid, GEMM_THREADS, 0, s>>>(g);
  else if (!ak && bk) gemm_kernel<false, true><<<grid, GEMM_THREADS, 0, s>>>(g);
  else gemm_kernel<false, false><<<grid, GEMM_THREADS, 0, s>>>(g);
  PE_TRY_LAUNCH("gemm_kernel");
  if (split > 1) {
    const int64_t total = (int64_t)M * N;
    gemm_splitk_reduce<<<(unsigned)((total + 31) / 32), dim3(32, 8), 0, s>>>(g, (int)split);
    PE_TRY_LAUNCH("gemm_splitk_reduce");
  }
  return PE_OK;
}

extern "C" pe_status pe_nn_im2col3(const void *X, int32_t B, int32_t H, int32_t W, int32_t C,
                                   void *col, int32_t backward, void *stream) {
  NN_CHECK_STREAM;
  if (!X || !col || B <= 0 || H <= 0 || W <= 0 || C <= 0)
    return pe_fail(PE_EINVAL, "pe_nn_im2col3: bad arguments");
  const bool v8 = (C % 8) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(col) & 15) == 0;
  const bf16 *x = static_cast<const bf16 *>(X);
  bf16 *y = static_cast<bf16 *>(col);
  if (!backward) {
    const int64_t n = (int64_t)B * H * W * 9 * (v8 ? C / 8 : C);
    if (v8) im2col3_kernel<8><<<grid1(n, 256), 256, 0, s>>>(x, B, H, W, C, y);
    else im2col3_kernel<1><<<grid1(n, 256), 256, 0, s>>>(x, B, H, W, C, y);
    PE_TRY_LAUNCH("im2col3_kernel");
  } else {  // X is dcol [P][9C], col is dX [P][C]
    const int64_t n = (int64_t)B * H * W * (v8 ? C / 8 : C);
    if (v8) col2im3_kernel<8><<<grid1(n, 256), 256, 0, s>>>(x, B, H, W, C, y);
    else col2im3_kernel<1><<<grid1(n, 256), 256, 0, s>>>(x, B, H, W, C, y);
    PE_TRY_LAUNCH("col2im3_kernel");
  }
  return PE_OK;
}

static bool al4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

extern "C" pe_status pe_nn_dwconv7(const void *X, const float *w, const float *bias, int32_t B,
                                   int32_t H, int32_t W, int32_t C, void *Y, void *stream) {
  NN_CHECK_STREAM;
  if (!X || !w || !Y || B <= 0 || H <= 0 || W <= 0 || C <= 0 || (C & 1) || !al4(X) || !al4(Y) ||
      (reinterpret_cast<uintptr_t>(w) & 7))
    return pe_fail(PE_EINVAL, "pe_nn_dwconv7: bad arguments (C even, aligned buffers)");
  const int per_row = ((W + 7) / 8) * (C / 2);
  dim3 grid((per_row + 255) / 256, (unsigned)(B * H < 65535 ? B * H : 65535));
  dw7_kernel<false><<<grid, 256, 0, s>>>(static_cast<const bf162 *>(X), w, bias, B, H, W, C,
                                         static_cast<bf162 *>(Y));
  PE_TRY_LAUNCH("dw7_kernel");
  return PE_OK;
}

// Chunks (image rows per partial) of the weight gradient: fixed by the shape.
static int dw_chunks(int32_t B, int32_t H) {
  int64_t r = (int64_t)B * H;
  return (int)(r < 1024 ? (r < 1 ? 1 : r) : 1024);
}

extern "C" size_t pe_nn_dwconv7_bwd_workspace(int32_t B, int32_t H, int32_t W, int32_t C) {
  (void)W;
  return (size_t)dw_chunks(B, H) * 50 * C * sizeof(float) + 256;
}

// dX (nullable), dw [7][7][C] and db [C] (FP32, overwritten).
extern "C" pe_status pe_nn_dwconv7_bwd(const void *X, const void *dY, const float *w, int32_t B,
                                       int32_t H, int32_t W, int32_t C, void *dX, float *dw,
                                       float *db, void *ws, size_t ws_bytes, void *stream) {
  NN_CHECK_STREAM;
  if (!X || !dY || !w || B <= 0 || H <= 0 || W <= 0 || C <= 0 || (C & 1) || !al4(X) ||
      !al4(dY) || (dX && !al4(dX)) || (reinterpret_cast<uintptr_t>(w) & 7))
    return pe_fail(PE_EINVAL, "pe_nn_dwconv7_bwd: bad arguments (C even, aligned buffers)");
  if (dX) {
    const int per_row = ((W + 7) / 8) * (C / 2);
    dim3 grid((per_row + 255) / 256, (unsigned)(B * H < 65535 ? B * H : 65535));
    dw7_kernel<true><<<grid, 256, 0, s>>>(static_cast<const bf162 *>(dY), w, nullptr, B, H, W, C,
                                          static_cast<bf162 *>(dX));
    PE_TRY_LAUNCH("dw7_kernel");
  }
  if (dw || db) {
    const int chunks = dw_chunks(B, H);
    size_t need = (size_t)chunks * 50 * C * sizeof(float);
    if (!ws || ws_bytes < need) return pe_fail(PE_ENOMEM, "pe_nn_dwconv7_bwd: workspace");
    float *part = static_cast<float *>(ws);
    const int cp2 = C / 2, bx = cp2 < 32 ? cp2 : 32;
    dim3 grid((unsigned)chunks, (unsigned)((cp2 + bx - 1) / bx));
    dw7_wgrad_kernel<<<grid, dim3(bx, 7), 0, s>>>(static_cast<const bf162 *>(X),
                                                  static_cast<const bf162 *>(dY), B, H, W, C, part);
    PE_TRY_LAUNCH("dw7_wgrad_kernel");
    // part[chunk][50][C]: taps 0..48 -> dw, 49 -> db; sum the chunks in
    // order into chunk 0 (a block reads only the columns it writes)
    sum_chunks_kernel<<<(unsigned)((50 * C + 31) / 32), dim3(32, 32), 0, s>>>(part, chunks,
                                                                          50 * (int64_t)C, part, 0);
    PE_TRY_LAUNCH("sum_chunks_kernel");
    if (dw) PE_TRY_CUDA(cudaMemcpyAsync(dw, part, sizeof(float) * 49 * C, cudaMemcpyDeviceToDevice, s));
    if (db)
      PE_TRY_CUDA(cudaMemcpyAsync(db, part + 49 * C, sizeof(float) * C, cudaMemcpyDeviceToDevice, s));
  }
  return PE_OK;
}

extern "C" pe_status pe_nn_layernorm(const void *X, const float *gamma, const float *beta,
                                     int64_t P, int32_t C, float eps, void *Y, float *mean,
                                     float *rstd, void *stream) {
  NN_CHECK_STREAM;
  if (!X || !gamma || !beta || !Y || !mean || !rstd || P <= 0 || C <= 0 || C > 256)
    return pe_fail(PE_EINVAL, "pe_nn_layernorm: bad arguments (C <= 256)");
  const bool al16 = (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  if (al16 && C == 32) {   // (64 channels in registers would cap a thread at 255 registers)
    ln_fwd_narrow_kernel<32><<<grid1(P, 256), 256, 0, s>>>(
        static_cast<const bf16 *>(X), gamma, beta, P, eps, static_cast<bf16 *>(Y), mean, rstd);
    PE_TRY_LAUNCH("ln_fwd_narrow_kernel");
  } else {
    ln_fwd_kernel<<<grid1(P * 32, 256), 256, 0, s>>>(static_cast<const bf16 *>(X), gamma, beta, P,
                                                     C, eps, static_cast<bf16 *>(Y), mean, rstd);
    PE_TRY_LAUNCH("ln_fwd_kernel");
  }
  return PE_OK;
}

extern "C" size_t pe_nn_layernorm_bwd_workspace(int64_t P, int32_t C) {
  int64_t warps = (int64_t)grid1(P * 32, 256) * 8;
  return (size_t)warps * 2 * C * sizeof(float) + 256;
}

// dX and dgamma, dbeta (FP32, overwritten).
extern "C" pe_status pe_nn_layernorm_bwd(const void *dY, const void *X, const float *gamma,
                                         const float *mean, const float *rstd, int64_t P, int32_t C,
                                         void *dX, float *dgamma, float *dbeta, void *ws,
                                         size_t ws_bytes, void *stream) {
  NN_CHECK_STREAM;
  if (!dY || !X || !gamma || !mean || !rstd || !dX || P <= 0 || C <= 0 || C > 256)
    return pe_fail(PE_EINVAL, "pe_nn_layernorm_bwd: bad arguments (C <= 256)");
  int blocks = grid1(P * 32, 256);
  int64_t warps = (int64_t)blocks * 8;
  size_t need = (size_t)warps * 2 * C * sizeof(float);
  if (!ws || ws_bytes < need) return pe_fail(PE_ENOMEM, "pe_nn_layernorm_bwd: workspace");
  float *part = static_cast<float *>(ws);
  ln_bwd_kernel<<<blocks, 256, 0, s>>>(static_cast<const bf16 *>(dY), static_cast<const bf16 *>(X),
                                       gamma, mean, rstd, P, C, static_cast<bf16 *>(dX), part);
  PE_TRY_LAUNCH("ln_bwd_kernel");
  // part[warp][2][C]: sum over warps in order
  sum_chunks_kernel<<<(unsigned)((2 * C + 31) / 32), dim3(32, 32), 0, s>>>(part, (int)warps,
                                                                        2 * (int64_t)C, part, 0);
  PE_TRY_LAUNCH("sum_chunks_kernel");
  if (dgamma) PE_TRY_CUDA(cudaMemcpyAsync(dgamma, part, sizeof(float) * C, cudaMemcpyDeviceToDevice, s));
  if (dbeta) PE_TRY_CUDA(cudaMemcpyAsync(dbeta, part + C, sizeof(float) * C, cudaMemcpyDeviceToDevice, s));
  return PE_OK;
}

// Row chunks of a column sum: fixed by M.
static int64_t colsum_chunks(int64_t M) {
  int64_t c = (M + 255) / 256;
  return c < 1 ? 1 : (c > 1024 ? 1024 : c);
}

extern "C" size_t pe_nn_colsum_workspace(int64_t M, int32_t N) {
  return (size_t)colsum_chunks(M) * N * sizeof(float) + 256;
}

// out[n] = (accumulate ? out[n] : 0) + sum_m X[m * ld + n] (fixed order).
extern "C" pe_status pe_nn_colsum(const void *X, int64_t M, int32_t N, int64_t ld, float *out,
                                  int32_t accumulate, void *ws, size_t ws_bytes, void *stream) {
  NN_CHECK_STREAM;
  if (!X || !out || M <= 0 || N <= 0 || ld < N) return pe_fail(PE_EINVAL, "pe_nn_colsum: bad arguments");
  const int64_t chunks = colsum_chunks(M);
  size_t need = (size_t)chunks * N * sizeof(float);
  if (!ws || ws_bytes < need) return pe_fail(PE_ENOMEM, "pe_nn_colsum: workspace");
  float *part = static_cast<float *>(ws);
  const int64_t rpc = (M + chunks - 1) / chunks;
  const bool pair = (N % 2 == 0) && (ld % 2 == 0) && al4(X);
  const bf16 *x = static_cast<const bf16 *>(X);
  if (pair) {
    colsum_kernel<true><<<dim3((N / 2 + 31) / 32, (unsigned)chunks), dim3(32, 8), 0, s>>>(
        x, M, N, ld, rpc, part);
  } else {
    colsum_kernel<false><<<dim3((N + 31) / 32, (unsigned)chunks), dim3(32, 8), 0, s>>>(
        x, M, N, ld, rpc, part);
  }
  PE_TRY_LAUNCH("colsum_kernel");
  sum_chunks_kernel<<<(unsigned)((N + 31) / 32), dim3(32, 32), 0, s>>>(part, (int)chunks, N, out,
                                                                      accumulate);
  PE_TRY_LAUNCH("sum_chunks_kernel");
  return PE_OK;
}

extern "C" pe_status pe_nn_gelu_bwd(const void *dA, const void *Z, int64_t n, void *dZ,
                                    void *stream) {
  NN_CHECK_STREAM;
  if (!dA || !Z || !dZ || n <= 0) return pe_fail(PE_EINVAL, "pe_nn_gelu_bwd: bad arguments");
  gelu_bwd_kernel<<<grid1(n, 256), 256, 0, s>>>(static_cast<const bf16 *>(dA),
                                                static_cast<const bf16 *>(Z), n,
                                                static_cast<bf16 *>(dZ));
  PE_TRY_LAUNCH("gelu_bwd_kernel");
  return PE_OK;
}

extern "C" pe_status pe_nn_maxpool2(const void *X, int32_t B, int32_t H, int32_t W, int32_t C,
                                    void *Y, uint8_t *arg, int32_t backward, void *stream) {
  NN_CHECK_STREAM;
  if (!X || !Y || !arg || B <= 0 || H < 2 || W < 2 || C <= 0 || (H & 1) || (W & 1))
    return pe_fail(PE_EINVAL, "pe_nn_maxpool2: bad arguments (even H, W)");
  if (!backward) {
    maxpool2_fwd_kernel<<<grid1((int64_t)B * H * W * C / 4, 256), 256, 0, s>>>(
        static_cast<const bf16 *>(X), B, H, W, C, static_cast<bf16 *>(Y), arg);
    PE_TRY_LAUNCH("maxpool2_fwd_kernel");
  } else {  // X = dY (pooled), Y = dX (full)
    maxpool2_bwd_kernel<<<grid1((int64_t)B * H * W * C, 256), 256, 0, s>>>(
        static_cast<const bf16 *>(X), arg, B, H, W, C, static_cast<bf16 *>(Y));
    PE_TRY_LAUNCH("maxpool2_bwd_kernel");
  }
  return PE_OK;
}

// Forward: src [B][H][W][4C] -> dst [B][2H][2W][ld_big] at channel offset off.
// Backward: src = the big gradient, dst = [B][H][W][4C].
extern "C" pe_status pe_nn_pixel_shuffle2(const void *src, int32_t B, int32_t H, int32_t W,
                                          int32_t C, void *dst, int64_t ld_big, int32_t off,
                                          int32_t backward, void *stream) {
  NN_CHECK_STREAM;
  if (!src || !dst || B <= 0 || H <= 0 || W <= 0 || C <= 0 || off < 0 || off + C > ld_big)
    return pe_fail(PE_EINVAL, "pe_nn_pixel_shuffle2: bad arguments");
  {
    const bf16 *big = static_cast<const bf16 *>(backward ? src : dst);
    const bool v8 = C % 8 == 0 && off % 8 == 0 && ld_big % 8 == 0 &&
                    (reinterpret_cast<uintptr_t>(big) & 15) == 0;
    const int64_t n = (int64_t)B * 4 * H * W * (v8 ? C / 8 : C);
    if (v8)
      pixel_shuffle2_kernel<8><<<grid1(n, 256), 256, 0, s>>>(
          static_cast<const bf16 *>(src), B, H, W, C, static_cast<bf16 *>(dst), ld_big, off,
          backward ? 1 : 0);
    else
      pixel_shuffle2_kernel<1><<<grid1(n, 256), 256, 0, s>>>(
          static_cast<const bf16 *>(src), B, H, W, C, static_cast<bf16 *>(dst), ld_big, off,
          backward ? 1 : 0);
  }
  PE_TRY_LAUNCH("pixel_shuffle2_kernel");
  return PE_OK;
}

extern "C" pe_status pe_nn_copy_channels(const void *src, int64_t lds, int32_t soff, void *dst,
                                         int64_t ldd, int32_t doff, int64_t P, int32_t C,
                                         int32_t accumulate, void *stream) {
  NN_CHECK_STREAM;
  if (!src || !dst || P <= 0 || C <= 0) return pe_fail(PE_EINVAL, "pe_nn_copy_channels: bad arguments");
  const bool v8 = C % 8 == 0 && soff % 8 == 0 && doff % 8 == 0 && lds % 8 == 0 && ldd % 8 == 0 &&
                  (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
  if (v8)
    copy_channels_kernel<8><<<grid1(P * (C / 8), 256), 256, 0, s>>>(
        static_cast<const bf16 *>(src), lds, soff, static_cast<bf16 *>(dst), ldd, doff, P, C,
        accumulate);
  else
    copy_channels_kernel<1><<<grid1(P * C, 256), 256, 0, s>>>(
        static_cast<const bf16 *>(src), lds, soff, static_cast<bf16 *>(dst), ldd, doff, P, C,
        accumulate);
  PE_TRY_LAUNCH("copy_channels_kernel");
  return PE_OK;
}

extern "C" pe_status pe_nn_transpose(const void *src, int32_t R, int32_t Cc, void *dst,
                                     void *stream) {
  NN_CHECK_STREAM;
  if (!src || !dst || R <= 0 || Cc <= 0) return pe_fail(PE_EINVAL, "pe_nn_transpose: bad arguments");
  if ((R + 31) / 32 > 65535) return pe_fail(PE_EINVAL, "pe_nn_transpose: too many rows");
  dim3 grid((unsigned)((Cc + 31) / 32), (unsigned)((R + 31) / 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(static_cast<const bf16 *>(src), R, Cc,
                                                static_cast<bf16 *>(dst));
  PE_TRY_LAUNCH("transpose_kernel");
  return PE_OK;
}

extern "C" pe_status pe_nn_to_bf16(const float *x, int64_t n, void *y, void *stream) {
  NN_CHECK_STREAM;
  if (!x || !y || n <= 0) return pe_fail(PE_EINVAL, "pe_nn_to_bf16: bad arguments");
  f32_to_bf16_kernel<<<grid1(n, 256), 256, 0, s>>>(x, n, static_cast<bf16 *>(y));
  PE_TRY_LAUNCH("f32_to_bf16_kernel");
  return PE_OK;
}

extern "C" pe_status pe_nn_adamw(float *p, const float *g, float *m, float *v, void *p_bf16,
                                 int64_t n, float lr, float beta1, float beta2, float eps,
                                 float weight_decay, int32_t step, void *stream) {
  NN_CHECK_STREAM;
  if (!p || !g || !m || !v || n <= 0 || step < 1) return pe_fail(PE_EINVAL, "pe_nn_adamw: bad arguments");
  float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
  adamw_kernel<<<grid1(n, 256), 256, 0, s>>>(p, g, m, v, static_cast<bf16 *>(p_bf16), n, lr, beta1,
                                             beta2, eps, weight_decay, bc1, bc2);
  PE_TRY_LAUNCH("adamw_kernel");
  return PE_OK;
}

static int loss_blocks(int64_t P) { return grid1(P, 256, 4); }

extern "C" size_t pe_nn_unet_losses_workspace(int32_t B, int32_t H, int32_t W) {
  int64_t P = (int64_t)B * H * W;
  return (size_t)(2 * P + 4 * loss_blocks(P) + 8) * sizeof(float) + 1024;
}

// Eq. 17-21: loss[0] = L, loss[1..4] = L1..L4 (device FP32); gradients of L
// with respect to the head outputs (FP32, overwritten).
extern "C" pe_status pe_nn_unet_losses(const float *depth, const float *normal, const float *logit,
                                       const float *d_gt, const float *n_gt, const float *m_gt,
                                       int32_t B, int32_t H, int32_t W, float alpha, float gamma,
                                       const float *lambdas, float *loss, float *g_depth,
                                       float *g_normal, float *g_logit, void *ws, size_t ws_bytes,
                                       void *stream) {
  NN_CHECK_STREAM;
  if (!depth || !normal || !logit || !d_gt || !n_gt || !m_gt || !lambdas || !loss || !g_depth ||
      !g_normal || !g_logit || B <= 0 || H < 3 || W < 3)
    return pe_fail(PE_EINVAL, "pe_nn_unet_losses: bad arguments");
  int64_t P = (int64_t)B * H * W;
  if (!ws || ws_bytes < pe_nn_unet_losses_workspace(B, H, W))
    return pe_fail(PE_ENOMEM, "pe_nn_unet_losses: workspace");
  float *f = static_cast<float *>(ws);
  loss_args a;
  memset(&a, 0, sizeof(a));
  a.d = depth;
  a.n = normal;
  a.z = logit;
  a.d_gt = d_gt;
  a.n_gt = n_gt;
  a.m_gt = m_gt;
  a.B = B;
  a.H = H;
  a.W = W;
  a.alpha = alpha;
  a.gamma = gamma;
  a.w1 = lambdas[0];
  a.w2 = lambdas[1];
  a.w3 = lambdas[2];
  a.w4 = lambdas[3];
  a.g_d = g_depth;
  a.g_n = g_normal;
  a.g_z = g_logit;
  a.c4u = f;
  a.c4v = f + P;
  int blocks = loss_blocks(P);
  a.part = f + 2 * P;
  float *counts = f + 2 * P + 4 * blocks;
  a.counts = counts;
  // two 64-bit counters after the three counts (the offset is a multiple of 8 bytes)
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(counts + 4);
  PE_TRY_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s));
  loss_count_kernel<<<grid1(P, 256), 256, 0, s>>>(a, cnt);
  PE_TRY_LAUNCH("loss_count_kernel");
  loss_count_finish<<<1, 1, 0, s>>>(cnt, P, counts);
  PE_TRY_LAUNCH("loss_count_finish");
  loss_pass1_kernel<<<blocks, 256, 0, s>>>(a);
  PE_TRY_LAUNCH("loss_pass1_kernel");
  loss_pass2_kernel<<<grid1(P, 256), 256, 0, s>>>(a);
  PE_TRY_LAUNCH("loss_pass2_kernel");
  loss_total_kernel<<<1, 32, 0, s>>>(a.part, blocks, a.w1, a.w2, a.w3, a.w4, loss);
  PE_TRY_LAUNCH("loss_total_kernel");
  return PE_OK;
}
