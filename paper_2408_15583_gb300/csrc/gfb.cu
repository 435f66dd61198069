// a2/a3: screen-based point-ray intersection (Alg. 1) as a scatter splat.
//
// Alg. 1 gathers, per ray tube, the points within the tube and keeps the one
// nearest the tube's origin.  With every candidate kept (K unbounded) that is
// a minimum over (point, pixel) pairs, so it can be computed by scattering:
// each point visits the pixels its footprint covers, tests the exact ray,
// and lowers the pixel's 64-bit key (float bits of depth << 32 | index) with
// atomicMin.  Depths are positive, so the key order is the depth order and
// ties go to the smaller index: the result does not depend on thread order.
#include "pe_internal.cuh"

namespace {

constexpr int kSplatThreads = 256;

// Surfel (mode 0) or tube (mode 1) test of point c against pixel (i, j).
__device__ __forceinline__ bool splat_test(const pe_view &V, int i, int j, pe_f3 c, pe_f3 n,
                                           float R, int mode, float &depth) {
  pe_f3 o = pe_pixel_origin(V, i, j);
  pe_f3 d = pe_v3(V.d);
  if (mode == 0) {
    pe_f3 x, e;
    return pe_hit_disk(o, d, c, n, R, 0.0f, depth, x, e);
  }
  // tube: distance of c to the central ray below delta, in front, score |c - o|
  pe_f3 q = pe_sub3(c, o);
  float t = pe_dot(q, d);
  pe_f3 x = pe_ray_at(o, t, d);
  pe_f3 e = pe_sub3(x, c);
  if (!(pe_dot(e, e) < pe_mul(R, R))) return false;
  if (!(t > 0.0f)) return false;
  depth = pe_sqrt(pe_dot(q, q));
  return true;
}

// Surfel mode runs in two passes over the points.  Pass 1 splats the disks
// that face the view (n . d <= 0); a tile pass then records, per 8 x 8
// pixel tile, the largest depth among its keys (+inf if a pixel is still
// empty); pass 2 splats the back-facing disks, except those whose nearest
// possible depth (centre depth - R) exceeds that largest depth over every
// tile their footprint touches: every candidate key of such a disk is
// larger than the key already in its pixel, so skipping it changes nothing
// (keys only decrease).  Behind a closed surface that is most back-facing
// disks.  pass 0: every point in one pass (tube mode).
constexpr int kTile = 8;

// A point's footprint on a screen: every pixel whose ray can hit the disk
// lies within R of the centre's projection (an orthographic projection does
// not enlarge a disk); one extra pixel of margin covers rounding.  (Not part
// of the exact test.)  False for a point with no pixel on the screen.
struct footprint {
  pe_f3 c, nn;
  float R, ci, cj, dc;
  int i0, i1, j0, j1;
};

__device__ __forceinline__ bool point_footprint(const pe_view &V, const float *__restrict__ pos,
                                                const float *__restrict__ nrm,
                                                const float *__restrict__ rad, int64_t p,
                                                int mode, float delta, footprint &F) {
  F.c = {__ldg(pos + 3 * p), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2)};
  F.nn = {0.f, 0.f, 0.f};
  if (mode == 0) {
    F.nn = {__ldg(nrm + 3 * p), __ldg(nrm + 3 * p + 1), __ldg(nrm + 3 * p + 2)};
    F.R = __ldg(rad + p);
  } else {
    F.R = delta;
  }
  if (!(F.R >= 0.0f)) return false;
  const float qx = F.c.x - V.o[0], qy = F.c.y - V.o[1], qz = F.c.z - V.o[2];
  const float inv = __fdividef(1.0f, V.pitch);  // (bounds only: 2 ulp is far below their margin)
  F.ci = (qx * V.u[0] + qy * V.u[1] + qz * V.u[2]) * inv + 0.5f * V.W - 0.5f;
  F.cj = (qx * V.v[0] + qy * V.v[1] + qz * V.v[2]) * inv + 0.5f * V.H - 0.5f;
  F.dc = qx * V.d[0] + qy * V.d[1] + qz * V.d[2];
  if (!(fabsf(F.ci) < 1e30f) || !(fabsf(F.cj) < 1e30f)) return false;  // NaN / inf
  const float rp = F.R * inv + 1.0f;
  const float fi0 = fmaxf(floorf(F.ci - rp), 0.0f), fi1 = fminf(ceilf(F.ci + rp), (float)(V.W - 1));
  const float fj0 = fmaxf(floorf(F.cj - rp), 0.0f), fj1 = fminf(ceilf(F.cj + rp), (float)(V.H - 1));
  if (!(fi0 <= fi1) || !(fj0 <= fj1)) return false;
  F.i0 = (int)fi0;
  F.i1 = (int)fi1;
  F.j0 = (int)fj0;
  F.j1 = (int)fj1;
  return true;
}

// Whether this pass splats the point: pass 0 every point; pass 1 disks
// facing the view (n . d <= 0); pass 2 the others, unless hidden: a hit
// point lies within R of c, so its depth is at least the centre's minus R
// (the slack covers the float32 rounding of both depths: pixel origin, hit
// parameter, centre projection), and if that exceeds the largest key depth
// of every tile the footprint touches, no candidate key can win.
__device__ __forceinline__ bool in_pass(const pe_view &V, const footprint &F, int pass,
                                        const float *__restrict__ hv, int tw) {
  if (pass == 0) return true;
  const float facing = F.nn.x * V.d[0] + F.nn.y * V.d[1] + F.nn.z * V.d[2];
  if (pass == 1) return !(facing > 0.0f);
  if (!(facing > 0.0f)) return false;
  const float tmin = F.dc - F.R - 1e-5f * (fabsf(F.dc) + F.R + V.pitch * (float)(V.W + V.H));
  float hmax = -INFINITY;
  for (int ty = F.j0 / kTile; ty <= F.j1 / kTile; ++ty)
    for (int tx = F.i0 / kTile; tx <= F.i1 / kTile; ++tx) hmax = fmaxf(hmax, hv[ty * tw + tx]);
  return !(tmin > hmax);
}

// Every pixel of the footprint whose exact test passes lowers its key;
// n_test / n_hit count the exact tests and the key updates.
__device__ __forceinline__ void splat_point(const pe_view &V, const footprint &F, int64_t p,
                                            int mode, unsigned long long *__restrict__ kv,
                                            long long &n_test, long long &n_hit) {
  // Per row, the columns whose ray can hit: the screen points (a, b)
  // (metres from c's projection along u, v) hitting the disk satisfy
  //   a^2 nw^2 + (a nu + b nv)^2 + b^2 nw^2 <= R^2 nw^2
  // (n in the view frame; the tube is the circle nu = nv = 0, nw = 1),
  // solved for a with R widened far beyond the rounding of the exact test,
  // which still decides every pixel.  Near edge-on disks keep the square.
  const pe_f3 nn = F.nn;
  float nu = 0.0f, nv = 0.0f, nw = 1.0f;
  if (mode == 0) {
    nu = nn.x * V.u[0] + nn.y * V.u[1] + nn.z * V.u[2];
    nv = nn.x * V.v[0] + nn.y * V.v[1] + nn.z * V.v[2];
    nw = -(nn.x * V.d[0] + nn.y * V.d[1] + nn.z * V.d[2]);
  }
  const float inv = __fdividef(1.0f, V.pitch);
  const float Rw = F.R * 1.0001f + 0.02f * V.pitch;
  const float qa = nw * nw + nu * nu;
  const bool rows = qa > 1e-3f;
  for (int j = F.j0; j <= F.j1; ++j) {
    int ia = F.i0, ib = F.i1;
    if (rows) {
      const float b = ((float)j - F.cj) * V.pitch;
      const float qb = 2.0f * b * nu * nv;
      const float qc = b * b * (nw * nw + nv * nv) - Rw * Rw * nw * nw;
      const float disc = qb * qb - 4.0f * qa * qc;
      if (disc < 0.0f) continue;
      // (fast square root and reciprocal: the bounds keep 0.05 px of slack)
      const float sq = disc > 0.0f ? disc * rsqrtf(disc) : 0.0f, inv2a = __fdividef(0.5f, qa);
      const float alo = (-qb - sq) * inv2a, ahi = (-qb + sq) * inv2a;
      ia = max(ia, (int)floorf(F.ci + alo * inv - 0.05f));
      ib = min(ib, (int)ceilf(F.ci + ahi * inv + 0.05f));
    }
    n_test += ib - ia + 1 > 0 ? ib - ia + 1 : 0;
    for (int i = ia; i <= ib; ++i) {
      float depth;
      if (!splat_test(V, i, j, F.c, nn, F.R, mode, depth)) continue;
      ++n_hit;
      unsigned long long key =
          ((unsigned long long)__float_as_uint(depth) << 32) | (unsigned long long)p;
      // the result is unused, so the atomic is a fire-and-forget reduction
      // in L2: the thread does not wait for it (reading the key first to
      // skip losing updates made every covered pixel wait on an L2 round
      // trip)
      atomicMin(kv + (int64_t)j * V.W + i, key);
    }
  }
}

// Each warp examines 32 points at a time and queues, in shared memory, the
// ones this pass splats; whenever 32 are queued its lanes splat one each.
// A pass that keeps a fraction of the points (the facing split, culled or
// off-screen points) thus still keeps every lane busy.
__global__ void __launch_bounds__(kSplatThreads)
    splat_kernel(const __grid_constant__ pe_view_batch vb, const float *__restrict__ pos,
                 const float *__restrict__ nrm, const float *__restrict__ rad, int64_t n,
                 int mode, float delta, int pass, const float *__restrict__ hz,
                 unsigned long long *__restrict__ keys, long long *__restrict__ stats,
                 const uint32_t *__restrict__ order) {
  __shared__ int64_t queue[kSplatThreads / 32][64];
  long long n_test = 0, n_hit = 0;
  const int vi = blockIdx.y;
  const pe_view &V = vb.v[vi];
  unsigned long long *kv = keys + (int64_t)vi * V.W * V.H;
  const int tw = (V.W + kTile - 1) / kTile, th = (V.H + kTile - 1) / kTile;
  const float *hv = hz ? hz + (int64_t)vi * tw * th : nullptr;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  int64_t *q = queue[wq];
  int count = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    // the point this lane examines: the i-th of the processing order (a
    // permutation, or the identity); its key holds its own index either way
    const int64_t i = base + lane;
    const int64_t p = i < n ? (order ? (int64_t)__ldg(order + i) : i) : n;
    footprint F;
    const bool keep = i < n && p < n && point_footprint(V, pos, nrm, rad, p, mode, delta, F) &&
                      in_pass(V, F, pass, hv, tw);
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) q[count + __popc(m & ((1u << lane) - 1u))] = p;
    count += __popc(m);
    __syncwarp();
    if (count >= 32) {
      const int64_t pp = q[lane];
      footprint G;
      point_footprint(V, pos, nrm, rad, pp, mode, delta, G);
      splat_point(V, G, pp, mode, kv, n_test, n_hit);
      __syncwarp();
      if (lane < count - 32) q[lane] = q[lane + 32];
      count -= 32;
      __syncwarp();
    }
  }
  if (lane < count) {
    const int64_t pp = q[lane];
    footprint G;
    point_footprint(V, pos, nrm, rad, pp, mode, delta, G);
    splat_point(V, G, pp, mode, kv, n_test, n_hit);
  }
  if (stats) {  // one atomic per warp and counter
    for (int o = 16; o > 0; o >>= 1) {
      n_test += __shfl_down_sync(0xffffffffu, n_test, o);
      n_hit += __shfl_down_sync(0xffffffffu, n_hit, o);
    }
    if (lane == 0) {
      if (n_test) atomicAdd(reinterpret_cast<unsigned long long *>(stats + 5), (unsigned long long)n_test);
      if (n_hit) atomicAdd(reinterpret_cast<unsigned long long *>(stats + 6), (unsigned long long)n_hit);
    }
  }
}

// hz[v][ty][tx] = the largest depth among the keys of tile (tx, ty) of view
// v, +inf if a pixel of the tile has no key yet.  One warp per 32 x 8
// pixels (four tiles side by side): lanes read coalesced rows.
__global__ void tile_max_kernel(const unsigned long long *__restrict__ keys, int n_views, int W,
                                int H, float *__restrict__ hz) {
  const int tw = (W + kTile - 1) / kTile, th = (H + kTile - 1) / kTile;
  const int gw = (tw + 3) / 4;  // warp groups per tile row
  const int64_t n_warps = (int64_t)n_views * th * gw;
  const int lane = threadIdx.x & 31;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_warps;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int v = (int)(w / ((int64_t)th * gw));
    const int r = (int)(w % ((int64_t)th * gw));
    const int ty = r / gw, gx = r % gw;
    const int i = gx * 32 + lane;
    float m = -INFINITY;
    if (i < W) {
      const unsigned long long *kv = keys + (int64_t)v * W * H;
      for (int jj = 0; jj < kTile; ++jj) {
        const int j = ty * kTile + jj;
        if (j >= H) break;
        const unsigned long long k = kv[(int64_t)j * W + i];
        m = fmaxf(m, k == ~0ull ? INFINITY : __uint_as_float((uint32_t)(k >> 32)));
      }
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    const int tx = gx * 4 + lane / kTile;
    if ((lane & (kTile - 1)) == 0 && tx < tw) hz[((int64_t)v * th + ty) * tw + tx] = m;
  }
}

__global__ void resolve_kernel(const __grid_constant__ pe_view_batch vb,
                               const unsigned long long *__restrict__ keys,
                               const float *__restrict__ nrm, int mode, int64_t per_view,
                               float4 *__restrict__ nd, uint32_t *__restrict__ hit,
                               uint8_t *__restrict__ mask) {
  int64_t total = per_view * vb.n;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long key = keys[g];
    const pe_view &V = vb.v[g / per_view];
    float4 o4 = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
    uint32_t idx = PE_NONE;
    if (key != ~0ull) {
      idx = (uint32_t)(key & 0xffffffffull);
      o4.w = __uint_as_float((uint32_t)(key >> 32));
      if (mode == 0) {
        pe_f3 n = {__ldg(nrm + 3 * (int64_t)idx), __ldg(nrm + 3 * (int64_t)idx + 1),
                   __ldg(nrm + 3 * (int64_t)idx + 2)};
        if (pe_dot(n, pe_v3(V.d)) > 0.0f) n = pe_neg3(n);
        o4.x = n.x;
        o4.y = n.y;
        o4.z = n.z;
      }
    }
    if (nd) nd[g] = o4;
    if (hit) hit[g] = idx;
    if (mask) mask[g] = idx != PE_NONE;
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

size_t pe_splat_tiles(int32_t n_views, int32_t W, int32_t H) {
  return (size_t)n_views * ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
}

pe_status pe_launch_splat(const pe_view_batch &vb, const float *pos, const float *nrm,
                          const float *rad, int64_t n, int mode, float delta, float *hz,
                          unsigned long long *keys, int64_t *stats, cudaStream_t s,
                          const uint32_t *order) {
  long long *st = reinterpret_cast<long long *>(stats);
  if (n <= 0) return PE_OK;
  int64_t blocks_needed = (n + kSplatThreads - 1) / kSplatThreads;
  // enough blocks to fill the GPU across the batch; points loop grid-stride
  int64_t per_view = (int64_t)sm_count() * 8 / (vb.n > 0 ? vb.n : 1);
  if (per_view < 1) per_view = 1;
  int gx = (int)(blocks_needed < per_view ? blocks_needed : per_view);
  dim3 grid(gx, vb.n);
  const bool two = mode == 0 && hz != nullptr;
  pe_event_before("splat_kernel", s);
  splat_kernel<<<grid, kSplatThreads, 0, s>>>(vb, pos, nrm, rad, n, mode, delta, two ? 1 : 0,
                                               nullptr, keys, st, order);
  pe_event_after("splat_kernel", s);
  PE_TRY_LAUNCH("splat_kernel");
  if (two) {
    const int th = (vb.H + kTile - 1) / kTile, gw = ((vb.W + kTile - 1) / kTile + 3) / 4;
    const int64_t warps = (int64_t)vb.n * th * gw;
    int blocks = (int)((warps * 32 + 255) / 256);
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    tile_max_kernel<<<blocks, 256, 0, s>>>(keys, vb.n, vb.W, vb.H, hz);
    PE_TRY_LAUNCH("tile_max_kernel");
    pe_event_before("splat_kernel", s);
    splat_kernel<<<grid, kSplatThreads, 0, s>>>(vb, pos, nrm, rad, n, mode, delta, 2, hz, keys,
                                                 st, order);
    pe_event_after("splat_kernel", s);
    PE_TRY_LAUNCH("splat_kernel");
  }
  return PE_OK;
}

static bool same_size(const pe_view *views, int32_t n) {
  for (int i = 1; i < n; ++i)
    if (views[i].W != views[0].W || views[i].H != views[0].H) return false;
  return true;
}

// Workspace: the keys (unless the caller keeps them), then the tiles of the
// two-pass splat.
extern "C" size_t pe_build_gfb_workspace(int32_t n_views, const pe_view *views) {
  if (n_views < 1 || !views) return 0;
  int64_t tot = 0, tiles = 0;
  for (int i = 0; i < n_views; ++i) {
    tot += (int64_t)views[i].W * views[i].H;
    tiles += (int64_t)((views[i].W + kTile - 1) / kTile) * ((views[i].H + kTile - 1) / kTile);
  }
  pe_carve c{nullptr, 0};
  c.take<unsigned long long>((size_t)tot);
  c.take<float>((size_t)tiles);
  return c.bytes() + 256;
}

extern "C" pe_status pe_build_gfb(const pe_view *views, int32_t n_views, const float *pos,
                                  const float *nrm, const float *rad, int64_t n_points,
                                  int32_t mode, float delta, void *ws, size_t ws_bytes,
                                  float *gfb_nd, uint32_t *gfb_hit, uint8_t *gfb_mask,
                                  uint64_t *keys_out, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!views || n_views < 1 || n_views > PE_MAX_BATCH)
    return pe_fail(PE_EINVAL, "pe_build_gfb: n_views must be in [1, %d]", PE_MAX_BATCH);
  if (!same_size(views, n_views))
    return pe_fail(PE_EINVAL, "pe_build_gfb: all views of a call must share W x H");
  if (views[0].W <= 0 || views[0].H <= 0 || !(views[0].pitch > 0))
    return pe_fail(PE_EINVAL, "pe_build_gfb: bad screen size or pitch");
  if (n_points < 0 || n_points >= (int64_t)PE_NONE)
    return pe_fail(PE_EINVAL, "pe_build_gfb: n_points out of range");
  if (mode != 0 && mode != 1) return pe_fail(PE_EINVAL, "pe_build_gfb: mode must be 0 or 1");
  if (n_points > 0 && (!pos || (mode == 0 && (!nrm || !rad))))
    return pe_fail(PE_EINVAL, "pe_build_gfb: surfel mode needs pos, nrm and rad");
  if (mode == 1 && !(delta > 0)) return pe_fail(PE_EINVAL, "pe_build_gfb: delta must be > 0");
  if (gfb_nd && !pe_aligned(gfb_nd, 16))
    return pe_fail(PE_EINVAL, "pe_build_gfb: gfb_nd must be 16-byte aligned");
  size_t need = pe_build_gfb_workspace(n_views, views);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_build_gfb: workspace needs %zu bytes (256-aligned)", need);

  pe_view_batch vb;
  memset(&vb, 0, sizeof(vb));
  vb.n = n_views;
  vb.W = views[0].W;
  vb.H = views[0].H;
  for (int i = 0; i < n_views; ++i) vb.v[i] = views[i];
  int64_t per_view = (int64_t)vb.W * vb.H;
  pe_carve wc{static_cast<char *>(ws), 0};
  unsigned long long *ws_keys = wc.take<unsigned long long>((size_t)(per_view * n_views));
  float *hz = wc.take<float>(pe_splat_tiles(vb.n, vb.W, vb.H));
  unsigned long long *keys = keys_out ? reinterpret_cast<unsigned long long *>(keys_out) : ws_keys;
  PE_TRY_CUDA(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * per_view * n_views, s));
  pe_status st = pe_launch_splat(vb, pos, nrm, rad, n_points, mode, delta, hz, keys, nullptr, s);
  if (st != PE_OK) return st;
  if (gfb_nd || gfb_hit || gfb_mask) {
    int64_t total = per_view * n_views;
    int blocks = (int)((total + 255) / 256);
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    resolve_kernel<<<blocks, 256, 0, s>>>(vb, keys, nrm, mode, per_view,
                                          reinterpret_cast<float4 *>(gfb_nd), gfb_hit,
                                          gfb_mask);
    PE_TRY_LAUNCH("resolve_kernel");
  }
  return PE_OK;
}
