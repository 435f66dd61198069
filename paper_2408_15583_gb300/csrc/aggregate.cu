// a4: GFB aggregation (Alg. 3, aggregation steps): edge filter, voxel fusion, Eq. 22
// splat radius, owner-pixel placement, and the bounding pyramids the march
// uses in place of the paper's splat acceleration structure.
//
// Fusion is a counting sort on a dense G^3 voxel grid (G <= 256): count
// contributors per voxel, exclusive scan, scatter pixel keys into voxel
// segments, then one thread per segment orders its keys by (view, pixel) and
// sums in FP64 in that order -- the same order as a sort by
// (voxel, view, pixel), so the result is bit-identical whatever the atomic
// order of the scatter.
#include <cstring>

#include "pe_internal.cuh"

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kSegLocal = 64;

__device__ __forceinline__ int view_of(const pe_geom_layout &L, int64_t g) {
  int v = 0;
  while (v + 1 < L.nv && g >= L.pix_off[v + 1]) ++v;
  return v;
}

// ---- Canny edges of the views' depth maps (edge mode 1) --------------------
// The same arithmetic, in the same order, as the reference statement: 5x5
// binomial smoothing over valid pixels (absent samples take the centre's
// depth), Sobel on the smoothed map, suppression across the gradient's
// sector, thresholds 8 tau L and half of it, hysteresis over 8 neighbours.
__device__ __forceinline__ bool canny_in(const pe_geom_layout &L, const uint8_t *mask, int64_t off,
                                         const pe_view &V, int i, int j) {
  return i >= 0 && j >= 0 && i < V.W && j < V.H && mask[off + (int64_t)j * V.W + i];
}

__global__ void canny_smooth_kernel(const __grid_constant__ pe_geom_layout L,
                                    const float4 *__restrict__ nd,
                                    const uint8_t *__restrict__ mask, float *__restrict__ S) {
  const int64_t total = L.pix_off[L.nv];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[g]) continue;
    const int v = view_of(L, g);
    const pe_view &V = L.view[v];
    const int64_t off = L.pix_off[v], p = g - off;
    const int i = (int)(p % V.W), j = (int)(p / V.W);
    const float t = nd[g].w;
    const int b[5] = {1, 4, 6, 4, 1};
    float acc = 0.0f;
    for (int dj = -2; dj <= 2; ++dj)
      for (int di = -2; di <= 2; ++di) {
        const float dq = canny_in(L, mask, off, V, i + di, j + dj)
                             ? nd[off + (int64_t)(j + dj) * V.W + (i + di)].w
                             : t;
        const float w = pe_div((float)(b[dj + 2] * b[di + 2]), 256.0f);
        acc = pe_add(acc, pe_mul(w, dq));
      }
    S[g] = acc;
  }
}

__global__ void canny_grad_kernel(const __grid_constant__ pe_geom_layout L,
                                  const uint8_t *__restrict__ mask, const float *__restrict__ S,
                                  float *__restrict__ Gm, uint8_t *__restrict__ sec) {
  const int64_t total = L.pix_off[L.nv];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[g]) continue;
    const int v = view_of(L, g);
    const pe_view &V = L.view[v];
    const int64_t off = L.pix_off[v], p = g - off;
    const int i = (int)(p % V.W), j = (int)(p / V.W);
    auto cs = [&](int di, int dj) -> float {
      return canny_in(L, mask, off, V, i + di, j + dj) ? S[off + (int64_t)(j + dj) * V.W + (i + di)]
                                                        : S[g];
    };
    const float gx = pe_add(pe_add(pe_sub(cs(1, -1), cs(-1, -1)), pe_mul(2.0f, pe_sub(cs(1, 0), cs(-1, 0)))),
                            pe_sub(cs(1, 1), cs(-1, 1)));
    const float gy = pe_add(pe_add(pe_sub(cs(-1, 1), cs(-1, -1)), pe_mul(2.0f, pe_sub(cs(0, 1), cs(0, -1)))),
                            pe_sub(cs(1, 1), cs(1, -1)));
    Gm[g] = pe_sqrt(pe_add(pe_mul(gx, gx), pe_mul(gy, gy)));
    const float ax = fabsf(gx), ay = fabsf(gy);
    uint8_t sc;
    if (ay <= pe_mul(0.41421356f, ax)) sc = 0;
    else if (ay >= pe_mul(2.41421356f, ax)) sc = 2;
    else sc = ((gx > 0.0f) == (gy > 0.0f)) ? 1 : 3;
    sec[g] = sc;
  }
}

__global__ void canny_nms_kernel(const __grid_constant__ pe_geom_layout L,
                                 const uint8_t *__restrict__ mask, const float *__restrict__ Gm,
                                 const uint8_t *__restrict__ sec, float tau,
                                 uint8_t *__restrict__ state) {
  const int64_t total = L.pix_off[L.nv];
  const int nx[4] = {1, 1, 0, 1}, ny[4] = {0, 1, 1, -1};
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint8_t st = 0;
    if (mask[g]) {
      const int v = view_of(L, g);
      const pe_view &V = L.view[v];
      const int64_t off = L.pix_off[v], p = g - off;
      const int i = (int)(p % V.W), j = (int)(p / V.W);
      const int a = sec[g];
      const float gm = Gm[g];
      const float g1 = canny_in(L, mask, off, V, i + nx[a], j + ny[a])
                           ? Gm[off + (int64_t)(j + ny[a]) * V.W + (i + nx[a])] : 0.0f;
      const float g2 = canny_in(L, mask, off, V, i - nx[a], j - ny[a])
                           ? Gm[off + (int64_t)(j - ny[a]) * V.W + (i - nx[a])] : 0.0f;
      if (gm > 0.0f && gm >= g1 && gm >= g2) {
        const float high = pe_mul(pe_mul(8.0f, tau), V.pitch), low = pe_mul(0.5f, high);
        st = gm >= high ? 2 : (gm >= low ? 1 : 0);
      }
    }
    state[g] = st;
  }
}

// One hysteresis pass: a weak pixel with a strong 8-neighbour becomes strong.
// Passes repeat until none changes; the fixed point is the set of weak pixels
// connected to a strong one, whatever the order of the updates.
__global__ void canny_hyst_kernel(const __grid_constant__ pe_geom_layout L,
                                  uint8_t *__restrict__ state, unsigned int *changed) {
  const int64_t total = L.pix_off[L.nv];
  unsigned int ch = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (state[g] != 1) continue;
    const int v = view_of(L, g);
    const pe_view &V = L.view[v];
    const int64_t off = L.pix_off[v], p = g - off;
    const int i = (int)(p % V.W), j = (int)(p / V.W);
    bool up = false;
    for (int dj = -1; dj <= 1 && !up; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || jj < 0 || ii >= V.W || jj >= V.H) continue;
        if (state[off + (int64_t)jj * V.W + ii] == 2) {
          up = true;
          break;
        }
      }
    if (up) {
      state[g] = 2;
      ++ch;
    }
  }
  if (ch) atomicAdd(changed, ch);
}

// Edge rule + voxel of the pixel's surface point; counts contributors.
__global__ void fuse_classify_kernel(const __grid_constant__ pe_geom_layout L,
                                     const float4 *__restrict__ nd,
                                     const uint8_t *__restrict__ mask, float tau,
                                     const uint8_t *__restrict__ canny_state,
                                     float bx, float by, float bz, float inv_vox, int G,
                                     uint32_t *__restrict__ vox_of, uint32_t *__restrict__ count) {
  int64_t total = L.pix_off[L.nv];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t vox = PE_NONE;
    if (mask[g]) {
      int v = view_of(L, g);
      const pe_view &V = L.view[v];
      int64_t off = L.pix_off[v], p = g - off;
      int i = (int)(p % V.W), j = (int)(p / V.W);
      float t = nd[g].w;
      // edge mode 1: Canny edges replace the depth-jump part of the rule
      float tauL = canny_state ? INFINITY : pe_mul(tau, V.pitch);
      bool edge = canny_state && canny_state[g] == 2;
      const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int ii = i + di[k], jj = j + dj[k];
        if (ii < 0 || jj < 0 || ii >= V.W || jj >= V.H) {
          edge = true;
          continue;
        }
        int64_t q = off + (int64_t)jj * V.W + ii;
        if (!mask[q]) {
          edge = true;
          continue;
        }
        float dt = fabsf(pe_sub(nd[q].w, t));
        if (dt > tauL) edge = true;
      }
      if (!edge) {
        pe_f3 o = pe_pixel_origin(V, i, j);
        pe_f3 x = pe_ray_at(o, t, pe_v3(V.d));
        float f[3] = {pe_mul(pe_sub(x.x, bx), inv_vox), pe_mul(pe_sub(x.y, by), inv_vox),
                      pe_mul(pe_sub(x.z, bz), inv_vox)};
        int ix[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float c = floorf(fminf(fmaxf(f[k], -1.0f), (float)G));
          int ci = (int)c;
          ix[k] = ci < 0 ? 0 : (ci > G - 1 ? G - 1 : ci);
        }
        vox = (uint32_t)((ix[0] * G + ix[1]) * G + ix[2]);
        atomicAdd(count + vox, 1u);
      }
    }
    vox_of[g] = vox;
  }
}

// ---- exclusive scan over n uint32 (n up to 2^24 + 1) ------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *total) {
  __shared__ uint32_t warp_sums[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  uint32_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + v - x;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_tile_sums(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) s += in[base + k];
  uint32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of the tile sums in one block (n_tiles <= kScanTile).
__global__ void __launch_bounds__(kScanThreads)
    scan_tile_offsets(uint32_t *__restrict__ sums, int64_t n_tiles) {
  int64_t base = (int64_t)threadIdx.x * kScanPer;
  uint32_t loc[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    loc[k] = base + k < n_tiles ? sums[base + k] : 0;
    s += loc[k];
  }
  uint32_t run = block_exclusive_scan(s, nullptr);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n_tiles) sums[base + k] = run;
    run += loc[k];
  }
}

// out[i] = sum of in[0..i) for i in [0, n]; out has n + 1 entries.
__global__ void __launch_bounds__(kScanThreads)
    scan_apply(const uint32_t *__restrict__ in, int64_t n, const uint32_t *__restrict__ tile_off,
               uint32_t *__restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  uint32_t loc[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    loc[k] = base + k < n ? in[base + k] : 0;
    s += loc[k];
  }
  uint32_t run = block_exclusive_scan(s, nullptr) + tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = run;
    if (base + k == n - 1) out[n] = run + loc[k];
    run += loc[k];
  }
}

// Scatter each kept pixel's key (voxel << 40 | view << 32 | pixel) into its
// voxel's segment (order inside a segment is arbitrary here).
__global__ void fuse_scatter_kernel(const __grid_constant__ pe_geom_layout L,
                                    const uint32_t *__restrict__ vox_of,
                                    const uint32_t *__restrict__ offs, uint32_t *__restrict__ count,
                                    unsigned long long *__restrict__ entries) {
  int64_t total = L.pix_off[L.nv];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t vox = vox_of[g];
    if (vox == PE_NONE) continue;
    int v = view_of(L, g);
    uint32_t slot = offs[vox] + atomicSub(count + vox, 1u) - 1u;
    entries[slot] = ((unsigned long long)vox << 40) | ((unsigned long long)v << 32) |
                    (unsigned long long)(g - L.pix_off[v]);
  }
}

// Eq. 22 for one contributor in FP64: s = sqrt(|n| |p| / |n . p|),
// R = sqrt(2) L s if s < 2.5 else 3.535 L.
__device__ __forceinline__ double eq22(pe_f3 n, pe_f3 p, double L) {
  double nx = n.x, ny = n.y, nz = n.z, px = p.x, py = p.y, pz = p.z;
  double nn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), __dmul_rn(nz, nz)));
  double pp = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz)));
  double np = __dadd_rn(__dadd_rn(__dmul_rn(nx, px), __dmul_rn(ny, py)), __dmul_rn(nz, pz));
  if (np < 0) np = -np;
  double s = np > 0 ? __dsqrt_rn(__ddiv_rn(__dmul_rn(nn, pp), np)) : __longlong_as_double(0x7ff0000000000000ll);
  if (s < 2.5) return __dmul_rn(__dmul_rn(1.4142135623730951, L), s);
  return __dmul_rn(3.535, L);
}

struct seg_acc {
  double sp[3], sn[3], rmax;
  pe_f3 n0;
  bool first;
};

__device__ __forceinline__ void seg_add(seg_acc &a, const pe_geom_layout &L,
                                        const float4 *__restrict__ nd, unsigned long long key) {
  int v = (int)((key >> 32) & 0xff);
  int64_t p = (int64_t)(key & 0xffffffffull);
  const pe_view &V = L.view[v];
  float4 q = nd[L.pix_off[v] + p];
  int i = (int)(p % V.W), j = (int)(p / V.W);
  pe_f3 x = pe_ray_at(pe_pixel_origin(V, i, j), q.w, pe_v3(V.d));
  pe_f3 n = {q.x, q.y, q.z};
  if (a.first) {
    a.n0 = n;
    a.first = false;
  }
  if (pe_dot(n, a.n0) < 0.0f) n = pe_neg3(n);
  a.sp[0] = __dadd_rn(a.sp[0], (double)x.x);
  a.sp[1] = __dadd_rn(a.sp[1], (double)x.y);
  a.sp[2] = __dadd_rn(a.sp[2], (double)x.z);
  a.sn[0] = __dadd_rn(a.sn[0], (double)n.x);
  a.sn[1] = __dadd_rn(a.sn[1], (double)n.y);
  a.sn[2] = __dadd_rn(a.sn[2], (double)n.z);
  double r = eq22(n, pe_v3(V.d), (double)V.pitch);
  if (r > a.rmax) a.rmax = r;
}

// One thread per voxel segment: order the keys, FP64 sums in that order,
// Eq. 22 maximum, write the splat at the owner pixel.
// One voxel segment (entries [s, offs[vox + 1]) of voxel vox, s = offs[vox]):
// the fused splat at its owner pixel.
__device__ __forceinline__ void fuse_one_segment(const pe_geom_layout &L,
                                                 const float4 *__restrict__ nd,
                                                 const unsigned long long *__restrict__ entries,
                                                 const uint32_t *__restrict__ offs, int64_t s,
                                                 float4 *__restrict__ cr, float4 *__restrict__ nf) {
  const uint32_t vox = (uint32_t)(entries[s] >> 40);
  int64_t len = (int64_t)offs[vox + 1] - s;
  seg_acc a;
  a.sp[0] = a.sp[1] = a.sp[2] = a.sn[0] = a.sn[1] = a.sn[2] = 0.0;
  a.rmax = 0.0;
  a.first = true;
  unsigned long long owner;
  if (len <= kSegLocal) {
    unsigned long long buf[kSegLocal];
    for (int64_t e = 0; e < len; ++e) {
      unsigned long long k = entries[s + e];
      int64_t m = e;
      while (m > 0 && buf[m - 1] > k) {
        buf[m] = buf[m - 1];
        --m;
      }
      buf[m] = k;
    }
    owner = buf[0];
    for (int64_t e = 0; e < len; ++e) seg_add(a, L, nd, buf[e]);
  } else {
    // long segment: visit keys in increasing order by repeated minimum
    unsigned long long last = 0;
    bool have = false;
    owner = ~0ull;
    for (int64_t e = 0; e < len; ++e) {
      unsigned long long best = ~0ull;
      for (int64_t f = 0; f < len; ++f) {
        unsigned long long k = entries[s + f];
        if ((!have || k > last) && k < best) best = k;
      }
      if (!have) owner = best;
      seg_add(a, L, nd, best);
      last = best;
      have = true;
    }
  }
  double cnt = (double)len;
  double m = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.sn[0], a.sn[0]), __dmul_rn(a.sn[1], a.sn[1])),
                                  __dmul_rn(a.sn[2], a.sn[2])));
  const pe_f3 nrm = {__double2float_rn(__ddiv_rn(a.sn[0], m)),
                     __double2float_rn(__ddiv_rn(a.sn[1], m)),
                     __double2float_rn(__ddiv_rn(a.sn[2], m))};
  // Owner: the contributing view facing the fused normal most directly, by
  // |n . d_v| in quarters (floor(4 |n . d_v|), so near-equal views tie),
  // the smaller (view, pixel) key on a tie; the first entry if the normal
  // vanishes.  Owners of neighbouring voxels then mostly come from the same
  // view, which keeps each stretch of surface in few pyramids.
  if (m > 0.0) {
    float bs = -1.0f;
    unsigned long long bk = owner;
    auto consider = [&](unsigned long long k) {
      const pe_view &V = L.view[(int)((k >> 32) & 0xff)];
      const float sc = floorf(__fmul_rn(fabsf(pe_dot(nrm, pe_f3{V.d[0], V.d[1], V.d[2]})), 4.0f));
      if (sc > bs || (sc == bs && k < bk)) {
        bs = sc;
        bk = k;
      }
    };
    for (int64_t e = 0; e < len; ++e) consider(entries[s + e]);
    owner = bk;
  }
  int v0 = (int)((owner >> 32) & 0xff);
  int64_t id = L.pix_off[v0] + (int64_t)(owner & 0xffffffffull);
  cr[id] = make_float4(__double2float_rn(__ddiv_rn(a.sp[0], cnt)),
                       __double2float_rn(__ddiv_rn(a.sp[1], cnt)),
                       __double2float_rn(__ddiv_rn(a.sp[2], cnt)), __double2float_rn(a.rmax));
  nf[id] = make_float4(nrm.x, nrm.y, nrm.z, (float)len);
}

// One segment per lane: each warp examines 32 entries at a time and queues,
// in shared memory, the ones that start a voxel's segment; whenever 32 are
// queued its lanes take one each (a segment's work is a serial chain of FP64
// sums, so a lane per segment, not per entry, keeps the warp full).
constexpr int kFuseThreads = 128;

__global__ void __launch_bounds__(kFuseThreads)
    fuse_segment_kernel(const __grid_constant__ pe_geom_layout L, const float4 *__restrict__ nd,
                        const unsigned long long *__restrict__ entries,
                        const uint32_t *__restrict__ offs, int64_t nvox,
                        float4 *__restrict__ cr, float4 *__restrict__ nf) {
  __shared__ uint32_t queue[kFuseThreads / 32][64];
  const int64_t n_entries = offs[nvox];  // kept pixels, written by scan_apply
  const int lane = threadIdx.x & 31;
  uint32_t *q = queue[threadIdx.x >> 5];
  int count = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_entries;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = base + lane;
    bool head = false;
    if (s < n_entries) head = offs[(uint32_t)(entries[s] >> 40)] == (uint32_t)s;
    const unsigned m = __ballot_sync(0xffffffffu, head);
    if (head) q[count + __popc(m & ((1u << lane) - 1u))] = (uint32_t)s;
    count += __popc(m);
    __syncwarp();
    if (count >= 32) {
      fuse_one_segment(L, nd, entries, offs, q[lane], cr, nf);
      __syncwarp();
      if (lane < count - 32) q[lane] = q[lane + 32];
      count -= 32;
      __syncwarp();
    }
  }
  if (lane < count) fuse_one_segment(L, nd, entries, offs, q[lane], cr, nf);
}

// Leaf boxes: bounds of the owned splats' spheres in the view's (u, v, d)
// frame, padded for rounding.  Empty tiles get lo = +inf, hi = -inf.
// Leaf boxes: per axis of the view frame, the union of the splats' disk
// extents (a disk, not its bounding sphere: thin along the axes its normal
// faces), padded; a leaf's lo.w holds the bit pattern of its occupancy mask
// (bit jj * PE_LEAF + ii set when slot (ii, jj) holds a splat) and hi.w its
// reach: the largest pixel distance from a slot to its splat's projected
// centre plus the splat's (padded) radius in pixels, so that a ray hitting a
// splat passes within `reach` pixels of the splat's slot.
static_assert(PE_LEAF * PE_LEAF <= 32, "leaf occupancy mask is one 32-bit word");
__global__ void pyramid_leaf_kernel(const __grid_constant__ pe_geom_layout L, int v,
                                    float4 *__restrict__ nodes) {
  const pe_view &V = L.view[v];
  int tw = L.tw[v][0], th = L.th[v][0];
  const float4 *cr = L.cr + L.pix_off[v];
  const float4 *nf = L.nf + L.pix_off[v];
  float pad = L.pad[v];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tw * th; t += gridDim.x * blockDim.x) {
    int tx = t % tw, ty = t / tw;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    uint32_t occ = 0;
    float reach = 0.0f;
    const float inv_pitch = 1.0f / V.pitch;
    for (int jj = 0; jj < PE_LEAF; ++jj) {
      int j = ty * PE_LEAF + jj;
      if (j >= V.H) break;
      for (int ii = 0; ii < PE_LEAF; ++ii) {
        int i = tx * PE_LEAF + ii;
        if (i >= V.W) break;
        float4 c = cr[(int64_t)j * V.W + i];
        if (!(c.w > 0.0f)) continue;
        occ |= 1u << (jj * PE_LEAF + ii);
        float qx = c.x - V.o[0], qy = c.y - V.o[1], qz = c.z - V.o[2];
        float a[3] = {qx * V.u[0] + qy * V.u[1] + qz * V.u[2],
                      qx * V.v[0] + qy * V.v[1] + qz * V.v[2],
                      qx * V.d[0] + qy * V.d[1] + qz * V.d[2]};
        float r = c.w * 1.000001f + pad;
        // reach: pixel distance (Chebyshev) from this slot to the splat's
        // projected centre plus its radius in pixels
        const float ci = a[0] * inv_pitch + 0.5f * V.W - 0.5f, cj = a[1] * inv_pitch + 0.5f * V.H - 0.5f;
        reach = fmaxf(reach, fmaxf(fabsf(ci - (float)i), fabsf(cj - (float)j)) + r * inv_pitch);
        // the disk's extent along axis e is R sqrt(1 - (n.e)^2) (its points
        // are c + y with y across n, |y| <= R); the 1e-6 under the root
        // (1e-3 R at a face-on axis) covers the rounding of n
        const float4 n = nf[(int64_t)j * V.W + i];
        const float ne[3] = {n.x * V.u[0] + n.y * V.u[1] + n.z * V.u[2],
                             n.x * V.v[0] + n.y * V.v[1] + n.z * V.v[2],
                             n.x * V.d[0] + n.y * V.d[1] + n.z * V.d[2]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float ek = c.w * 1.000001f * sqrtf(fmaxf(1.0f - ne[k] * ne[k], 0.0f) + 1e-6f) + pad;
          lo[k] = fminf(lo[k], a[k] - ek);
          hi[k] = fmaxf(hi[k], a[k] + ek);
        }
      }
    }
    int64_t nid = L.node_off[v][0] + t;
    nodes[2 * nid] = make_float4(lo[0], lo[1], lo[2], __uint_as_float(occ));
    nodes[2 * nid + 1] = make_float4(hi[0], hi[1], hi[2], reach);
  }
}

__global__ void pyramid_up_kernel(const __grid_constant__ pe_geom_layout L, int v, int l,
                                  float4 *__restrict__ nodes) {
  int tw = L.tw[v][l], th = L.th[v][l];
  int cw = L.tw[v][l - 1], ch = L.th[v][l - 1];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tw * th; t += gridDim.x * blockDim.x) {
    int tx = t % tw, ty = t / tw;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    for (int j = 0; j < PE_FAN; ++j)
      for (int i = 0; i < PE_FAN; ++i) {
        int cx = tx * PE_FAN + i, cy = ty * PE_FAN + j;
        if (cx >= cw || cy >= ch) continue;
        int64_t c = L.node_off[v][l - 1] + (int64_t)cy * cw + cx;
        float4 a = nodes[2 * c], b = nodes[2 * c + 1];
        lo.x = fminf(lo.x, a.x);
        lo.y = fminf(lo.y, a.y);
        lo.z = fminf(lo.z, a.z);
        hi.x = fmaxf(hi.x, b.x);
        hi.y = fmaxf(hi.y, b.y);
        hi.z = fmaxf(hi.z, b.z);
        hi.w = fmaxf(hi.w, b.w);  // largest reach below
      }
    int64_t nid = L.node_off[v][l] + t;
    nodes[2 * nid] = lo;
    nodes[2 * nid + 1] = hi;
  }
}

// Node slabs: for the pyramid nodes of levels 0..kSlabLevels-1 (up to
// 64 x 64 pixels), an axis n (the normalised sum of the node's splat
// normals, each turned toward its view) and the interval of heights
// n . (x - view origin) that the points x of the node's disks take: a disk
// (c, R, normal m) spans n . (c - o) +- R sqrt(1 - (n . m)^2), padded by
// 1e-6 under the root (the rounding of m) and by the view's absolute box
// pad.  Over a smooth patch the slab is far thinner than the node's box, so
// a ray that leaves the patch is rejected as soon as it is above the slab.
// One warp per node (all those levels of all views in one launch), sums in
// a fixed order, so the slabs are the same on every run.  Higher nodes, a
// node without splats and a node whose normals cancel get no slab (lower
// bound -inf).
constexpr int kSlabLevels = 5;

__global__ void __launch_bounds__(128)
    pyramid_slab_kernel(const __grid_constant__ pe_geom_layout L, int64_t n_slab_nodes,
                        float4 *__restrict__ slab, float *__restrict__ slab_hi) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n_slab_nodes) return;  // uniform over the warp
  // warp w -> (view, level, node): views in order, levels 0.. within each
  int v = 0, l = 0;
  int64_t k = w;
  for (v = 0; v < L.nv; ++v) {
    bool found = false;
    for (l = 0; l < min(L.nlev[v], kSlabLevels); ++l) {
      const int64_t cnt = (int64_t)L.tw[v][l] * L.th[v][l];
      if (k < cnt) {
        found = true;
        break;
      }
      k -= cnt;
    }
    if (found) break;
  }
  const int64_t nid = L.node_off[v][l] + k;
  const pe_view &V = L.view[v];
  const int tx = (int)(k % L.tw[v][l]), ty = (int)(k / L.tw[v][l]);
  const int span = PE_LEAF << l;
  const int i0 = tx * span, j0 = ty * span;
  const int iw = min(span, V.W - i0), jh = min(span, V.H - j0);
  const int npx = iw * jh;
  const float4 *cr = L.cr + L.pix_off[v];
  const float4 *nf = L.nf + L.pix_off[v];
  // pass 1: the axis
  float sx = 0.f, sy = 0.f, sz = 0.f, cnt = 0.f;
  for (int q = lane; q < npx; q += 32) {
    const int64_t g = (int64_t)(j0 + q / iw) * V.W + (i0 + q % iw);
    if (!(cr[g].w > 0.0f)) continue;
    const float4 m = nf[g];
    const float sg = (m.x * V.d[0] + m.y * V.d[1] + m.z * V.d[2]) > 0.0f ? -1.0f : 1.0f;
    sx += sg * m.x;
    sy += sg * m.y;
    sz += sg * m.z;
    cnt += 1.0f;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(FULL, sx, o);
    sy += __shfl_xor_sync(FULL, sy, o);
    sz += __shfl_xor_sync(FULL, sz, o);
    cnt += __shfl_xor_sync(FULL, cnt, o);
  }
  const float len = sqrtf(sx * sx + sy * sy + sz * sz);
  if (!(cnt > 0.0f) || !(len > 1e-3f * cnt)) {
    if (lane == 0) {
      slab[nid] = make_float4(0.f, 0.f, 1.f, -INFINITY);
      slab_hi[nid] = INFINITY;
    }
    return;
  }
  const float nx = sx / len, ny = sy / len, nz = sz / len;
  // pass 2: the heights
  const float pad = L.pad[v];
  float lo = INFINITY, hi = -INFINITY;
  for (int q = lane; q < npx; q += 32) {
    const int64_t g = (int64_t)(j0 + q / iw) * V.W + (i0 + q % iw);
    const float4 c = cr[g];
    if (!(c.w > 0.0f)) continue;
    const float4 m = nf[g];
    const float h = nx * (c.x - V.o[0]) + ny * (c.y - V.o[1]) + nz * (c.z - V.o[2]);
    const float nm = nx * m.x + ny * m.y + nz * m.z;
    const float e = c.w * 1.000001f * sqrtf(fmaxf(1.0f - nm * nm, 0.0f) + 1e-6f) + pad;
    lo = fminf(lo, h - e);
    hi = fmaxf(hi, h + e);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
  }
  if (lane == 0) {
    slab[nid] = make_float4(nx, ny, nz, lo - pad);
    slab_hi[nid] = hi + pad;
  }
}

// No slab for the nodes above kSlabLevels.
__global__ void slab_clear_kernel(float4 *__restrict__ slab, float *__restrict__ slab_hi,
                                  int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    slab[i] = make_float4(0.f, 0.f, 1.f, -INFINITY);
    slab_hi[i] = INFINITY;
  }
}

// The cells of the coarse grid that splat g marks: per world axis k the disk
// reaches R sqrt(1 - n_k^2) from its centre, padded by 1 % of a cell and the
// view's box pad (for rounding); cells clamped to the grid, `outside` when
// the padded box leaves it.  The view mask, the cell slabs' axes and their
// heights all take the same cells.
struct cell_box {
  int lo[3], hi[3];
  bool outside;
};
__device__ __forceinline__ cell_box splat_cells(const pe_geom_layout &L, float4 c, float4 nn,
                                                int v) {
  const int n = L.vg_n;
  const float cell = L.vg_cell;
  const float cc[3] = {c.x, c.y, c.z}, nk[3] = {nn.x, nn.y, nn.z};
  cell_box b;
  b.outside = false;
  for (int k = 0; k < 3; ++k) {
    const float pad = c.w * 1.00001f * sqrtf(fmaxf(1.0f - nk[k] * nk[k], 0.0f) + 1e-6f) +
                      1e-2f * cell + L.pad[v];
    float a = floorf((cc[k] - pad - L.vg_min[k]) / cell);
    float e = floorf((cc[k] + pad - L.vg_min[k]) / cell);
    if (!(a >= 0.0f) || !(e <= (float)(n - 1))) b.outside = true;
    b.lo[k] = (int)fminf(fmaxf(a, 0.0f), (float)(n - 1));
    b.hi[k] = (int)fminf(fmaxf(e, 0.0f), (float)(n - 1));
  }
  return b;
}

// Fixed-point scale of the cell axis sums (a normal component times 2^32,
// summed in 64-bit integers: the sum does not depend on the atomics' order;
// 2^28 terms at most, far below overflow).
constexpr float kAxisScale = 4294967296.0f;

// Coarse view-occupancy grid: every splat marks its cells with its owner
// view's bit (vmask[n^3] for splats reaching outside the grid), adds its
// normal, turned toward its view, to each cell's axis sum and counts itself
// there.
__global__ void vgrid_kernel(const __grid_constant__ pe_geom_layout L, uint32_t *__restrict__ vmask,
                             unsigned long long *__restrict__ axis_sum,
                             unsigned int *__restrict__ axis_cnt) {
  const int n = L.vg_n;
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t total = L.pix_off[L.nv];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    float4 c = L.cr[g];
    if (!(c.w > 0.0f)) continue;
    const int v = view_of(L, g);
    const uint32_t bit = 1u << v;
    const float4 nn = L.nf[g];
    const pe_view &V = L.view[v];
    const float sg = (nn.x * V.d[0] + nn.y * V.d[1] + nn.z * V.d[2]) > 0.0f ? -1.0f : 1.0f;
    const unsigned long long qx = (unsigned long long)__float2ll_rn(sg * nn.x * kAxisScale);
    const unsigned long long qy = (unsigned long long)__float2ll_rn(sg * nn.y * kAxisScale);
    const unsigned long long qz = (unsigned long long)__float2ll_rn(sg * nn.z * kAxisScale);
    const cell_box b = splat_cells(L, c, nn, v);
    if (b.outside) atomicOr(vmask + n3, bit);
    for (int x = b.lo[0]; x <= b.hi[0]; ++x)
      for (int y = b.lo[1]; y <= b.hi[1]; ++y)
        for (int z = b.lo[2]; z <= b.hi[2]; ++z) {
          const int64_t cid = ((int64_t)x * n + y) * n + z;
          atomicOr(vmask + cid, bit);
          atomicAdd(axis_sum + 3 * cid, qx);
          atomicAdd(axis_sum + 3 * cid + 1, qy);
          atomicAdd(axis_sum + 3 * cid + 2, qz);
          atomicAdd(axis_cnt + cid, 1u);
        }
  }
}

// A float as an unsigned key with the same order (for atomicMin/Max).
__device__ __forceinline__ unsigned int f_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_f(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Per cell: the axis (normalised sum; none for an empty cell or when the
// normals cancel, as for the node slabs), and the height keys' start values.
__global__ void cell_axis_kernel(int64_t n3, const unsigned long long *__restrict__ axis_sum,
                                 const unsigned int *__restrict__ axis_cnt,
                                 float4 *__restrict__ axis, unsigned int *__restrict__ hkey) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double inv = 1.0 / (double)kAxisScale;
    const double sx = (double)(long long)axis_sum[3 * i] * inv;
    const double sy = (double)(long long)axis_sum[3 * i + 1] * inv;
    const double sz = (double)(long long)axis_sum[3 * i + 2] * inv;
    const double cnt = (double)axis_cnt[i];
    const double len = sqrt(sx * sx + sy * sy + sz * sz);
    if (cnt > 0.0 && len > 1e-3 * cnt)
      axis[i] = make_float4((float)(sx / len), (float)(sy / len), (float)(sz / len), 1.0f);
    else
      axis[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    hkey[2 * i] = 0xffffffffu;  // lowest height: min over keys
    hkey[2 * i + 1] = 0u;       // highest height: max over keys
  }
}

// Heights axis . (x - cell centre) over the disks a cell counts: the centre's
// height +- R sqrt(1 - (axis . m)^2), padded like the node slabs.
__global__ void cell_height_kernel(const __grid_constant__ pe_geom_layout L,
                                   const float4 *__restrict__ axis,
                                   unsigned int *__restrict__ hkey) {
  const int n = L.vg_n;
  const float cell = L.vg_cell;
  const int64_t total = L.pix_off[L.nv];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    float4 c = L.cr[g];
    if (!(c.w > 0.0f)) continue;
    const int v = view_of(L, g);
    const float4 m = L.nf[g];
    const cell_box b = splat_cells(L, c, m, v);
    const float rx = c.x - L.vg_min[0], ry = c.y - L.vg_min[1], rz = c.z - L.vg_min[2];
    for (int x = b.lo[0]; x <= b.hi[0]; ++x)
      for (int y = b.lo[1]; y <= b.hi[1]; ++y)
        for (int z = b.lo[2]; z <= b.hi[2]; ++z) {
          const int64_t cid = ((int64_t)x * n + y) * n + z;
          const float4 a = axis[cid];
          if (a.w == 0.0f) continue;
          const float h = a.x * (rx - (x + 0.5f) * cell) + a.y * (ry - (y + 0.5f) * cell) +
                          a.z * (rz - (z + 0.5f) * cell);
          const float am = a.x * m.x + a.y * m.y + a.z * m.z;
          const float e = c.w * 1.000001f * sqrtf(fmaxf(1.0f - am * am, 0.0f) + 1e-6f) + L.pad[v];
          atomicMin(hkey + 2 * cid, f_key(h - e));
          atomicMax(hkey + 2 * cid + 1, f_key(h + e));
        }
  }
}

// The cell slabs in the form the march tests (see pe_geom_layout::cslab),
// padded by 1e-3 of a cell and 1e-5 of the grid's coordinate magnitude: far
// above the rounding of the heights here and of the ray positions in the
// march, so every point of a counted disk passes.
__global__ void cell_slab_kernel(int64_t n3, const float4 *__restrict__ axis,
                                 const unsigned int *__restrict__ hkey, float pad,
                                 float4 *__restrict__ cslab) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = axis[i];
    const unsigned int klo = hkey[2 * i], khi = hkey[2 * i + 1];
    if (a.w == 0.0f || klo == 0xffffffffu) {
      cslab[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float lo = key_f(klo), hi = key_f(khi);
    const float half = 0.5f * (hi - lo) + pad;
    const float mid = 0.5f * (hi + lo);
    cslab[i] = make_float4(a.x / half, a.y / half, a.z / half, mid / half);
  }
}

int grid_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

struct agg_ws {
  uint32_t *count, *offs, *tile, *vox_of;
  unsigned long long *entries;
  uint8_t *canny_state;     // edge mode 1 (the other Canny buffers alias
  unsigned int *changed;    // entries and vox_of, which the fusion fills later)
  unsigned long long *axis_sum;  // cell slabs: [n^3][3] fixed-point normal sums
  unsigned int *axis_cnt;        // [n^3]
  float4 *axis;                  // [n^3] axis, w = 1 when the cell has one
  unsigned int *hkey;            // [n^3][2] lowest / highest height keys
};

agg_ws carve_agg(pe_carve &c, int64_t total_pix, int G) {
  agg_ws w;
  int64_t nv = (int64_t)G * G * G;
  w.count = c.take<uint32_t>((size_t)nv);
  w.offs = c.take<uint32_t>((size_t)nv + 1);
  w.tile = c.take<uint32_t>((size_t)((nv + kScanTile - 1) / kScanTile));
  w.vox_of = c.take<uint32_t>((size_t)total_pix);
  w.entries = c.take<unsigned long long>((size_t)total_pix);
  w.canny_state = c.take<uint8_t>((size_t)total_pix);
  w.changed = c.take<unsigned int>(1);
  const int64_t n3 = (int64_t)PE_VGRID * PE_VGRID * PE_VGRID;
  w.axis_sum = c.take<unsigned long long>((size_t)n3 * 3);
  w.axis_cnt = c.take<unsigned int>((size_t)n3);
  w.axis = c.take<float4>((size_t)n3);
  w.hkey = c.take<unsigned int>((size_t)n3 * 2);
  return w;
}

}  // namespace

// out[i] = sum of in[0..i) for i in [0, n] (n + 1 entries; n <= 2^24) with
// tile scratch of (n + 4095) / 4096 uint32.
pe_status pe_exclusive_scan_u32(const uint32_t *in, int64_t n, uint32_t *tile, uint32_t *out,
                                cudaStream_t s) {
  const int64_t n_tiles = (n + kScanTile - 1) / kScanTile;
  if (n < 1 || n_tiles > kScanTile) return pe_fail(PE_EUNSUPPORTED, "scan: too many entries");
  scan_tile_sums<<<(int)n_tiles, kScanThreads, 0, s>>>(in, n, tile);
  PE_TRY_LAUNCH("scan_tile_sums");
  scan_tile_offsets<<<1, kScanThreads, 0, s>>>(tile, n_tiles);
  PE_TRY_LAUNCH("scan_tile_offsets");
  scan_apply<<<(int)n_tiles, kScanThreads, 0, s>>>(in, n, tile, out);
  PE_TRY_LAUNCH("scan_apply");
  return PE_OK;
}

extern "C" size_t pe_aggregate_workspace(int32_t n_views, const pe_view *views,
                                         int32_t fuse_grid) {
  pe_geom_layout L;
  if (!pe_make_layout(n_views, views, &L) || fuse_grid < 1 || fuse_grid > 256) return 0;
  pe_carve c{nullptr, 0};
  carve_agg(c, L.pix_off[L.nv], fuse_grid);
  return c.bytes() + 256;
}

extern "C" pe_status pe_aggregate_views(const pe_view *views, int32_t n_views,
                                        const float *gfb_nd, const uint8_t *gfb_mask,
                                        const pe_params *prm, void *ws, size_t ws_bytes,
                                        pe_geom *out, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!views || !gfb_nd || !gfb_mask || !prm || !out)
    return pe_fail(PE_EINVAL, "pe_aggregate_views: null argument");
  pe_geom_layout L;
  if (!pe_make_layout(n_views, views, &L))
    return pe_fail(PE_EINVAL, "pe_aggregate_views: 1 <= n_views <= %d with valid views",
                   PE_MAX_VIEWS);
  int G = prm->fuse_grid;
  if (G < 1 || G > 256) return pe_fail(PE_EINVAL, "pe_aggregate_views: fuse_grid in [1, 256]");
  if (!(prm->inv_voxel > 0.0f) || !isfinite(prm->inv_voxel) || !isfinite(prm->bbox_min[0]) ||
      !isfinite(prm->bbox_min[1]) || !isfinite(prm->bbox_min[2]))
    return pe_fail(PE_EINVAL, "pe_aggregate_views: the fusion grid needs a finite origin and "
                              "inv_voxel > 0 (a point set of positive extent)");
  if (!pe_aligned(gfb_nd, 16)) return pe_fail(PE_EINVAL, "pe_aggregate_views: gfb_nd alignment");
  if (out->n_views != n_views || !out->blob_dev)
    return pe_fail(PE_EINVAL, "pe_aggregate_views: out must name the same views and a blob");
  for (int v = 0; v < n_views; ++v)
    if (memcmp(&out->views[v], &views[v], sizeof(pe_view)) != 0)
      return pe_fail(PE_EINVAL, "pe_aggregate_views: out->views differ from views");
  size_t o_cr, o_nf, o_nodes, o_vm, o_slab, o_slab_hi, o_cslab, tot;
  pe_layout_offsets(L, &o_cr, &o_nf, &o_nodes, &o_vm, &o_slab, &o_slab_hi, &o_cslab, &tot);
  if (out->blob_bytes < tot || !pe_aligned(out->blob_dev, 256))
    return pe_fail(PE_ENOMEM, "pe_aggregate_views: geometry blob needs %zu bytes", tot);
  size_t need = pe_aggregate_workspace(n_views, views, G);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_aggregate_views: workspace needs %zu bytes", need);

  char *blob = static_cast<char *>(out->blob_dev);
  float4 *cr = reinterpret_cast<float4 *>(blob + o_cr);
  float4 *nf = reinterpret_cast<float4 *>(blob + o_nf);
  float4 *nodes = reinterpret_cast<float4 *>(blob + o_nodes);
  uint32_t *vmask = reinterpret_cast<uint32_t *>(blob + o_vm);
  float4 *slab = reinterpret_cast<float4 *>(blob + o_slab);
  float *slab_hi = reinterpret_cast<float *>(blob + o_slab_hi);
  float4 *cslab = reinterpret_cast<float4 *>(blob + o_cslab);
  L.cr = cr;
  L.nf = nf;
  L.nodes = nodes;
  // the coarse grid covers the fusion box with one spare cell on each side
  const float ext = (float)((double)G / (double)prm->inv_voxel);
  L.vg_n = PE_VGRID;
  L.vg_cell = ext / (float)(PE_VGRID - 2);
  for (int k = 0; k < 3; ++k) L.vg_min[k] = prm->bbox_min[k] - L.vg_cell;
  L.vmask = vmask;

  int64_t total_pix = L.pix_off[n_views];
  int64_t nvox = (int64_t)G * G * G;
  pe_carve c{static_cast<char *>(ws), 0};
  agg_ws w = carve_agg(c, total_pix, G);
  const float4 *nd = reinterpret_cast<const float4 *>(gfb_nd);
  int cap = sms() * 16;

  PE_TRY_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * nvox, s));
  PE_TRY_CUDA(cudaMemsetAsync(cr, 0, sizeof(float4) * total_pix, s));
  PE_TRY_CUDA(cudaMemsetAsync(nf, 0, sizeof(float4) * total_pix, s));
  const uint8_t *cstate = nullptr;
  if (prm->edge_mode == 1) {
    float *S = reinterpret_cast<float *>(w.entries), *Gm = S + total_pix;
    uint8_t *sec = reinterpret_cast<uint8_t *>(w.vox_of);
    canny_smooth_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, nd, gfb_mask, S);
    PE_TRY_LAUNCH("canny_smooth_kernel");
    canny_grad_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, gfb_mask, S, Gm, sec);
    PE_TRY_LAUNCH("canny_grad_kernel");
    canny_nms_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, gfb_mask, Gm, sec,
                                                                    prm->edge_tau, w.canny_state);
    PE_TRY_LAUNCH("canny_nms_kernel");
    // hysteresis: batches of passes until a batch changes nothing
    bool converged = false;
    for (int batch = 0; batch < 4096 && !converged; ++batch) {
      PE_TRY_CUDA(cudaMemsetAsync(w.changed, 0, sizeof(unsigned int), s));
      for (int k = 0; k < 8; ++k) {
        canny_hyst_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, w.canny_state,
                                                                         w.changed);
        PE_TRY_LAUNCH("canny_hyst_kernel");
      }
      unsigned int h = 0;
      PE_TRY_CUDA(cudaMemcpyAsync(&h, w.changed, sizeof(h), cudaMemcpyDeviceToHost, s));
      PE_TRY_CUDA(cudaStreamSynchronize(s));
      converged = h == 0;
    }
    if (!converged) return pe_fail(PE_EOVERFLOW, "pe_aggregate_views: Canny hysteresis did not converge");
    cstate = w.canny_state;
  } else if (prm->edge_mode != 0) {
    return pe_fail(PE_EINVAL, "pe_aggregate_views: edge_mode must be 0 or 1");
  }
  fuse_classify_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(
      L, nd, gfb_mask, prm->edge_tau, cstate, prm->bbox_min[0], prm->bbox_min[1],
      prm->bbox_min[2], prm->inv_voxel, G, w.vox_of, w.count);
  PE_TRY_LAUNCH("fuse_classify_kernel");
  int64_t n_tiles = (nvox + kScanTile - 1) / kScanTile;
  if (n_tiles > kScanTile) return pe_fail(PE_EUNSUPPORTED, "voxel grid too large for the scan");
  scan_tile_sums<<<(int)n_tiles, kScanThreads, 0, s>>>(w.count, nvox, w.tile);
  PE_TRY_LAUNCH("scan_tile_sums");
  scan_tile_offsets<<<1, kScanThreads, 0, s>>>(w.tile, n_tiles);
  PE_TRY_LAUNCH("scan_tile_offsets");
  scan_apply<<<(int)n_tiles, kScanThreads, 0, s>>>(w.count, nvox, w.tile, w.offs);
  PE_TRY_LAUNCH("scan_apply");
  fuse_scatter_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, w.vox_of, w.offs,
                                                                     w.count, w.entries);
  PE_TRY_LAUNCH("fuse_scatter_kernel");
  // segment heads are found by slot; the kernel reads the entry count
  // offs[nvox] on the device (at most total_pix)
  fuse_segment_kernel<<<grid_for(total_pix, kFuseThreads, cap), kFuseThreads, 0, s>>>(
      L, nd, w.entries, w.offs, nvox, cr, nf);
  PE_TRY_LAUNCH("fuse_segment_kernel");
  const int64_t n3 = (int64_t)PE_VGRID * PE_VGRID * PE_VGRID;
  PE_TRY_CUDA(cudaMemsetAsync(vmask, 0, sizeof(uint32_t) * ((size_t)n3 + 1), s));
  PE_TRY_CUDA(cudaMemsetAsync(w.axis_sum, 0, sizeof(unsigned long long) * 3 * (size_t)n3, s));
  PE_TRY_CUDA(cudaMemsetAsync(w.axis_cnt, 0, sizeof(unsigned int) * (size_t)n3, s));
  vgrid_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, vmask, w.axis_sum, w.axis_cnt);
  PE_TRY_LAUNCH("vgrid_kernel");
  cell_axis_kernel<<<grid_for(n3, 256, cap), 256, 0, s>>>(n3, w.axis_sum, w.axis_cnt, w.axis,
                                                          w.hkey);
  PE_TRY_LAUNCH("cell_axis_kernel");
  cell_height_kernel<<<grid_for(total_pix, 256, cap), 256, 0, s>>>(L, w.axis, w.hkey);
  PE_TRY_LAUNCH("cell_height_kernel");
  {
    float mag = 0.0f;
    for (int k = 0; k < 3; ++k)
      mag = fmaxf(mag, fabsf(L.vg_min[k]) + L.vg_cell * (float)L.vg_n);
    const float pad = 1e-3f * L.vg_cell + 1e-5f * mag;
    cell_slab_kernel<<<grid_for(n3, 256, cap), 256, 0, s>>>(n3, w.axis, w.hkey, pad, cslab);
    PE_TRY_LAUNCH("cell_slab_kernel");
  }
  out->vgrid_n = L.vg_n;
  out->vgrid_cell = L.vg_cell;
  for (int k = 0; k < 3; ++k) out->vgrid_min[k] = L.vg_min[k];
  for (int v = 0; v < n_views; ++v) {
    pyramid_leaf_kernel<<<grid_for((int64_t)L.tw[v][0] * L.th[v][0], 128, cap), 128, 0, s>>>(
        L, v, nodes);
    PE_TRY_LAUNCH("pyramid_leaf_kernel");
    for (int l = 1; l < L.nlev[v]; ++l) {
      pyramid_up_kernel<<<grid_for((int64_t)L.tw[v][l] * L.th[v][l], 128, cap), 128, 0, s>>>(
          L, v, l, nodes);
      PE_TRY_LAUNCH("pyramid_up_kernel");
    }
  }
  slab_clear_kernel<<<grid_for(L.n_nodes, 256, cap), 256, 0, s>>>(slab, slab_hi, L.n_nodes);
  PE_TRY_LAUNCH("slab_clear_kernel");
  int64_t n_slab = 0;
  for (int v = 0; v < n_views; ++v)
    for (int l = 0; l < L.nlev[v] && l < kSlabLevels; ++l) n_slab += (int64_t)L.tw[v][l] * L.th[v][l];
  pyramid_slab_kernel<<<(unsigned)((n_slab * 32 + 127) / 128), 128, 0, s>>>(L, n_slab, slab,
                                                                          slab_hi);
  PE_TRY_LAUNCH("pyramid_slab_kernel");
  return PE_OK;
}
