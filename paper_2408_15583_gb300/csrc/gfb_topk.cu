// Alg. 1 with a finite heap of K points per ray tube, as written: of the
// candidates of a tube (points within delta of its central ray, in front of
// the screen) the K nearest the central ray are kept, and of those the one
// nearest the tube's origin gives the pixel's depth.  (The default tube mode
// of pe_build_gfb keeps every candidate, K unbounded.)
//
// Three passes per batch of views, all scatter-then-gather:
//   count  every point visits the pixels its tube footprint covers and
//          counts the pixels it is a candidate of;
//   fill   after an exclusive scan, the same visit writes 64-bit keys
//          (float bits of the squared distance to the central ray << 32 |
//          point index) into the pixel's segment;
//   select one thread per pixel keeps the K smallest keys of its segment,
//          recomputes their distances to the origin and keeps the nearest
//          (ties: smaller index), writing the pixel's depth key.
// The tube test is the same arithmetic as the default tube mode, so K >= the
// number of candidates reproduces it bit for bit.
#include <cstring>

#include "pe_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxK = 64;

// Tube test of point c against pixel (i, j): squared distance to the
// central ray (rank) and distance to the origin (depth).
__device__ __forceinline__ bool tube_terms(const pe_view &V, int i, int j, pe_f3 c, float delta,
                                           float &a, float &depth) {
  const pe_f3 o = pe_pixel_origin(V, i, j);
  const pe_f3 d = pe_v3(V.d);
  const pe_f3 q = pe_sub3(c, o);
  const float t = pe_dot(q, d);
  const pe_f3 x = pe_ray_at(o, t, d);
  const pe_f3 e = pe_sub3(x, c);
  a = pe_dot(e, e);
  if (!(a < pe_mul(delta, delta))) return false;
  if (!(t > 0.0f)) return false;
  depth = pe_sqrt(pe_dot(q, q));
  return true;
}

// Visit every (point, pixel) candidate pair of view blockIdx.y.  PASS 0:
// count per pixel; PASS 1: write the rank key into the pixel's segment.
template <int PASS>
__global__ void __launch_bounds__(kThreads)
    topk_visit(const __grid_constant__ pe_view_batch vb, const float *__restrict__ pos, int64_t n,
               float delta, uint32_t *__restrict__ count, const uint32_t *__restrict__ offs,
               uint32_t *__restrict__ cursor, unsigned long long *__restrict__ list,
               uint32_t capacity, unsigned int *err) {
  const int vi = blockIdx.y;
  const pe_view &V = vb.v[vi];
  const int W = V.W, H = V.H;
  const int64_t pix0 = (int64_t)vi * W * H;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const pe_f3 c = {__ldg(pos + 3 * p), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2)};
    // footprint: pixels whose ray passes within delta of c (one pixel of
    // margin for rounding; not part of the test)
    const float qx = c.x - V.o[0], qy = c.y - V.o[1], qz = c.z - V.o[2];
    const float inv = 1.0f / V.pitch;
    const float ci = (qx * V.u[0] + qy * V.u[1] + qz * V.u[2]) * inv + 0.5f * W - 0.5f;
    const float cj = (qx * V.v[0] + qy * V.v[1] + qz * V.v[2]) * inv + 0.5f * H - 0.5f;
    if (!(fabsf(ci) < 1e30f) || !(fabsf(cj) < 1e30f)) continue;
    const float rp = delta * inv + 1.0f;
    const float fi0 = fmaxf(floorf(ci - rp), 0.0f), fi1 = fminf(ceilf(ci + rp), (float)(W - 1));
    const float fj0 = fmaxf(floorf(cj - rp), 0.0f), fj1 = fminf(ceilf(cj + rp), (float)(H - 1));
    if (!(fi0 <= fi1) || !(fj0 <= fj1)) continue;
    for (int j = (int)fj0; j <= (int)fj1; ++j)
      for (int i = (int)fi0; i <= (int)fi1; ++i) {
        float a, depth;
        if (!tube_terms(V, i, j, c, delta, a, depth)) continue;
        const int64_t g = pix0 + (int64_t)j * W + i;
        if (PASS == 0) {
          atomicAdd(count + g, 1u);
        } else {
          const uint32_t slot = offs[g] + atomicAdd(cursor + g, 1u);
          if (slot < capacity)
            list[slot] = ((unsigned long long)__float_as_uint(a) << 32) | (unsigned long long)p;
          else
            pe_raise(err, PE_ERR_OVERFLOW);
        }
      }
  }
}

__global__ void __launch_bounds__(kThreads)
    topk_select(const __grid_constant__ pe_view_batch vb, const float *__restrict__ pos,
                float delta, int K, const uint32_t *__restrict__ offs,
                const unsigned long long *__restrict__ list, uint32_t capacity,
                unsigned long long *__restrict__ keys) {
  const int64_t per = (int64_t)vb.W * vb.H, total = per * vb.n;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int vi = (int)(g / per);
    const int64_t r = g % per;
    const int i = (int)(r % vb.W), j = (int)(r / vb.W);
    uint32_t b = offs[g], e = offs[g + 1];
    if (e > capacity) e = capacity;
    unsigned long long best[kMaxK];
    int cnt = 0;
    for (uint32_t m = b; m < e; ++m) {
      const unsigned long long k = list[m];
      if (cnt == K && !(k < best[K - 1])) continue;
      int at = cnt < K ? cnt++ : K - 1;
      while (at > 0 && best[at - 1] > k) {
        best[at] = best[at - 1];
        --at;
      }
      best[at] = k;
    }
    unsigned long long out = ~0ull;
    for (int m = 0; m < cnt; ++m) {
      const uint32_t p = (uint32_t)(best[m] & 0xffffffffull);
      const pe_f3 c = {__ldg(pos + 3 * (int64_t)p), __ldg(pos + 3 * (int64_t)p + 1),
                       __ldg(pos + 3 * (int64_t)p + 2)};
      float a, depth;
      if (!tube_terms(vb.v[vi], i, j, c, delta, a, depth)) continue;  // cannot happen
      const unsigned long long key = ((unsigned long long)__float_as_uint(depth) << 32) | p;
      if (key < out) out = key;
    }
    keys[g] = out;
  }
}

int64_t footprint_bound(const pe_view &v, float delta) {
  const int64_t s = 2 * ((int64_t)ceil(delta / v.pitch) + 1) + 1;
  return s * s;
}

struct topk_ws {
  uint32_t *count, *offs, *cursor, *tile;
  unsigned long long *list;
  uint32_t capacity;
};

bool carve_topk(pe_carve &c, const pe_view *views, int32_t n_views, int64_t n_points, float delta,
                topk_ws *w) {
  const int64_t per = (int64_t)views[0].W * views[0].H;
  const int64_t pix = per * n_views;
  int64_t cap = 0;
  for (int v = 0; v < n_views; ++v) cap += n_points * footprint_bound(views[v], delta);
  if (cap > (int64_t)UINT32_MAX - 1) return false;
  w->count = c.take<uint32_t>((size_t)pix);
  w->offs = c.take<uint32_t>((size_t)pix + 1);
  w->cursor = c.take<uint32_t>((size_t)pix);
  w->tile = c.take<uint32_t>((size_t)((pix + 4095) / 4096 + 1));
  w->list = c.take<unsigned long long>((size_t)(cap > 0 ? cap : 1));
  w->capacity = (uint32_t)cap;
  return true;
}

}  // namespace

extern "C" size_t pe_build_gfb_topk_workspace(int32_t n_views, const pe_view *views,
                                              int64_t n_points, float delta) {
  if (!views || n_views < 1 || n_views > PE_MAX_BATCH || n_points < 0 || !(delta > 0)) return 0;
  pe_carve c{nullptr, 0};
  topk_ws w;
  if (!carve_topk(c, views, n_views, n_points, delta, &w)) return 0;
  return c.bytes() + 256;
}

extern "C" pe_status pe_build_gfb_topk(const pe_view *views, int32_t n_views, const float *pos,
                                       int64_t n_points, float delta, int32_t K, void *ws,
                                       size_t ws_bytes, uint64_t *keys_out, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!views || n_views < 1 || n_views > PE_MAX_BATCH)
    return pe_fail(PE_EINVAL, "pe_build_gfb_topk: n_views must be in [1, %d]", PE_MAX_BATCH);
  for (int i = 1; i < n_views; ++i)
    if (views[i].W != views[0].W || views[i].H != views[0].H)
      return pe_fail(PE_EINVAL, "pe_build_gfb_topk: all views of a call must share W x H");
  if (views[0].W <= 0 || views[0].H <= 0 || !(views[0].pitch > 0) || !keys_out)
    return pe_fail(PE_EINVAL, "pe_build_gfb_topk: bad screen or output");
  if (n_points < 0 || n_points >= (int64_t)PE_NONE || (n_points > 0 && !pos))
    return pe_fail(PE_EINVAL, "pe_build_gfb_topk: points");
  if (!(delta > 0) || K < 1 || K > kMaxK)
    return pe_fail(PE_EINVAL, "pe_build_gfb_topk: delta > 0 and K in [1, %d]", kMaxK);
  const int64_t per = (int64_t)views[0].W * views[0].H, pix = per * n_views;
  if (pix + 1 > (1ll << 24)) return pe_fail(PE_EUNSUPPORTED, "pe_build_gfb_topk: too many pixels");
  const size_t need = pe_build_gfb_topk_workspace(n_views, views, n_points, delta);
  if (need == 0) return pe_fail(PE_EUNSUPPORTED, "pe_build_gfb_topk: candidate list too long");
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_build_gfb_topk: workspace needs %zu bytes", need);
  pe_carve c{static_cast<char *>(ws), 0};
  topk_ws w;
  carve_topk(c, views, n_views, n_points, delta, &w);
  pe_view_batch vb;
  memset(&vb, 0, sizeof(vb));
  vb.n = n_views;
  vb.W = views[0].W;
  vb.H = views[0].H;
  for (int i = 0; i < n_views; ++i) vb.v[i] = views[i];
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(keys_out);
  PE_TRY_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * pix, s));
  PE_TRY_CUDA(cudaMemsetAsync(w.cursor, 0, sizeof(uint32_t) * pix, s));
  unsigned int *err = pe_err_word();
  int64_t b = (n_points + kThreads - 1) / kThreads;
  dim3 grid((unsigned)(b < 1 ? 1 : (b < 2048 ? b : 2048)), (unsigned)n_views);
  if (n_points > 0) {
    topk_visit<0><<<grid, kThreads, 0, s>>>(vb, pos, n_points, delta, w.count, nullptr, nullptr,
                                            nullptr, 0, err);
    PE_TRY_LAUNCH("topk_visit");
  }
  pe_status st = pe_exclusive_scan_u32(w.count, pix, w.tile, w.offs, s);
  if (st != PE_OK) return st;
  if (n_points > 0) {
    topk_visit<1><<<grid, kThreads, 0, s>>>(vb, pos, n_points, delta, nullptr, w.offs, w.cursor,
                                            w.list, w.capacity, err);
    PE_TRY_LAUNCH("topk_visit");
  }
  int64_t pb = (pix + kThreads - 1) / kThreads;
  topk_select<<<(int)(pb < 65535 ? pb : 65535), kThreads, 0, s>>>(vb, pos, delta, K, w.offs,
                                                                    w.list, w.capacity, keys);
  PE_TRY_LAUNCH("topk_select");
  return PE_OK;
}
