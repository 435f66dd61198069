// Between GFBs and the learned completion network (a8):
//   pe_learned_pairs  coarse tube-mode depth keys (Alg. 1) -> normalised network
//                     input; dense surfel GFB -> depth / normal (uvw frame,
//                     Sec. III-A) / mask targets;
//   pe_gfb_hits       a GFB (network output or coarse depth) -> the last-hit
//                     records the PO sum reads (single bounce, Sec. III-A:
//                     "insert depth, normal and intersection indicator into
//                     Eq. 14").  Without normals, Eq. 16 gives them from depth.
// Depth is normalised per view as (t - t_near) / t_scale.
#include <cuda_bf16.h>

#include <cstring>

#include "pe_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace {

struct io_views {
  int32_t n, W, H;
  pe_view v[PE_MAX_BATCH];
  float t_near[PE_MAX_BATCH], t_scale[PE_MAX_BATCH];
};

__global__ void pairs_kernel(const __grid_constant__ io_views V, const unsigned long long *keys,
                             const float4 *nd, bf16 *x, float *d_gt, float *n_gt, float *m_gt) {
  const int64_t per = (int64_t)V.W * V.H, total = per * V.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / per);
    const float tn = V.t_near[a], ts = V.t_scale[a];
    if (keys && x) {
      unsigned long long k = keys[t];
      float dep = k == ~0ull ? 0.0f : (__uint_as_float((uint32_t)(k >> 32)) - tn) / ts;
      x[t] = __float2bfloat16_rn(dep);
    }
    if (nd) {
      float4 q = nd[t];
      bool hit = isfinite(q.w);
      const pe_view &vw = V.v[a];
      if (d_gt) d_gt[t] = hit ? (q.w - tn) / ts : 0.0f;
      if (m_gt) m_gt[t] = hit ? 1.0f : 0.0f;
      if (n_gt) {
        float nu = 0.f, nv = 0.f, nw = 0.f;
        if (hit) {
          nu = q.x * vw.u[0] + q.y * vw.u[1] + q.z * vw.u[2];
          nv = q.x * vw.v[0] + q.y * vw.v[1] + q.z * vw.v[2];
          nw = -(q.x * vw.d[0] + q.y * vw.d[1] + q.z * vw.d[2]);
        }
        n_gt[3 * t] = nu;
        n_gt[3 * t + 1] = nv;
        n_gt[3 * t + 2] = nw;
      }
    }
  }
}

__global__ void gfb_hits_kernel(const __grid_constant__ io_views V, const float *depth,
                                const float *maskv, float thresh, const float *nuvw, pe_hits h) {
  const int W = V.W, H = V.H;
  const int64_t per = (int64_t)W * H, total = per * V.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / per);
    const int64_t p = t % per;
    const int i = (int)(p % W), j = (int)(p / W);
    const pe_view &vw = V.v[a];
    const float tn = V.t_near[a], ts = V.t_scale[a];
    const bool hit = maskv[t] > thresh;
    const float L = vw.pitch;
    pe_f3 u = {L * vw.u[0], L * vw.u[1], L * vw.u[2]};
    pe_f3 v = {L * vw.v[0], L * vw.v[1], L * vw.v[2]};
    pe_f3 d = {vw.d[0], vw.d[1], vw.d[2]};
    pe_f3 x = {0.f, 0.f, 0.f}, n = {0.f, 0.f, 0.f};
    if (hit) {
      float tt = tn + ts * depth[t];
      pe_f3 o = pe_pixel_origin(vw, i, j);
      x = {o.x + tt * d.x, o.y + tt * d.y, o.z + tt * d.z};
      float cu, cv, cw;
      if (nuvw) {
        cu = nuvw[3 * t];
        cv = nuvw[3 * t + 1];
        cw = nuvw[3 * t + 2];
      } else {
        // Eq. 16: n ~ w + t_u u + t_v v with t_u, t_v the depth derivatives
        // (central differences where both neighbours are hits, else one-sided)
        auto dep = [&](int ii, int jj, float &out) -> bool {
          if (ii < 0 || jj < 0 || ii >= W || jj >= H) return false;
          int64_t q = a * per + (int64_t)jj * W + ii;
          if (!(maskv[q] > thresh)) return false;
          out = tn + ts * depth[q];
          return true;
        };
        float l, r, dn, up;
        bool hl = dep(i - 1, j, l), hr = dep(i + 1, j, r), hd = dep(i, j - 1, dn), hu = dep(i, j + 1, up);
        float tu = 0.f, tv = 0.f;
        if (hl && hr) tu = (r - l) / (2.f * L);
        else if (hr) tu = (r - tt) / L;
        else if (hl) tu = (tt - l) / L;
        if (hd && hu) tv = (up - dn) / (2.f * L);
        else if (hu) tv = (up - tt) / L;
        else if (hd) tv = (tt - dn) / L;
        cu = tu;
        cv = tv;
        cw = 1.0f;
      }
      n = {cu * vw.u[0] + cv * vw.v[0] - cw * vw.d[0], cu * vw.u[1] + cv * vw.v[1] - cw * vw.d[1],
           cu * vw.u[2] + cv * vw.v[2] - cw * vw.d[2]};
      float nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
      if (nn > 0.f) {
        n = {n.x / nn, n.y / nn, n.z / nn};
        if (n.x * d.x + n.y * d.y + n.z * d.z > 0.f) n = {-n.x, -n.y, -n.z};
      } else {
        n = {-d.x, -d.y, -d.z};
      }
    }
    h.M[t] = hit ? 1 : 0;
    h.psi[t] = 1;
    float *pp = h.p + 3 * t, *np = h.n + 3 * t, *kp = h.k + 3 * t, *up_ = h.u + 3 * t, *vp = h.v + 3 * t;
    pp[0] = x.x; pp[1] = x.y; pp[2] = x.z;
    np[0] = n.x; np[1] = n.y; np[2] = n.z;
    kp[0] = d.x; kp[1] = d.y; kp[2] = d.z;
    up_[0] = u.x; up_[1] = u.y; up_[2] = u.z;
    vp[0] = v.x; vp[1] = v.y; vp[2] = v.z;
    h.path[t] = hit ? (double)d.x * x.x + (double)d.y * x.y + (double)d.z * x.z : 0.0;
  }
}

bool fill_views(io_views &V, const pe_view *views, int32_t n, const float *t_near,
                const float *t_scale) {
  if (!views || n < 1 || n > PE_MAX_BATCH || !t_near || !t_scale) return false;
  memset(&V, 0, sizeof(V));
  V.n = n;
  V.W = views[0].W;
  V.H = views[0].H;
  for (int i = 0; i < n; ++i) {
    if (views[i].W != V.W || views[i].H != V.H || !(t_scale[i] > 0)) return false;
    V.v[i] = views[i];
    V.t_near[i] = t_near[i];
    V.t_scale[i] = t_scale[i];
  }
  return true;
}

int grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

extern "C" pe_status pe_learned_pairs(const pe_view *views, int32_t n_views, const float *t_near,
                                      const float *t_scale, const uint64_t *tube_keys,
                                      const float *surfel_nd, void *x_bf16, float *d_gt,
                                      float *n_gt, float *m_gt, void *stream) {
  io_views V;
  if (!fill_views(V, views, n_views, t_near, t_scale))
    return pe_fail(PE_EINVAL, "pe_learned_pairs: bad views or normalisation");
  if (!(tube_keys && x_bf16) && !surfel_nd) return pe_fail(PE_EINVAL, "pe_learned_pairs: nothing to do");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pairs_kernel<<<grid_n((int64_t)V.W * V.H * n_views), 256, 0, s>>>(
      V, reinterpret_cast<const unsigned long long *>(tube_keys),
      reinterpret_cast<const float4 *>(surfel_nd), static_cast<bf16 *>(x_bf16), d_gt, n_gt, m_gt);
  PE_TRY_LAUNCH("pairs_kernel");
  return PE_OK;
}

extern "C" pe_status pe_gfb_hits(const pe_view *views, int32_t n_views, const float *t_near,
                                 const float *t_scale, const float *depth, const float *mask,
                                 float threshold, const float *normal_uvw, const pe_hits *hits,
                                 void *stream) {
  io_views V;
  if (!fill_views(V, views, n_views, t_near, t_scale))
    return pe_fail(PE_EINVAL, "pe_gfb_hits: bad views or normalisation");
  if (!depth || !mask || !hits || hits->n_rays < (int64_t)V.W * V.H * n_views || !hits->p ||
      !hits->n || !hits->k || !hits->u || !hits->v || !hits->path || !hits->M || !hits->psi)
    return pe_fail(PE_EINVAL, "pe_gfb_hits: bad buffers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gfb_hits_kernel<<<grid_n((int64_t)V.W * V.H * n_views), 256, 0, s>>>(V, depth, mask, threshold,
                                                                       normal_uvw, *hits);
  PE_TRY_LAUNCH("gfb_hits_kernel");
  return PE_OK;
}
