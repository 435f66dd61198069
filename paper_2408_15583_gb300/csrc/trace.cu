// a5: GFB-assisted multiple-bounce computation (Alg. 3, bounce loop).
//
// Rays march through the aggregated splats of every view.  Each splat lives
// at its owner pixel of one view, and every view keeps a pyramid of
// conservative bounding boxes in its own (u, v, d) frame (4x4-pixel leaves,
// 2x2 fan-out).  A coarse 3D occupancy grid gives each query the views whose
// splats lie along it and, per view, the stretch of the ray that passes
// through their cells.  A query descends each of those views' pyramids with
// the box test limited to that stretch and to t <= t_best + r, tests the splats of the leaves it reaches with
// the exact float32 ray/disk test, and finally applies Eq. 23 to the
// candidates within r of the nearest hit.  Because the boxes only cull and
// the candidate set and its selection do not depend on visiting order, the
// hit ids equal those of a brute-force search over all splats.
//
// Every pass (bounce 1 from the geometry, each later bounce, the shadow rays:
// with mb = 2 inside the bounce-2 pass) runs one warp per 8x4 tile of the
// incidence screen, one block per 128 rays; a lane is live when its ray's
// bounce count M says so.  Per-ray state lives in the last-hit records, so a ray that
// misses simply keeps its previous record.
#include <cstring>

#include "pe_internal.cuh"

namespace {

constexpr int kTraceThreads = 128;

struct march_args {
  pe_geom_layout L;
  pe_view_batch vb;
  pe_hits h;
  const unsigned long long *keys;
  const float *nrm;
  int32_t bounce;
  int32_t mb;
  int32_t implicit1;  // bounce 2 takes the bounce-1 records from the keys
  float eps;
  float r_ov;
  unsigned int *err;
  long long *stats;
};

// A ray in a view's (u, v, d) frame: reciprocal direction and -origin/dir,
// so a slab bound is one FMA.
struct vray {
  float ix, iy, iz, nx, ny, nz;
};

// A direction component for the slab form.  An exact zero (a ray
// perpendicular to a view axis, e.g. d = (0, 0, -1) against a top view)
// would give a reciprocal of +-inf, and the slab ends lo * inf - a * inf
// would be NaN or -inf: fminf/fmaxf drop the NaN and keep -inf, which
// rejects a box that holds the ray.  A magnitude of at least 1e-20 keeps
// every end finite (|a| * 1e20 is far below FLT_MAX) with the sign of
// (lo - a), so a box holding the ray spans beyond any parameter the walk
// uses; only a ray within 1e-17 m of a face sees a shorter slab, far
// inside the boxes' padding.
__device__ __forceinline__ float slab_dir(float x) {
  return fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x;
}

struct qstate {
  float tb;
  uint32_t ib;
  int nc;
  float ct[PE_MAX_CAND];
  uint32_t cid[PE_MAX_CAND];
};

// The ray's parameters inside a node's box in the view frame, within
// [t0, t1]: [tn, tf], empty when tn > tf.
__device__ __forceinline__ void box_range(float4 lo, float4 hi, const vray &r, float t0, float t1,
                                          float &tn, float &tf) {
  float ax = fmaf(lo.x, r.ix, r.nx), bx = fmaf(hi.x, r.ix, r.nx);
  float ay = fmaf(lo.y, r.iy, r.ny), by = fmaf(hi.y, r.iy, r.ny);
  float az = fmaf(lo.z, r.iz, r.nz), bz = fmaf(hi.z, r.iz, r.nz);
  tn = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), t0));
  tf = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), t1));
  if (lo.x > hi.x) tn = INFINITY;  // an empty node
}

// [tn, tf] narrowed to the parameters where the ray lies inside the node's
// slab (axis sl.xyz, heights [sl.w, shi] above the view origin; q = ray
// origin - view origin).  The fast reciprocal's relative error (2 ulp)
// moves the ends by ~1e-7 t, far inside the slab's padding; a direction
// within 1e-20 of the slab's plane keeps a finite reciprocal (slab_dir), so
// a ray along the plane is inside for all t or for none.
__device__ __forceinline__ bool slab_cut(float4 sl, float shi, pe_f3 q, pe_f3 d, float tn,
                                         float tf) {
  const float sd = sl.x * d.x + sl.y * d.y + sl.z * d.z;
  const float s0 = sl.x * q.x + sl.y * q.y + sl.z * q.z;
  const float rs = __fdividef(1.0f, slab_dir(sd));
  const float ta = (sl.w - s0) * rs, tb = (shi - s0) * rs;
  return fmaxf(tn, fminf(ta, tb)) <= fminf(tf, fmaxf(ta, tb));
}

// Whether any active lane's ray meets node `nid` (box lo/hi): the box test,
// then, for a box some lane meets, the node's slab (when it has one; the
// branch is uniform over the warp, whose lanes test the same node).
__device__ __forceinline__ bool warp_meets(const pe_geom_layout &L, int64_t nid, float4 lo,
                                           float4 hi, const vray &r, pe_f3 q, pe_f3 d, bool lv,
                                           float t0, float t1) {
  const unsigned FULL = 0xffffffffu;
  float tn, tf;
  box_range(lo, hi, r, t0, t1, tn, tf);
  bool h = lv && tn <= tf;
  if (!__any_sync(FULL, h)) return false;
  const float4 sl = __ldg(L.slab + nid);
  if (sl.w > -INFINITY) {
    const float shi = __ldg(L.slab_hi + nid);
    h = h && slab_cut(sl, shi, q, d, tn, tf);
    return __any_sync(FULL, h);
  }
  return true;
}

__device__ __forceinline__ void note_hit(qstate &S, float t, uint32_t id, float r_ov,
                                         unsigned int *err) {
  if (t < S.tb || (t == S.tb && id < S.ib)) {
    S.tb = t;
    S.ib = id;
  }
  float lim = pe_add(S.tb, r_ov);
  if (!(t <= lim)) return;
  if (S.nc == PE_MAX_CAND) {  // drop entries the shrinking limit excludes
    int k = 0;
    for (int m = 0; m < S.nc; ++m)
      if (S.ct[m] <= lim) {
        S.ct[k] = S.ct[m];
        S.cid[k] = S.cid[m];
        ++k;
      }
    S.nc = k;
  }
  if (S.nc < PE_MAX_CAND) {
    S.ct[S.nc] = t;
    S.cid[S.nc] = id;
    ++S.nc;
  } else {
    pe_raise(err, PE_ERR_OVERFLOW);
  }
}

// Views owning splats along the ray (t > tmin), from the coarse occupancy
// grid by a 3D DDA; all views when there is no grid.  The splats were marked
// in every cell their padded sphere overlaps, so a cell the ray crosses
// carries the bit of every splat it can hit there.  Per view, tv[v] gets the
// ray-parameter interval from the entry of the first to the exit of the last
// cell carrying its bit (unbounded for views marked outside the grid, empty
// for views not crossed): a hit on that view's splats lies inside it, since
// the points of the ray within the marking pad of the hit point all lie in
// marked cells.  tv is indexed [v * stride].
__device__ uint32_t view_mask(const pe_geom_layout &L, pe_f3 o, pe_f3 d, float tmin, float2 *tv,
                              int stride) {
  const int n = L.vg_n;
  for (int v = 0; v < L.nv; ++v) tv[v * stride] = make_float2(INFINITY, -INFINITY);
  if (n == 0) {
    for (int v = 0; v < L.nv; ++v) tv[v * stride] = make_float2(-INFINITY, INFINITY);
    return 0xffffffffu;
  }
  const uint32_t outside = __ldg(L.vmask + (int64_t)n * n * n);
  for (uint32_t b = outside; b; b &= b - 1) tv[(__ffs(b) - 1) * stride] = make_float2(-INFINITY, INFINITY);
  uint32_t m = outside;
  const float cell = L.vg_cell;
  const float oo[3] = {o.x - L.vg_min[0], o.y - L.vg_min[1], o.z - L.vg_min[2]};
  const float dd[3] = {d.x, d.y, d.z};
  const float size = cell * n;
  float t0 = tmin - 1e-3f * cell, t1 = INFINITY;
  float inv[3];
  for (int k = 0; k < 3; ++k) {
    // fast reciprocal: the cell boundaries it places move by ~1e-7 of t,
    // far inside the marking pad and the walk's slack
    inv[k] = __fdividef(1.0f, slab_dir(dd[k]));  // finite; exact zeros take the branch below
    float a = (0.0f - oo[k]) * inv[k], b = (size - oo[k]) * inv[k];
    if (dd[k] == 0.0f) {
      if (oo[k] < 0.0f || oo[k] > size) return m;
      continue;
    }
    t0 = fmaxf(t0, fminf(a, b));
    t1 = fminf(t1, fmaxf(a, b));
  }
  if (!(t0 <= t1)) return m;
  // the DDA state per axis in named registers (a runtime axis index into
  // small arrays would put them in local memory)
  int ix[3], st[3];
  float tmax[3], tdel[3];
  const float icell = __fdividef(1.0f, cell);
  for (int k = 0; k < 3; ++k) {
    float p = oo[k] + t0 * dd[k];
    int c = (int)floorf(p * icell);
    ix[k] = c < 0 ? 0 : (c > n - 1 ? n - 1 : c);
    if (dd[k] > 0.0f) {
      st[k] = 1;
      tmax[k] = ((ix[k] + 1) * cell - oo[k]) * inv[k];
      tdel[k] = cell * inv[k];
    } else if (dd[k] < 0.0f) {
      st[k] = -1;
      tmax[k] = (ix[k] * cell - oo[k]) * inv[k];
      tdel[k] = -cell * inv[k];
    } else {
      st[k] = 0;
      tmax[k] = INFINITY;
      tdel[k] = INFINITY;
    }
  }
  int x0 = ix[0], x1 = ix[1], x2 = ix[2];
  float m0 = tmax[0], m1 = tmax[1], m2 = tmax[2];
  const float d0 = tdel[0], d1 = tdel[1], d2 = tdel[2];
  const int s0 = st[0], s1 = st[1], s2 = st[2];
  float t_in = t0;
  bool ended = false;
  for (int it = 0; it < 3 * n + 3; ++it) {
    // the axis whose boundary comes first (ties as x < y < z order of the
    // comparisons: k = m0 < m1 ? (m0 < m2 ? 0 : 2) : (m1 < m2 ? 1 : 2))
    const bool k0 = m0 < m1 && m0 < m2;
    const bool k1 = !(m0 < m1) && m1 < m2;
    const float t_out = k0 ? m0 : (k1 ? m1 : m2);
    const int64_t cid = ((int64_t)x0 * n + x1) * n + x2;
    uint32_t b = __ldg(L.vmask + cid) & ~outside;
    float s_in = t_in, s_out = t_out;
    if (b) {
      // the cell's slab: the ray's stretch through the cell that lies inside
      // it, [s_in, s_out] (|hs + t hd| <= 1 in the slab's scaled heights);
      // a stretch outside the slab meets none of the cell's disks, so the
      // cell adds no view
      const float4 cs = __ldg(L.cslab + cid);
      const float qx = fmaf(-((float)x0 + 0.5f), cell, oo[0]);
      const float qy = fmaf(-((float)x1 + 0.5f), cell, oo[1]);
      const float qz = fmaf(-((float)x2 + 0.5f), cell, oo[2]);
      const float hs = fmaf(cs.x, qx, fmaf(cs.y, qy, fmaf(cs.z, qz, -cs.w)));
      const float hd = fmaf(cs.x, dd[0], fmaf(cs.y, dd[1], cs.z * dd[2]));
      const float r = __fdividef(1.0f, slab_dir(hd));
      const float ta = (-1.0f - hs) * r, tb = (1.0f - hs) * r;
      s_in = fmaxf(s_in, fminf(ta, tb));
      s_out = fminf(s_out, fmaxf(ta, tb));
      if (!(s_in <= s_out)) b = 0u;
    }
    for (uint32_t r = b; r; r &= r - 1) {
      const int v = __ffs(r) - 1;
      float2 &T = tv[v * stride];
      if (!((m >> v) & 1u)) T.x = s_in;
      T.y = s_out;
    }
    m |= b;
    if (t_out > t1) {
      ended = true;
      break;
    }
    if (k0) {
      x0 += s0;
      m0 = m0 + d0;
    } else if (k1) {
      x1 += s1;
      m1 = m1 + d1;
    } else {
      x2 += s2;
      m2 = m2 + d2;
    }
    if ((unsigned)x0 >= (unsigned)n || (unsigned)x1 >= (unsigned)n || (unsigned)x2 >= (unsigned)n) {
      ended = true;
      break;
    }
    t_in = t_out;
  }
  if (!ended)  // cannot happen for a line through an n^3 grid; stay conservative
    for (uint32_t r = m; r; r &= r - 1) tv[(__ffs(r) - 1) * stride].y = INFINITY;
  return m;
}

// Walk every view's pyramid with the whole warp (packet traversal).  The 32
// rays of a warp are neighbours on the ray screen, so they need nearly the
// same nodes: the warp descends the union of the nodes any active lane's
// box test accepts, box and splat data are loaded once per warp (uniform
// addresses), and each lane tests its own ray exactly.  Extra tests never
// change a lane's result (the minimum and the candidate set are
// order-independent), so hits stay bit-exact.  Per-level child masks replace
// a stack.  ANY: a lane stops at its first hit with t > tmin (shadow rays).
// Every lane of the warp must call this together.
// The walk of view v is limited to the lane's interval tv[v] from the grid,
// widened by a slack far above the rounding of both parameterisations.
// `tv` is the block's dynamic shared memory, L.nv x blockDim.x entries.
template <bool ANY>
__device__ void walk(const pe_geom_layout &L, pe_f3 o, pe_f3 d, float tmin, float r_ov,
                     bool active, qstate &S, bool &hit_any, unsigned int *err,
                     long long &n_splat, long long &n_node, long long &n_view) {
  static_assert(PE_FAN == 2, "the register-resident traversal assumes a 2x2 fan-out");
  static_assert(2 * PE_LEAF * PE_LEAF == 32, "a leaf is fetched by one warp: 16 centres + 16 normals");
  const unsigned FULL = 0xffffffffu;
  extern __shared__ float2 tv_all[];
  float2 *tv = tv_all + threadIdx.x;
  const int stride = blockDim.x;
  const uint32_t mine = active ? view_mask(L, o, d, tmin, tv, stride) : 0u;
  const uint32_t vm = __reduce_or_sync(FULL, mine);
  const uint32_t all_views = (L.nv >= 32) ? 0xffffffffu : ((1u << L.nv) - 1u);
  if (active) n_view += __popc(mine & all_views);
  const float t_slack = L.vg_n ? 1e-2f * L.vg_cell : 0.0f;
  for (int v = 0; v < L.nv; ++v) {
    if (!((vm >> v) & 1u)) continue;
    bool live = active && !(ANY && hit_any);
    if (!__any_sync(FULL, live)) return;
    const pe_view &V = L.view[v];
    const float pad = L.pad[v];
    float2 T = active ? tv[v * stride] : make_float2(INFINITY, -INFINITY);
    T.x = T.x - (t_slack + 1e-5f * fminf(fabsf(T.x), 1e30f));  // infinities stay
    T.y = T.y + (t_slack + 1e-5f * fminf(fabsf(T.y), 1e30f));
    pe_f3 q = {o.x - V.o[0], o.y - V.o[1], o.z - V.o[2]};
    // (the FMA slab form moves a face by ~1e-7 |origin|, far inside the
    // boxes' padding of 1e-5 of the view's span)
    vray r;
    // (fast reciprocals: 2 ulp, far inside the boxes' padding)
    r.ix = __fdividef(1.0f, slab_dir(d.x * V.u[0] + d.y * V.u[1] + d.z * V.u[2]));
    r.iy = __fdividef(1.0f, slab_dir(d.x * V.v[0] + d.y * V.v[1] + d.z * V.v[2]));
    r.iz = __fdividef(1.0f, slab_dir(d.x * V.d[0] + d.y * V.d[1] + d.z * V.d[2]));
    r.nx = -(q.x * V.u[0] + q.y * V.u[1] + q.z * V.u[2]) * r.ix;
    r.ny = -(q.x * V.v[0] + q.y * V.v[1] + q.z * V.v[2]) * r.iy;
    r.nz = -(q.x * V.d[0] + q.y * V.d[1] + q.z * V.d[2]) * r.iz;
    const float t0 = fmaxf(tmin - pad - 1e-6f * fabsf(tmin), T.x);
    const int top = L.nlev[v] - 1;
    const int64_t poff = L.pix_off[v];
    auto t_far = [&]() -> float {
      float lim = pe_add(S.tb, r_ov);
      return ANY ? T.y : fminf(fmaf(fabsf(lim), 1e-6f, lim) + pad, T.y);
    };
    // Start set: the nodes (sx + {0, 1}, sy + {0, 1}) of the lowest level ls
    // at which the leaf slots that a lane's ray can reach in this view span
    // at most two nodes per axis.  A ray hitting a splat passes within the
    // view's reach (root hi.w, in pixels) of the splat's slot, and the hit
    // lies on the lane's stretch [t0, T.y] of the ray, so the slots lie in
    // the projection of that stretch widened by the reach.  The warp's union
    // of those rectangles, [rx0, rx1] x [ry0, ry1] in leaf tiles, bounds the
    // start set and filters the children of every node the walk expands (a
    // node whose tiles miss it holds no splat a lane can hit).  Lanes whose
    // stretch is unbounded keep the root and the whole screen.
    const float4 rhi = __ldg(L.nodes + 2 * L.node_off[v][top] + 1);
    int ls = top, sx = 0, sy = 0;
    int rx0 = 0, ry0 = 0, rx1 = L.tw[v][0] - 1, ry1 = L.th[v][0] - 1;
    {
      const bool lv = active && !(ANY && hit_any) && T.x <= T.y;
      const bool fin = isfinite(t0) && isfinite(T.y);
      if (top > 0 && __all_sync(FULL, !lv || fin)) {
        int lx0 = 0x7fffffff, ly0 = 0x7fffffff, lx1 = -1, ly1 = -1;
        if (lv) {
          const float il = __fdividef(1.0f, V.pitch), reach = rhi.w + 2.0f;
          const float au = q.x * V.u[0] + q.y * V.u[1] + q.z * V.u[2];
          const float av = q.x * V.v[0] + q.y * V.v[1] + q.z * V.v[2];
          const float du = d.x * V.u[0] + d.y * V.u[1] + d.z * V.u[2];
          const float dv = d.x * V.v[0] + d.y * V.v[1] + d.z * V.v[2];
          const float cu = 0.5f * V.W - 0.5f, cv = 0.5f * V.H - 0.5f;
          const float u0 = fmaf(t0, du, au) * il + cu, u1 = fmaf(T.y, du, au) * il + cu;
          const float v0 = fmaf(t0, dv, av) * il + cv, v1 = fmaf(T.y, dv, av) * il + cv;
          const float tw0 = (float)L.tw[v][0], th0 = (float)L.th[v][0];
          const float fx0 = fminf(fmaxf(floorf((fminf(u0, u1) - reach) / PE_LEAF), -1.0f), tw0);
          const float fx1 = fminf(fmaxf(floorf((fmaxf(u0, u1) + reach) / PE_LEAF), -1.0f), tw0);
          const float fy0 = fminf(fmaxf(floorf((fminf(v0, v1) - reach) / PE_LEAF), -1.0f), th0);
          const float fy1 = fminf(fmaxf(floorf((fmaxf(v0, v1) + reach) / PE_LEAF), -1.0f), th0);
          // a stretch whose slots all lie off the screen reaches no splat
          if (fx1 >= 0.0f && fx0 < tw0 && fy1 >= 0.0f && fy0 < th0) {
            lx0 = (int)fmaxf(fx0, 0.0f);
            lx1 = (int)fminf(fx1, tw0 - 1.0f);
            ly0 = (int)fmaxf(fy0, 0.0f);
            ly1 = (int)fminf(fy1, th0 - 1.0f);
          }
        }
        lx0 = __reduce_min_sync(FULL, lx0);
        ly0 = __reduce_min_sync(FULL, ly0);
        lx1 = __reduce_max_sync(FULL, lx1);
        ly1 = __reduce_max_sync(FULL, ly1);
        if (lx1 < 0) continue;  // no lane reaches a slot of this view
        rx0 = lx0;
        rx1 = lx1;
        ry0 = ly0;
        ry1 = ly1;
        ls = 0;
        while (ls < top && ((lx1 >> ls) - (lx0 >> ls) > 1 || (ly1 >> ls) - (ly0 >> ls) > 1)) ++ls;
        sx = lx0 >> ls;
        sy = ly0 >> ls;
      }
    }
    // Traversal state, all in registers: `expand` asks to expand node
    // (px, py) of level l (its four children at level l-1 are box-tested
    // together; the accepted ones become pending bits [4(l-1), 4(l-1)+4) of
    // `masks`).  Otherwise the pending bits of level l < ls are children of
    // node (px, py) at level l+1, and those of level ls are the start set;
    // going up one level halves (px, py).  The walk ends when it climbs
    // above the start level.  occ4: the occupancy masks (lo.w, 16 bits each)
    // of the four nodes last tested at level 0, i.e. of the pending leaves,
    // so a leaf visit needs no reload of its node.
    uint64_t masks = 0, occ4 = 0;
    int l = ls + 1, px = 0, py = 0;
    bool expand = true;
    int leaf_x = 0, leaf_y = 0, leaf_c = 0;
    for (;;) {
      if (expand) {
        expand = false;
        const int cl = l - 1;
        const int cw = L.tw[v][cl];
        const int64_t base = L.node_off[v][cl];
        float4 blo[4], bhi[4];
        bool ex[4];
        int64_t cid[4];
        // the children (bx + {0, 1}, by + {0, 1}) that lie in the warp's
        // rectangle at this level (which also keeps them on the screen:
        // rx1 >> cl < tw[cl])
        const int bx = cl == ls ? sx : 2 * px, by = cl == ls ? sy : 2 * py;
        const int xhi = rx1 >> cl, yhi = ry1 >> cl, xlo = rx0 >> cl, ylo = ry0 >> cl;
        const bool in_x0 = bx >= xlo && bx <= xhi, in_x1 = bx + 1 >= xlo && bx + 1 <= xhi;
        const bool in_y0 = by >= ylo && by <= yhi, in_y1 = by + 1 >= ylo && by + 1 <= yhi;
        ex[0] = in_x0 && in_y0;
        ex[1] = in_x1 && in_y0;
        ex[2] = in_x0 && in_y1;
        ex[3] = in_x1 && in_y1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int cx = bx + (c & 1), cy = by + (c >> 1);
          cid[c] = base + (ex[c] ? (int64_t)cy * cw + cx : 0);
          blo[c] = __ldg(L.nodes + 2 * cid[c]);
          bhi[c] = __ldg(L.nodes + 2 * cid[c] + 1);
        }
        bool lv = active && !(ANY && hit_any);
        float t1 = t_far();
        uint32_t m = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          n_node += lv && ex[c];
          if (ex[c] && warp_meets(L, cid[c], blo[c], bhi[c], r, q, d, lv, t0, t1)) m |= 1u << c;
        }
        if (cl == 0) {
          occ4 = 0;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            occ4 |= (uint64_t)(__float_as_uint(blo[c].w) & 0xffffu) << (16 * c);
        }
        masks |= (uint64_t)m << (4 * cl);
        l = cl;
      }
      while (l <= ls && ((masks >> (4 * l)) & 0xfull) == 0) {
        ++l;
        px >>= 1;
        py >>= 1;
      }
      if (l > ls) break;
      const int c = __ffs((uint32_t)((masks >> (4 * l)) & 0xfull)) - 1;
      masks &= ~(1ull << (4 * l + c));
      const int cx = l == ls ? sx + (c & 1) : 2 * px + (c & 1);
      const int cy = l == ls ? sy + (c >> 1) : 2 * py + (c >> 1);
      if (l > 0) {
        px = cx;
        py = cy;
        expand = true;
        continue;
      }
      leaf_x = cx;
      leaf_y = cy;
      leaf_c = c;
      // leaf tile: test its splats (the occupied slots of the leaf's mask).
      // The warp fetches the whole leaf at once: lane b loads slot b's
      // centre/radius and lane 16 + b its normal (one memory round trip per
      // leaf, not one per slot); each slot is then broadcast by shuffles,
      // which move bits unchanged.  A conservative pre-test in plain float
      // arithmetic (distance of the centre to the ray line <= R, and the hit
      // parameter window [tc - R, tc + R] reaching (tmin, t_best + r]) skips
      // the exact test for splats no lane can hit; its slack covers the
      // rounding of both tests, so it never drops a hit the exact test takes.
      const int tx = leaf_x, ty = leaf_y;
      bool lv = active && !(ANY && hit_any);
      const uint32_t occ0 = (uint32_t)(occ4 >> (16 * leaf_c)) & 0xffffu;
      float4 mine = make_float4(0.f, 0.f, 0.f, 0.f);
      {
        const int lane = threadIdx.x & 31, b = lane & (PE_LEAF * PE_LEAF - 1);
        if ((occ0 >> b) & 1u) {
          const int i = tx * PE_LEAF + b % PE_LEAF, j = ty * PE_LEAF + b / PE_LEAF;
          const int64_t g = poff + (int64_t)j * V.W + i;
          mine = __ldg((lane < PE_LEAF * PE_LEAF ? L.cr : L.nf) + g);
        }
      }
      for (uint32_t occ = occ0; occ; occ &= occ - 1) {
        const int b = __ffs(occ) - 1;
        const int i = tx * PE_LEAF + b % PE_LEAF, j = ty * PE_LEAF + b / PE_LEAF;
        {
          int64_t g = poff + (int64_t)j * V.W + i;
          float4 c;
          c.x = __shfl_sync(FULL, mine.x, b);
          c.y = __shfl_sync(FULL, mine.y, b);
          c.z = __shfl_sync(FULL, mine.z, b);
          c.w = __shfl_sync(FULL, mine.w, b);
          float qx = c.x - o.x, qy = c.y - o.y, qz = c.z - o.z;
          float tc = qx * d.x + qy * d.y + qz * d.z;
          float qq = qx * qx + qy * qy + qz * qz;
          float ll = qq - tc * tc;
          float Rs = c.w * 1.0001f + 1e-3f * pad;
          float sl = 1e-5f * (fabsf(tc) + c.w) + pad;
          bool pass = lv && ll <= Rs * Rs + 1e-6f * qq && tc + Rs + sl > tmin &&
                      tc + Rs + sl >= T.x && tc - Rs - sl <= T.y;
          if (!ANY) {
            float lim = pe_add(S.tb, r_ov);
            pass = pass && tc - Rs - sl <= fmaf(fabsf(lim), 1e-6f, lim);
          }
          if (!__any_sync(FULL, pass)) continue;
          float4 n;
          n.x = __shfl_sync(FULL, mine.x, PE_LEAF * PE_LEAF + b);
          n.y = __shfl_sync(FULL, mine.y, PE_LEAF * PE_LEAF + b);
          n.z = __shfl_sync(FULL, mine.z, PE_LEAF * PE_LEAF + b);
          n.w = __shfl_sync(FULL, mine.w, PE_LEAF * PE_LEAF + b);
          if (!pass) continue;
          ++n_splat;
          float t;
          pe_f3 x, ee;
          if (!pe_hit_disk(o, d, {c.x, c.y, c.z}, {n.x, n.y, n.z}, c.w, tmin, t, x, ee)) continue;
          if (ANY) {
            hit_any = true;
            lv = false;
          } else {
            note_hit(S, t, (uint32_t)g, r_ov, err);
          }
        }
      }
      if (ANY && !__any_sync(FULL, active && !hit_any)) return;
    }
  }
}

// Eq. 23 on the final candidate set: select the hit closest to its splat's
// centre relative to R (ties: smaller t, smaller id); blend the normals in
// splat-id order with weights 1 - rho, normalise, turn against the ray.
// Every lane of the warp must call this together (inactive lanes: active=0).
__device__ bool nearest(const pe_geom_layout &L, pe_f3 o, pe_f3 d, float tmin, float r_ov,
                        bool active, unsigned int *err, pe_f3 &xo, pe_f3 &no, uint32_t &ido,
                        long long &n_splat, long long &n_node, long long &n_view) {
  qstate S;
  S.tb = INFINITY;
  S.ib = PE_NONE;
  S.nc = 0;
  bool unused = false;
  walk<false>(L, o, d, tmin, r_ov, active, S, unused, err, n_splat, n_node, n_view);
  if (!active || S.ib == PE_NONE) return false;
  float lim = pe_add(S.tb, r_ov);
  int k = 0;
  for (int m = 0; m < S.nc; ++m)
    if (S.ct[m] <= lim) S.cid[k++] = S.cid[m];
  for (int a = 1; a < k; ++a) {  // insertion sort by id
    uint32_t x = S.cid[a];
    int b = a;
    while (b > 0 && S.cid[b - 1] > x) {
      S.cid[b] = S.cid[b - 1];
      --b;
    }
    S.cid[b] = x;
  }
  pe_f3 m = {0.f, 0.f, 0.f}, nsel = {0.f, 0.f, 0.f}, xsel = {0.f, 0.f, 0.f};
  float best_rho = INFINITY, best_t = INFINITY;
  uint32_t sel = PE_NONE;
  for (int a = 0; a < k; ++a) {
    uint32_t g = S.cid[a];
    float4 c = __ldg(L.cr + g), n4 = __ldg(L.nf + g);
    float t;
    pe_f3 x, e;
    pe_hit_disk(o, d, {c.x, c.y, c.z}, {n4.x, n4.y, n4.z}, c.w, tmin, t, x, e);
    float rho = pe_div(pe_sqrt(pe_dot(e, e)), c.w);
    pe_f3 nn = {n4.x, n4.y, n4.z};
    if (pe_dot(nn, d) > 0.0f) nn = pe_neg3(nn);
    float w = pe_sub(1.0f, rho);
    m.x = pe_add(m.x, pe_mul(w, nn.x));
    m.y = pe_add(m.y, pe_mul(w, nn.y));
    m.z = pe_add(m.z, pe_mul(w, nn.z));
    if (rho < best_rho || (rho == best_rho && t < best_t)) {
      best_rho = rho;
      best_t = t;
      sel = g;
      xsel = x;
      nsel = nn;
    }
  }
  float mm = pe_dot(m, m);
  if (mm == 0.0f) {
    no = nsel;
  } else {
    float s = pe_sqrt(mm);
    no = {pe_div(m.x, s), pe_div(m.y, s), pe_div(m.z, s)};
    if (pe_dot(no, d) > 0.0f) no = pe_neg3(no);
  }
  xo = xsel;
  ido = sel;
  return true;
}

__device__ __forceinline__ double seg_len(pe_f3 a, pe_f3 b) {
  double dx = __dsub_rn((double)b.x, (double)a.x);
  double dy = __dsub_rn((double)b.y, (double)a.y);
  double dz = __dsub_rn((double)b.z, (double)a.z);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ __forceinline__ void st3(float *a, int64_t i, pe_f3 v) {
  a[3 * i] = v.x;
  a[3 * i + 1] = v.y;
  a[3 * i + 2] = v.z;
}
__device__ __forceinline__ pe_f3 ld3(const float *a, int64_t i) {
  return {a[3 * i], a[3 * i + 1], a[3 * i + 2]};
}

// Per-block partial counters: each warp adds its own, and the last warp of
// the block to finish sums them and issues one atomic per non-zero counter
// (a grid of one block per 128 rays would otherwise pile millions of atomics
// onto five addresses; no barrier at the end, so a warp done with its walk
// does not wait for the block's slowest).  stats_begin() runs first in the
// kernel, by every thread.
struct stats_acc {
  long long v[kTraceThreads / 32][5];
  unsigned int done;
};

__device__ __forceinline__ void stats_begin(stats_acc &acc) {
  if (threadIdx.x == 0) acc.done = 0u;
  __syncthreads();
}

__device__ __forceinline__ void flush_stats(long long *stats, stats_acc &acc, long long a,
                                            long long b, long long c, long long d, long long e) {
  if (!stats) return;  // a kernel argument: uniform over the block
  long long v[5] = {a, b, c, d, e};
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  unsigned int last = 0;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) acc.v[w][k] = v[k];
    __threadfence_block();
    last = atomicAdd(&acc.done, 1u) == (blockDim.x >> 5) - 1u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence_block();
  if (lane < 5) {
    long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += ((volatile long long *)acc.v[i])[lane];
    if (t) atomicAdd(reinterpret_cast<unsigned long long *>(stats + lane), (unsigned long long)t);
  }
}

// Thread t of a batch -> (view, pixel) so that each warp covers an 8x4 tile
// of one screen (neighbouring rays in a warp).
struct tile_map {
  int tiles_x, tiles_y;
  int64_t per_view_threads, n_threads;
};
__host__ __device__ __forceinline__ tile_map make_tile_map(int W, int H, int n_views) {
  tile_map m;
  m.tiles_x = (W + 7) / 8;
  m.tiles_y = (H + 3) / 4;
  m.per_view_threads = (int64_t)m.tiles_x * m.tiles_y * 32;
  m.n_threads = m.per_view_threads * n_views;
  return m;
}
__device__ __forceinline__ bool tile_pixel(const tile_map &m, int W, int H, int64_t t, int &view,
                                           int &i, int &j) {
  view = (int)(t / m.per_view_threads);
  int64_t r = t % m.per_view_threads;
  int tile = (int)(r >> 5), lane = (int)(r & 31);
  i = (tile % m.tiles_x) * 8 + (lane & 7);
  j = (tile / m.tiles_x) * 4 + (lane >> 3);
  return i < W && j < H;
}

// Bounce 1 by marching the splats from the incidence screen (the first
// bounce taken from the aggregated geometry, in 8x4 tiles for the warp's
// walk).  Writes every slot's M and Psi, and the rest of the record for the
// rays that hit.
__global__ void __launch_bounds__(kTraceThreads)
    primary_kernel(const __grid_constant__ march_args A) {
  const int W = A.vb.W, H = A.vb.H;
  const int64_t per_view = (int64_t)W * H;
  const tile_map tm = make_tile_map(W, H, A.vb.n);
  __shared__ stats_acc sacc;
  stats_begin(sacc);
  long long nq = 0, ns = 0, nn = 0, nv = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < tm.n_threads;
       base += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = base + threadIdx.x;
    int vi = 0, i = 0, j = 0;
    bool active = t < tm.n_threads && tile_pixel(tm, W, H, t, vi, i, j);
    if (!active) vi = 0;
    const pe_view &V = A.vb.v[vi];
    const int64_t slot = (int64_t)vi * per_view + (int64_t)j * W + i;
    pe_f3 o = pe_pixel_origin(V, i, j);
    pe_f3 d = pe_v3(V.d);
    pe_f3 u = {pe_mul(V.pitch, V.u[0]), pe_mul(V.pitch, V.u[1]), pe_mul(V.pitch, V.u[2])};
    pe_f3 v = {pe_mul(V.pitch, V.v[0]), pe_mul(V.pitch, V.v[1]), pe_mul(V.pitch, V.v[2])};
    bool hit = false;
    pe_f3 x = {0.f, 0.f, 0.f}, n = {0.f, 0.f, 0.f};
    uint32_t id = PE_NONE;
    nq += active;
    hit = nearest(A.L, o, d, 0.0f, A.r_ov, active, A.err, x, n, id, ns, nn, nv);
    if (active) {
      A.h.M[slot] = hit ? 1 : 0;
      A.h.psi[slot] = 1;
      if (A.h.ids) A.h.ids[slot] = id;
      // a miss (M = 0) ends the ray: nothing reads the rest of its record
      if (hit) {
        st3(A.h.p, slot, x);
        st3(A.h.n, slot, n);
        st3(A.h.k, slot, d);
        st3(A.h.u, slot, u);
        st3(A.h.v, slot, v);
        A.h.path[slot] = pe_path_start(d, x);
      }
    }
  }
  flush_stats(A.stats, sacc, nq, 0, ns, nn, nv);
}

// Bounce 1 from the incidence screen's GFB keys, one thread per slot in
// slot order: no walk, so no tiles; a warp reads 32 consecutive keys and
// writes 32 consecutive records (whole cache lines), and the kernel's few
// registers keep the SMs full of loads and stores in flight.
__global__ void __launch_bounds__(kTraceThreads)
    primary_gfb_kernel(const __grid_constant__ march_args A) {
  const int W = A.vb.W;
  const int64_t per_view = (int64_t)W * A.vb.H;
  const int64_t n = per_view * A.vb.n;
  __shared__ stats_acc sacc;
  stats_begin(sacc);
  long long nq = 0;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int vi = (int)(slot / per_view);
    const int64_t r = slot - (int64_t)vi * per_view;
    const int j = (int)(r / W), i = (int)(r - (int64_t)j * W);
    const pe_view &V = A.vb.v[vi];
    ++nq;
    const unsigned long long key = __ldcs(A.keys + slot);
    A.h.psi[slot] = 1;
    if (key == ~0ull) {
      A.h.M[slot] = 0;
      if (A.h.ids) A.h.ids[slot] = PE_NONE;
      continue;
    }
    pe_f3 x, nn, d, u, v;
    double path;
    pe_primary_record(V, i, j, key, A.nrm, x, nn, d, u, v, path);
    A.h.M[slot] = 1;
    if (A.h.ids) A.h.ids[slot] = (uint32_t)(key & 0xffffffffull);
    st3(A.h.p, slot, x);
    st3(A.h.n, slot, nn);
    st3(A.h.k, slot, d);
    st3(A.h.u, slot, u);
    st3(A.h.v, slot, v);
    A.h.path[slot] = path;
  }
  flush_stats(A.stats, sacc, nq, 0, 0, 0, 0);
}

// One bounce (b >= 2).  Threads map to slots by the same 8x4 tiles as bounce
// 1, and a lane is live when its ray hit at bounce b - 1 (M = b - 1).  A warp
// is thus always one tile of one screen: its rays are neighbours whose
// reflections stay close, so the warp's union walk is nearly each lane's own.
// (A compacted queue of live rays would mix tiles from anywhere on the
// screen into one warp; the per-lane results are the same either way.)
// Warps with no live lane only read M.  With mb = 2 this pass also runs the
// shadow rays of Psi (Eq. 14): the rays with two hits are its own hits, and
// their lanes walk from the new hit toward the receiver with an any-hit walk
// (saving a pass over every tile when few rays hit twice).
__global__ void __launch_bounds__(kTraceThreads, 8) march_kernel(const __grid_constant__ march_args A) {
  const int W = A.vb.W, H = A.vb.H;
  const int64_t per_view = (int64_t)W * H;
  const tile_map tm = make_tile_map(W, H, A.vb.n);
  const int64_t n_rays = A.h.n_rays;
  __shared__ stats_acc sacc;
  stats_begin(sacc);
  long long nq = 0, nsh = 0, ns = 0, nn = 0, nv = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < tm.n_threads;
       base += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = base + threadIdx.x;
    int vi = 0, i = 0, j = 0;
    bool active = t < tm.n_threads && tile_pixel(tm, W, H, t, vi, i, j);
    const uint32_t slot = active ? (uint32_t)((int64_t)vi * per_view + (int64_t)j * W + i) : 0u;
    // implicit bounce-1 records: the ray is live when its pixel's key holds
    // a hit, and this pass writes M and Psi of every pixel (the primary pass
    // does not run)
    const bool pix = active;
    // with mb = 2 this pass also runs the shadow rays (the rays with two
    // hits are exactly its hits); with more bounces a pass of their own
    // does (rays settle at different bounces, and one walk per warp over
    // all of them, from their stored records, measured faster)
    const bool last = A.bounce == A.mb && A.mb == 2;
    unsigned long long key = ~0ull;
    int m0 = 0;  // the ray's bounce count before this pass
    if (A.implicit1) {
      if (pix) {
        key = __ldcs(A.keys + slot);
        const bool h1 = key != ~0ull;
        A.h.M[slot] = h1 ? 1 : 0;  // raised to 2 below on a hit
        A.h.psi[slot] = 1;
        if (A.h.ids) A.h.ids[slot] = h1 ? (uint32_t)(key & 0xffffffffull) : PE_NONE;
      }
      active = pix && key != ~0ull;
      m0 = active ? 1 : 0;
      nq += pix;  // the pixel's bounce-1 lookup
    } else {
      m0 = pix ? A.h.M[slot] : 0;
      active = pix && m0 == A.bounce - 1;
    }
    if (!__any_sync(0xffffffffu, active || (last && m0 >= 2))) continue;
    pe_f3 p = {0.f, 0.f, 0.f}, n = {0.f, 0.f, 1.f}, d = {0.f, 0.f, 1.f};
    pe_f3 u = {0.f, 0.f, 0.f}, v = {0.f, 0.f, 0.f};
    if (active) {
      if (A.implicit1) {
        double path0;  // recomputed below for a hit (fewer registers live across the walk)
        pe_primary_record(A.vb.v[vi], i, j, key, A.nrm, p, n, d, u, v, path0);
      } else {
        p = ld3(A.h.p, slot);
        n = ld3(A.h.n, slot);
        d = ld3(A.h.k, slot);
        u = ld3(A.h.u, slot);
        v = ld3(A.h.v, slot);
      }
      pe_f3 rd = pe_reflect(d, n);
      float len = pe_sqrt(pe_dot(rd, rd));
      d = {pe_div(rd.x, len), pe_div(rd.y, len), pe_div(rd.z, len)};
      u = pe_reflect(u, n);
      v = pe_reflect(v, n);
    }
    pe_f3 x, n2;
    uint32_t id;
    nq += active;
    bool hit = nearest(A.L, p, d, A.eps, A.r_ov, active, A.err, x, n2, id, ns, nn, nv);
    if (hit) {
      // the bounce-1 path d . p (the primary record's, bit for bit)
      const double path0 =
          A.implicit1 ? pe_path_start(pe_v3(A.vb.v[slot / per_view].d), p) : A.h.path[slot];
      A.h.path[slot] = __dadd_rn(path0, seg_len(p, x));
      st3(A.h.p, slot, x);
      st3(A.h.n, slot, n2);
      st3(A.h.k, slot, d);
      st3(A.h.u, slot, u);
      st3(A.h.v, slot, v);
      A.h.M[slot] = A.bounce;
      if (A.h.ids) A.h.ids[(int64_t)(A.bounce - 1) * n_rays + slot] = id;
    }
    // Psi (mb = 2) of every ray with two hits: a shadow ray from its last hit
    // toward the receiver (w, the reverse of the view's direction); rays with
    // one hit keep Psi = 1.  (The general form: this pass's hit x, the origin
    // p of a ray that missed here, or the stored record of a ray settled
    // earlier.)
    const bool need = last && (hit || m0 >= 2);
    if (__any_sync(0xffffffffu, need)) {
      const pe_view &V = A.vb.v[need ? slot / per_view : 0];
      const pe_f3 w = {-V.d[0], -V.d[1], -V.d[2]};
      const pe_f3 o = hit ? x : (active ? p : (need ? ld3(A.h.p, slot) : p));
      qstate S;
      S.tb = INFINITY;
      S.ib = PE_NONE;
      S.nc = 0;
      nsh += need;
      bool blocked = false;
      walk<true>(A.L, o, w, A.eps, A.r_ov, need, S, blocked, A.err, ns, nn, nv);
      if (need) A.h.psi[slot] = blocked ? 0 : 1;
    }
  }
  flush_stats(A.stats, sacc, nq, nsh, ns, nn, nv);
}

// Psi: shadow ray from the last hit toward the receiver (monostatic: w),
// a pass of its own when mb >= 3 (with mb = 2 the march runs it).
__global__ void __launch_bounds__(kTraceThreads, 8) shadow_kernel(const __grid_constant__ march_args A) {
  const int W = A.vb.W, H = A.vb.H;
  const int64_t per_view = (int64_t)W * H;
  const tile_map tm = make_tile_map(W, H, A.vb.n);
  __shared__ stats_acc sacc;
  stats_begin(sacc);
  long long nsh = 0, ns = 0, nn = 0, nv = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < tm.n_threads;
       base += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = base + threadIdx.x;
    int vi = 0, i = 0, j = 0;
    bool active = t < tm.n_threads && tile_pixel(tm, W, H, t, vi, i, j);
    if (!active) vi = 0;
    const int64_t slot = (int64_t)vi * per_view + (int64_t)j * W + i;
    active = active && A.h.M[slot] >= 2;
    if (!__any_sync(0xffffffffu, active)) continue;
    const pe_view &V = A.vb.v[vi];
    pe_f3 w = {-V.d[0], -V.d[1], -V.d[2]};
    pe_f3 p = active ? ld3(A.h.p, slot) : pe_f3{0.f, 0.f, 0.f};
    qstate S;
    S.tb = INFINITY;
    S.ib = PE_NONE;
    S.nc = 0;
    nsh += active;
    bool blocked = false;
    walk<true>(A.L, p, w, A.eps, A.r_ov, active, S, blocked, A.err, ns, nn, nv);
    if (active) A.h.psi[slot] = blocked ? 0 : 1;
  }
  flush_stats(A.stats, sacc, 0, nsh, ns, nn, nv);
}

// Psi toward other receivers (bistatic Eq. 14): a shadow ray from each
// ray's last hit along its group's receiver direction; slots in raster order.
struct shadow_dirs_args {
  pe_geom_layout L;
  const float *p;
  const int32_t *M;
  int64_t rpg;
  int32_t n_groups;
  float eps;
  float dir[PE_MAX_BATCH][3];
  uint8_t *psi;
  unsigned int *err;
  long long *stats;
  int32_t only_bounce;  // > 0: only rays whose last hit is that bounce
};

__global__ void __launch_bounds__(kTraceThreads, 8)
    shadow_dirs_kernel(const __grid_constant__ shadow_dirs_args A) {
  const int64_t total = A.rpg * A.n_groups;
  __shared__ stats_acc sacc;
  stats_begin(sacc);
  long long nsh = 0, ns = 0, nn = 0, nv = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = base + threadIdx.x;
    const bool in = t < total;
    const bool active = in && A.M[t] >= 1 && (A.only_bounce <= 0 || A.M[t] == A.only_bounce);
    const int g = in ? (int)(t / A.rpg) : 0;
    const pe_f3 w = {A.dir[g][0], A.dir[g][1], A.dir[g][2]};
    const pe_f3 p = active ? pe_f3{A.p[3 * t], A.p[3 * t + 1], A.p[3 * t + 2]}
                           : pe_f3{0.f, 0.f, 0.f};
    qstate S;
    S.tb = INFINITY;
    S.ib = PE_NONE;
    S.nc = 0;
    nsh += active;
    bool blocked = false;
    walk<true>(A.L, p, w, A.eps, 0.0f, active, S, blocked, A.err, ns, nn, nv);
    if (in) A.psi[t] = (active && !blocked) ? 1 : 0;
  }
  flush_stats(A.stats, sacc, 0, nsh, ns, nn, nv);
}


// One block per 128 threads of the pass, no grid-stride cap: the walks of
// the bounce and shadow passes are long and live rays cluster on the
// target, so a capped grid (each warp revisiting the same tile column down
// the screen) left most warps idle while a few carried the target's tiles;
// with one warp per tile the block scheduler fills the SMs as blocks finish.
int grid_all(int64_t n) {
  int64_t b = (n + kTraceThreads - 1) / kTraceThreads;
  if (b < 1) b = 1;
  return (int)(b < 0x7fffffff ? b : 0x7fffffff);
}

// A streaming pass: enough blocks of kTraceThreads to fill every SM several
// times over, each looping over the slots with a grid stride.
int grid_stream(int64_t n) {
  static int sm = 0;
  if (!sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (sm <= 0) sm = 1;
  }
  const int64_t cap = (int64_t)sm * 16;
  const int64_t b = (n + kTraceThreads - 1) / kTraceThreads;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}


bool geom_layout(const pe_geom *g, pe_geom_layout *L) {
  if (!g || !g->blob_dev) return false;
  if (!pe_make_layout(g->n_views, g->views, L)) return false;
  size_t a, b, c, d, e, f, cs, t;
  pe_layout_offsets(*L, &a, &b, &c, &d, &e, &f, &cs, &t);
  if (g->blob_bytes < t) return false;
  char *blob = static_cast<char *>(g->blob_dev);
  L->cr = reinterpret_cast<const float4 *>(blob + a);
  L->nf = reinterpret_cast<const float4 *>(blob + b);
  L->nodes = reinterpret_cast<const float4 *>(blob + c);
  L->vmask = reinterpret_cast<const uint32_t *>(blob + d);
  L->slab = reinterpret_cast<const float4 *>(blob + e);
  L->slab_hi = reinterpret_cast<const float *>(blob + f);
  L->cslab = reinterpret_cast<const float4 *>(blob + cs);
  if (g->vgrid_n == PE_VGRID && g->vgrid_cell > 0.0f) {
    L->vg_n = g->vgrid_n;
    L->vg_cell = g->vgrid_cell;
    for (int k = 0; k < 3; ++k) L->vg_min[k] = g->vgrid_min[k];
  } else {
    L->vg_n = 0;      // no grid: every view is walked
  }
  return true;
}

}  // namespace

pe_status pe_launch_trace(const pe_view_batch &vb, const unsigned long long *keys,
                          const float *nrm, const pe_geom *geom, int32_t mb,
                          const pe_params &prm, const pe_hits &h, int64_t *stats,
                          cudaStream_t s, bool implicit1) {
  march_args A;
  memset(&A, 0, sizeof(A));
  bool have_geom = geom != nullptr;
  if (have_geom && !geom_layout(geom, &A.L))
    return pe_fail(PE_EINVAL, "trace: invalid geometry (views or blob size)");
  if (!have_geom && (mb > 1 || prm.first_bounce_from_geom))
    return pe_fail(PE_EINVAL, "trace: bounces beyond the first need the aggregated geometry");
  A.vb = vb;
  A.h = h;
  A.keys = keys;
  A.nrm = nrm;
  A.mb = mb;
  A.eps = prm.eps;
  A.r_ov = prm.overlap_r;
  A.err = pe_err_word();
  A.stats = reinterpret_cast<long long *>(stats);
  const int64_t n_rays = (int64_t)vb.W * vb.H * vb.n;
  if (h.ids) PE_TRY_CUDA(cudaMemsetAsync(h.ids, 0xff, sizeof(uint32_t) * n_rays * mb, s));
  A.bounce = 1;
  implicit1 = implicit1 && mb >= 2 && !prm.first_bounce_from_geom && have_geom;
  const int64_t n_thr = make_tile_map(vb.W, vb.H, vb.n).n_threads;
  // per-lane ray intervals of every view (walk's shared memory)
  const size_t tv_bytes = have_geom ? (size_t)A.L.nv * kTraceThreads * sizeof(float2) : 0;
  if (implicit1) {
    // no bounce-1 records: the bounce-2 pass takes them from the keys
  } else if (prm.first_bounce_from_geom) {
    pe_event_before("primary_kernel", s);
    primary_kernel<<<grid_all(n_thr), kTraceThreads, tv_bytes, s>>>(A);
    pe_event_after("primary_kernel", s);
    PE_TRY_LAUNCH("primary_kernel");
  } else {
    pe_event_before("primary_kernel", s);
    primary_gfb_kernel<<<grid_stream(n_rays), kTraceThreads, 0, s>>>(A);
    pe_event_after("primary_kernel", s);
    PE_TRY_LAUNCH("primary_gfb_kernel");
  }
  for (int b = 2; b <= mb; ++b) {
    A.bounce = b;
    A.implicit1 = implicit1 && b == 2;
    pe_event_before("march_kernel", s);
    march_kernel<<<grid_all(n_thr), kTraceThreads, tv_bytes, s>>>(A);
    pe_event_after("march_kernel", s);
    PE_TRY_LAUNCH("march_kernel");
  }
  if (mb >= 3) {  // (with mb = 2 the march ran the shadow rays)
    pe_event_before("shadow_kernel", s);
    shadow_kernel<<<grid_all(n_thr), kTraceThreads, tv_bytes, s>>>(A);
    pe_event_after("shadow_kernel", s);
    PE_TRY_LAUNCH("shadow_kernel");
  }
  return PE_OK;
}

pe_status pe_launch_shadow_dirs(const pe_geom *geom, const pe_hits &h, int32_t n_groups,
                                int64_t rpg, const float *dirs, float eps, int32_t only_bounce,
                                uint8_t *psi, int64_t *stats, cudaStream_t s) {
  if (n_groups < 1 || n_groups > PE_MAX_BATCH || rpg < 1)
    return pe_fail(PE_EINVAL, "shadow: 1..%d groups", PE_MAX_BATCH);
  shadow_dirs_args A;
  memset(&A, 0, sizeof(A));
  if (!geom_layout(geom, &A.L)) return pe_fail(PE_EINVAL, "shadow: invalid geometry");
  A.p = h.p;
  A.M = h.M;
  A.rpg = rpg;
  A.n_groups = n_groups;
  A.eps = eps;
  for (int g = 0; g < n_groups; ++g)
    for (int k = 0; k < 3; ++k) A.dir[g][k] = dirs[3 * g + k];
  A.psi = psi;
  A.err = pe_err_word();
  A.stats = reinterpret_cast<long long *>(stats);
  A.only_bounce = only_bounce;
  const size_t tv_bytes = (size_t)A.L.nv * kTraceThreads * sizeof(float2);
  shadow_dirs_kernel<<<grid_all(rpg * n_groups), kTraceThreads, tv_bytes, s>>>(A);
  PE_TRY_LAUNCH("shadow_dirs_kernel");
  return PE_OK;
}

extern "C" size_t pe_trace_workspace(int32_t n_views, const pe_view *views) {
  if (n_views < 1 || !views) return 0;
  return 256;  // nothing beyond the record buffers is needed at present
}

extern "C" pe_status pe_trace_bounces(const pe_view *views, int32_t n_views,
                                      const uint64_t *keys, const float *nrm,
                                      const pe_geom *geom, int32_t max_bounces,
                                      const pe_params *prm, void *ws, size_t ws_bytes,
                                      const pe_hits *hits, int64_t *stats, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!views || n_views < 1 || n_views > PE_MAX_BATCH || !prm || !hits)
    return pe_fail(PE_EINVAL, "pe_trace_bounces: bad arguments");
  for (int i = 1; i < n_views; ++i)
    if (views[i].W != views[0].W || views[i].H != views[0].H)
      return pe_fail(PE_EINVAL, "pe_trace_bounces: all screens must share W x H");
  if (max_bounces < 1 || max_bounces > 64)
    return pe_fail(PE_EINVAL, "pe_trace_bounces: max_bounces in [1, 64]");
  int64_t n_rays = (int64_t)views[0].W * views[0].H * n_views;
  if (n_rays >= (int64_t)PE_NONE) return pe_fail(PE_EINVAL, "pe_trace_bounces: too many rays");
  if (hits->n_rays != n_rays || !hits->p || !hits->n || !hits->k || !hits->u || !hits->v ||
      !hits->path || !hits->M || !hits->psi)
    return pe_fail(PE_EINVAL, "pe_trace_bounces: hits must hold n_views*W*H records");
  if (!prm->first_bounce_from_geom && (!keys || !nrm))
    return pe_fail(PE_EINVAL, "pe_trace_bounces: bounce 1 from the GFB needs keys and nrm");
  size_t need = pe_trace_workspace(n_views, views);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_trace_bounces: workspace needs %zu bytes", need);
  pe_view_batch vb;
  memset(&vb, 0, sizeof(vb));
  vb.n = n_views;
  vb.W = views[0].W;
  vb.H = views[0].H;
  for (int i = 0; i < n_views; ++i) vb.v[i] = views[i];
  pe_hits h = *hits;
  h.max_bounces = max_bounces;
  return pe_launch_trace(vb, reinterpret_cast<const unsigned long long *>(keys), nrm, geom,
                         max_bounces, *prm, h, stats, s);
}
