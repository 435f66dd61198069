// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstddef>

#include "pointemray.h"

#define PE_MAX_LEVELS 12
#define PE_LEAF 4          // leaf tile edge in pixels
#ifndef PE_FAN
#define PE_FAN 2           // tiles per pyramid level edge
#endif
#define PE_NONE 0xFFFFFFFFu

// Device error word bits (pe_stream_check maps them to pe_status).
#define PE_ERR_OVERFLOW 1u
#define PE_ERR_TIMEOUT 2u

// ---------------------------------------------------------------------------
// Host helpers (defined in api.cu)
// ---------------------------------------------------------------------------
pe_status pe_fail(pe_status s, const char *fmt, ...);
unsigned int *pe_err_word();  // device address of the error word, current device

#define PE_TRY_CUDA(call)                                                    \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return pe_fail(PE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

void pe_count_launch();
// Diagnostic event pairs around a named kernel's launches (api.cu).
void pe_event_before(const char *kernel, cudaStream_t s);
void pe_event_after(const char *kernel, cudaStream_t s);

#define PE_TRY_LAUNCH(what)                                                  \
  do {                                                                       \
    pe_count_launch();                                                       \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess)                                                   \
      return pe_fail(PE_ECUDA, "%s launch: %s", what, cudaGetErrorString(e_)); \
  } while (0)

// Bump allocator over a caller buffer (base may be null to measure).
struct pe_carve {
  char *base;
  size_t off;
  template <class T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
  size_t bytes() const { return (off + 255) & ~size_t(255); }
};

inline bool pe_aligned(const void *p, size_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// ---------------------------------------------------------------------------
// Views of a batch (kernel parameter, passed __grid_constant__)
// ---------------------------------------------------------------------------
struct pe_view_batch {
  int32_t n;
  int32_t W, H;            // common screen size (all views of the batch)
  pe_view v[PE_MAX_BATCH];
};

// Geometry layout: splat planes and bounding pyramids of the aggregated views.
struct pe_geom_layout {
  int32_t nv;
  pe_view view[PE_MAX_VIEWS];
  int64_t pix_off[PE_MAX_VIEWS + 1];
  int32_t nlev[PE_MAX_VIEWS];
  int32_t tw[PE_MAX_VIEWS][PE_MAX_LEVELS];
  int32_t th[PE_MAX_VIEWS][PE_MAX_LEVELS];
  int64_t node_off[PE_MAX_VIEWS][PE_MAX_LEVELS];  // in nodes (2 float4 each)
  int64_t n_nodes;
  float pad[PE_MAX_VIEWS];  // absolute box padding per view (metres)
  const float4 *cr;         // splat centre, radius
  const float4 *nf;         // splat normal, count
  const float4 *nodes;      // [n_nodes][2] lo, hi in (u, v, d) frame
  // [n_nodes]: a slab bounding every disk below the node, {axis, lower
  // bound} with the upper bound in slab_hi; heights n . (x - view origin);
  // lower bound -inf: no slab for that node
  const float4 *slab;
  const float *slab_hi;
  // coarse view-occupancy grid: vmask[(ix*n + iy)*n + iz], vmask[n^3] = views
  // with splats outside the grid; n = 0: no grid (walk every view)
  const uint32_t *vmask;
  // per cell of that grid, a slab bounding every disk the cell's mask counts:
  // {axis / h, mid / h} with heights axis . (x - cell centre) within mid +- h
  // (padded); a point x of those disks has |cslab.xyz . (x - centre) -
  // cslab.w| <= 1.  All zeros: no slab (every point passes).
  const float4 *cslab;
  float vg_min[3];
  float vg_cell;
  int32_t vg_n;
};

// Fills everything but the pointers; returns false on bad views.
bool pe_make_layout(int32_t nv, const pe_view *views, pe_geom_layout *L);

// Exclusive scan of n uint32 into out[0..n] (out[n] = total), n <= 2^24;
// tile holds (n + 4095) / 4096 entries of scratch.
pe_status pe_exclusive_scan_u32(const uint32_t *in, int64_t n, uint32_t *tile, uint32_t *out,
                                cudaStream_t s);
// Blob byte offsets of the arrays for a layout.
void pe_layout_offsets(const pe_geom_layout &L, size_t *off_cr, size_t *off_nf,
                       size_t *off_nodes, size_t *off_vmask, size_t *off_slab,
                       size_t *off_slab_hi, size_t *off_cslab, size_t *total);

// ---------------------------------------------------------------------------
// Launchers shared between entry points
// ---------------------------------------------------------------------------
// Splat into keys (set to all ones by the caller).  Surfel mode with hz
// (pe_splat_tiles(n_views, W, H) floats of scratch) runs the two-pass splat
// that skips back-facing disks hidden behind the first pass's keys; hz =
// null: one pass.
size_t pe_splat_tiles(int32_t n_views, int32_t W, int32_t H);
// stats (nullable): [5] += exact pixel tests, [6] += key updates.  order
// (nullable): the processing order of the points (a permutation of 0..n-1);
// the keys do not depend on it.
pe_status pe_launch_splat(const pe_view_batch &vb, const float *pos, const float *nrm,
                          const float *rad, int64_t n, int mode, float delta, float *hz,
                          unsigned long long *keys, int64_t *stats, cudaStream_t s,
                          const uint32_t *order = nullptr);

// implicit1 (bounce 1 from the GFB keys, mb >= 2): no bounce-1 records are
// written; the bounce-2 pass takes each ray's bounce-1 record from its key
// and writes M and Psi of every slot (the records of later hits as usual).
pe_status pe_launch_trace(const pe_view_batch &vb, const unsigned long long *keys,
                          const float *nrm, const pe_geom *geom, int32_t mb,
                          const pe_params &prm, const pe_hits &h,
                          int64_t *stats, cudaStream_t s, bool implicit1 = false);

// Psi toward receiver direction dirs[g] (host [n_groups][3]) for every slot
// of group g (rays_per_group consecutive slots): 1 unless a splat is hit from
// the slot's last hit (M >= 1; M == only_bounce if only_bounce > 0) along
// dirs[g] with t > eps; 0 for the other slots.
pe_status pe_launch_shadow_dirs(const pe_geom *geom, const pe_hits &h, int32_t n_groups,
                                int64_t rays_per_group, const float *dirs, float eps,
                                int32_t only_bounce, uint8_t *psi, int64_t *stats,
                                cudaStream_t s);
size_t pe_po_ws_bytes(int32_t n_groups, int64_t rays_per_group, int32_t n_freq);
// Bounce-1 records held implicitly by the incidence GFB (pe_rcs_sweep): a
// slot whose last hit is bounce 1 (M == 1) takes its record from its key
// (pe_primary_record) instead of the record arrays, which then hold only the
// records of later bounces.  views: host, one per group of the launch, each
// group's slots in raster order (rays_per_group = W * H).
struct pe_gfb_src {
  const unsigned long long *keys;  // device [n_groups][W * H]
  const float *nrm;                // device point normals [n][3]
  const pe_view *views;            // host [n_groups]
};

// stats (nullable): [7] += contributing rays x frequencies (the Eq. 14 terms).
pe_status pe_launch_po(const pe_hits &h, int32_t n_groups, int64_t rays_per_group,
                       const float *ks, const double *freqs, int32_t n_freq, void *ws,
                       size_t ws_bytes, double *E, cudaStream_t s, int64_t *stats = nullptr,
                       const pe_gfb_src *gfb1 = nullptr);

// ---------------------------------------------------------------------------
// Device helpers: IEEE binary32 without contraction, left to right.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
struct pe_f3 {
  float x, y, z;
};
__device__ __forceinline__ float pe_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float pe_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float pe_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float pe_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float pe_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float pe_dot(pe_f3 a, pe_f3 b) {
  return pe_add(pe_add(pe_mul(a.x, b.x), pe_mul(a.y, b.y)), pe_mul(a.z, b.z));
}
__device__ __forceinline__ pe_f3 pe_sub3(pe_f3 a, pe_f3 b) {
  return {pe_sub(a.x, b.x), pe_sub(a.y, b.y), pe_sub(a.z, b.z)};
}
// o + t d
__device__ __forceinline__ pe_f3 pe_ray_at(pe_f3 o, float t, pe_f3 d) {
  return {pe_add(o.x, pe_mul(t, d.x)), pe_add(o.y, pe_mul(t, d.y)),
          pe_add(o.z, pe_mul(t, d.z))};
}
__device__ __forceinline__ pe_f3 pe_neg3(pe_f3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ pe_f3 pe_v3(const float *p) { return {p[0], p[1], p[2]}; }

// Centre of pixel (i, j): ((o + a u) + b v), a = ((i + 0.5) - W/2) L.
__device__ __forceinline__ pe_f3 pe_pixel_origin(const pe_view &V, int i, int j) {
  float fi = pe_sub(pe_add((float)i, 0.5f), pe_mul(0.5f, (float)V.W));
  float fj = pe_sub(pe_add((float)j, 0.5f), pe_mul(0.5f, (float)V.H));
  float a = pe_mul(fi, V.pitch), b = pe_mul(fj, V.pitch);
  return {pe_add(pe_add(V.o[0], pe_mul(a, V.u[0])), pe_mul(b, V.v[0])),
          pe_add(pe_add(V.o[1], pe_mul(a, V.u[1])), pe_mul(b, V.v[1])),
          pe_add(pe_add(V.o[2], pe_mul(a, V.u[2])), pe_mul(b, V.v[2]))};
}

// Ray o + t d against a two-sided disk (c, n, R): plane not parallel, hit
// point inside the disk, t > tmin.  Returns t (and x, e = x - c) on a hit.
__device__ __forceinline__ bool pe_hit_disk(pe_f3 o, pe_f3 d, pe_f3 c, pe_f3 n, float R,
                                            float tmin, float &t, pe_f3 &x, pe_f3 &e) {
  float den = pe_dot(d, n);
  if (den == 0.0f) return false;
  pe_f3 q = pe_sub3(c, o);
  t = pe_div(pe_dot(q, n), den);
  x = pe_ray_at(o, t, d);
  e = pe_sub3(x, c);
  if (!(pe_dot(e, e) <= pe_mul(R, R))) return false;
  if (!(t > tmin)) return false;
  return true;
}

// Image-method path length at the first hit, k . p in FP64.
__device__ __forceinline__ double pe_path_start(pe_f3 d, pe_f3 p) {
  return __dadd_rn(__dadd_rn(__dmul_rn((double)d.x, (double)p.x), __dmul_rn((double)d.y, (double)p.y)),
                   __dmul_rn((double)d.z, (double)p.z));
}

// The bounce-1 record of pixel (i, j) of view V from its GFB key (a hit:
// key != ~0): hit point at the key's depth along the pixel's ray, the key
// point's normal turned against the ray, incoming direction d, tube vectors
// pitch u and pitch v, path d . p.  The one definition of those values:
// written by the primary pass, or recomputed from the key where the records
// are implicit, bit for bit the same.  pe_primary_geom: the record without
// its path.
__device__ __forceinline__ void pe_primary_geom(const pe_view &V, int i, int j,
                                                unsigned long long key,
                                                const float *__restrict__ nrm, pe_f3 &p,
                                                pe_f3 &n, pe_f3 &k, pe_f3 &u, pe_f3 &v) {
  const pe_f3 o = pe_pixel_origin(V, i, j);
  k = pe_v3(V.d);
  const uint32_t id = (uint32_t)(key & 0xffffffffull);
  p = pe_ray_at(o, __uint_as_float((uint32_t)(key >> 32)), k);
  n = {__ldg(nrm + 3 * (int64_t)id), __ldg(nrm + 3 * (int64_t)id + 1),
       __ldg(nrm + 3 * (int64_t)id + 2)};
  if (pe_dot(n, k) > 0.0f) n = pe_neg3(n);
  u = {pe_mul(V.pitch, V.u[0]), pe_mul(V.pitch, V.u[1]), pe_mul(V.pitch, V.u[2])};
  v = {pe_mul(V.pitch, V.v[0]), pe_mul(V.pitch, V.v[1]), pe_mul(V.pitch, V.v[2])};
}
__device__ __forceinline__ void pe_primary_record(const pe_view &V, int i, int j,
                                                  unsigned long long key,
                                                  const float *__restrict__ nrm, pe_f3 &p,
                                                  pe_f3 &n, pe_f3 &k, pe_f3 &u, pe_f3 &v,
                                                  double &path) {
  pe_primary_geom(V, i, j, key, nrm, p, n, k, u, v);
  path = pe_path_start(k, p);
}

// Reflection a - (2 (a . n)) n (Eq. 4; also H and the tube vectors).
__device__ __forceinline__ pe_f3 pe_reflect(pe_f3 a, pe_f3 n) {
  float s = pe_mul(2.0f, pe_dot(a, n));
  return {pe_sub(a.x, pe_mul(s, n.x)), pe_sub(a.y, pe_mul(s, n.y)),
          pe_sub(a.z, pe_mul(s, n.z))};
}

__device__ __forceinline__ void pe_raise(unsigned int *err, unsigned int bit) {
  if (err) atomicOr(err, bit);
}
#endif
