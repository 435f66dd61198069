/*
 * pointemray.h -- C ABI of the GB300 (sm_103a) SBR-on-points library.
 *
 * The library implements the data-parallel path of PointEMRay (Yang, Liu, Yu,
 * Cui, arXiv 2408.15583): screen-based point-ray intersection that splats
 * oriented points into geometric frame buffers (GFBs), GFB-assisted multiple
 * bounce computation, and the physical-optics (PO) field sum that gives the
 * radar cross section (RCS) of a PEC target under plane-wave excitation.
 *
 * Conventions (every entry point):
 *   - Pointers named *_dev are DEVICE pointers owned by the caller; pointers
 *     without the suffix are HOST pointers read during the call only.  The
 *     library never allocates or frees caller-visible memory; scratch memory
 *     is the caller's `ws` buffer of at least the size the matching
 *     *_workspace() query returns (256-byte aligned).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is asynchronous on `stream`.  Argument errors are
 *     returned synchronously; device-side conditions (candidate-list
 *     overflow, bounded waits that timed out) are reported by
 *     pe_stream_check().  No C++ exception crosses the ABI.
 *   - Arrays are row-major.  Points are float32 [N][3] (x,y,z).  A view's
 *     pixel (i, j) (column i along u, row j along v) has linear index
 *     j * W + i.  Several views are stored back to back in view order.
 *   - Float arithmetic that decides a hit (ray/disk tests, depth keys,
 *     reflections, Eq. 23) follows one fixed IEEE-754 binary32 operation order
 *     without contraction, so hit indices and bounce counts are reproducible
 *     bit for bit and independent of launch configuration.
 *   - Calls on different streams may run concurrently; they share the
 *     device-side error word read by pe_stream_check().
 */
#ifndef POINTEMRAY_H
#define POINTEMRAY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PE_ABI_VERSION 1
#define PE_MAX_VIEWS 16       /* views per aggregated geometry            */
#define PE_MAX_BATCH 64       /* views (angles) per pe_build_gfb call      */
#define PE_MAX_CAND 64        /* Eq. 23 overlap candidates kept per query  */

typedef enum {
  PE_OK = 0,
  PE_EINVAL = 1,        /* bad argument (null pointer, size, alignment)    */
  PE_ENOMEM = 2,        /* workspace smaller than the query returned        */
  PE_ECUDA = 3,         /* a CUDA runtime call failed (see pe_last_error)   */
  PE_ETIMEOUT = 4,      /* a bounded device wait gave up                    */
  PE_EOVERFLOW = 5,     /* a fixed-capacity device list overflowed          */
  PE_EUNSUPPORTED = 6   /* valid request outside what the library supports */
} pe_status;

/* An orthographic ray screen (the paper's uvwo frame, Sec. III-A around
 * Eq. 15-16): u, v, w orthonormal with u x v = w, w pointing from the target
 * toward the transmitter.  `o` is the screen centre, placed outside the
 * target; rays leave pixel centres o + a u + b v along d = -w, where
 * a = ((i + 0.5) - W/2) * pitch and b = ((j + 0.5) - H/2) * pitch.
 * All values are float32 (hosts compute them in FP64 and round once). */
typedef struct {
  float o[3], u[3], v[3], d[3];
  float pitch;
  int32_t W, H;
} pe_view;

/* Method parameters (values the paper leaves open are chosen by the caller).
 *   delta      ray-tube radius of Alg. 1 (tube mode), metres;
 *   eps        minimum travel distance of reflected rays (Sec. III-B, Fig. 4b);
 *   overlap_r  radius r of the Eq. 23 overlap sphere, metres;
 *   edge_tau   edge rule (edge_mode 0): a GFB pixel is an edge if a
 *              4-neighbour is outside the image or empty, or differs in depth
 *              by more than edge_tau * pitch;
 *   fuse_grid  voxel grid size G of the fusion step (Sec. III-B: 256);
 *   bbox_min   voxel grid origin (float32), inv_voxel = G / (longest bbox edge)
 *              as float32 (finite and > 0: a point set of zero extent has no
 *              grid, and pe_aggregate_views returns PE_EINVAL);
 *   first_bounce_from_geom  0: bounce 1 from the incidence view's GFB
 *              (PO path of Sec. III-A); 1: bounce 1 traced against the
 *              aggregated splats as in Alg. 3;
 *   edge_mode  0: the edge rule above; 1: a Canny filter on each view's depth
 *              map (the paper's choice, Sec. III-B): 5x5 binomial smoothing,
 *              Sobel gradient, suppression across the gradient, thresholds
 *              8 edge_tau pitch (high) and half of it (low), hysteresis over 8
 *              neighbours; a pixel next to the image border or an empty pixel
 *              is an edge in both modes.  Mode 1 synchronises the stream
 *              while the hysteresis converges. */
typedef struct {
  float delta;
  float eps;
  float overlap_r;
  float edge_tau;
  int32_t fuse_grid;
  float bbox_min[3];
  float inv_voxel;
  int32_t first_bounce_from_geom;
  int32_t edge_mode;
} pe_params;

/* Aggregated splat geometry (Alg. 3, aggregation steps).  One caller-allocated device
 * blob holds, for each view v (pixel offset off_v = sum of earlier W*H):
 *   splat_cr[off_v + p] = {cx, cy, cz, R}   (R = 0: no splat owned here)
 *   splat_nf[off_v + p] = {nx, ny, nz, count}
 * and a conservative bounding-box pyramid per view (leaf tiles of 4x4 pixels,
 * each level 2x2 tiles of the one below; a leaf's lo.w holds the bit pattern
 * of its occupancy mask) in that view's (u, v, d) frame.
 * A splat's id is its owner pixel's global index off_v + p.
 * The blob also holds a coarse 32^3 grid over the fusion bounding box: per
 * cell, a bit mask of the views that own a splat whose (padded) sphere
 * overlaps the cell, plus one mask of views with splats outside the grid,
 * and per cell a slab (an axis and an interval of heights along it) bounding
 * every disk its mask counts; rays only descend the pyramids of views met
 * along their path, within the stretches of the ray inside those slabs.
 * Layout is fully determined by the views; use pe_geom_bytes() to size it.
 * vgrid_* are written by pe_aggregate_views (callers leave them zero). */
#ifndef PE_VGRID
#define PE_VGRID 32
#endif
typedef struct {
  int32_t n_views;
  pe_view views[PE_MAX_VIEWS];
  void *blob_dev;          /* caller-owned, pe_geom_bytes() bytes, 256-aligned */
  size_t blob_bytes;
  float vgrid_min[3];      /* grid origin (metres); 0 cells = no grid */
  float vgrid_cell;        /* cell edge (metres) */
  int32_t vgrid_n;         /* cells per axis (PE_VGRID) or 0 */
} pe_geom;

/* Per-ray last-hit records (Alg. 3 hitRecord; Eq. 14 inputs), indexed by ray
 * slot = view * W * H + pixel.  All device pointers, caller-owned.
 *   p, n, k, u, v : float32 [n][3]  last hit point, normal (turned against the
 *                   incoming ray), incoming direction k^(M-1), incoming tube
 *                   vectors u^(M-1), v^(M-1) (screen cell vectors pitch*u,
 *                   pitch*v reflected at every bounce);
 *   path          : float64 [n]     image-method path length d^(M)
 *                   (k^(0) . p^(1) + sum |p^(m) - p^(m-1)|);
 *   M             : int32 [n]       bounces (0 = the ray missed: Phi = 0);
 *   psi           : uint8 [n]       visibility of the receiver (Psi);
 *   ids           : uint32 [mb][n]  hit id per bounce (point index for a
 *                   GFB bounce, splat id for a splat bounce, 0xFFFFFFFF after
 *                   the last); may be NULL.
 * M, psi (and ids) are written for every slot; p, n, k, u, v and path only
 * for rays that hit (M >= 1) and are undefined where M = 0. */
typedef struct {
  float *p, *n, *k, *u, *v;
  double *path;
  int32_t *M;
  uint8_t *psi;
  uint32_t *ids;
  int64_t n_rays;
  int32_t max_bounces;
} pe_hits;

/* Device counters of a trace (int64): [0] executed intersection queries
 * (primary GFB lookups + march queries, misses included), [1] shadow queries,
 * [2] exact ray/splat tests, [3] pyramid node tests, [4] views whose
 * splats lie along the query's ray per the coarse occupancy grid (the
 * pyramids its walk searches, each over the stretch of the ray crossing
 * that view's occupied cells); pe_rcs_sweep also counts its incidence
 * splats: [5] exact per-pixel ray/disk tests, [6] 64-bit key updates
 * (atomicMin, one per test that hits), and its field sums: [7] Eq. 14
 * terms (rays with a contribution x frequencies). */
#define PE_STATS_WORDS 8

/* Alg. 1 (screen-based PRI, tube mode) with a finite heap of K points per
 * ray tube, as the paper writes it: of the candidates of pixel (i, j)'s tube
 * (points within delta of its central ray, in front of the screen) the K
 * nearest the central ray (squared distance in FP32, ties: smaller index)
 * are kept, and of those the one nearest the tube's origin (Length(p - o),
 * ties: smaller index) gives the pixel's key, in pe_build_gfb's format
 * (float bits of the depth << 32 | point index; all ones = no candidate).
 * pe_build_gfb's tube mode is the unbounded heap (K >= every candidate
 * count gives the same keys).  pos_dev FP32 [n][3]; keys_dev [n_views][H][W]
 * uint64 (caller-allocated); all views of one W x H; 1 <= K <= 64;
 * n_views * W * H < 2^24; ws of
 * pe_build_gfb_topk_workspace() bytes (0: the candidate list would exceed
 * 2^32 entries, PE_EUNSUPPORTED). */
size_t pe_build_gfb_topk_workspace(int32_t n_views, const pe_view *views, int64_t n_points,
                                   float delta);
pe_status pe_build_gfb_topk(const pe_view *views, int32_t n_views, const float *pos_dev,
                            int64_t n_points, float delta, int32_t K, void *ws, size_t ws_bytes,
                            uint64_t *keys_dev, void *stream);

/* Surfel attributes (the per-point inputs of Alg. 1 in surfel mode; the
 * paper's splatting baseline takes a radius from the point spacing and
 * normals from local PCA, Sec. IV-A), computed on the GPU:
 *   radius[i] = mean distance from p_i to its k_r nearest other points;
 *   normal[i] = unit eigenvector of the smallest eigenvalue of the
 *               covariance of the k_n nearest points (p_i included), turned
 *               to agree with ref_nrm[i] (nullable) or else to point away
 *               from the bounding-box centre.
 * pos_dev: FP32 [n][3]; radius_dev [n], normal_dev [n][3] (FP32, either may
 * be null).  Neighbours are exact: ordered by the FP32 squared distance
 * (dx*dx + dy*dy) + dz*dz, ties by index; distances summed in FP64 in that
 * order; mean and covariance in FP64.  Requires 1 <= k_r <= 31, 3 <= k_n <=
 * 32, n >= max(k_r + 1, k_n), n < 2^32; ws of
 * pe_point_attributes_workspace(n) bytes (256-byte aligned). */
size_t pe_point_attributes_workspace(int64_t n_points);

/* A spatially coherent processing order of the points (no counterpart in the
 * paper): order_dev[0..n) = a permutation of 0..n-1 grouping the points by
 * their cell of a 32^3 grid over their bounding box (cells in raster order,
 * x slowest and z fastest; the order within a cell is unspecified).  Neighbouring points then
 * project to footprints of similar size, so the lanes of a splat warp stay
 * busy together (pe_sweep.point_order).  ws of pe_order_points_workspace(n)
 * bytes (256-byte aligned); 1 <= n < 2^32; positions are clamped into the
 * grid (a non-finite one lands in an edge cell). */
size_t pe_order_points_workspace(int64_t n_points);
pe_status pe_order_points(const float *pos_dev, int64_t n_points, void *ws, size_t ws_bytes,
                          uint32_t *order_dev, void *stream);
pe_status pe_point_attributes(const float *pos_dev, int64_t n_points, int32_t k_r, int32_t k_n,
                              const float *ref_nrm_dev, void *ws, size_t ws_bytes,
                              float *radius_dev, float *normal_dev, void *stream);

/* Unit-throughput probe (no counterpart in the paper): launches one probe
 * of `blocks` x 256 threads on `stream` and returns the number of operations
 * it performs (the caller times the launch with events on that stream), or
 * -1 with pe_last_error set on a bad argument.
 *   kind 0  FP32 FMA: n_iter x 8 independent fmaf chains per thread (flops,
 *           an FMA counted as 2);
 *   kind 1  __sinf: n_iter x 8 independent chains per thread (sines; the
 *           PO term's sine/cosine path);
 *   kind 2  FP64 FMA: as kind 0 in double (flops);
 *   kind 3  L2 reads: n_iter passes of 16-byte loads cached in L2 only over
 *           the first scratch_bytes - 16 bytes (bytes read; the caller zeroes
 *           the buffer, sizes it below the L2 and runs a warm-up launch);
 *   kind 4  64-bit atomicMin, result unused (the splat's form): n_iter per
 *           thread at hashed addresses of a power-of-two table in scratch
 *           (atomics);
 *   kind 5  packed FP32x2 FMA (__ffma2_rn): n_iter x 8 independent chains
 *           of float pairs per thread (flops, a pair's FMA counted as 4).
 * scratch_dev: device buffer of at least 4096 bytes, 256-byte aligned, that
 * every kind may write; blocks in [1, 2^20]; n_iter in [1, 2^24]. */
int64_t pe_probe_units(int32_t kind, int32_t blocks, int32_t n_iter, void *scratch_dev,
                       size_t scratch_bytes, void *stream);

/* Library version of this header's ABI. */
int pe_abi_version(void);

/* Number of CUDA kernels this library has launched in the calling process
 * (all threads, all devices) -- a diagnostic counter with no counterpart in
 * the paper. */
int64_t pe_kernel_launches(void);

/* Diagnostics (no counterpart in the paper): make the library record CUDA
 * events around the next launches of one of its kernels on the calling host
 * thread.  `kernel` names it ("march_kernel" (the bounces after the first;
 * with max_bounces = 2 also the shadow rays), "po_kernel", "splat_kernel",
 * "primary_kernel", "shadow_kernel");
 * events[2k] / events[2k+1] (created by the
 * caller, cudaEvent_t passed as void*) are recorded on the launching stream
 * immediately before / after the k-th such launch, for k < n_pairs.  Pass
 * n_pairs = 0 to stop.  Returns the pairs recorded since the last call. */
int32_t pe_set_kernel_events(const char *kernel, void **events, int32_t n_pairs);

/* Human-readable text of the last error on the calling host thread. */
const char *pe_last_error(void);

/* Synchronise `stream` and return the first device-side condition raised by
 * kernels since the last check (PE_EOVERFLOW, PE_ETIMEOUT), or PE_ECUDA if
 * the stream reports an error; clears the device error word. */
pe_status pe_stream_check(void *stream);

/* ---------------------------------------------------------------------------
 * a2/a3  Screen-based point-ray intersection (Alg. 1) -> GFBs.
 * ------------------------------------------------------------------------- */

/* Workspace bytes for pe_build_gfb over these views: one uint64 depth key per
 * pixel plus 256 bytes. */
size_t pe_build_gfb_workspace(int32_t n_views, const pe_view *views);

/* Splat every point into every view (Alg. 1 with every candidate kept, i.e.
 * K unbounded: the nearest candidate per pixel is a min over a packed 64-bit
 * key (float bits of depth) << 32 | point index, so ties go to the smaller
 * index and the result is deterministic).
 *   mode 0 (surfel): point i is a two-sided disk of radius rad_dev[i] with
 *     normal nrm_dev[i]; depth = ray parameter t of the hit (t > 0);
 *   mode 1 (tube, Alg. 1): a point is a candidate when its distance to the
 *     pixel's central ray is < delta and it lies in front; depth =
 *     |point - ray origin| (Alg. 1's Length(p - o)); nrm/rad may be NULL.
 * Outputs (device, per view back to back, any may be NULL):
 *   gfb_nd_dev  float32 [pix][4] = (nx, ny, nz, depth): the hit point's
 *               normal turned to face the view (n . d < 0); (0,0,0,+inf) on a
 *               miss; tube mode stores a zero normal;
 *   gfb_hit_dev uint32 [pix] point index or 0xFFFFFFFF;
 *   gfb_mask_dev uint8 [pix] 1 on a hit;
 *   keys_dev    uint64 [pix] the raw keys (UINT64_MAX on a miss).
 * Requires 1 <= n_views <= PE_MAX_BATCH, all views of the call of one W x H
 * (PE_EINVAL otherwise; views of several sizes take one call per size, and
 * pe_aggregate_views fuses their outputs concatenated), n_points < 2^32 - 1. */
pe_status pe_build_gfb(const pe_view *views, int32_t n_views,
                       const float *pos_dev, const float *nrm_dev,
                       const float *rad_dev, int64_t n_points, int32_t mode,
                       float delta, void *ws, size_t ws_bytes,
                       float *gfb_nd_dev, uint32_t *gfb_hit_dev,
                       uint8_t *gfb_mask_dev, uint64_t *keys_dev, void *stream);

/* ---------------------------------------------------------------------------
 * a4  GFB aggregation: edge filter, voxel fusion, splats (Alg. 3, aggregation steps,
 *     Eq. 22).
 * ------------------------------------------------------------------------- */

/* Bytes of the pe_geom blob for these views. */
size_t pe_geom_bytes(int32_t n_views, const pe_view *views);

/* Workspace bytes for pe_aggregate_views (dense G^3 voxel counters + one
 * entry per GFB pixel + scan scratch). */
size_t pe_aggregate_workspace(int32_t n_views, const pe_view *views,
                              int32_t fuse_grid);

/* Fuse the GFBs of n_views views (as written by pe_build_gfb: gfb_nd_dev and
 * gfb_mask_dev, views back to back) into splats.  Edge pixels are dropped;
 * every remaining pixel's surface point o + depth * d falls in a voxel of the
 * fuse_grid^3 grid; each non-empty voxel becomes one splat whose centre is
 * the mean of its points and whose normal is the normalised mean of their
 * normals (each first turned into the hemisphere of the voxel's first
 * contributor), both summed in FP64 in (view, pixel) order, and whose radius
 * is the largest Eq. 22 value over its contributors (L = the contributor's
 * view pitch, p = its view direction).  The splat is stored at its owner
 * pixel: among the contributing views the one facing the fused normal most
 * directly (largest floor(4 |n . d_v|), FP32; the lower view on a tie), at
 * its first pixel in (view, pixel) order (the first contributor if the
 * normal vanishes).
 * Then the bounding
 * pyramids are built.  out->views/n_views/blob_dev must be set by the caller
 * (views identical to `views`).  Requires n_views <= PE_MAX_VIEWS,
 * fuse_grid <= 256, a finite bbox_min and a finite inv_voxel > 0
 * (PE_EINVAL otherwise). */
pe_status pe_aggregate_views(const pe_view *views, int32_t n_views,
                             const float *gfb_nd_dev, const uint8_t *gfb_mask_dev,
                             const pe_params *params, void *ws, size_t ws_bytes,
                             pe_geom *out, void *stream);

/* ---------------------------------------------------------------------------
 * a5  GFB-assisted multiple-bounce computation (Alg. 3, bounce loop, Eq. 2-4,
 *     Eq. 23) and the visibility test Psi (Eq. 14).
 * ------------------------------------------------------------------------- */

/* Workspace bytes for pe_trace_bounces over n_views ray screens of this size
 * (currently a constant 256: the bounce state lives in the hit records). */
size_t pe_trace_workspace(int32_t n_views, const pe_view *views);

/* Trace every pixel ray of n_views ray screens (e.g. one per monostatic
 * angle).  Bounce 1: from the screen's own GFB keys (keys_dev as written by
 * pe_build_gfb for these views, surfel mode) with the point's normal nrm_dev
 * turned to face the view, or -- when params->first_bounce_from_geom -- by
 * marching the splats from the screen (tmin 0; keys/nrm may be NULL).
 * Bounces 2..max_bounces: reflect the direction, the tube vectors and the
 * polarisation at the current normal (Eq. 2-4: a - 2 (a . n) n), march the
 * splats from the hit point (t > eps), take the nearest hit t* and, among the
 * hits with t <= t* + overlap_r, the one whose hit point is closest to its
 * splat's centre relative to its radius (ties: smaller t, then smaller id);
 * the normal is the Eq. 23 blend of the candidates' normals (each turned
 * against the ray, weights 1 - |p_i - c_i| / R_i, summed in splat-id order,
 * normalised, turned against the ray).  A miss ends the ray.
 * Psi: for rays with M >= 2 a shadow ray from the last hit toward the
 * receiver (monostatic: along w, t > eps) is tested against the splats;
 * Psi = 1 for M = 1 (the incident ray itself reached that point).
 * Outputs go to `hits` (n_rays = n_views * W * H; all views same W, H).
 * stats_dev: int64 [PE_STATS_WORDS] counters, accumulated (caller zeroes), or
 * NULL.  geom may be NULL when max_bounces == 1 and bounce 1 comes from the
 * GFB. */
pe_status pe_trace_bounces(const pe_view *views, int32_t n_views,
                           const uint64_t *keys_dev, const float *nrm_dev,
                           const pe_geom *geom, int32_t max_bounces,
                           const pe_params *params, void *ws, size_t ws_bytes,
                           const pe_hits *hits, int64_t *stats_dev, void *stream);

/* ---------------------------------------------------------------------------
 * a6  Physical-optics field sum (Eq. 5-14).
 * ------------------------------------------------------------------------- */

/* Workspace bytes for pe_po_field. */
size_t pe_po_workspace(int32_t n_groups, int64_t rays_per_group, int32_t n_freq);

/* For each group g of rays_per_group consecutive ray slots (e.g. one
 * monostatic angle) with observation direction ks[g] (unit, host float32
 * [n_groups][3], toward the receiver) and each frequency f (host float64
 * [n_freq], Hz), the Eq. 14 sum without its factor -j eta0 k0 / (2 pi):
 *   Sigma = sum_l Phi_l Psi_l |u' x v'| sinc(q.u'/2) sinc(q.v'/2)
 *           [(n x h) x ks] x ks exp(-j k (d_l - ks . p_l)),
 * q = k (k_in - ks), u', v' from Eq. 12-13 with k_in, sinc(x) = sin(x)/x,
 * for the two transmit polarisations V (E along theta_hat = screen u; magnetic
 * polarisation -v/|v|) and H (E along phi_hat = screen v; h = u/|u|), with u,
 * v the propagated tube vectors.  E_dev: float64 [n_groups][n_freq][2][3][2]
 * (pol, xyz, re/im), device.  Per-term arithmetic is float32 with the phase
 * argument in double-float and reduced modulo 2 pi; sums are compensated in
 * float32 per thread and reduced in float64 in a fixed order (deterministic).
 * A bounce-1 record (M = 1) seen in backscatter (ks = -k exactly) has
 * d - ks . p = 2 k . p; that is formed from its k and p as a float pair, and
 * its path field is not read.
 * RCS: sigma = k^2/pi |e_rx . Sigma|^2. */
pe_status pe_po_field(const pe_hits *hits, int32_t n_groups, int64_t rays_per_group,
                      const float *ks, const double *freqs_hz, int32_t n_freq,
                      void *ws, size_t ws_bytes, double *E_dev, void *stream);

/* Bistatic observation grids: for each group g (rays_per_group slots, as in
 * pe_po_field) and each of n_obs receiver directions obs_dirs[g][o] (unit,
 * toward the receiver; host float32 [n_groups][n_obs][3]), Psi is tested per
 * ray toward that receiver -- a shadow ray from the ray's last hit (M >= 1)
 * against the aggregated splats of `geom`, blocked by any hit with t > eps
 * (Eq. 14's Psi, Sec. II-C) -- and the Eq. 14 sum of pe_po_field is formed
 * with ks = obs_dirs[g][o].  With only_bounce > 0 only rays whose last hit
 * is that bounce (M == only_bounce) contribute: tracing with max_bounces =
 * b for b = 1..mb and summing gives PO at every bounce (Eq. 14 applied at
 * each hit instead of the last).  hits->psi is not read.  E_dev: float64
 * [n_groups][n_obs][n_freq][2][3][2].  n_groups <= PE_MAX_BATCH; ws of
 * pe_po_field_bistatic_workspace() bytes.  The monostatic receiver
 * (obs = -d of the group's view) gives pe_po_field's result except that
 * single-bounce rays are shadow-tested too. */
size_t pe_po_field_bistatic_workspace(int32_t n_groups, int64_t rays_per_group, int32_t n_freq);
pe_status pe_po_field_bistatic(const pe_hits *hits, int32_t n_groups, int64_t rays_per_group,
                               const float *obs_dirs, int32_t n_obs, const pe_geom *geom,
                               float eps, int32_t only_bounce, const double *freqs_hz,
                               int32_t n_freq, void *ws, size_t ws_bytes, double *E_dev,
                               void *stream);

/* PO at every bounce (the variant of Eq. 14 that applies it at each hit of a
 * ray, not only at the last; Sec. II-C, Eq. 14, Alg. 3).  For each b =
 * 1..max_bounces the n_views monostatic screens are traced to b bounces
 * (bounce 1 from the GFB keys, or from the geometry when
 * prm->first_bounce_from_geom), the rays whose b-th hit is their last
 * (M == b) are shadow-tested toward the screen's own transmitter (-d) from
 * that hit, and Eq. 14 is summed over them; the b fields are added in
 * increasing b (one FP64 addition each, so the result is deterministic).
 * views: host [n_views] screens of one W x H; keys: device uint64
 * [n_views][H][W] from pe_build_gfb (NULL with first_bounce_from_geom); nrm:
 * device [N][3]; geom: the aggregated splats (required); freqs_hz: host
 * [n_freq] > 0.  E_dev: device float64 [n_views][n_freq][2 pol][3][re, im],
 * overwritten.  ws: device, 256-byte aligned, of
 * pe_po_field_every_bounce_workspace() bytes (0 = invalid arguments).
 * Errors: PE_EINVAL (arguments), PE_ENOMEM (workspace), PE_ECUDA. */
size_t pe_po_field_every_bounce_workspace(int32_t n_views, const pe_view *views, int32_t n_freq);
pe_status pe_po_field_every_bounce(const pe_view *views, int32_t n_views, const uint64_t *keys,
                                   const float *nrm, const pe_geom *geom, int32_t max_bounces,
                                   const pe_params *prm, const double *freqs_hz, int32_t n_freq,
                                   void *ws, size_t ws_bytes, double *E_dev, void *stream);

/* pe_po_field without a workspace -- for callers that cannot allocate device
 * memory for the library (their memory belongs to a host application's own
 * pool, or allocation is not allowed where they call from).  The paper has no
 * counterpart; this is an interface convenience.  Same arguments, result and
 * arithmetic as pe_po_field, minus ws/ws_bytes: the partial sums live in a
 * fixed 16 MiB device array inside the library, which every GPU that loads
 * the library keeps until the process exits.  Requests whose partial sums
 * need more than 16 MiB (pe_po_workspace() - 256 > 16 MiB) return PE_EINVAL
 * with a message.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, once per device, with that device current);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: after a cudaDeviceReset() on a device, do not call
 * this entry point on that device again (the kept address belongs to the
 * destroyed context).  All calls share the one
 * array: calls whose work overlaps on the GPU (different streams, or
 * different host threads on the same device) race and corrupt each other's
 * results; serialise them.  Nothing in the array needs clearing between
 * calls. */
pe_status pe_po_field_static(const pe_hits *hits, int32_t n_groups, int64_t rays_per_group,
                             const float *ks, const double *freqs_hz, int32_t n_freq,
                             double *E_dev, void *stream);

/* ---------------------------------------------------------------------------
 * a1/a7  Monostatic RCS sweep (whole path: a1-a6 per batch of angles).
 * ------------------------------------------------------------------------- */

/* A monostatic sweep: incidence (theta_deg[a], phi_deg[a]); ray screen
 * W x H centred at `centre`, half-width `extent` (>= the target's bounding
 * radius), pitch = 2 extent / W; frequencies; bounces. */
typedef struct {
  int32_t n_angles;
  const double *theta_deg;   /* host [n_angles] */
  const double *phi_deg;     /* host [n_angles] */
  int32_t W, H;
  double centre[3];
  double extent;
  int32_t n_freq;
  const double *freqs_hz;    /* host [n_freq] */
  int32_t max_bounces;
  int32_t angle_batch;       /* angles per batch (1..PE_MAX_BATCH), 0 = auto
                                (as many as fit ~16 GB of ray records, or
                                ~8 GB per set of batch buffers when there
                                are two: see pe_rcs_sweep) */
  const uint32_t *point_order; /* device [n_points] or NULL: the order in which
                                the incidence splat takes the points (a
                                permutation, e.g. from pe_order_points); the
                                keys, which hold the points' own indices, do
                                not depend on it */
} pe_sweep;

/* The view of a monostatic incidence (a1): w = (sin t cos p, sin t sin p,
 * cos t), u = theta_hat, v = phi_hat, pitch = 2 extent / W, screen centre
 * centre + (extent + pitch) w, d = -w; computed in FP64, rounded to float32. */
pe_status pe_view_from_angles(double theta_deg, double phi_deg, const double centre[3],
                              double extent, int32_t W, int32_t H, pe_view *out);

/* Workspace bytes for pe_rcs_sweep. */
size_t pe_rcs_sweep_workspace(const pe_sweep *sweep);

/* Run the sweep on the scene (points, surfel normals, radii: device) and the
 * aggregated geometry `geom` (NULL allowed when max_bounces == 1):
 * per batch of angles, splat the points into the incidence screens
 * (bounce 1), trace bounces 2..mb, test Psi, and sum the PO field.
 * E_dev: float64 [n_angles][n_freq][2][3][2] (device, required);
 * sigma_dev: float64 [n_angles][n_freq][2 tx][2 rx] m^2 (device, nullable),
 * tx/rx in (V, H); stats_dev as in pe_trace_bounces (nullable).
 * With more than one batch and n_freq >= 8 the workspace holds two sets of
 * batch buffers and the library sums one batch's field on a second CUDA
 * stream of its own (created and released within the call) while the next
 * batch traces on `stream`; `stream` waits for that work before the call's
 * later operations, so the results are ordered on `stream` as usual. */
pe_status pe_rcs_sweep(const pe_sweep *sweep, const float *pos_dev,
                       const float *nrm_dev, const float *rad_dev, int64_t n_points,
                       const pe_geom *geom, const pe_params *params, void *ws,
                       size_t ws_bytes, double *E_dev, double *sigma_dev,
                       int64_t *stats_dev, void *stream);

/* ---------------------------------------------------------------------------
 * a8  Learned GFB completion (Sec. III-A: a U-Net with ConvNeXt blocks (ref 49),
 *     max-pooling down, sub-pixel convolution up (ref 51), a shared encoder and
 *     three decoders for depth, normal (uvw frame) and hit mask; losses
 *     Eq. 17-21; AdamW training, Sec. IV-A).  Layer primitives composed by the
 *     caller.  Activations are BF16 (passed as void*) in NHWC layout (channels
 *     fastest); accumulation and master weights are FP32.  Reductions over
 *     pixels (weight, bias, LayerNorm and loss sums) use fixed-order partial
 *     sums in the caller's workspace, so results are deterministic.
 * ------------------------------------------------------------------------- */

/* C[m,n] = epi(alpha * sum_k A(m,k) B(k,n)) with A(m,k) = A[m*sam + k*sak],
 * B(k,n) = B[k*sbk + n*sbn] (BF16, any strides: row- or column-major
 * operands), tensor-core products accumulated in FP32.  epi adds bias[n]
 * (FP32, nullable), R[m*ldr+n] (BF16 residual, nullable), beta * C_old (FP32
 * C only), then, if gelu = 1, stores the pre-activation to Z (BF16, nullable)
 * and applies GELU (exact erf form); if gelu = 2, multiplies by GELU'(Z[m*ldz
 * + n]) (Z read, required: the backward of GELU fused into the data
 * gradient).  C is FP32 (c_f32 = 1) or BF16 with row
 * stride ldc.  Long K is split across blocks (deterministic split-K) using ws
 * of pe_nn_gemm_workspace() bytes. */
size_t pe_nn_gemm_workspace(int32_t M, int32_t N, int64_t K);
/* Which contraction kernel pe_nn_gemm uses (process-wide; returns the
 * previous setting; other values only query): 0 = the tcgen05 tensor-core
 * kernel (TMA-staged operands, accumulator in tensor memory) whenever both
 * operands are K-contiguous with 16-byte aligned rows and no split-K is
 * needed, else the mma.sync kernel (default); 1 = the mma.sync kernel only.
 * Both give the same result up to FP32 summation order. */
int32_t pe_nn_gemm_path(int32_t path);
/* Diagnostics (no counterpart in the paper): the number of polls each
 * bounded mbarrier wait of the tcgen05 GEMM's main loop and epilogue makes
 * before it gives up (process-wide; polls < 0 restores the default of 2^22,
 * 0 makes every such wait give up at once).  A wait that gives up skips the
 * rest of the tile, waits (with the default limit) for the copies and
 * products it has issued, frees its tensor memory and sets the status word:
 * the next pe_stream_check() returns PE_ETIMEOUT and clears it, and later
 * calls run normally.  For tests of that path; PE_EINVAL above 2^32 - 1. */
pe_status pe_nn_set_wait_limit(int64_t polls);
pe_status pe_nn_gemm(int32_t M, int32_t N, int64_t K, const void *A, int64_t sam, int64_t sak,
                     const void *B, int64_t sbk, int64_t sbn, void *C, int64_t ldc,
                     int32_t c_f32, const float *bias, const void *R, int64_t ldr, void *Z,
                     int64_t ldz, int32_t gelu, float alpha, float beta, void *ws,
                     size_t ws_bytes, void *stream);

/* 3x3 convolution support, zero padding 1: forward writes col[p][(ky*3+kx)*C + c]
 * (BF16 [B*H*W][9C]) from X [B][H][W][C]; backward (backward = 1) reads X as
 * dcol and writes col as dX [B][H][W][C] (sum over the taps that read each
 * input pixel). */
pe_status pe_nn_im2col3(const void *X, int32_t B, int32_t H, int32_t W, int32_t C, void *col,
                        int32_t backward, void *stream);

/* Depthwise 7x7 convolution, zero padding 3, weights w[ky][kx][c] FP32, bias
 * FP32 (nullable).  Backward: dX (nullable), dw [49][C] and db [C] (FP32,
 * overwritten, nullable) with ws of pe_nn_dwconv7_bwd_workspace() bytes. */
pe_status pe_nn_dwconv7(const void *X, const float *w, const float *bias, int32_t B, int32_t H,
                        int32_t W, int32_t C, void *Y, void *stream);
size_t pe_nn_dwconv7_bwd_workspace(int32_t B, int32_t H, int32_t W, int32_t C);
pe_status pe_nn_dwconv7_bwd(const void *X, const void *dY, const float *w, int32_t B, int32_t H,
                            int32_t W, int32_t C, void *dX, float *dw, float *db, void *ws,
                            size_t ws_bytes, void *stream);

/* LayerNorm over the C channels of each of P pixels (C <= 256), gamma/beta
 * FP32; saves per-pixel mean and 1/std (FP32) for the backward, which writes
 * dX and dgamma, dbeta (FP32, overwritten, nullable). */
pe_status pe_nn_layernorm(const void *X, const float *gamma, const float *beta, int64_t P,
                          int32_t C, float eps, void *Y, float *mean, float *rstd,
                          void *stream);
size_t pe_nn_layernorm_bwd_workspace(int64_t P, int32_t C);
pe_status pe_nn_layernorm_bwd(const void *dY, const void *X, const float *gamma,
                              const float *mean, const float *rstd, int64_t P, int32_t C,
                              void *dX, float *dgamma, float *dbeta, void *ws, size_t ws_bytes,
                              void *stream);

/* Bias gradients: out[n] = (accumulate ? out[n] : 0) + sum_m X[m*ld + n]. */
size_t pe_nn_colsum_workspace(int64_t M, int32_t N);
pe_status pe_nn_colsum(const void *X, int64_t M, int32_t N, int64_t ld, float *out,
                       int32_t accumulate, void *ws, size_t ws_bytes, void *stream);

/* dst [Cc][R] = transpose of src [R][Cc] (BF16, row-major, distinct buffers). */
pe_status pe_nn_transpose(const void *src, int32_t R, int32_t Cc, void *dst, void *stream);

/* dZ = dA * GELU'(Z) elementwise (BF16). */
pe_status pe_nn_gelu_bwd(const void *dA, const void *Z, int64_t n, void *dZ, void *stream);

/* 2x2 max-pooling (even H, W) with the argmax (0..3, row-major in the window)
 * kept in arg [B][H/2][W/2][C]; backward (backward = 1): X = dY, Y = dX. */
pe_status pe_nn_maxpool2(const void *X, int32_t B, int32_t H, int32_t W, int32_t C, void *Y,
                         uint8_t *arg, int32_t backward, void *stream);

/* Sub-pixel convolution's shuffle (ref 51): out[b][2y+i][2x+j][off + c] =
 * in[b][y][x][4c + 2i + j], the output having ld_big channels (so the result
 * can land in one half of a concatenation); backward = 1 runs the reverse. */
pe_status pe_nn_pixel_shuffle2(const void *src, int32_t B, int32_t H, int32_t W, int32_t C,
                               void *dst, int64_t ld_big, int32_t off, int32_t backward,
                               void *stream);

/* dst[p][doff + c] = (accumulate ? dst : 0) + src[p][soff + c], c < C (BF16). */
pe_status pe_nn_copy_channels(const void *src, int64_t lds, int32_t soff, void *dst, int64_t ldd,
                              int32_t doff, int64_t P, int32_t C, int32_t accumulate,
                              void *stream);

/* FP32 -> BF16 copy. */
pe_status pe_nn_to_bf16(const float *x, int64_t n, void *y, void *stream);

/* AdamW (ref 53) with decoupled weight decay and bias correction at `step`
 * (>= 1); also refreshes the BF16 copy p_bf16 (nullable). */
pe_status pe_nn_adamw(float *p, const float *g, float *m, float *v, void *p_bf16, int64_t n,
                      float lr, float beta1, float beta2, float eps, float weight_decay,
                      int32_t step, void *stream);

/* Eq. 17-21 on FP32 head outputs (depth [P], normal [P][3], mask logit [P])
 * against d_gt [P], n_gt [P][3], m_gt [P] in {0,1}, P = B*H*W: L1 (squared
 * depth error), L2 (|n_p x n_g| / (|n_p||n_g|)) and L4 (the same for the
 * vectors (d_u, d_v, 1) of central differences, on hit pixels whose 4
 * neighbours are hits) are means over ground-truth hits, L3 (alpha-balanced
 * focal loss) a mean over all pixels; loss[0] = sum lambdas[i] * L(i+1),
 * loss[1..4] = L1..L4 (device FP32); g_* = dL/d(outputs) (FP32, overwritten).
 * |a x b| is evaluated as sqrt(|a x b|^2 + 1e-12) and norms products get
 * +1e-8, so the losses are differentiable everywhere. */
size_t pe_nn_unet_losses_workspace(int32_t B, int32_t H, int32_t W);
pe_status pe_nn_unet_losses(const float *depth, const float *normal, const float *logit,
                            const float *d_gt, const float *n_gt, const float *m_gt, int32_t B,
                            int32_t H, int32_t W, float alpha, float gamma, const float *lambdas,
                            float *loss, float *g_depth, float *g_normal, float *g_logit,
                            void *ws, size_t ws_bytes, void *stream);

/* Training pairs and GFB <-> hit records for n_views screens of one size.
 * Depth is normalised per view: (t - t_near[v]) / t_scale[v] (host arrays).
 * pe_learned_pairs: x_bf16 [P] = normalised depth of the tube-mode keys
 * (pe_build_gfb mode 1; 0 where empty); from a surfel GFB (float4 n, depth;
 * pe_build_gfb mode 0) d_gt, m_gt [P] and n_gt [P][3] = (n.u, n.v, n.w).
 * pe_gfb_hits: single-bounce last-hit records (Sec. III-A, Eq. 14) of a GFB
 * given as normalised depth [P], a hit indicator mask [P] (> threshold) and
 * normals in the uvw frame [P][3] (turned to face the view), or -- when
 * normal_uvw is NULL -- normals from the depth derivatives by Eq. 16. */
pe_status pe_learned_pairs(const pe_view *views, int32_t n_views, const float *t_near,
                           const float *t_scale, const uint64_t *tube_keys,
                           const float *surfel_nd, void *x_bf16, float *d_gt, float *n_gt,
                           float *m_gt, void *stream);
pe_status pe_gfb_hits(const pe_view *views, int32_t n_views, const float *t_near,
                      const float *t_scale, const float *depth, const float *mask,
                      float threshold, const float *normal_uvw, const pe_hits *hits,
                      void *stream);

#ifdef __cplusplus
}
#endif

#endif /* POINTEMRAY_H */
