/*
 * PointEMRay CPU oracle -- generic core, included twice by oracle.c with
 *   R = float  (FP32 geometry mode: the op order every float expression below
 *               is written in is the one the bit-exact parity targets), and
 *   R = double (FP64 physics mode).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is a plain, slow, brute-force statement
 * of the method (the searches can take their candidates from a uniform grid
 * instead of every element, with the same result: oracle_grid.h).  It is compiled with -ffp-contract=off and without fast-math
 * so every float expression rounds once per operation, left to right.
 *
 * Passages followed (PointEMRay, arXiv 2408.15583):
 *   - screen / uvwo frame: Sec. III-A, around Eq. 15-16;
 *   - point-ray intersection (GFB): Alg. 1 (screen-based PRI), surfel reading
 *     of "assigning finite surface areas to points" (Sec. III-A intro);
 *   - edge filter, voxel fusion, splat radius: Alg. 3, aggregation steps, Eq. 22;
 *   - ray-splat intersection with overlap sphere and normal blend: Eq. 23,
 *     Fig. 4; minimum travel distance epsilon: Sec. III-B;
 *   - reflection: Eq. 2-4;  visibility Psi: Sec. II-C, Eq. 14.
 */

typedef struct {
  R o[3], u[3], v[3], d[3];
  R L;
  int W, H;
} SFX(view);

static void SFX(load_view)(const or_view *in, SFX(view) *v) {
  for (int k = 0; k < 3; ++k) {
    v->o[k] = (R)in->o[k];
    v->u[k] = (R)in->u[k];
    v->v[k] = (R)in->v[k];
    v->d[k] = (R)in->d[k];
  }
  v->L = (R)in->pitch;
  v->W = in->W;
  v->H = in->H;
}

static inline R SFX(dot)(const R *a, const R *b) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* Centre of pixel (i, j) on the screen plane: the origin of its ray.
 * Screen coordinates are measured from the screen centre in units of the
 * pitch L along u (columns i) and v (rows j). */
static void SFX(pixel_origin)(const SFX(view) *v, int i, int j, R *o) {
  R fi = ((R)i + (R)0.5) - (R)0.5 * (R)v->W;
  R fj = ((R)j + (R)0.5) - (R)0.5 * (R)v->H;
  R a = fi * v->L;
  R b = fj * v->L;
  for (int k = 0; k < 3; ++k) o[k] = (v->o[k] + a * v->u[k]) + b * v->v[k];
}

/* Ray o + t d against a two-sided disk (centre c, normal n, radius rad).
 * Hit iff the plane is not parallel, the plane point lies inside the disk and
 * t > tmin.  On a hit, *t and x (the hit point) and e = x - c are returned. */
static int SFX(hit_disk)(const R *o, const R *d, const R *c, const R *n, R rad,
                         R tmin, R *t_out, R *x, R *e) {
  R den = SFX(dot)(d, n);
  if (den == (R)0) return 0;
  R q[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
  R t = SFX(dot)(q, n) / den;
  for (int k = 0; k < 3; ++k) x[k] = o[k] + t * d[k];
  for (int k = 0; k < 3; ++k) e[k] = x[k] - c[k];
  if (!(SFX(dot)(e, e) <= rad * rad)) return 0;
  if (!(t > tmin)) return 0;
  *t_out = t;
  return 1;
}

/* Ray tube of radius delta around the central ray o + t d (Alg. 1): a point c
 * is a candidate iff its distance to the central ray is below delta and it
 * lies in front of the screen; its score is Length(c - o). */
static int SFX(hit_tube)(const R *o, const R *d, const R *c, R delta, R *score) {
  R q[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
  R t = SFX(dot)(q, d);
  R x[3], e[3];
  for (int k = 0; k < 3; ++k) x[k] = o[k] + t * d[k];
  for (int k = 0; k < 3; ++k) e[k] = x[k] - c[k];
  if (!(SFX(dot)(e, e) < delta * delta)) return 0;
  if (!(t > (R)0)) return 0;
  *score = SQRT(SFX(dot)(q, q));
  return 1;
}

/* One candidate of Alg. 1 for the pixel ray (o, d): point s as a disk of
 * radius rad[s] with normal nrm[s] (surfel mode 0) or as a point within a
 * tube of radius dl around the ray (tube mode 1).  The nearest candidate is
 * kept; equal depths go to the smaller point index. */
static void SFX(gfb_consider)(const R *o, const R *d, const float *pos, const float *nrm,
                              const float *rad, int mode, R dl, int64_t s, R *best,
                              int64_t *bi) {
  R c[3] = {(R)pos[3 * s], (R)pos[3 * s + 1], (R)pos[3 * s + 2]};
  R t;
  if (mode == 0) {
    R nn[3] = {(R)nrm[3 * s], (R)nrm[3 * s + 1], (R)nrm[3 * s + 2]};
    R x[3], e[3];
    if (!SFX(hit_disk)(o, d, c, nn, (R)rad[s], (R)0, &t, x, e)) return;
  } else {
    if (!SFX(hit_tube)(o, d, c, dl, &t)) return;
  }
  if (t < *best || (t == *best && s < *bi)) {
    *best = t;
    *bi = s;
  }
}

/* Alg. 1 (PRI) for the listed pixels of one view: the nearest candidate over
 * all points (ties: smaller point index), by brute force, or over the points
 * a uniform grid lists along the pixel's ray (use_grid; same result, see
 * oracle_grid.h).  Surfel mode (mode 0): each point is a disk of radius
 * rad[i] with normal nrm[i]; tube mode (mode 1): a tube of radius delta
 * around each pixel's ray.  Outputs: depth (t or tube score, +inf on a miss),
 * hit index (-1 on a miss) and, in surfel mode, the hit point's normal turned
 * to face the view (n . d < 0). */
static void SFX(gfb)(const or_view *vin, const float *pos, const float *nrm,
                     const float *rad, int64_t n, int mode, double delta,
                     const int64_t *pix, int64_t npix, int use_grid, double *depth_out,
                     int64_t *idx_out, double *nrm_out) {
  SFX(view) v;
  SFX(load_view)(vin, &v);
  R dl = (R)delta;
  or_grid grid;
  memset(&grid, 0, sizeof(grid));
  if (use_grid) {
    double *gc = (double *)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double *gr = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double scale = 0.0;
    for (int64_t s = 0; s < n; ++s) {
      for (int k = 0; k < 3; ++k) {
        gc[3 * s + k] = (double)pos[3 * s + k];
        if (fabs(gc[3 * s + k]) > scale) scale = fabs(gc[3 * s + k]);
      }
      gr[s] = mode == 0 ? (double)rad[s] : (double)dl;
    }
    scale += fabs(vin->o[0]) + fabs(vin->o[1]) + fabs(vin->o[2]) +
             (double)(vin->W + vin->H) * vin->pitch;
    or_grid_build(&grid, gc, gr, n, scale);
    free(gc);
    free(gr);
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < npix; ++q) {
    int64_t p = pix ? pix[q] : q;
    int i = (int)(p % v.W), j = (int)(p / v.W);
    R o[3];
    SFX(pixel_origin)(&v, i, j, o);
    R best = (R)INFINITY;
    int64_t bi = -1;
    if (!use_grid) {
      for (int64_t s = 0; s < n; ++s) SFX(gfb_consider)(o, v.d, pos, nrm, rad, mode, dl, s, &best, &bi);
    } else {
      double od[3] = {(double)o[0], (double)o[1], (double)o[2]};
      double dd[3] = {(double)v.d[0], (double)v.d[1], (double)v.d[2]};
      or_walk w;
      const int32_t *it;
      int64_t cnt;
      for (or_walk_begin(&w, &grid, od, dd, 0.0); or_walk_cell(&w, (double)best, &it, &cnt);
           or_walk_step(&w))
        for (int64_t e = 0; e < cnt; ++e)
          SFX(gfb_consider)(o, v.d, pos, nrm, rad, mode, dl, it[e], &best, &bi);
    }
    depth_out[q] = (double)best;
    idx_out[q] = bi;
    if (nrm_out) {
      if (bi >= 0 && mode == 0) {
        R nn[3] = {(R)nrm[3 * bi], (R)nrm[3 * bi + 1], (R)nrm[3 * bi + 2]};
        int flip = SFX(dot)(nn, v.d) > (R)0;
        for (int k = 0; k < 3; ++k) nrm_out[3 * q + k] = (double)(flip ? -nn[k] : nn[k]);
      } else {
        for (int k = 0; k < 3; ++k) nrm_out[3 * q + k] = 0.0;
      }
    }
  }
  or_grid_free(&grid);
}

/* Alg. 1 with a finite heap of K points per ray tube, as written: the
 * candidates (points within delta of the central ray, in front of the
 * screen) are ranked by their squared distance to the central ray (ties:
 * smaller point index); of the K best, the one nearest the tube's origin
 * (Length(p - o), ties: smaller index) gives the depth.  Same arithmetic as
 * hit_tube.  Outputs as gfb in tube mode. */
static void SFX(gfb_topk)(const or_view *vin, const float *pos, int64_t n, double delta, int K,
                          const int64_t *pix, int64_t npix, double *depth_out,
                          int64_t *idx_out) {
  SFX(view) v;
  SFX(load_view)(vin, &v);
  R dl = (R)delta;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < npix; ++q) {
    int64_t p = pix ? pix[q] : q;
    int i = (int)(p % v.W), j = (int)(p / v.W);
    R o[3];
    SFX(pixel_origin)(&v, i, j, o);
    R ka[64], ks[64];
    int64_t ki[64];
    int cnt = 0;
    for (int64_t s = 0; s < n; ++s) {
      R c[3] = {(R)pos[3 * s], (R)pos[3 * s + 1], (R)pos[3 * s + 2]};
      R qv[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
      R t = SFX(dot)(qv, v.d);
      R x[3], e[3];
      for (int k = 0; k < 3; ++k) x[k] = o[k] + t * v.d[k];
      for (int k = 0; k < 3; ++k) e[k] = x[k] - c[k];
      R a = SFX(dot)(e, e);
      if (!(a < dl * dl)) continue;
      if (!(t > (R)0)) continue;
      if (cnt == K && !(a < ka[K - 1])) continue; /* equal a: the smaller index stays */
      int at = cnt < K ? cnt++ : K - 1;
      while (at > 0 && ka[at - 1] > a) {
        ka[at] = ka[at - 1];
        ki[at] = ki[at - 1];
        ks[at] = ks[at - 1];
        --at;
      }
      ka[at] = a;
      ki[at] = s;
      ks[at] = SQRT(SFX(dot)(qv, qv));
    }
    R best = (R)INFINITY;
    int64_t bi = -1;
    for (int e = 0; e < cnt; ++e)
      if (ks[e] < best || (ks[e] == best && ki[e] < bi)) {
        best = ks[e];
        bi = ki[e];
      }
    depth_out[q] = (double)best;
    idx_out[q] = bi;
  }
}

/* ---------------------------------------------------------------------------
 * Alg. 3, aggregation steps: edge filtering, voxel fusion, conversion to splats.
 * ------------------------------------------------------------------------- */

/* Edge rule (the paper names a Canny operator without thresholds): a hit
 * pixel is an edge if a 4-neighbour is outside the image or empty, or if a
 * neighbour's depth differs by more than tau * L. */
/* Canny edges of one view's depth map (edge mode 1; the paper removes GFB
 * edges with a Canny filter before fusion, Sec. III-B, without its
 * parameters).  On valid pixels only: 5x5 binomial smoothing ([1 4 6 4 1]^2 /
 * 256; samples outside the image or empty take the centre's depth), Sobel
 * gradient of the smoothed map (samples outside/empty take the centre's
 * value), magnitude sqrt(gx^2 + gy^2), non-maximum suppression along the
 * gradient's sector (0, 45, 90, 135 degrees by tan 22.5 and tan 67.5; absent
 * neighbours count 0; ties kept), thresholds high = 8 tau L (the Sobel
 * response to a slope of tau pitches per pixel) and low = high / 2,
 * hysteresis over the 8 neighbours.  edge[p] = 1 for Canny edge pixels. */
static R SFX(cs)(const R *S, const uint8_t *mask, int W, int H, int i, int j, int di, int dj) {
  int ii = i + di, jj = j + dj;
  if (ii < 0 || jj < 0 || ii >= W || jj >= H || !mask[(int64_t)jj * W + ii])
    return S[(int64_t)j * W + i];
  return S[(int64_t)jj * W + ii];
}

static void SFX(canny)(const R *depth, const uint8_t *mask, int W, int H, R L, R tau,
                       uint8_t *edge) {
  const int64_t n = (int64_t)W * H;
  R *S = (R *)calloc((size_t)n + 1, sizeof(R));
  R *Gm = (R *)calloc((size_t)n + 1, sizeof(R));
  uint8_t *sec = (uint8_t *)calloc((size_t)n + 1, 1);
  uint8_t *st = (uint8_t *)calloc((size_t)n + 1, 1);
  int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  static const int b[5] = {1, 4, 6, 4, 1};
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      int64_t p = (int64_t)j * W + i;
      if (!mask[p]) continue;
      R acc = (R)0;
      for (int dj = -2; dj <= 2; ++dj)
        for (int di = -2; di <= 2; ++di) {
          int ii = i + di, jj = j + dj;
          int in = ii >= 0 && jj >= 0 && ii < W && jj < H && mask[(int64_t)jj * W + ii];
          R dq = in ? depth[(int64_t)jj * W + ii] : depth[p];
          R w = (R)(b[dj + 2] * b[di + 2]) / (R)256;
          acc = acc + w * dq;
        }
      S[p] = acc;
    }
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      int64_t p = (int64_t)j * W + i;
      if (!mask[p]) continue;
#define CS(a, c) SFX(cs)(S, mask, W, H, i, j, a, c)
      R gx = ((CS(1, -1) - CS(-1, -1)) + (R)2 * (CS(1, 0) - CS(-1, 0))) + (CS(1, 1) - CS(-1, 1));
      R gy = ((CS(-1, 1) - CS(-1, -1)) + (R)2 * (CS(0, 1) - CS(0, -1))) + (CS(1, 1) - CS(1, -1));
#undef CS
      Gm[p] = SQRT(gx * gx + gy * gy);
      R ax = gx < (R)0 ? -gx : gx, ay = gy < (R)0 ? -gy : gy;
      if (ay <= (R)0.41421356f * ax) sec[p] = 0;
      else if (ay >= (R)2.41421356f * ax) sec[p] = 2;
      else sec[p] = ((gx > (R)0) == (gy > (R)0)) ? 1 : 3;
    }
  const R high = ((R)8 * tau) * L, low = (R)0.5 * high;
  static const int nx[4] = {1, 1, 0, 1}, ny[4] = {0, 1, 1, -1};
  int64_t top = 0;
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      int64_t p = (int64_t)j * W + i;
      if (!mask[p]) continue;
      R g = Gm[p], g1 = (R)0, g2 = (R)0;
      int a = sec[p];
      int i1 = i + nx[a], j1 = j + ny[a], i2 = i - nx[a], j2 = j - ny[a];
      if (i1 >= 0 && j1 >= 0 && i1 < W && j1 < H && mask[(int64_t)j1 * W + i1]) g1 = Gm[(int64_t)j1 * W + i1];
      if (i2 >= 0 && j2 >= 0 && i2 < W && j2 < H && mask[(int64_t)j2 * W + i2]) g2 = Gm[(int64_t)j2 * W + i2];
      if (!(g > (R)0 && g >= g1 && g >= g2)) continue;
      st[p] = g >= high ? 2 : (g >= low ? 1 : 0);
      if (st[p] == 2) stack[top++] = p;
    }
  while (top > 0) { /* hysteresis: weak pixels connected to a strong one */
    int64_t p = stack[--top];
    int i = (int)(p % W), j = (int)(p / W);
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        int ii = i + di, jj = j + dj;
        if (ii < 0 || jj < 0 || ii >= W || jj >= H) continue;
        int64_t q = (int64_t)jj * W + ii;
        if (st[q] == 1) {
          st[q] = 2;
          stack[top++] = q;
        }
      }
  }
  for (int64_t p = 0; p < n; ++p) edge[p] = st[p] == 2;
  free(S);
  free(Gm);
  free(sec);
  free(st);
  free(stack);
}

static int SFX(is_edge)(const R *depth, const uint8_t *mask, int W, int H, int i,
                        int j, R tauL) {
  static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  R t = depth[(int64_t)j * W + i];
  for (int k = 0; k < 4; ++k) {
    int ii = i + di[k], jj = j + dj[k];
    if (ii < 0 || jj < 0 || ii >= W || jj >= H) return 1;
    int64_t q = (int64_t)jj * W + ii;
    if (!mask[q]) return 1;
    R dt = depth[q] - t;
    if (dt < (R)0) dt = -dt;
    if (dt > tauL) return 1;
  }
  return 0;
}

typedef struct {
  uint64_t key;  /* voxel << 40 | view << 32 | pixel */
  R p[3];
  R n[3];
  int view;
} SFX(entry);

static int SFX(cmp_entry)(const void *a, const void *b) {
  uint64_t ka = ((const SFX(entry) *)a)->key, kb = ((const SFX(entry) *)b)->key;
  return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

typedef struct {
  int64_t id;
  R c[3], n[3], r;
  int32_t count;
} SFX(splat);

static int SFX(cmp_splat)(const void *a, const void *b) {
  int64_t ka = ((const SFX(splat) *)a)->id, kb = ((const SFX(splat) *)b)->id;
  return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

/* Eq. 22 for one contributor: s = sqrt(|n| |p| / |n . p|), R = sqrt(2) L s
 * for s < 2.5 else 3.535 L.  Evaluated in FP64 from the stored values. */
static double SFX(eq22)(const R *n, const R *p, double L) {
  double nx = (double)n[0], ny = (double)n[1], nz = (double)n[2];
  double px = (double)p[0], py = (double)p[1], pz = (double)p[2];
  double nn = sqrt((nx * nx + ny * ny) + nz * nz);
  double pp = sqrt((px * px + py * py) + pz * pz);
  double np = (nx * px + ny * py) + nz * pz;
  if (np < 0) np = -np;
  double s = (np > 0) ? sqrt((nn * pp) / np) : INFINITY;
  if (s < 2.5) return (1.4142135623730951 * L) * s;
  return 3.535 * L;
}

/* Fuse the listed GFBs into splats.  depth/nrm/mask are the views' buffers
 * concatenated in view order (row-major H x W each).  Returns the number of
 * splats written (sorted by splat id = global owner pixel index). */
static int64_t SFX(aggregate)(int nv, const or_view *views, const double *depth_in,
                              const double *nrm_in, const uint8_t *mask,
                              double tau, int edge_mode, const double *bmin, double inv_vox,
                              int G, int64_t *out_id, double *out_c,
                              double *out_n, double *out_r, int32_t *out_count,
                              uint8_t *keep_out) {
  int64_t total = 0;
  for (int v = 0; v < nv; ++v) total += (int64_t)views[v].W * views[v].H;
  R *depth = (R *)malloc(sizeof(R) * (size_t)(total > 0 ? total : 1));
  for (int64_t q = 0; q < total; ++q) depth[q] = (R)depth_in[q];
  SFX(entry) *ent = (SFX(entry) *)malloc(sizeof(SFX(entry)) * (size_t)(total > 0 ? total : 1));
  int64_t ne = 0, off = 0;
  R bm[3] = {(R)bmin[0], (R)bmin[1], (R)bmin[2]};
  R iv = (R)inv_vox;
  for (int v = 0; v < nv; ++v) {
    SFX(view) V;
    SFX(load_view)(&views[v], &V);
    R tauL = (R)tau * V.L;
    uint8_t *cedge = NULL;
    if (edge_mode == 1) {
      cedge = (uint8_t *)calloc((size_t)V.W * V.H + 1, 1);
      SFX(canny)(depth + off, mask + off, V.W, V.H, V.L, (R)tau, cedge);
      tauL = (R)INFINITY; /* the border part of the edge rule stays */
    }
    for (int j = 0; j < V.H; ++j)
      for (int i = 0; i < V.W; ++i) {
        int64_t q = off + (int64_t)j * V.W + i;
        uint8_t keep = 0;
        if (mask[q] && !SFX(is_edge)(depth + off, mask + off, V.W, V.H, i, j, tauL) &&
            !(cedge && cedge[(int64_t)j * V.W + i])) {
          keep = 1;
          R o[3], p[3];
          SFX(pixel_origin)(&V, i, j, o);
          R t = depth[q];
          for (int k = 0; k < 3; ++k) p[k] = o[k] + t * V.d[k];
          int64_t ix[3];
          for (int k = 0; k < 3; ++k) {
            R f = (p[k] - bm[k]) * iv;
            int64_t c = (int64_t)FLOOR(f);
            if (c < 0) c = 0;
            if (c > G - 1) c = G - 1;
            ix[k] = c;
          }
          uint64_t vox = (uint64_t)((ix[0] * G + ix[1]) * G + ix[2]);
          SFX(entry) *E = &ent[ne++];
          E->key = (vox << 40) | ((uint64_t)v << 32) | (uint64_t)((int64_t)j * V.W + i);
          for (int k = 0; k < 3; ++k) {
            E->p[k] = p[k];
            E->n[k] = (R)nrm_in[3 * q + k];
          }
          E->view = v;
        }
        if (keep_out) keep_out[q] = keep;
      }
    free(cedge);
    off += (int64_t)V.W * V.H;
  }
  qsort(ent, (size_t)ne, sizeof(SFX(entry)), SFX(cmp_entry));
  int64_t *voff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
  voff[0] = 0;
  for (int v = 0; v < nv; ++v) voff[v + 1] = voff[v] + (int64_t)views[v].W * views[v].H;
  SFX(splat) *sp = (SFX(splat) *)malloc(sizeof(SFX(splat)) * (size_t)(ne > 0 ? ne : 1));
  int64_t ns = 0;
  for (int64_t a = 0; a < ne;) {
    uint64_t vox = ent[a].key >> 40;
    int64_t b = a;
    while (b < ne && (ent[b].key >> 40) == vox) ++b;
    /* segment [a, b) in (view, pixel) order */
    const SFX(entry) *E0 = &ent[a];
    double sp3[3] = {0, 0, 0}, sn3[3] = {0, 0, 0}, rmax = 0.0;
    for (int64_t e = a; e < b; ++e) {
      const SFX(entry) *E = &ent[e];
      R nn[3] = {E->n[0], E->n[1], E->n[2]};
      if (SFX(dot)(nn, E0->n) < (R)0)
        for (int k = 0; k < 3; ++k) nn[k] = -nn[k];
      for (int k = 0; k < 3; ++k) {
        sp3[k] = sp3[k] + (double)E->p[k];
        sn3[k] = sn3[k] + (double)nn[k];
      }
      SFX(view) V;
      SFX(load_view)(&views[E->view], &V);
      double r = SFX(eq22)(nn, V.d, (double)V.L);
      if (r > rmax) rmax = r;
    }
    double cnt = (double)(b - a);
    double m = sqrt((sn3[0] * sn3[0] + sn3[1] * sn3[1]) + sn3[2] * sn3[2]);
    SFX(splat) *S = &sp[ns++];
    for (int k = 0; k < 3; ++k) {
      S->c[k] = (R)(sp3[k] / cnt);
      S->n[k] = (R)(sn3[k] / m);
    }
    /* owner: among the contributing views, the one facing the fused normal
     * most directly, by |n . d_v| in quarters (floor(4 |n . d_v|), so that
     * near-equal views tie), the lower view on a tie, and within it its
     * first (lowest) pixel; the first entry if the normal vanishes */
    const SFX(entry) *Eo = E0;
    if (m > 0.0) {
      R best = (R)-1;
      for (int64_t e = a; e < b; ++e) {
        SFX(view) V;
        SFX(load_view)(&views[ent[e].view], &V);
        R sc = SFX(dot)(S->n, V.d);
        if (sc < (R)0) sc = -sc;
        sc = FLOOR(sc * (R)4);
        if (sc > best) {
          best = sc;
          Eo = &ent[e];
        }
      }
    }
    int v0 = (int)((Eo->key >> 32) & 0xff);
    S->id = voff[v0] + (int64_t)(Eo->key & 0xffffffffu);
    S->r = (R)rmax;
    S->count = (int32_t)(b - a);
    a = b;
  }
  qsort(sp, (size_t)ns, sizeof(SFX(splat)), SFX(cmp_splat));
  for (int64_t s = 0; s < ns; ++s) {
    out_id[s] = sp[s].id;
    for (int k = 0; k < 3; ++k) {
      out_c[3 * s + k] = (double)sp[s].c[k];
      out_n[3 * s + k] = (double)sp[s].n[k];
    }
    out_r[s] = (double)sp[s].r;
    out_count[s] = sp[s].count;
  }
  free(sp);
  free(voff);
  free(ent);
  free(depth);
  return ns;
}

/* ---------------------------------------------------------------------------
 * Alg. 3, bounce loop: bounce tracing against splats, Eq. 23 overlap selection.
 * ------------------------------------------------------------------------- */

typedef struct {
  const R *c, *n, *r;
  const int64_t *id;
  int64_t ns;
  const or_grid *grid; /* NULL: every search is brute force over all splats */
} SFX(splatset);

/* First pass of the nearest-hit search: splat s against the ray; the nearest
 * hit with t > tmin is kept (equal t: the smaller storage index, which is the
 * smaller splat id). */
static void SFX(first_hit)(const SFX(splatset) *S, const R *o, const R *d, R tmin, int64_t s,
                           R *tb, int64_t *sb) {
  R t, x[3], e[3];
  if (!SFX(hit_disk)(o, d, S->c + 3 * s, S->n + 3 * s, S->r[s], tmin, &t, x, e)) return;
  if (t < *tb || (t == *tb && s < *sb)) {
    *tb = t;
    *sb = s;
  }
}

/* The splats the search must consider for the ray o + t d up to t_stop: all
 * of them (brute force) or those listed in the grid cells the ray crosses
 * before t_stop, sorted by storage index without repeats. */
static void SFX(candidates)(const SFX(splatset) *S, const R *o, const R *d, R tmin, R t_stop,
                            or_list *L) {
  L->n = 0;
  if (!S->grid) {
    for (int64_t s = 0; s < S->ns; ++s) or_list_push(L, (int32_t)s);
    return;
  }
  double od[3] = {(double)o[0], (double)o[1], (double)o[2]};
  double dd[3] = {(double)d[0], (double)d[1], (double)d[2]};
  or_walk w;
  const int32_t *it;
  int64_t cnt;
  for (or_walk_begin(&w, S->grid, od, dd, (double)tmin - S->grid->slack);
       or_walk_cell(&w, (double)t_stop, &it, &cnt); or_walk_step(&w))
    for (int64_t e = 0; e < cnt; ++e) or_list_push(L, it[e]);
  or_list_sort_unique(L);
}

/* Nearest ray-splat hit with t > tmin, then Eq. 23: among the hits whose t is
 * within r_ov of the nearest, pick the one closest (relative to its radius)
 * to its splat's centre, and blend the candidates' normals with weights
 * 1 - |p_i - c_i| / R_i (each normal first turned against the ray; blend in
 * splat-id order; result normalised and turned against the ray).
 * Splats are stored in id order. */
static int SFX(nearest)(const SFX(splatset) *S, const R *o, const R *d, R tmin,
                        R r_ov, R *p_out, R *n_out, int64_t *id_out) {
  R tb = (R)INFINITY;
  int64_t sb = -1;
  if (!S->grid) {
    for (int64_t s = 0; s < S->ns; ++s) SFX(first_hit)(S, o, d, tmin, s, &tb, &sb);
  } else {
    double od[3] = {(double)o[0], (double)o[1], (double)o[2]};
    double dd[3] = {(double)d[0], (double)d[1], (double)d[2]};
    or_walk w;
    const int32_t *it;
    int64_t cnt;
    for (or_walk_begin(&w, S->grid, od, dd, (double)tmin - S->grid->slack);
         or_walk_cell(&w, (double)tb, &it, &cnt); or_walk_step(&w))
      for (int64_t e = 0; e < cnt; ++e) SFX(first_hit)(S, o, d, tmin, it[e], &tb, &sb);
  }
  if (sb < 0) return 0;
  R lim = tb + r_ov;
  or_list L = {NULL, 0, 0};
  SFX(candidates)(S, o, d, tmin, lim, &L);
  R m[3] = {0, 0, 0};
  R best_rho = (R)INFINITY, best_t = (R)INFINITY;
  int64_t ssel = -1;
  R xsel[3] = {0, 0, 0}, nsel[3] = {0, 0, 0};
  for (int64_t e = 0; e < L.n; ++e) {
    const int64_t s = L.v[e];
    R t, x[3], ev[3];
    if (!SFX(hit_disk)(o, d, S->c + 3 * s, S->n + 3 * s, S->r[s], tmin, &t, x, ev)) continue;
    if (!(t <= lim)) continue;
    R rho = SQRT(SFX(dot)(ev, ev)) / S->r[s];
    const R *ns = S->n + 3 * s;
    R nn[3] = {ns[0], ns[1], ns[2]};
    if (SFX(dot)(nn, d) > (R)0)
      for (int k = 0; k < 3; ++k) nn[k] = -nn[k];
    R w = (R)1 - rho;
    for (int k = 0; k < 3; ++k) m[k] = m[k] + w * nn[k];
    if (rho < best_rho || (rho == best_rho && t < best_t)) {
      best_rho = rho;
      best_t = t;
      ssel = s;
      for (int k = 0; k < 3; ++k) {
        xsel[k] = x[k];
        nsel[k] = nn[k];
      }
    }
  }
  free(L.v);
  R mm = SFX(dot)(m, m);
  if (mm == (R)0) {
    for (int k = 0; k < 3; ++k) n_out[k] = nsel[k];
  } else {
    R s = SQRT(mm);
    for (int k = 0; k < 3; ++k) n_out[k] = m[k] / s;
    if (SFX(dot)(n_out, d) > (R)0)
      for (int k = 0; k < 3; ++k) n_out[k] = -n_out[k];
  }
  for (int k = 0; k < 3; ++k) p_out[k] = xsel[k];
  *id_out = S->id[ssel];
  return 1;
}

static int SFX(any_hit)(const SFX(splatset) *S, const R *o, const R *d, R tmin) {
  if (!S->grid) {
    for (int64_t s = 0; s < S->ns; ++s) {
      R t, x[3], e[3];
      if (SFX(hit_disk)(o, d, S->c + 3 * s, S->n + 3 * s, S->r[s], tmin, &t, x, e)) return 1;
    }
    return 0;
  }
  double od[3] = {(double)o[0], (double)o[1], (double)o[2]};
  double dd[3] = {(double)d[0], (double)d[1], (double)d[2]};
  or_walk w;
  const int32_t *it;
  int64_t cnt;
  for (or_walk_begin(&w, S->grid, od, dd, (double)tmin - S->grid->slack);
       or_walk_cell(&w, INFINITY, &it, &cnt); or_walk_step(&w))
    for (int64_t e = 0; e < cnt; ++e) {
      R t, x[3], ev[3];
      const int64_t s = it[e];
      if (SFX(hit_disk)(o, d, S->c + 3 * s, S->n + 3 * s, S->r[s], tmin, &t, x, ev)) return 1;
    }
  return 0;
}

/* Grid over the splats (centres, radii) for searches from rays whose
 * coordinates stay below `extra` in magnitude beyond the splats' own. */
static void SFX(splat_grid)(or_grid *g, const double *sc, const double *sr, int64_t ns,
                            double extra) {
  double scale = 0.0;
  for (int64_t s = 0; s < 3 * ns; ++s)
    if (fabs(sc[s]) > scale && isfinite(sc[s])) scale = fabs(sc[s]);
  or_grid_build(g, sc, sr, ns, scale + extra);
}

/* Eq. 4 (and H^r = R H^i, tube vectors likewise): a - 2 (a . n) n. */
static void SFX(reflect)(const R *a, const R *n, R *out) {
  R s = (R)2 * SFX(dot)(a, n);
  for (int k = 0; k < 3; ++k) out[k] = a[k] - s * n[k];
}

/* Trace the listed pixel rays of view `vin` (Alg. 3, bounce loop).
 * Bounce 1 comes from the view's GFB (first_t/first_idx/first_n, as produced
 * by gfb() for the same pixels) or, if first_t is NULL, from the splats with
 * tmin = 0.  Bounces 2..mb march through the splats with tmin = eps.
 * Outputs per ray: M (number of hits), hit ids per bounce ([nr][mb], -1 after
 * the last), the last-hit record (p, n, incoming k, incoming tube vectors u, v),
 * the image-method path length (FP64) and Psi (shadow test toward -d for
 * M >= 2 when do_shadow; 1 otherwise). */
static void SFX(trace)(const or_view *vin, const int64_t *pix, int64_t nr,
                       const double *first_t, const int64_t *first_idx,
                       const double *first_n, const double *sc, const double *sn,
                       const double *sr, const int64_t *sid, int64_t ns, int mb,
                       double eps, double r_ov, int do_shadow, int use_grid, int32_t *M_out,
                       int64_t *ids_out, double *p_out, double *n_out, double *k_out,
                       double *u_out, double *v_out, double *path_out,
                       uint8_t *psi_out) {
  SFX(view) V;
  SFX(load_view)(vin, &V);
  R *c = (R *)malloc(sizeof(R) * (size_t)(3 * ns + 1));
  R *n = (R *)malloc(sizeof(R) * (size_t)(3 * ns + 1));
  R *r = (R *)malloc(sizeof(R) * (size_t)(ns + 1));
  for (int64_t s = 0; s < 3 * ns; ++s) {
    c[s] = (R)sc[s];
    n[s] = (R)sn[s];
  }
  for (int64_t s = 0; s < ns; ++s) r[s] = (R)sr[s];
  or_grid grid;
  memset(&grid, 0, sizeof(grid));
  if (use_grid)
    SFX(splat_grid)(&grid, sc, sr, ns,
                    fabs(vin->o[0]) + fabs(vin->o[1]) + fabs(vin->o[2]) +
                        (double)(vin->W + vin->H) * vin->pitch);
  SFX(splatset) S = {c, n, r, sid, ns, use_grid ? &grid : NULL};
  R E = (R)eps, RO = (R)r_ov;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < nr; ++q) {
    int64_t pq = pix ? pix[q] : q;
    int i = (int)(pq % V.W), j = (int)(pq / V.W);
    R o[3], d[3], u[3], v[3], p[3], nn[3];
    SFX(pixel_origin)(&V, i, j, o);
    for (int k = 0; k < 3; ++k) {
      d[k] = V.d[k];
      u[k] = V.L * V.u[k];
      v[k] = V.L * V.v[k];
    }
    for (int b = 0; b < mb; ++b) ids_out[q * mb + b] = -1;
    int64_t id;
    int hit;
    if (first_t) {
      hit = first_idx[q] >= 0;
      if (hit) {
        R t = (R)first_t[q];
        for (int k = 0; k < 3; ++k) {
          p[k] = o[k] + t * d[k];
          nn[k] = (R)first_n[3 * q + k];
        }
        id = first_idx[q];
      }
    } else {
      hit = SFX(nearest)(&S, o, d, (R)0, RO, p, nn, &id);
    }
    int M = 0;
    double path = 0.0;
    R kin[3] = {0, 0, 0}, uin[3] = {0, 0, 0}, vin3[3] = {0, 0, 0};
    if (hit) {
      M = 1;
      ids_out[q * mb] = id;
      path = ((double)d[0] * (double)p[0] + (double)d[1] * (double)p[1]) +
             (double)d[2] * (double)p[2];
      for (int k = 0; k < 3; ++k) {
        kin[k] = d[k];
        uin[k] = u[k];
        vin3[k] = v[k];
      }
      for (int b = 2; b <= mb; ++b) {
        R rd[3], ru[3], rv[3];
        SFX(reflect)(d, nn, rd);
        R len = SQRT(SFX(dot)(rd, rd));
        for (int k = 0; k < 3; ++k) d[k] = rd[k] / len;
        SFX(reflect)(u, nn, ru);
        SFX(reflect)(v, nn, rv);
        for (int k = 0; k < 3; ++k) {
          u[k] = ru[k];
          v[k] = rv[k];
        }
        R p2[3], n2[3];
        int64_t id2;
        if (!SFX(nearest)(&S, p, d, E, RO, p2, n2, &id2)) break;
        double dx = (double)p2[0] - (double)p[0];
        double dy = (double)p2[1] - (double)p[1];
        double dz = (double)p2[2] - (double)p[2];
        path = path + sqrt((dx * dx + dy * dy) + dz * dz);
        for (int k = 0; k < 3; ++k) {
          p[k] = p2[k];
          nn[k] = n2[k];
          kin[k] = d[k];
          uin[k] = u[k];
          vin3[k] = v[k];
        }
        M = b;
        ids_out[q * mb + (b - 1)] = id2;
      }
    }
    M_out[q] = M;
    uint8_t psi = 1;
    if (M >= 2 && do_shadow) {
      R w[3] = {-V.d[0], -V.d[1], -V.d[2]};
      psi = SFX(any_hit)(&S, p, w, E) ? 0 : 1;
    }
    psi_out[q] = psi;
    for (int k = 0; k < 3; ++k) {
      p_out[3 * q + k] = M ? (double)p[k] : 0.0;
      n_out[3 * q + k] = M ? (double)nn[k] : 0.0;
      k_out[3 * q + k] = (double)kin[k];
      u_out[3 * q + k] = (double)uin[k];
      v_out[3 * q + k] = (double)vin3[k];
    }
    path_out[q] = path;
  }
  or_grid_free(&grid);
  free(c);
  free(n);
  free(r);
}

/* Psi for other receivers (bistatic observation, Eq. 14): for each ray with
 * at least one hit and each direction dirs[o] toward a receiver, 1 unless a
 * splat is hit along that direction from the ray's last hit point with
 * t > eps.  p: [nr][3] last-hit points, M: [nr] hit counts; psi_out:
 * [nobs][nr] (0 for rays without a hit). */
static void SFX(shadow_dirs)(const double *sc, const double *sn, const double *sr,
                             const int64_t *sid, int64_t ns, const double *p, const int32_t *M,
                             int64_t nr, const double *dirs, int nobs, double eps,
                             int use_grid, uint8_t *psi_out) {
  R *c = (R *)malloc(sizeof(R) * (size_t)(3 * ns + 1));
  R *n = (R *)malloc(sizeof(R) * (size_t)(3 * ns + 1));
  R *r = (R *)malloc(sizeof(R) * (size_t)(ns + 1));
  for (int64_t s = 0; s < 3 * ns; ++s) {
    c[s] = (R)sc[s];
    n[s] = (R)sn[s];
  }
  for (int64_t s = 0; s < ns; ++s) r[s] = (R)sr[s];
  or_grid grid;
  memset(&grid, 0, sizeof(grid));
  if (use_grid) {
    double extra = 0.0;
    for (int64_t q = 0; q < 3 * nr; ++q)
      if (fabs(p[q]) > extra && isfinite(p[q])) extra = fabs(p[q]);
    SFX(splat_grid)(&grid, sc, sr, ns, extra);
  }
  SFX(splatset) S = {c, n, r, sid, ns, use_grid ? &grid : NULL};
  const R E = (R)eps;
  for (int o = 0; o < nobs; ++o) {
    const R w[3] = {(R)dirs[3 * o], (R)dirs[3 * o + 1], (R)dirs[3 * o + 2]};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < nr; ++q) {
      uint8_t psi = 0;
      if (M[q] >= 1) {
        const R pq[3] = {(R)p[3 * q], (R)p[3 * q + 1], (R)p[3 * q + 2]};
        psi = SFX(any_hit)(&S, pq, w, E) ? 0 : 1;
      }
      psi_out[(int64_t)o * nr + q] = psi;
    }
  }
  or_grid_free(&grid);
  free(c);
  free(n);
  free(r);
}
