/*
 * PointEMRay CPU oracle -- uniform-grid candidate lists (TEST INFRASTRUCTURE
 * ONLY).
 *
 * The oracle's searches (nearest surfel per pixel ray for Alg. 1, nearest
 * splat and the Eq. 23 candidate set per bounce ray, any splat along a shadow
 * ray) are brute force over every element.  At the workloads' full sizes that
 * is 10^11 and more disk tests, so the same searches can draw their candidates
 * from a uniform 3D grid instead: every element (a disk of radius R, or a
 * point with a tube of radius delta around the ray) is listed in every cell
 * that its bounding box, padded, overlaps; a ray walks the cells it crosses in
 * order of its parameter t (a 3D DDA, Amanatides & Woo 1987) and tests the
 * listed elements with the very same per-element test as the brute-force loop.
 * Only the set of elements tested changes, never the test or the rule that
 * picks among the hits, so the result equals the brute-force result bit for
 * bit:
 *   - a valid hit point lies within R of its element's centre (the disk test
 *     itself guarantees it, up to the rounding of its own arithmetic), so the
 *     point of the ray at the hit's t lies in a cell that lists the element;
 *     the padding covers the rounding of the FP32 hit point and of the walk;
 *   - the walk visits cells in increasing t and stops only once a cell is
 *     entered beyond the current bound (nearest t plus a slack), so every cell
 *     holding a point of the ray with t at or below the bound has been
 *     visited.
 * The grid is pure acceleration: all of its arithmetic is FP64 and none of it
 * reaches an output.  Its results are tested against the brute-force path
 * bit for bit on small cases.
 */

typedef struct {
  double lo[3];     /* grid origin */
  double cell;      /* cubic cell edge */
  double inv;       /* 1 / cell */
  int n[3];         /* cells per axis */
  int64_t *start;   /* [cells + 1]: the list of cell k is item[start[k] .. start[k+1]) */
  int32_t *item;    /* element indices, ascending within a cell */
  double slack;     /* t slack of the walk's stopping rule */
  int ok;           /* 0: no element with a finite box (every search misses) */
} or_grid;

static int or_cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static void or_grid_free(or_grid *g) {
  free(g->start);
  free(g->item);
  g->start = NULL;
  g->item = NULL;
}

/* Grid over n elements with centres c[3*i..] and radii r[i] (the element's
 * reach from its centre).  Elements with a non-finite centre or radius are
 * left out: the per-element tests never accept them (every comparison with a
 * NaN is false).  Cell edge: twice the median radius, grown if the grid would
 * exceed about 8M cells.  scale bounds the magnitude of the coordinates the
 * searches will use (elements and ray origins); it sets the padding. */
static void or_grid_build(or_grid *g, const double *c, const double *r, int64_t n,
                          double scale) {
  memset(g, 0, sizeof(*g));
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double *rs = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int64_t nf = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double *ci = c + 3 * i;
    if (!(isfinite(ci[0]) && isfinite(ci[1]) && isfinite(ci[2]) && isfinite(r[i]))) continue;
    double ri = fabs(r[i]);
    for (int k = 0; k < 3; ++k) {
      if (ci[k] - ri < lo[k]) lo[k] = ci[k] - ri;
      if (ci[k] + ri > hi[k]) hi[k] = ci[k] + ri;
    }
    rs[nf++] = ri;
  }
  if (nf == 0) {
    free(rs);
    g->ok = 0;
    return;
  }
  qsort(rs, (size_t)nf, sizeof(double), or_cmp_double);
  double ext = 0.0;
  for (int k = 0; k < 3; ++k)
    if (hi[k] - lo[k] > ext) ext = hi[k] - lo[k];
  double cell = 2.0 * rs[nf / 2];
  free(rs);
  if (!(cell > 0.0)) cell = ext > 0.0 ? ext / cbrt((double)nf) : 1.0;
  if (!(cell > 0.0)) cell = 1.0;
  /* padding: far above the rounding of FP32 hit points (a few ulps of the
   * largest coordinate) and of the FP64 walk */
  double pad = 1e-3 * cell + 1e-5 * scale;
  for (;;) {
    double cells = 1.0;
    for (int k = 0; k < 3; ++k) cells *= floor((hi[k] - lo[k] + 2.0 * pad) / cell) + 1.0;
    if (cells <= 8.0e6) break;
    cell *= 1.25;
    pad = 1e-3 * cell + 1e-5 * scale;
  }
  for (int k = 0; k < 3; ++k) {
    g->lo[k] = lo[k] - pad;
    g->n[k] = (int)floor((hi[k] - lo[k] + 2.0 * pad) / cell) + 1;
  }
  g->cell = cell;
  g->inv = 1.0 / cell;
  g->slack = 1e-3 * cell + 1e-5 * scale;
  const int64_t nc = (int64_t)g->n[0] * g->n[1] * g->n[2];
  g->start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  /* two passes: count, then fill in ascending element order */
  for (int pass = 0; pass < 2; ++pass) {
    int64_t *fill = NULL;
    if (pass == 1) {
      for (int64_t k = 0; k < nc; ++k) g->start[k + 1] += g->start[k];
      g->item = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->start[nc] > 0 ? g->start[nc] : 1));
      fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
      memcpy(fill, g->start, sizeof(int64_t) * (size_t)nc);
    }
    for (int64_t i = 0; i < n; ++i) {
      const double *ci = c + 3 * i;
      if (!(isfinite(ci[0]) && isfinite(ci[1]) && isfinite(ci[2]) && isfinite(r[i]))) continue;
      double ri = fabs(r[i]) + pad;
      int a[3], b[3];
      for (int k = 0; k < 3; ++k) {
        a[k] = (int)floor((ci[k] - ri - g->lo[k]) * g->inv);
        b[k] = (int)floor((ci[k] + ri - g->lo[k]) * g->inv);
        if (a[k] < 0) a[k] = 0;
        if (b[k] > g->n[k] - 1) b[k] = g->n[k] - 1;
      }
      for (int x = a[0]; x <= b[0]; ++x)
        for (int y = a[1]; y <= b[1]; ++y)
          for (int z = a[2]; z <= b[2]; ++z) {
            int64_t k = ((int64_t)x * g->n[1] + y) * g->n[2] + z;
            if (pass == 0)
              g->start[k + 1] += 1;
            else
              g->item[fill[k]++] = (int32_t)i;
          }
    }
    free(fill);
  }
  g->ok = 1;
}

/* Walk of the cells a ray o + t d (t >= t0) crosses, in increasing t. */
typedef struct {
  const or_grid *g;
  int ix[3], step[3];
  double tmax[3], tdelta[3];
  double t_in;      /* t at which the current cell is entered */
  double t_end;     /* t at which the ray leaves the grid */
  int live;
} or_walk;

static void or_walk_begin(or_walk *w, const or_grid *g, const double *o, const double *d,
                          double t0) {
  w->g = g;
  w->live = 0;
  if (!g->ok) return;
  double te = t0, tx = INFINITY;
  for (int k = 0; k < 3; ++k) {
    double a = g->lo[k], b = g->lo[k] + g->n[k] * g->cell;
    if (d[k] == 0.0) {
      if (o[k] < a || o[k] > b) return;
      continue;
    }
    double t1 = (a - o[k]) / d[k], t2 = (b - o[k]) / d[k];
    if (t1 > t2) {
      double s = t1;
      t1 = t2;
      t2 = s;
    }
    if (t1 > te) te = t1;
    if (t2 < tx) tx = t2;
  }
  if (!(te <= tx)) return;
  for (int k = 0; k < 3; ++k) {
    double pk = o[k] + te * d[k];
    int i = (int)floor((pk - g->lo[k]) * g->inv);
    if (i < 0) i = 0;
    if (i > g->n[k] - 1) i = g->n[k] - 1;
    w->ix[k] = i;
    if (d[k] > 0.0) {
      w->step[k] = 1;
      w->tmax[k] = (g->lo[k] + (i + 1) * g->cell - o[k]) / d[k];
      w->tdelta[k] = g->cell / d[k];
    } else if (d[k] < 0.0) {
      w->step[k] = -1;
      w->tmax[k] = (g->lo[k] + i * g->cell - o[k]) / d[k];
      w->tdelta[k] = -g->cell / d[k];
    } else {
      w->step[k] = 0;
      w->tmax[k] = INFINITY;
      w->tdelta[k] = INFINITY;
    }
  }
  w->t_in = te;
  w->t_end = tx;
  w->live = 1;
}

/* The current cell's element list, or 0 once the walk has left the grid or
 * the current cell is entered beyond t_stop + slack.  Advance with
 * or_walk_step after using it. */
static int or_walk_cell(const or_walk *w, double t_stop, const int32_t **items, int64_t *count) {
  if (!w->live || w->t_in > t_stop + w->g->slack) return 0;
  const or_grid *g = w->g;
  int64_t k = ((int64_t)w->ix[0] * g->n[1] + w->ix[1]) * g->n[2] + w->ix[2];
  *items = g->item + g->start[k];
  *count = g->start[k + 1] - g->start[k];
  return 1;
}

static void or_walk_step(or_walk *w) {
  int a = 0;
  if (w->tmax[1] < w->tmax[a]) a = 1;
  if (w->tmax[2] < w->tmax[a]) a = 2;
  double t = w->tmax[a];
  w->ix[a] += w->step[a];
  w->tmax[a] += w->tdelta[a];
  if (w->ix[a] < 0 || w->ix[a] >= w->g->n[a] || !(t <= w->t_end) || w->step[a] == 0) {
    w->live = 0;
    return;
  }
  w->t_in = t;
}

/* A growable list of element indices (per query), sorted and de-duplicated
 * on request. */
typedef struct {
  int32_t *v;
  int64_t n, cap;
} or_list;

static void or_list_push(or_list *L, int32_t x) {
  if (L->n == L->cap) {
    L->cap = L->cap ? 2 * L->cap : 64;
    L->v = (int32_t *)realloc(L->v, sizeof(int32_t) * (size_t)L->cap);
  }
  L->v[L->n++] = x;
}

static int or_cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static void or_list_sort_unique(or_list *L) {
  if (L->n < 2) return;
  qsort(L->v, (size_t)L->n, sizeof(int32_t), or_cmp_i32);
  int64_t m = 1;
  for (int64_t i = 1; i < L->n; ++i)
    if (L->v[i] != L->v[m - 1]) L->v[m++] = L->v[i];
  L->n = m;
}
