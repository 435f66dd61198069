/*
 * PointEMRay CPU oracle (TEST INFRASTRUCTURE ONLY -- only tests/, the smoke
 * check and the benchmark's CPU-baseline leg load this library).
 *
 * A plain, slow, brute-force statement of the SBR-on-points method of
 * PointEMRay (arXiv 2408.15583), written from the paper:
 *   - geometry (GFB, fusion, bounce tracing) in oracle_core.h, compiled twice:
 *     or_*_f32 (FP32 geometry, the bit-exact target of the GPU path) and
 *     or_*_f64 (FP64 physics reference);
 *   - the physical-optics field sum of Eq. 5-14 here, always in FP64 with
 *     Neumaier-compensated sums over rays.
 * Shares no code with the CUDA path.  Build: gcc -O2 -ffp-contract=off
 * (no fast-math) -fopenmp -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double o[3], u[3], v[3], d[3];
  double pitch;
  int32_t W, H;
} or_view;

#include "oracle_grid.h"

#define R float
#define SFX(x) x##_f32
#define SQRT sqrtf
#define FLOOR floorf
#include "oracle_core.h"
#undef R
#undef SFX
#undef SQRT
#undef FLOOR

#define R double
#define SFX(x) x##_f64
#define SQRT sqrt
#define FLOOR floor
#include "oracle_core.h"
#undef R
#undef SFX
#undef SQRT
#undef FLOOR

int or_abi_version(void) { return 1; }

/* Threads the oracle's parallel loops use from now on (n >= 1), when built
 * with OpenMP; returns the number in force (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
#endif
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void or_gfb(int fp64, const or_view *v, const float *pos, const float *nrm,
            const float *rad, int64_t n, int mode, double delta,
            const int64_t *pix, int64_t npix, int use_grid, double *depth, int64_t *idx,
            double *nrm_out) {
  if (fp64)
    gfb_f64(v, pos, nrm, rad, n, mode, delta, pix, npix, use_grid, depth, idx, nrm_out);
  else
    gfb_f32(v, pos, nrm, rad, n, mode, delta, pix, npix, use_grid, depth, idx, nrm_out);
}

void or_gfb_topk(int fp64, const or_view *v, const float *pos, int64_t n, double delta, int K,
                 const int64_t *pix, int64_t npix, double *depth, int64_t *idx) {
  if (fp64)
    gfb_topk_f64(v, pos, n, delta, K, pix, npix, depth, idx);
  else
    gfb_topk_f32(v, pos, n, delta, K, pix, npix, depth, idx);
}

int64_t or_aggregate(int fp64, int nv, const or_view *views, const double *depth,
                     const double *nrm, const uint8_t *mask, double tau, int edge_mode,
                     const double *bmin, double inv_vox, int G, int64_t *out_id,
                     double *out_c, double *out_n, double *out_r,
                     int32_t *out_count, uint8_t *keep) {
  if (fp64)
    return aggregate_f64(nv, views, depth, nrm, mask, tau, edge_mode, bmin, inv_vox, G,
                         out_id, out_c, out_n, out_r, out_count, keep);
  return aggregate_f32(nv, views, depth, nrm, mask, tau, edge_mode, bmin, inv_vox, G, out_id,
                       out_c, out_n, out_r, out_count, keep);
}

void or_trace(int fp64, const or_view *v, const int64_t *pix, int64_t nr,
              const double *first_t, const int64_t *first_idx,
              const double *first_n, const double *sc, const double *sn,
              const double *sr, const int64_t *sid, int64_t ns, int mb, double eps,
              double r_ov, int do_shadow, int use_grid, int32_t *M, int64_t *ids, double *p,
              double *n, double *k, double *u, double *vv, double *path,
              uint8_t *psi) {
  if (fp64)
    trace_f64(v, pix, nr, first_t, first_idx, first_n, sc, sn, sr, sid, ns, mb,
              eps, r_ov, do_shadow, use_grid, M, ids, p, n, k, u, vv, path, psi);
  else
    trace_f32(v, pix, nr, first_t, first_idx, first_n, sc, sn, sr, sid, ns, mb,
              eps, r_ov, do_shadow, use_grid, M, ids, p, n, k, u, vv, path, psi);
}

void or_shadow_dirs(int fp64, const double *sc, const double *sn, const double *sr,
                    const int64_t *sid, int64_t ns, const double *p, const int32_t *M, int64_t nr,
                    const double *dirs, int nobs, double eps, int use_grid, uint8_t *psi) {
  if (fp64)
    shadow_dirs_f64(sc, sn, sr, sid, ns, p, M, nr, dirs, nobs, eps, use_grid, psi);
  else
    shadow_dirs_f32(sc, sn, sr, sid, ns, p, M, nr, dirs, nobs, eps, use_grid, psi);
}

/* ---------------------------------------------------------------------------
 * Physical optics (Sec. II-B, II-C).
 * ------------------------------------------------------------------------- */

static const double OR_C0 = 299792458.0;
static const double OR_PI = 3.14159265358979323846;

static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* sinc(x) = sin(x)/x, sinc(0) = 1: the unnormalised sinc that results from
 * integrating exp(-j q u) over an interval of length U (Eq. 10-11). */
static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* Neumaier-compensated accumulator (Neumaier 1974, the improved Kahan
 * summation): s carries the running sum, c the rounding errors of its
 * additions, each recovered exactly by the Fast2Sum of the larger and the
 * smaller operand; the sum is s + c. */
typedef struct {
  double s, c;
} or_acc;
static void acc_add(or_acc *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

/* The field's accumulator over a list of terms, for its pins: out[0] = the
 * compensated sum s + c, out[1] = s alone (the plain left-to-right sum). */
void or_acc_sum(const double *x, int64_t n, double *out) {
  or_acc a = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) acc_add(&a, x[i]);
  out[0] = a.s + a.c;
  out[1] = a.s;
}

/* Eq. 14 without the common factor -j eta0 k0 / (2 pi):
 *   Sigma(f, pol) = sum_l Phi_l Psi_l |u' x v'| sinc(q.u'/2) sinc(q.v'/2)
 *                   [(n x h) x ks] x ks exp(-j k (d - ks . p))
 * with q = k (k_in - ks) and u', v' from Eq. 12-13 (k_in is the ray's
 * direction of travel into its last hit).  Two transmit polarisations: for a
 * screen frame (u_hat, v_hat, w_hat) with propagation -w_hat, the electric
 * field along theta_hat = u_hat (V) has magnetic polarisation -v_hat and the
 * one along phi_hat = v_hat (H) has +u_hat; both are carried by the
 * propagated tube vectors, so h_V = -v/|v| and h_H = u/|u|.
 * Output E[obs][f][pol(V,H)][xyz][re,im]. */
void or_po_field(int64_t nr, const double *p, const double *n, const double *k,
                 const double *u, const double *v, const double *path,
                 const uint8_t *use, int nf, const double *freqs, int nobs,
                 const double *ks_dirs, double *E) {
  /* every (receiver, frequency) sample is its own sum over the rays, in ray
   * order, so the samples can be computed in parallel */
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int o = 0; o < nobs; ++o) {
    for (int f = 0; f < nf; ++f) {
      const double *ks = ks_dirs + 3 * o;
      double kw = 2.0 * OR_PI * freqs[f] / OR_C0;
      or_acc acc[2][3][2];
      memset(acc, 0, sizeof(acc));
      for (int64_t l = 0; l < nr; ++l) {
        if (!use[l]) continue;
        const double *pl = p + 3 * l, *nl = n + 3 * l, *kl = k + 3 * l;
        const double *ul = u + 3 * l, *vl = v + 3 * l;
        double nk = dot3(nl, kl);
        if (nk == 0.0) continue;
        double up[3], vp[3], nu = dot3(nl, ul) / nk, nv = dot3(nl, vl) / nk;
        for (int c = 0; c < 3; ++c) {
          up[c] = ul[c] - kl[c] * nu;
          vp[c] = vl[c] - kl[c] * nv;
        }
        double cr[3];
        cross3(up, vp, cr);
        double area = sqrt(dot3(cr, cr));
        double q[3];
        for (int c = 0; c < 3; ++c) q[c] = kw * (kl[c] - ks[c]);
        double amp = area * sinc(0.5 * dot3(q, up)) * sinc(0.5 * dot3(q, vp));
        double ph = kw * (path[l] - dot3(ks, pl));
        double cre = cos(ph), cim = -sin(ph);
        double lu = sqrt(dot3(ul, ul)), lv = sqrt(dot3(vl, vl));
        double h[2][3];
        for (int c = 0; c < 3; ++c) {
          h[0][c] = -vl[c] / lv; /* V: E along theta_hat */
          h[1][c] = ul[c] / lu;  /* H: E along phi_hat   */
        }
        for (int pol = 0; pol < 2; ++pol) {
          double a[3], b[3], vec[3];
          cross3(nl, h[pol], a);
          cross3(a, ks, b);
          cross3(b, ks, vec);
          for (int c = 0; c < 3; ++c) {
            acc_add(&acc[pol][c][0], amp * vec[c] * cre);
            acc_add(&acc[pol][c][1], amp * vec[c] * cim);
          }
        }
      }
      for (int pol = 0; pol < 2; ++pol)
        for (int c = 0; c < 3; ++c)
          for (int ri = 0; ri < 2; ++ri)
            E[((((int64_t)o * nf + f) * 2 + pol) * 3 + c) * 2 + ri] =
                acc[pol][c][ri].s + acc[pol][c][ri].c;
    }
  }
}

/* ---------------------------------------------------------------------------
 * Surfel attributes (the inputs of Alg. 1 in surfel mode): the K nearest
 * points of every point by brute force.  Squared distance in FP32 as
 * (dx*dx + dy*dy) + dz*dz with dx = p_j - p_i; neighbours ordered by
 * (squared distance, index); the point itself is included (distance 0).
 * For the points queries[0..nq) (all points, nq = n, when queries is null);
 * out_idx / out_d2: [nq][K].
 * ------------------------------------------------------------------------- */
void or_knn(const float *pos, int64_t n, const int64_t *queries, int64_t nq, int K,
            int64_t *out_idx, float *out_d2) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t qi = 0; qi < nq; ++qi) {
    const int64_t i = queries ? queries[qi] : qi;
    float bd[64];
    int64_t bi[64];
    int cnt = 0;
    const float qx = pos[3 * i], qy = pos[3 * i + 1], qz = pos[3 * i + 2];
    for (int64_t j = 0; j < n; ++j) {
      float dx = pos[3 * j] - qx, dy = pos[3 * j + 1] - qy, dz = pos[3 * j + 2] - qz;
      float d2 = (dx * dx + dy * dy) + dz * dz;
      if (cnt == K && !(d2 < bd[K - 1] || (d2 == bd[K - 1] && j < bi[K - 1]))) continue;
      int at = cnt < K ? cnt++ : K - 1;
      while (at > 0 && (bd[at - 1] > d2 || (bd[at - 1] == d2 && bi[at - 1] > j))) {
        bd[at] = bd[at - 1];
        bi[at] = bi[at - 1];
        --at;
      }
      bd[at] = d2;
      bi[at] = j;
    }
    for (int e = 0; e < K; ++e) {
      out_idx[qi * K + e] = e < cnt ? bi[e] : -1;
      out_d2[qi * K + e] = e < cnt ? bd[e] : INFINITY;
    }
  }
}
