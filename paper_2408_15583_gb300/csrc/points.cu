// Surfel attributes on the GPU: the per-point inputs of Alg. 1 in surfel
// mode, computed from the point cloud alone.
//   radius[i]  mean distance to the k_r nearest other points;
//   normal[i]  the smallest principal axis of the k_n nearest points
//              (itself included), turned to agree with a reference normal
//              or away from the bounding-box centre.
//
// Exact k-nearest-neighbour search on a uniform grid: the bounding box
// (reduced on the device) is cut into G^3 cubic cells, the points are
// counting-sorted into cells, and each point searches shells of cells of
// growing Chebyshev radius until its k-th distance is below the distance to
// every unsearched cell.  Neighbours are ordered by (FP32 squared distance,
// index), with the squared distance evaluated in one fixed order, so the
// neighbour lists -- and the radii, summed in FP64 in list order -- equal a
// brute-force search bit for bit.  Queries run in cell order, so a warp's
// points are neighbours and read the same cells.
#include <cstring>

#include "pe_internal.cuh"

namespace {

constexpr int KMAX = 32;
constexpr int kPtThreads = 128;
constexpr int kBoxBlocks = 256;

struct grid_info {
  float lo[3], ctr[3];
  float h, inv_h;
  int G;
};

__device__ __forceinline__ float d2_of(float qx, float qy, float qz, const float *p) {
  const float dx = __fsub_rn(p[0], qx), dy = __fsub_rn(p[1], qy), dz = __fsub_rn(p[2], qz);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__global__ void bbox_partial(const float *__restrict__ pos, int64_t n, float *__restrict__ part) {
  __shared__ float red[6][kPtThreads];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], pos[3 * i + k]);
      hi[k] = fmaxf(hi[k], pos[3 * i + k]);
    }
  for (int k = 0; k < 3; ++k) {
    red[k][threadIdx.x] = lo[k];
    red[3 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = red[threadIdx.x][0];
    for (int t = 1; t < kPtThreads; ++t)
      v = threadIdx.x < 3 ? fminf(v, red[threadIdx.x][t]) : fmaxf(v, red[threadIdx.x][t]);
    part[blockIdx.x * 6 + threadIdx.x] = v;
  }
}

// Cubic cells of side h = (largest extent / G) (1 + 2^-10): the farthest
// point falls in cell G - 1.
__global__ void bbox_final(const float *__restrict__ part, int blocks, int G, grid_info *gi) {
  if (threadIdx.x != 0) return;
  float lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = part[k];
    hi[k] = part[3 + k];
    for (int b = 1; b < blocks; ++b) {
      lo[k] = fminf(lo[k], part[b * 6 + k]);
      hi[k] = fmaxf(hi[k], part[b * 6 + 3 + k]);
    }
  }
  float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
  if (!(ext > 0.0f)) ext = 1.0f;
  grid_info g;
  for (int k = 0; k < 3; ++k) {
    g.lo[k] = lo[k];
    g.ctr[k] = 0.5f * (lo[k] + hi[k]);
  }
  g.G = G;
  g.h = ext / (float)G * (1.0f + 1.0f / 1024.0f);
  g.inv_h = 1.0f / g.h;
  *gi = g;
}

__device__ __forceinline__ int cell_1d(const grid_info &g, float x, int k) {
  int c = (int)floorf((x - g.lo[k]) * g.inv_h);
  return c < 0 ? 0 : (c > g.G - 1 ? g.G - 1 : c);
}

__global__ void count_cells(const float *__restrict__ pos, int64_t n, const grid_info *gip,
                            uint32_t *__restrict__ count, uint32_t *__restrict__ cell_of) {
  const grid_info g = *gip;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = ((uint32_t)cell_1d(g, pos[3 * i], 0) * g.G + cell_1d(g, pos[3 * i + 1], 1)) * g.G +
                       cell_1d(g, pos[3 * i + 2], 2);
    cell_of[i] = c;
    atomicAdd(count + c, 1u);
  }
}

__global__ void scatter_cells(int64_t n, const uint32_t *__restrict__ cell_of,
                              const uint32_t *__restrict__ offs, uint32_t *__restrict__ cursor,
                              uint32_t *__restrict__ sorted) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cell_of[i];
    sorted[offs[c] + atomicAdd(cursor + c, 1u)] = (uint32_t)i;
  }
}

// Smallest-eigenvalue unit eigenvector of the symmetric 3x3 matrix
// (a00 a01 a02; a11 a12; a22) by the trigonometric solution of the
// characteristic cubic and the largest cross product of two rows of
// A - lambda I.  (0, 0, 1) when A is a multiple of the identity.
__device__ void smallest_axis(double a00, double a01, double a02, double a11, double a12,
                              double a22, double out[3]) {
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double q = (a00 + a11 + a22) / 3.0;
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  if (!(p2 > 0.0)) {
    out[0] = 0.0;
    out[1] = 0.0;
    out[2] = 1.0;
    return;
  }
  const double p = sqrt(p2 / 6.0);
  const double ip = 1.0 / p;
  const double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip,
               c12 = a12 * ip;
  double r = 0.5 * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) +
                    c02 * (c01 * c12 - c11 * c02));
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  const double lam = q + 2.0 * p * cos(phi + 2.0943951023931957);  // + 2 pi / 3: smallest
  const double r0[3] = {a00 - lam, a01, a02}, r1[3] = {a01, a11 - lam, a12},
               r2[3] = {a02, a12, a22 - lam};
  double best[3] = {0.0, 0.0, 1.0}, bn = 0.0;
  const double *rows[3][2] = {{r0, r1}, {r0, r2}, {r1, r2}};
  for (int k = 0; k < 3; ++k) {
    const double *u = rows[k][0], *v = rows[k][1];
    const double c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                         u[0] * v[1] - u[1] * v[0]};
    const double nn = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (nn > bn) {
      bn = nn;
      best[0] = c[0];
      best[1] = c[1];
      best[2] = c[2];
    }
  }
  const double s = bn > 0.0 ? 1.0 / sqrt(bn) : 1.0;
  out[0] = best[0] * s;
  out[1] = best[1] * s;
  out[2] = best[2] * s;
}

struct knn_args {
  const float *pos;
  int64_t n;
  const grid_info *gi;
  const uint32_t *offs, *sorted;
  int K, k_r, k_n;
  const float *ref;
  float *rad, *nrm;
  unsigned int *err;
};

__global__ void __launch_bounds__(kPtThreads) knn_kernel(const knn_args A) {
  const grid_info g = *A.gi;
  const int G = g.G;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < A.n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = A.sorted[t];
    const float qx = A.pos[3 * (int64_t)i], qy = A.pos[3 * (int64_t)i + 1],
                qz = A.pos[3 * (int64_t)i + 2];
    const int c[3] = {cell_1d(g, qx, 0), cell_1d(g, qy, 1), cell_1d(g, qz, 2)};
    const float q[3] = {qx, qy, qz};
    float bd[KMAX];
    uint32_t bi[KMAX];
    int cnt = 0;
    const int K = A.K;
    for (int s = 0; s <= G; ++s) {
      // the cells at Chebyshev distance s from c (inside the grid)
      for (int dz = -s; dz <= s; ++dz) {
        const int z = c[2] + dz;
        if (z < 0 || z >= G) continue;
        for (int dy = -s; dy <= s; ++dy) {
          const int y = c[1] + dy;
          if (y < 0 || y >= G) continue;
          const bool face = dz == -s || dz == s || dy == -s || dy == s;
          for (int dx = -s; dx <= s; dx += face ? 1 : (s > 0 ? 2 * s : 1)) {
            const int x = c[0] + dx;
            if (x < 0 || x >= G) continue;
            const uint32_t cell = ((uint32_t)x * G + y) * G + z;
            const uint32_t b = A.offs[cell], e = A.offs[cell + 1];
            for (uint32_t m = b; m < e; ++m) {
              const uint32_t j = A.sorted[m];
              const float d2 = d2_of(qx, qy, qz, A.pos + 3 * (int64_t)j);
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
          }
        }
      }
      // stop once the k-th distance is below the distance to every cell
      // outside the searched block (faces at the grid's edge bound nothing)
      float bound = INFINITY;
      for (int k = 0; k < 3; ++k) {
        const float slack = 1e-4f * g.h + 1e-6f * (fabsf(g.lo[k]) + (float)G * g.h);
        if (c[k] - s > 0) bound = fminf(bound, q[k] - (g.lo[k] + (float)(c[k] - s) * g.h) - slack);
        if (c[k] + s + 1 < G)
          bound = fminf(bound, (g.lo[k] + (float)(c[k] + s + 1) * g.h) - q[k] - slack);
      }
      if (bound == INFINITY) break;  // every cell searched
      if (cnt == K && bound > 0.0f && bd[K - 1] <= bound * bound) break;
    }
    if (cnt < K) {  // fewer than K points in the cloud: rejected on the host
      pe_raise(A.err, PE_ERR_OVERFLOW);
      continue;
    }
    if (A.rad) {
      double sum = 0.0;
      int used = 0;
      for (int e = 0; e < K && used < A.k_r; ++e) {
        if (bi[e] == i) continue;
        sum += sqrt((double)bd[e]);
        ++used;
      }
      A.rad[i] = (float)(sum / (double)A.k_r);
    }
    if (A.nrm) {
      double m[3] = {0.0, 0.0, 0.0};
      for (int e = 0; e < A.k_n; ++e)
        for (int k = 0; k < 3; ++k) m[k] += (double)A.pos[3 * (int64_t)bi[e] + k];
      for (int k = 0; k < 3; ++k) m[k] /= (double)A.k_n;
      double a00 = 0, a01 = 0, a02 = 0, a11 = 0, a12 = 0, a22 = 0;
      for (int e = 0; e < A.k_n; ++e) {
        const float *p = A.pos + 3 * (int64_t)bi[e];
        const double x = (double)p[0] - m[0], y = (double)p[1] - m[1], z = (double)p[2] - m[2];
        a00 += x * x;
        a01 += x * y;
        a02 += x * z;
        a11 += y * y;
        a12 += y * z;
        a22 += z * z;
      }
      double v[3];
      smallest_axis(a00, a01, a02, a11, a12, a22, v);
      double w[3];
      if (A.ref) {
        for (int k = 0; k < 3; ++k) w[k] = (double)A.ref[3 * (int64_t)i + k];
      } else {
        for (int k = 0; k < 3; ++k) w[k] = (double)q[k] - (double)g.ctr[k];
      }
      if (v[0] * w[0] + v[1] * w[1] + v[2] * w[2] < 0.0)
        for (int k = 0; k < 3; ++k) v[k] = -v[k];
      for (int k = 0; k < 3; ++k) A.nrm[3 * (int64_t)i + k] = (float)v[k];
    }
  }
}

int grid_res(int64_t n) {
  // about (2.5 n^(1/3))^3 cells: a surface sampled by n points puts a few
  // dozen points in each occupied cell
  double g = 2.5 * cbrt((double)n);
  int G = (int)g;
  return G < 4 ? 4 : (G > 255 ? 255 : G);
}

struct pt_ws {
  float *part;
  grid_info *gi;
  uint32_t *count, *offs, *cursor, *tile, *cell_of, *sorted;
};

pt_ws carve(pe_carve &c, int64_t n) {
  const int G = grid_res(n);
  const int64_t cells = (int64_t)G * G * G;
  pt_ws w;
  w.part = c.take<float>(kBoxBlocks * 6);
  w.gi = c.take<grid_info>(1);
  w.count = c.take<uint32_t>((size_t)cells);
  w.offs = c.take<uint32_t>((size_t)cells + 1);
  w.cursor = c.take<uint32_t>((size_t)cells);
  w.tile = c.take<uint32_t>((size_t)((cells + 4095) / 4096 + 1));
  w.cell_of = c.take<uint32_t>((size_t)n);
  w.sorted = c.take<uint32_t>((size_t)n);
  return w;
}

}  // namespace

namespace {

// The processing order of pe_order_points: the same counting sort into a
// 32^3 grid over the bounding box, cells in raster order (a warp's 32 points
// then mostly share a cell of about 1/32 of the target's extent).
constexpr int kOrderGrid = 32;

pt_ws carve_order(pe_carve &c, int64_t n) {
  const int64_t cells = (int64_t)kOrderGrid * kOrderGrid * kOrderGrid;
  pt_ws w;
  w.part = c.take<float>(kBoxBlocks * 6);
  w.gi = c.take<grid_info>(1);
  w.count = c.take<uint32_t>((size_t)cells);
  w.offs = c.take<uint32_t>((size_t)cells + 1);
  w.cursor = c.take<uint32_t>((size_t)cells);
  w.tile = c.take<uint32_t>((size_t)((cells + 4095) / 4096 + 1));
  w.cell_of = c.take<uint32_t>((size_t)n);
  w.sorted = nullptr;  // the caller's order buffer
  return w;
}

}  // namespace

extern "C" size_t pe_order_points_workspace(int64_t n_points) {
  if (n_points < 1 || n_points >= (int64_t)UINT32_MAX) return 0;
  pe_carve c{nullptr, 0};
  carve_order(c, n_points);
  return c.bytes() + 256;
}

extern "C" pe_status pe_order_points(const float *pos, int64_t n_points, void *ws, size_t ws_bytes,
                                     uint32_t *order, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!pos || !order || n_points < 1 || n_points >= (int64_t)UINT32_MAX)
    return pe_fail(PE_EINVAL, "pe_order_points: bad arguments");
  const size_t need = pe_order_points_workspace(n_points);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_order_points: workspace needs %zu bytes", need);
  pe_carve c{static_cast<char *>(ws), 0};
  pt_ws w = carve_order(c, n_points);
  const int64_t cells = (int64_t)kOrderGrid * kOrderGrid * kOrderGrid;
  bbox_partial<<<kBoxBlocks, kPtThreads, 0, s>>>(pos, n_points, w.part);
  PE_TRY_LAUNCH("bbox_partial");
  bbox_final<<<1, 32, 0, s>>>(w.part, kBoxBlocks, kOrderGrid, w.gi);
  PE_TRY_LAUNCH("bbox_final");
  PE_TRY_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * cells, s));
  PE_TRY_CUDA(cudaMemsetAsync(w.cursor, 0, sizeof(uint32_t) * cells, s));
  int64_t b = (n_points + 255) / 256;
  const int blocks = (int)(b < 4096 ? b : 4096);
  count_cells<<<blocks, 256, 0, s>>>(pos, n_points, w.gi, w.count, w.cell_of);
  PE_TRY_LAUNCH("count_cells");
  pe_status st = pe_exclusive_scan_u32(w.count, cells, w.tile, w.offs, s);
  if (st != PE_OK) return st;
  scatter_cells<<<blocks, 256, 0, s>>>(n_points, w.cell_of, w.offs, w.cursor, order);
  PE_TRY_LAUNCH("scatter_cells");
  return PE_OK;
}

extern "C" size_t pe_point_attributes_workspace(int64_t n_points) {
  if (n_points < 1) return 0;
  pe_carve c{nullptr, 0};
  carve(c, n_points);
  return c.bytes() + 256;
}

extern "C" pe_status pe_point_attributes(const float *pos, int64_t n_points, int32_t k_r,
                                         int32_t k_n, const float *ref_nrm, void *ws,
                                         size_t ws_bytes, float *radius, float *normal,
                                         void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!pos || n_points < 1 || n_points >= (int64_t)UINT32_MAX || (!radius && !normal))
    return pe_fail(PE_EINVAL, "pe_point_attributes: bad arguments");
  if ((radius && (k_r < 1 || k_r > KMAX - 1)) || (normal && (k_n < 3 || k_n > KMAX)))
    return pe_fail(PE_EINVAL, "pe_point_attributes: k_r in [1, %d], k_n in [3, %d]", KMAX - 1, KMAX);
  const int K = (radius ? k_r + 1 : 0) > (normal ? k_n : 0) ? k_r + 1 : (normal ? k_n : 0);
  if (n_points < K)
    return pe_fail(PE_EINVAL, "pe_point_attributes: needs at least %d points", K);
  const size_t need = pe_point_attributes_workspace(n_points);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_point_attributes: workspace needs %zu bytes", need);
  pe_carve c{static_cast<char *>(ws), 0};
  pt_ws w = carve(c, n_points);
  const int G = grid_res(n_points);
  const int64_t cells = (int64_t)G * G * G;
  bbox_partial<<<kBoxBlocks, kPtThreads, 0, s>>>(pos, n_points, w.part);
  PE_TRY_LAUNCH("bbox_partial");
  bbox_final<<<1, 32, 0, s>>>(w.part, kBoxBlocks, G, w.gi);
  PE_TRY_LAUNCH("bbox_final");
  PE_TRY_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * cells, s));
  PE_TRY_CUDA(cudaMemsetAsync(w.cursor, 0, sizeof(uint32_t) * cells, s));
  int64_t b = (n_points + 255) / 256;
  const int blocks = (int)(b < 4096 ? b : 4096);
  count_cells<<<blocks, 256, 0, s>>>(pos, n_points, w.gi, w.count, w.cell_of);
  PE_TRY_LAUNCH("count_cells");
  pe_status st = pe_exclusive_scan_u32(w.count, cells, w.tile, w.offs, s);
  if (st != PE_OK) return st;
  scatter_cells<<<blocks, 256, 0, s>>>(n_points, w.cell_of, w.offs, w.cursor, w.sorted);
  PE_TRY_LAUNCH("scatter_cells");
  knn_args A;
  memset(&A, 0, sizeof(A));
  A.pos = pos;
  A.n = n_points;
  A.gi = w.gi;
  A.offs = w.offs;
  A.sorted = w.sorted;
  A.K = K;
  A.k_r = k_r;
  A.k_n = k_n;
  A.ref = ref_nrm;
  A.rad = radius;
  A.nrm = normal;
  A.err = pe_err_word();
  int64_t qb = (n_points + kPtThreads - 1) / kPtThreads;
  pe_event_before("knn_kernel", s);
  knn_kernel<<<(int)(qb < 65535 * 16 ? qb : 65535 * 16), kPtThreads, 0, s>>>(A);
  pe_event_after("knn_kernel", s);
  PE_TRY_LAUNCH("knn_kernel");
  return PE_OK;
}
