// a6: physical-optics aperture field sum (Eq. 5-14) over rays x frequencies.
//
// Per ray, the frequency-independent parts of Eq. 14 are computed once and
// staged in shared memory: the projected tube vectors of Eq. 12-13, the
// parallelogram area |u' x v'|, the sinc arguments per unit wavenumber, the
// two polarisations' vector factors [(n x h) x ks] x ks, and the phase path
// d - ks . p (FP64, split into a float hi/lo pair).  The vector factor is
// perpendicular to ks (it is minus the part of n x h across ks), so it is
// kept as its two coordinates in an orthonormal basis (e1, e2) of the plane
// across ks.  Threads then run one frequency each over the staged rays:
// sinc x sinc, the phase k (d - ks.p) as a double-float product reduced
// modulo 2 pi, one sincos, eight multiply-adds.  Each thread keeps float sums
// compensated with TwoSum every few terms; the block reduces the threads'
// (hi + lo) in FP64 in a fixed order and a second kernel sums the blocks in a
// fixed order and turns the two coordinates back into the field's three
// Cartesian components, so the field is deterministic.
#include <cstring>

#include "pe_internal.cuh"

namespace {

constexpr int kPoThreads = 256;
constexpr int kPoGroups = 64;    // groups (angles) per launch
constexpr int kPoFreqs = 256;    // frequencies per launch
#ifndef PE_PO_FLUSH
#define PE_PO_FLUSH 64
#endif
constexpr int kFlush = PE_PO_FLUSH;  // terms between TwoSum flushes
constexpr int kAcc = 8;          // sums per (ray, frequency): 2 pol x (e1, e2) x (re, im)
constexpr float kTwoPi = 6.28318530717958647692f;

struct po_consts {
  int32_t ng, nf;
  int32_t fl;            // frequency lanes per block (power of two <= 64)
  int32_t n_chunks;
  int64_t rpg, chunk;    // rays per group, rays per block (multiple of 256)
  int32_t g0;            // first group of this launch (slot offset g0 * rpg)
  int32_t rl_shift;      // log2 of the ray lanes per block (256 / fl)
  float ks[kPoGroups][3];
  float e1[kPoGroups][3], e2[kPoGroups][3];  // orthonormal basis across ks
  float k[kPoFreqs];                  // wavenumber (rad/m), for the sinc arguments
  float khi[kPoFreqs], klo[kPoFreqs];  // k / 2 pi = f / c (revolutions/m) as a float pair
  float k2[kPoFreqs];                  // k^2 (uniform grids: the sinc series variable)
  float dkhi, dklo;                    // uniform grids: the step of k / 2 pi, a float pair
  float kmax;                          // the launch's largest k
  long long *stats;                    // nullable: [7] += contributing rays x nf
  // implicit bounce-1 records (pe_gfb_src): null keys1 = every record is
  // in the arrays; else a slot with M == 1 takes its record from its key
  const unsigned long long *keys1;
  const float *nrm1;
  pe_view view1[kPoGroups];            // the launch's groups' views
  int32_t mono1[kPoGroups];            // ks == -d of that view, bit for bit
};

// Adds this thread's count of contributing rays, times the launch's
// frequencies, to stats[7] (one atomic per warp).  Every thread of the block
// calls it at the end of the kernel.
__device__ __forceinline__ void count_terms(const po_consts &C, long long rays) {
  if (!C.stats) return;  // a kernel argument: uniform over the block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rays += __shfl_down_sync(0xffffffffu, rays, o);
  if ((threadIdx.x & 31) == 0 && rays)
    atomicAdd(reinterpret_cast<unsigned long long *>(C.stats + 7),
              (unsigned long long)(rays * C.nf));
}

// sin(x)/x: Taylor series through x^8 for |x| < 0.5 (truncation < 3e-11),
// otherwise the hardware sine divided by x.
__device__ __forceinline__ float sincf_(float x) {
  float ax = fabsf(x);
  if (ax < 0.5f) {
    float x2 = x * x;
    return 1.0f + x2 * (-1.0f / 6.0f + x2 * (1.0f / 120.0f + x2 * (-1.0f / 5040.0f +
                                                                  x2 * (1.0f / 362880.0f))));
  }
  return __fdividef(__sinf(x), x);
}

__device__ __forceinline__ void two_sum_into(float &hi, float &lo, float b) {
  float s = hi + b;
  float bp = s - hi;
  float e = (hi - (s - bp)) + (b - bp);
  hi = s;
  lo += e;
}

__device__ __forceinline__ pe_f3 cross(pe_f3 a, pe_f3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float dotf(pe_f3 a, pe_f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// 2 (a . b) as an unevaluated float pair hi + lo (|lo| <= ulp(hi) / 2) in
// FP32 operations alone: each product split exactly by an FMA (TwoProduct),
// the three products added by Knuth's TwoSum with their low parts gathered;
// the error stays below 2^-44 of the largest product (a phase error below
// 1e-10 revolutions at 18 GHz 30 m from the origin).  (FP64 issues at 1/64 of
// the FP32 rate on sm_103a, and the FP64 form of this dot product, with its
// conversions, cost the field sum as much as a third of its time.)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
__device__ __forceinline__ void twice_dot_pair(pe_f3 a, pe_f3 b, float &hi, float &lo) {
  const float p0 = __fmul_rn(a.x, b.x), p1 = __fmul_rn(a.y, b.y), p2 = __fmul_rn(a.z, b.z);
  const float e0 = __fmaf_rn(a.x, b.x, -p0), e1 = __fmaf_rn(a.y, b.y, -p1),
              e2 = __fmaf_rn(a.z, b.z, -p2);
  float s, t0, t1;
  two_sum(p0, p1, s, t0);
  two_sum(s, p2, s, t1);
  const float l = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), e2), __fadd_rn(t0, t1));
  two_sum(s, l, hi, lo);
  hi = __fmul_rn(2.0f, hi);
  lo = __fmul_rn(2.0f, lo);
}

// The words of slot `slot` that decide its record: bounce count, Psi and,
// where bounce-1 records are implicit, its GFB key (loaded whatever M is, so
// the three loads are independent).
struct ray_words {
  int32_t M;
  uint32_t psi;
  unsigned long long key;
};
__device__ __forceinline__ ray_words load_words(const pe_hits &h, const po_consts &C,
                                                int64_t slot) {
  ray_words w;
  w.M = h.M[slot];
  w.psi = h.psi[slot];
  w.key = C.keys1 ? __ldg(C.keys1 + slot) : 0ull;
  return w;
}

// The frequency-independent factors of ray `slot` (Eq. 12-14): the sinc
// arguments per unit wavenumber (au, av), the phase path d - ks.p as a float
// pair (dh, dl) and the area-weighted vector factors of both polarisations in
// the basis (e1, e2).  False for a ray without a contribution (a miss,
// Psi = 0, or a tube edge-on to the surface).
// (r: the slot's index within its group g of the launch.)
__device__ __forceinline__ bool ray_factors(const pe_hits &h, int64_t slot, const ray_words &w,
                                            pe_f3 ks, pe_f3 e1, pe_f3 e2, float &au, float &av,
                                            float &dh, float &dl, float V[4], const po_consts &C,
                                            int g, int64_t r) {
  const int32_t M = w.M;
  if (!(M >= 1 && w.psi != 0)) return false;
  pe_f3 kk, n, u, v, p;
  const bool implicit = M == 1 && C.keys1;
  bool twice;  // backscatter from a bounce-1 record (below)
  if (implicit) {
    const pe_view &W = C.view1[g];
    const int j = (int)(r / W.W), i = (int)(r - (int64_t)j * W.W);
    pe_primary_geom(W, i, j, w.key, C.nrm1, p, n, kk, u, v);
    twice = C.mono1[g] != 0;
  } else {
    kk = {h.k[3 * slot], h.k[3 * slot + 1], h.k[3 * slot + 2]};
    n = {h.n[3 * slot], h.n[3 * slot + 1], h.n[3 * slot + 2]};
    u = {h.u[3 * slot], h.u[3 * slot + 1], h.u[3 * slot + 2]};
    v = {h.v[3 * slot], h.v[3 * slot + 1], h.v[3 * slot + 2]};
    p = {h.p[3 * slot], h.p[3 * slot + 1], h.p[3 * slot + 2]};
    twice = M == 1 && ks.x == -kk.x && ks.y == -kk.y && ks.z == -kk.z;
  }
  // (the field is summed to a relative tolerance, so the per-ray factors use
  // the fast reciprocal and reciprocal square root: a few ulp each)
  float nk = dotf(n, kk);
  if (nk == 0.0f) return false;
  const float ink = __fdividef(1.0f, nk);
  float su = dotf(n, u) * ink, sv = dotf(n, v) * ink;
  pe_f3 up = {u.x - kk.x * su, u.y - kk.y * su, u.z - kk.z * su};
  pe_f3 vp = {v.x - kk.x * sv, v.y - kk.y * sv, v.z - kk.z * sv};
  pe_f3 cr = cross(up, vp);
  const float c2 = dotf(cr, cr);
  float area = c2 > 0.0f ? c2 * rsqrtf(c2) : 0.0f;
  pe_f3 q = {kk.x - ks.x, kk.y - ks.y, kk.z - ks.z};
  au = 0.5f * dotf(q, up);
  av = 0.5f * dotf(q, vp);
  const float ilu = rsqrtf(dotf(u, u)), ilv = rsqrtf(dotf(v, v));
  // [(n x h) x ks] x ks in the basis (e1, e2): for unit ks,
  // (m x ks) x ks = ks (m . ks) - m, and e1, e2 lie across ks, so its
  // coordinates are -m . e = -h . (e x n) with m = n x h (h = -v/|v| for V,
  // u/|u| for H): two cross products per ray instead of six.
  const pe_f3 g1 = cross(e1, n), g2 = cross(e2, n);
  const float sv_ = area * ilv, su_ = -area * ilu;
  V[0] = sv_ * dotf(v, g1);
  V[1] = sv_ * dotf(v, g2);
  V[2] = su_ * dotf(u, g1);
  V[3] = su_ * dotf(u, g2);
  // Backscatter from a bounce-1 record (ks = -k exactly): the path of such a
  // record is k . p by its definition, so d - ks . p = 2 k . p, taken from
  // the record's k and p as a float pair whether the record is implicit or
  // written (the two give the same bits).  Every other record: its FP64 path.
  if (twice) {
    twice_dot_pair(kk, p, dh, dl);
  } else {
    const double path = implicit ? pe_path_start(kk, p) : h.path[slot];
    const double ksp =
        (double)ks.x * (double)p.x + (double)ks.y * (double)p.y + (double)ks.z * (double)p.z;
    const double delta = path - ksp;
    dh = (float)delta;
    dl = (float)(delta - (double)dh);
  }
  return true;
}

// One (ray, frequency) term of Eq. 14 added to the float sums b: sinc x sinc,
// the phase in revolutions (k / 2 pi) (d - ks.p) as a double-float product
// (ph - rint(ph) is exact for |ph| < 2^23; er carries the low parts), one
// sincos, eight multiply-adds.
__device__ __forceinline__ void add_term(float kf, float khi, float klo, float au, float av,
                                         float dhi, float dlo, const float V[4], float b[kAcc]) {
  // the common case, both arguments small, as one branch: the product of the
  // two Taylor series of sin(x)/x in x^2 (each through x^8, truncation
  // < 2.5e-11 per factor, < 5e-11 for the product)
  const float xa = kf * au, xb = kf * av;
  float s;
  if (fmaxf(fabsf(xa), fabsf(xb)) < 0.5f) {
    const float ta = xa * xa, tb = xb * xb;
    float pa = fmaf(ta, 1.0f / 362880.0f, -1.0f / 5040.0f);
    float pb = fmaf(tb, 1.0f / 362880.0f, -1.0f / 5040.0f);
    pa = fmaf(pa, ta, 1.0f / 120.0f);
    pb = fmaf(pb, tb, 1.0f / 120.0f);
    pa = fmaf(pa, ta, -1.0f / 6.0f);
    pb = fmaf(pb, tb, -1.0f / 6.0f);
    pa = fmaf(pa, ta, 1.0f);
    pb = fmaf(pb, tb, 1.0f);
    s = pa * pb;
  } else {
    s = sincf_(xa) * sincf_(xb);
  }
  const float ph = khi * dhi;
  const float er = fmaf(khi, dhi, -ph) + fmaf(khi, dlo, klo * dhi);
  const float red = (ph - rintf(ph)) + er;
  float sn, cs;
  __sincosf(red * kTwoPi, &sn, &cs);
  const float re = s * cs, im = -s * sn;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    b[2 * i] = fmaf(V[i], re, b[2 * i]);
    b[2 * i + 1] = fmaf(V[i], im, b[2 * i + 1]);
  }
}

__global__ void __launch_bounds__(kPoThreads, 4)
    po_kernel(const pe_hits h, const __grid_constant__ po_consts C, double *__restrict__ part) {
  // per staged ray: {au, av, dh, dl}, {Va.e1, Va.e2, Vc.e1, Vc.e2}: two
  // broadcast 16-byte loads per term
  __shared__ float4 s_ray[2][kPoThreads];
  __shared__ int s_warp[kPoThreads / 32];
  __shared__ double s_red[kPoThreads][kAcc];

  const int g = blockIdx.y;  // group within this launch
  const int chunk = blockIdx.x;
  const int tid = threadIdx.x;
  const int FL = C.fl, RL = kPoThreads / FL;
  const int lane_f = tid % FL, lane_r = tid / FL;
  const pe_f3 ks = {C.ks[g][0], C.ks[g][1], C.ks[g][2]};
  const pe_f3 e1 = {C.e1[g][0], C.e1[g][1], C.e1[g][2]};
  const pe_f3 e2 = {C.e2[g][0], C.e2[g][1], C.e2[g][2]};
  const int64_t r_begin = (int64_t)chunk * C.chunk;
  int64_t r_end = r_begin + C.chunk;
  if (r_end > C.rpg) r_end = C.rpg;
  const int64_t slot0 = (int64_t)(C.g0 + g) * C.rpg;
  long long n_rays = 0;  // contributing rays (counted in the first frequency chunk)

  for (int f0 = 0; f0 < C.nf; f0 += FL) {
    const int f = f0 + lane_f;
    const bool f_ok = f < C.nf;
    const float kf = f_ok ? C.k[f] : 0.0f, khi = f_ok ? C.khi[f] : 0.0f,
                klo = f_ok ? C.klo[f] : 0.0f;
    float hi[kAcc], lo[kAcc], b[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) hi[i] = lo[i] = b[i] = 0.0f;
    int pending = 0;

    if (FL == 1) {
      // one frequency: each thread takes its own rays, nothing to share
      for (int64_t r = r_begin + tid; r < r_end; r += kPoThreads) {
        float au, av, dh, dl, V[4];
        if (!ray_factors(h, slot0 + r, load_words(h, C, slot0 + r), ks, e1, e2, au, av, dh, dl, V,
                         C, g, r))
          continue;
        n_rays += f0 == 0;
        add_term(kf, khi, klo, au, av, dh, dl, V, b);
        if (++pending == kFlush) {
#pragma unroll
          for (int i = 0; i < kAcc; ++i) {
            two_sum_into(hi[i], lo[i], b[i]);
            b[i] = 0.0f;
          }
          pending = 0;
        }
      }
    } else {
      for (int64_t sb = r_begin; sb < r_end; sb += kPoThreads) {
        // ---- stage the frequency-independent per-ray factors --------------
        const int64_t r = sb + tid;
        float au = 0, av = 0, dh = 0, dl = 0, V[4] = {0, 0, 0, 0};
        const bool valid = r < r_end && ray_factors(h, slot0 + r, load_words(h, C, slot0 + r), ks,
                                                    e1, e2, au, av, dh, dl, V, C, g, r);
        // stable compaction of the valid rays (order = slot order)
        unsigned m = __ballot_sync(0xffffffffu, valid);
        int wid = tid >> 5, lane = tid & 31;
        __syncthreads();  // previous sub-batch's readers are done
        if (lane == 0) s_warp[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kPoThreads / 32; ++w) {
          if (w < wid) before += s_warp[w];
          total += s_warp[w];
        }
        if (tid == 0 && f0 == 0) n_rays += total;
        if (valid) {
          int at = before + __popc(m & ((1u << lane) - 1u));
          s_ray[0][at] = make_float4(au, av, dh, dl);
          s_ray[1][at] = make_float4(V[0], V[1], V[2], V[3]);
        }
        __syncthreads();
        // ---- one frequency per thread over the staged rays ---------------
        // chunks of at most kFlush terms; the compensated flush is checked
        // per chunk (between flushes a float sum holds fewer than 2 kFlush
        // terms)
        if (f_ok) {
          for (int j0 = lane_r; j0 < total; j0 += kFlush * RL) {
            const int jn = min(total, j0 + kFlush * RL);
#pragma unroll 2
            for (int j = j0; j < jn; j += RL) {
              const float4 r0 = s_ray[0][j], r1 = s_ray[1][j];
              const float Vs[4] = {r1.x, r1.y, r1.z, r1.w};
              add_term(kf, khi, klo, r0.x, r0.y, r0.z, r0.w, Vs, b);
            }
            pending += ((jn - j0 - 1) >> C.rl_shift) + 1;
            if (pending >= kFlush) {
#pragma unroll
              for (int i = 0; i < kAcc; ++i) {
                two_sum_into(hi[i], lo[i], b[i]);
                b[i] = 0.0f;
              }
              pending = 0;
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kAcc; ++i) two_sum_into(hi[i], lo[i], b[i]);
    // ---- fixed-order FP64 reduction over the ray lanes -------------------
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s_red[tid][i] = (double)hi[i] + (double)lo[i];
    __syncthreads();
    if (tid < FL && f0 + tid < C.nf) {
      double acc[kAcc];
#pragma unroll
      for (int i = 0; i < kAcc; ++i) acc[i] = 0.0;
      for (int rl = 0; rl < RL; ++rl)
#pragma unroll
        for (int i = 0; i < kAcc; ++i) acc[i] += s_red[rl * FL + tid][i];
      int64_t o = (((int64_t)g * C.n_chunks + chunk) * C.nf + (f0 + tid)) * kAcc;
#pragma unroll
      for (int i = 0; i < kAcc; ++i) part[o + i] = acc[i];
    }
    __syncthreads();
  }
  count_terms(C, n_rays);
}

// ---------------------------------------------------------------------------
// Uniform frequency grids (k_f = k_0 + f dk): each thread takes kFt
// consecutive frequencies of a ray.  The phase factor of its first frequency
// is computed as above (double-float phase in revolutions, one sincos); the
// next ones follow by rotation, e^{-j k_{f+1} d} = e^{-j k_f d} e^{-j dk d},
// with the ray's rotation e^{-j dk d} staged once per ray (re-anchored at
// every thread's first frequency, so the float32 rotation drifts over at most
// kFt - 1 steps).  The two sinc factors are one power series in t = k^2:
// sinc(k a) sinc(k b) = sum_n c_n t^n, whose coefficients through t^6 are
// staged per ray.  With |k a|, |k b| <= 1 the tail n >= 7 stays below
// sum_{n>=7} 2^(2n+1) / (2n+2)! < 1.6e-9 (the sum over i + j = n of
// 1 / ((2i+1)! (2j+1)!) is 2^(2n+1) / (2n+2)!); a ray with a larger argument
// anywhere in the launch takes the direct form instead.  (Through t^4 the
// range would be |k a|, |k b| < 0.5, which leaves about half of a sphere's
// rays, those beyond 45 degrees incidence, to the direct form at a 2 mm
// pitch and 12 GHz.)  Per term: six multiply-adds of the series, four of the
// rotation, two for the complex amplitude and eight for the sums.
// ---------------------------------------------------------------------------
#ifndef PE_PO_FT
#define PE_PO_FT 2   // frequencies per thread of the rotation kernel
#endif
#ifndef PE_PO_SMC
#define PE_PO_SMC 1  // 1: the compensated sums live in shared memory, not registers
#endif
#ifndef PE_PO_MINB
#define PE_PO_MINB 3  // resident blocks per SM the rotation kernel's registers allow
#endif
#ifndef PE_PO_ROT
#define PE_PO_ROT 1  // 0: every grid takes the direct kernel
#endif
#ifndef PE_PO_JU
#define PE_PO_JU 1   // rays per unrolled step of the series pass
#endif
constexpr int kFt = PE_PO_FT;
constexpr int kJu = PE_PO_JU;

constexpr int kSer = 6;        // series coefficients beyond the constant 1
constexpr float kSerRange = 1.0f;  // largest |k a|, |k b| of a series ray

__device__ __forceinline__ void series_coeffs(float au, float av, float c[kSer]) {
  // sinc x = sum_i (-1)^i x^(2i) / (2i+1)!.  With a_i = A^i / (2i+1)!,
  // b_j = B^j / (2j+1)! (A = au^2, B = av^2; a_i = a_(i-1) A / (2i (2i+1)))
  // the product's coefficient of t^n is (-1)^n sum_{i+j=n} a_i b_j.
  const float A = au * au, B = av * av;
  float a[kSer + 1], b[kSer + 1];
  a[0] = b[0] = 1.0f;
#pragma unroll
  for (int i = 1; i <= kSer; ++i) {
    const float r = 1.0f / (float)((2 * i) * (2 * i + 1));
    a[i] = a[i - 1] * A * r;
    b[i] = b[i - 1] * B * r;
  }
#pragma unroll
  for (int n = 1; n <= kSer; ++n) {
    float x = 0.0f;
#pragma unroll
    for (int i = 0; i <= n; ++i) x = fmaf(a[i], b[n - i], x);
    c[n - 1] = (n & 1) ? -x : x;
  }
}

// One term: the complex amplitude sc e^{-j phase} (pr, pi) into the eight
// sums b (V[i] x re, im), then the phase factor rotated by the ray's step.
__device__ __forceinline__ void rot_term(float sc, float4 V, float4 r2, float &pr, float &pi,
                                         float *b) {
  const float re = sc * pr, im = sc * pi;
  b[0] = fmaf(V.x, re, b[0]);
  b[1] = fmaf(V.x, im, b[1]);
  b[2] = fmaf(V.y, re, b[2]);
  b[3] = fmaf(V.y, im, b[3]);
  b[4] = fmaf(V.z, re, b[4]);
  b[5] = fmaf(V.z, im, b[5]);
  b[6] = fmaf(V.w, re, b[6]);
  b[7] = fmaf(V.w, im, b[7]);
  const float nr = fmaf(pr, r2.z, -pi * r2.w);
  pi = fmaf(pr, r2.w, pi * r2.z);
  pr = nr;
}

// The reduced phase (revolutions in [-1/2, 1/2] plus the carried low part)
// of the float-pair product (khi + klo)(dhi + dlo), as in add_term.
__device__ __forceinline__ float rev_phase(float khi, float klo, float dhi, float dlo) {
  const float ph = khi * dhi;
  const float er = fmaf(khi, dhi, -ph) + fmaf(khi, dlo, klo * dhi);
  return (ph - rintf(ph)) + er;
}

template <int FT, bool SMC>
__global__ void __launch_bounds__(kPoThreads, PE_PO_MINB)
    po_rot_kernel(const pe_hits h, const __grid_constant__ po_consts C, double *__restrict__ part) {
  // SMC: the per-thread compensated sums (hi, lo) in dynamic shared memory,
  // [2][FT * kAcc][kPoThreads] floats, instead of registers
  extern __shared__ float s_hl[];
  // per staged ray: the series {c1..c4}, the area-weighted vector factors
  // {Va.e1, Va.e2, Vc.e1, Vc.e2}, {dh, dl, rotation re, im}, and {c5, c6}
  // for a series ray or the sinc arguments (au, av) for the direct form
  __shared__ float4 s_ray[3][kPoThreads];
  __shared__ float2 s_arg[kPoThreads];
  __shared__ int s_warp[2 * (kPoThreads / 32)];
  __shared__ double s_red[kPoThreads][kAcc];

  const int g = blockIdx.y;
  const int chunk = blockIdx.x;
  const int tid = threadIdx.x;
  const int FL = C.fl, RL = kPoThreads / FL;  // frequency-chunk lanes, ray lanes
  const int lane_f = tid % FL, lane_r = tid / FL;
  const pe_f3 ks = {C.ks[g][0], C.ks[g][1], C.ks[g][2]};
  const pe_f3 e1 = {C.e1[g][0], C.e1[g][1], C.e1[g][2]};
  const pe_f3 e2 = {C.e2[g][0], C.e2[g][1], C.e2[g][2]};
  const int64_t r_begin = (int64_t)chunk * C.chunk;
  int64_t r_end = r_begin + C.chunk;
  if (r_end > C.rpg) r_end = C.rpg;
  const int64_t slot0 = (int64_t)(C.g0 + g) * C.rpg;
  const int n_fc = (C.nf + FT - 1) / FT;  // frequency chunks of the launch
  long long n_rays = 0;  // contributing rays (counted in the first frequency chunk)

  for (int c0 = 0; c0 < n_fc; c0 += FL) {
    const int f1 = (c0 + lane_f) * FT;  // this thread's first frequency
    const bool f_ok = f1 < C.nf;
    float t2[FT], kq[FT], ik[FT];
#pragma unroll
    for (int q = 0; q < FT; ++q) {
      t2[q] = f1 + q < C.nf ? C.k2[f1 + q] : 0.0f;
      kq[q] = C.k[min(f1 + q, C.nf - 1)];
      ik[q] = __frcp_rn(kq[q]);  // (frequencies are > 0)
    }
    const float khi = f_ok ? C.khi[f1] : 0.0f, klo = f_ok ? C.klo[f1] : 0.0f;
    constexpr int NA = FT * kAcc;
    float hi[SMC ? 1 : NA], lo[SMC ? 1 : NA], b[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) b[i] = 0.0f;
    if (SMC) {
#pragma unroll
      for (int i = 0; i < NA; ++i) s_hl[i * kPoThreads + tid] = s_hl[(NA + i) * kPoThreads + tid] = 0.0f;
    } else {
#pragma unroll
      for (int i = 0; i < NA; ++i) hi[SMC ? 0 : i] = lo[SMC ? 0 : i] = 0.0f;
    }
    int pending = 0;

    for (int64_t sb = r_begin; sb < r_end; sb += kPoThreads) {
      // ---- stage the frequency-independent per-ray factors ----------------
      const int64_t r = sb + tid;
      float au = 0, av = 0, dh = 0, dl = 0, V[4] = {0, 0, 0, 0};
      const bool valid = r < r_end && ray_factors(h, slot0 + r, load_words(h, C, slot0 + r), ks,
                                                  e1, e2, au, av, dh, dl, V, C, g, r);
      // two stable compactions: rays whose sinc arguments stay in the series'
      // range for every frequency of the launch first, the others after them
      const bool ser = valid && fmaxf(fabsf(au), fabsf(av)) * C.kmax <= kSerRange;
      const unsigned ma = __ballot_sync(0xffffffffu, ser);
      const unsigned mb = __ballot_sync(0xffffffffu, valid && !ser);
      int wid = tid >> 5, lane = tid & 31;
      __syncthreads();  // previous sub-batch's readers are done
      if (lane == 0) {
        s_warp[wid] = __popc(ma);
        s_warp[kPoThreads / 32 + wid] = __popc(mb);
      }
      __syncthreads();
      int before_a = 0, n_a = 0, before_b = 0, n_b = 0;
      for (int w = 0; w < kPoThreads / 32; ++w) {
        if (w < wid) {
          before_a += s_warp[w];
          before_b += s_warp[kPoThreads / 32 + w];
        }
        n_a += s_warp[w];
        n_b += s_warp[kPoThreads / 32 + w];
      }
      if (tid == 0 && c0 == 0) n_rays += n_a + n_b;
      if (valid) {
        const unsigned below = (1u << lane) - 1u;
        const int at = ser ? before_a + __popc(ma & below) : n_a + before_b + __popc(mb & below);
        float4 r0;
        float2 r3;
        if (ser) {
          float c[kSer];
          series_coeffs(au, av, c);
          r0 = make_float4(c[0], c[1], c[2], c[3]);
          r3 = make_float2(c[4], c[5]);
        } else {
          // the direct form as sin(k A) sin(k B) / (k^2 A B) with A >= B the
          // two arguments' sizes (sinc is even) and the reciprocals staged,
          // so that a term takes no division; a B whose factor stays in the
          // one-factor series' range (|k B| < 0.5) takes that series in t
          // (through x^8, tail below 3e-11) and flags the ray by A > 0
          float A = fabsf(au), B = fabsf(av);
          if (B > A) {
            const float x = A;
            A = B;
            B = x;
          }
          if (B * C.kmax < 0.5f) {
            const float B2 = B * B, B4 = B2 * B2;
            r0 = make_float4(-B2 * (1.0f / 6.0f), B4 * (1.0f / 120.0f), -B4 * B2 * (1.0f / 5040.0f),
                             B4 * B4 * (1.0f / 362880.0f));
            r3 = make_float2(A, __frcp_rn(A));
          } else {
            r0 = make_float4(__frcp_rn(A * B), 0.0f, 0.0f, 0.0f);
            r3 = make_float2(-A, B);
          }
        }
        float rs, rc;
        __sincosf(rev_phase(C.dkhi, C.dklo, dh, dl) * kTwoPi, &rs, &rc);
        s_ray[0][at] = r0;
        s_ray[1][at] = make_float4(V[0], V[1], V[2], V[3]);
        s_ray[2][at] = make_float4(dh, dl, rc, -rs);
        s_arg[at] = r3;
      }
      __syncthreads();
      // ---- FT frequencies per thread over the staged rays ---------------
      if (f_ok) {
        for (int pass = 0; pass < 2; ++pass) {
          const int jb = pass == 0 ? 0 : n_a, je = pass == 0 ? n_a : n_a + n_b;
          for (int j0 = jb + lane_r; j0 < je; j0 += kFlush * RL) {
            const int jn = min(je, j0 + kFlush * RL);
            if (pass == 0) {
#pragma unroll kJu
              for (int j = j0; j < jn; j += RL) {
                const float4 r0 = s_ray[0][j], r1 = s_ray[1][j], r2 = s_ray[2][j];
                const float2 c56 = s_arg[j];
                float sn, cs;
                __sincosf(rev_phase(khi, klo, r2.x, r2.y) * kTwoPi, &sn, &cs);
                float pr = cs, pi = -sn;  // e^{-j phase} at frequency f1
#pragma unroll
                for (int q = 0; q < FT; ++q) {
                  const float t = t2[q];
                  const float sc = fmaf(
                      fmaf(fmaf(fmaf(fmaf(fmaf(c56.y, t, c56.x), t, r0.w), t, r0.z), t, r0.y), t,
                           r0.x),
                      t, 1.0f);
                  rot_term(sc, r1, r2, pr, pi, b + q * kAcc);
                }
              }
            } else {
              for (int j = j0; j < jn; j += RL) {
                const float4 r0 = s_ray[0][j], r1 = s_ray[1][j], r2 = s_ray[2][j];
                const float2 arg = s_arg[j];
                float sn, cs;
                __sincosf(rev_phase(khi, klo, r2.x, r2.y) * kTwoPi, &sn, &cs);
                float pr = cs, pi = -sn;
                if (arg.x > 0.0f) {  // sinc(k B) by its series (a warp shares the ray when FL = 32)
#pragma unroll
                  for (int q = 0; q < FT; ++q) {
                    const float t = t2[q];
                    const float sb = fmaf(fmaf(fmaf(fmaf(r0.w, t, r0.z), t, r0.y), t, r0.x), t, 1.0f);
                    const float sc = sb * __sinf(kq[q] * arg.x) * (arg.y * ik[q]);
                    rot_term(sc, r1, r2, pr, pi, b + q * kAcc);
                  }
                } else {
#pragma unroll
                  for (int q = 0; q < FT; ++q) {
                    const float sc =
                        __sinf(kq[q] * -arg.x) * __sinf(kq[q] * arg.y) * (r0.x * ik[q] * ik[q]);
                    rot_term(sc, r1, r2, pr, pi, b + q * kAcc);
                  }
                }
              }
            }
            pending += ((jn - j0 - 1) >> C.rl_shift) + 1;
            if (pending >= kFlush) {
#pragma unroll
              for (int i = 0; i < NA; ++i) {
                if (SMC) {
                  float x = s_hl[i * kPoThreads + tid], y = s_hl[(NA + i) * kPoThreads + tid];
                  two_sum_into(x, y, b[i]);
                  s_hl[i * kPoThreads + tid] = x;
                  s_hl[(NA + i) * kPoThreads + tid] = y;
                } else {
                  two_sum_into(hi[SMC ? 0 : i], lo[SMC ? 0 : i], b[i]);
                }
                b[i] = 0.0f;
              }
              pending = 0;
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      if (SMC) {
        float x = s_hl[i * kPoThreads + tid], y = s_hl[(NA + i) * kPoThreads + tid];
        two_sum_into(x, y, b[i]);
        s_hl[i * kPoThreads + tid] = x;
        s_hl[(NA + i) * kPoThreads + tid] = y;
      } else {
        two_sum_into(hi[SMC ? 0 : i], lo[SMC ? 0 : i], b[i]);
      }
    }
    // ---- fixed-order FP64 reduction over the ray lanes, per frequency ----
#pragma unroll
    for (int q = 0; q < FT; ++q) {
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kAcc; ++i) {
        const int a = q * kAcc + i;
        s_red[tid][i] = SMC ? (double)s_hl[a * kPoThreads + tid] +
                                  (double)s_hl[(NA + a) * kPoThreads + tid]
                            : (double)hi[SMC ? 0 : a] + (double)lo[SMC ? 0 : a];
      }
      __syncthreads();
      const int f = (c0 + tid) * FT + q;
      if (tid < FL && c0 + tid < n_fc && f < C.nf) {
        double acc[kAcc];
#pragma unroll
        for (int i = 0; i < kAcc; ++i) acc[i] = 0.0;
        for (int rl = 0; rl < RL; ++rl)
#pragma unroll
          for (int i = 0; i < kAcc; ++i) acc[i] += s_red[rl * FL + tid][i];
        int64_t o = (((int64_t)g * C.n_chunks + chunk) * C.nf + f) * kAcc;
#pragma unroll
        for (int i = 0; i < kAcc; ++i) part[o + i] = acc[i];
      }
    }
    __syncthreads();
  }
  count_terms(C, n_rays);
}

// E[g0+g][f][12] = the chunks' sums (fixed order) taken back from the basis
// (e1, e2) across ks to Cartesian components: for polarisation p, component
// x and re/im r, E = e1[x] S[p][e1][r] + e2[x] S[p][e2][r].
__global__ void po_reduce_kernel(const double *__restrict__ part, const __grid_constant__ po_consts C,
                                 int nf_total, int f_base, double *__restrict__ E) {
  const int64_t n = (int64_t)C.ng * C.nf;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(t % C.nf);
    const int g = (int)(t / C.nf);
    double S[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) S[i] = 0.0;
    for (int c = 0; c < C.n_chunks; ++c) {
      const double *q = part + (((int64_t)g * C.n_chunks + c) * C.nf + f) * kAcc;
#pragma unroll
      for (int i = 0; i < kAcc; ++i) S[i] += q[i];
    }
    double *e = E + (((int64_t)(C.g0 + g) * nf_total) + f_base + f) * 12;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int r = 0; r < 2; ++r)
          e[(p * 3 + x) * 2 + r] = __dadd_rn(__dmul_rn((double)C.e1[g][x], S[(p * 2) * 2 + r]),
                                             __dmul_rn((double)C.e2[g][x], S[(p * 2 + 1) * 2 + r]));
  }
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

// An orthonormal basis (e1, e2) of the plane across the unit vector ks, in
// FP64, rounded to float (both the kernel's projection and the reduction's
// reconstruction use these float values).  e1 is the coordinate axis least
// aligned with ks with its ks part removed; e2 = ks x e1.
void transverse_basis(const float ksf[3], float e1f[3], float e2f[3]) {
  double k[3] = {ksf[0], ksf[1], ksf[2]};
  const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  for (int i = 0; i < 3; ++i) k[i] = kn > 0 ? k[i] / kn : (i == 2 ? 1.0 : 0.0);
  int m = 0;
  for (int i = 1; i < 3; ++i)
    if (fabs(k[i]) < fabs(k[m])) m = i;
  double a[3] = {0.0, 0.0, 0.0};
  a[m] = 1.0;
  const double ak = a[0] * k[0] + a[1] * k[1] + a[2] * k[2];
  double e1[3] = {a[0] - ak * k[0], a[1] - ak * k[1], a[2] - ak * k[2]};
  const double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int i = 0; i < 3; ++i) e1[i] /= n1;
  const double e2[3] = {k[1] * e1[2] - k[2] * e1[1], k[2] * e1[0] - k[0] * e1[2],
                        k[0] * e1[1] - k[1] * e1[0]};
  for (int i = 0; i < 3; ++i) {
    e1f[i] = (float)e1[i];
    e2f[i] = (float)e2[i];
  }
}

void po_shape(int32_t ng, int64_t rpg, int32_t nf, int *fl, int *n_chunks, int64_t *chunk) {
  int f = 1;
  while (f < nf && f < 64) f <<= 1;
  *fl = f;
  int64_t max_chunks = (rpg + kPoThreads - 1) / kPoThreads;
  int64_t target = ((int64_t)sms() * 8 + ng - 1) / (ng > 0 ? ng : 1);
  if (target < 1) target = 1;
  int64_t nc = target < max_chunks ? target : max_chunks;
  if (nc < 1) nc = 1;
  int64_t ch = (rpg + nc - 1) / nc;
  ch = (ch + kPoThreads - 1) / kPoThreads * kPoThreads;
  nc = (rpg + ch - 1) / ch;
  if (nc < 1) nc = 1;
  *n_chunks = (int)nc;
  *chunk = ch;
}

}  // namespace

size_t pe_po_ws_bytes(int32_t n_groups, int64_t rpg, int32_t n_freq) {
  // the partial sums of the largest launch (any group count up to 64)
  int nf = n_freq < kPoFreqs ? n_freq : kPoFreqs;
  int gmax = n_groups < kPoGroups ? n_groups : kPoGroups;
  size_t most = 0;
  for (int ng = 1; ng <= gmax; ++ng) {
    int fl, nc;
    int64_t ch;
    po_shape(ng, rpg, nf, &fl, &nc, &ch);
    size_t b = (size_t)ng * nc * nf * kAcc;
    if (b > most) most = b;
  }
  pe_carve c{nullptr, 0};
  c.take<double>(most);
  return c.bytes();
}

pe_status pe_launch_po(const pe_hits &h, int32_t n_groups, int64_t rpg, const float *ks,
                       const double *freqs, int32_t n_freq, void *ws, size_t ws_bytes,
                       double *E, cudaStream_t s, int64_t *stats, const pe_gfb_src *gfb1) {
  if (n_groups < 1 || rpg < 1 || n_freq < 1) return PE_OK;
  if (ws_bytes < pe_po_ws_bytes(n_groups, rpg, n_freq))
    return pe_fail(PE_ENOMEM, "po: workspace too small");
  if (gfb1) {
    if (!gfb1->keys || !gfb1->nrm || !gfb1->views)
      return pe_fail(PE_EINVAL, "po: implicit bounce-1 records need keys, normals and views");
    for (int g = 0; g < n_groups; ++g)
      if ((int64_t)gfb1->views[g].W * gfb1->views[g].H != rpg)
        return pe_fail(PE_EINVAL, "po: implicit bounce-1 records need W * H rays per group");
  }
  double *part = static_cast<double *>(ws);
  const double two_pi = 2.0 * M_PI;
  const double c0 = 299792458.0;
  for (int g0 = 0; g0 < n_groups; g0 += kPoGroups) {
    int ng = n_groups - g0 < kPoGroups ? n_groups - g0 : kPoGroups;
    for (int fb = 0; fb < n_freq; fb += kPoFreqs) {
      int nf = n_freq - fb < kPoFreqs ? n_freq - fb : kPoFreqs;
      po_consts C;
      memset(&C, 0, sizeof(C));
      C.ng = ng;
      C.nf = nf;
      po_shape(ng, rpg, nf, &C.fl, &C.n_chunks, &C.chunk);
      C.rpg = rpg;
      C.g0 = g0;
      C.stats = reinterpret_cast<long long *>(stats);
      for (int g = 0; g < ng; ++g) {
        for (int k = 0; k < 3; ++k) C.ks[g][k] = ks[3 * (g0 + g) + k];
        transverse_basis(C.ks[g], C.e1[g], C.e2[g]);
      }
      if (gfb1) {
        C.keys1 = gfb1->keys;
        C.nrm1 = gfb1->nrm;
        for (int g = 0; g < ng; ++g) {
          C.view1[g] = gfb1->views[g0 + g];
          C.mono1[g] = 1;
          for (int k = 0; k < 3; ++k)
            if (!(C.ks[g][k] == -C.view1[g].d[k])) C.mono1[g] = 0;
        }
      }
      C.rl_shift = __builtin_ctz((unsigned)(kPoThreads / C.fl));
      double kmax = 0.0;
      for (int f = 0; f < nf; ++f) {
        const double kd = two_pi * freqs[fb + f] / c0;
        const double kr = freqs[fb + f] / c0;  // k / 2 pi
        C.k[f] = (float)kd;
        C.khi[f] = (float)kr;
        C.klo[f] = (float)(kr - (double)C.khi[f]);
        C.k2[f] = (float)(kd * kd);
        kmax = fmax(kmax, kd);
      }
      C.kmax = (float)(kmax * (1.0 + 1e-6));
      // a uniform grid (every frequency within 1e-9 of its place on the
      // line through the first and the last) takes the rotation kernel
      bool uniform = PE_PO_ROT && nf >= kFt;
      const double df = nf > 1 ? (freqs[fb + nf - 1] - freqs[fb]) / (double)(nf - 1) : 0.0;
      for (int f = 0; uniform && f < nf; ++f)
        uniform = fabs(freqs[fb + f] - (freqs[fb] + f * df)) <= 1e-9 * fabs(freqs[fb + f]);
      dim3 grid(C.n_chunks, ng);
      if (uniform) {
        const double dkr = df / c0;
        C.dkhi = (float)dkr;
        C.dklo = (float)(dkr - (double)C.dkhi);
        const int n_fc = (nf + kFt - 1) / kFt;
        int fl = 1;
        while (fl < n_fc && fl < 64) fl <<= 1;
        C.fl = fl;
        C.rl_shift = __builtin_ctz((unsigned)(kPoThreads / C.fl));
        const size_t smem = PE_PO_SMC ? sizeof(float) * 2 * kFt * kAcc * kPoThreads : 0;
        static bool attr = false;
        if (!attr && smem > 0) {
          PE_TRY_CUDA(cudaFuncSetAttribute(po_rot_kernel<kFt, PE_PO_SMC != 0>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          attr = true;
        }
        pe_event_before("po_kernel", s);
        po_rot_kernel<kFt, PE_PO_SMC != 0><<<grid, kPoThreads, smem, s>>>(h, C, part);
        pe_event_after("po_kernel", s);
        PE_TRY_LAUNCH("po_rot_kernel");
      } else {
        pe_event_before("po_kernel", s);
        po_kernel<<<grid, kPoThreads, 0, s>>>(h, C, part);
        pe_event_after("po_kernel", s);
        PE_TRY_LAUNCH("po_kernel");
      }
      int64_t n = (int64_t)ng * nf;
      int blocks = (int)((n + 127) / 128);
      po_reduce_kernel<<<blocks, 128, 0, s>>>(part, C, n_freq, fb, E);
      PE_TRY_LAUNCH("po_reduce_kernel");
    }
  }
  return PE_OK;
}

extern "C" size_t pe_po_workspace(int32_t n_groups, int64_t rays_per_group, int32_t n_freq) {
  if (n_groups < 1 || rays_per_group < 1 || n_freq < 1) return 0;
  return pe_po_ws_bytes(n_groups, rays_per_group, n_freq) + 256;
}

extern "C" pe_status pe_po_field(const pe_hits *hits, int32_t n_groups, int64_t rays_per_group,
                                 const float *ks, const double *freqs, int32_t n_freq, void *ws,
                                 size_t ws_bytes, double *E, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!hits || !ks || !freqs || !E || n_groups < 1 || rays_per_group < 1 || n_freq < 1)
    return pe_fail(PE_EINVAL, "pe_po_field: bad arguments");
  if (hits->n_rays < (int64_t)n_groups * rays_per_group || !hits->p || !hits->n || !hits->k ||
      !hits->u || !hits->v || !hits->path || !hits->M || !hits->psi)
    return pe_fail(PE_EINVAL, "pe_po_field: hits must hold n_groups * rays_per_group records");
  for (int f = 0; f < n_freq; ++f)
    if (!(freqs[f] > 0)) return pe_fail(PE_EINVAL, "pe_po_field: frequencies must be > 0");
  size_t need = pe_po_workspace(n_groups, rays_per_group, n_freq);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_po_field: workspace needs %zu bytes", need);
  return pe_launch_po(*hits, n_groups, rays_per_group, ks, freqs, n_freq, ws, ws_bytes, E, s);
}

// ---------------------------------------------------------------------------
// Bistatic observation: the Eq. 14 sum toward n_obs receiver directions per
// group, each with Psi tested toward its own receiver.
// ---------------------------------------------------------------------------

namespace {
struct bistatic_ws {
  uint8_t *psi;
  double *Eo;
  char *po;
  size_t po_bytes;
};

bistatic_ws carve_bistatic(pe_carve &c, int32_t n_groups, int64_t rpg, int32_t n_freq) {
  bistatic_ws w;
  w.psi = c.take<uint8_t>((size_t)(n_groups * rpg));
  w.Eo = c.take<double>((size_t)n_groups * n_freq * 12);
  w.po_bytes = pe_po_ws_bytes(n_groups, rpg, n_freq);
  w.po = c.take<char>(w.po_bytes);
  return w;
}
}  // namespace

extern "C" size_t pe_po_field_bistatic_workspace(int32_t n_groups, int64_t rays_per_group,
                                                 int32_t n_freq) {
  if (n_groups < 1 || rays_per_group < 1 || n_freq < 1) return 0;
  pe_carve c{nullptr, 0};
  carve_bistatic(c, n_groups, rays_per_group, n_freq);
  return c.bytes() + 256;
}

extern "C" pe_status pe_po_field_bistatic(const pe_hits *hits, int32_t n_groups,
                                          int64_t rays_per_group, const float *obs_dirs,
                                          int32_t n_obs, const pe_geom *geom, float eps,
                                          int32_t only_bounce, const double *freqs,
                                          int32_t n_freq, void *ws, size_t ws_bytes, double *E,
                                          void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!hits || !obs_dirs || !freqs || !E || !geom || n_groups < 1 || n_groups > PE_MAX_BATCH ||
      rays_per_group < 1 || n_obs < 1 || n_freq < 1 || !(eps >= 0.0f))
    return pe_fail(PE_EINVAL, "pe_po_field_bistatic: bad arguments (1..%d groups)", PE_MAX_BATCH);
  if (hits->n_rays < (int64_t)n_groups * rays_per_group || !hits->p || !hits->n || !hits->k ||
      !hits->u || !hits->v || !hits->path || !hits->M)
    return pe_fail(PE_EINVAL, "pe_po_field_bistatic: hits must hold n_groups * rays_per_group records");
  for (int f = 0; f < n_freq; ++f)
    if (!(freqs[f] > 0)) return pe_fail(PE_EINVAL, "pe_po_field_bistatic: frequencies must be > 0");
  const size_t need = pe_po_field_bistatic_workspace(n_groups, rays_per_group, n_freq);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_po_field_bistatic: workspace needs %zu bytes", need);
  pe_carve c{static_cast<char *>(ws), 0};
  bistatic_ws w = carve_bistatic(c, n_groups, rays_per_group, n_freq);
  float dirs[PE_MAX_BATCH * 3];
  const size_t row = sizeof(double) * 12 * n_freq;
  for (int o = 0; o < n_obs; ++o) {
    for (int g = 0; g < n_groups; ++g)
      for (int k = 0; k < 3; ++k) dirs[3 * g + k] = obs_dirs[((int64_t)g * n_obs + o) * 3 + k];
    pe_status st = pe_launch_shadow_dirs(geom, *hits, n_groups, rays_per_group, dirs, eps,
                                         only_bounce, w.psi, nullptr, s);
    if (st != PE_OK) return st;
    pe_hits h = *hits;
    h.psi = w.psi;
    st = pe_launch_po(h, n_groups, rays_per_group, dirs, freqs, n_freq, w.po, w.po_bytes, w.Eo, s);
    if (st != PE_OK) return st;
    // E[g][o][f][12] <- Eo[g][f][12]
    PE_TRY_CUDA(cudaMemcpy2DAsync(E + (int64_t)o * n_freq * 12, row * n_obs, w.Eo, row, row,
                                  (size_t)n_groups, cudaMemcpyDeviceToDevice, s));
  }
  return PE_OK;
}

// ---------------------------------------------------------------------------
// PO at every bounce: Eq. 14 applied at each hit of a ray instead of its last
// one.  For b = 1..max_bounces the rays are traced to b bounces; those whose
// b-th hit is their last (M == b) contribute Eq. 14 at that hit, with Psi
// tested toward the monostatic receiver; the b fields are summed in b order.
// ---------------------------------------------------------------------------

namespace {
struct every_ws {
  pe_hits h;
  uint8_t *psi;
  double *Eb;
  char *po;
  size_t po_bytes;
};

every_ws carve_every(pe_carve &c, int32_t n_views, int64_t per, int32_t n_freq) {
  every_ws w;
  memset(&w, 0, sizeof(w));
  const int64_t n = per * n_views;
  w.h.p = c.take<float>((size_t)n * 3);
  w.h.n = c.take<float>((size_t)n * 3);
  w.h.k = c.take<float>((size_t)n * 3);
  w.h.u = c.take<float>((size_t)n * 3);
  w.h.v = c.take<float>((size_t)n * 3);
  w.h.path = c.take<double>((size_t)n);
  w.h.M = c.take<int32_t>((size_t)n);
  w.h.psi = c.take<uint8_t>((size_t)n);
  w.h.ids = nullptr;
  w.h.n_rays = n;
  w.psi = c.take<uint8_t>((size_t)n);
  w.Eb = c.take<double>((size_t)n_views * n_freq * 12);
  w.po_bytes = pe_po_ws_bytes(n_views, per, n_freq);
  w.po = c.take<char>(w.po_bytes);
  return w;
}

// E[i] += Eb[i] (one FP64 addition per element, in bounce order).
__global__ void field_add_kernel(double *__restrict__ E, const double *__restrict__ Eb, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    E[i] = __dadd_rn(E[i], Eb[i]);
}
}  // namespace

extern "C" size_t pe_po_field_every_bounce_workspace(int32_t n_views, const pe_view *views,
                                                     int32_t n_freq) {
  if (n_views < 1 || n_views > PE_MAX_BATCH || !views || n_freq < 1) return 0;
  pe_carve c{nullptr, 0};
  carve_every(c, n_views, (int64_t)views[0].W * views[0].H, n_freq);
  return c.bytes() + 256;
}

extern "C" pe_status pe_po_field_every_bounce(const pe_view *views, int32_t n_views,
                                              const uint64_t *keys, const float *nrm,
                                              const pe_geom *geom, int32_t max_bounces,
                                              const pe_params *prm, const double *freqs,
                                              int32_t n_freq, void *ws, size_t ws_bytes,
                                              double *E, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!views || n_views < 1 || n_views > PE_MAX_BATCH || !prm || !geom || !freqs || !E ||
      n_freq < 1 || max_bounces < 1 || max_bounces > 64 || !(prm->eps >= 0.0f))
    return pe_fail(PE_EINVAL, "pe_po_field_every_bounce: bad arguments");
  for (int i = 1; i < n_views; ++i)
    if (views[i].W != views[0].W || views[i].H != views[0].H)
      return pe_fail(PE_EINVAL, "pe_po_field_every_bounce: all screens must share W x H");
  const int64_t per = (int64_t)views[0].W * views[0].H;
  if (per < 1 || per * n_views >= (int64_t)PE_NONE)
    return pe_fail(PE_EINVAL, "pe_po_field_every_bounce: screen size");
  if (!prm->first_bounce_from_geom && (!keys || !nrm))
    return pe_fail(PE_EINVAL, "pe_po_field_every_bounce: bounce 1 from the GFB needs keys and nrm");
  for (int f = 0; f < n_freq; ++f)
    if (!(freqs[f] > 0))
      return pe_fail(PE_EINVAL, "pe_po_field_every_bounce: frequencies must be > 0");
  const size_t need = pe_po_field_every_bounce_workspace(n_views, views, n_freq);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_po_field_every_bounce: workspace needs %zu bytes", need);
  pe_carve c{static_cast<char *>(ws), 0};
  every_ws w = carve_every(c, n_views, per, n_freq);
  pe_view_batch vb;
  memset(&vb, 0, sizeof(vb));
  vb.n = n_views;
  vb.W = views[0].W;
  vb.H = views[0].H;
  float dirs[PE_MAX_BATCH * 3];
  for (int i = 0; i < n_views; ++i) {
    vb.v[i] = views[i];
    for (int k = 0; k < 3; ++k) dirs[3 * i + k] = -views[i].d[k];
  }
  const int64_t nE = (int64_t)n_views * n_freq * 12;
  for (int b = 1; b <= max_bounces; ++b) {
    pe_hits h = w.h;
    h.max_bounces = b;
    pe_status st = pe_launch_trace(vb, reinterpret_cast<const unsigned long long *>(keys), nrm,
                                   geom, b, *prm, h, nullptr, s);
    if (st != PE_OK) return st;
    st = pe_launch_shadow_dirs(geom, h, n_views, per, dirs, prm->eps, b, w.psi, nullptr, s);
    if (st != PE_OK) return st;
    h.psi = w.psi;
    st = pe_launch_po(h, n_views, per, dirs, freqs, n_freq, w.po, w.po_bytes, b == 1 ? E : w.Eb,
                      s);
    if (st != PE_OK) return st;
    if (b > 1) {
      field_add_kernel<<<(int)((nE + 255) / 256), 256, 0, s>>>(E, w.Eb, nE);
      PE_TRY_LAUNCH("field_add_kernel");
    }
  }
  return PE_OK;
}
