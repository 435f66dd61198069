// a1/a7: monostatic RCS sweep -- the whole path per batch of angles:
// incidence screens (a1) -> splat the points (a2, bounce 1) -> bounces 2..mb
// and Psi through the aggregated splats (a5) -> PO field (a6) -> sigma.
#include <cstring>

#include "pe_internal.cuh"

namespace {

// sigma[a][f][tx][rx] = k^2/pi |e_rx . Sigma_tx|^2, e_V = u (theta_hat),
// e_H = v (phi_hat) of the angle's screen.
__global__ void sigma_kernel(const __grid_constant__ pe_view_batch vb, const double *__restrict__ E,
                             const double *__restrict__ kw, int nf, int a0,
                             double *__restrict__ sigma) {
  int n = vb.n * nf;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int a = t / nf, f = t % nf;
    const pe_view &V = vb.v[a];
    const double *e = E + ((int64_t)(a0 + a) * nf + f) * 12;
    double k = kw[f];
    double c = k * k / M_PI;
    for (int tx = 0; tx < 2; ++tx)
      for (int rx = 0; rx < 2; ++rx) {
        const float *er = rx == 0 ? V.u : V.v;
        double re = 0, im = 0;
        for (int q = 0; q < 3; ++q) {
          re += (double)er[q] * e[(tx * 3 + q) * 2];
          im += (double)er[q] * e[(tx * 3 + q) * 2 + 1];
        }
        sigma[(((int64_t)(a0 + a) * nf + f) * 2 + tx) * 2 + rx] = c * (re * re + im * im);
      }
  }
}

// The buffers of one batch of angles: incidence keys and tile depths, ray
// records, PO partial sums.
struct batch_ws {
  unsigned long long *keys;
  float *hz;
  pe_hits h;
  void *po;
  size_t po_bytes;
};

// With more than one batch and a field sum of some size (at least
// kLaneFreqs frequencies) the sweep keeps two sets of batch buffers
// ("lanes"): the PO sum of one batch runs on a second stream while the next
// batch splats and traces on the caller's, so the ALU-bound field sum and the
// latency-bound march share the SMs (sphere workload, 64 frequencies: 80.0
// -> 74.9 ms per step).  With few frequencies the sum is short and the
// smaller batches of two lanes cost more than the overlap gains.
constexpr int kLaneFreqs = 8;
struct sweep_ws {
  batch_ws lane[2];
  int n_lanes;
  double *kw;
};

// Ray-record bytes per angle of a batch.
int64_t record_bytes(const pe_sweep *sw) {
  return (int64_t)sw->W * sw->H * (8 + 60 + 8 + 4 + 1 + 8) + 4096;
}

// Angles per batch: the caller's, else as many as fit ray records of about
// 16 GB (a few percent of the device's memory; more angles per launch
// amortise each pass's tail: the composite sweep at 2048^2 rays runs 168 ms
// with 5 angles per batch, 144 ms with 39), split over two lanes when the
// sweep takes more than one batch and its field sum is of some size.
int batch_of(const pe_sweep *sw) {
  if (sw->angle_batch > 0) return sw->angle_batch < PE_MAX_BATCH ? sw->angle_batch : PE_MAX_BATCH;
  const int64_t bytes = record_bytes(sw);
  int64_t b = ((int64_t)16 << 30) / bytes;
  if (b < 1) b = 1;
  if (b > PE_MAX_BATCH) b = PE_MAX_BATCH;
  if (b >= sw->n_angles) return sw->n_angles;
  if (sw->n_freq < kLaneFreqs) return (int)b;
  b = ((int64_t)8 << 30) / bytes;  // two lanes
  if (b < 1) b = 1;
  if (b > PE_MAX_BATCH) b = PE_MAX_BATCH;
  return (int)b;
}

int lanes_of(const pe_sweep *sw, int B) {
  return sw->n_angles > B && sw->n_freq >= kLaneFreqs ? 2 : 1;
}

sweep_ws carve_sweep(pe_carve &c, const pe_sweep *sw, int B) {
  sweep_ws w;
  memset(&w, 0, sizeof(w));
  w.n_lanes = lanes_of(sw, B);
  int64_t n = (int64_t)sw->W * sw->H * B;
  for (int l = 0; l < w.n_lanes; ++l) {
    batch_ws &b = w.lane[l];
    b.keys = c.take<unsigned long long>((size_t)n);
    b.hz = c.take<float>(pe_splat_tiles(B, sw->W, sw->H));
    b.h.p = c.take<float>((size_t)n * 3);
    b.h.n = c.take<float>((size_t)n * 3);
    b.h.k = c.take<float>((size_t)n * 3);
    b.h.u = c.take<float>((size_t)n * 3);
    b.h.v = c.take<float>((size_t)n * 3);
    b.h.path = c.take<double>((size_t)n);
    b.h.M = c.take<int32_t>((size_t)n);
    b.h.psi = c.take<uint8_t>((size_t)n);
    b.h.ids = nullptr;
    b.h.n_rays = n;
    b.h.max_bounces = sw->max_bounces;
    b.po_bytes = pe_po_ws_bytes(B, (int64_t)sw->W * sw->H, sw->n_freq);
    b.po = c.take<char>(b.po_bytes);
  }
  w.kw = c.take<double>((size_t)sw->n_freq);
  return w;
}

// The second stream and its events, released when the call returns (the
// runtime frees them once the work queued on them has completed).
struct lane_sync {
  cudaStream_t s2 = nullptr;
  cudaEvent_t traced = nullptr, done[2] = {nullptr, nullptr};
  ~lane_sync() {
    if (traced) cudaEventDestroy(traced);
    for (int l = 0; l < 2; ++l)
      if (done[l]) cudaEventDestroy(done[l]);
    if (s2) cudaStreamDestroy(s2);
  }
};

bool sweep_ok(const pe_sweep *sw) {
  return sw && sw->n_angles >= 1 && sw->theta_deg && sw->phi_deg && sw->W > 0 && sw->H > 0 &&
         (int64_t)sw->W * sw->H * PE_MAX_BATCH < (int64_t)PE_NONE && sw->extent > 0 &&
         sw->n_freq >= 1 && sw->freqs_hz && sw->max_bounces >= 1 && sw->max_bounces <= 64;
}

}  // namespace

extern "C" size_t pe_rcs_sweep_workspace(const pe_sweep *sw) {
  if (!sweep_ok(sw)) return 0;
  pe_carve c{nullptr, 0};
  carve_sweep(c, sw, batch_of(sw));
  return c.bytes() + 256;
}

extern "C" pe_status pe_rcs_sweep(const pe_sweep *sw, const float *pos, const float *nrm,
                                  const float *rad, int64_t n_points, const pe_geom *geom,
                                  const pe_params *prm, void *ws, size_t ws_bytes, double *E,
                                  double *sigma, int64_t *stats, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!sweep_ok(sw) || !prm || !E) return pe_fail(PE_EINVAL, "pe_rcs_sweep: bad sweep");
  if (n_points < 0 || n_points >= (int64_t)PE_NONE || (n_points > 0 && (!pos || !nrm || !rad)))
    return pe_fail(PE_EINVAL, "pe_rcs_sweep: points");
  for (int f = 0; f < sw->n_freq; ++f)
    if (!(sw->freqs_hz[f] > 0)) return pe_fail(PE_EINVAL, "pe_rcs_sweep: frequencies must be > 0");
  if (sw->max_bounces > 1 && !geom)
    return pe_fail(PE_EINVAL, "pe_rcs_sweep: max_bounces > 1 needs the aggregated geometry");
  size_t need = pe_rcs_sweep_workspace(sw);
  if (!ws || ws_bytes < need || !pe_aligned(ws, 256))
    return pe_fail(PE_ENOMEM, "pe_rcs_sweep: workspace needs %zu bytes", need);
  const int B = batch_of(sw);
  pe_carve c{static_cast<char *>(ws), 0};
  sweep_ws w = carve_sweep(c, sw, B);
  const int64_t per = (int64_t)sw->W * sw->H;

  double kw_h[4096];
  const double two_pi = 2.0 * M_PI;
  for (int f0 = 0; f0 < sw->n_freq; f0 += 4096) {
    int nf = sw->n_freq - f0 < 4096 ? sw->n_freq - f0 : 4096;
    for (int f = 0; f < nf; ++f) kw_h[f] = two_pi * sw->freqs_hz[f0 + f] / 299792458.0;
    // pageable source: the call returns once kw_h has been staged
    PE_TRY_CUDA(cudaMemcpyAsync(w.kw + f0, kw_h, sizeof(double) * nf, cudaMemcpyHostToDevice, s));
  }

  lane_sync ls;
  if (w.n_lanes == 2) {
    PE_TRY_CUDA(cudaStreamCreateWithFlags(&ls.s2, cudaStreamNonBlocking));
    PE_TRY_CUDA(cudaEventCreateWithFlags(&ls.traced, cudaEventDisableTiming));
    for (int l = 0; l < 2; ++l)
      PE_TRY_CUDA(cudaEventCreateWithFlags(&ls.done[l], cudaEventDisableTiming));
  }
  bool used[2] = {false, false};
  for (int a0 = 0, bi = 0; a0 < sw->n_angles; a0 += B, ++bi) {
    int nb = sw->n_angles - a0 < B ? sw->n_angles - a0 : B;
    const int L = bi % w.n_lanes;
    batch_ws &W = w.lane[L];
    pe_view_batch vb;
    memset(&vb, 0, sizeof(vb));
    vb.n = nb;
    vb.W = sw->W;
    vb.H = sw->H;
    float ks[PE_MAX_BATCH * 3];
    for (int a = 0; a < nb; ++a) {
      pe_status st = pe_view_from_angles(sw->theta_deg[a0 + a], sw->phi_deg[a0 + a], sw->centre,
                                         sw->extent, sw->W, sw->H, &vb.v[a]);
      if (st != PE_OK) return st;
      for (int k = 0; k < 3; ++k) ks[3 * a + k] = -vb.v[a].d[k];
    }
    // the lane's buffers are free once its previous batch's field is summed
    if (used[L]) PE_TRY_CUDA(cudaStreamWaitEvent(s, ls.done[L], 0));
    pe_hits h = W.h;
    h.n_rays = per * nb;
    if (!prm->first_bounce_from_geom) {
      PE_TRY_CUDA(cudaMemsetAsync(W.keys, 0xff, sizeof(unsigned long long) * per * nb, s));
      pe_status st = pe_launch_splat(vb, pos, nrm, rad, n_points, 0, 0.0f, W.hz, W.keys, stats, s,
                                     sw->point_order);
      if (st != PE_OK) return st;
    }
    // bounce-1 records stay implicit in the incidence GFB (bounce 1 from the
    // keys and a march to follow): the bounce-2 pass and the PO sum take them
    // from the keys, and only later hits are written as records
    const bool implicit1 = !prm->first_bounce_from_geom && sw->max_bounces >= 2;
    pe_status st =
        pe_launch_trace(vb, W.keys, nrm, geom, sw->max_bounces, *prm, h, stats, s, implicit1);
    if (st != PE_OK) return st;
    // PO: E rows [a0, a0 + nb), on the second stream when there is one
    cudaStream_t sp = s;
    if (w.n_lanes == 2) {
      PE_TRY_CUDA(cudaEventRecord(ls.traced, s));
      PE_TRY_CUDA(cudaStreamWaitEvent(ls.s2, ls.traced, 0));
      sp = ls.s2;
    }
    const pe_gfb_src src{W.keys, nrm, vb.v};
    st = pe_launch_po(h, nb, per, ks, sw->freqs_hz, sw->n_freq, W.po, W.po_bytes,
                      E + (int64_t)a0 * sw->n_freq * 12, sp, stats, implicit1 ? &src : nullptr);
    if (st != PE_OK) return st;
    if (sigma) {
      int n = nb * sw->n_freq;
      sigma_kernel<<<(n + 127) / 128, 128, 0, sp>>>(vb, E, w.kw, sw->n_freq, a0, sigma);
      PE_TRY_LAUNCH("sigma_kernel");
    }
    if (w.n_lanes == 2) {
      PE_TRY_CUDA(cudaEventRecord(ls.done[L], ls.s2));
      used[L] = true;
    }
  }
  // the caller's stream continues once every field sum has finished
  for (int l = 0; l < 2; ++l)
    if (used[l]) PE_TRY_CUDA(cudaStreamWaitEvent(s, ls.done[l], 0));
  return PE_OK;
}
