// Status, error reporting, view set-up (a1) and the aggregated-geometry
// layout shared by the aggregation and tracing entry points.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pe_internal.cuh"

static thread_local char g_last_error[512] = "";

pe_status pe_fail(pe_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return s;
}

// One error word per device; kernels OR condition bits into it.
static __device__ unsigned int g_pe_err_word;

unsigned int *pe_err_word() {
  static std::mutex mu;
  static unsigned int *addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pe_err_word) != cudaSuccess) return nullptr;
    addr[dev] = static_cast<unsigned int *>(p);
  }
  return addr[dev];
}

extern "C" int pe_abi_version(void) { return PE_ABI_VERSION; }

static std::atomic<long long> g_launches{0};
void pe_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" int64_t pe_kernel_launches(void) { return (int64_t)g_launches.load(); }

extern "C" const char *pe_last_error(void) { return g_last_error; }

// Diagnostic event recording (calling host thread only).
namespace {
thread_local char t_ev_kernel[64] = "";
thread_local void **t_ev = nullptr;
thread_local int32_t t_ev_pairs = 0, t_ev_done = 0;
}  // namespace

extern "C" int32_t pe_set_kernel_events(const char *kernel, void **events, int32_t n_pairs) {
  int32_t done = t_ev_done;
  t_ev_done = 0;
  if (!kernel || !events || n_pairs <= 0) {
    t_ev = nullptr;
    t_ev_pairs = 0;
    t_ev_kernel[0] = 0;
    return done;
  }
  snprintf(t_ev_kernel, sizeof(t_ev_kernel), "%s", kernel);
  t_ev = events;
  t_ev_pairs = n_pairs;
  return done;
}

void pe_event_before(const char *kernel, cudaStream_t s) {
  if (t_ev && t_ev_done < t_ev_pairs && strcmp(kernel, t_ev_kernel) == 0)
    cudaEventRecord(static_cast<cudaEvent_t>(t_ev[2 * t_ev_done]), s);
}

void pe_event_after(const char *kernel, cudaStream_t s) {
  if (t_ev && t_ev_done < t_ev_pairs && strcmp(kernel, t_ev_kernel) == 0) {
    cudaEventRecord(static_cast<cudaEvent_t>(t_ev[2 * t_ev_done + 1]), s);
    ++t_ev_done;
  }
}

extern "C" pe_status pe_stream_check(void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PE_TRY_CUDA(cudaStreamSynchronize(s));
  unsigned int *w = pe_err_word();
  if (!w) return pe_fail(PE_ECUDA, "error word unavailable");
  unsigned int h = 0;
  PE_TRY_CUDA(cudaMemcpyAsync(&h, w, sizeof(h), cudaMemcpyDeviceToHost, s));
  PE_TRY_CUDA(cudaMemsetAsync(w, 0, sizeof(h), s));
  PE_TRY_CUDA(cudaStreamSynchronize(s));
  if (h & PE_ERR_TIMEOUT) return pe_fail(PE_ETIMEOUT, "a bounded device wait gave up");
  if (h & PE_ERR_OVERFLOW)
    return pe_fail(PE_EOVERFLOW, "a fixed-capacity device list overflowed");
  return PE_OK;
}

// a1: monostatic incidence view, FP64 on the host, rounded once to float32.
extern "C" pe_status pe_view_from_angles(double theta_deg, double phi_deg,
                                         const double centre[3], double extent,
                                         int32_t W, int32_t H, pe_view *out) {
  if (!centre || !out || W <= 0 || H <= 0 || !(extent > 0))
    return pe_fail(PE_EINVAL, "pe_view_from_angles: bad arguments");
  const double rad = M_PI / 180.0;
  double th = theta_deg * rad, ph = phi_deg * rad;
  double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
  double w[3] = {st * cp, st * sp, ct};
  double u[3] = {ct * cp, ct * sp, -st};
  double v[3] = {-sp, cp, 0.0};
  double L = (2.0 * extent) / (double)W;
  double D = extent + L;
  for (int k = 0; k < 3; ++k) {
    out->o[k] = (float)(centre[k] + D * w[k]);
    out->u[k] = (float)u[k];
    out->v[k] = (float)v[k];
    out->d[k] = (float)(-w[k]);
  }
  out->pitch = (float)L;
  out->W = W;
  out->H = H;
  return PE_OK;
}

// ---------------------------------------------------------------------------
// Geometry layout
// ---------------------------------------------------------------------------
bool pe_make_layout(int32_t nv, const pe_view *views, pe_geom_layout *L) {
  if (nv < 1 || nv > PE_MAX_VIEWS || !views) return false;
  memset(L, 0, sizeof(*L));
  L->nv = nv;
  int64_t off = 0, nodes = 0;
  for (int v = 0; v < nv; ++v) {
    const pe_view &V = views[v];
    if (V.W <= 0 || V.H <= 0 || !(V.pitch > 0)) return false;
    L->view[v] = V;
    L->pix_off[v] = off;
    off += (int64_t)V.W * V.H;
    int tw = (V.W + PE_LEAF - 1) / PE_LEAF, th = (V.H + PE_LEAF - 1) / PE_LEAF;
    int l = 0;
    for (;;) {
      if (l >= PE_MAX_LEVELS) return false;
      L->tw[v][l] = tw;
      L->th[v][l] = th;
      L->node_off[v][l] = nodes;
      nodes += (int64_t)tw * th;
      if (tw == 1 && th == 1) break;
      tw = (tw + PE_FAN - 1) / PE_FAN;
      th = (th + PE_FAN - 1) / PE_FAN;
      ++l;
    }
    L->nlev[v] = l + 1;
    // Absolute padding of the boxes: covers the float32 rounding of the
    // frame transforms of splats and rays (coordinates up to |o| + 2 W pitch).
    double o_abs = fabs((double)V.o[0]) + fabs((double)V.o[1]) + fabs((double)V.o[2]);
    double span = 2.0 * (double)V.pitch * (double)(V.W > V.H ? V.W : V.H);
    L->pad[v] = (float)(1e-5 * (o_abs + span));
  }
  L->pix_off[nv] = off;
  L->n_nodes = nodes;
  return true;
}

void pe_layout_offsets(const pe_geom_layout &L, size_t *off_cr, size_t *off_nf,
                       size_t *off_nodes, size_t *off_vmask, size_t *off_slab,
                       size_t *off_slab_hi, size_t *off_cslab, size_t *total) {
  pe_carve c{nullptr, 0};
  int64_t np = L.pix_off[L.nv];
  c.take<float4>((size_t)np);
  *off_cr = 0;
  size_t a = c.bytes();
  c.take<float4>((size_t)np);
  *off_nf = a;
  size_t b = c.bytes();
  c.take<float4>((size_t)L.n_nodes * 2);
  *off_nodes = b;
  size_t d = c.bytes();
  c.take<uint32_t>((size_t)PE_VGRID * PE_VGRID * PE_VGRID + 1);
  *off_vmask = d;
  size_t e = c.bytes();
  c.take<float4>((size_t)L.n_nodes);
  *off_slab = e;
  size_t f = c.bytes();
  c.take<float>((size_t)L.n_nodes);
  *off_slab_hi = f;
  size_t g = c.bytes();
  c.take<float4>((size_t)PE_VGRID * PE_VGRID * PE_VGRID);
  *off_cslab = g;
  *total = c.bytes();
}

extern "C" size_t pe_geom_bytes(int32_t n_views, const pe_view *views) {
  pe_geom_layout L;
  if (!pe_make_layout(n_views, views, &L)) return 0;
  size_t a, b, c, d, e, f, g, t;
  pe_layout_offsets(L, &a, &b, &c, &d, &e, &f, &g, &t);
  return t;
}
