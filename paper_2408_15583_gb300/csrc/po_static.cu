// pe_po_field_static: the PO field sum with its scratch in a fixed device
// array instead of a caller workspace.
//
// Why it exists: some callers cannot hand the library a freshly allocated
// workspace -- for example a host application whose device memory is owned by
// its own pool and that forbids allocations from plug-ins, a latency-critical
// loop that must not call cudaMalloc (it can synchronise the device), or a
// wrapper that has no way to size and keep a buffer alive between calls.  This
// entry point needs only the inputs and the output: the block partial sums of
// the field live in g_po_scratch below, a file-scope device array that every
// GPU loading the library holds until the process exits.
#include <mutex>

#include "pe_internal.cuh"

// Capacity of the scratch, in doubles (16 MiB).  A call needs
// n_groups * n_chunks * min(n_freq, 256) * 12 doubles of partial sums, where
// n_chunks depends on the rays per group (at most about 1216 / n_groups chunks
// per group); requests above the capacity are rejected.
#define PE_PO_STATIC_DOUBLES (2u * 1024u * 1024u)

static __device__ __align__(256) double g_po_scratch[PE_PO_STATIC_DOUBLES];

// Device address of g_po_scratch for the current device, looked up once per
// device (the host-side name of the array is not a device address) and kept
// for the life of the process; a cudaDeviceReset() destroys the context the
// address belongs to, so the header rules out calls after a reset.
static double *po_scratch_address() {
  static std::mutex mu;
  static double *addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_po_scratch);
    if (e != cudaSuccess) {
      pe_fail(PE_ECUDA, "pe_po_field_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return nullptr;
    }
    addr[dev] = static_cast<double *>(p);
  }
  return addr[dev];
}

extern "C" pe_status pe_po_field_static(const pe_hits *hits, int32_t n_groups,
                                        int64_t rays_per_group, const float *ks,
                                        const double *freqs, int32_t n_freq, double *E,
                                        void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!hits || !ks || !freqs || !E || n_groups < 1 || rays_per_group < 1 || n_freq < 1)
    return pe_fail(PE_EINVAL, "pe_po_field_static: bad arguments");
  if (hits->n_rays < (int64_t)n_groups * rays_per_group || !hits->p || !hits->n || !hits->k ||
      !hits->u || !hits->v || !hits->path || !hits->M || !hits->psi)
    return pe_fail(PE_EINVAL,
                   "pe_po_field_static: hits must hold n_groups * rays_per_group records");
  for (int f = 0; f < n_freq; ++f)
    if (!(freqs[f] > 0)) return pe_fail(PE_EINVAL, "pe_po_field_static: frequencies must be > 0");
  const size_t need = pe_po_ws_bytes(n_groups, rays_per_group, n_freq);
  const size_t cap = sizeof(double) * (size_t)PE_PO_STATIC_DOUBLES;
  if (need > cap)
    return pe_fail(PE_EINVAL,
                   "pe_po_field_static: request needs %zu bytes of scratch, above the fixed "
                   "%zu; use pe_po_field with a workspace or fewer groups/frequencies",
                   need, cap);
  double *scratch = po_scratch_address();
  if (!scratch) return PE_ECUDA;
  // Nothing in the scratch has to start at zero: every partial sum the reduce
  // reads is written by the field kernel of the same call.
  return pe_launch_po(*hits, n_groups, rays_per_group, ks, freqs, n_freq, scratch, cap, E, s);
}
