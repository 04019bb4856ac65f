// K_hat = M_hat^dag M_hat in FP64 without any device allocation.
//
// For callers that cannot allocate device memory themselves: code whose
// device memory is owned by a host application's own pool manager, code
// that cannot afford the implicit device-wide synchronisation of cudaMalloc
// in a latency-critical loop, or code that must not fail on allocation under
// memory pressure.  Such a caller passes its own gauge field, input and
// output; the two intermediate half spinors K_hat needs live in one
// file-scope device array of fixed size instead of a context's workspace.
//
// Limits and sharing rules:
//   - the lattice may have at most NOALLOC_MAX_VH = 32768 sites per parity
//     (e.g. 16^4); larger lattices are rejected with WD_ERR_ARG before any
//     launch.  The array (2 x 12 x 32768 complex doubles = 12.6 MB) is held
//     on every device that loads the library until the process exits;
//   - every call shares the array, which keeps the contents of the last call;
//     both intermediate vectors are fully written before they are read, so
//     nothing needs clearing; calls that overlap on the GPU (different
//     streams, or other threads) race on the array and must be serialised by
//     the caller;
//   - on its first call on a device the entry point looks up the array's
//     device address (cudaGetSymbolAddress) with that device current; make
//     that first call before any stream capture.  The address is kept per
//     device index for the life of the process, so it belongs to the device's
//     primary context: after cudaDeviceReset, or under a driver-API context
//     other than the primary one, it no longer names the array and the entry
//     point must not be used.
#include <mutex>

#include "dslash_impl.cuh"

namespace wd {
namespace {

constexpr long NOALLOC_MAX_VH = 32768;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[2 * 12 * NOALLOC_MAX_VH];

std::mutex g_noalloc_mutex;
double2* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(double2** out) {
  int dev = 0;
  WD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(WD_ERR_ARG, "mdagm_apply_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return WD_OK;
}

template <bool DAG, bool XPAY>
int launch(cudaStream_t s, const Geom& g, int out_par, const double2* gauge, const double2* in, double2* out,
           const double2* y, double alpha) {
  using A = HopArgs<SpF64, SpF64, SpF64, GF64>;
  SpF64 I{const_cast<double2*>(in), g.Vh}, O{out, g.Vh}, Y{const_cast<double2*>(y ? y : in), g.Vh};
  A a{g, out_par, I, O, Y, GF64{gauge, g.Vh}, alpha, Reduce{nullptr, nullptr, nullptr}, nullptr};
  k_hop<double, DAG, XPAY, false, 128, SpF64, SpF64, SpF64, GF64><<<nblocks(g.Vh, HOP_THREADS), HOP_THREADS, 0, s>>>(a);
  WD_CUDA(cudaGetLastError());
  return WD_OK;
}

}  // namespace
}  // namespace wd

using namespace wd;

extern "C" int mdagm_apply_noalloc(const int dims[4], const double* gauge_eo, double kappa, const double* in,
                                   double* out, void* stream) {
  if (!dims || !gauge_eo || !in || !out) return fail(WD_ERR_ARG, "mdagm_apply_noalloc: null argument");
  for (int m = 0; m < 4; ++m)
    if (dims[m] < 2 || dims[m] % 2 != 0)
      return fail(WD_ERR_ARG, "mdagm_apply_noalloc: every lattice extent must be even and >= 2");
  Geom g;
  for (int m = 0; m < 4; ++m) g.L[m] = dims[m];
  g.Lh = dims[0] / 2;
  g.V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  g.Vh = g.V / 2;
  if (g.Vh > NOALLOC_MAX_VH)
    return fail(WD_ERR_ARG, "mdagm_apply_noalloc: lattice has more than 32768 sites per parity "
                            "(the fixed scratch size); use mdagm_apply with a context instead");
  double2* scratch = nullptr;
  WD_TRY(scratch_address(&scratch));
  double2* t1 = scratch;                   // odd sites
  double2* t2 = scratch + 12 * g.Vh;       // even sites
  const cudaStream_t s = (cudaStream_t)stream;
  const double2* G = (const double2*)gauge_eo;
  const double2* x = (const double2*)in;
  double2* y = (double2*)out;
  const double a = -kappa * kappa;
  WD_TRY((launch<false, false>(s, g, 1, G, x, t1, nullptr, 0.0)));   // t1 = D_oe x
  WD_TRY((launch<false, true>(s, g, 0, G, t1, t2, x, a)));           // t2 = x - k^2 D_eo t1 = M_hat x
  WD_TRY((launch<true, false>(s, g, 1, G, t2, t1, nullptr, 0.0)));   // t1 = D^dag_oe t2
  WD_TRY((launch<true, true>(s, g, 0, G, t1, y, t2, a)));            // out = M_hat^dag t2
  return WD_OK;
}
