// fsim_fock_build_noalloc: the Fock build (J, K from D) for callers that must
// not allocate device memory while they run -- for example a server whose
// memory pool already owns the whole device budget, a loop that cannot afford
// the device-wide synchronisation that cudaMalloc/cudaFree bring, or a host
// whose allocator forbids raw cudaMalloc.  The paper has no counterpart; it is
// an interface addition of this library.
//
// The build needs scratch beyond its inputs and outputs: the FP64 J and K
// accumulators (2 N^2 doubles) and, in mixed precision, an FP32 copy of D
// (N^2 floats).  Here that scratch is one file-scope device array of fixed
// size, so the call never allocates:
//   * capacity: N <= kNoAllocMaxN basis functions (5 MiB in total); every GPU
//     that loads the library keeps this array until the process exits;
//   * the array is shared by every call on a device and keeps the previous
//     call's contents; the accumulators are cleared at the start of each call;
//     calls whose GPU work overlaps (e.g. on two streams at once) race on it;
//   * host code cannot use the array's name as a device address: set-up
//     fetches it with cudaGetSymbolAddress once per device, with that device
//     current.  The first allocating build of a basis does this
//     (noalloc_scratch_prepare, called when the basis allocates its own
//     scratch), so the module that holds the array is loaded then and a later
//     non-allocating call loads nothing; a first call on a device that never
//     ran that set-up looks the address up itself, which may load the 5 MiB
//     array, so it belongs in set-up too, before any stream capture.
#include <mutex>

#include "fsim_internal.h"

namespace fsim {
int fock_build_into(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o, double* Jacc,
                    double* Kacc, float* D32);
}  // namespace fsim

namespace {

constexpr int kNoAllocMaxN = 512;
constexpr size_t kAccBytes = (size_t)kNoAllocMaxN * kNoAllocMaxN * sizeof(double);
constexpr size_t kD32Bytes = (size_t)kNoAllocMaxN * kNoAllocMaxN * sizeof(float);
constexpr size_t kScratchBytes = 2 * kAccBytes + kD32Bytes;

static __device__ __align__(256) unsigned char g_fock_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (once per device).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    fsim::set_error("fsim_fock_build_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
    return FSIM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    fsim::set_error("fsim_fock_build_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return FSIM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fock_scratch);
    if (e != cudaSuccess || !p) {
      fsim::set_error("fsim_fock_build_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FSIM_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FSIM_OK;
}

}  // namespace

int fsim::noalloc_scratch_prepare() {
  void* p = nullptr;
  return scratch_address(&p);
}

extern "C" int fsim_fock_build_noalloc(fsim_basis* b, const double* D, double* J, double* K,
                                       const fsim_fock_opts* opts) {
  if (!b || !D || !J || !K || !opts) {
    fsim::set_error("fsim_fock_build_noalloc: null pointer");
    return FSIM_EINVAL;
  }
  if (opts->ptr_mode != FSIM_PTR_DEVICE) {
    fsim::set_error("fsim_fock_build_noalloc: D, J, K must be device pointers (ptr_mode FSIM_PTR_DEVICE)");
    return FSIM_EINVAL;
  }
  if (opts->timing) {
    fsim::set_error("fsim_fock_build_noalloc: per-kernel timing is not available here (it creates CUDA events)");
    return FSIM_EINVAL;
  }
  if (b->spherical) {
    fsim::set_error("fsim_fock_build_noalloc: spherical bases are not supported (use fsim_fock_build)");
    return FSIM_EINVAL;
  }
  if (b->nbf > kNoAllocMaxN) {
    fsim::set_error("fsim_fock_build_noalloc: %d basis functions exceed the fixed scratch capacity of %d", b->nbf,
                    kNoAllocMaxN);
    return FSIM_EINVAL;
  }
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) {
    fsim::set_error("fsim_fock_build_noalloc: the basis lives on device %d, device %d is current", b->device, cur);
    return FSIM_EINVAL;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FSIM_OK) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  // layout for this N: J_acc (N^2 doubles), K_acc (N^2 doubles), D in FP32 (N^2 floats)
  const size_t n2 = (size_t)b->nbf * b->nbf;
  double* Jacc = reinterpret_cast<double*>(p);
  double* Kacc = Jacc + n2;
  float* D32 = reinterpret_cast<float*>(Kacc + n2);
  return fsim::fock_build_into(b, D, J, K, *opts, Jacc, Kacc, D32);
}
