// wpcd_kapply_noalloc: the Faddeev kernel application y = O P0 Vt (g o x)
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a stream is being
// captured into a CUDA graph (allocation calls are not capturable), hosts
// that run the library inside an application whose device memory is owned
// by a fixed-size pool or a foreign allocator, and real-time loops that must
// not touch the allocator after start-up.  wpcd_kapply takes its two
// intermediate vectors from cudaMalloc on every call; this variant takes
// them from a fixed array in device memory that the library reserves when
// it is loaded.
//
// The array is a file-scope __device__ variable of WPCD_NOALLOC_MAX_DIM x 2
// complex doubles (4 MiB).  Every GPU that loads the library holds it until
// the process exits.  In host code its name is only a host-side stand-in,
// so its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; that first call should therefore come before any stream
// capture.  All calls share the array and it keeps the last call's contents;
// both intermediates are fully overwritten by every call, so nothing has to
// start at zero, but calls whose executions overlap on the GPU (different
// streams, or concurrent host threads on one device) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "wpcd_internal.h"

namespace {

// intermediates Vt (g o x) and P0 (...) of one application: 2 x dim complex
__device__ __align__(256) double2 g_kapply_scratch[2 * WPCD_NOALLOC_MAX_DIM];

constexpr int kMaxDevices = 64;
double2 *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

wpcd_status scratch_for_device(int device, double2 **out) {
  if (device < 0 || device >= kMaxDevices) return wpcd::set_error(WPCD_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_kapply_scratch);  // the device is current (caller)
    if (e != cudaSuccess) return wpcd::cuda_error(e, "cudaGetSymbolAddress (no-alloc scratch)");
    g_scratch_addr[device] = static_cast<double2 *>(p);
  }
  *out = g_scratch_addr[device];
  return WPCD_OK;
}

}  // namespace

extern "C" wpcd_status wpcd_kapply_noalloc(const wpcd_problem *pr, const wpcd_P *P, const double *g,
                                           const double *x, double *y, void *stream) {
  wpcd::clear_error();
  WPCD_GUARD_BEGIN
  if (!pr || !P || !x || !y || x == y) return wpcd::set_error(WPCD_EINVAL, "bad kapply arguments");
  if (!wpcd::P_fits(P, pr)) return wpcd::set_error(WPCD_EINVAL, "P was assembled on another lattice or for another channel count");
  const int64_t dim = (int64_t)pr->n_ch * pr->N * pr->M;
  if (dim > WPCD_NOALLOC_MAX_DIM)
    return wpcd::set_error(WPCD_EINVAL,
                           "problem dimension exceeds WPCD_NOALLOC_MAX_DIM (131072) of the no-alloc scratch");
  cudaError_t e = cudaSetDevice(pr->device);
  if (e != cudaSuccess) return wpcd::cuda_error(e, "cudaSetDevice");
  double2 *scratch = nullptr;
  wpcd_status st = scratch_for_device(pr->device, &scratch);
  if (st != WPCD_OK) return st;
  return wpcd::kapply_scratch(pr, P, g, x, y, reinterpret_cast<double *>(scratch),
                              reinterpret_cast<double *>(scratch + dim), static_cast<cudaStream_t>(stream));
  WPCD_GUARD_END
}
