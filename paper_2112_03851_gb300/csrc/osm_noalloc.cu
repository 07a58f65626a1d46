// osm_apply_noalloc: the subdomain operator y = A x without any device
// allocation by the library during or for the call.
//
// Some callers cannot call cudaMalloc at the point where they need the
// operator.  A plug-in that runs inside a host framework usually finds the
// device memory already reserved by that framework's caching allocator,
// which also caps what a component may take; a cudaMalloc of its own would
// bypass that accounting and can fail once the framework holds the memory.
// A caller with a fixed memory budget decided at start-up (a service that
// must not allocate while serving) is in the same position.  This entry
// point serves them: besides the caller's input and output it touches only a
// fixed scratch array that is part of the library image itself.
//
// The scratch lives in the file-scope array below.  Every GPU that loads this
// library holds it (8 MiB) until the process exits.  In host code the array's
// name is only a host-side stand-in, so the first call on each device looks
// up the array's device address with cudaGetSymbolAddress (with that device
// current) and passes that address to the kernels; that first call should
// therefore come before any stream capture.  All calls share the array and it
// keeps the last call's contents: the part of it that must start at zero is
// cleared by every call, and calls that overlap on the GPU (two streams, two
// threads) race on it.  The call synchronises the handle's stream before it
// returns, so y is ready when it does.
#include <cuda_runtime.h>

#include <mutex>

#include "osm_internal.h"

namespace {

// Two vectors of at most kNoAllocMaxRows padded rows each.
constexpr int64_t kNoAllocMaxRows = int64_t(1) << 19;
static __device__ __align__(256) double g_apply_scratch[2 * kNoAllocMaxRows];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" osm_status osm_apply_noalloc(osm_handle h, int32_t op, const double* x, double* y) {
  cudaStream_t stream = nullptr;
  int64_t vec_rows = 0;
  int device = -1;
  const osm::DevProblem* d = osm::handle_problem(h, &stream, &vec_rows, &device);
  if (!d || !x || !y || (op != 0 && op != 1)) return OSM_E_ARG;
  if (vec_rows > kNoAllocMaxRows) {
    osm::handle_set_error(h, "osm_apply_noalloc: problem exceeds the fixed scratch of 524288 padded rows "
                             "(osm_info vec_rows); use osm_apply");
    return OSM_E_ARG;
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != device) e = cudaErrorInvalidDevice;
  double* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(cur, &scratch);
  double* w = scratch;
  double* ys = scratch + kNoAllocMaxRows;
  // padding rows of the scattered input must read as zero
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(double) * vec_rows, stream);
  if (e == cudaSuccess) e = osm::launch_apply_scratch(*d, op, x, y, w, ys, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    osm::handle_set_error(h, cudaGetErrorString(e));
    return OSM_E_CUDA;
  }
  return OSM_OK;
}
