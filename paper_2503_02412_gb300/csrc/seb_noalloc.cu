// Allocation-free pose query: forward and hand-written backward in one call, for callers
// that cannot allocate device memory (a real-time loop running under a fixed memory budget,
// or a host that embeds the library behind an allocator it does not own).  The per-pose state
// the backward reuses, which seb_query_poses normally writes to a caller buffer, lives here in
// a file-scope device array instead.
//
// Limits and sharing:
//   - the array holds at most kNoAllocMaxPoses poses (4 MiB); larger batches are rejected;
//   - every GPU that loads the library keeps the array until the process exits;
//   - all calls share it: two calls whose kernels overlap on the GPU (different streams, no
//     ordering between them) race on it.  Calls on one stream are safe;
//   - nothing in it must start at zero: the forward writes the record of every pose the
//     backward then reads, within the same call;
//   - the first call on a device (with n >= 1) resolves the array's device address
//     (cudaGetSymbolAddress with that device current) and caches it.  With lazy module loading
//     that lookup also loads the module and its 4 MiB array onto the device, so it may fail for
//     lack of device memory: make that first call once at start-up, before any stream capture
//     and before the memory budget is taken.
#include <mutex>
#include <string.h>

#include "seb_internal.h"

namespace {

constexpr int64_t kNoAllocMaxPoses = SEB_NOALLOC_MAX_POSES;

// Per-pose saved state of the forward, read back by the backward (SEB_QUERY_SAVED floats each).
static __device__ __align__(256) float g_saved_scratch[kNoAllocMaxPoses * SEB_QUERY_SAVED];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's name
// is only a host-side stand-in, so the address has to come from the runtime.
int scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    seb::set_error("cudaGetDevice: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    seb::set_error("device index %d beyond %d", dev, kMaxDevices);
    return SEB_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_saved_scratch);
    if (e != cudaSuccess || !p) {
      seb::set_error("cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      return SEB_ERR_CUDA;
    }
    g_scratch_dev[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_dev[dev];
  return SEB_OK;
}

}  // namespace

extern "C" int seb_query_poses_grad_noalloc(const seb_params* p, const void* elev, int64_t oi, int64_t oj,
                                            const float* poses, int64_t n, const float* grad_out, float* out,
                                            uint8_t* flags, float* grad_pose, seb_stream_t stream) {
  SEB_RANGE();
  if (!p || !elev || n < 0 || (n > 0 && (!poses || !grad_out || !out || !flags || !grad_pose))) {
    seb::set_error("seb_query_poses_grad_noalloc: NULL pointer or negative count");
    return SEB_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxPoses) {
    seb::set_error("seb_query_poses_grad_noalloc: %lld poses exceed the %lld-pose scratch; split the batch "
                   "or use seb_query_poses with a caller buffer",
                   (long long)n, (long long)kNoAllocMaxPoses);
    return SEB_ERR_INVALID_ARG;
  }
  // the same lattice, validation and launch record as seb_query_poses (no heap memory)
  seb::QTab Q;
  seb::QLaunch L;
  int rc = seb::query_setup(*p, elev, oi, oj, poses, n, &Q, &L);
  if (rc) return rc;
  if (n == 0) return SEB_OK;
  float* saved = nullptr;
  rc = scratch_address(&saved);
  if (rc) return rc;
  L.out = out;
  L.flags = flags;
  L.saved = saved;
  cudaError_t e = seb::launch_query(Q, L, p->elev_dtype, false, (cudaStream_t)stream);
  if (e == cudaSuccess) {
    L.gout = grad_out;
    L.gpose = grad_pose;
    e = seb::launch_query(Q, L, p->elev_dtype, true, (cudaStream_t)stream);
  }
  if (e != cudaSuccess) {
    seb::set_error("seb_query_poses_grad_noalloc launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}
