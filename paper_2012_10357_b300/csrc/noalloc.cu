// LBVH build that allocates nothing: pr_lbvh_build_noalloc.
//
// pr_lbvh_build takes the scratch of its radix-sort path from the
// stream-ordered pool at call time. Some callers cannot let a library
// allocate device memory while they run: applications whose device memory is
// owned by their own allocator under a fixed budget (every byte must come from
// that pool, so an outside allocation can fail or push them over budget), and
// latency-sensitive loops in which an allocation's possible device
// synchronisation or pool growth is not acceptable. For them this variant
// keeps its scratch in one file-scope device array of fixed size, held until
// the process exits. The array lives in this file's module, which CUDA may
// load lazily: the first call on a device (whatever n) looks its address up,
// which loads the module and reserves the array there if that has not
// happened yet. The address is kept per device for the life of the process,
// so destroying the primary context (cudaDeviceReset) while the library is in
// use is not supported.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/proceduray.h"
#include "internal.h"

namespace {

constexpr size_t a256c(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch of the radix-sort path for PR_LBVH_NOALLOC_MAX_BOXES boxes: key and
// value double buffers, refit counters and two parent arrays (7 x n words),
// per-tile digit histograms and the centroid-bounds partials.
constexpr size_t kMaxBoxes = PR_LBVH_NOALLOC_MAX_BOXES;
constexpr size_t kScratchBytes = 7 * a256c(4 * kMaxBoxes) +
                                 a256c(4 * 256 * ((kMaxBoxes + pr::kSortTile - 1) / pr::kSortTile)) +
                                 a256c(4 * 6 * pr::kMaxPartials) + 256;

// Shared by every call on a device; contents persist between calls.
static __device__ __align__(256) unsigned char g_lbvh_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_lbvh_scratch on the current device, looked up once per
// device. In host code the array's name is only a host-side stand-in.
pr_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    pr_internal_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return PR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    pr_internal_set_error("pr_lbvh_build_noalloc: device ordinal beyond 63");
    return PR_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_lbvh_scratch);
    if (e != cudaSuccess || !p) {
      pr_internal_set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return PR_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PR_OK;
}

}  // namespace

extern "C" pr_status pr_lbvh_build_noalloc(const float* boxes, uint32_t n, float* nodes, uint32_t* perm,
                                           uint32_t* codes, float* root_box, void* stream) {
  if (n == 0) return PR_OK;
  if (n > PR_LBVH_NOALLOC_MAX_BOXES) {
    pr_internal_set_error("pr_lbvh_build_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                          std::to_string(PR_LBVH_NOALLOC_MAX_BOXES) + " boxes; use pr_lbvh_build");
    return PR_ERR_INVALID_ARG;
  }
  if (!boxes || !perm || !codes || !root_box || (n > 1 && !nodes)) {
    pr_internal_set_error("pr_lbvh_build_noalloc: null device pointer");
    return PR_ERR_INVALID_ARG;
  }
  if (((uintptr_t)nodes & 15) || ((uintptr_t)root_box & 15)) {
    pr_internal_set_error("pr_lbvh_build_noalloc: nodes and root_box must be 16-byte aligned");
    return PR_ERR_INVALID_ARG;
  }
  if (pr::build_scratch_bytes(n) > kScratchBytes) {
    pr_internal_set_error("pr_lbvh_build_noalloc: scratch layout larger than the fixed array");
    return PR_ERR_INVALID_ARG;
  }
  // the per-device set-up runs on the first call, also when this call needs no scratch
  void* scratch = nullptr;
  pr_status s = scratch_address(&scratch);
  if (s != PR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  pr::LevelDesc J;
  J.boxes = boxes;
  J.gather = nullptr;
  J.n = n;
  J.leaf_ref_base = 0;
  J.nodes = reinterpret_cast<float4*>(nodes);
  J.perm = perm;
  J.codes = codes;
  J.root_box = root_box;
  if (n <= pr::kSmallMax) {
    pr::launch_build_small_one(J, st);           // one CTA, shared memory only
  } else {
    // the refit counters must start at zero: the radix-sort path clears them
    // with cudaMemsetAsync on `stream` before its refit kernel
    pr::launch_build_large(J, pr::carve_build_scratch(scratch, n), st);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    pr_internal_set_error(std::string("pr_lbvh_build_noalloc launch: ") + cudaGetErrorString(e));
    return PR_ERR_CUDA;
  }
  return PR_OK;
}
