// Batched forward zoom for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: code running inside
// another application's real-time video pipeline or render loop, where a
// device allocation may synchronise the device and stall every other stream,
// or a plugin that is handed image pointers but no allocator.  The batched
// entry point normally needs a caller-provided workspace (the tile queue); this
// variant keeps that queue in a fixed array in this library's own device
// memory instead, so the caller passes only the images.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (WENO_NOALLOC_SCRATCH_BYTES bytes) until the process exits.
// In host code its name is only a host-side stand-in, so the device address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.
#include <mutex>

#include "wd_batched.h"
#include "wd_common.cuh"
#include "wd_fwd.h"
#include "wdweno.h"

using namespace wdweno;

namespace {

// Queue head, tile total and the prefix sum of tiles of up to
// WENO_NOALLOC_MAX_IMAGES images, rounded up to 16 bytes exactly as
// batched_workspace_bytes rounds it: the batched call checks the workspace
// size against that rounded figure.
constexpr size_t kQueueBytesAtMax =
    (16 + 8 * (size_t(WENO_NOALLOC_MAX_IMAGES) + 1) + 15) & ~size_t(15);
static_assert(kQueueBytesAtMax <= WENO_NOALLOC_SCRATCH_BYTES, "scratch too small");

static __device__ __align__(256) unsigned char g_queue_scratch[WENO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_queue_scratch on the current device, looked up on the
// first call for that device.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WENO_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_queue_scratch) != cudaSuccess || !p) return WENO_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return WENO_OK;
}

}  // namespace

extern "C" int weno_zoom2x_batched_noalloc(int count, const weno_image* d_in, weno_dtype in_t,
                                           const weno_image* d_out, weno_dtype out_t,
                                           const weno_params* p, int rows_per_tile,
                                           int tile_width, void* stream) {
  if (count > WENO_NOALLOC_MAX_IMAGES) return WENO_ERANGE;
  if (count < 0) return WENO_EINVAL;
  if (count == 0) return WENO_OK;
  void* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != WENO_OK) return rc;
  // The batched path clears the queue head and rewrites the prefix sums on
  // every call, so the array needs no clearing here.
  // The whole array is offered as the workspace; the batched call checks it
  // against batched_workspace_bytes(count), which is at most kQueueBytesAtMax.
  return weno_zoom2x_batched(count, d_in, in_t, d_out, out_t, p, scratch,
                             WENO_NOALLOC_SCRATCH_BYTES, rows_per_tile, tile_width, stream);
}
