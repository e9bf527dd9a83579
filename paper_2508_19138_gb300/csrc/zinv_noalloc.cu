// Allocation-free variant of the batched block inverse.
//
// Some callers cannot allocate device memory at the point where they need an inverse: code
// running under a memory pool or allocator that must not be re-entered, code that has already
// handed all free memory to its own arena, or a host thread that must not take the CUDA driver's
// allocation lock in a latency-critical loop.  For them this entry point runs the same blocked
// Gauss-Jordan inversion as bt_zinv_batched, but its scratch (pivot rows and the panel copy)
// lives in one fixed array compiled into the library instead of a caller-provided workspace.
//
// Properties a caller must know:
//   * the array has BT_ZINV_NOALLOC_SCRATCH_BYTES bytes and exists on every GPU that loads the
//     library, for the life of the process;
//   * its device address is looked up once per device (cudaGetSymbolAddress) on the first call
//     made with that device current.  Under CUDA's default lazy module loading, that lookup is
//     also what loads this file's device code on the device, and with it reserves the array:
//     the driver allocates then, and can fail with BT_ERR_CUDA if the device is already full.
//     So make the first call on each device before any pool or arena takes the free memory, and
//     before any stream capture; later calls allocate nothing;
//   * all calls share the array: two calls whose work overlaps on the GPU (different streams,
//     or different host threads) race on it; calls on one stream are ordered and safe;
//   * nothing in the array needs to start at zero: every word is written before it is read,
//     and the array keeps whatever the last call left there;
//   * a request whose scratch would not fit is rejected with BT_ERR_BUDGET, nothing launched.
#include <mutex>

#include "bt_common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_zinv_scratch[BT_ZINV_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_zinv_scratch for the current device (host code cannot use the symbol's
// name as an address: there it names a host-side stand-in).
bt_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_zinv_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return BT_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BT_OK;
}

}  // namespace

extern "C" bt_status bt_zinv_batched_noalloc(int n, void* A, long long strideA, int batch, int* info_device,
                                             void* stream) {
  if (n < 0 || batch < 0 || (n > 0 && batch > 0 && !A)) return BT_ERR_INVALID_ARG;
  if (batch > 1 && strideA < (long long)n * n) return BT_ERR_INVALID_ARG;
  if (n == 0 || batch == 0) return BT_OK;
  const size_t need = bt::zinv_workspace_bytes(n, batch);
  if (need > (size_t)BT_ZINV_NOALLOC_SCRATCH_BYTES) return BT_ERR_BUDGET;
  void* scratch = nullptr;
  if (need > 0) BT_TRY(scratch_for_current_device(&scratch));
  return bt::zinv(static_cast<cudaStream_t>(stream), n, static_cast<zd*>(A), strideA, batch, info_device, scratch,
                  need > 0 ? (size_t)BT_ZINV_NOALLOC_SCRATCH_BYTES : 0, nullptr);
}
