// Split-precision complex GEMM (placeholder until the tcgen05 kernel lands).
#include "bt_common.cuh"
namespace bt {
size_t split_workspace_bytes(int, int, int, int, int) { return 0; }
bt_status split_zgemm(cudaStream_t, int, int, int, zd, Operand, Operand, zd, zd*, int, long long, int, int, void*,
                      size_t, const int*) {
  return BT_ERR_UNSUPPORTED;
}
}  // namespace bt
extern "C" bt_status bt_split_zgemm_workspace_bytes(int, int, int, int, int, size_t* bytes) {
  if (bytes) *bytes = 0;
  return BT_ERR_UNSUPPORTED;
}
extern "C" bt_status bt_split_zgemm_batched(int, int, int, double, double, const void*, int, long long, int, const void*,
                                            int, long long, int, double, double, void*, int, long long, int, int, void*,
                                            size_t, void*) {
  return BT_ERR_UNSUPPORTED;
}
