// FP64 issue-rate probe: the two ways GB300 can do FP64 multiply-adds, each kept busy on
// registers only (no memory traffic), so that their ceilings can be compared directly.
//   which 0: DFMA, 8 independent chains per thread (fma.rn.f64)
//   which 1: DMMA, the FP64 tensor instruction mma.sync.aligned.m8n8k4 (512 flops per warp-wide
//            instruction), 4 independent accumulator tiles per warp
// A complex GEMM built on either cannot run faster than its probe's rate, which is what decides
// between them for the FP64 products of the sweeps (the paper's hardware has an FP64 tensor rate
// far above its FMA rate; GB300 does not).  Not part of the method: a measurement aid.
#include "bt_common.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_probe_kernel(int iters, double seed, double* out) {
  double a[8], b = 1.0 + 1e-9 * threadIdx.x, c = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 12345.678) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) dmma_probe_kernel(int iters, double seed, double* out) {
  double a = seed + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * blockIdx.x;
  double d[4][2];
#pragma unroll
  for (int t = 0; t < 4; ++t) { d[t][0] = 0.0; d[t][1] = 0.0; }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[t][0]), "+d"(d[t][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 4; ++t) s += d[t][0] + d[t][1];
  if (s == 12345.678) out[0] = s;
}

}  // namespace

extern "C" bt_status bt_debug_fp64_rate(int which, int iters, double* tflops, double* ms, void* stream) {
  if ((which != 0 && which != 1) || iters < 1 || !tflops) return BT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  BT_CUDA_TRY(cudaGetDevice(&dev));
  BT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * 8;
  double* out = nullptr;
  BT_CUDA_TRY(cudaMallocAsync(&out, sizeof(double), st));
  cudaEvent_t e0, e1;
  BT_CUDA_TRY(cudaEventCreate(&e0));
  BT_CUDA_TRY(cudaEventCreate(&e1));
  auto launch = [&]() {
    if (which == 0) dfma_probe_kernel<<<grid, kThreads, 0, st>>>(iters, 0.5, out);
    else dmma_probe_kernel<<<grid, kThreads, 0, st>>>(iters, 0.5, out);
    bt::count_launch();
  };
  launch();  // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  bt_status rc = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess ? BT_OK : BT_ERR_CUDA;
  float t = 0.f;
  if (rc == BT_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = BT_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (rc != BT_OK) return rc;
  const double threads = (double)grid * kThreads;
  // DFMA: 8 fma per thread per iteration, 2 flops each.  DMMA: per warp 4 instructions of
  // 8 x 8 x 4 multiply-adds (512 flops) per iteration.
  const double flops = which == 0 ? threads * iters * 8.0 * 2.0 : threads / 32.0 * iters * 4.0 * 512.0;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return BT_OK;
}

// Measurement aid: the current device's preferred L1 / shared-memory split for kernels that set
// no carveout of their own (cudaDeviceSetCacheConfig; state of this process's context only).
extern "C" bt_status bt_debug_cache_config(int config) {
  if (config < 0 || config > 3) return BT_ERR_INVALID_ARG;
  BT_CUDA_TRY(cudaDeviceSetCacheConfig(static_cast<cudaFuncCache>(config)));
  return BT_OK;
}
