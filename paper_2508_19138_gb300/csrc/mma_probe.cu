// Measurement aid, not part of the method: the issue rate of single-CTA tcgen05.mma (kind::f16,
// M = 128, N = 224, K = 16; 4 MMAs and one commit per 64-deep K block, the tensor-core GEMM's
// issue pattern) from one thread, with operands already in shared memory (no copies), while
// `busy` other warps of the CTA run dependent FP32 / 64-bit integer multiply-add chains (the
// instruction mix of the GEMM's accumulator drain) and, with `wait`, a ring-stage mbarrier wait
// that always succeeds before each K block.  Reports the tensor pipe's busy fraction: ideal
// cycles (N / 2 per MMA at 8192 flop per clock and SM) over measured cycles, mean over CTAs.
#include <vector>

#include "bt_common.cuh"
#include "sm103_ptx.cuh"

namespace {

constexpr int kProbeStages = 4;
constexpr uint32_t kProbeStage = 45056;  // 16 KB A + 28 KB B
constexpr int kProbeThreads = 640;       // MMA warp, TMEM warp, 2 idle, up to 16 busy warps

__global__ void __launch_bounds__(kProbeThreads, 1) mma_issue_probe_kernel(int iters, int busy, int wait,
                                                                           unsigned long long* out) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kProbeStages * kProbeStage);
  uint64_t* drain = bar + kProbeStages;
  uint64_t* sink = drain + 1;  // per-K-block commits land here; nothing waits on it
  volatile int* done = reinterpret_cast<volatile int*>(drain + 2);
  uint32_t* slot = reinterpret_cast<uint32_t*>(drain + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < (int)(kProbeStages * kProbeStage / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(sm)[i] = 0u;  // bf16 zeros
  if (threadIdx.x == 0) {
    for (int s = 0; s < kProbeStages; ++s) bt::ptx::mbar_init(&bar[s], 1);
    bt::ptx::mbar_init(drain, 1);
    bt::ptx::mbar_init(sink, 1);
    *done = 0;
    bt::ptx::fence_barrier_init();
  }
  if (warp == 1) {
    bt::ptx::tmem_alloc(slot, 512);
    bt::ptx::tmem_relinquish();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bt::ptx::tc_fence_before();
  __syncthreads();
  bt::ptx::tc_fence_after();
  const uint32_t tmem = *slot;
  if (threadIdx.x == 0)
    for (int s = 0; s < kProbeStages; ++s) bt::ptx::mbar_arrive(&bar[s]);  // phase 0 of every stage completes
  __syncthreads();
  if (warp == 1 && lane == 0) {
    const uint32_t idesc = bt::ptx::idesc_bf16_f32(128, 224);
    const uint32_t base = bt::ptx::smem_u32(sm);
    volatile int never = 0;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
      const int st = it & (kProbeStages - 1);
      if (wait) bt::ptx::mbar_wait_bounded(&bar[st], 0, &never, 2000000000ull);
      bt::ptx::tc_fence_after();
      const uint32_t a = base + (uint32_t)st * kProbeStage;
      const uint64_t ad = bt::ptx::sdesc_kmajor_sw128(a), bd = bt::ptx::sdesc_kmajor_sw128(a + 16384);
#pragma unroll
      for (int k = 0; k < 4; ++k) bt::ptx::umma_f16(tmem, ad + 2u * k, bd + 2u * k, idesc, (it | k) ? 1u : 0u);
      bt::ptx::umma_commit(sink);
    }
    bt::ptx::umma_commit(drain);
    bt::ptx::mbar_wait_bounded(drain, 0, &never, 2000000000ull);
    out[blockIdx.x] = (unsigned long long)(clock64() - t0);
    *done = 1;
  } else if (warp >= 4 && warp < 4 + busy) {
    float f = 1.0f + lane;
    unsigned long long acc = lane;
    while (!*done) {
#pragma unroll 16
      for (int i = 0; i < 64; ++i) {
        f = fmaf(f, 1.0000001f, 12582912.0f);
        acc += (unsigned long long)__float_as_uint(f) * 3u;
      }
    }
    if (acc == 12345ull) out[gridDim.x] = acc;  // keeps the chains alive
  }
  bt::ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    bt::ptx::tc_fence_after();
    bt::ptx::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

extern "C" bt_status bt_debug_mma_issue_rate(int busy_warps, int wait, double* frac, void* stream) {
  if (busy_warps < 0 || busy_warps > 16 || !frac) return BT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  BT_CUDA_TRY(cudaGetDevice(&dev));
  BT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = 1024 + kProbeStages * kProbeStage + 128;
  BT_CUDA_TRY(cudaFuncSetAttribute(mma_issue_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned long long* d = nullptr;
  BT_CUDA_TRY(cudaMallocAsync(&d, sizeof(unsigned long long) * (sms + 1), st));
  const int iters = 8192;
  mma_issue_probe_kernel<<<sms, kProbeThreads, smem, st>>>(iters, busy_warps, wait ? 1 : 0, d);
  bt::count_launch();
  std::vector<unsigned long long> h((size_t)sms);
  bt_status rc = cudaGetLastError() == cudaSuccess &&
                         cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost,
                                         st) == cudaSuccess &&
                         cudaStreamSynchronize(st) == cudaSuccess
                     ? BT_OK
                     : BT_ERR_CUDA;
  cudaFreeAsync(d, st);
  if (rc != BT_OK) return rc;
  double cyc = 0.0;
  for (int i = 0; i < sms; ++i) cyc += (double)h[(size_t)i];
  cyc /= sms;
  *frac = cyc > 0.0 ? 448.0 * iters / cyc : 0.0;
  return BT_OK;
}
