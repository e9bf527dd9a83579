// Shared device/host helpers of the sm_103a kernels: complex128 arithmetic on double2,
// launch checks, and the internal launcher declarations used across translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include "../../include/bt_selinv.h"

typedef double2 zd;  // complex128: x = re, y = im

__host__ __device__ __forceinline__ zd zmake(double r, double i) { zd z; z.x = r; z.y = i; return z; }
__host__ __device__ __forceinline__ zd zadd(zd a, zd b) { return zmake(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zd zsub(zd a, zd b) { return zmake(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zd zmul(zd a, zd b) {
  return zmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ zd zconj(zd a) { return zmake(a.x, -a.y); }
__host__ __device__ __forceinline__ zd zscale(zd a, double s) { return zmake(a.x * s, a.y * s); }
// acc += a * b with four fused multiply-adds
__device__ __forceinline__ void zfma(zd& acc, zd a, zd b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// 1 / a, scaled to avoid overflow of |a|^2 (Smith's method)
__host__ __device__ __forceinline__ zd zinv(zd a) {
  double ar = a.x, ai = a.y;
  if (fabs(ar) >= fabs(ai)) {
    double r = ai / ar, d = ar + ai * r;
    return zmake(1.0 / d, -r / d);
  } else {
    double r = ar / ai, d = ai + ar * r;
    return zmake(r / d, -1.0 / d);
  }
}
__host__ __device__ __forceinline__ double zabs1(zd a) { return fabs(a.x) + fabs(a.y); }

#define BT_CUDA_TRY(expr)                                      \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return BT_ERR_CUDA;                 \
  } while (0)

#define BT_TRY(expr)                                           \
  do {                                                         \
    bt_status _s = (expr);                                     \
    if (_s != BT_OK) return _s;                                \
  } while (0)

namespace bt {

// Kernel launches issued by this library (process-wide counter).
void count_launch();
long long launches_total();

// One GEMM operand: element (r, c) of op(X) for batch entry b is
//   op == BT_OP_N : X[b*stride + r*ld + c]
//   op == BT_OP_C : conj(X[b*stride + c*ld + r])
struct Operand {
  const zd* p;
  int ld;
  long long stride;
  int op;
};

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b]; rows m, cols n, depth k.  active[b] == 0 skips
// batch entry b (active may be null).  FP64 (DFMA) kernel.
bt_status zgemm(cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta,
                zd* C, int ldc, long long strideC, int batch, const int* active, int tile = 0);

// C = alpha op(A) op(B) + beta C for a square n x n C whose exact value is anti-Hermitian
// (alpha real, beta C anti-Hermitian, op(A) op(B) anti-Hermitian): the tiles on and above the
// diagonal are computed, the others written as -(upper)^H.  Complex alpha: plain zgemm.
bt_status zgemm_antiherm(cudaStream_t st, int n, int k, zd alpha, Operand A, Operand B, zd beta, zd* C, int ldc,
                         long long strideC, int batch, const int* active, int tile = 0);

// Which kernel runs a complex product: FP64 DFMA (slices == 0) or the sliced bf16 tensor-core
// product with `slices` slices per operand and its workspace.
struct Engine {
  int slices = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* err = nullptr;  // sliced products: one device word set to BT_ERR_TIMEOUT by a bounded wait
  int tile = 0;        // FP64 products: output tile 16 or 32 (0: 32 unless that leaves SMs idle)
  int panel = 0;       // inversions: panel width below the default (0: the default)
};

// Split-precision (sliced bf16 tensor-core) variant of zgemm; see split_gemm.cu.
size_t split_workspace_bytes(int m, int n, int k, int slices, int batch);
// A bounded wait that expires sets err[b * err_stride] = BT_ERR_TIMEOUT for the batch entry b of
// the CTA (err may be null; err_stride 0 makes it one word for the whole call).
//
// An operand may come pre-sliced (SlicedOp: sliced once by slice_op, reused by every product it
// enters while its values stay the same); its shape, slice count, batch and k must match the
// product's, and k <= 1024 (one K chunk).
struct SlicedOp {
  uint32_t* t = nullptr;  // slice words
  int* e = nullptr;       // line exponents
  int role = -1;          // 0: rows of op(A) (At operand), 1: columns of op(B) (Bt operand)
  int lines = 0, kc = 0, S = 0, batch = 0;
  bool shared = false;    // one operand for every batch entry (sliced once)
  bool valid() const { return t != nullptr; }
};
size_t sliced_op_bytes(int role, int lines, int k, int slices, int batch);
bt_status slice_op(cudaStream_t st, int role, int lines, int k, Operand X, int batch, int slices, void* buf,
                   size_t bytes, SlicedOp* out);
bt_status split_zgemm(cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta,
                      zd* C, int ldc, long long strideC, int batch, int slices, void* ws,
                      size_t ws_bytes, const int* active, int* err = nullptr, long long err_stride = 0,
                      const SlicedOp* preA = nullptr, const SlicedOp* preB = nullptr);

// C = alpha op(A) op(B) + beta C on the engine's kernel.
bt_status gemm(const Engine& eng, cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta,
               zd* C, int ldc, long long strideC, int batch, const int* active);
// The anti-Hermitian variant (zgemm_antiherm on the FP64 engine; the sliced engine computes all of C).
bt_status gemm_antiherm(const Engine& eng, cudaStream_t st, int n, int k, zd alpha, Operand A, Operand B, zd beta,
                        zd* C, int ldc, long long strideC, int batch, const int* active);

// In-place batched inverse (Gauss-Jordan, partial pivoting).  info[b] |= error code.  The
// rank-kb updates of the blocked variant run on `eng` (FP64 unless given).
// `wide`: workspace for the wider panels used when the updates run sliced (Engine::slices > 0).
size_t zinv_workspace_bytes(int n, int batch, bool wide = false);
bt_status zinv(cudaStream_t st, int n, zd* A, long long strideA, int batch, int* info, void* ws,
               size_t ws_bytes, const int* active, const Engine* eng = nullptr);

// Graph mode of the decimation: `st` is being captured into a CUDA graph, and the iteration
// loop is captured as a conditional while node whose body (one iteration and the convergence
// test) is recorded on `body_stream`; the device decides when to stop.  body_launches returns
// the kernels of one pass of the body.
struct LoopCapture {
  cudaStream_t body_stream = nullptr;
  long long body_launches = 0;
};

// One Newton step on decimated surface functions (see decimate.cu): for the leads whose
// decimation took more than `after` iterations, e_s <- e_s + d with d solving the linearised
// equation d - (n x) d (x n') = m - n x n' - e_s (a Stein equation, solved by doubling).
struct Polish {
  int after = -1;                 // < 0: no lead is polished
  int* iters = nullptr;           // [batch] device: doubling iterations per lead (0 = not polished)
  long long lead_iterations = 0;  // direct mode: doubling iterations summed over the leads
  int selected = 0;               // direct mode: leads that took the step
  long long body_launches = 0;    // graph mode: kernels of one pass of the doubling loop
  const Engine* engine = nullptr; // products of the step (null: FP64)
};

// Sancho-Rubio decimation for `batch` leads.  With `loop` (graph capture), iters_host_max and
// lead_iterations are not written: the per-lead counts are in `iters` on the device.
size_t decimate_workspace_bytes(int bs, int batch, bool wide = false);
bt_status decimate(cudaStream_t st, int bs, int batch, const zd* m, const zd* n, const zd* np,
                   double tol, int maxit, zd* x, zd* sigma, int* iters, int* info, void* ws,
                   size_t ws_bytes, int* iters_host_max, int* h_pinned, const int* mask = nullptr,
                   long long* lead_iterations = nullptr, const Engine* eng = nullptr,
                   LoopCapture* loop = nullptr, Polish* polish = nullptr);

// X = R + A X B for `batch` independent bs x bs problems (B = A^H when B is null), by doubling:
// X <- X + A X B, A <- A A, B <- B B until bs^2 max|A| max|B| <= tol.  X holds R on entry; A and B
// are overwritten.  mask[l] == 0 leaves problem l alone (mask may be null); ok[l] = 1 where the
// doubling converged within maxit, else 0 (X is then a partial sum); iters[l] = doublings.
// With `loop` (graph capture) the doubling loop is a conditional while node (its body's kernel
// count in *body_launches) and the counts are left on the device; otherwise *lead_iterations =
// doublings summed over the problems.
size_t stein_workspace_bytes(int bs, int batch);
bt_status stein(cudaStream_t st, int bs, int batch, zd* A, zd* B, zd* X, double tol, int maxit, const int* mask,
                int* ok, int* iters, void* ws, size_t ws_bytes, int* h_pinned, long long* lead_iterations,
                const Engine* eng = nullptr, LoopCapture* loop = nullptr, long long* body_launches = nullptr);
bt_status invert_mask(cudaStream_t st, int batch, const int* a, int* out);  // out = !a
// info[l] = ok[l] ? 0 : code (masked-out problems, mask[l] == 0, get 0)
bt_status status_from_ok(cudaStream_t st, int batch, const int* ok, const int* mask, int code, int* info);
// Fixed-point iteration x <- (m - n x n')^{-1} (Eq. 5) from the given x for leads with run[l];
// conv[l] = 1 where it converged to tol within nfpi iterations.
bt_status fixed_point(cudaStream_t st, int bs, int batch, const zd* m, const zd* n, const zd* np, zd* x,
                      const int* run, int* conv, int nfpi, double tol, int* info, void* ws, size_t ws_bytes,
                      int* h_pinned, long long* lead_iterations, const Engine* eng = nullptr);

// Context creation with an optional lent workspace (serving arena); see selinv.cu.
bt_status ctx_create(const bt_selinv_desc* desc, void* cuda_stream, void* ext_ws, size_t ext_bytes, bt_ctx** out,
                     std::string* err);
size_t ctx_workspace_bytes(const bt_selinv_desc& d);

}  // namespace bt
