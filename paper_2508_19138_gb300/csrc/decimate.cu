// Sancho-Rubio decimation for the retarded open-boundary condition (Sec. 4.2, Eq. 4):
//     x = (m - n x n')^{-1}
// for a batch of independent semi-infinite leads (cells with diagonal block m, coupling n from a
// cell to the next one away from the device and n' back).  Every iteration removes every second
// cell of the lead (Sancho, Lopez Sancho, Rubio 1985, the method the paper cites):
//     g = e^{-1};  e_s -= a g b;  e -= a g b + b g a;  a <- -a g a;  b <- -b g b
// from a = n, b = n', e = e_s = m, until max|a|, max|b| <= tol * max(|n|, |n'|); then
// x = e_s^{-1} and the boundary block sigma = n x n'.
//
// The per-lead convergence test is a max-|.|^2 reduction (integer keys, warp shuffles, one
// atomicMax per CTA over many CTAs per lead); converged leads drop out of every later launch
// through an `active` mask, and
// the host stops as soon as the device-side count of active leads reaches zero.  The loop is
// bounded by maxit; leads still active then get BT_ERR_NOT_CONVERGED (never a hang).
// In graph mode the same loop is a conditional while node of the captured graph: a one-thread
// kernel at the end of each iteration sets the loop condition from that count and the device
// iteration counter, so a whole solve runs without returning to the host.
//
// Newton polish.  Decimation in FP64 loses accuracy where a lead mode decays slowly (energies
// near a band edge at small eta): a rounding error made early is carried through the 2^k
// decimated cells, and the surface function comes out up to ~1e-8 off (checked against an
// extended-precision decimation).  For leads whose decimation took more than `after` iterations
// one Newton step on e_s restores FP64 accuracy: with x = e_s^{-1} the residual of
// e_s = m - n e_s^{-1} n' is r = m - n x n' - e_s, and the correction d solves the linearised
// equation d - (n x) d (x n') = r, a Stein equation X = R + A X B solved by doubling
// (X <- X + A X B, A <- A A, B <- B B: after k steps X sums the first 2^k terms).  Then
// e_s <- e_s + d and x = e_s^{-1}.  The same doubling solves the Stein equation of the W
// contacts (Eq. 7).
#include <cstring>
#include <utility>
#include <vector>

#include "bt_common.cuh"

namespace bt {
namespace {

constexpr int NT = 256;

// Per-lead maxima of squared moduli over bs^2 elements, spread over (chunks x leads) CTAs.  The
// maxima are kept as the bit patterns of non-negative doubles, which order like the doubles:
// integer max reductions and one atomicMax per CTA, so the only FP64 work is |z|^2 (two
// instructions per element on GB300's narrow FP64 pipe).  A component with an all-ones exponent
// (Inf / NaN) sets the lead's non-finite flag.
//   kind 0: keys[2l] = max |X|^2, keys[2l+1] = max |Y|^2
//   kind 1: keys[2l] = max |X - Y|^2, keys[2l+1] = max |X|^2
__device__ __forceinline__ unsigned long long sq_key(zd a) {
  return (unsigned long long)__double_as_longlong(fma(a.x, a.x, a.y * a.y));
}
__device__ __forceinline__ int nonfinite_bits(zd a) {
  const unsigned long long x = (unsigned long long)__double_as_longlong(a.x),
                           y = (unsigned long long)__double_as_longlong(a.y);
  return ((x & 0x7FF0000000000000ull) == 0x7FF0000000000000ull) ||
         ((y & 0x7FF0000000000000ull) == 0x7FF0000000000000ull);
}
__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}

template <int KIND>
__global__ void __launch_bounds__(NT) lead_max_kernel(long long bs2, const zd* __restrict__ X,
                                                      const zd* __restrict__ Y, const int* __restrict__ active,
                                                      unsigned long long* __restrict__ keys, int* __restrict__ flags) {
  __shared__ unsigned long long sh0[NT / 32], sh1[NT / 32];
  const int l = blockIdx.y;
  if (active && active[l] == 0) return;
  unsigned long long k0 = 0, k1 = 0;
  int bad = 0;
  const zd* x = X + (long long)l * bs2;
  const zd* y = Y + (long long)l * bs2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const zd u = x[i], v = y[i];
    bad |= nonfinite_bits(u) | nonfinite_bits(v);
    unsigned long long a, b;
    if (KIND == 0) { a = sq_key(u); b = sq_key(v); }
    else { a = sq_key(zsub(u, v)); b = sq_key(u); }
    k0 = a > k0 ? a : k0;
    k1 = b > k1 ? b : k1;
  }
  bad = __syncthreads_or(bad);
  k0 = warp_umax(k0);
  k1 = warp_umax(k1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sh0[w] = k0; sh1[w] = k1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < NT / 32; ++i) { k0 = sh0[i] > k0 ? sh0[i] : k0; k1 = sh1[i] > k1 ? sh1[i] : k1; }
    atomicMax(&keys[2 * l], k0);
    atomicMax(&keys[2 * l + 1], k1);
    if (bad) atomicOr(&flags[l], 1);
  }
}

__device__ __forceinline__ double key_sqrt(unsigned long long k) { return sqrt(__longlong_as_double((long long)k)); }

bt_status lead_max(cudaStream_t st, int kind, long long bs2, int batch, const zd* X, const zd* Y, const int* active,
                   unsigned long long* keys, int* flags) {
  BT_CUDA_TRY(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * 2 * batch, st));
  BT_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * batch, st));
  long long chunks = (bs2 + NT * 8 - 1) / (NT * 8);
  if (chunks > 64) chunks = 64;
  dim3 g((unsigned)chunks, (unsigned)batch);
  if (kind == 0) lead_max_kernel<0><<<g, NT, 0, st>>>(bs2, X, Y, active, keys, flags);
  else lead_max_kernel<1><<<g, NT, 0, st>>>(bs2, X, Y, active, keys, flags);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

// ref[l] = max(max|n|, max|n'|)
__global__ void ref_kernel(int batch, const unsigned long long* __restrict__ keys, double* __restrict__ ref) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch) return;
  ref[l] = key_sqrt(keys[2 * l] > keys[2 * l + 1] ? keys[2 * l] : keys[2 * l + 1]);
}

// convergence test of one iteration: lead l leaves the active set once max|a|,|b| <= tol*ref
__global__ void check_kernel(int batch, const unsigned long long* __restrict__ keys, const int* __restrict__ flags,
                             const double* __restrict__ ref, double tol, int it, int* __restrict__ active,
                             int* __restrict__ iters, int* __restrict__ info, int* __restrict__ n_active) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch || active[l] == 0) return;
  const double v = key_sqrt(keys[2 * l] > keys[2 * l + 1] ? keys[2 * l] : keys[2 * l + 1]);
  iters[l] = it;
  if (flags[l] || info[l] != 0) {
    if (info[l] == 0) info[l] = BT_ERR_NONFINITE;
    active[l] = 0;
  } else if (v <= tol * ref[l]) {
    active[l] = 0;
  } else {
    atomicAdd(n_active, 1);
  }
}

// es -= t; e -= t  (active leads only)
__global__ void sub2_kernel(long long bs2, int batch, const zd* __restrict__ t, zd* __restrict__ es,
                            zd* __restrict__ e, const int* __restrict__ active) {
  const int l = blockIdx.y;
  if (active[l] == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)l * bs2 + i;
    es[o] = zsub(es[o], t[o]);
    e[o] = zsub(e[o], t[o]);
  }
}

// active[l] = mask[l] (all leads without a mask); state of masked-out leads is left alone
__global__ void init_kernel(int batch, const int* __restrict__ mask, int* active, int* iters, int* info) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch) return;
  const int on = mask ? (mask[l] != 0) : 1;
  active[l] = on;
  if (on) { iters[l] = 0; info[l] = 0; }
}

__global__ void finish_kernel(int batch, const int* active, int* info) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < batch && active[l] != 0 && info[l] == 0) info[l] = BT_ERR_NOT_CONVERGED;
}

// dst[l] = src[l] for leads with mask[l] != 0 (all leads without a mask)
__global__ void masked_copy_kernel(long long bs2, const zd* __restrict__ src, zd* __restrict__ dst,
                                   const int* __restrict__ mask) {
  const int l = blockIdx.y;
  if (mask && mask[l] == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x)
    dst[(long long)l * bs2 + i] = src[(long long)l * bs2 + i];
}

// Fixed-point convergence test: lead l converged when max|x_new - x| <= tol * max|x_new|.  A
// lead whose geometric extrapolation (rate = this update / previous update) cannot reach the
// tolerance within the remaining iterations is given up (left for decimation).
__global__ void fpi_check_kernel(int batch, const unsigned long long* __restrict__ keys,
                                 const int* __restrict__ flags, double tol, int it, int nfpi,
                                 int* __restrict__ active, int* __restrict__ conv, double* __restrict__ prev,
                                 int* __restrict__ n_active) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch || active[l] == 0) return;
  const double d = flags[l] ? __longlong_as_double(0x7ff8000000000000ll) : key_sqrt(keys[2 * l]);
  const double r = key_sqrt(keys[2 * l + 1]);
  // linear convergence with rate rho = d_k / d_{k-1}: the distance to the fixed point is
  // about d rho / (1 - rho).  The first update has no rate: accept it only 10x below tol.
  const double rate = it > 1 && prev[l] > 0.0 ? d / prev[l] : 0.0;
  const double err = it > 1 ? (rate < 1.0 ? d * rate / (1.0 - rate) : INFINITY) : 10.0 * d;
  if (d <= tol * r && err <= tol * r) {
    active[l] = 0;
    conv[l] = 1;
  } else {
    const bool hopeless =
        isnan(d) || (it > 1 && (rate >= 1.0 || d * pow(rate, (double)(nfpi - it)) > tol * r * (1.0 - rate)));
    if (hopeless || it >= nfpi) { active[l] = 0; conv[l] = 0; }
    else atomicAdd(n_active, 1);
    prev[l] = d;
  }
}

// Graph mode: the convergence test reads the iteration number from the device counter.
__global__ void check_dev_kernel(int batch, const unsigned long long* __restrict__ keys, const int* __restrict__ flags,
                                 const double* __restrict__ ref, double tol, const int* __restrict__ itc,
                                 int* __restrict__ active, int* __restrict__ iters, int* __restrict__ info,
                                 int* __restrict__ n_active) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch || active[l] == 0) return;
  const double v = key_sqrt(keys[2 * l] > keys[2 * l + 1] ? keys[2 * l] : keys[2 * l + 1]);
  iters[l] = *itc;
  if (flags[l] || info[l] != 0) {
    if (info[l] == 0) info[l] = BT_ERR_NONFINITE;
    active[l] = 0;
  } else if (v <= tol * ref[l]) {
    active[l] = 0;
  } else {
    atomicAdd(n_active, 1);
  }
}

// Graph mode: iteration counter and loop condition (continue while leads are active and the
// iteration cap is not reached).  One thread.
__global__ void loop_ctl_kernel(cudaGraphConditionalHandle h, const int* __restrict__ n_active, int* itc, int maxit) {
  const int it = *itc;
  *itc = it + 1;
  cudaGraphSetConditional(h, (*n_active > 0 && it < maxit) ? 1u : 0u);
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

__global__ void not_kernel(int batch, const int* __restrict__ a, int* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < batch) out[l] = a[l] ? 0 : 1;
}

// ---- Stein doubling and the Newton polish ----

// problems selected by the mask (all without one) start active, not converged, no iterations
__global__ void stein_init_kernel(int batch, const int* __restrict__ mask, int* active, int* ok, int* iters) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch) return;
  const int on = mask ? (mask[l] != 0) : 1;
  active[l] = on;
  ok[l] = 0;
  if (iters) iters[l] = 0;
}

// convergence test after one doubling step: the next increment A X B is bounded by
// bs^2 max|A| max|X| max|B|, so problem l is done once bs^2 max|A| max|B| <= tol
__device__ __forceinline__ void stein_test(int l, const unsigned long long* keys, const int* flags, double bs2,
                                           double tol, int it, int* active, int* ok, int* iters, int* n_active) {
  if (iters) iters[l] = it;
  if (flags[l]) {
    active[l] = 0;  // non-finite: no correction
  } else if (key_sqrt(keys[2 * l]) * key_sqrt(keys[2 * l + 1]) * bs2 <= tol) {
    active[l] = 0;
    ok[l] = 1;
  } else {
    atomicAdd(n_active, 1);
  }
}

__global__ void stein_check_kernel(int batch, const unsigned long long* __restrict__ keys, const int* __restrict__ flags,
                                   double bs2, double tol, int it, int* __restrict__ active, int* __restrict__ ok,
                                   int* __restrict__ iters, int* __restrict__ n_active) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch || active[l] == 0) return;
  stein_test(l, keys, flags, bs2, tol, it, active, ok, iters, n_active);
}

// graph mode: the iteration number comes from the device counter
__global__ void stein_check_dev_kernel(int batch, const unsigned long long* __restrict__ keys,
                                       const int* __restrict__ flags, double bs2, double tol,
                                       const int* __restrict__ itc, int* __restrict__ active, int* __restrict__ ok,
                                       int* __restrict__ iters, int* __restrict__ n_active) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch || active[l] == 0) return;
  stein_test(l, keys, flags, bs2, tol, *itc, active, ok, iters, n_active);
}

// leads to polish: selected by the decimation mask, decimated without error, and with more than
// `after` iterations
__global__ void polish_mask_kernel(int batch, const int* __restrict__ mask, const int* __restrict__ iters,
                                   const int* __restrict__ info, int after, int* __restrict__ pm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= batch) return;
  pm[l] = (mask ? mask[l] != 0 : 1) && info[l] == 0 && iters[l] > after;
}

// X = m - es - t (the residual r of the Newton step, t = n x n') for selected leads
__global__ void residual_kernel(long long bs2, const zd* __restrict__ m, const zd* __restrict__ es,
                                const zd* __restrict__ t, zd* __restrict__ X, const int* __restrict__ sel) {
  const int l = blockIdx.y;
  if (sel[l] == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)l * bs2 + i;
    X[o] = zsub(zsub(m[o], es[o]), t[o]);
  }
}

// es += X for leads whose doubling converged
__global__ void add_masked_kernel(long long bs2, zd* __restrict__ es, const zd* __restrict__ X,
                                  const int* __restrict__ sel) {
  const int l = blockIdx.y;
  if (sel[l] == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)l * bs2 + i;
    es[o] = zadd(es[o], X[o]);
  }
}

struct SteinWs {
  zd *T, *A2, *B2;
  unsigned long long* keys;
  int* flags;
  int* active;
  int* n_active;
  int* itc;
};

struct DecimWs {
  zd *a, *b, *a2, *b2, *e, *es, *g, *ag, *bg, *t;
  double* ref;
  unsigned long long* keys;
  int* flags;
  int* active;
  int* n_active;
  int* itc;  // graph mode: iteration counter
  int* pm;   // Newton polish: leads selected
  int* ok;   // Newton polish: leads whose doubling converged
  int* itc2; // graph mode: iteration counter of the polish loop
  void* inv_ws;
  size_t inv_bytes;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t carve(void* base, int bs, int batch, bool wide, DecimWs* w) {
  const size_t mat = align256((size_t)batch * bs * bs * sizeof(zd));
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) { char* q = p ? p + off : nullptr; off += align256(bytes); return q; };
  zd** mats[] = {&w->a, &w->b, &w->a2, &w->b2, &w->e, &w->es, &w->g, &w->ag, &w->bg, &w->t};
  for (zd** m : mats) *m = reinterpret_cast<zd*>(take(mat));
  w->ref = reinterpret_cast<double*>(take(sizeof(double) * batch));
  w->keys = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * 2 * batch));
  w->flags = reinterpret_cast<int*>(take(sizeof(int) * batch));
  w->active = reinterpret_cast<int*>(take(sizeof(int) * batch));
  w->n_active = reinterpret_cast<int*>(take(sizeof(int)));
  w->itc = reinterpret_cast<int*>(take(sizeof(int)));
  w->pm = reinterpret_cast<int*>(take(sizeof(int) * batch));
  w->ok = reinterpret_cast<int*>(take(sizeof(int) * batch));
  w->itc2 = reinterpret_cast<int*>(take(sizeof(int)));
  w->inv_bytes = zinv_workspace_bytes(bs, batch, wide);
  w->inv_ws = take(w->inv_bytes);
  return off;
}

// One decimation iteration on the active leads.  With `fixed` the new a, b are copied back into
// w.a, w.b (the buffers stay where a captured graph expects them); otherwise the buffers swap.
bt_status decimate_step(cudaStream_t st, int bs, int batch, DecimWs& w, int* info, const Engine& E, bool fixed) {
  const long long bs2 = (long long)bs * bs, S = bs2;
  const size_t mat_bytes = (size_t)batch * bs2 * sizeof(zd);
  const zd one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0), zero = zmake(0.0, 0.0);
  BT_CUDA_TRY(cudaMemcpyAsync(w.g, w.e, mat_bytes, cudaMemcpyDeviceToDevice, st));
  BT_TRY(zinv(st, bs, w.g, S, batch, info, w.inv_ws, w.inv_bytes, w.active, &E));
  // ag = a g, bg = b g
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{w.a, bs, S, BT_OP_N}, Operand{w.g, bs, S, BT_OP_N}, zero, w.ag, bs, S, batch, w.active));
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{w.b, bs, S, BT_OP_N}, Operand{w.g, bs, S, BT_OP_N}, zero, w.bg, bs, S, batch, w.active));
  // t = a g b; es -= t; e -= t
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{w.ag, bs, S, BT_OP_N}, Operand{w.b, bs, S, BT_OP_N}, zero, w.t, bs, S, batch, w.active));
  {
    dim3 g((unsigned)((bs2 + 255) / 256 < 64 ? (bs2 + 255) / 256 : 64), batch);
    sub2_kernel<<<g, 256, 0, st>>>(bs2, batch, w.t, w.es, w.e, w.active); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
  }
  // e -= b g a
  BT_TRY(gemm(E, st, bs, bs, bs, mone, Operand{w.bg, bs, S, BT_OP_N}, Operand{w.a, bs, S, BT_OP_N}, one, w.e, bs, S, batch, w.active));
  // a2 = -a g a, b2 = -b g b
  BT_TRY(gemm(E, st, bs, bs, bs, mone, Operand{w.ag, bs, S, BT_OP_N}, Operand{w.a, bs, S, BT_OP_N}, zero, w.a2, bs, S, batch, w.active));
  BT_TRY(gemm(E, st, bs, bs, bs, mone, Operand{w.bg, bs, S, BT_OP_N}, Operand{w.b, bs, S, BT_OP_N}, zero, w.b2, bs, S, batch, w.active));
  if (fixed) {
    BT_CUDA_TRY(cudaMemcpyAsync(w.a, w.a2, mat_bytes, cudaMemcpyDeviceToDevice, st));
    BT_CUDA_TRY(cudaMemcpyAsync(w.b, w.b2, mat_bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    std::swap(w.a, w.a2);
    std::swap(w.b, w.b2);
  }
  BT_CUDA_TRY(cudaMemsetAsync(w.n_active, 0, sizeof(int), st));
  BT_TRY(lead_max(st, 0, bs2, batch, w.a, w.b, w.active, w.keys, w.flags));
  return BT_OK;
}

// Graph mode: a loop as a conditional while node of the graph being captured on st.  The body
// (one iteration, ending with a kernel that sets the loop condition through the handle) is
// recorded by body(bst, handle) on the loop's body stream; the body runs at least once.
template <class Body>
bt_status while_node(cudaStream_t st, LoopCapture& loop, long long* body_launches, Body body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  BT_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  if (cs != cudaStreamCaptureStatusActive || !g) return BT_ERR_INVALID_ARG;
  cudaGraphConditionalHandle h;
  BT_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  // the parameter union has no default constructor: zeroed storage, fields set by name
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  std::memset(pbuf, 0, sizeof(pbuf));
  cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(pbuf);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  BT_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p));
  BT_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  cudaStream_t bst = loop.body_stream;
  BT_CUDA_TRY(cudaStreamBeginCaptureToGraph(bst, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const long long l0 = launches_total();
  bt_status rc = body(bst, h);
  if (rc == BT_OK && cudaGetLastError() != cudaSuccess) rc = BT_ERR_CUDA;
  if (body_launches) *body_launches = launches_total() - l0;
  cudaGraph_t got = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(bst, &got);
  if (rc != BT_OK) return rc;
  return ce == cudaSuccess ? BT_OK : BT_ERR_CUDA;
}

// Graph mode: the decimation loop as a conditional while node.
bt_status decimate_loop_graph(cudaStream_t st, LoopCapture& loop, int bs, int batch, double tol, int maxit,
                              DecimWs& w, int* iters, int* info, const Engine& E) {
  set_int_kernel<<<1, 1, 0, st>>>(w.itc, 1); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return while_node(st, loop, &loop.body_launches, [&](cudaStream_t bst, cudaGraphConditionalHandle h) {
    BT_TRY(decimate_step(bst, bs, batch, w, info, E, true));
    check_dev_kernel<<<(batch + 255) / 256, 256, 0, bst>>>(batch, w.keys, w.flags, w.ref, tol, w.itc, w.active, iters,
                                                           info, w.n_active); count_launch();
    loop_ctl_kernel<<<1, 1, 0, bst>>>(h, w.n_active, w.itc, maxit); count_launch();
    return BT_OK;
  });
}

// One doubling step of X = R + A X B on the active problems: X += (A X) B, then A <- A A and
// B <- B B (B = A^H when herm).  With `fixed` the squares are copied back into A, B (the buffers
// stay where a captured graph expects them); otherwise the pointers swap.  Ends with the
// max-|.| reduction of the new A, B.
bt_status stein_step(cudaStream_t st, int bs, int batch, zd*& A, zd*& B, bool herm, zd* X, SteinWs& w,
                     const Engine& E, bool fixed) {
  const long long bs2 = (long long)bs * bs, S = bs2;
  const size_t mat_bytes = (size_t)batch * bs2 * sizeof(zd);
  const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{A, bs, S, BT_OP_N}, Operand{X, bs, S, BT_OP_N}, zero, w.T, bs, S, batch, w.active));
  const Operand opB = herm ? Operand{A, bs, S, BT_OP_C} : Operand{B, bs, S, BT_OP_N};
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{w.T, bs, S, BT_OP_N}, opB, one, X, bs, S, batch, w.active));
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{A, bs, S, BT_OP_N}, Operand{A, bs, S, BT_OP_N}, zero, w.A2, bs, S, batch, w.active));
  if (!herm)
    BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{B, bs, S, BT_OP_N}, Operand{B, bs, S, BT_OP_N}, zero, w.B2, bs, S, batch, w.active));
  if (fixed) {
    BT_CUDA_TRY(cudaMemcpyAsync(A, w.A2, mat_bytes, cudaMemcpyDeviceToDevice, st));
    if (!herm) BT_CUDA_TRY(cudaMemcpyAsync(B, w.B2, mat_bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    std::swap(A, w.A2);
    if (!herm) std::swap(B, w.B2);
  }
  BT_CUDA_TRY(cudaMemsetAsync(w.n_active, 0, sizeof(int), st));
  return lead_max(st, 0, bs2, batch, A, herm ? A : B, w.active, w.keys, w.flags);
}

// The doubling loop: direct (one read-back of the active count per step) or, with `loop`, a
// conditional while node.  ok[l] = 1 where problem l converged.  The swapped buffers of the
// direct loop leave A, B pointing at either copy: their contents are scratch afterwards.
bt_status stein_loop(cudaStream_t st, int bs, int batch, zd* A, zd* B, bool herm, zd* X, double tol, int maxit,
                     const int* mask, int* ok, int* iters, SteinWs& w, int* h_pinned, long long* lead_iterations,
                     const Engine& E, LoopCapture* loop, long long* body_launches, int* n_selected = nullptr) {
  const double bs2 = (double)bs * bs;
  stein_init_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, mask, w.active, ok, iters); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  if (loop) {
    set_int_kernel<<<1, 1, 0, st>>>(w.itc, 1); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
    return while_node(st, *loop, body_launches, [&](cudaStream_t bst, cudaGraphConditionalHandle h) {
      zd *a = A, *b = B;
      BT_TRY(stein_step(bst, bs, batch, a, b, herm, X, w, E, true));
      stein_check_dev_kernel<<<(batch + 255) / 256, 256, 0, bst>>>(batch, w.keys, w.flags, bs2, tol, w.itc, w.active,
                                                                   ok, iters, w.n_active); count_launch();
      loop_ctl_kernel<<<1, 1, 0, bst>>>(h, w.n_active, w.itc, maxit); count_launch();
      return BT_OK;
    });
  }
  int running = batch;
  if (mask) {
    std::vector<int> hm(batch);
    if (cudaMemcpyAsync(hm.data(), mask, sizeof(int) * batch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return BT_ERR_CUDA;
    running = 0;
    for (int v : hm) running += v != 0;
  }
  if (n_selected) *n_selected = running;
  long long its = 0;
  zd *a = A, *b = B;
  SteinWs ws = w;  // the direct loop swaps buffers; the caller's struct keeps its pointers
  for (int it = 1; it <= maxit && running > 0; ++it) {
    its += running;
    BT_TRY(stein_step(st, bs, batch, a, b, herm, X, ws, E, false));
    stein_check_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, ws.keys, ws.flags, bs2, tol, it, ws.active, ok,
                                                            iters, ws.n_active); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
    BT_CUDA_TRY(cudaMemcpyAsync(h_pinned, ws.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_CUDA_TRY(cudaStreamSynchronize(st));
    running = *h_pinned;
  }
  if (lead_iterations) *lead_iterations = its;
  return BT_OK;
}

// Newton step on the decimated leads with more than pol.after iterations (see the file header).
// On entry x = e_s^{-1} for every decimated lead; on return x and e_s are corrected where the
// doubling converged.
constexpr double kPolishTol = 1e-12;  // relative size of the neglected doubling terms
constexpr int kPolishMaxit = 64;
bt_status polish_step(cudaStream_t st, int bs, int batch, const zd* m, const zd* n, const zd* np, zd* x,
                      const int* mask, const int* iters, int* info, DecimWs& w, int* h_pinned, const Engine& E,
                      LoopCapture* loop, Polish& pol) {
  const long long bs2 = (long long)bs * bs, S = bs2;
  const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
  polish_mask_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, mask, iters, info, pol.after, w.pm); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  // A = n x, B = x n', t = A n' = n x n', residual X = m - e_s - t
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{n, bs, S, BT_OP_N}, Operand{x, bs, S, BT_OP_N}, zero, w.a, bs, S, batch, w.pm));
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{x, bs, S, BT_OP_N}, Operand{np, bs, S, BT_OP_N}, zero, w.b, bs, S, batch, w.pm));
  BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{w.a, bs, S, BT_OP_N}, Operand{np, bs, S, BT_OP_N}, zero, w.t, bs, S, batch, w.pm));
  dim3 g((unsigned)((bs2 + 255) / 256 < 64 ? (bs2 + 255) / 256 : 64), batch);
  residual_kernel<<<g, 256, 0, st>>>(bs2, m, w.es, w.t, w.g, w.pm); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  SteinWs sw{w.ag, w.a2, w.b2, w.keys, w.flags, w.active, w.n_active, w.itc2};
  BT_TRY(stein_loop(st, bs, batch, w.a, w.b, false, w.g, kPolishTol, kPolishMaxit, w.pm, w.ok, pol.iters, sw, h_pinned,
                    &pol.lead_iterations, E, loop, &pol.body_launches, &pol.selected));
  // e_s += d, x = e_s^{-1} where the doubling converged
  add_masked_kernel<<<g, 256, 0, st>>>(bs2, w.es, w.g, w.ok); count_launch();
  masked_copy_kernel<<<g, 256, 0, st>>>(bs2, w.es, x, w.ok); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return zinv(st, bs, x, S, batch, info, w.inv_ws, w.inv_bytes, w.ok, &E);
}

// Direct mode: host-driven loop, one convergence read-back per iteration.
bt_status decimate_loop_host(cudaStream_t st, int bs, int batch, double tol, int maxit, DecimWs& w, int* iters,
                             int* info, const Engine& E, const int* mask, int* h_pinned, int* iters_host_max,
                             long long* lead_iterations) {
  int* h_active = h_pinned;
  if (!h_active) BT_CUDA_TRY(cudaMallocHost(&h_active, sizeof(int)));
  int it = 0;
  long long lead_its = 0;
  int running = batch;  // leads entering the next iteration (upper bound before the first test)
  bt_status rc = BT_OK;
  if (mask) {
    // count the masked-in leads so a fully memoized chunk runs no iteration at all
    std::vector<int> hm(batch);
    if (cudaMemsetAsync(w.n_active, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemcpyAsync(hm.data(), mask, sizeof(int) * batch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = BT_ERR_CUDA;
    running = 0;
    for (int v : hm) running += v != 0;
  }
  for (it = 1; rc == BT_OK && it <= maxit && running > 0; ++it) {
    lead_its += running;
    if ((rc = decimate_step(st, bs, batch, w, info, E, false)) != BT_OK) break;
    check_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, w.keys, w.flags, w.ref, tol, it, w.active, iters, info,
                                                      w.n_active); count_launch();
    if (cudaGetLastError() != cudaSuccess) { rc = BT_ERR_CUDA; break; }
    if (cudaMemcpyAsync(h_active, w.n_active, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) { rc = BT_ERR_CUDA; break; }
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = BT_ERR_CUDA; break; }
    running = *h_active;
    if (running == 0) break;
  }
  if (!h_pinned) cudaFreeHost(h_active);
  if (rc != BT_OK) return rc;
  if (iters_host_max) *iters_host_max = it > maxit ? maxit : (it > 0 ? it : 0);
  if (lead_iterations) *lead_iterations = lead_its;
  return BT_OK;
}

}  // namespace

size_t decimate_workspace_bytes(int bs, int batch, bool wide) {
  DecimWs w;
  return carve(nullptr, bs, batch, wide, &w);
}

bt_status decimate(cudaStream_t st, int bs, int batch, const zd* m, const zd* n, const zd* np, double tol,
                   int maxit, zd* x, zd* sigma, int* iters, int* info, void* ws, size_t ws_bytes,
                   int* iters_host_max, int* h_pinned, const int* mask, long long* lead_iterations,
                   const Engine* eng, LoopCapture* loop, Polish* polish) {
  const Engine fp64;
  const Engine& E = eng ? *eng : fp64;
  if (bs <= 0 || batch <= 0 || maxit <= 0 || batch > 65535) return BT_ERR_INVALID_ARG;
  if (loop && (mask || !loop->body_stream)) return BT_ERR_INVALID_ARG;
  // wide inversion panels when the products run sliced and the workspace was sized for them
  const bool wide = E.slices > 0 && ws_bytes >= decimate_workspace_bytes(bs, batch, true);
  if (!ws || ws_bytes < decimate_workspace_bytes(bs, batch, wide)) return BT_ERR_INVALID_ARG;
  DecimWs w;
  carve(ws, bs, batch, wide, &w);
  const long long bs2 = (long long)bs * bs;
  const size_t mat_bytes = (size_t)batch * bs2 * sizeof(zd);
  BT_CUDA_TRY(cudaMemcpyAsync(w.a, n, mat_bytes, cudaMemcpyDeviceToDevice, st));
  BT_CUDA_TRY(cudaMemcpyAsync(w.b, np, mat_bytes, cudaMemcpyDeviceToDevice, st));
  BT_CUDA_TRY(cudaMemcpyAsync(w.e, m, mat_bytes, cudaMemcpyDeviceToDevice, st));
  BT_CUDA_TRY(cudaMemcpyAsync(w.es, m, mat_bytes, cudaMemcpyDeviceToDevice, st));
  init_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, mask, w.active, iters, info); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  BT_TRY(lead_max(st, 0, bs2, batch, n, np, nullptr, w.keys, w.flags));
  ref_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, w.keys, w.ref); count_launch();
  BT_CUDA_TRY(cudaGetLastError());

  if (loop) {
    BT_TRY(decimate_loop_graph(st, *loop, bs, batch, tol, maxit, w, iters, info, E));
  } else {
    BT_TRY(decimate_loop_host(st, bs, batch, tol, maxit, w, iters, info, E, mask, h_pinned, iters_host_max,
                              lead_iterations));
  }
  finish_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, w.active, info); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  // x = e_s^{-1} (decimated leads);  sigma = n x n'
  {
    dim3 g((unsigned)((bs2 + 255) / 256 < 64 ? (bs2 + 255) / 256 : 64), batch);
    masked_copy_kernel<<<g, 256, 0, st>>>(bs2, w.es, x, mask); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
  }
  const long long S = bs2;
  const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
  BT_TRY(zinv(st, bs, x, S, batch, info, w.inv_ws, w.inv_bytes, mask, &E));
  if (polish && polish->after >= 0) {
    int* hp = h_pinned;
    if (!loop && !hp && cudaMallocHost(&hp, 64) != cudaSuccess) return BT_ERR_CUDA;
    // the step's products run on polish->engine: FP64, or sliced with 8 slices when the
    // decimation's products are sliced (its residual then limits the step at ~1e-9 relative,
    // well inside the split path's tolerance, for a twentieth of the FP64 cost)
    const Engine fp64_step;
    const Engine& PE = polish->engine ? *polish->engine : fp64_step;
    const bt_status ps = polish_step(st, bs, batch, m, n, np, x, mask, iters, info, w, hp, PE, loop, *polish);
    if (hp != h_pinned) cudaFreeHost(hp);
    BT_TRY(ps);
  }
  if (sigma) {
    BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{n, bs, S, BT_OP_N}, Operand{x, bs, S, BT_OP_N}, zero, w.t, bs, S, batch, nullptr));
    BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{w.t, bs, S, BT_OP_N}, Operand{np, bs, S, BT_OP_N}, zero, sigma, bs, S, batch, nullptr));
  }
  return BT_OK;
}


size_t stein_workspace_bytes(int bs, int batch) {
  const size_t mat = align256((size_t)batch * bs * bs * sizeof(zd));
  return 3 * mat + align256(sizeof(unsigned long long) * 2 * batch) + 2 * align256(sizeof(int) * batch) +
         2 * align256(sizeof(int));
}

bt_status stein(cudaStream_t st, int bs, int batch, zd* A, zd* B, zd* X, double tol, int maxit, const int* mask,
                int* ok, int* iters, void* ws, size_t ws_bytes, int* h_pinned, long long* lead_iterations,
                const Engine* eng, LoopCapture* loop, long long* body_launches) {
  const Engine fp64;
  const Engine& E = eng ? *eng : fp64;
  if (bs <= 0 || batch <= 0 || batch > 65535 || maxit <= 0 || !A || !X || !ok) return BT_ERR_INVALID_ARG;
  if (!ws || ws_bytes < stein_workspace_bytes(bs, batch)) return BT_ERR_INVALID_ARG;
  if (!loop && !h_pinned) return BT_ERR_INVALID_ARG;
  const size_t mat = align256((size_t)batch * bs * bs * sizeof(zd));
  char* p = static_cast<char*>(ws);
  SteinWs w;
  w.T = reinterpret_cast<zd*>(p); p += mat;
  w.A2 = reinterpret_cast<zd*>(p); p += mat;
  w.B2 = reinterpret_cast<zd*>(p); p += mat;
  w.keys = reinterpret_cast<unsigned long long*>(p); p += align256(sizeof(unsigned long long) * 2 * batch);
  w.flags = reinterpret_cast<int*>(p); p += align256(sizeof(int) * batch);
  w.active = reinterpret_cast<int*>(p); p += align256(sizeof(int) * batch);
  w.n_active = reinterpret_cast<int*>(p); p += align256(sizeof(int));
  w.itc = reinterpret_cast<int*>(p);
  long long body = 0;
  BT_TRY(stein_loop(st, bs, batch, A, B, B == nullptr, X, tol, maxit, mask, ok, iters, w, h_pinned, lead_iterations,
                    E, loop, &body));
  if (body_launches) *body_launches = body;
  return BT_OK;
}

__global__ void status_from_ok_kernel(int batch, const int* __restrict__ ok, const int* __restrict__ mask, int code,
                                      int* __restrict__ info) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < batch) info[l] = (mask && mask[l] == 0) || ok[l] ? 0 : code;
}

bt_status status_from_ok(cudaStream_t st, int batch, const int* ok, const int* mask, int code, int* info) {
  status_from_ok_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, ok, mask, code, info);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status invert_mask(cudaStream_t st, int batch, const int* a, int* out) {
  not_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, a, out);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status fixed_point(cudaStream_t st, int bs, int batch, const zd* m, const zd* n, const zd* np, zd* x,
                      const int* run, int* conv, int nfpi, double tol, int* info, void* ws, size_t ws_bytes,
                      int* h_pinned, long long* lead_iterations, const Engine* eng) {
  const Engine fp64;
  const Engine& E = eng ? *eng : fp64;
  if (bs <= 0 || batch <= 0 || batch > 65535) return BT_ERR_INVALID_ARG;
  // wide inversion panels when the products run sliced and the workspace was sized for them
  const bool wide = E.slices > 0 && ws_bytes >= decimate_workspace_bytes(bs, batch, true);
  if (!ws || ws_bytes < decimate_workspace_bytes(bs, batch, wide)) return BT_ERR_INVALID_ARG;
  DecimWs w;
  carve(ws, bs, batch, wide, &w);
  const long long bs2 = (long long)bs * bs;
  const size_t mat_bytes = (size_t)batch * bs2 * sizeof(zd);
  const long long S = bs2;
  const zd one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0), zero = zmake(0.0, 0.0);
  BT_CUDA_TRY(cudaMemsetAsync(conv, 0, sizeof(int) * batch, st));
  BT_CUDA_TRY(cudaMemcpyAsync(w.active, run, sizeof(int) * batch, cudaMemcpyDeviceToDevice, st));
  BT_CUDA_TRY(cudaMemsetAsync(w.ref, 0, sizeof(double) * batch, st));  // previous update sizes
  std::vector<int> hm(batch);
  if (cudaMemcpyAsync(hm.data(), run, sizeof(int) * batch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BT_ERR_CUDA;
  int running = 0;
  for (int v : hm) running += v != 0;
  long long lead_its = 0;
  dim3 gcopy((unsigned)((bs2 + 255) / 256 < 64 ? (bs2 + 255) / 256 : 64), batch);
  for (int it = 1; it <= nfpi && running > 0; ++it) {
    lead_its += running;
    // x_new = (m - n x n')^{-1}   (Eq. 5)
    BT_TRY(gemm(E, st, bs, bs, bs, one, Operand{n, bs, S, BT_OP_N}, Operand{x, bs, S, BT_OP_N}, zero, w.t, bs, S, batch, w.active));
    BT_CUDA_TRY(cudaMemcpyAsync(w.g, m, mat_bytes, cudaMemcpyDeviceToDevice, st));
    BT_TRY(gemm(E, st, bs, bs, bs, mone, Operand{w.t, bs, S, BT_OP_N}, Operand{np, bs, S, BT_OP_N}, one, w.g, bs, S, batch, w.active));
    BT_TRY(zinv(st, bs, w.g, S, batch, info, w.inv_ws, w.inv_bytes, w.active, &E));
    // the test reads the current mask; copy x_new -> x for the leads still iterating first
    masked_copy_kernel<<<gcopy, 256, 0, st>>>(bs2, x, w.e, w.active); count_launch();  // keep x_k
    masked_copy_kernel<<<gcopy, 256, 0, st>>>(bs2, w.g, x, w.active); count_launch();
    BT_CUDA_TRY(cudaMemsetAsync(w.n_active, 0, sizeof(int), st));
    BT_TRY(lead_max(st, 1, bs2, batch, x, w.e, w.active, w.keys, w.flags));
    fpi_check_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, w.keys, w.flags, tol, it, nfpi, w.active, conv, w.ref,
                                                          w.n_active); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
    BT_CUDA_TRY(cudaMemcpyAsync(h_pinned, w.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_CUDA_TRY(cudaStreamSynchronize(st));
    running = *h_pinned;
  }
  if (lead_iterations) *lead_iterations = lead_its;
  return BT_OK;
}

}  // namespace bt

extern "C" bt_status bt_decimate_workspace_bytes(int bs, int batch, size_t* bytes) {
  if (!bytes || bs <= 0 || batch <= 0) return BT_ERR_INVALID_ARG;
  *bytes = bt::decimate_workspace_bytes(bs, batch, false);
  return BT_OK;
}

extern "C" bt_status bt_decimate_batched(int bs, int batch, const void* m, const void* n, const void* n_prime,
                                         double tol, int maxit, void* x, void* sigma, int* iters_device,
                                         int* info_device, void* workspace, size_t workspace_bytes, void* stream) {
  if (!m || !n || !n_prime || !x || !iters_device || !info_device) return BT_ERR_INVALID_ARG;
  if (!(tol > 0.0)) tol = 1e-14;
  if (maxit <= 0) maxit = 100;
  bt::Polish pol;
  pol.after = 14;  // leads with more decimation iterations get the Newton step
  return bt::decimate(static_cast<cudaStream_t>(stream), bs, batch, static_cast<const zd*>(m),
                      static_cast<const zd*>(n), static_cast<const zd*>(n_prime), tol, maxit, static_cast<zd*>(x),
                      static_cast<zd*>(sigma), iters_device, info_device, workspace, workspace_bytes, nullptr, nullptr,
                      nullptr, nullptr, nullptr, nullptr, &pol);
}
