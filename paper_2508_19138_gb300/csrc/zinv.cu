// Batched in-place inversion of complex128 blocks: the x^R_i = (Schur complement)^{-1} of the
// RGF forward pass (Sec. 3.2.2, Eq. 8) and the g = e^{-1} of the decimation (Eq. 4).
//
// Algorithm: Gauss-Jordan elimination with partial (row) pivoting, i.e. the block LU of the
// pivot column carried to the full inverse in one sweep.  Pivot = max |re| + |im| over the
// not-yet-pivoted rows of the current column, first index on ties (LAPACK's izamax rule); the
// pivot sequence is the one LU with partial pivoting picks.  Row exchanges are undone at the
// end as column exchanges in reverse order.
//
//  * n <= kSmallN: one CTA per matrix, the whole matrix resident in shared memory.
//  * larger n: blocked.  For each panel of kb columns one CTA per matrix eliminates the n x kb
//    panel in shared memory (all rows, pivots searched in rows >= j); the remaining columns
//    then receive the panel's row exchanges and the rank-kb update
//        A[:, C] += P[:, K] * A_old[K, C]   (rows K of C zeroed first)
//    as one batched FP64 GEMM, so the O(n^3) part runs on the GEMM kernel.
#include <cooperative_groups.h>

#include <mutex>

#include "bt_common.cuh"

namespace bt {
namespace {

constexpr int kSmallN = 96;
constexpr int NT = 256;
constexpr size_t kSmemLimit = 227 * 1024;

// block-wide argmax of v over threads (ties -> smaller index); result broadcast
__device__ __forceinline__ void block_argmax(double& v, int& idx, double* sv, int* si) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, v, off);
    int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[w] = v; si[w] = idx; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? sv[lane] : -1.0;
    idx = lane < nw ? si[lane] : 0x7fffffff;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, v, off);
      int oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) { sv[0] = v; si[0] = idx; }
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  __syncthreads();
}

__device__ __forceinline__ int pivot_code(zd piv) {
  if (!isfinite(piv.x) || !isfinite(piv.y)) return BT_ERR_NONFINITE;
  if (piv.x == 0.0 && piv.y == 0.0) return BT_ERR_SINGULAR;
  return 0;
}

// One Gauss-Jordan step on a row-major panel P (rows 0..n-1, columns 0..kb-1, leading
// dimension ld) in shared memory, pivot column jj, pivot row searched in rows >= j.
// Returns the pivot row; *code gets a failure code (thread 0 view).
__device__ int gj_step(zd* P, int n, int kb, int ld, int j, int jj, zd* colj, zd* rowj, double* sv, int* si,
                       int* code) {
  // pivot search
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int r = j + threadIdx.x; r < n; r += blockDim.x) {
    double v = zabs1(P[r * ld + jj]);
    if (!(v <= 1.0e308)) v = 1.0e308;  // NaN / Inf: still a candidate, flagged below
    if (v > best) { best = v; bi = r; }
  }
  block_argmax(best, bi, sv, si);
  const int p = bi;
  if (p != j) {
    for (int c = threadIdx.x; c < kb; c += blockDim.x) {
      zd t = P[j * ld + c];
      P[j * ld + c] = P[p * ld + c];
      P[p * ld + c] = t;
    }
  }
  __syncthreads();
  const zd piv = P[j * ld + jj];
  const int pc = pivot_code(piv);
  if (pc && threadIdx.x == 0 && *code == 0) *code = pc;
  const zd ip = pc ? zmake(0.0, 0.0) : zinv(piv);
  for (int r = threadIdx.x; r < n; r += blockDim.x) colj[r] = P[r * ld + jj];
  for (int c = threadIdx.x; c < kb; c += blockDim.x) rowj[c] = zmul(P[j * ld + c], ip);
  __syncthreads();
  const int total = n * kb;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    zd* pe = P + r * ld + c;
    if (r == j) {
      *pe = (c == jj) ? ip : rowj[c];
    } else if (c == jj) {
      *pe = zmul(zmake(-colj[r].x, -colj[r].y), ip);
    } else {
      zd a = *pe;
      const zd f = colj[r], g = rowj[c];
      a.x = fma(-f.x, g.x, a.x);
      a.x = fma(f.y, g.y, a.x);
      a.y = fma(-f.x, g.y, a.y);
      a.y = fma(-f.y, g.x, a.y);
      *pe = a;
    }
  }
  __syncthreads();
  return p;
}

// Whole matrix in shared memory (n <= kSmallN).
__global__ void __launch_bounds__(NT) zinv_small_kernel(int n, zd* __restrict__ A, long long sA, int* info,
                                                        const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (active && active[b] == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = n + 1;
  zd* P = reinterpret_cast<zd*>(smem_raw);
  zd* colj = P + n * ld;
  zd* rowj = colj + n;
  int* perm = reinterpret_cast<int*>(rowj + n);
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int code;
  zd* Ag = A + sA * b;
  if (threadIdx.x == 0) code = 0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) P[(e / n) * ld + (e % n)] = Ag[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    int p = gj_step(P, n, n, ld, j, j, colj, rowj, sv, si, &code);
    if (threadIdx.x == 0) perm[j] = p;
  }
  __syncthreads();
  // undo the row exchanges as column exchanges, last first
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    for (int j = n - 1; j >= 0; --j) {
      const int p = perm[j];
      if (p != j) {
        zd t = P[r * ld + j];
        P[r * ld + j] = P[r * ld + p];
        P[r * ld + p] = t;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ag[e] = P[(e / n) * ld + (e % n)];
  if (threadIdx.x == 0 && code && info && info[b] == 0) info[b] = code;
}

// Panel of kb columns eliminated by a cluster of CL CTAs: CTA r of the cluster holds rows
// [r R, r R + R) of the panel in its shared memory (R = ceil(n / CL)), so the panel's FP64
// updates use CL SMs instead of one.  Per column: each CTA proposes its best pivot candidate,
// all CTAs read every candidate through distributed shared memory and agree on the same pivot
// (max |re| + |im|, first index on ties), read the pivot row and exchange rows j and p through
// DSMEM, then update their own rows.  Two cluster barriers per column; no spin-waits.
template <int CL>
__global__ void __launch_bounds__(NT) gj_panel_cluster_kernel(int n, int k0, int kb, zd* __restrict__ A,
                                                              long long sA, int* __restrict__ perm_all, int* info,
                                                              const int* __restrict__ active) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / CL;
  if (active && active[b] == 0) return;  // uniform over the cluster
  const int R = (n + CL - 1) / CL;
  const int r0 = rank * R;
  const int rows = max(0, min(R, n - r0));
  const int ld = kb + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zd* P = reinterpret_cast<zd*>(smem_raw);  // [R][ld]
  zd* colj = P + (size_t)R * ld;            // [R]
  zd* rowj = colj + R;                      // [kb]
  zd* pivrow = rowj + kb;                   // [kb]
  zd* swapbuf = pivrow + kb;                // [kb]
  __shared__ double cand_v;
  __shared__ int cand_i;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int code;
  __shared__ int gp;
  zd* Ag = A + sA * b;
  int* perm = perm_all + (long long)n * b;
  if (threadIdx.x == 0) code = 0;
  for (int e = threadIdx.x; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    P[r * ld + c] = Ag[(long long)(r0 + r) * n + k0 + c];
  }
  __syncthreads();
  for (int jj = 0; jj < kb; ++jj) {
    const int j = k0 + jj;
    // local pivot candidate among rows >= j
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      if (r0 + r < j) continue;
      double v = zabs1(P[r * ld + jj]);
      if (!(v <= 1.0e308)) v = 1.0e308;
      if (v > best) { best = v; bi = r0 + r; }
    }
    block_argmax(best, bi, sv, si);
    if (threadIdx.x == 0) { cand_v = best; cand_i = bi; }
    cluster.sync();  // candidates visible
    if (threadIdx.x < 32) {  // lane q reads CTA q's candidate (all remote loads in parallel)
      const int q = threadIdx.x;
      double v = q < CL ? *cluster.map_shared_rank(&cand_v, q) : -1.0;
      int p = q < CL ? *cluster.map_shared_rank(&cand_i, q) : 0x7fffffff;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, off);
        const int oi = __shfl_down_sync(0xffffffffu, p, off);
        if (ov > v || (ov == v && oi < p)) { v = ov; p = oi; }
      }
      if (q == 0) gp = p;
    }
    __syncthreads();
    const int p = gp;
    const int own_p = p / R, own_j = j / R;
    {
      const zd* rp = cluster.map_shared_rank(P, own_p) + (size_t)(p - own_p * R) * ld;
      for (int c = threadIdx.x; c < kb; c += blockDim.x) pivrow[c] = rp[c];
      if (rank == own_p && p != j) {
        const zd* rj = cluster.map_shared_rank(P, own_j) + (size_t)(j - own_j * R) * ld;
        for (int c = threadIdx.x; c < kb; c += blockDim.x) swapbuf[c] = rj[c];
      }
    }
    cluster.sync();  // every read of rows p and j and of the candidates is done
    if (p != j) {
      if (rank == own_j)
        for (int c = threadIdx.x; c < kb; c += blockDim.x) P[(j - r0) * ld + c] = pivrow[c];
      if (rank == own_p)
        for (int c = threadIdx.x; c < kb; c += blockDim.x) P[(p - r0) * ld + c] = swapbuf[c];
    }
    const zd piv = pivrow[jj];
    const int pc = pivot_code(piv);
    if (pc && threadIdx.x == 0 && code == 0) code = pc;
    const zd ip = pc ? zmake(0.0, 0.0) : zinv(piv);
    if (rank == 0 && threadIdx.x == 0) perm[j] = p;
    for (int c = threadIdx.x; c < kb; c += blockDim.x) rowj[c] = zmul(pivrow[c], ip);
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += blockDim.x) colj[r] = P[r * ld + jj];
    __syncthreads();
    for (int e = threadIdx.x; e < rows * kb; e += blockDim.x) {
      const int r = e / kb, c = e - r * kb;
      zd* pe = P + r * ld + c;
      if (r0 + r == j) {
        *pe = (c == jj) ? ip : rowj[c];
      } else if (c == jj) {
        *pe = zmul(zmake(-colj[r].x, -colj[r].y), ip);
      } else {
        zd a = *pe;
        const zd f = colj[r], g = rowj[c];
        a.x = fma(-f.x, g.x, a.x);
        a.x = fma(f.y, g.y, a.x);
        a.y = fma(-f.x, g.y, a.y);
        a.y = fma(-f.y, g.x, a.y);
        *pe = a;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    Ag[(long long)(r0 + r) * n + k0 + c] = P[r * ld + c];
  }
  if (rank == 0 && threadIdx.x == 0 && code && info && info[b] == 0) info[b] = code;
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

constexpr int kPanelCluster = 8;
constexpr int kClusterMinN = 192;  // below this a single CTA holds the panel comfortably
size_t cluster_panel_smem(int n, int kb) {
  const int R = (n + kPanelCluster - 1) / kPanelCluster;
  return (size_t)R * (kb + 1) * sizeof(zd) + (size_t)(R + 3 * kb) * sizeof(zd) + 16;
}

// Panel of kb columns starting at k0: eliminated in shared memory, written back in place.
__global__ void __launch_bounds__(NT) gj_panel_kernel(int n, int k0, int kb, zd* __restrict__ A, long long sA,
                                                      int* __restrict__ perm_all, int* info,
                                                      const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (active && active[b] == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = kb + 1;
  zd* P = reinterpret_cast<zd*>(smem_raw);
  zd* colj = P + n * ld;
  zd* rowj = colj + n;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int code;
  zd* Ag = A + sA * b;
  int* perm = perm_all + (long long)n * b;
  if (threadIdx.x == 0) code = 0;
  for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    P[r * ld + c] = Ag[(long long)r * n + k0 + c];
  }
  __syncthreads();
  for (int jj = 0; jj < kb; ++jj) {
    int p = gj_step(P, n, kb, ld, k0 + jj, jj, colj, rowj, sv, si, &code);
    if (threadIdx.x == 0) perm[k0 + jj] = p;
  }
  for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    Ag[(long long)r * n + k0 + c] = P[r * ld + c];
  }
  if (threadIdx.x == 0 && code && info && info[b] == 0) info[b] = code;
}

// Row exchanges of the panel applied to the columns outside it; rows K copied to T and zeroed.
__global__ void gj_swap_copy_kernel(int n, int k0, int kb, zd* __restrict__ A, long long sA,
                                    const int* __restrict__ perm_all, zd* __restrict__ T, long long sT,
                                    const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && active[b] == 0) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || (c >= k0 && c < k0 + kb)) return;
  zd* Ag = A + sA * b;
  const int* perm = perm_all + (long long)n * b;
  for (int jj = 0; jj < kb; ++jj) {
    const int j = k0 + jj, p = perm[j];
    if (p != j) {
      zd t = Ag[(long long)j * n + c];
      Ag[(long long)j * n + c] = Ag[(long long)p * n + c];
      Ag[(long long)p * n + c] = t;
    }
  }
  zd* Tb = T + sT * b;
  for (int jj = 0; jj < kb; ++jj) {
    Tb[(long long)jj * n + c] = Ag[(long long)(k0 + jj) * n + c];
    Ag[(long long)(k0 + jj) * n + c] = zmake(0.0, 0.0);
  }
}

// Row exchanges undone as column exchanges in reverse order; one thread per row.
__global__ void gj_unscramble_kernel(int n, zd* __restrict__ A, long long sA, const int* __restrict__ perm_all,
                                     const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && active[b] == 0) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  zd* row = A + sA * b + (long long)r * n;
  const int* perm = perm_all + (long long)n * b;
  for (int j = n - 1; j >= 0; --j) {
    const int p = perm[j];
    if (p != j) {
      zd t = row[j];
      row[j] = row[p];
      row[p] = t;
    }
  }
}

int panel_width(int n) {
  // The panel elimination costs ~n kb^2 complex FMAs per panel on ONE SM per matrix (4 n^2 kb
  // DFMA per inverse), the rank-kb updates n^3 on all SMs; kb = 16 balances the two on GB300's
  // slow FP64 pipe (kb = 32 made the panels ~27 % of a split-precision step).
  for (int kb = 16; kb >= 4; kb >>= 1) {
    size_t need = (size_t)n * (kb + 1) * sizeof(zd) + (size_t)(n + kb) * sizeof(zd) + 1024;
    if (need <= kSmemLimit) return kb;
  }
  return 0;
}

size_t small_smem(int n) { return (size_t)n * (n + 1) * sizeof(zd) + 2 * (size_t)n * sizeof(zd) + n * sizeof(int) + 16; }
size_t panel_smem(int n, int kb) { return (size_t)n * (kb + 1) * sizeof(zd) + (size_t)(n + kb) * sizeof(zd) + 16; }

// The dynamic shared-memory limits are per-function device state: set them once per device to
// the largest size any launch uses (setting them per launch races between host threads that
// invert different block sizes concurrently, e.g. the serving workers).
bt_status set_smem_limits() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return BT_OK;
  const int small_max = (int)small_smem(kSmallN);
  const int panel_max = (int)(kSmemLimit - 1024);  // leaves room for the kernels' static shared memory
  if (cudaFuncSetAttribute(zinv_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, small_max) != cudaSuccess ||
      cudaFuncSetAttribute(gj_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_max) != cudaSuccess)
    return BT_ERR_CUDA;
  done[dev] = true;
  return BT_OK;
}

}  // namespace

size_t zinv_workspace_bytes(int n, int batch) {
  if (n <= kSmallN) return 0;
  int kb = panel_width(n);
  if (kb == 0) return 0;
  // perm [batch][n] ints (rounded to 256 B) + T [batch][kb][n] complex
  size_t perm = ((size_t)batch * n * sizeof(int) + 255) / 256 * 256;
  return perm + (size_t)batch * kb * n * sizeof(zd);
}

bt_status zinv(cudaStream_t st, int n, zd* A, long long sA, int batch, int* info, void* ws, size_t ws_bytes,
               const int* active, const Engine* eng) {
  const Engine fp64;
  const Engine& E = eng ? *eng : fp64;
  if (n < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (n == 0 || batch == 0) return BT_OK;
  if (batch > 2147483647 / 2) return BT_ERR_INVALID_ARG;
  BT_TRY(set_smem_limits());
  if (n <= kSmallN) {
    size_t sm = small_smem(n);
    zinv_small_kernel<<<batch, NT, sm, st>>>(n, A, sA, info, active); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
    return BT_OK;
  }
  const int kb = panel_width(n);
  if (kb == 0) return BT_ERR_UNSUPPORTED;
  if (ws_bytes < zinv_workspace_bytes(n, batch) || ws == nullptr) return BT_ERR_INVALID_ARG;
  if (batch > 65535) return BT_ERR_INVALID_ARG;
  int* perm = static_cast<int*>(ws);
  size_t perm_bytes = ((size_t)batch * n * sizeof(int) + 255) / 256 * 256;
  zd* T = reinterpret_cast<zd*>(static_cast<char*>(ws) + perm_bytes);
  const long long sT = (long long)kb * n;
  const bool clustered = n >= kClusterMinN;
  for (int k0 = 0; k0 < n; k0 += kb) {
    const int w = (n - k0) < kb ? (n - k0) : kb;
    if (clustered) {
      // one cluster of kPanelCluster CTAs per matrix (rows of the panel split across SMs)
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(batch * kPanelCluster));
      cfg.blockDim = dim3(NT);
      cfg.dynamicSmemBytes = cluster_panel_smem(n, w);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kPanelCluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      BT_CUDA_TRY(cudaLaunchKernelEx(&cfg, gj_panel_cluster_kernel<kPanelCluster>, n, k0, w, A, sA, perm, info,
                                     active));
      count_launch();
    } else {
      gj_panel_kernel<<<batch, NT, panel_smem(n, w), st>>>(n, k0, w, A, sA, perm, info, active); count_launch();
    }
    BT_CUDA_TRY(cudaGetLastError());
    dim3 g((n + 255) / 256, batch);
    gj_swap_copy_kernel<<<g, 256, 0, st>>>(n, k0, w, A, sA, perm, T, sT, active); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
    // A[:, C] += A[:, K] * T[:, C] for the column ranges left and right of the panel
    Operand P{A + k0, n, sA, BT_OP_N};
    if (k0 > 0) {
      Operand Tl{T, n, sT, BT_OP_N};
      BT_TRY(gemm(E, st, n, k0, w, zmake(1.0, 0.0), P, Tl, zmake(1.0, 0.0), A, n, sA, batch, active));
    }
    const int c1 = k0 + w;
    if (c1 < n) {
      Operand Tr{T + c1, n, sT, BT_OP_N};
      BT_TRY(gemm(E, st, n, n - c1, w, zmake(1.0, 0.0), P, Tr, zmake(1.0, 0.0), A + c1, n, sA, batch, active));
    }
  }
  dim3 g((n + 255) / 256, batch);
  gj_unscramble_kernel<<<g, 256, 0, st>>>(n, A, sA, perm, active); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt

extern "C" bt_status bt_zinv_workspace_bytes(int n, int batch, size_t* bytes) {
  if (!bytes || n < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  *bytes = bt::zinv_workspace_bytes(n, batch);
  return BT_OK;
}

extern "C" bt_status bt_zinv_batched(int n, void* A, long long strideA, int batch, int* info_device, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  if (n < 0 || batch < 0 || (n > 0 && batch > 0 && !A)) return BT_ERR_INVALID_ARG;
  if (batch > 1 && strideA < (long long)n * n) return BT_ERR_INVALID_ARG;
  return bt::zinv(static_cast<cudaStream_t>(stream), n, static_cast<zd*>(A), strideA, batch, info_device, workspace,
                  workspace_bytes, nullptr);
}
