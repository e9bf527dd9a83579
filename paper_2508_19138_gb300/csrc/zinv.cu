// Batched in-place inversion of complex128 blocks: the x^R_i = (Schur complement)^{-1} of the
// RGF forward pass (Sec. 4.3.2, Eq. 9) and the g = e^{-1} of the decimation (Eq. 4).
//
// Algorithm: Gauss-Jordan elimination with partial (row) pivoting, i.e. the block LU of the
// pivot column carried to the full inverse in one sweep.  Pivot = max |re| + |im| over the
// not-yet-pivoted rows of the current column, first index on ties (LAPACK's izamax rule); the
// pivot sequence is the one LU with partial pivoting picks.  Row exchanges are undone at the
// end as column exchanges in reverse order.
//
//  * n <= kSmallN: one CTA per matrix, the whole matrix resident in shared memory.
//  * larger n: blocked.  For each panel of kb columns the n x kb panel is eliminated in shared
//    memory (all rows, pivots searched in rows >= j) — by one CTA per matrix, or for
//    n >= kClusterMinN by a thread-block cluster per matrix with the rows split across its
//    SMs; the remaining columns then receive the panel's row exchanges and the rank-kb update
//        A[:, C] += P[:, K] * A_old[K, C]   (rows K of C zeroed first)
//    as one batched GEMM (FP64, or sliced on the tensor cores), so the O(n^3) part runs on
//    the GEMM kernels.
#include <cooperative_groups.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "bt_common.cuh"

namespace bt {
namespace {

constexpr int kSmallN = 96;
constexpr int kClusterMinN = 192;  // below this a single CTA holds the panel comfortably
constexpr int NT = 256;
constexpr size_t kSmemLimit = 227 * 1024;

// block-wide argmax of the key k over threads (ties -> smaller index); result broadcast.
// Keys are compared as integers (see pivot_key).
__device__ __forceinline__ void block_argmax(unsigned long long& k, int& idx, unsigned long long* sk, int* si) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long ok = __shfl_down_sync(0xffffffffu, k, off);
    const int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ok > k || (ok == k && oi < idx)) { k = ok; idx = oi; }
  }
  if (lane == 0) { sk[w] = k; si[w] = idx; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    k = lane < nw ? sk[lane] : 0ull;
    idx = lane < nw ? si[lane] : 0x7fffffff;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ok = __shfl_down_sync(0xffffffffu, k, off);
      const int oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ok > k || (ok == k && oi < idx)) { k = ok; idx = oi; }
    }
    if (lane == 0) { sk[0] = k; si[0] = idx; }
  }
  __syncthreads();
  k = sk[0];
  idx = si[0];
  __syncthreads();
}

// Pivot key of a candidate entry: the bits of |re| + |im| (non-negative doubles order like their
// bit patterns), Inf / NaN clamped to the largest finite value so that they are still chosen and
// then flagged.  Integer compares keep the pivot search off GB300's narrow FP64 pipe.
__device__ __forceinline__ unsigned long long pivot_key(zd a) {
  const unsigned long long k = (unsigned long long)__double_as_longlong(zabs1(a));
  return k >= 0x7FF0000000000000ull ? 0x7FEFFFFFFFFFFFFFull : k;
}
// (key, pos) ordering of pivot candidates: larger key, then smaller position
__device__ __forceinline__ bool cand_better(unsigned long long k1, int p1, unsigned long long k2, int p2) {
  return k1 > k2 || (k1 == k2 && p1 < p2);
}

// 1 / a for a finite, non-zero a with one real reciprocal: a is scaled by an exact power of two
// 2^-e so that s = |a 2^-e|^2 lies in [1, 8), then 1/a = conj(a 2^-e) 2^-e / s.  A handful of dependent
// FP64 operations instead of the three divisions of Smith's method (used when the exponent is at
// the ends of the range, where the scaling itself could leave the normal numbers).
__device__ __forceinline__ zd zrecip_fast(zd a) {
  const unsigned long long bx = (unsigned long long)__double_as_longlong(a.x) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long by = (unsigned long long)__double_as_longlong(a.y) & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(((bx > by ? bx : by) >> 52) & 0x7FF);  // biased exponent of max(|re|, |im|)
  if (e < 64 || e > 2046 - 64) return zinv(a);
  const double sc = __longlong_as_double((long long)(2046 - e) << 52);  // 2^(1023 - e)
  const double xr = a.x * sc, xi = a.y * sc;                              // exact, max in [1, 2)
  const double s = fma(xr, xr, xi * xi);
  const double t = __drcp_rn(s) * sc;
  return zmake(xr * t, -xi * t);
}

__device__ __forceinline__ int pivot_code(zd piv) {
  if (!isfinite(piv.x) || !isfinite(piv.y)) return BT_ERR_NONFINITE;
  if (piv.x == 0.0 && piv.y == 0.0) return BT_ERR_SINGULAR;
  return 0;
}

// One Gauss-Jordan step on a row-major panel P (rows 0..n-1, columns 0..kb-1, leading
// dimension ld) in shared memory, pivot column jj, pivot row searched in rows >= j.
// Returns the pivot row; *code gets a failure code (thread 0 view).  The pivot's reciprocal is
// formed once (thread 0) and broadcast.
__device__ int gj_step(zd* P, int n, int kb, int ld, int j, int jj, zd* colj, zd* rowj, unsigned long long* sk,
                       int* si, zd* s_ip, int* code) {
  // pivot search (rows scanned in increasing order: strict > keeps the first on ties)
  unsigned long long best = 0;
  int bi = 0x7fffffff;
  for (int r = j + threadIdx.x; r < n; r += blockDim.x) {
    const unsigned long long k = pivot_key(P[r * ld + jj]);
    if (bi == 0x7fffffff || k > best) { best = k; bi = r; }
  }
  block_argmax(best, bi, sk, si);
  const int p = bi;
  if (p != j) {
    for (int c = threadIdx.x; c < kb; c += blockDim.x) {
      zd t = P[j * ld + c];
      P[j * ld + c] = P[p * ld + c];
      P[p * ld + c] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const zd piv = P[j * ld + jj];
    const int pc = pivot_code(piv);
    if (pc && *code == 0) *code = pc;
    *s_ip = pc ? zmake(0.0, 0.0) : zinv(piv);
  }
  __syncthreads();
  const zd ip = *s_ip;
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
  __shared__ unsigned long long sk[32];
  __shared__ int si[32];
  __shared__ int code;
  __shared__ zd s_ip;
  zd* Ag = A + sA * b;
  if (threadIdx.x == 0) code = 0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) P[(e / n) * ld + (e % n)] = Ag[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    int p = gj_step(P, n, n, ld, j, j, colj, rowj, sk, si, &s_ip, &code);
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
// updates use CL SMs instead of one.  Rows are not exchanged while the panel is eliminated:
// every CTA keeps the same position map of the row exchanges (row_at / pos_of), and the pivot
// search of column j runs over the rows whose current position is >= j, ties going to the
// smaller position, which selects the pivot sequence of elimination with physical exchanges.
// Per column: warp 0 of each CTA publishes its best candidate (key, position and the row's kb
// entries) in a buffer of parity j & 1, one cluster barrier, then every CTA reads all candidates
// and their rows through distributed shared memory in one round of independent loads, picks the
// winner (its row index from the replicated position map) and updates its own rows.
// A buffer of parity j & 1 is rewritten two columns later, after the barrier of column j + 1,
// which no CTA passes before every CTA has finished reading it.  At the end each CTA writes its
// rows to their final positions.  perm[] records the exchanges as the LAPACK-style sequence
// (row j swapped with row perm[j], in order), as the rest of the blocked inverse expects.
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
  zd* pub = P + (size_t)R * ld;             // [2][kb]  published candidate rows
  zd* rowj = pub + 2 * kb;                  // [kb]     scaled pivot row
  int* pos_of = reinterpret_cast<int*>(rowj + kb);  // [n] current position of each row
  int* row_at = pos_of + n;                          // [n] row at each position
  __shared__ unsigned long long cand_key[2];
  __shared__ int cand_pos[2];
  __shared__ zd s_ip;
  __shared__ int s_q, s_code;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  zd* Ag = A + sA * b;
  int* perm = perm_all + (long long)n * b;
  if (tid == 0) s_code = 0;
  for (int r = tid; r < n; r += blockDim.x) { pos_of[r] = r; row_at[r] = r; }
  for (int e = tid; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    P[r * ld + c] = Ag[(long long)(r0 + r) * n + k0 + c];
  }
  __syncthreads();
  // row update layout: 4 threads per row, columns c = sub, sub + 4, ...
  const int sub = tid & 3;
  const int rows_per_pass = blockDim.x >> 2;
  for (int jj = 0; jj < kb; ++jj) {
    const int j = k0 + jj, par = jj & 1;
    if (warp == 0) {
      // best local candidate among rows at positions >= j: (key, position) reduced over the warp;
      // its row is row_at[position] (the position maps are the same in every CTA)
      unsigned long long bk = 0;
      int bp = 0x7fffffff;
      for (int r = lane; r < rows; r += 32) {
        const int pos = pos_of[r0 + r];
        if (pos < j) continue;
        const unsigned long long k = pivot_key(P[r * ld + jj]);
        if (bp == 0x7fffffff || cand_better(k, pos, bk, bp)) { bk = k; bp = pos; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, off);
        const int op = __shfl_xor_sync(0xffffffffu, bp, off);
        if (op != 0x7fffffff && (bp == 0x7fffffff || cand_better(ok, op, bk, bp))) { bk = ok; bp = op; }
      }
      if (lane == 0) { cand_key[par] = bk; cand_pos[par] = bp; }
      if (bp != 0x7fffffff) {
        const int br = row_at[bp];
        for (int c = lane; c < kb; c += 32) pub[par * kb + c] = P[(br - r0) * ld + c];
      }
    }
    cluster.sync();  // candidates of column j visible cluster-wide
    if (warp == 0) {
      // one round of remote reads, all issued before any is used: lane l reads the candidate of
      // CTA l % CL, and entry l of every CTA's candidate row; the winner's row is then selected
      // locally (lanes >= kb read a valid entry they do not use)
      const int qr = lane & (CL - 1);
      const int cl = lane < kb ? lane : kb - 1;
      unsigned long long bk = *cluster.map_shared_rank(&cand_key[par], qr);
      int bp = *cluster.map_shared_rank(&cand_pos[par], qr);
      int bq = qr;
      zd cv[CL];
#pragma unroll
      for (int q = 0; q < CL; ++q) cv[q] = cluster.map_shared_rank(pub, q)[par * kb + cl];
#pragma unroll
      for (int off = CL / 2; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, off);
        const int op = __shfl_xor_sync(0xffffffffu, bp, off);
        const int oq = __shfl_xor_sync(0xffffffffu, bq, off);
        if (op != 0x7fffffff && (bp == 0x7fffffff || cand_better(ok, op, bk, bp))) { bk = ok; bp = op; bq = oq; }
      }
      // every lane now holds the winner (position j itself is always a candidate)
      const int br = row_at[bp];
      zd wv = cv[0];
#pragma unroll
      for (int q = 1; q < CL; ++q)
        if (bq == q) wv = cv[q];
      const zd piv = zmake(__shfl_sync(0xffffffffu, wv.x, jj), __shfl_sync(0xffffffffu, wv.y, jj));
      const int pc = pivot_code(piv);
      zd ip = zmake(0.0, 0.0);
      if (lane == 0 && !pc) ip = zrecip_fast(piv);  // one lane: GB300's FP64 pipe is narrow
      ip = zmake(__shfl_sync(0xffffffffu, ip.x, 0), __shfl_sync(0xffffffffu, ip.y, 0));
      if (lane < kb) rowj[lane] = lane == jj ? ip : zmul(wv, ip);
      if (lane == 0) {
        s_ip = ip;
        s_q = br;
        if (pc && s_code == 0) s_code = pc;
        // exchange positions j and bp
        const int cur = bp, rj = row_at[j];
        if (rank == 0) perm[j] = cur;
        row_at[cur] = rj;
        pos_of[rj] = cur;
        row_at[j] = br;
        pos_of[br] = j;
      }
    }
    __syncthreads();
    const zd ip = s_ip;
    const int q = s_q;
    for (int rb = 0; rb < rows; rb += rows_per_pass) {  // uniform trip count (the __syncwarp below)
      const int r = rb + (tid >> 2);
      const bool act = r < rows;
      const zd f = act ? P[r * ld + jj] : zmake(0.0, 0.0);
      __syncwarp();
      if (act) {
        if (r0 + r == q) {
          for (int c = sub; c < kb; c += 4) P[r * ld + c] = rowj[c];
        } else {
          for (int c = sub; c < kb; c += 4) {
            if (c == jj) {
              P[r * ld + c] = zmul(zmake(-f.x, -f.y), ip);
            } else {
              zd a = P[r * ld + c];
              const zd g = rowj[c];
              a.x = fma(-f.x, g.x, a.x);
              a.x = fma(f.y, g.y, a.x);
              a.y = fma(-f.x, g.y, a.y);
              a.y = fma(-f.y, g.x, a.y);
              P[r * ld + c] = a;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // rows to their final positions (pos_of is a permutation: disjoint destinations)
  for (int e = tid; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    Ag[(long long)pos_of[r0 + r] * n + k0 + c] = P[r * ld + c];
  }
  if (rank == 0 && tid == 0 && s_code && info && info[b] == 0) info[b] = s_code;
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

constexpr int kPanelCluster = 8;  // largest cluster (portable size)
size_t cluster_panel_smem(int n, int kb, int cl) {
  const int R = (n + cl - 1) / cl;
  return (size_t)R * (kb + 1) * sizeof(zd) + (size_t)(3 * kb) * sizeof(zd) + 2 * (size_t)n * sizeof(int) + 16;
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
  __shared__ unsigned long long sk[32];
  __shared__ int si[32];
  __shared__ int code;
  __shared__ zd s_ip;
  zd* Ag = A + sA * b;
  int* perm = perm_all + (long long)n * b;
  if (threadIdx.x == 0) code = 0;
  for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    P[r * ld + c] = Ag[(long long)r * n + k0 + c];
  }
  __syncthreads();
  for (int jj = 0; jj < kb; ++jj) {
    int p = gj_step(P, n, kb, ld, k0 + jj, jj, colj, rowj, sk, si, &s_ip, &code);
    if (threadIdx.x == 0) perm[k0 + jj] = p;
  }
  for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    Ag[(long long)r * n + k0 + c] = P[r * ld + c];
  }
  if (threadIdx.x == 0 && code && info && info[b] == 0) info[b] = code;
}

// Row exchanges of the panel (the LAPACK-style sequence perm[k0..k0+kb)) applied to the columns
// outside it as one permutation of the touched rows (at most 2 kb): all touched entries of a
// column are read first (independent loads, 8 rows in flight per column), then written to their
// new rows.  Rows K of those columns are copied to T and zeroed; T's panel columns are zeroed,
// so that one rank-kb GEMM over all n columns leaves the panel columns unchanged.
// Block = 32 columns x 8 row slots of one matrix.
constexpr int kSwapCols = 32;
constexpr int kSwapRows = 8;
constexpr int kMaxTouched = 64;  // 2 * the largest panel width
__global__ void __launch_bounds__(kSwapCols * kSwapRows) gj_swap_copy_kernel(int n, int k0, int kb,
                                                                             zd* __restrict__ A, long long sA,
                                                                             const int* __restrict__ perm_all,
                                                                             zd* __restrict__ T, long long sT,
                                                                             const int* __restrict__ active) {
  __shared__ int pos[kMaxTouched], src[kMaxTouched];
  __shared__ int cnt;
  __shared__ zd stage[kMaxTouched][kSwapCols + 1];
  const int b = blockIdx.y;
  if (active && active[b] == 0) return;
  const int* perm = perm_all + (long long)n * b;
  const int tx = threadIdx.x % kSwapCols, ty = threadIdx.x / kSwapCols;
  if (threadIdx.x == 0) {
    // pos[i] <- the row src[i] after the exchanges, for every touched row
    int m = 0;
    for (int jj = 0; jj < kb; ++jj) {
      const int j = k0 + jj, p = perm[j];
      int ij = -1, ip = -1;
      for (int i = 0; i < m; ++i) {
        if (pos[i] == j) ij = i;
        if (pos[i] == p) ip = i;
      }
      if (ij < 0) { pos[m] = j; src[m] = j; ij = m++; }
      if (ip < 0) { pos[m] = p; src[m] = p; ip = m++; }
      const int t = src[ij];
      src[ij] = src[ip];
      src[ip] = t;
    }
    cnt = m;
  }
  __syncthreads();
  const int c = blockIdx.x * kSwapCols + tx;
  const bool col_ok = c < n;
  const bool panel = c >= k0 && c < k0 + kb;
  zd* Ag = A + sA * b;
  zd* Tb = T + sT * b;
  const int m = cnt;
  if (col_ok && !panel)
    for (int i = ty; i < m; i += kSwapRows) stage[i][tx] = Ag[(long long)src[i] * n + c];
  __syncthreads();  // every touched entry of these columns read before any is written
  if (!col_ok) return;
  if (panel) {
    for (int jj = ty; jj < kb; jj += kSwapRows) Tb[(long long)jj * n + c] = zmake(0.0, 0.0);
    return;
  }
  for (int i = ty; i < m; i += kSwapRows) {
    const int q = pos[i];
    if (q >= k0 && q < k0 + kb) {
      Tb[(long long)(q - k0) * n + c] = stage[i][tx];
      Ag[(long long)q * n + c] = zmake(0.0, 0.0);
    } else {
      Ag[(long long)q * n + c] = stage[i][tx];
    }
  }
}

// Row exchanges undone as column exchanges in reverse order, composed into one column
// permutation: out[r][c] = row_r[src[c]].  One row per warp (blockDim / 32 rows per block), each
// staged in shared memory (coalesced read, gather from shared memory, coalesced write).
constexpr int kUnscrRows = 4;
__global__ void __launch_bounds__(32 * kUnscrRows) gj_unscramble_kernel(int n, zd* __restrict__ A, long long sA,
                                                                        const int* __restrict__ perm_all,
                                                                        const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrows = blockDim.x >> 5;
  zd* rows = reinterpret_cast<zd*>(smem_raw);                  // [nrows][n]
  int* src = reinterpret_cast<int*>(rows + (size_t)nrows * n);  // [n]
  const int b = blockIdx.y;
  if (active && active[b] == 0) return;
  const int* perm = perm_all + (long long)n * b;
  for (int c = threadIdx.x; c < n; c += blockDim.x) src[c] = c;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = n - 1; j >= 0; --j) {
      const int p = perm[j];
      if (p != j) { const int t = src[j]; src[j] = src[p]; src[p] = t; }
    }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * nrows + warp;
  if (r >= n) return;
  zd* row = A + sA * b + (long long)r * n;
  zd* buf = rows + (size_t)warp * n;
  for (int c = lane; c < n; c += 32) buf[c] = row[c];
  __syncwarp();
  for (int c = lane; c < n; c += 32) row[c] = buf[src[c]];
}

int panel_width(int n, bool wide) {
  // The panel elimination costs ~n kb^2 complex FMAs per panel on the SMs of one matrix's
  // cluster (4 n^2 kb DFMA per inverse), the rank-kb updates n^3 on all SMs.  On GB300's slow
  // FP64 pipe kb = 16 balances the two when the updates are FP64 GEMMs; when they run sliced on
  // the tensor cores (wide), kb = 32 fills one 64-deep K block of the split GEMM (K' = 2 kb)
  // and halves the number of update launches.
  for (int kb = wide ? 32 : 16; kb >= 4; kb >>= 1) {
    size_t need = (size_t)n * (kb + 1) * sizeof(zd) + (size_t)(n + kb) * sizeof(zd) + 1024;
    if (need <= kSmemLimit || n >= kClusterMinN) return kb;
  }
  return 0;
}

size_t unscramble_smem(int n, int rows) { return (size_t)rows * n * sizeof(zd) + (size_t)n * sizeof(int); }
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
      cudaFuncSetAttribute(gj_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_max) != cudaSuccess ||
      cudaFuncSetAttribute(gj_panel_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_max) !=
          cudaSuccess ||
      cudaFuncSetAttribute(gj_panel_cluster_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_max) !=
          cudaSuccess ||
      cudaFuncSetAttribute(gj_panel_cluster_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_max) !=
          cudaSuccess ||
      cudaFuncSetAttribute(gj_unscramble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_max) != cudaSuccess)
    return BT_ERR_CUDA;
  done[dev] = true;
  return BT_OK;
}

// Cluster size of the panel kernel (2, 4 or 8 CTAs per matrix): the largest for which every
// matrix of the batch gets its cluster at once, by the occupancy the hardware reports for that
// cluster size and shared-memory size (the panel CTAs are small, so two clusters can share SMs:
// 32 matrices run 8-CTA clusters at two CTAs per SM instead of 4-CTA clusters at one).
// A test / measurement override (bt_debug_panel_cluster) forces a size.
std::atomic<int> g_panel_cluster{0};

template <int CL>
int max_active_clusters(int n, int kb, int batch) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;  // (device, shared bytes) -> clusters
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const int smem = (int)cluster_panel_smem(n, kb, CL);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, smem});
  if (it != cache.end()) return it->second;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(batch * CL));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, gj_panel_cluster_kernel<CL>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    nc = 0;
  }
  cache[{dev, smem}] = nc;
  return nc;
}

int panel_cluster_size(int n, int kb, int batch) {
  const int forced = g_panel_cluster.load();
  if (forced == 2 || forced == 4 || forced == 8) return forced;
  if (max_active_clusters<8>(n, kb, batch) >= batch) return 8;
  if (max_active_clusters<4>(n, kb, batch) >= batch) return 4;
  return 2;
}

}  // namespace

size_t zinv_workspace_bytes(int n, int batch, bool wide) {
  if (n <= kSmallN) return 0;
  int kb = panel_width(n, wide);
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
  // wide panels when the updates run sliced and the workspace was sized for them
  const bool wide = E.slices > 0 && ws_bytes >= zinv_workspace_bytes(n, batch, true);
  int kb = panel_width(n, wide);
  if (kb == 0) return BT_ERR_UNSUPPORTED;
  // a narrower panel (autotuner) fits the workspace sized for the default one
  if (E.panel >= 4 && E.panel < kb) kb = E.panel;
  if (ws_bytes < zinv_workspace_bytes(n, batch, wide) || ws == nullptr) return BT_ERR_INVALID_ARG;
  if (batch > 65535) return BT_ERR_INVALID_ARG;
  int* perm = static_cast<int*>(ws);
  size_t perm_bytes = ((size_t)batch * n * sizeof(int) + 255) / 256 * 256;
  zd* T = reinterpret_cast<zd*>(static_cast<char*>(ws) + perm_bytes);
  const long long sT = (long long)kb * n;
  const bool clustered = n >= kClusterMinN;
  int cl = kPanelCluster;
  if (clustered) {
    cl = panel_cluster_size(n, kb, batch);
    if (cluster_panel_smem(n, kb, cl) > kSmemLimit - 1024) return BT_ERR_UNSUPPORTED;
  }
  for (int k0 = 0; k0 < n; k0 += kb) {
    const int w = (n - k0) < kb ? (n - k0) : kb;
    if (clustered) {
      // one cluster of cl CTAs per matrix (rows of the panel split across SMs): the largest
      // cluster for which every matrix of the batch is resident at once
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(batch * cl));
      cfg.blockDim = dim3(NT);
      cfg.dynamicSmemBytes = cluster_panel_smem(n, w, cl);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cl;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cl == 8) {
        BT_CUDA_TRY(cudaLaunchKernelEx(&cfg, gj_panel_cluster_kernel<8>, n, k0, w, A, sA, perm, info, active));
      } else if (cl == 4) {
        BT_CUDA_TRY(cudaLaunchKernelEx(&cfg, gj_panel_cluster_kernel<4>, n, k0, w, A, sA, perm, info, active));
      } else {
        BT_CUDA_TRY(cudaLaunchKernelEx(&cfg, gj_panel_cluster_kernel<2>, n, k0, w, A, sA, perm, info, active));
      }
      count_launch();
    } else {
      gj_panel_kernel<<<batch, NT, panel_smem(n, w), st>>>(n, k0, w, A, sA, perm, info, active); count_launch();
    }
    BT_CUDA_TRY(cudaGetLastError());
    dim3 g((n + kSwapCols - 1) / kSwapCols, batch);
    gj_swap_copy_kernel<<<g, kSwapCols * kSwapRows, 0, st>>>(n, k0, w, A, sA, perm, T, sT, active); count_launch();
    BT_CUDA_TRY(cudaGetLastError());
    // A[:, all] += A[:, K] * T: T's panel columns are zero, so the panel columns keep their values
    Operand P{A + k0, n, sA, BT_OP_N};
    Operand Tall{T, n, sT, BT_OP_N};
    BT_TRY(gemm(E, st, n, n, w, zmake(1.0, 0.0), P, Tall, zmake(1.0, 0.0), A, n, sA, batch, active));
  }
  int urows = kUnscrRows;
  while (urows > 1 && unscramble_smem(n, urows) > kSmemLimit - 1024) --urows;
  if (unscramble_smem(n, urows) > kSmemLimit - 1024) return BT_ERR_UNSUPPORTED;
  dim3 g((n + urows - 1) / urows, batch);
  gj_unscramble_kernel<<<g, 32 * urows, unscramble_smem(n, urows), st>>>(n, A, sA, perm, active); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt

extern "C" void bt_debug_panel_cluster(int cl) { bt::g_panel_cluster.store(cl); }

extern "C" bt_status bt_zinv_workspace_bytes(int n, int batch, size_t* bytes) {
  if (!bytes || n < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  *bytes = bt::zinv_workspace_bytes(n, batch, false);
  return BT_OK;
}

extern "C" bt_status bt_zinv_batched(int n, void* A, long long strideA, int batch, int* info_device, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  if (n < 0 || batch < 0 || (n > 0 && batch > 0 && !A)) return BT_ERR_INVALID_ARG;
  if (batch > 1 && strideA < (long long)n * n) return BT_ERR_INVALID_ARG;
  return bt::zinv(static_cast<cudaStream_t>(stream), n, static_cast<zd*>(A), strideA, batch, info_device, workspace,
                  workspace_bytes, nullptr);
}
