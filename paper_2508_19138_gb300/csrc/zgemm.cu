// Batched complex128 GEMM on the FP64 pipe (DFMA): the dense block products of the RGF
// forward / backward passes (Sec. 4.3.2, Eq. 9-12) and of the decimation (Eq. 4).
//
// GB300 note: the FP64 pipe of this part issues about 2 DFMA per clock per SM (measured
// ~1.2 TFLOP/s for the whole GPU; the FP64 mma.sync path measured ~1.05 TFLOP/s), so this
// kernel is bound by FP64 issue, not by memory.  Two consequences:
//  * the complex product uses three real products instead of four (Gauss's trick, the "3M"
//    method): t1 = Re a Re b, t2 = Im a Im b, t3 = (Re a + Im a)(Re b + Im b), Re c = t1 - t2,
//    Im c = t3 - t1 - t2.  The sums Re + Im are formed once per element when a tile is staged
//    in shared memory, so the inner loop issues 3 DFMA per complex multiply-add instead of 4
//    (error bound u |a||b| per term with |.| the 1-norm of re/im, Higham 2002, Sec. 23.2.4);
//  * what matters otherwise is keeping every SM busy with whole tiles: 32 x 32 output tiles
//    divide the workload block sizes (32, 416 = 13 x 32, 1024) without ragged waste, and the
//    batch (energies x blocks) gives >= 152 CTAs; where it would not (small blocks, few
//    energies), 16 x 16 tiles of 64 threads are used instead.
// Tiles are staged through shared memory with a register prefetch of the next k-slab.
// zgemm_antiherm: the same kernel over the upper tiles only, for products whose exact result is
// anti-Hermitian (the lesser / greater sandwiches), the lower tiles written as mirror images.
#include <atomic>

#include "bt_common.cuh"

namespace bt {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int BK = 16;
// TILE x TILE output tiles, (TILE/2)^2 threads with 2 x 2 outputs each: 32 (256 threads) for the
// large blocks, 16 (64 threads) when the 32-tiles would leave SMs idle (small blocks, few energies).
template <int TILE>
struct Shape {
  static constexpr int BM = TILE, BN = TILE, NT = TILE * TILE / 4, H = TILE / 2;
  static constexpr int EA = BM * BK / NT, EB = BN * BK / NT;  // staged elements per thread
};

// TRI: C (square, n x n) is known to be anti-Hermitian (C_ji = -conj(C_ij)) in exact arithmetic,
// e.g. the sandwiches x^R B^<> x^R^H of Eq. 10 and 12: only the tiles on and above the diagonal
// are computed (blockIdx.x runs over them row by row), every tile above the diagonal also
// writes its mirror image -(tile)^H below it (staged through shared memory so that the
// transposed store stays coalesced), and the diagonal tiles are made exactly anti-Hermitian.
// About half of the FP64 work of the product.
template <int OPA, int OPB, bool TRI, int TILE>
__global__ void __launch_bounds__(Shape<TILE>::NT) zgemm_kernel(int m, int n, int k, zd alpha, const zd* __restrict__ A,
                                                   int lda, long long sA, const zd* __restrict__ B, int ldb,
                                                   long long sB, zd beta, zd* __restrict__ C, int ldc,
                                                   long long sC, const int* __restrict__ active) {
  constexpr int BM = Shape<TILE>::BM, BN = Shape<TILE>::BN, NT = Shape<TILE>::NT, H = Shape<TILE>::H;
  constexpr int EA = Shape<TILE>::EA, EB = Shape<TILE>::EB;
  const int bz = blockIdx.z;
  if (active && active[bz] == 0) return;
  int m0, n0;
  if (TRI) {
    const int T = (n + BN - 1) / BN;
    int idx = blockIdx.x, tr = 0;
    while (idx >= T - tr) { idx -= T - tr; ++tr; }
    m0 = tr * BM;
    n0 = (tr + idx) * BN;
  } else {
    m0 = blockIdx.y * BM;
    n0 = blockIdx.x * BN;
  }
  A += sA * bz;
  B += sB * bz;
  C += sC * bz;
  // real, imaginary and re + im planes of the staged tiles
  __shared__ double Ar[BK][BM + 1], Ai[BK][BM + 1], Ap[BK][BM + 1];
  __shared__ double Br[BK][BN + 1], Bi[BK][BN + 1], Bp[BK][BN + 1];
  const int t = threadIdx.x;
  const int tx = t % H, ty = t / H;

  double t1[2][2], t2[2][2], t3[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;

  zd ra[EA], rb[EB];  // prefetch registers: the thread's elements of A and of B per k-slab
  auto load_a = [&](int k0) {
#pragma unroll
    for (int s = 0; s < EA; ++s) {
      int e = t + NT * s;
      int r, c;
      if (OPA == BT_OP_N) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      int gr = m0 + r, gc = k0 + c;
      zd v = zmake(0.0, 0.0);
      if (gr < m && gc < k) {
        if (OPA == BT_OP_N) v = A[(long long)gr * lda + gc];
        else v = zconj(A[(long long)gc * lda + gr]);
      }
      ra[s] = v;
    }
  };
  auto load_b = [&](int k0) {
#pragma unroll
    for (int s = 0; s < EB; ++s) {
      int e = t + NT * s;
      int r, c;
      if (OPB == BT_OP_N) { r = e / BN; c = e % BN; } else { c = e / BK; r = e % BK; }
      int gr = k0 + r, gc = n0 + c;
      zd v = zmake(0.0, 0.0);
      if (gr < k && gc < n) {
        if (OPB == BT_OP_N) v = B[(long long)gr * ldb + gc];
        else v = zconj(B[(long long)gc * ldb + gr]);
      }
      rb[s] = v;
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int s = 0; s < EA; ++s) {
      int e = t + NT * s;
      int r, c;
      if (OPA == BT_OP_N) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      Ar[c][r] = ra[s].x;
      Ai[c][r] = ra[s].y;
      Ap[c][r] = ra[s].x + ra[s].y;
    }
#pragma unroll
    for (int s = 0; s < EB; ++s) {
      int e = t + NT * s;
      int r, c;
      if (OPB == BT_OP_N) { r = e / BN; c = e % BN; } else { c = e / BK; r = e % BK; }
      Br[r][c] = rb[s].x;
      Bi[r][c] = rb[s].y;
      Bp[r][c] = rb[s].x + rb[s].y;
    }
  };

  load_a(0);
  load_b(0);
  for (int k0 = 0; k0 < k; k0 += BK) {
    __syncthreads();
    store_tiles();
    __syncthreads();
    if (k0 + BK < k) {
      load_a(k0 + BK);
      load_b(k0 + BK);
    }
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double ar[2], ai[2], ap[2], br[2], bi[2], bp[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        ar[i] = Ar[kk][ty + H * i];
        ai[i] = Ai[kk][ty + H * i];
        ap[i] = Ap[kk][ty + H * i];
        br[i] = Br[kk][tx + H * i];
        bi[i] = Bi[kk][tx + H * i];
        bp[i] = Bp[kk][tx + H * i];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          t1[i][j] = fma(ar[i], br[j], t1[i][j]);
          t2[i][j] = fma(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fma(ap[i], bp[j], t3[i][j]);
        }
    }
  }
  zd acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = zmake(t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]);
  const bool beta_zero = (beta.x == 0.0 && beta.y == 0.0);
  const bool diag_tile = TRI && m0 == n0;  // written below, element by element
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    int gr = m0 + ty + H * i;
    if (gr >= m || diag_tile) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int gc = n0 + tx + H * j;
      if (gc >= n) continue;
      zd* cp = C + (long long)gr * ldc + gc;
      zd v = zmul(alpha, acc[i][j]);
      if (!beta_zero) v = zadd(v, zmul(beta, *cp));
      *cp = v;
    }
  }
  if (TRI) {
    // Tile above the diagonal: its mirror image C[n0 + c][m0 + r] = -conj(alpha acc[r][c]) +
    // beta C[n0 + c][m0 + r] (alpha, beta real).  Diagonal tile: its upper triangle as computed,
    // the strict lower triangle mirrored from it and the diagonal made imaginary, so that the
    // whole of C comes out exactly anti-Hermitian.  (Mirroring only whole tiles would turn the
    // Hermitian rounding noise that the operands carry into anti-Hermitian error; with every
    // output exactly anti-Hermitian no such noise builds up along the sweep.)
    __shared__ double Mr[TRI ? BN : 1][TRI ? BM + 1 : 1], Mi[TRI ? BN : 1][TRI ? BM + 1 : 1];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const zd v = zmul(alpha, acc[i][j]);
        if (diag_tile) {
          Mr[ty + H * i][tx + H * j] = v.x;
          Mi[ty + H * i][tx + H * j] = v.y;
        } else {
          Mr[tx + H * j][ty + H * i] = -v.x;
          Mi[tx + H * j][ty + H * i] = v.y;
        }
      }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < (BM * BN) / NT; ++s) {
      const int r = t / BN + (NT / BN) * s, c = t % BN;
      const int gr = (diag_tile ? m0 : n0) + r, gc = (diag_tile ? n0 : m0) + c;
      if (gr < m && gc < n) {
        zd* cp = C + (long long)gr * ldc + gc;
        zd v;
        if (!diag_tile || r < c) v = zmake(Mr[r][c], Mi[r][c]);
        else if (r > c) v = zmake(-Mr[c][r], Mi[c][r]);
        else v = zmake(0.0, Mi[r][r]);
        if (!beta_zero) v = zadd(v, zmul(beta, *cp));
        if (diag_tile && r == c) v.x = 0.0;
        *cp = v;
      }
    }
  }
}

template <bool TRI, int TILE>
bt_status launch_tile(cudaStream_t st, dim3 grid, int m, int n, int k, zd alpha, const Operand& A, const Operand& B,
                      zd beta, zd* C, int ldc, long long strideC, const int* active) {
  constexpr int NT = Shape<TILE>::NT;
  if (A.op == BT_OP_N && B.op == BT_OP_N)
    zgemm_kernel<BT_OP_N, BT_OP_N, TRI, TILE><<<grid, NT, 0, st>>>(m, n, k, alpha, A.p, A.ld, A.stride, B.p, B.ld, B.stride, beta, C, ldc, strideC, active);
  else if (A.op == BT_OP_N && B.op == BT_OP_C)
    zgemm_kernel<BT_OP_N, BT_OP_C, TRI, TILE><<<grid, NT, 0, st>>>(m, n, k, alpha, A.p, A.ld, A.stride, B.p, B.ld, B.stride, beta, C, ldc, strideC, active);
  else if (A.op == BT_OP_C && B.op == BT_OP_N)
    zgemm_kernel<BT_OP_C, BT_OP_N, TRI, TILE><<<grid, NT, 0, st>>>(m, n, k, alpha, A.p, A.ld, A.stride, B.p, B.ld, B.stride, beta, C, ldc, strideC, active);
  else
    zgemm_kernel<BT_OP_C, BT_OP_C, TRI, TILE><<<grid, NT, 0, st>>>(m, n, k, alpha, A.p, A.ld, A.stride, B.p, B.ld, B.stride, beta, C, ldc, strideC, active);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

int sm_count() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_relaxed);
  if (v == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 152;
    cached.store(v, std::memory_order_relaxed);
  }
  return v;
}

// Tiles of 32 unless they would leave SMs idle (fewer than two tiles per SM), then 16; `tile`
// (16 or 32, from the autotuner) overrides the rule.
template <bool TRI>
bt_status launch_zgemm(cudaStream_t st, int m, int n, int k, zd alpha, const Operand& A, const Operand& B, zd beta,
                       zd* C, int ldc, long long strideC, int batch, const int* active, int tile) {
  auto tiles = [&](int tl) {
    const long long tm = (m + tl - 1) / tl, tn = (n + tl - 1) / tl;
    return TRI ? tn * (tn + 1) / 2 : tm * tn;
  };
  const bool use16 = tile == 16 || (tile != 32 && tiles(32) * batch < 2LL * sm_count());
  if (use16) {
    const long long t16 = tiles(16);
    dim3 grid = TRI ? dim3((unsigned)t16, 1, batch) : dim3((n + 15) / 16, (m + 15) / 16, batch);
    return launch_tile<TRI, 16>(st, grid, m, n, k, alpha, A, B, beta, C, ldc, strideC, active);
  }
  dim3 grid = TRI ? dim3((unsigned)tiles(32), 1, batch) : dim3((n + 31) / 32, (m + 31) / 32, batch);
  return launch_tile<TRI, 32>(st, grid, m, n, k, alpha, A, B, beta, C, ldc, strideC, active);
}

}  // namespace

bt_status zgemm(cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta, zd* C,
                int ldc, long long strideC, int batch, const int* active, int tile) {
  if (m < 0 || n < 0 || k < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (m == 0 || n == 0 || batch == 0) return BT_OK;
  if (batch > 65535) {
    // split very large batches into several launches (grid z limit)
    for (int b0 = 0; b0 < batch; b0 += 65535) {
      int nbatch = batch - b0 < 65535 ? batch - b0 : 65535;
      Operand a = A, b = B;
      a.p += A.stride * b0;
      b.p += B.stride * b0;
      BT_TRY(zgemm(st, m, n, k, alpha, a, b, beta, C + strideC * b0, ldc, strideC, nbatch,
                   active ? active + b0 : nullptr, tile));
    }
    return BT_OK;
  }
  return launch_zgemm<false>(st, m, n, k, alpha, A, B, beta, C, ldc, strideC, batch, active, tile);
}

bt_status zgemm_antiherm(cudaStream_t st, int n, int k, zd alpha, Operand A, Operand B, zd beta, zd* C, int ldc,
                         long long strideC, int batch, const int* active, int tile) {
  if (n < 0 || k < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (n == 0 || batch == 0) return BT_OK;
  if (alpha.y != 0.0 || batch > 65535)
    return zgemm(st, n, n, k, alpha, A, B, beta, C, ldc, strideC, batch, active, tile);
  return launch_zgemm<true>(st, n, n, k, alpha, A, B, beta, C, ldc, strideC, batch, active, tile);
}

bt_status gemm_antiherm(const Engine& eng, cudaStream_t st, int n, int k, zd alpha, Operand A, Operand B, zd beta,
                       zd* C, int ldc, long long strideC, int batch, const int* active) {
  if (eng.slices > 0)
    return split_zgemm(st, n, n, k, alpha, A, B, beta, C, ldc, strideC, batch, eng.slices, eng.ws, eng.ws_bytes,
                       active, eng.err, 0);
  return zgemm_antiherm(st, n, k, alpha, A, B, beta, C, ldc, strideC, batch, active, eng.tile);
}

bt_status gemm(const Engine& eng, cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta,
               zd* C, int ldc, long long strideC, int batch, const int* active) {
  if (eng.slices > 0)
    return split_zgemm(st, m, n, k, alpha, A, B, beta, C, ldc, strideC, batch, eng.slices, eng.ws, eng.ws_bytes,
                       active, eng.err, 0);
  return zgemm(st, m, n, k, alpha, A, B, beta, C, ldc, strideC, batch, active, eng.tile);
}

}  // namespace bt

extern "C" bt_status bt_zgemm_batched(int m, int n, int k, double alpha_re, double alpha_im, const void* A, int lda,
                                      long long strideA, int opA, const void* B, int ldb, long long strideB, int opB,
                                      double beta_re, double beta_im, void* C, int ldc, long long strideC, int batch,
                                      void* stream) {
  if ((opA != BT_OP_N && opA != BT_OP_C) || (opB != BT_OP_N && opB != BT_OP_C)) return BT_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && batch > 0 && (!C || (k > 0 && (!A || !B)))) return BT_ERR_INVALID_ARG;
  int rowsA = opA == BT_OP_N ? k : m;  // minimal leading dimensions
  int rowsB = opB == BT_OP_N ? n : k;
  if (lda < (rowsA > 1 ? rowsA : 1) || ldb < (rowsB > 1 ? rowsB : 1) || ldc < (n > 1 ? n : 1))
    return BT_ERR_INVALID_ARG;
  bt::Operand a{static_cast<const zd*>(A), lda, strideA, opA};
  bt::Operand b{static_cast<const zd*>(B), ldb, strideB, opB};
  return bt::zgemm(static_cast<cudaStream_t>(stream), m, n, k, zmake(alpha_re, alpha_im), a, b,
                   zmake(beta_re, beta_im), static_cast<zd*>(C), ldc, strideC, batch, nullptr);
}
