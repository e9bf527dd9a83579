// Element-wise energy convolution by FFT (Sec. 4.4, Eq. 3).
//
// For every element series e (an (i, j) entry of a selected block, or of its packed upper
// triangle), c[m] = s * sum_k a[m - k] * b[k], a linear convolution over the energy index with a
// and b zero outside [0, na) and [0, nb).  The paper replaces the O(N_E^2) sum by FFTs; here each
// series is transformed in shared memory:
//   * L = the power of two >= na + nb - 1 (zero padding makes the circular convolution of length
//     L equal the linear one);
//   * a and b are loaded energy by energy into bit-reversed positions (the loads of one energy
//     cover TS adjacent elements, so a warp reads whole 32-byte sectors of the energy-major
//     arrays), then transformed by in-place radix-2 decimation-in-time stages;
//   * the spectra are multiplied (with s / L folded in), transformed back by decimation-in-
//     frequency stages (natural order in, bit-reversed order out), and the requested window of c
//     is written energy by energy;
//   * twiddles exp(-2 pi i r / L), r < L / 2, are tabulated once per CTA in shared memory; the
//     grid is persistent (a few CTAs per SM walking the element tiles).
// All arithmetic is FP64.  On GB300 the FP64 pipe, not HBM, bounds this kernel: a transform of
// length L costs about 5 L log2 L flops per series, three per convolution.
#include <atomic>

#include "bt_common.cuh"

namespace bt {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxL = 4096;
constexpr int kTileC = 2048;  // complex values per buffer per CTA: TS series of length L

__device__ __forceinline__ int bitrev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

struct ConvParams {
  int n_elem, na, nb, m0, n_out, L, log2L, TS;
  const zd* A;
  long long lda;
  const zd* B;
  long long ldb;
  zd* C;
  long long ldc;
  zd scale;  // s / L
  int reverse_b, conj_b;
};

__device__ __forceinline__ zd mul_mi(zd a) { return zmake(a.y, -a.x); }  // a * (-i)
__device__ __forceinline__ zd mul_pi(zd a) { return zmake(-a.y, a.x); }  // a * (+i)

// In-place FFT stages over TS series of length L held as x[t * L + i], two radix-2 stages per
// pass over the data (each thread takes the four points i0 + {0, h, 2h, 3h}): half the shared-
// memory round trips and barriers of single stages.  tw[r] = exp(-2 pi i r / L), r < L / 2.
//
// Forward, decimation in time (bit-reversed input, natural output), stages s and s + 1 (spans h
// and 2h), w1 = W_2h^r, w2 = W_4h^r, W_4h^(r+h) = -i w2:
//   a0 = x0 + w1 x1, a1 = x0 - w1 x1, a2 = x2 + w1 x3, a3 = x2 - w1 x3,
//   y0 = a0 + w2 a2, y2 = a0 - w2 a2, y1 = a1 - i w2 a3, y3 = a1 + i w2 a3.
// The first stage pair has w1 = w2 = 1 (no multiplications); an odd stage count starts with one
// single stage of trivial twiddles.
__device__ void fft_dit(zd* x, const zd* tw, int L, int log2L, int TS) {
  const int half = L >> 1, quarter = L >> 2;
  int s = 0;
  if (log2L & 1) {  // one radix-2 stage with w = 1
    for (int q = threadIdx.x; q < TS * half; q += blockDim.x) {
      const int t = q / half, j = q - t * half;
      zd* y = x + t * L + 2 * j;
      const zd u = y[0], v = y[1];
      y[0] = zadd(u, v);
      y[1] = zsub(u, v);
    }
    __syncthreads();
    s = 1;
  }
  for (; s + 1 < log2L; s += 2) {
    const int h = 1 << s;
    const int t1 = half >> s, t2 = half >> (s + 1);
    for (int q = threadIdx.x; q < TS * quarter; q += blockDim.x) {
      const int t = q / quarter, j = q - t * quarter;
      const int g = j >> s, r = j & (h - 1);
      zd* y = x + t * L + (g << (s + 2)) + r;
      const zd x0 = y[0], x1 = y[h], x2 = y[2 * h], x3 = y[3 * h];
      zd a0, a1, a2, a3, b2, b3;
      if (s == 0) {
        a0 = zadd(x0, x1); a1 = zsub(x0, x1); a2 = zadd(x2, x3); a3 = zsub(x2, x3);
        b2 = a2; b3 = mul_mi(a3);
      } else {
        const zd w1 = tw[r * t1], w2 = tw[r * t2];
        const zd v1 = zmul(x1, w1), v3 = zmul(x3, w1);
        a0 = zadd(x0, v1); a1 = zsub(x0, v1); a2 = zadd(x2, v3); a3 = zsub(x2, v3);
        b2 = zmul(a2, w2); b3 = mul_mi(zmul(a3, w2));
      }
      y[0] = zadd(a0, b2);
      y[2 * h] = zsub(a0, b2);
      y[h] = zadd(a1, b3);
      y[3 * h] = zsub(a1, b3);
    }
    __syncthreads();
  }
}

// Inverse, decimation in frequency (natural input, bit-reversed output), conjugate twiddles,
// stages s + 1 then s:
//   a0 = x0 + x2, a2 = (x0 - x2) conj(w2), a1 = x1 + x3, a3 = (x1 - x3) conj(w2) i,
//   y0 = a0 + a1, y1 = (a0 - a1) conj(w1), y2 = a2 + a3, y3 = (a2 - a3) conj(w1).
// The last stage pair has w1 = w2 = 1; an odd stage count ends with one single stage of w = 1.
__device__ void ifft_dif(zd* x, const zd* tw, int L, int log2L, int TS) {
  const int half = L >> 1, quarter = L >> 2;
  for (int s = log2L - 2; s >= (log2L & 1); s -= 2) {
    const int h = 1 << s;
    const int t1 = half >> s, t2 = half >> (s + 1);
    for (int q = threadIdx.x; q < TS * quarter; q += blockDim.x) {
      const int t = q / quarter, j = q - t * quarter;
      const int g = j >> s, r = j & (h - 1);
      zd* y = x + t * L + (g << (s + 2)) + r;
      const zd x0 = y[0], x1 = y[h], x2 = y[2 * h], x3 = y[3 * h];
      const zd a0 = zadd(x0, x2), a1 = zadd(x1, x3);
      zd a2 = zsub(x0, x2), a3 = mul_pi(zsub(x1, x3));
      zd y1 = zsub(a0, a1), y3;
      if (s == 0) {
        y3 = zsub(a2, a3);
      } else {
        const zd w1 = zconj(tw[r * t1]), w2 = zconj(tw[r * t2]);
        a2 = zmul(a2, w2);
        a3 = zmul(a3, w2);
        y1 = zmul(y1, w1);
        y3 = zmul(zsub(a2, a3), w1);
      }
      y[0] = zadd(a0, a1);
      y[h] = y1;
      y[2 * h] = zadd(a2, a3);
      y[3 * h] = y3;
    }
    __syncthreads();
  }
  if (log2L & 1) {  // the last radix-2 stage, w = 1
    for (int q = threadIdx.x; q < TS * half; q += blockDim.x) {
      const int t = q / half, j = q - t * half;
      zd* y = x + t * L + 2 * j;
      const zd u = y[0], v = y[1];
      y[0] = zadd(u, v);
      y[1] = zsub(u, v);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) conv_kernel(ConvParams p) {
  extern __shared__ zd sh[];
  const int L = p.L, TS = p.TS;
  zd* xa = sh;
  zd* xb = sh + TS * L;
  zd* tw = sh + 2 * TS * L;
  for (int r = threadIdx.x; r < (L >> 1); r += blockDim.x) {
    double sv, cv;
    sincospi(-2.0 * (double)r / (double)L, &sv, &cv);
    tw[r] = zmake(cv, sv);
  }
  __syncthreads();
  const int n_tiles = (p.n_elem + TS - 1) / TS;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int e0 = tile * TS;
    // load a and b into bit-reversed positions (zero padding beyond na / nb)
    for (int idx = threadIdx.x; idx < TS * L; idx += blockDim.x) {
      const int k = idx / TS, t = idx - k * TS;
      const int e = e0 + t;
      const int pos = t * L + bitrev(k, p.log2L);
      zd va = zmake(0.0, 0.0), vb = zmake(0.0, 0.0);
      if (e < p.n_elem) {
        if (k < p.na) va = p.A[(long long)k * p.lda + e];
        if (k < p.nb) {
          const int kb = p.reverse_b ? p.nb - 1 - k : k;
          vb = p.B[(long long)kb * p.ldb + e];
          if (p.conj_b) vb = zconj(vb);
        }
      }
      xa[pos] = va;
      xb[pos] = vb;
    }
    __syncthreads();
    fft_dit(xa, tw, L, p.log2L, TS);
    fft_dit(xb, tw, L, p.log2L, TS);
    for (int idx = threadIdx.x; idx < TS * L; idx += blockDim.x) xa[idx] = zmul(zmul(xa[idx], xb[idx]), p.scale);
    __syncthreads();
    ifft_dif(xa, tw, L, p.log2L, TS);
    for (int idx = threadIdx.x; idx < TS * p.n_out; idx += blockDim.x) {
      const int mi = idx / TS, t = idx - mi * TS;
      const int e = e0 + t;
      if (e < p.n_elem) p.C[(long long)mi * p.ldc + e] = xa[t * L + bitrev(p.m0 + mi, p.log2L)];
    }
    __syncthreads();
  }
}

}  // namespace

bt_status energy_convolve(cudaStream_t st, int n_elem, int na, int nb, int m0, int n_out, const zd* A, long long lda,
                          const zd* B, long long ldb, zd* C, long long ldc, zd scale, int reverse_b, int conj_b) {
  if (n_elem < 0 || na < 1 || nb < 1 || m0 < 0 || n_out < 0) return BT_ERR_INVALID_ARG;
  const long long full = (long long)na + nb - 1;
  if (m0 + (long long)n_out > full) return BT_ERR_INVALID_ARG;
  if (n_elem == 0 || n_out == 0) return BT_OK;
  if (!A || !B || !C || lda < n_elem || ldb < n_elem || ldc < n_elem) return BT_ERR_INVALID_ARG;
  int L = 1, log2L = 0;
  while (L < full) { L <<= 1; ++log2L; }
  if (L > kMaxL) return BT_ERR_UNSUPPORTED;
  if (L < 2) { L = 2; log2L = 1; }
  ConvParams p;
  p.n_elem = n_elem; p.na = na; p.nb = nb; p.m0 = m0; p.n_out = n_out; p.L = L; p.log2L = log2L;
  p.TS = L >= kTileC ? 1 : kTileC / L;
  p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc;
  p.scale = zscale(scale, 1.0 / L);
  p.reverse_b = reverse_b; p.conj_b = conj_b;
  const size_t smem = sizeof(zd) * (2 * (size_t)p.TS * L + L / 2);
  // the kernel's dynamic shared-memory limit, raised to the largest size asked for so far
  static std::atomic<int> configured_smem{0};
  if ((int)smem > configured_smem.load()) {
    BT_CUDA_TRY(cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_smem.store((int)smem);
  }
  int dev = 0, sms = 0, per_sm = 0;
  BT_CUDA_TRY(cudaGetDevice(&dev));
  BT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_kernel, kThreads, smem));
  const long long n_tiles = (n_elem + p.TS - 1) / p.TS;
  long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > n_tiles) grid = n_tiles;
  conv_kernel<<<(unsigned)grid, kThreads, smem, st>>>(p);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt

extern "C" bt_status bt_energy_convolve(int n_elem, int na, int nb, int m0, int n_out, const void* A, long long lda,
                                        const void* B, long long ldb, void* C, long long ldc, double scale_re,
                                        double scale_im, int flags, void* stream) {
  if (flags & ~(BT_CONV_REVERSE_B | BT_CONV_CONJ_B)) return BT_ERR_INVALID_ARG;
  return bt::energy_convolve(static_cast<cudaStream_t>(stream), n_elem, na, nb, m0, n_out, static_cast<const zd*>(A),
                             lda, static_cast<const zd*>(B), ldb, static_cast<zd*>(C), ldc,
                             zmake(scale_re, scale_im), (flags & BT_CONV_REVERSE_B) != 0, (flags & BT_CONV_CONJ_B) != 0);
}
