// Split-precision complex GEMM on the tcgen05 tensor cores (the BT_SPLIT products of the RGF
// sweeps): C = alpha op(A) op(B) + beta C with complex128 operands, computed as sums of exact
// bf16 slice products in the manner of Ozaki et al. (error-free splitting, 2012).
//
// Realification.  With K' = 2k interleaved (re, im) and the transposed product C^T:
//     Bt[2j  ][2p] = Re op(B)[p][j],  Bt[2j  ][2p+1] = -Im op(B)[p][j]
//     Bt[2j+1][2p] = Im op(B)[p][j],  Bt[2j+1][2p+1] =  Re op(B)[p][j]
//     At[i][2p] = Re op(A)[i][p],     At[i][2p+1] = Im op(A)[i][p]
// gives (Bt At^T)[2j][i] = Re C[i][j], [2j+1][i] = Im C[i][j]: one real GEMM, M = 2n rows
// (MMA "A" operand Bt), N = m columns (MMA "B" operand At), K = 2k, both operands K-major.
//
// Slicing.  Each row i of op(A) is scaled by 2^-eA_i (eA_i = max exponent of the row) and cut
// into S digits of 7 bits by integer arithmetic on the IEEE fields (truncated fixed point with
// 7S fraction bits); digit s is stored as bf16(sign * d_s * 2^(-7(s-1))), exact.  Columns of
// op(B) likewise with eB_j.  A slice product of digits is an integer < K' * 127^2 < 2^24 for
// K' <= 1040, so the tensor core's fp32 accumulation of a single slice pair is exact.
//
// Accumulation.  Pairs (s, t) with s + t <= S + 1 are used.  Pairs with s + t <= 5 are
// accumulated one per TMEM accumulator (exact); all remaining pairs share one accumulator
// (their fp32 rounding is below 2^-45 of the leading term).  Every accumulator is drained into
// per-thread int64 fixed-point sums (2^-36 units of the leading digit product), so the final
// value is assembled without floating-point cancellation; the FP64 pipe is touched only for
// the alpha / beta update of C.
//
// Kernel shape: one CTA per 128 x NT output tile of C^T and batch entry; warp 0 issues TMA
// loads (3-D tensor maps over [batch*S][rows][K'], 128-byte swizzle), warp 1 issues the
// tcgen05.mma instructions (M = 128, N = NT, K = 16) into a double-buffered TMEM accumulator,
// warps 2..9 drain the accumulators and write C.  All waits are bounded in time; on a timeout
// the CTA records BT_ERR_TIMEOUT, drains what it issued and frees its TMEM.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "bt_common.cuh"
#include "sm103_ptx.cuh"

namespace bt {
namespace {

constexpr int kDigitBits = 7;
constexpr int kMaxSlices = 8;
constexpr int kMaxPairs = kMaxSlices * (kMaxSlices + 1) / 2;
constexpr int kExactD = 5;       // pairs with s + t <= kExactD get their own accumulator
constexpr int kFixShift = 36;    // int64 fixed point: units of 2^-36 of a leading digit product
constexpr int kTileM = 128;
constexpr int kKBlock = 64;      // bf16 per 128-byte swizzle row
constexpr int kStages = 7;       // 7 x (16 + 16) KB covers the TMA latency at 224 clocks per stage
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kMaxKp = 1040;     // K' bound for exact fp32 accumulation of one slice pair
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

struct Schedule {
  int n_pairs;
  int n_groups;
  unsigned char s[kMaxPairs];          // slice of op(A) (1-based)
  unsigned char t[kMaxPairs];          // slice of op(B) (1-based)
  unsigned char group_end[kMaxPairs];  // pairs [group_end[g-1], group_end[g]) form group g
};

struct MmaParams {
  int m;          // rows of C (N side of the MMA)
  int n2;         // 2 * columns of C (M side)
  int Kp;         // padded K' (multiple of 8)
  int S;
  const int* eA;  // [batch][m] biased exponents of op(A) rows
  const int* eB;  // [batch][n] biased exponents of op(B) columns
  zd* C;
  int ldc;
  long long sC;
  zd alpha, beta;
  int beta_zero;
  int complex_coef;  // alpha or beta has an imaginary part
  int* err;          // per batch entry error slot (may be null)
  const int* active; // batch entries with active[b] == 0 are skipped (may be null)
  int a_shared;      // op(A) / op(B) shared by every batch entry: sliced once (batch index 0)
  int b_shared;
  Schedule sched;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// fp32 value -> int64 fixed point with kFixShift fraction bits, from the IEEE fields with
// integer instructions only (a float -> int64 conversion would run on GB300's slow FP64 pipe).
// Exact for the single-pair groups (integers times 2^-7(s+t-2), s+t <= 7); the shared group
// is truncated below 2^-36 of a leading digit product.
__device__ __forceinline__ long long f32_to_fix(float v) {
  const uint32_t bits = __float_as_uint(v);
  const int e = (int)((bits >> 23) & 0xFFu);
  if (e == 0) return 0;  // zero (denormals are far below the fixed-point resolution)
  const long long m = (long long)((bits & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 150 + kFixShift;  // value = m * 2^(e - 150)
  long long r;
  if (sh >= 0) r = sh < 40 ? (m << sh) : 0x7FFFFFFFFFFFFFFFll;  // |v| >= 2^27 cannot occur
  else r = sh > -32 ? (m >> -sh) : 0;
  return (bits >> 31) ? -r : r;
}

// int64 fixed-point value * 2^e -> double, integer arithmetic only (round to nearest even).
__device__ __forceinline__ double fix_to_double(long long v, int e) {
  if (v == 0) return 0.0;
  unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(a);
  a <<= lz;                                   // leading one at bit 63
  unsigned long long mant = a >> 11;          // 53 bits incl. the leading one
  const unsigned long long rem = a & 0x7FFull;
  int expo = 1023 + (63 - lz) + e;            // value = mant * 2^(63-lz-52) * 2^e
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) { mant >>= 1; ++expo; }
  }
  if (expo <= 0 || expo >= 2047) {            // outside the normal range: slow path
    const double r = ldexp((double)mant, expo - 1023 - 52);
    return sign ? -r : r;
  }
  const unsigned long long bits = sign | ((unsigned long long)expo << 52) | (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1)
    split_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const MmaParams p) {
  constexpr int kABytes = kTileM * 128;
  constexpr int kBBytes = NT * 128;
  constexpr int kHalf = NT / 2;
  constexpr int kChunks = kHalf / 8;
  static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "UMMA N");
  static_assert(2 * NT <= 256, "two accumulators must fit in 256 TMEM columns");
  constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(kTileM, NT);

  if (p.active && p.active[blockIdx.z] == 0) return;  // before any barrier or TMEM use
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM;  // rows of C^T
  const int n0 = blockIdx.y * NT;      // rows of C
  const int b = blockIdx.z;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], kEpiWarps);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 256);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int KB = (p.Kp + kKBlock - 1) / kKBlock;
  const Schedule& sc = p.sched;
  auto fail = [&]() {
    *abort_flag = 1;
    if (p.err) atomicCAS(&p.err[b], 0, (int)BT_ERR_TIMEOUT);
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      ptx::prefetch_tensormap(&tmA);
      ptx::prefetch_tensormap(&tmB);
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      const int n_items = sc.n_pairs * KB;
      for (int it = 0; it < n_items; ++it) {
        const int pi = it / KB, kb = it - pi * KB;
        if (!ptx::mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, kWaitLimitNs)) { fail(); break; }
        ptx::mbar_arrive_expect_tx(&full[stage], kABytes + kBBytes);
        ptx::tma_load_3d(sA + stage * kABytes, &tmA, &full[stage], kb * kKBlock, m0,
                         (p.b_shared ? 0 : b) * p.S + (sc.t[pi] - 1));
        ptx::tma_load_3d(sB + stage * kBBytes, &tmB, &full[stage], kb * kKBlock, n0,
                         (p.a_shared ? 0 : b) * p.S + (sc.s[pi] - 1));
        ++issued;
        if (++stage == kStages) { stage = 0; phase ^= 1u; }
      }
      if (*abort_flag) {
        // let the loads already in flight land before the CTA exits (bounded)
        volatile int never = 0;
        for (int idx = issued > kStages ? issued - kStages : 0; idx < issued; ++idx)
          ptx::mbar_wait_bounded(&full[idx % kStages], (uint32_t)((idx / kStages) & 1), &never, kWaitLimitNs);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int g = 0; g < sc.n_groups && ok; ++g) {
        const int ab = g & 1;
        if (g >= 2) {
          if (!ptx::mbar_wait_bounded(&tempty[ab], (uint32_t)(((g >> 1) - 1) & 1), abort_flag, kWaitLimitNs)) {
            fail();
            ok = false;
            break;
          }
        }
        ptx::tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(ab * NT);
        const int pb = g == 0 ? 0 : sc.group_end[g - 1], pe = sc.group_end[g];
        bool first = true;
        for (int pi = pb; pi < pe && ok; ++pi) {
          for (int kb = 0; kb < KB; ++kb) {
            if (!ptx::mbar_wait_bounded(&full[stage], phase, abort_flag, kWaitLimitNs)) { fail(); ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t a_addr = ptx::smem_u32(sA + stage * kABytes);
            const uint32_t b_addr = ptx::smem_u32(sB + stage * kBBytes);
#pragma unroll
            for (int k = 0; k < kKBlock / 16; ++k) {
              const uint64_t ad = ptx::sdesc_kmajor_sw128(a_addr + k * 32);
              const uint64_t bd = ptx::sdesc_kmajor_sw128(b_addr + k * 32);
              ptx::umma_f16(dcol, ad, bd, kIdesc, (first && k == 0) ? 0u : 1u);
            }
            first = false;
            ptx::umma_commit(&empty[stage]);
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
          }
        }
        if (ok) ptx::umma_commit(&tfull[ab]);
      }
      // every MMA this thread issued has completed once `drain` fires
      ptx::umma_commit(drain);
      volatile int never = 0;
      ptx::mbar_wait_bounded(drain, 0, &never, kWaitLimitNs);
    }
  } else {
    // ---------------- epilogue: TMEM -> int64 fixed point -> C ----------------
    const int ew = warp - 2;
    const int q = warp & 3;  // TMEM lanes [32q, 32q+32) are accessible to this warp
    const int half = ew >> 2;
    long long acc[kHalf];
#pragma unroll
    for (int c = 0; c < kHalf; ++c) acc[c] = 0;
    bool ok = true;
    for (int g = 0; g < sc.n_groups; ++g) {
      const int ab = g & 1;
      if (!ptx::mbar_wait_bounded(&tfull[ab], (uint32_t)((g >> 1) & 1), abort_flag, kWaitLimitNs)) {
        fail();
        ok = false;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * NT + half * kHalf);
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        uint32_t v[8];
        ptx::tmem_ld_x8(base + c * 8, v);
        ptx::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[c * 8 + j] += f32_to_fix(__uint_as_float(v[j]));
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[ab]);
    }
    if (ok) {
      const int r = q * 32 + lane;
      const int jp = m0 + r;  // row of C^T
      const bool row_ok = jp < p.n2;
      const int j = jp >> 1, part = jp & 1;
      const int n = p.n2 >> 1;
      const int EB = row_ok ? p.eB[(long long)(p.b_shared ? 0 : b) * n + j] : 1;
      zd* Cb = p.C + p.sC * b;
      const double ar = p.alpha.x, ai = p.alpha.y, br = p.beta.x, bi = p.beta.y;
#pragma unroll
      for (int c = 0; c < kHalf; ++c) {
        const int i = n0 + half * kHalf + c;
        const bool ok_el = row_ok && i < p.m;
        double v = 0.0;
        int EA = 1;
        if (ok_el) {
          EA = p.eA[(long long)(p.a_shared ? 0 : b) * p.m + i];
          // value = acc * 2^-36 * 2^(eA + eB - 14), eA = EA - 1022, eB = EB - 1022
          v = fix_to_double(acc[c], EA + EB - 2044 - 14 - kFixShift);
          if (EA >= 2047 || EB >= 2047) v = __longlong_as_double(0x7ff8000000000000ll);
        }
        double* cp = reinterpret_cast<double*>(Cb + (long long)(ok_el ? i : 0) * p.ldc + (ok_el ? j : 0)) + part;
        if (!p.complex_coef) {
          if (ok_el) {
            double out = ar == 1.0 ? v : (ar == -1.0 ? -v : ar * v);
            if (!p.beta_zero) out = fma(br, *cp, out);
            *cp = out;
          }
        } else {
          // complex alpha / beta: the partner lane (2j vs 2j+1) holds the other component
          const double vo = __shfl_xor_sync(0xffffffffu, v, 1);
          const double re = part ? vo : v, im = part ? v : vo;
          double cre = 0.0, cim = 0.0;
          if (ok_el && !p.beta_zero) {
            const zd old = Cb[(long long)i * p.ldc + j];
            cre = old.x;
            cim = old.y;
          }
          if (ok_el) {
            const double outr = ar * re - ai * im + (p.beta_zero ? 0.0 : br * cre - bi * cim);
            const double outi = ar * im + ai * re + (p.beta_zero ? 0.0 : br * cim + bi * cre);
            *cp = part ? outi : outr;
          }
        }
      }
    }
  }
  // ---------------- teardown ----------------
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 256);
  }
}

// ------------------------------------------------------------------------------------------
// slicing kernels
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int biased_exp(double v) {
  const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  return e == 0 ? 1 : e;
}

// element (r, c) of L = op(X): op N -> X[r][c], op C -> conj(X[c][r])
__device__ __forceinline__ zd load_op(const zd* X, int ld, int op, int r, int c) {
  return op == BT_OP_N ? X[(long long)r * ld + c] : zconj(X[(long long)c * ld + r]);
}

// Row maxima (rows != null) and column maxima (cols != null) of the biased exponents of L
// (R x Kc), tiles of 32 x 32 loaded coalesced for either orientation.
__global__ void exp_max_kernel(int R, int Kc, const zd* __restrict__ X, int ld, long long sX, int op,
                               int* __restrict__ rows, long long sRows, int* __restrict__ cols, long long sCols,
                               const int* __restrict__ active) {
  __shared__ int E[32][33];
  const int b = blockIdx.z;
  if (active && active[b] == 0) return;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const zd* Xb = X + sX * b;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int yy = ty; yy < 32; yy += 8) {
    // coalesced along the stored row: op N reads X[r][c] with c fastest; op C reads X[c][r] with r fastest
    int r, c;
    if (op == BT_OP_N) { r = r0 + yy; c = c0 + tx; } else { r = r0 + tx; c = c0 + yy; }
    int e = 0;
    if (r < R && c < Kc) {
      const zd v = load_op(Xb, ld, op, r, c);
      e = max(biased_exp(v.x), biased_exp(v.y));
    }
    if (op == BT_OP_N) E[yy][tx] = e; else E[tx][yy] = e;
  }
  __syncthreads();
  if (ty == 0) {
    int m = 0;
    if (rows && r0 + tx < R) {
      for (int c = 0; c < 32; ++c) m = max(m, E[tx][c]);
      atomicMax(&rows[sRows * b + r0 + tx], m);
    }
  } else if (ty == 1) {
    int m = 0;
    if (cols && c0 + tx < Kc) {
      for (int r = 0; r < 32; ++r) m = max(m, E[r][tx]);
      atomicMax(&cols[sCols * b + c0 + tx], m);
    }
  }
}

// Digits of |v| * 2^(-eRow) as a fixed-point number with 7S fraction bits (truncated);
// q[s] = sign * d_s * 2^(-7s) (pre-scaled by the slice position).
__device__ __forceinline__ void slice_value(double v, int Erow, int S, float* q) {
  const long long bits = __double_as_longlong(v);
  int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = (unsigned long long)bits & ((1ull << 52) - 1);
  if (E == 0) E = 1; else M |= (1ull << 52);
  const int F = kDigitBits * S;
  const int sh = E - Erow + F - 53;
  unsigned long long X;
  if (sh >= 0) X = M << sh;
  else if (-sh >= 64) X = 0;
  else X = M >> (-sh);
  const float sign = bits < 0 ? -1.0f : 1.0f;
  float scale = sign;
#pragma unroll
  for (int s = 1; s <= kMaxSlices; ++s) {
    if (s <= S) {
      const unsigned d = (unsigned)((X >> (F - kDigitBits * s)) & 127ull);
      q[s - 1] = scale * (float)d;
      scale *= 0.0078125f;  // 2^-7
    }
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// At slices: out[b][s][r][2p + c] for L = op(A) (R x Kc), row exponents erow[b][r].
__global__ void slice_rows_kernel(int R, int Rpad, int Kc, int Kp, const zd* __restrict__ X, int ld, long long sX,
                                  int op, const int* __restrict__ erow, int S, uint32_t* __restrict__ out,
                                  const int* __restrict__ active) {
  __shared__ zd T[32][33];
  const int b = blockIdx.z;
  if (active && active[b] == 0) return;
  const int r0 = blockIdx.y * 32, p0 = blockIdx.x * 32;
  const zd* Xb = X + sX * b;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int yy = ty; yy < 32; yy += 8) {
    int r, c;
    if (op == BT_OP_N) { r = r0 + yy; c = p0 + tx; } else { r = r0 + tx; c = p0 + yy; }
    zd v = zmake(0.0, 0.0);
    if (r < R && c < Kc) v = load_op(Xb, ld, op, r, c);
    if (op == BT_OP_N) T[yy][tx] = v; else T[tx][yy] = v;
  }
  __syncthreads();
  const int Kw = Kp >> 1;  // 32-bit words per output row
  const long long slice_words = (long long)Rpad * Kw;
  for (int yy = ty; yy < 32; yy += 8) {
    const int r = r0 + yy, p = p0 + tx;
    if (r >= Rpad || p >= Kw) continue;
    float qr[kMaxSlices], qi[kMaxSlices];
    const zd v = T[yy][tx];
    const bool in = r < R && p < Kc;  // padding rows / columns are written as zeros
    if (in) {
      const int Er = erow[(long long)b * R + r];
      slice_value(v.x, Er, S, qr);
      slice_value(v.y, Er, S, qi);
    }
    uint32_t* o = out + ((long long)b * S) * slice_words + (long long)r * Kw + p;
    for (int s = 0; s < S; ++s) o[s * slice_words] = in ? pack_bf16x2(qr[s], qi[s]) : 0u;
  }
}

// Bt slices: rows 2j (re) and 2j+1 (im) of out[b][s][2 Ncol][Kp] for L = op(B) (Kc x Ncol),
// column exponents ecol[b][j].
__global__ void slice_cols_kernel(int Kc, int Ncol, int NcolPad, int Kp, const zd* __restrict__ X, int ld,
                                  long long sX, int op, const int* __restrict__ ecol, int S,
                                  uint32_t* __restrict__ out, const int* __restrict__ active) {
  __shared__ zd T[32][33];  // T[j][p]
  const int b = blockIdx.z;
  if (active && active[b] == 0) return;
  const int j0 = blockIdx.y * 32, p0 = blockIdx.x * 32;
  const zd* Xb = X + sX * b;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int yy = ty; yy < 32; yy += 8) {
    // op N: L[p][j] = X[p][j] (coalesced along j);  op C: L[p][j] = conj(X[j][p]) (along p)
    int p, j;
    if (op == BT_OP_N) { p = p0 + yy; j = j0 + tx; } else { p = p0 + tx; j = j0 + yy; }
    zd v = zmake(0.0, 0.0);
    if (p < Kc && j < Ncol) v = load_op(Xb, ld, op, p, j);
    if (op == BT_OP_N) T[tx][yy] = v; else T[yy][tx] = v;
  }
  __syncthreads();
  const int Kw = Kp >> 1;
  const long long slice_words = (long long)2 * NcolPad * Kw;
  for (int yy = ty; yy < 32; yy += 8) {
    const int j = j0 + yy, p = p0 + tx;
    if (j >= NcolPad || p >= Kw) continue;
    float qr[kMaxSlices], qi[kMaxSlices];
    const zd v = T[yy][tx];
    const bool in = j < Ncol && p < Kc;  // padding rows / columns are written as zeros
    if (in) {
      const int Ec = ecol[(long long)b * Ncol + j];
      slice_value(v.x, Ec, S, qr);
      slice_value(v.y, Ec, S, qi);
    }
    uint32_t* o0 = out + ((long long)b * S) * slice_words + (long long)(2 * j) * Kw + p;
    uint32_t* o1 = o0 + Kw;
    for (int s = 0; s < S; ++s) {
      o0[s * slice_words] = in ? pack_bf16x2(qr[s], -qi[s]) : 0u;
      o1[s * slice_words] = in ? pack_bf16x2(qi[s], qr[s]) : 0u;
    }
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encode() {
  std::call_once(g_encode_once, []() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

bool encode_slices_map(CUtensorMap* map, void* base, int Kp, int rows, int depth, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)depth};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)kKBlock, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

Schedule make_schedule(int S) {
  Schedule sc{};
  int np = 0, ng = 0;
  // exact single-pair groups up to s + t = dx; the shared group's fp32 rounding (~2^-24 of
  // terms scaled by 2^-7(dx-1)) then stays below the slicing error for every S
  const int dx = S - 1 > kExactD ? S - 1 : kExactD;
  for (int d = 2; d <= dx && d <= S + 1; ++d)
    for (int s = 1; s <= S; ++s) {
      const int t = d - s;
      if (t < 1 || t > S) continue;
      sc.s[np] = (unsigned char)s;
      sc.t[np] = (unsigned char)t;
      ++np;
      sc.group_end[ng++] = (unsigned char)np;
    }
  const int np0 = np;
  for (int d = dx + 1; d <= S + 1; ++d)
    for (int s = 1; s <= S; ++s) {
      const int t = d - s;
      if (t < 1 || t > S) continue;
      sc.s[np] = (unsigned char)s;
      sc.t[np] = (unsigned char)t;
      ++np;
    }
  if (np > np0) sc.group_end[ng++] = (unsigned char)np;
  sc.n_pairs = np;
  sc.n_groups = ng;
  return sc;
}

int pick_nt(int m) {
  // Cost of one K=16 step of a 128 x NT tile: the MMA needs NT/2 clocks of tensor work and
  // reads (128 + NT) x 32 bytes of shared memory at ~128 B/clock, so the step costs
  // max(NT/2, 32 + NT/4) clocks.  Pick the N tile (multiple of 16, <= 128) that minimises
  // tiles x step cost for the m columns (e.g. m = 416 -> 112: 4 tiles, 7 % padding).
  int best = 16;
  double best_cost = 1e30;
  for (int nt = 128; nt >= 16; nt -= 16) {
    const int tiles = (m + nt - 1) / nt;
    const double step = nt / 2.0 > 32.0 + nt / 4.0 ? nt / 2.0 : 32.0 + nt / 4.0;
    const double cost = tiles * step;
    if (cost < best_cost - 1e-9) { best_cost = cost; best = nt; }
  }
  return best;
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct SplitWs {
  int *eA, *eB;
  uint32_t *At, *Bt;
};

int pad_k(int kc) { return ((2 * kc + kKBlock - 1) / kKBlock) * kKBlock; }
int pad_rows_n(int m, int nt) { return ((m + nt - 1) / nt) * nt; }
int pad_rows_m(int n) { return ((2 * n + kTileM - 1) / kTileM) * kTileM; }

size_t carve_ws(char* base, int m, int n, int kc, int S, int batch, SplitWs* w) {
  const int Kp = pad_k(kc);
  const int mp = pad_rows_n(m, pick_nt(m)), n2p = pad_rows_m(n);
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += al256(bytes); return p; };
  w->eA = reinterpret_cast<int*>(take(sizeof(int) * (size_t)batch * m));
  w->eB = reinterpret_cast<int*>(take(sizeof(int) * (size_t)batch * n));
  w->At = reinterpret_cast<uint32_t*>(take((size_t)batch * S * mp * Kp * 2));
  w->Bt = reinterpret_cast<uint32_t*>(take((size_t)batch * S * n2p * Kp * 2));
  return off;
}

template <int NT>
bt_status launch_mma(cudaStream_t st, const CUtensorMap& mA, const CUtensorMap& mB, const MmaParams& p, int batch) {
  const size_t smem = 1024 + (size_t)kStages * (kTileM * 128 + NT * 128) + 256;
  // per-function device state: set once per device (the value never changes for one NT)
  static std::mutex mu;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BT_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr_set[dev]) {
      if (cudaFuncSetAttribute(split_mma_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return BT_ERR_CUDA;
      attr_set[dev] = true;
    }
  }
  dim3 grid((p.n2 + kTileM - 1) / kTileM, (p.m + NT - 1) / NT, batch);
  split_mma_kernel<NT><<<grid, kThreads, smem, st>>>(mA, mB, p);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status launch_mma_nt(int nt, cudaStream_t st, const CUtensorMap& mA, const CUtensorMap& mB, const MmaParams& p,
                        int batch) {
  switch (nt) {
    case 16: return launch_mma<16>(st, mA, mB, p, batch);
    case 32: return launch_mma<32>(st, mA, mB, p, batch);
    case 48: return launch_mma<48>(st, mA, mB, p, batch);
    case 64: return launch_mma<64>(st, mA, mB, p, batch);
    case 80: return launch_mma<80>(st, mA, mB, p, batch);
    case 96: return launch_mma<96>(st, mA, mB, p, batch);
    case 112: return launch_mma<112>(st, mA, mB, p, batch);
    case 128: return launch_mma<128>(st, mA, mB, p, batch);
    default: return BT_ERR_UNSUPPORTED;
  }
}

constexpr int kMaxKc = 512;  // complex k per launch: K' = 2k <= 1024 <= 1040 (exact slice products)

}  // namespace

size_t split_workspace_bytes(int m, int n, int k, int slices, int batch) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return 0;
  const int S = slices > 0 ? slices : 6;
  const int kc = k < kMaxKc ? k : kMaxKc;
  SplitWs w;
  return carve_ws(nullptr, m, n, kc, S, batch, &w);
}

bt_status split_zgemm(cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta, zd* C, int ldc,
                      long long strideC, int batch, int slices, void* ws, size_t ws_bytes, const int* active) {
  const int S = slices > 0 ? slices : 6;
  if (S < 2 || S > kMaxSlices) return BT_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (m == 0 || n == 0 || batch == 0) return BT_OK;
  if (batch > 65535) return BT_ERR_INVALID_ARG;
  if (k == 0) {
    if (beta.x == 0.0 && beta.y == 0.0) {
      for (int b = 0; b < batch; ++b)
        BT_CUDA_TRY(cudaMemset2DAsync(C + strideC * b, sizeof(zd) * ldc, 0, sizeof(zd) * n, m, st));
      return BT_OK;
    }
    return zgemm(st, m, n, 0, alpha, A, B, beta, C, ldc, strideC, batch, active);  // C = beta C
  }
  if (!ws || ws_bytes < split_workspace_bytes(m, n, k, S, batch)) return BT_ERR_INVALID_ARG;
  if (!get_encode()) return BT_ERR_UNSUPPORTED;
  // K' = 2k must stay <= 1040 per launch for exact slice products: chunk k, accumulate into C
  for (int k0 = 0; k0 < k; k0 += kMaxKc) {
    const int kc = (k - k0) < kMaxKc ? (k - k0) : kMaxKc;
    const int Kp = pad_k(kc);
    const int nt = pick_nt(m);
    const int mp = pad_rows_n(m, nt), n2p = pad_rows_m(n);
    SplitWs w;
    carve_ws(static_cast<char*>(ws), m, n, kc, S, batch, &w);
    Operand a = A, bop = B;
    a.p = A.op == BT_OP_N ? A.p + k0 : A.p + (long long)k0 * A.ld;
    bop.p = B.op == BT_OP_N ? B.p + (long long)k0 * B.ld : B.p + k0;
    // an operand shared by every batch entry (stride 0, e.g. a Hamiltonian block) is sliced once
    const bool a_shared = A.stride == 0 && batch > 1, b_shared = B.stride == 0 && batch > 1;
    const int ba = a_shared ? 1 : batch, bb = b_shared ? 1 : batch;
    const int* act_a = a_shared ? nullptr : active;
    const int* act_b = b_shared ? nullptr : active;
    BT_CUDA_TRY(cudaMemsetAsync(w.eA, 0, sizeof(int) * (size_t)ba * m, st));
    BT_CUDA_TRY(cudaMemsetAsync(w.eB, 0, sizeof(int) * (size_t)bb * n, st));
    {
      dim3 g((kc + 31) / 32, (m + 31) / 32, ba);
      exp_max_kernel<<<g, 256, 0, st>>>(m, kc, a.p, a.ld, a.stride, a.op, w.eA, m, nullptr, 0, act_a);
      count_launch();
      dim3 g2((n + 31) / 32, (kc + 31) / 32, bb);
      exp_max_kernel<<<g2, 256, 0, st>>>(kc, n, bop.p, bop.ld, bop.stride, bop.op, nullptr, 0, w.eB, n, act_b);
      count_launch();
      BT_CUDA_TRY(cudaGetLastError());
    }
    {
      dim3 g((Kp / 2 + 31) / 32, (mp + 31) / 32, ba);
      slice_rows_kernel<<<g, 256, 0, st>>>(m, mp, kc, Kp, a.p, a.ld, a.stride, a.op, w.eA, S, w.At, act_a);
      count_launch();
      dim3 g2((Kp / 2 + 31) / 32, (n2p / 2 + 31) / 32, bb);
      slice_cols_kernel<<<g2, 256, 0, st>>>(kc, n, n2p / 2, Kp, bop.p, bop.ld, bop.stride, bop.op, w.eB, S, w.Bt,
                                            act_b);
      count_launch();
      BT_CUDA_TRY(cudaGetLastError());
    }
    CUtensorMap mA, mB;
    if (!encode_slices_map(&mA, w.Bt, Kp, n2p, batch * S, kTileM)) return BT_ERR_CUDA;
    if (!encode_slices_map(&mB, w.At, Kp, mp, batch * S, nt)) return BT_ERR_CUDA;
    MmaParams p{};
    p.m = m;
    p.n2 = 2 * n;
    p.Kp = Kp;
    p.S = S;
    p.eA = w.eA;
    p.eB = w.eB;
    p.C = C;
    p.ldc = ldc;
    p.sC = strideC;
    p.alpha = alpha;
    p.beta = k0 == 0 ? beta : zmake(1.0, 0.0);
    p.beta_zero = (p.beta.x == 0.0 && p.beta.y == 0.0) ? 1 : 0;
    p.complex_coef = (p.alpha.y != 0.0 || p.beta.y != 0.0) ? 1 : 0;
    p.err = nullptr;
    p.active = active;
    p.a_shared = a_shared ? 1 : 0;
    p.b_shared = b_shared ? 1 : 0;
    p.sched = make_schedule(S);
    BT_TRY(launch_mma_nt(nt, st, mA, mB, p, batch));
  }
  return BT_OK;
}

}  // namespace bt

extern "C" bt_status bt_split_zgemm_workspace_bytes(int m, int n, int k, int slices, int batch, size_t* bytes) {
  if (!bytes || m < 0 || n < 0 || k < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (slices != 0 && (slices < 2 || slices > 8)) return BT_ERR_INVALID_ARG;
  *bytes = bt::split_workspace_bytes(m, n, k, slices, batch);
  return BT_OK;
}

extern "C" bt_status bt_split_zgemm_batched(int m, int n, int k, double alpha_re, double alpha_im, const void* A,
                                            int lda, long long strideA, int opA, const void* B, int ldb,
                                            long long strideB, int opB, double beta_re, double beta_im, void* C,
                                            int ldc, long long strideC, int batch, int slices, void* workspace,
                                            size_t workspace_bytes, void* stream) {
  if ((opA != BT_OP_N && opA != BT_OP_C) || (opB != BT_OP_N && opB != BT_OP_C)) return BT_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || batch < 0) return BT_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && batch > 0 && (!C || (k > 0 && (!A || !B)))) return BT_ERR_INVALID_ARG;
  const int rowsA = opA == BT_OP_N ? k : m;
  const int rowsB = opB == BT_OP_N ? n : k;
  if (lda < (rowsA > 1 ? rowsA : 1) || ldb < (rowsB > 1 ? rowsB : 1) || ldc < (n > 1 ? n : 1))
    return BT_ERR_INVALID_ARG;
  bt::Operand a{static_cast<const zd*>(A), lda, strideA, opA};
  bt::Operand b{static_cast<const zd*>(B), ldb, strideB, opB};
  return bt::split_zgemm(static_cast<cudaStream_t>(stream), m, n, k, zmake(alpha_re, alpha_im), a, b,
                         zmake(beta_re, beta_im), static_cast<zd*>(C), ldc, strideC, batch, slices, workspace,
                         workspace_bytes, nullptr);
}
