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
// Slicing.  Each row i of op(A) is scaled by R_i = 2^(eA_i - 1022) (eA_i = largest biased
// exponent in the row, so every component is below R_i), rounded to a fixed-point integer
// X = round(|v| / R_i * 2^(7S-1)) by integer arithmetic on the IEEE fields, and written as S
// balanced base-128 digits d_1..d_S in [-64, 64] (X = sum_s d_s 128^(S-s)); digit s is stored as
// the bf16 integer sign * d_s.  Columns of op(B) likewise with eB_j.  Then
//     v ~= R * 2^-6 * sum_s d_s 2^(-7(s-1)),
// and a product of digits is an integer of magnitude <= 2^12.
//
// Accumulation.  Pairs (s, t) with s + t <= S + 1 are used.  Over one K segment of at most 960
// real terms, the pairs of one weight class w = s + t - 2 are summed in TMEM fp32 accumulators,
// as many per accumulator as keep its value an integer below 2^24, so the tensor core's fp32
// sum is exact.  An accumulator holding one pair (below 2^22) is drained by adding 1.5 * 2^23
// (one FFMA, which also applies the 2^-p pre-scale of the low-order pairs): the bits of that
// float are then 0x4B400000 + the integer, and one 32 x 32 -> 64-bit multiply-add accumulates
// them with the class weight 2^(F - 7w + p) into a per-thread uint64 fixed-point sum (units of
// 2^-F of a leading digit product, arithmetic mod 2^64); one holding several pairs is converted
// exactly (float -> int32) and added as a signed integer.  The known sum of the 0x4B400000
// biases is subtracted once at the end, giving the exact (to 2^-F) two's-complement value,
// converted to double once per output.
//
// Classes go two by two (w, w + 1) into dual jobs: item t holds the pairs (s, t) and (s + 1, t)
// of the two classes, whose At tiles are adjacent in a pipeline stage and whose accumulators are
// adjacent in TMEM, so one M = 128, N = 2 NT MMA per K step serves both and reads the Bt tile
// once.
//
// Kernel shape: a persistent grid of one CTA per SM walks the 128 x NT output tiles of C^T
// (all batch entries); warp 0 issues TMA loads (3-D tensor maps over [batch*S][rows][K'],
// 128-byte swizzle) through a ring of shared-memory stages, warp 1 issues tcgen05.mma (M = 128,
// N = NT or 2 NT, K = 16) into double-buffered TMEM accumulators, warps 2..17 drain the
// accumulators and write C.  The ring and the accumulators run on across tiles, so the write of one tile overlaps
// the MMAs of the next.  All waits are bounded in time; on a timeout the CTA records
// BT_ERR_TIMEOUT, drains what it issued and frees its TMEM.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <atomic>
#include "bt_common.cuh"
#include "sm103_ptx.cuh"

namespace bt {
namespace {

constexpr int kDigitBits = 7;
constexpr int kMaxSlices = 8;
constexpr int kMaxItems = 128;     // slice pairs (or pair couples) per tile
constexpr int kMaxJobs = 96;       // accumulations rounds (one or two drains each) per tile
constexpr int kSegBlocks = 15;     // K blocks per segment: 15 * 64 = 960 real terms, 960 * 2^12 < 2^22
constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;
constexpr int kTileM = 128;
constexpr int kKBlock = 64;      // bf16 per 128-byte swizzle row
constexpr int kEpiWarps = 16;   // 4 lane quarters x 4 column quarters of the accumulator
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
// measurement hook slots (bt_debug_split_profile): cycles of the MMA issuer waiting for a stage's
// TMA data / for a drained accumulator, its whole loop; the producer waiting for a free stage;
// epilogue warp 0 draining accumulators / writing C; tiles processed
enum ProfSlot : int { kProfMmaWaitFull = 0, kProfMmaWaitAcc, kProfMmaLoop, kProfTmaWaitEmpty, kProfEpiDrain,
                      kProfEpiWrite, kProfTiles, kProfSlots };

// One job = one accumulation round over K blocks [kb0, kb1) and the items [ib, ie), drained once:
//  * dual job: two TMEM accumulators (lanes) fed by items (t, s, s2): the pairs (s, t) and
//    (s2, t) share op(B)'s slice t, so each K block loads the Bt tile once for eight MMAs;
//  * single job: one accumulator summing the pairs (s, t) of its items.
// The pairs summed in one lane have equal weights.
struct Schedule {
  int n_jobs;
  unsigned char dual[kMaxJobs];
  unsigned char ib[kMaxJobs];
  unsigned char ie[kMaxJobs];
  unsigned char kb0[kMaxJobs];
  unsigned char kb1[kMaxJobs];
  unsigned char lsh[kMaxJobs][2];  // weight 2^(F - 7w) > 2^31 (2^30 for cvt): shift, not multiply
  unsigned char cvt[kMaxJobs][2];  // lane sums several pairs (may exceed 2^22): exact float -> int
  uint32_t mult[kMaxJobs][2];      // weight 2^(F - 7w) <= 2^31 (after the pre-scale)
  float fscale[kMaxJobs][2];       // 2^-p: pre-scale of pairs with F - 7w < 0
  unsigned char s[kMaxItems];      // slice of op(A) (1-based), lane 0
  unsigned char s2[kMaxItems];     // slice of op(A), lane 1 of a dual job
  unsigned char t[kMaxItems];      // slice of op(B) (1-based)
};

enum CoefMode : int {
  kCoefUnit = 0,       // alpha = +-1, beta = 0
  kCoefUnitAcc = 1,    // alpha = +-1, beta = 1
  kCoefReal = 2,       // real alpha, real beta
  kCoefComplex = 3,    // alpha or beta complex
};

struct MmaParams {
  int m;          // rows of C (N side of the MMA)
  int n2;         // 2 * columns of C (M side)
  int Kp;         // padded K' (multiple of 64)
  int S;
  int tiles_x;    // tiles along the 2n rows of C^T
  int tiles_y;    // tiles along the m rows of C
  int n_tiles;    // tiles_x * tiles_y * batch
  int pair;       // 1: CTA pairs (cta_group::2), a unit = two M tiles of one N tile
  int tiles_xu;   // units along the 2n rows: tiles_x, or ceil(tiles_x / 2) for pairs
  int n_units;    // tiles_xu * tiles_y * batch
  const int* eA;  // [batch][m] biased exponents of op(A) rows
  const int* eB;  // [batch][n] biased exponents of op(B) columns
  zd* C;
  int ldc;
  long long sC;
  zd alpha, beta;
  int coef_mode;
  int negate;                 // alpha = -1 (kCoefUnit / kCoefUnitAcc)
  unsigned long long bias;    // sum over groups of kMagicBits * weight (mod 2^64)
  int fix_bits;               // F: fixed-point units of 2^-F of a leading digit product
  int* err;          // error slots (may be null): batch entry b writes err[b * err_stride]
  long long err_stride;
  unsigned long long stall_ns;  // test hook: the MMA warp first waits this long on a barrier
                                // that nothing completes (0: off)
  unsigned long long* prof;     // measurement hook (may be null): SM clock cycles accumulated
                                // over all CTAs, see kProf* (counted by the PROF instantiations)
  const int* active; // batch entries with active[b] == 0 are skipped (may be null)
  int a_shared;      // op(A) / op(B) shared by every batch entry: sliced once (batch index 0)
  int b_shared;
  Schedule sched;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// int64 fixed-point value v * 2^e -> double: one hardware conversion (rounded to nearest even),
// then the power of two added to the exponent field (ldexp only when the result would leave the
// normal range).  About a tenth of the integer instructions of a software normalisation, which
// matters where the write of C dominates (short K).
__device__ __forceinline__ double fix_to_double(long long v, int e) {
  const double d = __ll2double_rn(v);
  const long long bits = __double_as_longlong(d);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return d;  // v == 0
  const int ne = ex + e;
  if (ne <= 0 || ne >= 2047) return ldexp(d, e);
  return __longlong_as_double(bits + ((long long)e << 52));
}

// Pipeline depth for an N tile: as many stages as fit in 227 KB of shared memory next to the
// 1 KB alignment pad and the barriers, at most 8.  A stage holds the Bt tile (128 rows) and the At
// rows of this CTA: both At tiles of a dual job on one CTA, one of them on each CTA of a pair.
__host__ __device__ constexpr int stage_bytes_for(int nt, int pair) {
  // pair 2: CTA pairs whose stages hold two K blocks
  return pair == 2 ? 2 * (kTileM * 128 + nt * 128) : kTileM * 128 + (pair ? 1 : 2) * nt * 128;
}
__host__ __device__ constexpr int stages_for(int nt, int pair) {
  return (227 * 1024 - 1024 - 256) / stage_bytes_for(nt, pair) < 8
             ? (227 * 1024 - 1024 - 256) / stage_bytes_for(nt, pair)
             : 8;
}
__host__ __device__ constexpr size_t smem_for(int nt, int pair) {
  return 1024 + (size_t)stages_for(nt, pair) * stage_bytes_for(nt, pair) + 256;
}

// Work unit u of a batched launch -> (rows of C^T, rows of C, batch entry) of this CTA; false for
// inactive entries.  One CTA: a unit is one 128 x NT tile.  A CTA pair: a unit is two M tiles
// (rows m0 and m0 + 128 of C^T, one per CTA of the pair) of the same N tile.
__device__ __forceinline__ bool unit_coords(const MmaParams& p, int nt, int u, int rank, int& m0, int& n0, int& b) {
  const int per_b = p.tiles_xu * p.tiles_y;
  b = u / per_b;
  const int r = u - b * per_b;
  const int ty = r / p.tiles_xu;
  const int tx = r - ty * p.tiles_xu;
  m0 = (p.pair ? 2 * tx + rank : tx) * kTileM;
  n0 = ty * nt;
  return !p.active || p.active[b] != 0;
}

template <int NT, int PAIR, bool PROF>
__global__ void __launch_bounds__(kThreads, 1)
    split_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmBh, const MmaParams p) {
  constexpr int kABytes = kTileM * 128;
  constexpr int kBBytes = NT * 128;
  // PAIR: 0 one CTA per tile; 1 CTA pairs; 2 CTA pairs with two K blocks per pipeline stage
  constexpr bool PAIRED = PAIR != 0;
  constexpr int KPS = PAIR == 2 ? 2 : 1;  // K blocks per stage
  constexpr int kStages = stages_for(NT, PAIR);
  constexpr int kStageBytes = stage_bytes_for(NT, PAIR);
  constexpr int kCols = NT / (kEpiWarps / 4);  // accumulator columns per epilogue thread
  constexpr int kWB = 4;  // outputs per write chunk (kCols is a multiple of 4)
  static_assert(kCols % 4 == 0, "accumulator columns per thread: a multiple of 4");
  static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "UMMA N");
  static_assert(4 * NT <= 512, "two double-buffered accumulator pairs must fit in TMEM");
  // one CTA: M = 128; a pair: M = 256, rows 0..127 in the leader (rank 0), 128..255 in its peer
  constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(PAIRED ? 2 * kTileM : kTileM, NT);
  constexpr uint32_t kIdesc2 = ptx::idesc_bf16_f32(PAIRED ? 2 * kTileM : kTileM, 2 * NT);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  // stage: Bt tile (A operand) + the At rows of this CTA (B operand)
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = PAIRED ? (int)ptx::cluster_ctarank() : 0;
  const bool leader = rank == 0;
  const int cta_unit0 = PAIRED ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;  // first unit of this CTA
  const int unit_step = PAIRED ? (int)(gridDim.x >> 1) : (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      // the leader's MMA reuses an accumulator once the epilogues of both CTAs drained it
      ptx::mbar_init(&tempty[a], PAIRED ? 2 * kEpiWarps : kEpiWarps);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 1) {
    if constexpr (PAIRED) {
      ptx::tmem_alloc_pair(tmem_slot, 512);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(tmem_slot, 512);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  // a pair: the peer's barriers and tensor memory exist before any copy or MMA targets them
  // (the cluster barrier is warp-aligned: every warp arrives converged)
  if constexpr (PAIRED) {
    __syncwarp();
    ptx::cluster_sync_all();
  } else {
    __syncthreads();
  }
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const Schedule& sc = p.sched;
  // every role of both CTAs walks the same units in the same order and skips the same entries
  auto fail = [&](int b) {
    *abort_flag = 1;
    if constexpr (PAIRED) {  // stop the peer too (its shared memory lives until the final barrier)
      const uint32_t peer = ptx::mapa_shared(ptx::smem_u32((const void*)abort_flag), (uint32_t)(rank ^ 1));
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer), "r"(1) : "memory");
    }
    if (p.err) atomicCAS(&p.err[(long long)b * p.err_stride], 0, (int)BT_ERR_TIMEOUT);
  };
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if constexpr (PAIRED) return ptx::mbar_wait_bounded_cluster(bar, parity, abort_flag, kWaitLimitNs);
    else return ptx::mbar_wait_bounded(bar, parity, abort_flag, kWaitLimitNs);
  };

  if (warp == 0) {
    // ---------------- TMA producer (each CTA loads its own rows) ----------------
    if (lane == 0) {
      ptx::prefetch_tensormap(&tmA);
      ptx::prefetch_tensormap(&tmB);
      if constexpr (PAIRED) ptx::prefetch_tensormap(&tmBh);
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      bool ok = true;
      long long t_empty = 0;
      for (int u = cta_unit0; u < p.n_units && ok; u += unit_step) {
        int m0, n0, b;
        if (!unit_coords(p, NT, u, rank, m0, n0, b)) continue;
        const int zA = (p.b_shared ? 0 : b) * p.S - 1, zB = (p.a_shared ? 0 : b) * p.S - 1;
        for (int g = 0; g < sc.n_jobs && ok; ++g) {
          const bool dual = sc.dual[g] != 0;
          // bytes landing in this CTA per stage; a pair's leader expects both CTAs' bytes
          const uint32_t own = (uint32_t)(kABytes + (PAIRED ? (dual ? kBBytes : kBBytes / 2)
                                                          : (dual ? 2 : 1) * kBBytes));
          const int ie = sc.ie[g], kb0 = sc.kb0[g], kb1 = sc.kb1[g];
          for (int it = sc.ib[g]; it < ie && ok; ++it) {
            const int ct = zA + sc.t[it], cs = zB + sc.s[it], cs2 = zB + sc.s2[it];
            for (int kb = kb0; kb < kb1; kb += KPS) {
              const int nk = (KPS == 2 && kb + 1 < kb1) ? 2 : 1;  // K blocks in this stage
              const long long c0 = PROF ? clock64() : 0;
              if (!wait(&empty[stage], phase ^ 1u)) {
                fail(b);
                ok = false;
                break;
              }
              if constexpr (PROF) t_empty += clock64() - c0;
              uint8_t* st = stages + stage * kStageBytes;
              if constexpr (PAIRED) {
                // stage: the Bt tiles of its K blocks, then their At tiles
                const uint32_t fb = ptx::mapa_shared(ptx::smem_u32(&full[stage]), 0u);  // the leader's
                if (leader) ptx::mbar_arrive_expect_tx(&full[stage], 2u * own * (uint32_t)nk);
                for (int h = 0; h < nk; ++h) {
                  const int kx = (kb + h) * kKBlock;
                  uint8_t* sb = st + KPS * kABytes + h * kBBytes;
                  ptx::tma_load_3d_pair(st + h * kABytes, &tmA, fb, kx, m0, ct);
                  if (dual) ptx::tma_load_3d_pair(sb, &tmB, fb, kx, n0, leader ? cs : cs2);
                  else ptx::tma_load_3d_pair(sb, &tmBh, fb, kx, n0 + rank * (NT / 2), cs);
                }
              } else {
                ptx::mbar_arrive_expect_tx(&full[stage], own);
                ptx::tma_load_3d(st, &tmA, &full[stage], kb * kKBlock, m0, ct);
                ptx::tma_load_3d(st + kABytes, &tmB, &full[stage], kb * kKBlock, n0, cs);
                if (dual) ptx::tma_load_3d(st + kABytes + kBBytes, &tmB, &full[stage], kb * kKBlock, n0, cs2);
              }
              ++issued;
              if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
          }
        }
      }
      if constexpr (PROF) atomicAdd(&p.prof[kProfTmaWaitEmpty], (unsigned long long)t_empty);
      if (*abort_flag) {
        // let the loads already in flight land before the CTA exits (bounded): one CTA waits for
        // its last stages' barriers; a pair's copies signal the leader, so both wait a while
        volatile int never = 0;
        if (!PAIRED) {
          for (int idx = issued > kStages ? issued - kStages : 0; idx < issued; ++idx)
            ptx::mbar_wait_bounded(&full[idx % kStages], (uint32_t)((idx / kStages) & 1), &never, kWaitLimitNs);
        } else {
          const uint64_t t0 = ptx::globaltimer_ns();
          while (ptx::globaltimer_ns() - t0 < 2000000ull && !never) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one CTA's, or the pair leader's) ----------------
    if (lane == 0 && leader) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t gc = 0;  // jobs started so far (all units)
      bool ok = true;
      long long t_full = 0, t_acc = 0, tiles = 0;
      // shared-memory descriptors of the current stage, kept as their low words (the start
      // address field, units of 16 bytes, and the leading byte offset) and advanced by adds: the
      // issuing thread's instructions per K block bound the tensor pipe's rate next to the
      // epilogue warps, so the loop below carries as few as possible
      const uint64_t d_stage0 = ptx::sdesc_kmajor_sw128(ptx::smem_u32(stages));
      const uint32_t d_hi = (uint32_t)(d_stage0 >> 32), a_lo0 = (uint32_t)d_stage0;
      constexpr uint32_t kStageLo = (uint32_t)kStageBytes >> 4, kBLo = (uint32_t)kABytes >> 4;
      uint32_t a_lo = a_lo0;
      const long long t_loop0 = PROF ? clock64() : 0;
      if (p.stall_ns) {
        // test hook: wait on `drain`, which nothing completes before the commit below, so the
        // bounded wait expires and the CTA takes its timeout path (abort, drain, free TMEM)
        for (int u = cta_unit0; u < p.n_units; u += unit_step) {
          int m0, n0, b;
          if (!unit_coords(p, NT, u, rank, m0, n0, b)) continue;
          if (!ptx::mbar_wait_bounded(drain, 0, abort_flag, p.stall_ns)) {
            fail(b);
            ok = false;
          }
          break;
        }
      }
      for (int u = cta_unit0; u < p.n_units && ok; u += unit_step) {
        int m0, n0, b;
        if (!unit_coords(p, NT, u, rank, m0, n0, b)) continue;
        ++tiles;
        for (int g = 0; g < sc.n_jobs && ok; ++g, ++gc) {
          const uint32_t ab = gc & 1u;
          const long long ca = PROF ? clock64() : 0;
          if (gc >= 2 && !wait(&tempty[ab], ((gc >> 1) - 1u) & 1u)) {
            fail(b);
            ok = false;
            break;
          }
          if constexpr (PROF) t_acc += clock64() - ca;
          ptx::tc_fence_after();
          const uint32_t dcol0 = tmem + (2u * ab) * (uint32_t)NT;
          // a dual job's two At tiles form one 2NT-row B operand (side by side in this CTA's
          // stage, or one per CTA of a pair) and its two accumulators sit side by side in TMEM:
          // one MMA with N = 2 NT per K step reads the Bt tile once for both lanes
          const uint32_t idesc = sc.dual[g] != 0 ? kIdesc2 : kIdesc;
          const int ie = sc.ie[g], kb0 = sc.kb0[g], kb1 = sc.kb1[g];
          uint32_t acc0 = 0u;  // the job's first MMA overwrites the accumulators
          for (int it = sc.ib[g]; it < ie && ok; ++it) {
            for (int kb = kb0; kb < kb1; kb += KPS) {
              const int nk = (KPS == 2 && kb + 1 < kb1) ? 2 : 1;  // K blocks in this stage
              const long long cf = PROF ? clock64() : 0;
              if (!wait(&full[stage], phase)) {
                fail(b);
                ok = false;
                break;
              }
              if constexpr (PROF) t_full += clock64() - cf;
              ptx::tc_fence_after();
              // K step k starts 32 bytes further: +2 in the descriptor's address field (stage
              // addresses are below 256 KB, so the 14-bit field cannot carry into the next one)
#pragma unroll
              for (int h = 0; h < KPS; ++h) {
                if (h < nk) {
                  const uint32_t alo = a_lo + (uint32_t)h * kBLo;
                  const uint32_t blo = a_lo + (uint32_t)KPS * kBLo + (uint32_t)h * ((uint32_t)kBBytes >> 4);
#pragma unroll
                  for (int k = 0; k < kKBlock / 16; ++k) {
                    const uint64_t ad = ((uint64_t)d_hi << 32) | (uint64_t)(alo + 2u * k);
                    const uint64_t bd = ((uint64_t)d_hi << 32) | (uint64_t)(blo + 2u * k);
                    const uint32_t acc = (h == 0 && k == 0) ? acc0 : 1u;
                    if constexpr (PAIRED)
                      ptx::umma_f16_pair(dcol0, ad, bd, idesc, acc);
                    else
                      ptx::umma_f16(dcol0, ad, bd, idesc, acc);
                  }
                }
              }
              acc0 = 1u;
              if constexpr (PAIRED) ptx::umma_commit_pair_mc(&empty[stage], (uint16_t)0x3);
              else ptx::umma_commit(&empty[stage]);
              if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
                a_lo = a_lo0;
              } else {
                a_lo += kStageLo;
              }
            }
          }
          if (ok) {
            if constexpr (PAIRED) ptx::umma_commit_pair_mc(&tfull[ab], (uint16_t)0x3);
            else ptx::umma_commit(&tfull[ab]);
          }
        }
      }
      // every MMA this thread issued has completed once `drain` fires
      if constexpr (PAIRED) ptx::umma_commit_pair_mc(drain, (uint16_t)0x1);
      else ptx::umma_commit(drain);
      volatile int never = 0;
      ptx::mbar_wait_bounded(drain, 0, &never, kWaitLimitNs);
      if constexpr (PROF) {
        atomicAdd(&p.prof[kProfMmaWaitFull], (unsigned long long)t_full);
        atomicAdd(&p.prof[kProfMmaWaitAcc], (unsigned long long)t_acc);
        atomicAdd(&p.prof[kProfMmaLoop], (unsigned long long)(clock64() - t_loop0));
        atomicAdd(&p.prof[kProfTiles], (unsigned long long)tiles);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> uint64 fixed point -> C (each CTA its own rows) ----------
    const int ew = warp - 2;
    const int q = warp & 3;  // TMEM lanes [32q, 32q+32) are accessible to this warp
    const int cq = ew >> 2;  // column quarter
    const int r = q * 32 + lane;
    uint32_t gc = 0;
    bool ok = true;
    long long t_drain = 0, t_write = 0;
    for (int u = cta_unit0; u < p.n_units && ok; u += unit_step) {
      int m0, n0, b;
      if (!unit_coords(p, NT, u, rank, m0, n0, b)) continue;
      unsigned long long acc[kCols];
#pragma unroll
      for (int c = 0; c < kCols; ++c) acc[c] = 0ull;
      for (int g = 0; g < sc.n_jobs; ++g, ++gc) {
        const uint32_t ab = gc & 1u;
        const bool got = wait(&tfull[ab], (gc >> 1) & 1u);
        // the warp-collective tcgen05.ld below needs every lane: one lane's timeout stops the warp
        if (!__all_sync(0xffffffffu, got)) {
          if (!got) fail(b);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const long long cd = PROF ? clock64() : 0;
        const int lanes = sc.dual[g] ? 2 : 1;
        for (int l = 0; l < lanes; ++l) {
          const float fs = sc.fscale[g][l];
          const uint32_t mu = sc.mult[g][l];
          const int lsh = sc.lsh[g][l];
          const bool cvt = sc.cvt[g][l] != 0;
          const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (2u * ab + (uint32_t)l) * (uint32_t)NT +
                                (uint32_t)(cq * kCols);
#pragma unroll
          // 8 columns per tcgen05.ld (and per wait), a last load of 4 when kCols is not a multiple
          // of 8: the fewer instructions the epilogue warps issue, the less they slow the MMA issuer
          auto add_cols = [&](int c0, const uint32_t* v, int w) {
            if (cvt) {
              // several pairs: an integer below 2^24, pre-scaled and rounded to int32 (exact for
              // the classes of weight >= 2^-F, as in the FFMA path otherwise)
              if (lsh == 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                  if (c < w) {
                    const int iv = __float2int_rn(__uint_as_float(v[c]) * fs);
                    acc[c0 + c] += (unsigned long long)((long long)iv * (long long)(int)mu);
                  }
                }
              } else {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                  if (c < w) acc[c0 + c] += (unsigned long long)(long long)__float2int_rn(__uint_as_float(v[c])) << lsh;
              }
            } else if (lsh == 0) {
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                if (c < w) {
                  const float t = fmaf(__uint_as_float(v[c]), fs, kMagic);
                  acc[c0 + c] += (unsigned long long)__float_as_uint(t) * (unsigned long long)mu;
                }
              }
            } else {
#pragma unroll
              for (int c = 0; c < 8; ++c)
                if (c < w) acc[c0 + c] += (unsigned long long)__float_as_uint(__uint_as_float(v[c]) + kMagic) << lsh;
            }
          };
#pragma unroll
          for (int c0 = 0; c0 + 8 <= kCols; c0 += 8) {
            uint32_t v[8];
            ptx::tmem_ld_x8(base + c0, v);
            ptx::tmem_wait_ld();
            add_cols(c0, v, 8);
          }
          if constexpr (kCols % 8 != 0) {
            constexpr int c0 = kCols - 4;
            uint32_t v[8];
            ptx::tmem_ld_x4(base + c0, v);
            ptx::tmem_wait_ld();
            add_cols(c0, v, 4);
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIRED) ptx::mbar_arrive_remote(ptx::mapa_shared(ptx::smem_u32(&tempty[ab]), 0u));
          else ptx::mbar_arrive(&tempty[ab]);
        }
        if constexpr (PROF) t_drain += clock64() - cd;
      }
      if (!ok) break;
      const long long cw = PROF ? clock64() : 0;
      // write this tile of C (overlaps the MMAs of the next tile)
      const int jp = m0 + r;  // row of C^T
      const bool row_ok = jp < p.n2;
      const int j = jp >> 1, part = jp & 1;
      const int n = p.n2 >> 1;
      const int EB = row_ok ? p.eB[(long long)(p.b_shared ? 0 : b) * n + j] : 1;
      zd* Cb = p.C + p.sC * b;
      const int* eAb = p.eA + (long long)(p.a_shared ? 0 : b) * p.m;
      const bool need_old = p.coef_mode == kCoefUnitAcc || (p.coef_mode == kCoefReal && p.beta.x != 0.0);
      // chunks of kWB outputs: every load of a chunk (exponents, old C) is issued before its
      // stores, so the loads overlap instead of waiting one by one behind possibly aliasing stores
#pragma unroll
      for (int c0 = 0; c0 < kCols; c0 += kWB) {
        int ea[kWB];
        double old[kWB];
#pragma unroll
        for (int u = 0; u < kWB; ++u) {
          const int i = n0 + cq * kCols + c0 + u;
          const bool ok_el = row_ok && i < p.m;
          ea[u] = ok_el ? eAb[i] : 1;
          old[u] = (need_old && ok_el) ? reinterpret_cast<const double*>(Cb + (long long)i * p.ldc + j)[part] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kWB; ++u) {
          const int c = c0 + u;
          const int i = n0 + cq * kCols + c;
          const bool ok_el = row_ok && i < p.m;
          double v = 0.0;
          if (ok_el) {
            const int EA = ea[u];
            long long a = (long long)(acc[c] - p.bias);
            if (p.negate) a = -a;
            // value = a * 2^-F * R_A * R_B * 2^-12, R = 2^(E - 1022)
            v = fix_to_double(a, EA + EB - 2044 - 12 - p.fix_bits);
            if (EA >= 2047 || EB >= 2047) v = __longlong_as_double(0x7ff8000000000000ll);
          }
          double* cp = reinterpret_cast<double*>(Cb + (long long)(ok_el ? i : 0) * p.ldc + (ok_el ? j : 0)) + part;
          if (p.coef_mode == kCoefUnit) {
            if (ok_el) *cp = v;
          } else if (p.coef_mode == kCoefUnitAcc) {
            if (ok_el) *cp = old[u] + v;
          } else if (p.coef_mode == kCoefReal) {
            if (ok_el) {
              const double out = p.alpha.x * v;
              *cp = p.beta.x == 0.0 ? out : fma(p.beta.x, old[u], out);
            }
          } else {
            // complex alpha / beta: the partner lane (2j vs 2j+1) holds the other component
            const double vo = __shfl_xor_sync(0xffffffffu, v, 1);
            const double re = part ? vo : v, im = part ? v : vo;
            const double ar = p.alpha.x, ai = p.alpha.y, br = p.beta.x, bi = p.beta.y;
            const bool bz = br == 0.0 && bi == 0.0;
            double cre = 0.0, cim = 0.0;
            if (ok_el && !bz) {
              const zd o = Cb[(long long)i * p.ldc + j];
              cre = o.x;
              cim = o.y;
            }
            if (ok_el) {
              const double outr = ar * re - ai * im + (bz ? 0.0 : br * cre - bi * cim);
              const double outi = ar * im + ai * re + (bz ? 0.0 : br * cim + bi * cre);
              *cp = part ? outi : outr;
            }
          }
        }
      }
      if constexpr (PROF) t_write += clock64() - cw;
    }
    if constexpr (PROF) {
      if (ew == 0 && lane == 0) {
        atomicAdd(&p.prof[kProfEpiDrain], (unsigned long long)t_drain);
        atomicAdd(&p.prof[kProfEpiWrite], (unsigned long long)t_write);
      }
    }
  }
  // ---------------- teardown ----------------
  ptx::tc_fence_before();
  if constexpr (PAIRED) {
    // the leader's MMAs write the peer's tensor memory and its commits signal the peer's
    // barriers: both CTAs are done with both before either frees its tensor memory
    __syncwarp();
    ptx::cluster_sync_all();
    if (warp == 1) {
      ptx::tc_fence_after();
      ptx::tmem_dealloc_pair(tmem, 512);
    }
    __syncwarp();
    ptx::cluster_sync_all();  // no CTA leaves while its peer may still address its shared memory
  } else {
    __syncthreads();
    if (warp == 1) {
      ptx::tc_fence_after();
      ptx::tmem_dealloc(tmem, 512);
    }
  }
}

// ------------------------------------------------------------------------------------------
// slicing kernels
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int biased_exp(double v) {
  const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  return e == 0 ? 1 : e;
}

// Balanced base-128 digits of v / R, R = 2^(Erow - 1022):  X = round(|v| / R * 2^(7S-1)) <=
// 2^(7S-1) (integer arithmetic on the IEEE fields), X = sum_s d_s 128^(S-s) with the lower digits
// in [-64, 63] and the leading digit in [0, 64];  q[s-1] = sign * d_s as an exact float, formed
// as (bits 0x4B400000 + d) - 1.5 * 2^23: one integer add and one FADD, no conversion instruction
// (conversions run on GB300's narrow FP64 / conversion pipe).
__device__ __forceinline__ float digit_float(int d) { return __int_as_float(0x4B400000 + d) - 12582912.0f; }
__device__ __forceinline__ void slice_value(double v, int Erow, int S, float* q) {
  const long long bits = __double_as_longlong(v);
  int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = (unsigned long long)bits & ((1ull << 52) - 1);
  if (E == 0) E = 1; else M |= (1ull << 52);
  // X2 = trunc(|v| / R * 2^(7S)) = M * 2^(E - Erow + 7S - 53); one bit beyond X for rounding
  const int sh = E - Erow + kDigitBits * S - 53;
  unsigned long long X2;
  if (sh >= 0) X2 = M << sh;
  else if (-sh >= 64) X2 = 0;
  else X2 = M >> (-sh);
  unsigned long long X = (X2 + 1ull) >> 1;
  const int sg = bits < 0 ? -1 : 1;
#pragma unroll
  for (int s = kMaxSlices; s >= 2; --s) {
    if (s <= S) {
      int d = (int)(X & 127ull);
      X >>= kDigitBits;
      if (d >= 64) { d -= 128; X += 1ull; }  // borrow from the next digit
      q[s - 1] = digit_float(sg * d);
    }
  }
  q[0] = digit_float(sg * (int)X);  // leading digit, <= 64
}

// Two exact small floats -> packed bf16 pair: their upper halves (the low 16 bits are zero).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Slicing works on "lines": the rows of op(A) (At operand) and the columns of op(B) (Bt
// operand), each of Kc complex elements, one exponent per line.  A line is contiguous in memory
// for op(A) = A and op(B) = B^H, strided (a memory column) otherwise.  Output rows hold Kw = Kp/2
// 32-bit words (bf16 pairs) per slice:
//   At: out[b][s][l][p]               = (Re, Im) digits of op(A)[l][p]
//   Bt: out[b][s][2l][p], [2l+1][p]   = (Re, -Im), (Im, Re) digits of op(B)[p][l]
// Words p in [Kc, Kw) are written as zeros; lines in [L, Lpad) are not written (the tensor maps
// end at line L, so TMA fills them with zeros).  The line exponents go to e[b][l].
template <bool kBt>
__device__ __forceinline__ void write_slices(uint32_t* __restrict__ out, long long slice_words, int Kw, int l, int p,
                                             int S, bool in, const float* qr, const float* qi) {
  uint32_t* o0 = out + (long long)(kBt ? 2 * l : l) * Kw + p;
#pragma unroll
  for (int s = 0; s < kMaxSlices; ++s) {
    if (s < S) {
      if (kBt) {
        o0[s * slice_words] = in ? pack_bf16x2(qr[s], -qi[s]) : 0u;
        o0[s * slice_words + Kw] = in ? pack_bf16x2(qi[s], qr[s]) : 0u;
      } else {
        o0[s * slice_words] = in ? pack_bf16x2(qr[s], qi[s]) : 0u;
      }
    }
  }
}

// Contiguous lines: one warp per line, grid (ceil(Lpad / 8), batch), 256 threads.
template <bool kBt>
__global__ void slice_lines_contig_kernel(int L, int Lpad, int Kc, int Kw, const zd* __restrict__ X, int ld,
                                          long long sX, int conj, int S, int* __restrict__ e,
                                          uint32_t* __restrict__ out, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && active[b] == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + warp;
  if (l >= L) return;  // lines in [L, Lpad) are read by TMA as out of range (zeros)
  const bool line_ok = true;
  const zd* line = X + sX * b + (long long)(line_ok ? l : 0) * ld;
  int E = 1;
  if (line_ok)
    for (int p = lane; p < Kc; p += 32) {
      const zd v = line[p];
      E = max(E, max(biased_exp(v.x), biased_exp(v.y)));
    }
  E = __reduce_max_sync(0xffffffffu, E);
  if (line_ok && lane == 0) e[(long long)b * L + l] = E;
  const long long slice_words = (long long)(kBt ? 2 : 1) * Lpad * Kw;
  uint32_t* ob = out + (long long)b * S * slice_words;
  for (int p = lane; p < Kw; p += 32) {
    const bool in = line_ok && p < Kc;
    float qr[kMaxSlices], qi[kMaxSlices];
    if (in) {
      const zd v = line[p];
      slice_value(v.x, E, S, qr);
      slice_value(conj ? -v.y : v.y, E, S, qi);
    }
    write_slices<kBt>(ob, slice_words, Kw, l, p, S, in, qr, qi);
  }
}

// Strided lines (memory columns), pass 1: e[b][l] = max biased exponent of line l, as atomicMax
// over CTAs of 32 lines x kExpRows rows (e zeroed before).  Grid (ceil(L / 32), ceil(Kc / kExpRows),
// batch), 256 threads.
constexpr int kExpRows = 64;
__global__ void line_exp_strided_kernel(int L, int Kc, const zd* __restrict__ X, int ld, long long sX,
                                        int* __restrict__ e, const int* __restrict__ active) {
  __shared__ int red[8][32];
  const int b = blockIdx.z;
  if (active && active[b] == 0) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int l = blockIdx.x * 32 + tx, p0 = blockIdx.y * kExpRows;
  const zd* Xb = X + sX * b;
  int E = 1;
  if (l < L)
    for (int p = p0 + ty; p < Kc && p < p0 + kExpRows; p += 8) {
      const zd v = Xb[(long long)p * ld + l];
      E = max(E, max(biased_exp(v.x), biased_exp(v.y)));
    }
  red[ty][tx] = E;
  __syncthreads();
  if (ty == 0 && l < L) {
#pragma unroll
    for (int y = 1; y < 8; ++y) E = max(E, red[y][tx]);
    atomicMax(&e[(long long)b * L + l], E);
  }
}

// Strided lines, pass 2: one 32-line x 32-word tile per CTA (grid (ceil(Lpad / 32), Kw / 32,
// batch), 256 threads): coalesced loads along the memory rows, shared-memory transpose, digits
// written along the output rows.
template <bool kBt>
__global__ void slice_lines_strided_kernel(int L, int Lpad, int Kc, int Kw, const zd* __restrict__ X, int ld,
                                           long long sX, int conj, int S, const int* __restrict__ e,
                                           uint32_t* __restrict__ out, const int* __restrict__ active) {
  __shared__ zd T[32][33];  // T[p][l]
  __shared__ int Eline[32];
  const int b = blockIdx.z;
  if (active && active[b] == 0) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int l0 = blockIdx.x * 32, p0 = blockIdx.y * 32;
  const zd* Xb = X + sX * b;
  if (ty == 0) Eline[tx] = l0 + tx < L ? e[(long long)b * L + l0 + tx] : 1;
  for (int yy = ty; yy < 32; yy += 8) {
    const int p = p0 + yy, l = l0 + tx;
    T[yy][tx] = (p < Kc && l < L) ? Xb[(long long)p * ld + l] : zmake(0.0, 0.0);
  }
  __syncthreads();
  const long long slice_words = (long long)(kBt ? 2 : 1) * Lpad * Kw;
  uint32_t* ob = out + (long long)b * S * slice_words;
  for (int yy = ty; yy < 32; yy += 8) {
    const int l = l0 + yy, p = p0 + tx;
    if (l >= L || p >= Kw) continue;  // lines in [L, Lpad): out of range for TMA, never written
    const bool in = l < L && p < Kc;
    float qr[kMaxSlices], qi[kMaxSlices];
    if (in) {
      const zd v = T[tx][yy];
      slice_value(v.x, Eline[yy], S, qr);
      slice_value(conj ? -v.y : v.y, Eline[yy], S, qi);
    }
    write_slices<kBt>(ob, slice_words, Kw, l, p, S, in, qr, qi);
  }
}

template <bool kBt>
bt_status slice_lines(cudaStream_t st, bool contiguous, int L, int Lpad, int Kc, int Kw, const zd* X, int ld,
                      long long sX, int conj, int S, int* e, uint32_t* out, int batch, const int* active) {
  if (contiguous) {
    dim3 g((L + 7) / 8, batch);
    slice_lines_contig_kernel<kBt><<<g, 256, 0, st>>>(L, Lpad, Kc, Kw, X, ld, sX, conj, S, e, out, active);
  } else {
    BT_CUDA_TRY(cudaMemsetAsync(e, 0, sizeof(int) * (size_t)batch * L, st));
    dim3 ge((L + 31) / 32, (Kc + kExpRows - 1) / kExpRows, batch);
    line_exp_strided_kernel<<<ge, 256, 0, st>>>(L, Kc, X, ld, sX, e, active);
    count_launch();
    dim3 g((L + 31) / 32, Kw / 32, batch);
    slice_lines_strided_kernel<kBt><<<g, 256, 0, st>>>(L, Lpad, Kc, Kw, X, ld, sX, conj, S, e, out, active);
  }
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
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

// rows: the rows that hold data; rows_alloc: the rows allocated per slice (a multiple of the
// tile).  Rows in [rows, rows_alloc) are never written: TMA reads them as zeros (out of range).
bool encode_slices_map(CUtensorMap* map, void* base, int Kp, int rows, int rows_alloc, int depth, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)depth};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows_alloc};
  cuuint32_t box[3] = {(cuuint32_t)kKBlock, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Jobs for every slice pair (s, t) with s + t <= S + 1 over each K segment of L <= kSegBlocks
// blocks (balanced).  A term of a pair's sum is a digit product of magnitude <= 2^12, so n pairs
// over L blocks of 64 real terms sum to an integer below n L 2^18: exact in the fp32 accumulator
// while n L < 64 (below 2^24), and inside the drain's magic-number range (below 2^22) while
// n L < 16.
//  * merged (default): the pairs of one weight class d = s + t share accumulators, up to 63 / L
//    each.  In long segments (L >= 8) classes go two by two (d, d + 1) into dual jobs: item
//    t = 1 .. d - 1 holds the pairs (d - t, t) (lane 0) and (d + 1 - t, t) (lane 1), which share
//    op(B)'s slice t; the pair (1, d) of class d + 1 left over goes into a single job, and so does
//    a class without a partner.  S = 6, L = 13: 7 jobs and 11 drains per tile instead of 12 and
//    21.  In short segments, where the drains outweigh the MMAs, one single job per class (S
//    drains).  Jobs are ordered longest first: a tile's C write overlaps the MMAs of the next
//    tile's first jobs.
//  * one pair per accumulator: in long segments (L >= 8) pairs of equal t and consecutive s go
//    two by two into dual jobs, a leftover pair into a single job; short segments: single jobs
//    summing up to 15 / L pairs of equal weight.
// A pair of weight class d enters the fixed-point sum with factor 2^(F - 7(d - 2)): a shift for
// factors above 2^31 (2^30 for a lane converted to a signed integer), a 32-bit multiplier down
// to 2^0, and below that a pre-scale 2^(F - 7(d - 2)) before the rounding to an integer
// (rounding below 2^-F of a leading digit product).
// F = min(7S - 9, 50 - log2(K')): resolution below the slicing error, and
// |sum| <= K' * 2^12 * 2^F * (1 + 2^-6) < 2^63.
bool make_schedule(int S, int KB, bool merge, Schedule* sc, unsigned long long* bias, int* fix_bits) {
  *sc = Schedule{};
  int lg = 0;
  while ((1 << lg) < KB * kKBlock) ++lg;
  int F = kDigitBits * S - 9;
  if (F > 50 - lg) F = 50 - lg;
  struct Spec {
    int kb0, kb1, dual, n;
    int d[2], cvt[2];
    int s[kMaxSlices], s2[kMaxSlices], t[kMaxSlices];  // a job holds at most S items
  };
  std::vector<Spec> jobs;
  auto open_job = [&](int kb0, int kb1, bool dual, int d0, int d1) -> Spec& {
    Spec j{};
    j.kb0 = kb0;
    j.kb1 = kb1;
    j.dual = dual ? 1 : 0;
    j.d[0] = d0;
    j.d[1] = d1;
    jobs.push_back(j);
    return jobs.back();
  };
  auto add_item = [](Spec& j, int s, int s2, int t) {
    if (j.n >= kMaxSlices) return false;
    j.s[j.n] = s;
    j.s2[j.n] = s2;
    j.t[j.n] = t;
    ++j.n;
    return true;
  };
  const int nseg = (KB + kSegBlocks - 1) / kSegBlocks;
  for (int seg = 0; seg < nseg; ++seg) {
    const int kb0 = (int)((long long)KB * seg / nseg), kb1 = (int)((long long)KB * (seg + 1) / nseg);
    const int L = kb1 - kb0;
    if (merge && L < 8) {
      // short segment: the drains outweigh the MMAs, so one accumulator per class (S drains)
      const int nmax = 63 / L;
      for (int d = 2; d <= S + 1; ++d) {
        Spec* j = nullptr;
        for (int s = 1; s <= S; ++s) {
          const int t = d - s;
          if (t < 1 || t > S) continue;
          if (!j || j->n == nmax) j = &open_job(kb0, kb1, false, d, 0);
          if (!add_item(*j, s, s, t)) return false;
        }
      }
    } else if (merge) {
      const int nmax = 63 / L;
      for (int d = 2; d <= S + 1; d += 2) {
        if (d + 1 <= S + 1) {
          for (int t0 = 1; t0 <= d - 1; t0 += nmax) {
            Spec& j = open_job(kb0, kb1, true, d, d + 1);
            for (int t = t0; t <= d - 1 && t < t0 + nmax; ++t)
              if (!add_item(j, d - t, d + 1 - t, t)) return false;
          }
          Spec& j = open_job(kb0, kb1, false, d + 1, 0);
          if (!add_item(j, 1, 1, d)) return false;
        } else {
          for (int s0 = 1; s0 <= d - 1; s0 += nmax) {
            Spec& j = open_job(kb0, kb1, false, d, 0);
            for (int s = s0; s <= d - 1 && s < s0 + nmax; ++s)
              if (!add_item(j, s, s, d - s)) return false;
          }
        }
      }
    } else if (15 / L == 1) {
      for (int t = 1; t <= S; ++t)
        for (int s = 1; s + t <= S + 1; s += 2) {
          const bool two = s + 1 + t <= S + 1;
          Spec& j = open_job(kb0, kb1, two, s + t, s + 1 + t);
          if (!add_item(j, s, two ? s + 1 : s, t)) return false;
        }
    } else {
      const int per_group = 15 / L;
      for (int d = 2; d <= S + 1; ++d) {
        Spec* j = nullptr;
        for (int s = 1; s <= S; ++s) {
          const int t = d - s;
          if (t < 1 || t > S) continue;
          if (!j || j->n == per_group) j = &open_job(kb0, kb1, false, d, 0);
          if (!add_item(*j, s, s, t)) return false;
        }
      }
    }
  }
  for (Spec& j : jobs) {
    const bool exact_magic = j.n * (j.kb1 - j.kb0) < 16;
    j.cvt[0] = j.cvt[1] = exact_magic ? 0 : 1;
  }
  if (merge)
    std::stable_sort(jobs.begin(), jobs.end(), [](const Spec& a, const Spec& b) {
      return a.n * (a.kb1 - a.kb0) * (1 + a.dual) > b.n * (b.kb1 - b.kb0) * (1 + b.dual);
    });
  if ((int)jobs.size() > kMaxJobs) return false;
  unsigned long long bs = 0;
  int ni = 0;
  for (int g = 0; g < (int)jobs.size(); ++g) {
    const Spec& j = jobs[g];
    if (ni + j.n > kMaxItems) return false;
    sc->dual[g] = (unsigned char)j.dual;
    sc->kb0[g] = (unsigned char)j.kb0;
    sc->kb1[g] = (unsigned char)j.kb1;
    sc->ib[g] = (unsigned char)ni;
    for (int i = 0; i < j.n; ++i, ++ni) {
      sc->s[ni] = (unsigned char)j.s[i];
      sc->s2[ni] = (unsigned char)j.s2[i];
      sc->t[ni] = (unsigned char)j.t[i];
    }
    sc->ie[g] = (unsigned char)ni;
    for (int l = 0; l < 1 + j.dual; ++l) {
      const int e = F - kDigitBits * (j.d[l] - 2);
      const bool cvt = j.cvt[l] != 0;
      const int shift_above = cvt ? 30 : 31;  // a signed int32 multiplier stays below 2^31
      sc->cvt[g][l] = cvt ? 1 : 0;
      sc->lsh[g][l] = (unsigned char)(e > shift_above ? e : 0);
      sc->mult[g][l] = e > shift_above ? 1u : (e >= 0 ? (1u << e) : 1u);
      sc->fscale[g][l] = e >= 0 ? 1.0f : ldexpf(1.0f, e);
      if (!cvt) bs += (unsigned long long)kMagicBits * ((unsigned long long)sc->mult[g][l] << sc->lsh[g][l]);
    }
  }
  sc->n_jobs = (int)jobs.size();
  *bias = bs;
  *fix_bits = F;
  return true;
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

int num_sms() {
  static std::mutex mu;
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (sms[dev] == 0 && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms[dev] = 0;
  return sms[dev];
}

// Clusters of two CTAs of the pair kernel that can be resident at once (per device and N tile).
template <int NT, int PAIR>
int pair_clusters() {
  static std::mutex mu;
  static int val[64];
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return val[dev];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem_for(NT, PAIR);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaFuncSetAttribute(split_mma_kernel<NT, PAIR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_for(NT, PAIR)) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&nc, split_mma_kernel<NT, PAIR, false>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    nc = 0;
  }
  val[dev] = nc;
  done[dev] = true;
  return nc;
}

template <int NT, int PAIR, bool PROF>
bt_status launch_mma(cudaStream_t st, const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mBh,
                     const MmaParams& p) {
  const size_t smem = smem_for(NT, PAIR);
  // per-function device state: set once per device (the value never changes for one NT)
  static std::mutex mu;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BT_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr_set[dev]) {
      if (cudaFuncSetAttribute(split_mma_kernel<NT, PAIR, PROF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem) != cudaSuccess)
        return BT_ERR_CUDA;
      attr_set[dev] = true;
    }
  }
  const int sms = num_sms();
  if (sms <= 0) return BT_ERR_CUDA;
  if constexpr (PAIR != 0) {
    // persistent: as many CTA pairs as can be resident, units walked in order
    const int nc = pair_clusters<NT, PAIR>();
    if (nc <= 0) return BT_ERR_UNSUPPORTED;
    const int clusters = p.n_units < nc ? p.n_units : nc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * clusters));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BT_CUDA_TRY(cudaLaunchKernelEx(&cfg, split_mma_kernel<NT, PAIR, PROF>, mA, mB, mBh, p));
  } else {
    // persistent: one CTA per SM (1 CTA fits per SM by shared memory), tiles walked in order
    const int grid = p.n_units < sms ? p.n_units : sms;
    split_mma_kernel<NT, 0, PROF><<<grid, kThreads, smem, st>>>(mA, mB, mBh, p);
  }
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

template <int PAIR>
bt_status launch_mma_nt(int nt, cudaStream_t st, const CUtensorMap& mA, const CUtensorMap& mB,
                        const CUtensorMap& mBh, const MmaParams& p) {
  // the measurement hook's counters are compiled into the block sizes of the measured workloads
  // only (N tiles of 112 and 128); other launches run uninstrumented
  if (p.prof && nt == 112) return launch_mma<112, PAIR, true>(st, mA, mB, mBh, p);
  if (p.prof && nt == 128) return launch_mma<128, PAIR, true>(st, mA, mB, mBh, p);
  switch (nt) {
    case 16: return launch_mma<16, PAIR, false>(st, mA, mB, mBh, p);
    case 32: return launch_mma<32, PAIR, false>(st, mA, mB, mBh, p);
    case 48: return launch_mma<48, PAIR, false>(st, mA, mB, mBh, p);
    case 64: return launch_mma<64, PAIR, false>(st, mA, mB, mBh, p);
    case 80: return launch_mma<80, PAIR, false>(st, mA, mB, mBh, p);
    case 96: return launch_mma<96, PAIR, false>(st, mA, mB, mBh, p);
    case 112: return launch_mma<112, PAIR, false>(st, mA, mB, mBh, p);
    case 128: return launch_mma<128, PAIR, false>(st, mA, mB, mBh, p);
    default: return BT_ERR_UNSUPPORTED;
  }
}

int pair_clusters_nt(int nt, int pair) {
  switch (nt * 4 + pair) {
#define BT_PAIR_CASE(N)                                 \
  case N * 4 + 1: return pair_clusters<N, 1>();        \
  case N * 4 + 2: return pair_clusters<N, 2>();
    BT_PAIR_CASE(16) BT_PAIR_CASE(32) BT_PAIR_CASE(48) BT_PAIR_CASE(64)
    BT_PAIR_CASE(80) BT_PAIR_CASE(96) BT_PAIR_CASE(112) BT_PAIR_CASE(128)
#undef BT_PAIR_CASE
    default: return 0;
  }
}

// CTA-pair mode (bt_debug_split_pair): 0 = the default rule, 1 = one CTA per tile always,
// 2 = pairs whenever the shape allows them, 3 = pairs with two K blocks per pipeline stage
std::atomic<int> g_pair_mode{0};
std::atomic<int> g_sched_mode{0};  // 0: merged class accumulators, 1: one pair per accumulator

constexpr int kMaxKc = 1024;  // complex k per launch (slice workspace); K' = 2k <= 2048 = 32 K blocks

}  // namespace

size_t split_workspace_bytes(int m, int n, int k, int slices, int batch) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return 0;
  const int S = slices > 0 ? slices : 6;
  const int kc = k < kMaxKc ? k : kMaxKc;
  SplitWs w;
  return carve_ws(nullptr, m, n, kc, S, batch, &w);
}

// test hook (bt_debug_split_stall): the MMA warp's stall before its first MMA (0 = off), for the
// next g_stall_left launches (negative: every launch)
std::atomic<unsigned long long*> g_prof{nullptr};  // bt_debug_split_profile: device counters
std::atomic<unsigned long long> g_stall_ns{0};
std::atomic<long long> g_stall_left{0};

unsigned long long stall_for_launch() {
  const unsigned long long ns = g_stall_ns.load();
  if (ns == 0) return 0;
  long long left = g_stall_left.load();
  while (left != 0) {
    if (left < 0) return ns;
    if (g_stall_left.compare_exchange_weak(left, left - 1)) return ns;
  }
  return 0;
}

size_t sliced_op_bytes(int role, int lines, int k, int slices, int batch) {
  if (lines <= 0 || k <= 0 || k > kMaxKc || batch <= 0 || (role != 0 && role != 1)) return 0;
  const int S = slices > 0 ? slices : 6;
  const int Kp = pad_k(k);
  const int rows = role == 0 ? pad_rows_n(lines, pick_nt(lines)) : pad_rows_m(lines);
  return al256(sizeof(int) * (size_t)batch * lines) + al256((size_t)batch * S * rows * Kp * 2);
}

bt_status slice_op(cudaStream_t st, int role, int lines, int k, Operand X, int batch, int slices, void* buf,
                   size_t bytes, SlicedOp* out) {
  const int S = slices > 0 ? slices : 6;
  if (!out || S < 2 || S > kMaxSlices || batch <= 0 || batch > 65535 || lines <= 0 || k <= 0 || k > kMaxKc ||
      (role != 0 && role != 1))
    return BT_ERR_INVALID_ARG;
  if (!buf || bytes < sliced_op_bytes(role, lines, k, S, batch)) return BT_ERR_INVALID_ARG;
  const int Kp = pad_k(k);
  SlicedOp o;
  o.role = role;
  o.lines = lines;
  o.kc = k;
  o.S = S;
  o.batch = batch;
  o.shared = X.stride == 0 && batch > 1;
  o.e = static_cast<int*>(buf);
  o.t = reinterpret_cast<uint32_t*>(static_cast<char*>(buf) + al256(sizeof(int) * (size_t)batch * lines));
  const int nb = o.shared ? 1 : batch;
  if (role == 0) {
    const int mp = pad_rows_n(lines, pick_nt(lines));
    BT_TRY(slice_lines<false>(st, X.op == BT_OP_N, lines, mp, k, Kp / 2, X.p, X.ld, X.stride, X.op == BT_OP_C, S, o.e,
                              o.t, nb, nullptr));
  } else {
    const int n2p = pad_rows_m(lines);
    BT_TRY(slice_lines<true>(st, X.op == BT_OP_C, lines, n2p / 2, k, Kp / 2, X.p, X.ld, X.stride, X.op == BT_OP_C, S,
                             o.e, o.t, nb, nullptr));
  }
  *out = o;
  return BT_OK;
}

bt_status split_zgemm(cudaStream_t st, int m, int n, int k, zd alpha, Operand A, Operand B, zd beta, zd* C, int ldc,
                      long long strideC, int batch, int slices, void* ws, size_t ws_bytes, const int* active,
                      int* err, long long err_stride, const SlicedOp* preA, const SlicedOp* preB) {
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
  if (preA && preA->valid() && (preA->role != 0 || preA->lines != m || preA->kc != k || preA->S != S ||
                                preA->batch != batch || k > kMaxKc || active))
    return BT_ERR_INVALID_ARG;
  if (preB && preB->valid() && (preB->role != 1 || preB->lines != n || preB->kc != k || preB->S != S ||
                                preB->batch != batch || k > kMaxKc || active))
    return BT_ERR_INVALID_ARG;
  const bool useA = preA && preA->valid(), useB = preB && preB->valid();
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
    const bool a_shared = useA ? preA->shared : (A.stride == 0 && batch > 1);
    const bool b_shared = useB ? preB->shared : (B.stride == 0 && batch > 1);
    const int ba = a_shared ? 1 : batch, bb = b_shared ? 1 : batch;
    const int* act_a = a_shared ? nullptr : active;
    const int* act_b = b_shared ? nullptr : active;
    // At from the rows of op(A): contiguous for op N;  Bt from the columns of op(B): contiguous for op C
    if (useA) {
      w.At = preA->t;
      w.eA = preA->e;
    } else {
      BT_TRY(slice_lines<false>(st, a.op == BT_OP_N, m, mp, kc, Kp / 2, a.p, a.ld, a.stride, a.op == BT_OP_C, S, w.eA,
                                w.At, ba, act_a));
    }
    if (useB) {
      w.Bt = preB->t;
      w.eB = preB->e;
    } else {
      BT_TRY(slice_lines<true>(st, bop.op == BT_OP_C, n, n2p / 2, kc, Kp / 2, bop.p, bop.ld, bop.stride,
                               bop.op == BT_OP_C, S, w.eB, w.Bt, bb, act_b));
    }
    // CTA pairs (cta_group::2: two M tiles share each At tile, half of it in each CTA), by
    // default with two K blocks per pipeline stage and only for an even number of M tiles (an odd
    // count pads one 128-row tile per pair column: at 2n = 832 one CTA per tile is faster), and
    // only when the device holds most of its SMs as pairs.  Measured at 1024^3 x 4: 0.724 ms
    // against 0.767 ms for one CTA per tile.
    const int tiles_x = n2p / kTileM;
    const int mode = g_pair_mode.load();
    bool pair = false;
    const int pair_kind = mode == 2 ? 1 : 2;
    const bool want = mode == 2 || mode == 3 || (mode == 0 && tiles_x % 2 == 0);
    if (want && tiles_x >= 2) {
      const int nc = pair_clusters_nt(nt, pair_kind);
      pair = nc > 0 && 2 * nc >= (num_sms() * 9) / 10;
    }
    CUtensorMap mA, mB, mBh;
    if (!encode_slices_map(&mA, w.Bt, Kp, 2 * n, n2p, batch * S, kTileM)) return BT_ERR_CUDA;
    if (!encode_slices_map(&mB, w.At, Kp, m, mp, batch * S, nt)) return BT_ERR_CUDA;
    // pairs: a single job's At tile is split in halves, one per CTA
    if (!encode_slices_map(&mBh, w.At, Kp, m, mp, batch * S, pair ? nt / 2 : nt)) return BT_ERR_CUDA;
    MmaParams p{};
    p.m = m;
    p.n2 = 2 * n;
    p.Kp = Kp;
    p.S = S;
    p.tiles_x = tiles_x;
    p.tiles_y = mp / nt;
    p.n_tiles = p.tiles_x * p.tiles_y * batch;
    p.pair = pair ? 1 : 0;
    p.tiles_xu = pair ? (tiles_x + 1) / 2 : tiles_x;
    p.n_units = p.tiles_xu * p.tiles_y * batch;
    p.eA = w.eA;
    p.eB = w.eB;
    p.C = C;
    p.ldc = ldc;
    p.sC = strideC;
    p.alpha = alpha;
    p.beta = k0 == 0 ? beta : zmake(1.0, 0.0);
    const bool unit = alpha.y == 0.0 && (alpha.x == 1.0 || alpha.x == -1.0);
    if (p.alpha.y != 0.0 || p.beta.y != 0.0) p.coef_mode = kCoefComplex;
    else if (unit && p.beta.x == 0.0) p.coef_mode = kCoefUnit;
    else if (unit && p.beta.x == 1.0) p.coef_mode = kCoefUnitAcc;
    else p.coef_mode = kCoefReal;
    p.negate = (unit && alpha.x == -1.0) ? 1 : 0;
    p.err = err;
    p.err_stride = err_stride;
    p.stall_ns = stall_for_launch();
    p.prof = g_prof.load();
    p.active = active;
    p.a_shared = a_shared ? 1 : 0;
    p.b_shared = b_shared ? 1 : 0;
    if (!make_schedule(S, Kp / kKBlock, g_sched_mode.load() == 0, &p.sched, &p.bias, &p.fix_bits))
      return BT_ERR_UNSUPPORTED;
    if (pair && pair_kind == 2) BT_TRY(launch_mma_nt<2>(nt, st, mA, mB, mBh, p));
    else if (pair) BT_TRY(launch_mma_nt<1>(nt, st, mA, mB, mBh, p));
    else BT_TRY(launch_mma_nt<0>(nt, st, mA, mB, mBh, p));
  }
  return BT_OK;
}

}  // namespace bt

extern "C" bt_status bt_debug_split_profile(int enable, unsigned long long* counters, int n_counters) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  unsigned long long* d = bt::g_prof.load();
  if (enable) {
    if (!d) {
      if (cudaMalloc(&d, sizeof(unsigned long long) * bt::kProfSlots) != cudaSuccess) return BT_ERR_OOM;
    }
    if (cudaMemset(d, 0, sizeof(unsigned long long) * bt::kProfSlots) != cudaSuccess) return BT_ERR_CUDA;
    bt::g_prof.store(d);
    return BT_OK;
  }
  if (!d) return BT_ERR_INVALID_ARG;
  bt::g_prof.store(nullptr);
  unsigned long long h[bt::kProfSlots] = {};
  const bool ok = cudaDeviceSynchronize() == cudaSuccess &&
                  cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d);
  if (!ok) return BT_ERR_CUDA;
  if (counters)
    for (int i = 0; i < n_counters && i < bt::kProfSlots; ++i) counters[i] = h[i];
  return BT_OK;
}

extern "C" void bt_debug_split_pair(int mode) { bt::g_pair_mode.store(mode >= 1 && mode <= 3 ? mode : 0); }

extern "C" void bt_debug_split_sched(int mode) { bt::g_sched_mode.store(mode == 1 ? 1 : 0); }

extern "C" int bt_debug_split_schedule(int slices, int k_blocks, int mode, int* jobs, int max_jobs, int* items,
                                       int max_items, int* fix_bits) {
  if (slices < 2 || slices > bt::kMaxSlices || k_blocks < 1 || k_blocks > 255) return -1;
  bt::Schedule sc;
  unsigned long long bias = 0;
  int F = 0;
  if (!bt::make_schedule(slices, k_blocks, mode != 1, &sc, &bias, &F)) return -1;
  if (fix_bits) *fix_bits = F;
  if (jobs)
    for (int g = 0; g < sc.n_jobs && g < max_jobs; ++g) {
      int* r = jobs + 8 * g;
      r[0] = sc.dual[g];
      r[1] = sc.ib[g];
      r[2] = sc.ie[g];
      r[3] = sc.kb0[g];
      r[4] = sc.kb1[g];
      r[5] = sc.cvt[g][0];
      r[6] = sc.cvt[g][1];
      r[7] = 0;
    }
  if (items)
    for (int i = 0; i < (sc.n_jobs ? sc.ie[sc.n_jobs - 1] : 0) && i < max_items; ++i) {
      items[3 * i] = sc.s[i];
      items[3 * i + 1] = sc.s2[i];
      items[3 * i + 2] = sc.t[i];
    }
  return sc.n_jobs;
}

extern "C" void bt_debug_split_stall(unsigned long long ns, long long launches) {
  bt::g_stall_left.store(launches);
  bt::g_stall_ns.store(ns);
}

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
                         workspace_bytes, nullptr, nullptr, 0);
}
