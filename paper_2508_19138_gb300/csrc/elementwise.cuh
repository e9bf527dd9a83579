// Declarations of the element-wise kernels of the sweep (assemble.cu).
#pragma once
#include "bt_common.cuh"

namespace bt {

// Arguments of the M~ block assembly: out[e] = use_z * z[e] * S - H_sign * H - sig_sign * sig
//                                              - diag(sigvec) - obc1 - obc2
// Each source pointer may be null; *_stride is the per-batch-entry element stride (0 = shared);
// *_conjT reads the conjugate transpose of the stored block.
struct MBlockArgs {
  zd* out = nullptr;
  long long out_stride = 0;
  const zd* z = nullptr;
  int use_z = 0;
  int S_identity = 0;
  const zd* S = nullptr;
  long long S_stride = 0;
  int S_conjT = 0;
  const zd* H = nullptr;
  long long H_stride = 0;
  int H_conjT = 0;
  double H_sign = 1.0;
  const zd* sig = nullptr;
  long long sig_stride = 0;
  int sig_conjT = 0;
  double sig_sign = 1.0;
  const zd* sigvec = nullptr;
  long long sigvec_stride = 0;
  const zd* obc1 = nullptr;
  const zd* obc2 = nullptr;
  long long obc_stride = 0;
};

// out[e] = sig (+ diag(sigvec)) + obc1 + obc2; with sig_packed, sig is an anti-Hermitian block
// stored by its upper triangle (entry (r, c >= r) at r bs - r (r - 1) / 2 + (c - r)).
struct BBlockArgs {
  zd* out = nullptr;
  long long out_stride = 0;
  const zd* sig = nullptr;
  long long sig_stride = 0;
  int sig_packed = 0;
  const zd* sigvec = nullptr;
  long long sigvec_stride = 0;
  const zd* obc1 = nullptr;
  const zd* obc2 = nullptr;
  long long obc_stride = 0;
};

bt_status energy_setup(cudaStream_t st, int n, const double* E, double eta, double muL, double muR, double kT, zd* z,
                       double* fL, double* fR);
bt_status assemble_m(cudaStream_t st, int bs, int batch, const MBlockArgs& a);
bt_status assemble_b(cudaStream_t st, int bs, int batch, const BBlockArgs& a);
bt_status obc_lesser_greater(cudaStream_t st, int bs, int E, const zd* sig, const double* fL, const double* fR,
                             zd* outL, zd* outG);
bt_status add_antiherm(cudaStream_t st, int bs, int batch, zd* X, long long sX, const zd* Y, long long sY, double sgn);
// X <- (X - X^H) / 2 per bs x bs block (exactly anti-Hermitian result)
bt_status antiherm_project(cudaStream_t st, int bs, int batch, zd* X, long long sX);
bt_status axpby(cudaStream_t st, long long n, int batch, double alpha, const zd* x, long long sx, double beta, zd* out,
                long long so);
bt_status write_blocks(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_blk, long long s_e,
                       zd* dst, long long d_blk, long long d_e, int mode);
bt_status write_diagvec(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_blk, long long s_e,
                        zd* dst, long long d_blk, long long d_e, int mode);  // diagonal entries only
// packed upper triangle of (X - X^H)/2, bs (bs + 1) / 2 entries per block
bt_status write_packed(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_blk, long long s_e,
                       zd* dst, long long d_e);
bt_status shift_diag(cudaStream_t st, int bs, int batch, zd* X, long long sX, double v);  // X += v I
// full anti-Hermitian blocks from packed upper triangles: nblk blocks per batch entry, the packed
// blocks bs (bs + 1) / 2 apart (s_e per entry), the full ones d_blk apart (d_e per entry)
bt_status unpack_antiherm(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_e, zd* dst,
                          long long d_blk, long long d_e);
bt_status merge_status(cudaStream_t st, int E, const int* info, int n_sources, long long src_stride, int* status);
// status[e] = *flag for every e when *flag != 0 (a chunk-wide error word that overrides the
// numerical failures recorded after it)
bt_status flag_status(cudaStream_t st, int E, const int* flag, int* status);

}  // namespace bt
