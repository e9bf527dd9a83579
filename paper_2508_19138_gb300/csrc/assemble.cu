// Element-wise kernels of the sweep: assembly of M~ and B^<> blocks (Sec. 4.3.1, Table 2),
// the lesser/greater boundary blocks by fluctuation-dissipation (Sec. 4.2), the anti-Hermitian
// corrections (y - y^H), (Z - Z^H) of Eq. 10 and 12, the projection onto anti-Hermitian blocks
// and the symmetrised write-out of Sec. 5.2 (full blocks, diagonal entries or packed upper
// triangles).
// All are memory-bound grid-stride loops over (element, batch entry) with coalesced accesses
// along the row-major block; transposed reads (X^H) go through the L1/L2 of the same block.
#include "elementwise.cuh"

namespace bt {
namespace {

__device__ __forceinline__ double fermi_dev(double E, double mu, double kT) {
  const double x = (E - mu) / kT;
  const double ex = exp(-fabs(x));
  return x > 0.0 ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
}

__global__ void energy_setup_kernel(int n, const double* __restrict__ E, double eta, double muL, double muR, double kT,
                                    zd* __restrict__ z, double* __restrict__ fL, double* __restrict__ fR) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = zmake(E[i], eta);
  fL[i] = fermi_dev(E[i], muL, kT);
  fR[i] = fermi_dev(E[i], muR, kT);
}

// out[e] = zS*S - H - sig (- obc1 - obc2) for one block position
__global__ void assemble_m_kernel(int bs, MBlockArgs a) {
  const int e = blockIdx.y;
  const long long bs2 = (long long)bs * bs;
  const zd z = a.z ? a.z[e] : zmake(0.0, 0.0);
  zd* out = a.out + a.out_stride * e;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    zd v = zmake(0.0, 0.0);
    if (a.use_z) {
      if (a.S) {
        zd s = a.S_conjT ? zconj(a.S[a.S_stride * e + (long long)c * bs + r]) : a.S[a.S_stride * e + i];
        v = zmul(z, s);
      } else if (a.S_identity && r == c) {
        v = z;
      }
    }
    if (a.H) {
      zd h = a.H_conjT ? zconj(a.H[a.H_stride * e + (long long)c * bs + r]) : a.H[a.H_stride * e + i];
      v = zsub(v, zscale(h, a.H_sign));
    }
    if (a.sig) {
      zd s = a.sig_conjT ? zconj(a.sig[a.sig_stride * e + (long long)c * bs + r]) : a.sig[a.sig_stride * e + i];
      v = zsub(v, zscale(s, a.sig_sign));
    }
    if (a.sigvec && r == c) v = zsub(v, a.sigvec[a.sigvec_stride * e + r]);
    if (a.obc1) v = zsub(v, a.obc1[a.obc_stride * e + i]);
    if (a.obc2) v = zsub(v, a.obc2[a.obc_stride * e + i]);
    out[i] = v;
  }
}

// out[e] = sig (blocks or diagonal vector) + obc
__global__ void assemble_b_kernel(int bs, BBlockArgs a) {
  const int e = blockIdx.y;
  const long long bs2 = (long long)bs * bs;
  zd* out = a.out + a.out_stride * e;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    zd v = zmake(0.0, 0.0);
    if (a.sig && !a.sig_packed) v = a.sig[a.sig_stride * e + i];
    if (a.sig && a.sig_packed) {
      const int lo = r < c ? r : c, hi = r < c ? c : r;
      const zd u = a.sig[a.sig_stride * e + (long long)lo * bs - (long long)lo * (lo - 1) / 2 + (hi - lo)];
      v = r <= c ? u : zmake(-u.x, u.y);  // lower triangle: -conj(upper)
    }
    if (a.sigvec && r == c) v = a.sigvec[a.sigvec_stride * e + r];
    if (a.obc1) v = zadd(v, a.obc1[a.obc_stride * e + i]);
    if (a.obc2) v = zadd(v, a.obc2[a.obc_stride * e + i]);
    out[i] = v;
  }
}

// lesser / greater boundary blocks: B^<_c = -f (s - s^H), B^>_c = (1 - f)(s - s^H)
__global__ void obc_lg_kernel(int bs, int E, const zd* __restrict__ sig, const double* __restrict__ fL,
                              const double* __restrict__ fR, zd* __restrict__ outL, zd* __restrict__ outG) {
  const int l = blockIdx.y;  // lead index: [0, E) left, [E, 2E) right
  const double f = l < E ? fL[l] : fR[l - E];
  const long long bs2 = (long long)bs * bs;
  const zd* s = sig + bs2 * l;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    const zd d = zsub(s[i], zconj(s[(long long)c * bs + r]));
    if (outL) outL[bs2 * l + i] = zscale(d, -f);
    if (outG) outG[bs2 * l + i] = zscale(d, 1.0 - f);
  }
}

// X += sgn * (Y - Y^H)
__global__ void add_antiherm_kernel(int bs, zd* __restrict__ X, long long sX, const zd* __restrict__ Y, long long sY,
                                    double sgn) {
  const int e = blockIdx.y;
  const long long bs2 = (long long)bs * bs;
  zd* x = X + sX * e;
  const zd* y = Y + sY * e;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    const zd d = zsub(y[i], zconj(y[(long long)c * bs + r]));
    x[i] = zadd(x[i], zscale(d, sgn));
  }
}

// X <- (X - X^H) / 2 in place: each pair (r, c), (c, r) with r <= c handled by one thread, so the
// result is exactly anti-Hermitian (diagonal purely imaginary).
__global__ void antiherm_project_kernel(int bs, zd* __restrict__ X, long long sX) {
  const int e = blockIdx.y;
  const long long bs2 = (long long)bs * bs;
  zd* x = X + sX * e;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    if (r > c) continue;
    if (r == c) {
      x[i].x = 0.0;
      continue;
    }
    const long long j = (long long)c * bs + r;
    const zd u = zscale(zsub(x[i], zconj(x[j])), 0.5);
    x[i] = u;
    x[j] = zmake(-u.x, u.y);
  }
}

// out = alpha * x  (+ beta * out unless beta == 0)
__global__ void axpby_kernel(long long n, double alpha, const zd* __restrict__ x, long long sx, double beta,
                             zd* __restrict__ out, long long so) {
  const int e = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    zd v = zscale(x[sx * e + i], alpha);
    if (beta != 0.0) v = zadd(v, zscale(out[so * e + i], beta));
    out[so * e + i] = v;
  }
}

// Packed upper triangle of (X - X^H)/2 per block (Sec. 5.2: the anti-Hermitian lesser / greater
// blocks stored by their upper triangle): row r holds columns r..bs-1, starting at
// r bs - r (r - 1) / 2; bs (bs + 1) / 2 entries per block.
__global__ void write_packed_kernel(int bs, int nblk, const zd* __restrict__ src, long long s_blk, long long s_e,
                                    zd* __restrict__ dst, long long d_e) {
  const int e = blockIdx.z, blk = blockIdx.y;
  const long long bs2 = (long long)bs * bs, pk = (long long)bs * (bs + 1) / 2;
  const zd* s = src + s_e * e + s_blk * blk;
  zd* d = dst + d_e * e + pk * blk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    if (c < r) continue;
    const long long o = (long long)r * bs - (long long)r * (r - 1) / 2 + (c - r);
    d[o] = zscale(zsub(s[i], zconj(s[(long long)c * bs + r])), 0.5);
  }
}

// Full anti-Hermitian blocks from their packed upper triangles.
__global__ void unpack_antiherm_kernel(int bs, const zd* __restrict__ src, long long s_e, zd* __restrict__ dst,
                                       long long d_blk, long long d_e) {
  const int e = blockIdx.z, blk = blockIdx.y;
  const long long bs2 = (long long)bs * bs, pk = (long long)bs * (bs + 1) / 2;
  const zd* s = src + s_e * e + pk * blk;
  zd* d = dst + d_e * e + d_blk * blk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
    const int lo = r < c ? r : c, hi = r < c ? c : r;
    const zd u = s[(long long)lo * bs - (long long)lo * (lo - 1) / 2 + (hi - lo)];
    d[i] = r <= c ? u : zmake(-u.x, u.y);
  }
}

// Write nblk blocks per batch entry: mode 0 copy, mode 1 (X - X^H)/2.
__global__ void write_blocks_kernel(int bs, int nblk, const zd* __restrict__ src, long long s_blk, long long s_e,
                                    zd* __restrict__ dst, long long d_blk, long long d_e, int mode) {
  const int e = blockIdx.z, blk = blockIdx.y;
  const long long bs2 = (long long)bs * bs;
  const zd* s = src + s_e * e + s_blk * blk;
  zd* d = dst + d_e * e + d_blk * blk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < bs2; i += (long long)gridDim.x * blockDim.x) {
    if (mode == 0) {
      d[i] = s[i];
    } else {
      const int r = (int)(i / bs), c = (int)(i - (long long)r * bs);
      d[i] = zscale(zsub(s[i], zconj(s[(long long)c * bs + r])), 0.5);
    }
  }
}

// Diagonal entries of nblk diagonal blocks per batch entry -> [nblk][bs] vectors; mode 1 keeps
// the anti-Hermitian part of the block, whose diagonal is i Im(x).
__global__ void write_diagvec_kernel(int bs, int nblk, const zd* __restrict__ src, long long s_blk, long long s_e,
                                     zd* __restrict__ dst, long long d_blk, long long d_e, int mode) {
  const int e = blockIdx.z, blk = blockIdx.y;
  const zd* s = src + s_e * e + s_blk * blk;
  zd* d = dst + d_e * e + d_blk * blk;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < bs; r += gridDim.x * blockDim.x) {
    const zd v = s[(long long)r * bs + r];
    d[r] = mode == 0 ? v : zmake(0.0, v.y);
  }
}

__global__ void merge_status_kernel(int E, const int* __restrict__ info, int n_sources, long long src_stride,
                                    int* __restrict__ status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int s = 0; s < n_sources; ++s) {
    const int v = info[src_stride * s + e];
    if (v != 0 && status[e] == 0) status[e] = v;
  }
}

__global__ void shift_diag_kernel(int bs, zd* __restrict__ X, long long sX, double v) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= bs) return;
  zd* x = X + sX * blockIdx.y + (long long)r * bs + r;
  x->x += v;
}

inline dim3 grid_for(long long n, int batch, int ythird = 1) {
  long long gx = (n + 255) / 256;
  if (gx > 256) gx = 256;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)batch, (unsigned)ythird);
}

}  // namespace

bt_status energy_setup(cudaStream_t st, int n, const double* E, double eta, double muL, double muR, double kT, zd* z,
                       double* fL, double* fR) {
  if (n <= 0) return BT_OK;
  energy_setup_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, E, eta, muL, muR, kT, z, fL, fR); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status assemble_m(cudaStream_t st, int bs, int batch, const MBlockArgs& a) {
  if (batch <= 0) return BT_OK;
  assemble_m_kernel<<<grid_for((long long)bs * bs, batch), 256, 0, st>>>(bs, a); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status assemble_b(cudaStream_t st, int bs, int batch, const BBlockArgs& a) {
  if (batch <= 0) return BT_OK;
  assemble_b_kernel<<<grid_for((long long)bs * bs, batch), 256, 0, st>>>(bs, a); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status unpack_antiherm(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_e, zd* dst,
                          long long d_blk, long long d_e) {
  if (batch <= 0 || nblk <= 0) return BT_OK;
  const long long bs2 = (long long)bs * bs;
  long long gx = (bs2 + 255) / 256;
  if (gx > 64) gx = 64;
  unpack_antiherm_kernel<<<dim3((unsigned)gx, nblk, batch), 256, 0, st>>>(bs, src, s_e, dst, d_blk, d_e);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status obc_lesser_greater(cudaStream_t st, int bs, int E, const zd* sig, const double* fL, const double* fR,
                             zd* outL, zd* outG) {
  if (E <= 0) return BT_OK;
  obc_lg_kernel<<<grid_for((long long)bs * bs, 2 * E), 256, 0, st>>>(bs, E, sig, fL, fR, outL, outG); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status antiherm_project(cudaStream_t st, int bs, int batch, zd* X, long long sX) {
  antiherm_project_kernel<<<grid_for((long long)bs * bs, batch), 256, 0, st>>>(bs, X, sX); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status add_antiherm(cudaStream_t st, int bs, int batch, zd* X, long long sX, const zd* Y, long long sY, double sgn) {
  if (batch <= 0) return BT_OK;
  add_antiherm_kernel<<<grid_for((long long)bs * bs, batch), 256, 0, st>>>(bs, X, sX, Y, sY, sgn); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status axpby(cudaStream_t st, long long n, int batch, double alpha, const zd* x, long long sx, double beta, zd* out,
                long long so) {
  if (batch <= 0 || n <= 0) return BT_OK;
  axpby_kernel<<<grid_for(n, batch), 256, 0, st>>>(n, alpha, x, sx, beta, out, so); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status write_blocks(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_blk, long long s_e,
                       zd* dst, long long d_blk, long long d_e, int mode) {
  if (batch <= 0 || nblk <= 0) return BT_OK;
  if (nblk > 65535 || batch > 65535) return BT_ERR_INVALID_ARG;
  dim3 g = grid_for((long long)bs * bs, nblk, batch);
  if (g.x > 64) g.x = 64;
  write_blocks_kernel<<<g, 256, 0, st>>>(bs, nblk, src, s_blk, s_e, dst, d_blk, d_e, mode); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status write_packed(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_blk, long long s_e,
                       zd* dst, long long d_e) {
  if (batch <= 0 || nblk <= 0) return BT_OK;
  if (nblk > 65535 || batch > 65535) return BT_ERR_INVALID_ARG;
  dim3 g = grid_for((long long)bs * bs, nblk, batch);
  if (g.x > 64) g.x = 64;
  write_packed_kernel<<<g, 256, 0, st>>>(bs, nblk, src, s_blk, s_e, dst, d_e); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status shift_diag(cudaStream_t st, int bs, int batch, zd* X, long long sX, double v) {
  if (batch <= 0) return BT_OK;
  shift_diag_kernel<<<dim3((bs + 127) / 128, batch), 128, 0, st>>>(bs, X, sX, v); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status write_diagvec(cudaStream_t st, int bs, int nblk, int batch, const zd* src, long long s_blk, long long s_e,
                        zd* dst, long long d_blk, long long d_e, int mode) {
  if (batch <= 0 || nblk <= 0) return BT_OK;
  if (nblk > 65535 || batch > 65535) return BT_ERR_INVALID_ARG;
  dim3 g((bs + 255) / 256, nblk, batch);
  write_diagvec_kernel<<<g, 256, 0, st>>>(bs, nblk, src, s_blk, s_e, dst, d_blk, d_e, mode);
  count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

__global__ void flag_status_kernel(int E, const int* __restrict__ flag, int* __restrict__ status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  // a timed-out product leaves everything computed after it meaningless: the flag takes precedence
  if (e < E && *flag != 0) status[e] = *flag;
}

bt_status flag_status(cudaStream_t st, int E, const int* flag, int* status) {
  if (E <= 0) return BT_OK;
  flag_status_kernel<<<(E + 127) / 128, 128, 0, st>>>(E, flag, status); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

bt_status merge_status(cudaStream_t st, int E, const int* info, int n_sources, long long src_stride, int* status) {
  if (E <= 0) return BT_OK;
  merge_status_kernel<<<(E + 127) / 128, 128, 0, st>>>(E, info, n_sources, src_stride, status); count_launch();
  BT_CUDA_TRY(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt
