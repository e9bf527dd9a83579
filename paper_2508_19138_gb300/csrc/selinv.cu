// Context, workspace and the recursive Green's function sweeps (Sec. 4.3.2) behind the C ABI.
//
// For a chunk of Ec energies every step below is ONE batched launch over the chunk (the
// energies are the data-parallel axis, Sec. 4.4 / 5.4):
//   a1  assembly of M~ = M - B^R_scatt - B^R_OBC and B^<> (Table 2, Sec. 4.3.1);
//       W system: V P^R and V P^<> V^H as block-tridiagonal products
//   a2  contact decimation (Eq. 4) for the 2 Ec leads, fluctuation-dissipation for B^<>_OBC
//   a3  forward pass, Eq. 9 (x^R_i) and Eq. 10 (x^<>_i, with y_i = M~_{i,i-1} x^R_{i-1} B_{i-1,i})
//   a4  backward pass, Eq. 11 (X^R_i), Eq. 12 (X^<>_i with Y_i, Z_i); first off-diagonal blocks
//         X^R_{i,i+1} = -x^R_i M~_{i,i+1} X^R_{i+1},   X^R_{i+1,i} = -X^R_{i+1} M~_{i+1,i} x^R_i
//         X^<>_{i,i+1} = -x^R_i M~_{i,i+1} X^<>_{i+1} - x^<>_i (X^R_{i+1} M~_{i+1,i})^H
//                        + x^R_i B^<>_{i,i+1} (X^R_{i+1})^H
//       W system: W^R = X^R V on the selected blocks (needs X^R_{i,i+-2})
//   a5  symmetrised write-out of the diagonal lesser/greater blocks (Sec. 5.2), as full blocks
//       or packed upper triangles
// All sweep products go through prod(), which runs the FP64 DFMA kernel or, with BT_SPLIT, the
// sliced bf16 tensor-core product; with symmetrised outputs the lesser/greater sandwiches come
// out exactly anti-Hermitian (Sec. 5.2 symmetry kept inside the sweep) and Z_i of Eq. 12 is
// formed from the first term of X^<>_{i,i+1}.  The inversions and the decimation run on the
// FP64 engine, or on a sliced one with split_scope = 1.  In graph mode a chunk's launches are
// captured once into a CUDA graph and replayed (run_chunk_graph).
#include <algorithm>
#include <cstring>
#include <functional>
#include <string>
#include <unordered_map>
#include <vector>

#include "elementwise.cuh"

struct bt_ctx {
  bt_selinv_desc d{};
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  // chunk workspace (E = max_energies, B2 = bs^2)
  zd *xR = nullptr, *xL = nullptr, *xG = nullptr;     // [E][N][B2]
  zd *Mu = nullptr, *Ml = nullptr;                    // [E][N-1][B2] assembled off-diagonal M~ (general / W)
  zd *XRu = nullptr, *XRl = nullptr;                  // [E][N-1][B2] kept for the W products
  zd *Md = nullptr;                                   // [E][N][B2] W: assembled M~ diagonal
  zd *BdL = nullptr, *BdG = nullptr, *BuL = nullptr, *BuG = nullptr;  // W: B^<> blocks
  zd *Td = nullptr, *Tu = nullptr, *Tl = nullptr;     // W: V P products [E][N or N-1][B2]
  zd *X2u = nullptr, *X2l = nullptr;                  // W: X^R_{i,i+2}, X^R_{i+2,i} [E][N-2][B2]
  zd* wl[11] = {};                                    // W contacts: lead temporaries [2E][B2]
  int *w_ok = nullptr, *w_info = nullptr;             // W contacts: Stein convergence, status [2E]
  zd* t[12] = {};                                     // [E][B2] temporaries
  zd *lead_m = nullptr, *lead_n = nullptr, *lead_np = nullptr, *lead_x = nullptr, *lead_sig = nullptr;
  zd *obcL = nullptr, *obcG = nullptr;                // [2E][B2]
  int *lead_iters = nullptr, *lead_info = nullptr;    // [2E]
  int* lead_piters = nullptr;                         // [2E] doubling iterations of the Newton step
  // contact memoization: surface functions of solved energies [cap][2][B2] + lead masks [2E]
  zd* memo_x = nullptr;
  int *lead_run = nullptr, *lead_conv = nullptr, *lead_dec = nullptr;
  std::unordered_map<uint64_t, int> memo_slot;        // energy bits -> slot
  std::vector<uint64_t> memo_key;                     // slot -> energy bits (0 = empty)
  std::vector<char> memo_used;
  int memo_next = 0;
  zd* z = nullptr;
  double *fL = nullptr, *fR = nullptr, *Edev = nullptr;
  int* tflag = nullptr;  // BT_ERR_TIMEOUT from a bounded wait of a sliced product in this chunk
  void* inv_ws = nullptr;
  size_t inv_bytes = 0;
  void* dec_ws = nullptr;
  size_t dec_bytes = 0;
  void* split_ws = nullptr;
  size_t split_bytes = 0;
  // sliced products: operands sliced once per sweep step and reused by the products they enter
  char* pre_a[2] = {nullptr, nullptr};
  char* pre_b[3] = {nullptr, nullptr, nullptr};
  size_t pre_a_bytes = 0, pre_b_bytes = 0;
  bt::Engine eng_kept;  // products of the inversions and the decimation (FP64 unless split_scope = 1)
  bt::Engine eng_polish;  // products of the Newton step after decimation (FP64, or 8 slices with split_scope = 1)
  int* h_pinned = nullptr;
  double* h_E = nullptr;
  bool pinned = true;   // host buffers from cudaMallocHost (else new[])
  bool owns_ws = true;  // workspace from cudaMalloc (else lent by a serving arena)
  // host-buffer entry point staging (allocated on first use), and the stream and events that
  // overlap the copies of one chunk's outputs with the next chunk's compute
  char* stage = nullptr;
  size_t stage_bytes = 0;
  // graph mode: the chunk's per-energy inputs copied to fixed addresses before each replay, so
  // that one captured graph serves every call with the same shapes and outputs (allocated on
  // first use)
  char* gstage = nullptr;
  size_t gstage_bytes = 0;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  cudaEvent_t ev_ready = nullptr;
  std::string err;
  bt_stats stats{};
  double flops = 0.0;
  // graph mode: captured chunks (least recently used first), the stream the decimation loop body
  // is captured on, and the per-lead iteration counts of the last replayed chunk (read back
  // asynchronously, folded into the statistics at the next synchronisation)
  struct Captured {
    std::vector<char> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double flops = 0.0;             // model flops without the decimation iterations
    long long launches = 0;         // kernels outside the decimation loop
    long long body_launches = 0;    // kernels per decimation iteration
    long long polish_body = 0;      // kernels per doubling iteration of the Newton step
    bool decim = false;
  };
  std::vector<Captured> graphs;
  cudaStream_t body_st = nullptr;
  bt::LoopCapture* loop = nullptr;  // non-null while a chunk is being captured
  int* h_iters = nullptr;           // [4E] pinned: decimation, then Newton-step iterations per lead
  long long cap_polish_body = 0;    // kernels of one pass of the Newton step's doubling loop (capture)
  bool pending = false;
  int pending_Ec = 0;
  long long pending_body = 0;
  long long pending_polish_body = 0;
  long long uncounted = 0;          // launches recorded during capture (not executed)
};

namespace {

thread_local std::string g_create_error;

size_t al(size_t x) { return (x + 255) / 256 * 256; }

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += al(count * sizeof(T));
    return p;
  }
};

bool is_split(const bt_selinv_desc& d) { return d.precision == BT_SPLIT; }
int slices_of(const bt_selinv_desc& d) { return d.split_slices > 0 ? d.split_slices : 6; }
// split_scope = 1: the products inside the inversions and the decimation carry one slice more
// than the sweep products; their errors are amplified by the condition of the inverted blocks
// (at S = 6 the 40 x 416 nanoribbon's retarded blocks came out 2e-8 off the oracle).
int kept_slices_of(const bt_selinv_desc& d) { return slices_of(d) < 8 ? slices_of(d) + 1 : 8; }

// Lays out the workspace; with base == nullptr only measures it.
size_t layout(bt_ctx* c, const bt_selinv_desc& d, char* base) {
  Carver cv(base);
  const size_t E = (size_t)d.max_energies, N = (size_t)d.nb, B2 = (size_t)d.bs * d.bs;
  const size_t N1 = N > 1 ? N - 1 : 1;
  bt_ctx tmp;
  bt_ctx* x = c ? c : &tmp;
  x->xR = cv.take<zd>(E * N * B2);
  x->xL = cv.take<zd>(E * N * B2);
  x->xG = cv.take<zd>(E * N * B2);
  x->Mu = cv.take<zd>(E * N1 * B2);
  x->Ml = cv.take<zd>(E * N1 * B2);
  for (int i = 0; i < 12; ++i) x->t[i] = cv.take<zd>(E * B2);
  if (d.system == BT_SYS_W) {
    x->XRu = cv.take<zd>(E * N1 * B2);
    x->XRl = cv.take<zd>(E * N1 * B2);
    x->Md = cv.take<zd>(E * N * B2);
    x->BdL = cv.take<zd>(E * N * B2);
    x->BdG = cv.take<zd>(E * N * B2);
    x->BuL = cv.take<zd>(E * N1 * B2);
    x->BuG = cv.take<zd>(E * N1 * B2);
    x->Td = cv.take<zd>(E * N * B2);
    x->Tu = cv.take<zd>(E * N1 * B2);
    x->Tl = cv.take<zd>(E * N1 * B2);
    const size_t N2 = N > 2 ? N - 2 : 1;
    x->X2u = cv.take<zd>(E * N2 * B2);
    x->X2l = cv.take<zd>(E * N2 * B2);
    if (d.obc) {
      for (int i = 0; i < 11; ++i) x->wl[i] = cv.take<zd>(2 * E * B2);
      x->w_ok = cv.take<int>(2 * E);
      x->w_info = cv.take<int>(2 * E);
    }
  }
  if (d.obc) {
    x->lead_m = cv.take<zd>(2 * E * B2);
    x->lead_n = cv.take<zd>(2 * E * B2);
    x->lead_np = cv.take<zd>(2 * E * B2);
    x->lead_x = cv.take<zd>(2 * E * B2);
    x->lead_sig = cv.take<zd>(2 * E * B2);
    x->obcL = cv.take<zd>(2 * E * B2);
    x->obcG = cv.take<zd>(2 * E * B2);
    x->lead_iters = cv.take<int>(2 * E);
    x->lead_info = cv.take<int>(2 * E);
    x->lead_piters = cv.take<int>(2 * E);
    x->dec_bytes = bt::decimate_workspace_bytes(d.bs, (int)(2 * E), is_split(d) && d.split_scope == 1);
    x->dec_ws = cv.take<char>(x->dec_bytes);
    if (d.obc_memo) {
      const size_t cap = (size_t)(d.memo_capacity > 0 ? d.memo_capacity : 4 * d.max_energies);
      x->memo_x = cv.take<zd>(cap * 2 * B2);
      x->lead_run = cv.take<int>(2 * E);
      x->lead_conv = cv.take<int>(2 * E);
      x->lead_dec = cv.take<int>(2 * E);
    }
  }
  x->z = cv.take<zd>(E);
  x->tflag = cv.take<int>(1);
  x->fL = cv.take<double>(E);
  x->fR = cv.take<double>(E);
  x->Edev = cv.take<double>(E);
  x->inv_bytes = bt::zinv_workspace_bytes(d.bs, (int)E, is_split(d) && d.split_scope == 1);
  x->inv_ws = cv.take<char>(x->inv_bytes);
  if (is_split(d)) {
    // sweep products batch E; with split_scope = 1 also the decimation's 2E leads
    const int sb = (d.split_scope == 1 && d.obc) ? (int)(2 * E) : (int)E;
    // split_scope = 1 with contacts: the Newton step after decimation runs with 8 slices
    const int ws_slices = d.split_scope == 1 ? (d.obc ? 8 : kept_slices_of(d)) : slices_of(d);
    x->split_bytes = bt::split_workspace_bytes(d.bs, d.bs, d.bs, ws_slices, sb);
    x->split_ws = cv.take<char>(x->split_bytes);
    if (d.bs <= 1024) {
      x->pre_a_bytes = bt::sliced_op_bytes(0, d.bs, d.bs, slices_of(d), (int)E);
      x->pre_b_bytes = bt::sliced_op_bytes(1, d.bs, d.bs, slices_of(d), (int)E);
      for (int i = 0; i < 2; ++i) x->pre_a[i] = cv.take<char>(x->pre_a_bytes);
      for (int i = 0; i < 3; ++i) x->pre_b[i] = cv.take<char>(x->pre_b_bytes);
    }
  }
  return cv.off;
}

bt_status validate_desc(const bt_selinv_desc* d, std::string* why) {
  auto fail = [&](const char* m) { if (why) *why = m; return BT_ERR_INVALID_ARG; };
  if (!d) return fail("desc is NULL");
  if (d->nb < 1) return fail("nb must be >= 1");
  if (d->bs < 1) return fail("bs must be >= 1");
  if (d->max_energies < 1 || d->max_energies > 32767) return fail("max_energies must be in [1, 32767]");
  if (d->system != BT_SYS_G && d->system != BT_SYS_W) return fail("unknown system");
  if (d->precision != BT_FP64 && d->precision != BT_SPLIT) return fail("unknown precision");
  if (d->precision == BT_SPLIT && (d->split_slices != 0 && (d->split_slices < 2 || d->split_slices > 8)))
    return fail("split_slices must be 0 or in [2, 8]");
  if (d->obc && d->nb < 2) return fail("contacts from the edge blocks need nb >= 2");
  if (d->obc && d->system == BT_SYS_G && !(d->kT > 0.0)) return fail("kT must be > 0 with contacts");
  if (d->obc_memo && !d->obc) return fail("contact memoization needs obc = 1");
  if (d->obc_memo && d->system != BT_SYS_G) return fail("contact memoization is for the G system");
  if (d->graph != 0 && d->graph != 1) return fail("graph must be 0 or 1");
  if (d->graph && d->obc_memo) return fail("graph mode and contact memoization are exclusive");
  if (d->split_scope != 0 && d->split_scope != 1) return fail("split_scope must be 0 or 1");
  if (d->gemm_tile != 0 && d->gemm_tile != 16 && d->gemm_tile != 32) return fail("gemm_tile must be 0, 16 or 32");
  if (d->inv_panel != 0 && d->inv_panel != 4 && d->inv_panel != 8 && d->inv_panel != 16 && d->inv_panel != 32)
    return fail("inv_panel must be 0, 4, 8, 16 or 32");
  if (d->obc_memo && d->memo_capacity > 1000000) return fail("memo_capacity too large");
  if (!(d->eta >= 0.0)) return fail("eta must be >= 0");
  if ((double)d->bs * d->bs * d->nb > 4.0e12) return fail("problem too large");
  return BT_OK;
}

struct Blk {  // one block operand for the chunk: pointer at energy 0 of the chunk, energy stride
  const zd* p = nullptr;
  long long es = 0;
  int op = BT_OP_N;
  double f = 1.0;  // real factor folded into alpha
  bool valid() const { return p != nullptr; }
};

inline bt::Operand opnd(const Blk& b, int bs) { return bt::Operand{b.p, bs, b.es, b.op}; }
inline Blk flip(Blk b) { b.op = b.op == BT_OP_N ? BT_OP_C : BT_OP_N; return b; }
inline Blk ws_blk(const zd* p, long long es) { Blk b; b.p = p; b.es = es; return b; }

struct Sweep {
  bt_ctx* c;
  int Ec;
  int N, bs;
  long long B2;
  bool needL, needG, needRlower, keepRoff, has_boff;
  std::function<bt_status(int, zd*, long long)> asmM;              // M~_ii -> dst (energy stride)
  std::function<bt_status(int, int, zd*, long long)> asmB;         // B_ii (which 0:<,1:>) -> dst
  std::function<Blk(int)> Mu, Ml;                                  // M~_{i,i+1}, M~_{i+1,i}
  std::function<Blk(int, int)> Bu;                                 // B_{i,i+1} (which)
  // outputs for this chunk (nullptr = not requested)
  zd *oRu = nullptr, *oRl = nullptr, *oLu = nullptr, *oGu = nullptr;
  long long oes_u = 0;  // energy stride of upper/lower outputs
  // W system: X^R_{i,i+2} and X^R_{i+2,i} (need keepRoff), [E][N-2][B2]
  zd *X2u = nullptr, *X2l = nullptr;
};

bt_status set_err(bt_ctx* c, bt_status s, const char* what) {
  if (s != BT_OK && c) c->err = what;
  return s;
}

// C = alpha op(A) op(B) + beta C for the chunk (bs x bs blocks).  antiherm: the exact result is
// anti-Hermitian (a lesser / greater sandwich x B x^H with B = -B^H, plus an anti-Hermitian C):
// with symmetrised outputs (Sec. 5.2) the result is made exactly anti-Hermitian — the FP64 engine
// computes only the blocks' upper half and mirrors it (about half of the product's FP64 work),
// the sliced engine projects its full result.
// `units`: block products of the paper's formulation that this product stands for (the model
// flop count is 8 b^3 per such product, however the kernels compute it).
// preA / preB: the operand already sliced (sliced products only; ignored by the FP64 engine).
bt_status prod(bt_ctx* c, int Ec, double alpha, const Blk& A, const Blk& B, double beta, zd* C, long long sC,
               bool antiherm = false, double units = 1.0, const bt::SlicedOp* preA = nullptr,
               const bt::SlicedOp* preB = nullptr) {
  const int bs = c->d.bs;
  const double a = alpha * A.f * B.f;
  c->flops += units * 8.0 * bs * (double)bs * bs * Ec;
  if (is_split(c->d)) {
    BT_TRY(bt::split_zgemm(c->st, bs, bs, bs, zmake(a, 0.0), opnd(A, bs), opnd(B, bs), zmake(beta, 0.0), C, bs, sC,
                           Ec, slices_of(c->d), c->split_ws, c->split_bytes, nullptr, c->tflag, 0, preA, preB));
    // the sliced product computes every entry; its result is projected onto the anti-Hermitian
    // matrices so that, as on the FP64 engine, the sandwiches come out exactly anti-Hermitian
    if (antiherm && c->d.symmetrize) return bt::antiherm_project(c->st, bs, Ec, C, sC);
    return BT_OK;
  }
  if (antiherm && c->d.symmetrize)
    return bt::zgemm_antiherm(c->st, bs, bs, zmake(a, 0.0), opnd(A, bs), opnd(B, bs), zmake(beta, 0.0), C, bs, sC, Ec,
                              nullptr, c->d.gemm_tile);
  return bt::zgemm(c->st, bs, bs, bs, zmake(a, 0.0), opnd(A, bs), opnd(B, bs), zmake(beta, 0.0), C, bs, sC, Ec,
                   nullptr, c->d.gemm_tile);
}

bt_status inv(bt_ctx* c, int Ec, zd* A, long long sA, int* info) {
  const int bs = c->d.bs;
  c->flops += 8.0 * bs * (double)bs * bs * Ec;
  return bt::zinv(c->st, bs, A, sA, Ec, info, c->inv_ws, c->inv_bytes, nullptr, &c->eng_kept);
}

// Forward (Eq. 9-10) and backward (Eq. 11-12) passes for one chunk.  x^R, x^<> live in
// c->xR/xL/xG and are overwritten by X^R, X^<> in the backward pass.
bt_status run_sweep(Sweep& s, int* status) {
  bt_ctx* c = s.c;
  const int Ec = s.Ec, N = s.N, bs = s.bs;
  const long long B2 = s.B2, NB2 = (long long)N * B2;
  zd** t = c->t;
  auto xR = [&](int i) { return c->xR + i * B2; };
  auto xLG = [&](int w, int i) { return (w == 0 ? c->xL : c->xG) + i * B2; };
  auto X = [&](zd* p, long long es) { return ws_blk(p, es); };
  const bool need[2] = {s.needL, s.needG};
  // sliced products: an operand that enters several products of a step is sliced once
  const bool reuse = is_split(c->d) && c->pre_a[0] != nullptr;
  auto slice_blk = [&](int role, const Blk& b, int slot, bt::SlicedOp* o) -> bt_status {
    char* buf = role == 0 ? c->pre_a[slot] : c->pre_b[slot];
    const size_t bytes = role == 0 ? c->pre_a_bytes : c->pre_b_bytes;
    return bt::slice_op(c->st, role, bs, bs, opnd(b, bs), Ec, slices_of(c->d), buf, bytes, o);
  };

  // ---------------- forward pass ----------------
  for (int i = 0; i < N; ++i) {
    zd* T1 = t[0];
    if (i > 0) BT_TRY(prod(c, Ec, 1.0, s.Ml(i - 1), X(xR(i - 1), NB2), 0.0, T1, B2));  // M~_{i,i-1} x^R_{i-1}
    BT_TRY(s.asmM(i, xR(i), NB2));
    if (i > 0) BT_TRY(prod(c, Ec, -1.0, X(T1, B2), s.Mu(i - 1), 1.0, xR(i), NB2));      // - ... M~_{i-1,i}
    BT_TRY(inv(c, Ec, xR(i), NB2, status));
    // x^R_i enters both the lesser and the greater sandwich, as op(A) and as op(B)^H
    bt::SlicedOp sxa, sxh;
    if (reuse && need[0] && need[1]) {
      BT_TRY(slice_blk(0, X(xR(i), NB2), 0, &sxa));
      BT_TRY(slice_blk(1, flip(X(xR(i), NB2)), 0, &sxh));
    }
    for (int w = 0; w < 2; ++w) {
      if (!need[w]) continue;
      zd *Bt = t[1], *Tq = t[2], *Y = t[3];
      BT_TRY(s.asmB(i, w, Bt, B2));
      if (i > 0) {
        BT_TRY(prod(c, Ec, 1.0, s.Ml(i - 1), X(xLG(w, i - 1), NB2), 0.0, Tq, B2));        // M~_{i,i-1} x^<>_{i-1}
        BT_TRY(prod(c, Ec, 1.0, X(Tq, B2), flip(s.Ml(i - 1)), 1.0, Bt, B2, true));        // ... M~_{i,i-1}^H
        if (s.has_boff) {
          Blk bu = s.Bu(i - 1, w);
          if (bu.valid()) {
            BT_TRY(prod(c, Ec, 1.0, X(T1, B2), bu, 0.0, Y, B2));                          // y_i
            BT_TRY(bt::add_antiherm(c->st, bs, Ec, Bt, B2, Y, B2, -1.0));                  // - (y - y^H)
          }
        }
      }
      BT_TRY(prod(c, Ec, 1.0, X(xR(i), NB2), X(Bt, B2), 0.0, Tq, B2, false, 1.0, &sxa));
      BT_TRY(prod(c, Ec, 1.0, X(Tq, B2), flip(X(xR(i), NB2)), 0.0, xLG(w, i), NB2, true, 1.0, nullptr,
                  &sxh));  // x^R (...) x^R^H
    }
  }
  // ---------------- backward pass ----------------
  const long long N1B2 = (long long)(N - 1) * B2;
  for (int i = N - 2; i >= 0; --i) {
    zd *U1 = t[0], *W1 = t[1], *V1 = t[2], *P = t[3], *Zt = t[4], *Z = t[5], *Yb = t[6];
    zd* XB[2] = {t[7], t[8]};
    zd* XRn = xR(i + 1);
    BT_TRY(prod(c, Ec, 1.0, X(xR(i), NB2), s.Mu(i), 0.0, U1, B2));                 // x^R_i M~_{i,i+1}
    BT_TRY(prod(c, Ec, 1.0, s.Ml(i), X(xR(i), NB2), 0.0, W1, B2));                 // M~_{i+1,i} x^R_i
    const bool anyLG = s.needL || s.needG;
    const bool both = s.needL && s.needG;
    const bool rl = s.needRlower || s.keepRoff;
    // operands of several products of this step, sliced once: U1 (op(A) of X^R_{i,i+1}, X^R_{i,i+2}
    // and both outputs' x^R M X^<> and Z_i), X^R_{i+1} (op(A) of X^R_{i+1,i} and V1), W1 (op(B)
    // of X^R_{i+1,i}, X^R_{i+2,i} and X^R_i), V1^H and U1^H (op(B) of both outputs' products)
    bt::SlicedOp su1, sxrn, sw1, sv1h, su1h;
    if (reuse) {
      if (anyLG || (s.X2u && i + 2 < N)) BT_TRY(slice_blk(0, X(U1, B2), 0, &su1));
      if (rl && anyLG) BT_TRY(slice_blk(0, X(XRn, NB2), 1, &sxrn));
      if (rl) BT_TRY(slice_blk(1, X(W1, B2), 0, &sw1));
    }
    // X^R_{i,i+1}
    zd* XRu;
    long long esu;
    if (s.keepRoff) { XRu = c->XRu + i * B2; esu = N1B2; }
    else if (s.oRu) { XRu = s.oRu + i * B2; esu = s.oes_u; }
    else { XRu = t[9]; esu = B2; }
    BT_TRY(prod(c, Ec, -1.0, X(U1, B2), X(XRn, NB2), 0.0, XRu, esu, false, 1.0, &su1));
    if (s.keepRoff && s.oRu) BT_TRY(bt::write_blocks(c->st, bs, 1, Ec, XRu, 0, esu, s.oRu + i * B2, 0, s.oes_u, 0));
    if (s.needRlower || s.keepRoff) {
      zd* XRl;
      long long esl;
      if (s.keepRoff) { XRl = c->XRl + i * B2; esl = N1B2; }
      else { XRl = s.oRl + i * B2; esl = s.oes_u; }
      BT_TRY(prod(c, Ec, -1.0, X(XRn, NB2), X(W1, B2), 0.0, XRl, esl, false, 1.0, &sxrn, &sw1));
      if (s.keepRoff && s.oRl) BT_TRY(bt::write_blocks(c->st, bs, 1, Ec, XRl, 0, esl, s.oRl + i * B2, 0, s.oes_u, 0));
    }
    if (s.X2u && i + 2 < N) {
      // X^R_{i,i+2} = -x^R_i M~_{i,i+1} X^R_{i+1,i+2};  X^R_{i+2,i} = -X^R_{i+2,i+1} M~_{i+1,i} x^R_i
      const long long N2B2 = (long long)(N - 2) * B2;
      BT_TRY(prod(c, Ec, -1.0, X(U1, B2), X(c->XRu + (i + 1) * B2, N1B2), 0.0, s.X2u + i * B2, N2B2, false, 1.0,
                  &su1));
      BT_TRY(prod(c, Ec, -1.0, X(c->XRl + (i + 1) * B2, N1B2), X(W1, B2), 0.0, s.X2l + i * B2, N2B2, false, 1.0,
                  nullptr, &sw1));
    }
    if (anyLG) BT_TRY(prod(c, Ec, 1.0, X(XRn, NB2), s.Ml(i), 0.0, V1, B2, false, 1.0, &sxrn));  // X^R_{i+1} M~_{i+1,i}
    if (reuse && both) {
      BT_TRY(slice_blk(1, flip(X(V1, B2)), 1, &sv1h));
      BT_TRY(slice_blk(1, flip(X(U1, B2)), 2, &su1h));
    }
    if (anyLG && s.has_boff) {
      for (int w = 0; w < 2; ++w) {
        if (!need[w]) continue;
        Blk bu = s.Bu(i, w);
        if (bu.valid()) BT_TRY(prod(c, Ec, 1.0, X(xR(i), NB2), bu, 0.0, XB[w], B2)); // x^R_i B_{i,i+1}
      }
    }
    BT_TRY(prod(c, Ec, -1.0, X(XRu, esu), X(W1, B2), 1.0, xR(i), NB2, false, 1.0, nullptr, &sw1));  // X^R_i (Eq. 11)
    for (int w = 0; w < 2; ++w) {
      if (!need[w]) continue;
      zd* xLi = xLG(w, i);
      zd* XLn = xLG(w, i + 1);
      zd* oU = w == 0 ? s.oLu : s.oGu;
      const bool bu_valid = s.has_boff && s.Bu(i, w).valid();
      BT_TRY(prod(c, Ec, 1.0, X(U1, B2), X(XLn, NB2), 0.0, P, B2, false, 1.0, &su1));  // x^R M X^<>_{i+1}
      // With exactly anti-Hermitian x^<>_i (symmetrised outputs: the sandwiches above are computed
      // so), Z_i = -X^R_{i,i+1} M~_{i+1,i} x^<>_i = U1 V1 x^<>_i = U1 D^H with
      // D = -x^<>_i V1^H, the first term of X^<>_{i,i+1}: one product instead of two.
      const bool z_from_d = c->d.symmetrize != 0;
      zd* d = oU ? oU + i * B2 : Zt;
      const long long des = oU ? s.oes_u : B2;
      if (oU || z_from_d) {
        BT_TRY(prod(c, Ec, -1.0, X(xLi, NB2), flip(X(V1, B2)), 0.0, d, des, false,    // D = - x^<> (X^R M)^H
                    oU ? 1.0 : 0.0, nullptr, &sv1h));
        if (z_from_d)
          BT_TRY(prod(c, Ec, 1.0, X(U1, B2), flip(X(d, des)), 0.0, Z, B2, false, 2.0, &su1));  // Z_i
      }
      if (oU) {
        BT_TRY(bt::axpby(c->st, B2, Ec, -1.0, P, B2, 1.0, d, s.oes_u));             // - x^R M X^<>
        if (bu_valid)
          BT_TRY(prod(c, Ec, 1.0, X(XB[w], B2), flip(X(XRn, NB2)), 1.0, d, s.oes_u));  // + x^R B X^R^H
      }
      if (!z_from_d) {
        BT_TRY(prod(c, Ec, 1.0, s.Ml(i), X(xLi, NB2), 0.0, Zt, B2));                // M~_{i+1,i} x^<>_i
        BT_TRY(prod(c, Ec, -1.0, X(XRu, esu), X(Zt, B2), 0.0, Z, B2));              // Z_i
      }
      BT_TRY(prod(c, Ec, 1.0, X(P, B2), flip(X(U1, B2)), 1.0, xLi, NB2, true, 1.0, nullptr, &su1h));  // + x M X M^H x^H
      BT_TRY(bt::add_antiherm(c->st, bs, Ec, xLi, NB2, Z, B2, 1.0));                // + (Z - Z^H)
      if (bu_valid) {
        BT_TRY(prod(c, Ec, -1.0, X(XB[w], B2), flip(X(XRu, esu)), 0.0, Yb, B2));    // Y_i
        BT_TRY(bt::add_antiherm(c->st, bs, Ec, xLi, NB2, Yb, B2, -1.0));            // - (Y - Y^H)
      }
    }
  }
  return BT_OK;
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================

extern "C" bt_status bt_selinv_workspace_bytes(const bt_selinv_desc* desc, size_t* bytes) {
  std::string why;
  if (!bytes) return BT_ERR_INVALID_ARG;
  bt_status s = validate_desc(desc, &why);
  if (s != BT_OK) return s;
  *bytes = layout(nullptr, *desc, nullptr);
  return BT_OK;
}

namespace bt {

// Creates a context.  With ext_ws == nullptr the workspace is allocated here (cudaMalloc) and
// host staging buffers are pinned; otherwise the caller lends ext_bytes of device memory at
// ext_ws (a serving arena) and host buffers are pageable, so creation allocates no device or
// pinned memory.
bt_status ctx_create(const bt_selinv_desc* desc, void* cuda_stream, void* ext_ws, size_t ext_bytes, bt_ctx** out,
                     std::string* err) {
  if (!out) { *err = "out is NULL"; return BT_ERR_INVALID_ARG; }
  *out = nullptr;
  bt_status s = validate_desc(desc, err);
  if (s != BT_OK) return s;
  bt_selinv_desc d = *desc;
  if (!(d.decim_tol > 0.0)) d.decim_tol = 1e-14;
  if (d.decim_maxit <= 0) d.decim_maxit = 100;
  if (d.memo_nfpi <= 0) d.memo_nfpi = 20;
  if (d.memo_capacity <= 0) d.memo_capacity = 4 * d.max_energies;
  if (d.decim_newton_after == 0) d.decim_newton_after = 14;
  const size_t need = layout(nullptr, d, nullptr);
  if (d.hbm_budget_bytes && need > d.hbm_budget_bytes) {
    *err = "workspace exceeds hbm_budget_bytes";
    return BT_ERR_BUDGET;
  }
  if (ext_ws && ext_bytes < need) {
    *err = "lent workspace is too small";
    return BT_ERR_INVALID_ARG;
  }
  bt_ctx* c = new (std::nothrow) bt_ctx();
  if (!c) { *err = "host allocation failed"; return BT_ERR_OOM; }
  c->d = d;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  if (ext_ws) {
    c->ws = static_cast<char*>(ext_ws);
    c->owns_ws = false;
  } else if (cudaMalloc(&c->ws, need) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    *err = "cudaMalloc of the workspace failed";
    return BT_ERR_OOM;
  }
  c->ws_bytes = need;
  layout(c, d, c->ws);
  if (ext_ws) {
    c->h_pinned = new int[16];
    c->h_E = new double[d.max_energies];
    c->pinned = false;
  } else if (cudaMallocHost(&c->h_pinned, 64) != cudaSuccess ||
             cudaMallocHost(&c->h_E, sizeof(double) * d.max_energies) != cudaSuccess) {
    cudaGetLastError();
    bt_selinv_destroy(c);
    *err = "pinned host allocation failed";
    return BT_ERR_OOM;
  }
  if (d.graph) {
    if (!c->st) {
      bt_selinv_destroy(c);
      *err = "graph mode needs a non-default stream (stream capture)";
      return BT_ERR_INVALID_ARG;
    }
    if (cudaStreamCreateWithFlags(&c->body_st, cudaStreamNonBlocking) != cudaSuccess ||
        (c->pinned ? cudaMallocHost(&c->h_iters, sizeof(int) * 4 * d.max_energies) != cudaSuccess
                   : (c->h_iters = new int[4 * d.max_energies]) == nullptr)) {
      cudaGetLastError();
      bt_selinv_destroy(c);
      *err = "graph mode set-up failed";
      return BT_ERR_CUDA;
    }
  }
  c->stats.workspace_bytes = need;
  if (is_split(d) && d.split_scope == 1)
    c->eng_kept = bt::Engine{kept_slices_of(d), c->split_ws, c->split_bytes, c->tflag};
  c->eng_kept.tile = d.gemm_tile;
  c->eng_kept.panel = d.inv_panel;
  c->eng_polish.tile = d.gemm_tile;
  if (is_split(d) && d.split_scope == 1) c->eng_polish = bt::Engine{8, c->split_ws, c->split_bytes, c->tflag};
  if (d.obc_memo) {
    c->memo_key.assign(d.memo_capacity, 0);
    c->memo_used.assign(d.memo_capacity, 0);
  }
  *out = c;
  return BT_OK;
}

size_t ctx_workspace_bytes(const bt_selinv_desc& d) { return layout(nullptr, d, nullptr); }

}  // namespace bt

extern "C" bt_status bt_selinv_create(const bt_selinv_desc* desc, void* cuda_stream, bt_ctx** out) {
  g_create_error.clear();
  return bt::ctx_create(desc, cuda_stream, nullptr, 0, out, &g_create_error);
}

extern "C" bt_status bt_selinv_destroy(bt_ctx* c) {
  if (!c) return BT_OK;
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  if (c->body_st) cudaStreamDestroy(c->body_st);
  if (c->h_iters) {
    if (c->pinned) cudaFreeHost(c->h_iters);
    else delete[] c->h_iters;
  }
  if (c->copy_st) cudaStreamSynchronize(c->copy_st);
  if (c->ws && c->owns_ws) cudaFree(c->ws);
  if (c->stage) cudaFree(c->stage);
  if (c->gstage) cudaFree(c->gstage);
  for (cudaEvent_t ev : {c->ev_done[0], c->ev_done[1], c->ev_ready})
    if (ev) cudaEventDestroy(ev);
  if (c->copy_st) cudaStreamDestroy(c->copy_st);
  if (c->pinned) {
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->h_E) cudaFreeHost(c->h_E);
  } else {
    delete[] c->h_pinned;
    delete[] c->h_E;
  }
  delete c;
  return BT_OK;
}

extern "C" const char* bt_selinv_last_error(const bt_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

namespace {

// Graph mode: folds the device-side decimation counts of the last replayed chunk into the
// statistics.  The caller has synchronised the stream.
void fold_pending(bt_ctx* c) {
  if (!c->pending) return;
  c->pending = false;
  long long it_max = 0, lead_its = 0, pit_max = 0, p_its = 0, p_leads = 0;
  const int L = 2 * c->pending_Ec;
  for (int l = 0; l < L; ++l) {
    const long long v = c->h_iters[l] > 0 ? c->h_iters[l] : 0;
    it_max = v > it_max ? v : it_max;
    lead_its += v;
    const long long p = c->h_iters[L + l] > 0 ? c->h_iters[L + l] : 0;
    pit_max = p > pit_max ? p : pit_max;
    p_its += p;
    p_leads += p > 0;
  }
  const double U = 8.0 * c->d.bs * (double)c->d.bs * c->d.bs;
  c->stats.decim_iterations += it_max;
  c->stats.lead_iterations += lead_its;
  c->stats.newton_leads += p_leads;
  c->stats.newton_iterations += p_its;
  // the doubling loop body runs at least once per replay
  c->stats.kernel_launches += c->pending_body * it_max + c->pending_polish_body * (pit_max > 0 ? pit_max : 1);
  c->flops += 7.0 * U * (double)lead_its + 4.0 * U * (double)(p_its + p_leads);
  c->stats.flops_model = c->flops;
}

}  // namespace

extern "C" bt_status bt_selinv_get_stats(const bt_ctx* c, bt_stats* out) {
  if (!c || !out) return BT_ERR_INVALID_ARG;
  if (c->pending) {
    bt_ctx* m = const_cast<bt_ctx*>(c);  // a handle is single-threaded; the read-back is folded here
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return BT_ERR_CUDA;
    fold_pending(m);
  }
  *out = c->stats;
  return BT_OK;
}

namespace {

// per-energy element extents of a bt_bt operand
long long diag_extent(const bt_bt& b, int nb, int bs) {
  if (b.layout == BT_LAYOUT_DIAGVEC) return (long long)nb * bs;
  if (b.layout == BT_LAYOUT_PACKED_UPPER) return (long long)nb * bs * (bs + 1) / 2;
  return (long long)nb * bs * bs;
}
long long off_extent(int nb, int bs) { return (long long)(nb > 1 ? nb - 1 : 0) * bs * bs; }

bt_status validate_operand(const bt_bt* b, bool required, bool allow_diagvec, const char* name, std::string* why,
                           bool allow_packed = false) {
  if (!b) {
    if (required) { *why = std::string(name) + " is required"; return BT_ERR_INVALID_ARG; }
    return BT_OK;
  }
  if (!b->diag && required) { *why = std::string(name) + ".diag is required"; return BT_ERR_INVALID_ARG; }
  if (b->layout == BT_LAYOUT_PACKED_UPPER) {
    // Sec. 5.2: an anti-Hermitian operand stored by the upper triangles of its diagonal blocks
    if (!allow_packed || b->symmetry != BT_SYM_ANTIHERMITIAN) {
      *why = std::string(name) + ": packed upper-triangle input is for anti-Hermitian lesser / greater operands";
      return BT_ERR_INVALID_ARG;
    }
    return BT_OK;
  }
  if (b->layout != BT_LAYOUT_BLOCKS && b->layout != BT_LAYOUT_DIAGVEC) { *why = std::string(name) + ": bad layout"; return BT_ERR_INVALID_ARG; }
  if (b->layout == BT_LAYOUT_DIAGVEC && !allow_diagvec) { *why = std::string(name) + ": diagonal-vector layout not accepted"; return BT_ERR_INVALID_ARG; }
  if (b->layout == BT_LAYOUT_DIAGVEC && (b->upper || b->lower)) { *why = std::string(name) + ": diagonal-vector layout has no off-diagonal blocks"; return BT_ERR_INVALID_ARG; }
  if (b->symmetry < BT_SYM_GENERAL || b->symmetry > BT_SYM_ANTIHERMITIAN) { *why = std::string(name) + ": bad symmetry"; return BT_ERR_INVALID_ARG; }
  if (b->upper && b->symmetry == BT_SYM_GENERAL && !b->lower) { *why = std::string(name) + ": general symmetry needs lower blocks"; return BT_ERR_INVALID_ARG; }
  return BT_OK;
}

// Offset an operand to energy e0 of the solve.
const zd* at_energy(const void* p, int per_energy, long long extent, long long e0) {
  if (!p) return nullptr;
  const zd* q = static_cast<const zd*>(p);
  return per_energy ? q + extent * e0 : q;
}

// a5: diagonal blocks of the chunk from the workspace [Ec][N][b][b] to the caller's output,
// as full blocks or as the diagonal-vector layout; mode 1 applies (X - X^H)/2.
bt_status write_diag_out(bt_ctx* c, int Ec, const zd* src, const bt_bt_out* o, long long e0, int mode) {
  if (!o || !o->diag) return BT_OK;
  const int N = c->d.nb, bs = c->d.bs;
  const long long B2 = (long long)bs * bs, NB2 = N * B2;
  if (o->layout == BT_LAYOUT_DIAGVEC)
    return bt::write_diagvec(c->st, bs, N, Ec, src, B2, NB2, static_cast<zd*>(o->diag) + e0 * N * bs, bs,
                             (long long)N * bs, mode);
  if (o->layout == BT_LAYOUT_PACKED_UPPER) {
    const long long pk = (long long)N * bs * (bs + 1) / 2;
    return bt::write_packed(c->st, bs, N, Ec, src, B2, NB2, static_cast<zd*>(o->diag) + e0 * pk, pk);
  }
  return bt::write_blocks(c->st, bs, N, Ec, src, B2, NB2, static_cast<zd*>(o->diag) + e0 * NB2, B2, NB2, mode);
}

// a2: Sancho-Rubio decimation of the chunk's 2 Ec leads (c->lead_m, lead_n, lead_np -> lead_x and
// lead_sig = n x n'), with the Newton step for slowly decaying leads; statistics and model flops.
bt_status decimate_leads(bt_ctx* c, int Ec, const int* dec_mask) {
  const bt_selinv_desc& d = c->d;
  const int bs = d.bs;
  const double U = 8.0 * bs * (double)bs * bs;
  int it_max = 0;
  long long lead_its = 0;
  bt::Polish pol;
  pol.after = d.decim_newton_after;
  pol.iters = c->lead_piters;
  pol.engine = &c->eng_polish;
  bt_status s = bt::decimate(c->st, bs, 2 * Ec, c->lead_m, c->lead_n, c->lead_np, d.decim_tol, d.decim_maxit, c->lead_x,
                             c->lead_sig, c->lead_iters, c->lead_info, c->dec_ws, c->dec_bytes, &it_max, c->h_pinned,
                             dec_mask, &lead_its, &c->eng_kept, c->loop, &pol);
  if (s != BT_OK) return set_err(c, s, "decimation failed to launch");
  c->stats.decim_iterations += it_max;
  c->stats.lead_iterations += lead_its;
  // 7 products per lead-iteration, then x = e_s^{-1} and n x n' for every lead
  c->flops += 7.0 * U * (double)lead_its + 3.0 * U * 2.0 * Ec;
  if (c->loop) {
    c->cap_polish_body += pol.body_launches;
  } else if (pol.after >= 0) {
    // Newton step: 4 products per doubling iteration; n x, x n', n x n' and the inverse per lead
    const long long p_leads = pol.lead_iterations > 0 ? pol.selected : 0;
    c->stats.newton_leads += p_leads;
    c->stats.newton_iterations += pol.lead_iterations;
    c->flops += 4.0 * U * (double)(pol.lead_iterations + p_leads);
  }
  return BT_OK;
}

// e0: the chunk's first energy in the outputs; ein: in the inputs (e0, or 0 for staged inputs)
bt_status solve_chunk_g(bt_ctx* c, const bt_bt* H, const bt_bt* S, const bt_bt* sR, const bt_bt* sL, const bt_bt* sG,
                        long long e0, long long ein, int Ec, const bt_bt_out* oR, const bt_bt_out* oL,
                        const bt_bt_out* oG, int* status) {
  const bt_selinv_desc& d = c->d;
  const int N = d.nb, bs = d.bs;
  const long long B2 = (long long)bs * bs, NB2 = N * B2, N1B2 = (long long)(N > 1 ? N - 1 : 0) * B2;
  cudaStream_t st = c->st;
  auto dstride = [&](const bt_bt* b) { return b && b->per_energy ? diag_extent(*b, N, bs) : 0LL; };
  auto ostride = [&](const bt_bt* b) { return b && b->per_energy ? off_extent(N, bs) : 0LL; };
  const zd* Hd = at_energy(H->diag, H->per_energy, diag_extent(*H, N, bs), ein);
  const zd* Hu = at_energy(H->upper, H->per_energy, off_extent(N, bs), ein);
  const zd* Hl = at_energy(H->lower, H->per_energy, off_extent(N, bs), ein);
  const zd *Sd = nullptr, *Su = nullptr, *Sl = nullptr;
  if (S) {
    Sd = at_energy(S->diag, S->per_energy, diag_extent(*S, N, bs), ein);
    Su = at_energy(S->upper, S->per_energy, off_extent(N, bs), ein);
    Sl = at_energy(S->lower, S->per_energy, off_extent(N, bs), ein);
  }
  const zd *Rd = nullptr, *Ru = nullptr, *Rl = nullptr;
  if (sR) {
    Rd = at_energy(sR->diag, sR->per_energy, diag_extent(*sR, N, bs), ein);
    Ru = at_energy(sR->upper, sR->per_energy, off_extent(N, bs), ein);
    Rl = at_energy(sR->lower, sR->per_energy, off_extent(N, bs), ein);
  }
  const bt_bt* sLG[2] = {sL, sG};
  const zd *LGd[2] = {nullptr, nullptr}, *LGu[2] = {nullptr, nullptr};
  for (int w = 0; w < 2; ++w)
    if (sLG[w]) {
      LGd[w] = at_energy(sLG[w]->diag, sLG[w]->per_energy, diag_extent(*sLG[w], N, bs), ein);
      LGu[w] = at_energy(sLG[w]->upper, sLG[w]->per_energy, off_extent(N, bs), ein);
    }

  // energies -> z, Fermi factors
  BT_TRY(bt::energy_setup(st, Ec, c->Edev, d.eta, d.mu_left, d.mu_right, d.kT, c->z, c->fL, c->fR));

  // Does M~ have per-energy off-diagonal blocks?  (S or Sigma^R with off-diagonal blocks, or
  // a per-energy H): then they are assembled into c->Mu / c->Ml, else M~_{i,i+1} = -H_{i,i+1}.
  const bool general_off = (S && Su) || (sR && Ru) || H->per_energy;
  auto h_off = [&](int i, bool upper, bt::MBlockArgs& a) {
    // a.H := H_{i,i+1} (upper) or H_{i+1,i} (lower)
    if (upper) { a.H = Hu ? Hu + i * B2 : nullptr; a.H_stride = ostride(H); return; }
    if (H->symmetry == BT_SYM_GENERAL) { a.H = Hl ? Hl + i * B2 : nullptr; a.H_stride = ostride(H); return; }
    a.H = Hu ? Hu + i * B2 : nullptr;
    a.H_stride = ostride(H);
    a.H_conjT = 1;
    a.H_sign = H->symmetry == BT_SYM_ANTIHERMITIAN ? -1.0 : 1.0;
  };
  auto off_args = [&](int i, bool upper, zd* out, long long out_stride) {
    bt::MBlockArgs a;
    a.out = out;
    a.out_stride = out_stride;
    a.z = c->z;
    h_off(i, upper, a);
    if (S && Su) {  // overlap: Hermitian unless given in full
      a.use_z = 1;
      if (upper || S->symmetry == BT_SYM_GENERAL) { a.S = (upper ? Su : Sl) + i * B2; }
      else { a.S = Su + i * B2; a.S_conjT = 1; }
      a.S_stride = ostride(S);
    }
    if (sR && Ru) {
      if (upper || sR->symmetry == BT_SYM_GENERAL) { a.sig = (upper ? Ru : Rl) + i * B2; }
      else { a.sig = Ru + i * B2; a.sig_conjT = 1; a.sig_sign = sR->symmetry == BT_SYM_ANTIHERMITIAN ? -1.0 : 1.0; }
      a.sig_stride = ostride(sR);
    }
    return a;
  };
  if (general_off) {
    for (int i = 0; i < N - 1; ++i) {
      BT_TRY(bt::assemble_m(st, bs, Ec, off_args(i, true, c->Mu + i * B2, N1B2)));
      BT_TRY(bt::assemble_m(st, bs, Ec, off_args(i, false, c->Ml + i * B2, N1B2)));
    }
  }
  auto diag_args = [&](int i, zd* out, long long out_stride, bool with_obc) {
    bt::MBlockArgs a;
    a.out = out;
    a.out_stride = out_stride;
    a.z = c->z;
    a.use_z = 1;
    if (S && Sd) { a.S = Sd + i * B2; a.S_stride = dstride(S); }
    else a.S_identity = 1;
    a.H = Hd + i * B2;
    a.H_stride = dstride(H);
    if (sR && Rd) {
      if (sR->layout == BT_LAYOUT_DIAGVEC) { a.sigvec = Rd + (long long)i * bs; a.sigvec_stride = dstride(sR); }
      else { a.sig = Rd + i * B2; a.sig_stride = dstride(sR); }
    }
    if (with_obc && d.obc) {
      a.obc_stride = B2;
      if (i == 0) a.obc1 = c->lead_sig;
      if (i == N - 1) a.obc2 = c->lead_sig + (long long)Ec * B2;
    }
    return a;
  };

  // ---------------- a2: contacts ----------------
  if (d.obc) {
    // left lead: m = M_11, n = M_21, n' = M_12;  right lead: m = M_NN, n = M_{N-1,N}, n' = M_{N,N-1}
    BT_TRY(bt::assemble_m(st, bs, Ec, diag_args(0, c->lead_m, B2, false)));
    BT_TRY(bt::assemble_m(st, bs, Ec, diag_args(N - 1, c->lead_m + Ec * B2, B2, false)));
    BT_TRY(bt::assemble_m(st, bs, Ec, off_args(0, false, c->lead_n, B2)));
    BT_TRY(bt::assemble_m(st, bs, Ec, off_args(0, true, c->lead_np, B2)));
    BT_TRY(bt::assemble_m(st, bs, Ec, off_args(N - 2, true, c->lead_n + Ec * B2, B2)));
    BT_TRY(bt::assemble_m(st, bs, Ec, off_args(N - 2, false, c->lead_np + Ec * B2, B2)));
    long long fpi_its = 0;
    const double U = 8.0 * bs * (double)bs * bs;
    const int* dec_mask = nullptr;
    std::vector<int> slots;
    if (d.obc_memo) {
      // Sec. 5.3: energies solved before start the fixed point (Eq. 5) from their kept surface
      // functions; leads that do not converge within memo_nfpi iterations are decimated.
      std::vector<int> run(2 * Ec, 0);
      slots.assign(Ec, -1);
      for (int e = 0; e < Ec; ++e) {
        uint64_t key;
        std::memcpy(&key, &c->h_E[e], sizeof(key));
        auto it = c->memo_slot.find(key);
        if (it == c->memo_slot.end()) continue;
        slots[e] = it->second;
        run[e] = run[Ec + e] = 1;
        for (int side = 0; side < 2; ++side)
          BT_CUDA_TRY(cudaMemcpyAsync(c->lead_x + (long long)(side * Ec + e) * B2,
                                      c->memo_x + ((long long)it->second * 2 + side) * B2, sizeof(zd) * B2,
                                      cudaMemcpyDeviceToDevice, st));
      }
      c->stats.memo_hits += (long long)std::count_if(slots.begin(), slots.end(), [](int v) { return v >= 0; });
      BT_CUDA_TRY(cudaMemcpyAsync(c->lead_run, run.data(), sizeof(int) * 2 * Ec, cudaMemcpyHostToDevice, st));
      BT_CUDA_TRY(cudaMemsetAsync(c->lead_info, 0, sizeof(int) * 2 * Ec, st));
      BT_TRY(bt::fixed_point(st, bs, 2 * Ec, c->lead_m, c->lead_n, c->lead_np, c->lead_x, c->lead_run, c->lead_conv,
                             // fixed-point target: 1e-12 of |x| (FP64 rounding already moves the
                             // surface function of an in-band lead by ~1e-13 at eta = 1e-6)
                             d.memo_nfpi, d.decim_tol > 1e-12 ? d.decim_tol : 1e-12, c->lead_info, c->dec_ws,
                             c->dec_bytes, c->h_pinned, &fpi_its,
                             &c->eng_kept));
      BT_TRY(bt::invert_mask(st, 2 * Ec, c->lead_conv, c->lead_dec));
      dec_mask = c->lead_dec;
      c->flops += 3.0 * U * (double)fpi_its;
    }
    BT_TRY(decimate_leads(c, Ec, dec_mask));
    c->stats.fpi_iterations += fpi_its;
    if (d.obc_memo) {
      // keep this chunk's surface functions (oldest entries evicted first)
      for (int e = 0; e < Ec; ++e) {
        uint64_t key;
        std::memcpy(&key, &c->h_E[e], sizeof(key));
        int slot = slots[e];
        if (slot < 0) {
          slot = c->memo_next;
          c->memo_next = (c->memo_next + 1) % d.memo_capacity;
          if (c->memo_used[slot]) c->memo_slot.erase(c->memo_key[slot]);
          c->memo_used[slot] = 1;
          c->memo_key[slot] = key;
          c->memo_slot[key] = slot;
        }
        for (int side = 0; side < 2; ++side)
          BT_CUDA_TRY(cudaMemcpyAsync(c->memo_x + ((long long)slot * 2 + side) * B2,
                                      c->lead_x + (long long)(side * Ec + e) * B2, sizeof(zd) * B2,
                                      cudaMemcpyDeviceToDevice, st));
      }
    }
    BT_TRY(bt::merge_status(st, Ec, c->lead_info, 2, Ec, status));
    BT_TRY(bt::obc_lesser_greater(st, bs, Ec, c->lead_sig, c->fL, c->fR, c->obcL, c->obcG));
  }

  // ---------------- a1 + a3 + a4 ----------------
  Sweep sw;
  sw.c = c;
  sw.Ec = Ec;
  sw.N = N;
  sw.bs = bs;
  sw.B2 = B2;
  sw.needL = oL && (oL->diag || oL->upper);
  sw.needG = oG && (oG->diag || oG->upper);
  sw.needRlower = oR && oR->lower;
  sw.keepRoff = false;
  sw.has_boff = (LGu[0] != nullptr) || (LGu[1] != nullptr);
  sw.oRu = oR && oR->upper ? static_cast<zd*>(oR->upper) + e0 * N1B2 : nullptr;
  sw.oRl = oR && oR->lower ? static_cast<zd*>(oR->lower) + e0 * N1B2 : nullptr;
  sw.oLu = oL && oL->upper ? static_cast<zd*>(oL->upper) + e0 * N1B2 : nullptr;
  sw.oGu = oG && oG->upper ? static_cast<zd*>(oG->upper) + e0 * N1B2 : nullptr;
  sw.oes_u = N1B2;
  sw.asmM = [&](int i, zd* dst, long long es) { return bt::assemble_m(st, bs, Ec, diag_args(i, dst, es, true)); };
  sw.asmB = [&](int i, int w, zd* dst, long long es) {
    bt::BBlockArgs a;
    a.out = dst;
    a.out_stride = es;
    if (LGd[w]) {
      if (sLG[w]->layout == BT_LAYOUT_DIAGVEC) { a.sigvec = LGd[w] + (long long)i * bs; a.sigvec_stride = dstride(sLG[w]); }
      else if (sLG[w]->layout == BT_LAYOUT_PACKED_UPPER) {
        a.sig = LGd[w] + (long long)i * bs * (bs + 1) / 2;
        a.sig_stride = dstride(sLG[w]);
        a.sig_packed = 1;
      } else { a.sig = LGd[w] + i * B2; a.sig_stride = dstride(sLG[w]); }
    }
    if (d.obc) {
      const zd* ob = w == 0 ? c->obcL : c->obcG;
      a.obc_stride = B2;
      if (i == 0) a.obc1 = ob;
      if (i == N - 1) a.obc2 = ob + (long long)Ec * B2;
    }
    return bt::assemble_b(st, bs, Ec, a);
  };
  if (general_off) {
    sw.Mu = [&](int i) { return ws_blk(c->Mu + i * B2, N1B2); };
    sw.Ml = [&](int i) { return ws_blk(c->Ml + i * B2, N1B2); };
  } else {
    sw.Mu = [&](int i) { Blk b; b.p = Hu + i * B2; b.es = 0; b.op = BT_OP_N; b.f = -1.0; return b; };
    sw.Ml = [&](int i) {
      Blk b;
      b.es = 0;
      if (H->symmetry == BT_SYM_GENERAL) { b.p = Hl + i * B2; b.op = BT_OP_N; b.f = -1.0; }
      else { b.p = Hu + i * B2; b.op = BT_OP_C; b.f = H->symmetry == BT_SYM_ANTIHERMITIAN ? 1.0 : -1.0; }
      return b;
    };
  }
  sw.Bu = [&](int i, int w) {
    Blk b;
    if (LGu[w]) { b.p = LGu[w] + i * B2; b.es = ostride(sLG[w]); }
    return b;
  };
  if (N > 1 && !Hu) return set_err(c, BT_ERR_INVALID_ARG, "H.upper is required for nb > 1");
  BT_TRY(run_sweep(sw, status));

  // ---------------- a5: write-out ----------------
  BT_TRY(write_diag_out(c, Ec, c->xR, oR, e0, 0));
  BT_TRY(write_diag_out(c, Ec, c->xL, oL, e0, d.symmetrize ? 1 : 0));
  BT_TRY(write_diag_out(c, Ec, c->xG, oG, e0, d.symmetrize ? 1 : 0));
  return BT_OK;
}


// W system (Table 2, right column): M~ = I - V P^R, B^<> = V P^<> V^H as block-tridiagonal
// products (Sec. 4.3.1; exact when the cell is longer than 3 r_cut), the RGF sweep on them, and
// W^R = X^R V on the selected blocks (X^R_{i,i+-2} from the backward pass).  W^<> = X^<>.
bt_status solve_chunk_w(bt_ctx* c, const bt_bt* V, const bt_bt* PR, const bt_bt* PL, const bt_bt* PG, long long e0,
                        long long ein, int Ec, const bt_bt_out* oR, const bt_bt_out* oL, const bt_bt_out* oG,
                        int* status) {
  const bt_selinv_desc& d = c->d;
  const int N = d.nb, bs = d.bs;
  const long long B2 = (long long)bs * bs, NB2 = N * B2, N1B2 = (long long)(N > 1 ? N - 1 : 0) * B2;
  const long long N2B2 = (long long)(N > 2 ? N - 2 : 0) * B2;
  cudaStream_t st = c->st;
  const zd* Vd = static_cast<const zd*>(V->diag);
  const zd* Vu = static_cast<const zd*>(V->upper);
  auto Vb = [&](int i, int j) {  // V_{ij}, |i-j| <= 1, V Hermitian
    Blk b;
    b.es = 0;
    if (i == j) { b.p = Vd + i * B2; }
    else if (j == i + 1) { b.p = Vu + i * B2; }
    else { b.p = Vu + j * B2; b.op = BT_OP_C; }
    return b;
  };
  auto Vh = [&](int i, int j) { return flip(Vb(i, j)); };  // (V_{ij})^H
  struct PT { const zd *d, *u, *l; long long ed, eo; int sym; };
  auto mkP = [&](const bt_bt* P) {
    PT p{};
    if (!P) return p;
    p.ed = P->per_energy ? diag_extent(*P, N, bs) : 0;
    p.eo = P->per_energy ? N1B2 : 0;
    p.d = at_energy(P->diag, P->per_energy, diag_extent(*P, N, bs), ein);
    p.u = at_energy(P->upper, P->per_energy, N1B2, ein);
    p.l = at_energy(P->lower, P->per_energy, N1B2, ein);
    p.sym = P->symmetry;
    return p;
  };
  auto Pb = [&](const PT& p, int i, int j) {  // P_{ij} for energy 0 of the chunk
    Blk b;
    if (i == j) { b.p = p.d + i * B2; b.es = p.ed; }
    else if (j == i + 1) { b.p = p.u + i * B2; b.es = p.eo; }
    else if (p.sym == BT_SYM_GENERAL) { b.p = p.l + j * B2; b.es = p.eo; }
    else { b.p = p.u + j * B2; b.es = p.eo; b.op = BT_OP_C; b.f = p.sym == BT_SYM_ANTIHERMITIAN ? -1.0 : 1.0; }
    return b;
  };
  auto W = [&](zd* p, long long es) { return ws_blk(p, es); };

  // ---- a1 (W): M~ = I - V P^R ----
  const PT pr = mkP(PR);
  const bool wobc = d.obc != 0;
  for (int i = 0; i < N; ++i) {
    zd* md = c->Md + i * B2;
    BT_TRY(prod(c, Ec, -1.0, Vb(i, i), Pb(pr, i, i), 0.0, md, NB2));
    if (i > 0) BT_TRY(prod(c, Ec, -1.0, Vb(i, i - 1), Pb(pr, i - 1, i), 1.0, md, NB2));
    if (i + 1 < N) BT_TRY(prod(c, Ec, -1.0, Vb(i, i + 1), Pb(pr, i + 1, i), 1.0, md, NB2));
    BT_TRY(bt::shift_diag(st, bs, Ec, md, NB2, 1.0));
    if (i + 1 < N) {
      zd* mu = c->Mu + i * B2;
      zd* ml = c->Ml + i * B2;
      BT_TRY(prod(c, Ec, -1.0, Vb(i, i), Pb(pr, i, i + 1), 0.0, mu, N1B2));
      BT_TRY(prod(c, Ec, -1.0, Vb(i, i + 1), Pb(pr, i + 1, i + 1), 1.0, mu, N1B2));
      BT_TRY(prod(c, Ec, -1.0, Vb(i + 1, i), Pb(pr, i, i), 0.0, ml, N1B2));
      BT_TRY(prod(c, Ec, -1.0, Vb(i + 1, i + 1), Pb(pr, i + 1, i), 1.0, ml, N1B2));
    }
  }
  const bool needL = oL && (oL->diag || oL->upper);
  const bool needG = oG && (oG->diag || oG->upper);
  const bool need[2] = {needL, needG};
  PT plg[2] = {mkP(PL), mkP(PG)};
  zd* Bd[2] = {c->BdL, c->BdG};
  zd* Bu[2] = {c->BuL, c->BuG};
  // P^<> given by the upper triangles of its diagonal blocks (Sec. 5.2): the chunk's diagonal
  // blocks are unpacked into the B^<> buffer, which is free until the B^<> assembly (the products
  // that read P^<> all run before it)
  const bt_bt* Plg[2] = {PL, PG};
  for (int w = 0; w < 2; ++w) {
    if (!need[w] || !Plg[w] || Plg[w]->layout != BT_LAYOUT_PACKED_UPPER) continue;
    BT_TRY(bt::unpack_antiherm(st, bs, N, Ec, plg[w].d, plg[w].ed, Bd[w], B2, NB2));
    plg[w].d = Bd[w];
    plg[w].ed = NB2;
  }

  // ---- W contacts (Sec. 4.2: the retarded boundary by Eq. 4, the lesser / greater boundary by
  // the Stein equation of Eq. 7) ----
  // Each lead repeats the device's edge cell of V and P and its coupling to the next cell inward:
  // the left lead cell 0 and coupling (0,1), the right lead cell N-1 and coupling (N-2,N-1).  M and
  // B^<> stay block-tridiagonal over the whole chain.  For a bulk lead cell k (virtual index 1,
  // neighbours 0 and 2; "away" is 0 on the left, 2 on the right), with m = M_kk, n = M_{k,away},
  // n' = M_{away,k}, b = B_kk and c = B_{away,k}:
  //   x = (m - n x n')^{-1} (decimation),  y = n x c,  a = x n,  q = x (b - y + y^H) x^H,
  //   w = q + a w a^H (Stein equation, doubling),  B^R_OBC = n x n',  B^<>_OBC = n w n^H - (y - y^H)
  // (the fixed point of the forward recursion of Eq. 9-10 run along the lead).  The edge cells'
  // own blocks of M and B^<> also take the products with the first lead cell, and the edge
  // blocks of W^R the term X^R_{0,-1} V_{-1,0} with X^R_{0,-1} = -X^R_00 M_{0,-1} x (mirrored on
  // the right).
  struct Rep { int d, u; };
  const Rep rep[2] = {{0, 0}, {N - 1, N - 2}};
  auto LV = [&](const Rep& r, int i, int j) {
    return i == j ? Vb(r.d, r.d) : (j == i + 1 ? Vb(r.u, r.u + 1) : Vb(r.u + 1, r.u));
  };
  auto LP = [&](const PT& p, const Rep& r, int i, int j) {
    return i == j ? Pb(p, r.d, r.d) : (j == i + 1 ? Pb(p, r.u, r.u + 1) : Pb(p, r.u + 1, r.u));
  };
  auto lead = [&](zd* base, int side) { return base + (long long)side * Ec * B2; };
  zd** wl = c->wl;
  zd* const nx = wl[5];  // n x per lead, kept for the W^R edge terms
  if (wobc) {
    for (int side = 0; side < 2; ++side) {
      const Rep& r = rep[side];
      const int away = side == 0 ? 0 : 2;
      zd* m = lead(c->lead_m, side);
      for (int a = 0; a < 3; ++a) BT_TRY(prod(c, Ec, -1.0, LV(r, 1, a), LP(pr, r, a, 1), a ? 1.0 : 0.0, m, B2));
      BT_TRY(bt::shift_diag(st, bs, Ec, m, B2, 1.0));
      bool first = true;
      for (int a = 0; a < 3; ++a)
        if (std::abs(a - away) <= 1) {
          BT_TRY(prod(c, Ec, -1.0, LV(r, 1, a), LP(pr, r, a, away), first ? 0.0 : 1.0, lead(c->lead_n, side), B2));
          first = false;
        }
      first = true;
      for (int a = 0; a < 3; ++a)
        if (std::abs(away - a) <= 1) {
          BT_TRY(prod(c, Ec, -1.0, LV(r, away, a), LP(pr, r, a, 1), first ? 0.0 : 1.0, lead(c->lead_np, side), B2));
          first = false;
        }
    }
    BT_TRY(decimate_leads(c, Ec, nullptr));
    BT_TRY(bt::merge_status(st, Ec, c->lead_info, 2, Ec, status));
    for (int side = 0; side < 2; ++side) {
      BT_TRY(prod(c, Ec, 1.0, W(lead(c->lead_n, side), B2), W(lead(c->lead_x, side), B2), 0.0, lead(nx, side), B2));
      BT_TRY(prod(c, Ec, 1.0, W(lead(c->lead_x, side), B2), W(lead(c->lead_n, side), B2), 0.0, lead(wl[6], side), B2));
    }
    const double U = 8.0 * bs * (double)bs * bs;
    for (int w = 0; w < 2; ++w) {
      if (!need[w]) continue;
      const PT& p = plg[w];
      zd* obc = w == 0 ? c->obcL : c->obcG;
      for (int side = 0; side < 2; ++side) {
        const Rep& r = rep[side];
        zd *T0 = lead(wl[0], side), *T1 = lead(wl[1], side), *T2 = lead(wl[2], side);
        zd *b = lead(wl[3], side), *cc = lead(wl[4], side);
        // T_{k,k-1}, T_kk, T_{k,k+1} of T = V P^<> in the lead
        BT_TRY(prod(c, Ec, 1.0, LV(r, 1, 0), LP(p, r, 0, 0), 0.0, T0, B2));
        BT_TRY(prod(c, Ec, 1.0, LV(r, 1, 1), LP(p, r, 1, 0), 1.0, T0, B2));
        for (int a = 0; a < 3; ++a) BT_TRY(prod(c, Ec, 1.0, LV(r, 1, a), LP(p, r, a, 1), a ? 1.0 : 0.0, T1, B2));
        BT_TRY(prod(c, Ec, 1.0, LV(r, 1, 1), LP(p, r, 1, 2), 0.0, T2, B2));
        BT_TRY(prod(c, Ec, 1.0, LV(r, 1, 2), LP(p, r, 2, 2), 1.0, T2, B2));
        // b = B_kk = sum_c T_{k,c} (V_{k,c})^H; c = B_{away,k} (periodic lead: T_{k-1,.} = T_{k,.+1})
        BT_TRY(prod(c, Ec, 1.0, W(T0, B2), flip(LV(r, 1, 0)), 0.0, b, B2));
        BT_TRY(prod(c, Ec, 1.0, W(T1, B2), flip(LV(r, 1, 1)), 1.0, b, B2));
        BT_TRY(prod(c, Ec, 1.0, W(T2, B2), flip(LV(r, 1, 2)), 1.0, b, B2));
        if (c->d.symmetrize) BT_TRY(bt::antiherm_project(st, bs, Ec, b, B2));
        if (side == 0) {
          BT_TRY(prod(c, Ec, 1.0, W(T1, B2), flip(LV(r, 1, 0)), 0.0, cc, B2));
          BT_TRY(prod(c, Ec, 1.0, W(T2, B2), flip(LV(r, 1, 1)), 1.0, cc, B2));
        } else {
          BT_TRY(prod(c, Ec, 1.0, W(T0, B2), flip(LV(r, 1, 1)), 0.0, cc, B2));
          BT_TRY(prod(c, Ec, 1.0, W(T1, B2), flip(LV(r, 1, 2)), 1.0, cc, B2));
        }
        // y = n x c;  b - (y - y^H);  q = x (b - y + y^H) x^H
        zd *y = lead(wl[7], side), *tq = lead(wl[8], side), *q = lead(wl[9], side);
        BT_TRY(prod(c, Ec, 1.0, W(lead(nx, side), B2), W(cc, B2), 0.0, y, B2));
        BT_TRY(bt::add_antiherm(st, bs, Ec, b, B2, y, B2, -1.0));
        BT_TRY(prod(c, Ec, 1.0, W(lead(c->lead_x, side), B2), W(b, B2), 0.0, tq, B2));
        BT_TRY(prod(c, Ec, 1.0, W(tq, B2), flip(W(lead(c->lead_x, side), B2)), 0.0, q, B2, true));
      }
      // w = q + a w a^H for all 2 Ec leads (a is consumed: copied first)
      BT_CUDA_TRY(cudaMemcpyAsync(wl[10], wl[6], sizeof(zd) * 2 * Ec * B2, cudaMemcpyDeviceToDevice, st));
      long long its = 0, body = 0;
      BT_TRY(bt::stein(st, bs, 2 * Ec, wl[10], nullptr, wl[9], 1e-14, 64, nullptr, c->w_ok, nullptr, c->dec_ws,
                       c->dec_bytes, c->h_pinned, &its, &c->eng_kept, c->loop, &body));
      c->cap_polish_body += body;
      c->flops += 3.0 * U * (double)its;
      BT_TRY(bt::status_from_ok(st, 2 * Ec, c->w_ok, nullptr, BT_ERR_NOT_CONVERGED, c->w_info));
      BT_TRY(bt::merge_status(st, Ec, c->w_info, 2, Ec, status));
      // B^<>_OBC = n w n^H - (y - y^H)
      for (int side = 0; side < 2; ++side) {
        zd* o = lead(obc, side);
        BT_TRY(prod(c, Ec, 1.0, W(lead(c->lead_n, side), B2), W(lead(wl[9], side), B2), 0.0, lead(wl[8], side), B2));
        BT_TRY(prod(c, Ec, 1.0, W(lead(wl[8], side), B2), flip(W(lead(c->lead_n, side), B2)), 0.0, o, B2, true));
        BT_TRY(bt::add_antiherm(st, bs, Ec, o, B2, lead(wl[7], side), B2, -1.0));
      }
    }
    // edge cells of M~: the products with the first lead cell, then - B^R_OBC
    BT_TRY(prod(c, Ec, -1.0, Vb(1, 0), Pb(pr, 0, 1), 1.0, c->Md, NB2));
    BT_TRY(prod(c, Ec, -1.0, Vb(N - 2, N - 1), Pb(pr, N - 1, N - 2), 1.0, c->Md + (N - 1) * B2, NB2));
    BT_TRY(bt::axpby(st, B2, Ec, -1.0, lead(c->lead_sig, 0), B2, 1.0, c->Md, NB2));
    BT_TRY(bt::axpby(st, B2, Ec, -1.0, lead(c->lead_sig, 1), B2, 1.0, c->Md + (N - 1) * B2, NB2));
  }

  // ---- a1 (W): B^<> = (V P^<>) V^H, diagonal and upper blocks ----
  for (int w = 0; w < 2; ++w) {
    if (!need[w]) continue;
    const PT& p = plg[w];
    for (int i = 0; i < N; ++i) {  // T = V P^<>
      zd* td = c->Td + i * B2;
      BT_TRY(prod(c, Ec, 1.0, Vb(i, i), Pb(p, i, i), 0.0, td, NB2));
      if (i > 0) BT_TRY(prod(c, Ec, 1.0, Vb(i, i - 1), Pb(p, i - 1, i), 1.0, td, NB2));
      if (i + 1 < N) BT_TRY(prod(c, Ec, 1.0, Vb(i, i + 1), Pb(p, i + 1, i), 1.0, td, NB2));
      if (i + 1 < N) {
        zd* tu = c->Tu + i * B2;
        zd* tl = c->Tl + i * B2;
        BT_TRY(prod(c, Ec, 1.0, Vb(i, i), Pb(p, i, i + 1), 0.0, tu, N1B2));
        BT_TRY(prod(c, Ec, 1.0, Vb(i, i + 1), Pb(p, i + 1, i + 1), 1.0, tu, N1B2));
        BT_TRY(prod(c, Ec, 1.0, Vb(i + 1, i), Pb(p, i, i), 0.0, tl, N1B2));
        BT_TRY(prod(c, Ec, 1.0, Vb(i + 1, i + 1), Pb(p, i + 1, i), 1.0, tl, N1B2));
      }
    }
    if (wobc) {
      // T_00 += V_{0,-1} P_{-1,0}, T_{N-1,N-1} += V_{N-1,N} P_{N,N-1};
      // T_{0,-1} = V_{0,-1} P_{-1,-1} + V_00 P_{0,-1},  T_{N-1,N} = V_{N-1,N} P_{N,N} + V_{N-1,N-1} P_{N-1,N}
      BT_TRY(prod(c, Ec, 1.0, Vb(1, 0), Pb(p, 0, 1), 1.0, c->Td, NB2));
      BT_TRY(prod(c, Ec, 1.0, Vb(N - 2, N - 1), Pb(p, N - 1, N - 2), 1.0, c->Td + (N - 1) * B2, NB2));
      BT_TRY(prod(c, Ec, 1.0, Vb(1, 0), Pb(p, 0, 0), 0.0, c->t[0], B2));
      BT_TRY(prod(c, Ec, 1.0, Vb(0, 0), Pb(p, 1, 0), 1.0, c->t[0], B2));
      BT_TRY(prod(c, Ec, 1.0, Vb(N - 2, N - 1), Pb(p, N - 1, N - 1), 0.0, c->t[1], B2));
      BT_TRY(prod(c, Ec, 1.0, Vb(N - 1, N - 1), Pb(p, N - 2, N - 1), 1.0, c->t[1], B2));
    }
    for (int i = 0; i < N; ++i) {  // B = T V^H
      zd* bd = Bd[w] + i * B2;
      BT_TRY(prod(c, Ec, 1.0, W(c->Td + i * B2, NB2), Vh(i, i), 0.0, bd, NB2));
      if (i > 0) BT_TRY(prod(c, Ec, 1.0, W(c->Tl + (i - 1) * B2, N1B2), Vh(i, i - 1), 1.0, bd, NB2));
      if (i + 1 < N) BT_TRY(prod(c, Ec, 1.0, W(c->Tu + i * B2, N1B2), Vh(i, i + 1), 1.0, bd, NB2));
      if (wobc && (i == 0 || i == N - 1)) {
        // T_{0,-1} (V_{0,-1})^H or T_{N-1,N} (V_{N-1,N})^H, and the boundary block B^<>_OBC
        const zd* obc = w == 0 ? c->obcL : c->obcG;
        for (int side = 0; side < 2; ++side) {
          if ((side == 0 && i != 0) || (side == 1 && i != N - 1)) continue;
          BT_TRY(prod(c, Ec, 1.0, W(c->t[side], B2), side == 0 ? Vh(1, 0) : Vh(N - 2, N - 1), 1.0, bd, NB2));
          BT_TRY(bt::axpby(st, B2, Ec, 1.0, lead(const_cast<zd*>(obc), side), B2, 1.0, bd, NB2));
        }
      }
      // B^<>_ii is anti-Hermitian as a sum of three products: made exactly so (Sec. 5.2) before the
      // sweep's anti-Hermitian products take it as an operand
      if (c->d.symmetrize) BT_TRY(bt::antiherm_project(c->st, bs, Ec, bd, NB2));
      if (i + 1 < N) {
        zd* bu = Bu[w] + i * B2;
        BT_TRY(prod(c, Ec, 1.0, W(c->Td + i * B2, NB2), Vh(i + 1, i), 0.0, bu, N1B2));
        BT_TRY(prod(c, Ec, 1.0, W(c->Tu + i * B2, N1B2), Vh(i + 1, i + 1), 1.0, bu, N1B2));
      }
    }
  }
  // ---- a3 + a4 ----
  Sweep sw;
  sw.c = c;
  sw.Ec = Ec;
  sw.N = N;
  sw.bs = bs;
  sw.B2 = B2;
  sw.needL = needL;
  sw.needG = needG;
  sw.needRlower = true;
  sw.keepRoff = true;
  sw.has_boff = N > 1;
  sw.oLu = oL && oL->upper ? static_cast<zd*>(oL->upper) + e0 * N1B2 : nullptr;
  sw.oGu = oG && oG->upper ? static_cast<zd*>(oG->upper) + e0 * N1B2 : nullptr;
  sw.oes_u = N1B2;
  sw.X2u = N > 2 ? c->X2u : nullptr;
  sw.X2l = N > 2 ? c->X2l : nullptr;
  sw.asmM = [&](int i, zd* dst, long long es) {
    return bt::write_blocks(st, bs, 1, Ec, c->Md + i * B2, 0, NB2, dst, 0, es, 0);
  };
  sw.asmB = [&](int i, int w, zd* dst, long long es) {
    return bt::write_blocks(st, bs, 1, Ec, Bd[w] + i * B2, 0, NB2, dst, 0, es, 0);
  };
  sw.Mu = [&](int i) { return ws_blk(c->Mu + i * B2, N1B2); };
  sw.Ml = [&](int i) { return ws_blk(c->Ml + i * B2, N1B2); };
  sw.Bu = [&](int i, int w) { return ws_blk(Bu[w] + i * B2, N1B2); };
  BT_TRY(run_sweep(sw, status));

  // ---- W^R = X^R V on the selected blocks ----
  if (oR && (oR->diag || oR->upper || oR->lower)) {
    auto XRd = [&](int i) { return W(c->xR + i * B2, NB2); };
    auto XRu = [&](int i) { return W(c->XRu + i * B2, N1B2); };
    auto XRl = [&](int i) { return W(c->XRl + i * B2, N1B2); };
    auto X2u = [&](int i) { return W(c->X2u + i * B2, N2B2); };
    auto X2l = [&](int i) { return W(c->X2l + i * B2, N2B2); };
    const bool rvec = oR->layout == BT_LAYOUT_DIAGVEC;
    // contacts: Q_L = n_L x_L V_{-1,0}, Q_R = n_R x_R V_{N,N-1}; W^R_{i,0} -= X^R_{i,0} Q_L and
    // W^R_{i,N-1} -= X^R_{i,N-1} Q_R for the selected blocks i (the lead cell's column of X^R V)
    zd* Q[2] = {lead(wl[10], 0), lead(wl[10], 1)};
    if (wobc) {
      BT_TRY(prod(c, Ec, 1.0, W(lead(nx, 0), B2), Vb(0, 1), 0.0, Q[0], B2));
      BT_TRY(prod(c, Ec, 1.0, W(lead(nx, 1), B2), Vb(N - 1, N - 2), 0.0, Q[1], B2));
    }
    for (int i = 0; i < N; ++i) {
      if (oR->diag) {
        // diagonal-vector output: form the block in a temporary, keep its diagonal
        zd* o = rvec ? c->t[0] : static_cast<zd*>(oR->diag) + (e0 * N + i) * B2;
        const long long es = rvec ? B2 : NB2;
        BT_TRY(prod(c, Ec, 1.0, XRd(i), Vb(i, i), 0.0, o, es));
        if (i > 0) BT_TRY(prod(c, Ec, 1.0, XRl(i - 1), Vb(i - 1, i), 1.0, o, es));
        if (i + 1 < N) BT_TRY(prod(c, Ec, 1.0, XRu(i), Vb(i + 1, i), 1.0, o, es));
        if (wobc && i == 0) BT_TRY(prod(c, Ec, -1.0, XRd(0), W(Q[0], B2), 1.0, o, es));
        if (wobc && i == N - 1) BT_TRY(prod(c, Ec, -1.0, XRd(N - 1), W(Q[1], B2), 1.0, o, es));
        if (rvec)
          BT_TRY(bt::write_diagvec(st, bs, 1, Ec, o, 0, B2, static_cast<zd*>(oR->diag) + (e0 * N + i) * bs, 0,
                                   (long long)N * bs, 0));
      }
      if (i + 1 < N && oR->upper) {
        zd* o = static_cast<zd*>(oR->upper) + (e0 * (N - 1) + i) * B2;
        BT_TRY(prod(c, Ec, 1.0, XRd(i), Vb(i, i + 1), 0.0, o, N1B2));
        BT_TRY(prod(c, Ec, 1.0, XRu(i), Vb(i + 1, i + 1), 1.0, o, N1B2));
        if (i + 2 < N) BT_TRY(prod(c, Ec, 1.0, X2u(i), Vb(i + 2, i + 1), 1.0, o, N1B2));
        if (wobc && i == N - 2) BT_TRY(prod(c, Ec, -1.0, XRu(N - 2), W(Q[1], B2), 1.0, o, N1B2));
      }
      if (i + 1 < N && oR->lower) {
        zd* o = static_cast<zd*>(oR->lower) + (e0 * (N - 1) + i) * B2;
        BT_TRY(prod(c, Ec, 1.0, XRl(i), Vb(i, i), 0.0, o, N1B2));
        BT_TRY(prod(c, Ec, 1.0, XRd(i + 1), Vb(i + 1, i), 1.0, o, N1B2));
        if (i > 0) BT_TRY(prod(c, Ec, 1.0, X2l(i - 1), Vb(i - 1, i), 1.0, o, N1B2));
        if (wobc && i == 0) BT_TRY(prod(c, Ec, -1.0, XRl(0), W(Q[0], B2), 1.0, o, N1B2));
      }
    }
  }
  // ---- a5 ----
  BT_TRY(write_diag_out(c, Ec, c->xL, oL, e0, d.symmetrize ? 1 : 0));
  BT_TRY(write_diag_out(c, Ec, c->xG, oG, e0, d.symmetrize ? 1 : 0));
  return BT_OK;
}

bt_status check_solve_args(bt_ctx* c, const bt_bt* H, const bt_bt* S, const bt_bt* sR, const bt_bt* sL, const bt_bt* sG,
                           const double* E, int n, const bt_bt_out* oR, const bt_bt_out* oL, const bt_bt_out* oG,
                           const int* status) {
  std::string why;
  auto fail = [&](const std::string& m) { c->err = m; return BT_ERR_INVALID_ARG; };
  if (n < 0) return fail("n_energies < 0");
  if (n > 0 && !E) return fail("energies_host is NULL");
  if (n > 0 && !status) return fail("status array is NULL");
  bt_status s;
  if ((s = validate_operand(H, true, false, c->d.system == BT_SYS_G ? "H" : "V", &why)) != BT_OK) return fail(why);
  if (c->d.nb > 1 && !H->upper) return fail("H/V upper blocks are required for nb > 1");
  if (c->d.system == BT_SYS_G) {
    if ((s = validate_operand(S, false, false, "S", &why)) != BT_OK) return fail(why);
    if ((s = validate_operand(sR, false, true, "sigR", &why)) != BT_OK) return fail(why);
    if ((s = validate_operand(sL, false, true, "sigL", &why, true)) != BT_OK) return fail(why);
    if ((s = validate_operand(sG, false, true, "sigG", &why, true)) != BT_OK) return fail(why);
    if (sL && sL->upper && sL->symmetry != BT_SYM_ANTIHERMITIAN) return fail("sigL off-diagonal blocks must be anti-Hermitian");
    if (sG && sG->upper && sG->symmetry != BT_SYM_ANTIHERMITIAN) return fail("sigG off-diagonal blocks must be anti-Hermitian");
  } else {
    if (S) return fail("S must be NULL for the W system");
    if (H->per_energy) return fail("V must be shared across energies");
    if (H->symmetry != BT_SYM_HERMITIAN) return fail("V must be Hermitian");
    if ((s = validate_operand(sR, true, false, "P^R", &why)) != BT_OK) return fail(why);
    if (c->d.nb > 1 && (!sR->upper || (sR->symmetry == BT_SYM_GENERAL && !sR->lower))) return fail("P^R off-diagonal blocks are required");
    if ((s = validate_operand(sL, false, false, "P^<", &why, true)) != BT_OK) return fail(why);
    if ((s = validate_operand(sG, false, false, "P^>", &why, true)) != BT_OK) return fail(why);
    if ((oL && (oL->diag || oL->upper) && !sL) || (oG && (oG->diag || oG->upper) && !sG))
      return fail("W^<> outputs need P^<>");
    if (c->d.nb > 1 && ((sL && (!sL->upper || sL->symmetry != BT_SYM_ANTIHERMITIAN)) ||
                        (sG && (!sG->upper || sG->symmetry != BT_SYM_ANTIHERMITIAN))))
      return fail("P^<> need anti-Hermitian off-diagonal blocks");
  }
  const bt_bt_out* outs[3] = {oR, oL, oG};
  for (int k = 0; k < 3; ++k) {
    const bt_bt_out* o = outs[k];
    if (!o) continue;
    if (o->layout != BT_LAYOUT_BLOCKS && o->layout != BT_LAYOUT_DIAGVEC && o->layout != BT_LAYOUT_PACKED_UPPER)
      return fail("bad output layout");
    if (o->layout == BT_LAYOUT_DIAGVEC && (o->upper || o->lower))
      return fail("diagonal-vector outputs have no off-diagonal blocks");
    if (o->layout == BT_LAYOUT_PACKED_UPPER && (k == 0 || !c->d.symmetrize || o->lower))
      return fail("packed upper-triangle storage is for symmetrised lesser/greater diagonal blocks (lower = NULL)");
  }
  (void)s;
  return BT_OK;
}

}  // namespace

namespace {

// Key of a captured chunk: every pointer and layout field the captured launches depend on (the
// energies themselves are uploaded outside the graph).
std::vector<char> chunk_key(long long e0, int Ec, const bt_bt* const* ins, int n_in, const bt_bt_out* const* outs,
                            int n_out, const int* status) {
  std::vector<char> k;
  auto put = [&](const void* p, size_t n) {
    const char* b = static_cast<const char*>(p);
    k.insert(k.end(), b, b + n);
  };
  put(&e0, sizeof(e0));
  put(&Ec, sizeof(Ec));
  for (int i = 0; i < n_in; ++i) {
    const char present = ins[i] != nullptr;
    put(&present, 1);
    if (present) {
      put(&ins[i]->diag, sizeof(void*));
      put(&ins[i]->upper, sizeof(void*));
      put(&ins[i]->lower, sizeof(void*));
      put(&ins[i]->layout, sizeof(int));
      put(&ins[i]->symmetry, sizeof(int));
      put(&ins[i]->per_energy, sizeof(int));
    }
  }
  for (int i = 0; i < n_out; ++i) {
    const char present = outs[i] != nullptr;
    put(&present, 1);
    if (present) {
      put(&outs[i]->diag, sizeof(void*));
      put(&outs[i]->upper, sizeof(void*));
      put(&outs[i]->lower, sizeof(void*));
      put(&outs[i]->layout, sizeof(int));
    }
  }
  put(&status, sizeof(status));
  return k;
}

constexpr size_t kMaxCaptured = 8;

// Graph mode: replays the chunk's captured graph, capturing it first when this combination of
// operands has not been seen (kMaxCaptured most recent kept).  The decimation loop is a
// conditional while node, so a replay needs no host round trip.
template <class Direct>
bt_status run_chunk_graph(bt_ctx* c, const bt_bt* H, const bt_bt* S, const bt_bt* sR, const bt_bt* sL,
                          const bt_bt* sG, long long e0, int Ec, const bt_bt_out* oR, const bt_bt_out* oL,
                          const bt_bt_out* oG, int* status, Direct direct) {
  const bt_bt* ins[5] = {H, S, sR, sL, sG};
  const bt_bt_out* outs[3] = {oR, oL, oG};
  std::vector<char> key = chunk_key(e0, Ec, ins, 5, outs, 3, status);
  size_t idx = c->graphs.size();
  for (size_t i = 0; i < c->graphs.size(); ++i)
    if (c->graphs[i].key == key) { idx = i; break; }
  if (idx == c->graphs.size()) {
    bt_ctx::Captured g;
    g.key = std::move(key);
    bt::LoopCapture loop;
    loop.body_stream = c->body_st;
    const double f0 = c->flops;
    const long long l0 = bt::launches_total();
    if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return set_err(c, BT_ERR_CUDA, "stream capture could not start");
    c->loop = c->d.obc ? &loop : nullptr;
    bt_status s = direct();
    c->loop = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->st, &g.graph);
    const long long recorded = bt::launches_total() - l0;
    c->uncounted += recorded;
    if (s != BT_OK || ce != cudaSuccess) {
      if (g.graph) cudaGraphDestroy(g.graph);
      cudaGetLastError();
      return s != BT_OK ? s : set_err(c, BT_ERR_CUDA, "stream capture failed");
    }
    if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g.graph);
      return set_err(c, BT_ERR_CUDA, "graph instantiation failed");
    }
    g.flops = c->flops - f0;
    c->flops = f0;  // counted again below, as for every replay
    g.body_launches = loop.body_launches;
    g.polish_body = c->cap_polish_body;
    g.launches = recorded - loop.body_launches - c->cap_polish_body;
    c->cap_polish_body = 0;
    g.decim = c->d.obc != 0;
    if (c->graphs.size() >= kMaxCaptured) {
      cudaGraphExecDestroy(c->graphs.front().exec);
      cudaGraphDestroy(c->graphs.front().graph);
      c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back(std::move(g));
    idx = c->graphs.size() - 1;
  } else if (idx + 1 != c->graphs.size()) {
    std::rotate(c->graphs.begin() + idx, c->graphs.begin() + idx + 1, c->graphs.end());
    idx = c->graphs.size() - 1;
  }
  const bt_ctx::Captured& g = c->graphs[idx];
  if (cudaGraphLaunch(g.exec, c->st) != cudaSuccess) return set_err(c, BT_ERR_CUDA, "graph launch failed");
  c->flops += g.flops;
  c->stats.kernel_launches += g.launches;
  if (g.decim) {
    if (cudaMemcpyAsync(c->h_iters, c->lead_iters, sizeof(int) * 2 * Ec, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
      return set_err(c, BT_ERR_CUDA, "iteration read-back failed");
    if (c->d.decim_newton_after >= 0) {
      if (cudaMemcpyAsync(c->h_iters + 2 * Ec, c->lead_piters, sizeof(int) * 2 * Ec, cudaMemcpyDeviceToHost,
                          c->st) != cudaSuccess)
        return set_err(c, BT_ERR_CUDA, "iteration read-back failed");
    } else {
      std::memset(c->h_iters + 2 * Ec, 0, sizeof(int) * 2 * Ec);
    }
    c->pending = true;
    c->pending_Ec = Ec;
    c->pending_body = g.body_launches;
    c->pending_polish_body = g.polish_body;
  }
  return BT_OK;
}

// Graph mode: copies energies [e0, e0 + Ec) of every per-energy input to the context's staging
// memory (device to device, stream-ordered before the replay) and points ins[k] at the copies, so
// that the captured graph reads fixed addresses whichever energies the call passes.
bt_status stage_inputs(bt_ctx* c, const bt_bt** ins, bt_bt* staged, long long e0, int Ec) {
  const int N = c->d.nb, bs = c->d.bs, Emax = c->d.max_energies;
  const long long oext = off_extent(N, bs);
  size_t need = 0;
  for (int k = 0; k < 5; ++k) {
    const bt_bt* b = ins[k];
    if (!b || !b->per_energy) continue;
    if (b->diag) need += al(sizeof(zd) * diag_extent(*b, N, bs) * Emax);
    if (b->upper) need += al(sizeof(zd) * oext * Emax);
    if (b->lower) need += al(sizeof(zd) * oext * Emax);
  }
  if (need == 0) return BT_OK;
  if (c->gstage_bytes < need) {
    // the stream is idle here (the caller synchronised it before staging the chunk's energies);
    // graphs captured on the old staging memory read it: they go with it
    for (auto& g : c->graphs) {
      cudaGraphExecDestroy(g.exec);
      cudaGraphDestroy(g.graph);
    }
    c->graphs.clear();
    if (c->gstage) cudaFree(c->gstage);
    c->gstage = nullptr;
    c->gstage_bytes = 0;
    if (cudaMalloc(&c->gstage, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, BT_ERR_OOM, "graph-mode input staging allocation failed");
    }
    c->gstage_bytes = need;
  }
  Carver cv(c->gstage);
  auto copy = [&](const void* src, long long ext, const void** dst) -> bool {
    zd* d = cv.take<zd>((size_t)(ext * Emax));
    *dst = d;
    return cudaMemcpyAsync(d, static_cast<const zd*>(src) + ext * e0, sizeof(zd) * ext * Ec, cudaMemcpyDeviceToDevice,
                           c->st) == cudaSuccess;
  };
  for (int k = 0; k < 5; ++k) {
    const bt_bt* b = ins[k];
    if (!b || !b->per_energy) continue;
    staged[k] = *b;
    if (b->diag && !copy(b->diag, diag_extent(*b, N, bs), &staged[k].diag)) return set_err(c, BT_ERR_CUDA, "input staging failed");
    if (b->upper && !copy(b->upper, oext, &staged[k].upper)) return set_err(c, BT_ERR_CUDA, "input staging failed");
    if (b->lower && !copy(b->lower, oext, &staged[k].lower)) return set_err(c, BT_ERR_CUDA, "input staging failed");
    ins[k] = &staged[k];
  }
  return BT_OK;
}

}  // namespace

extern "C" bt_status bt_selinv_solve(bt_ctx* c, const bt_bt* H, const bt_bt* S, const bt_bt* sigR, const bt_bt* sigL,
                                     const bt_bt* sigG, const double* energies_host, int n_energies,
                                     const bt_bt_out* outR, const bt_bt_out* outL, const bt_bt_out* outG,
                                     int* status_device) {
  if (!c) return BT_ERR_INVALID_ARG;
  c->err.clear();
  BT_TRY(check_solve_args(c, H, S, sigR, sigL, sigG, energies_host, n_energies, outR, outL, outG, status_device));
  if (n_energies == 0) return BT_OK;
  if (c->pending) {  // the previous solve's last replayed chunk: complete its statistics first
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return set_err(c, BT_ERR_CUDA, "stream error");
    fold_pending(c);
  }
  c->flops = 0.0;
  const long long launches0 = bt::launches_total();
  c->uncounted = 0;
  struct LaunchTally {  // attributes this call's launches to the context on every return path
    bt_ctx* c;
    long long l0;
    ~LaunchTally() { c->stats.kernel_launches += bt::launches_total() - l0 - c->uncounted; }
  } tally{c, launches0};
  if (cudaMemsetAsync(status_device, 0, sizeof(int) * (size_t)n_energies, c->st) != cudaSuccess)
    return set_err(c, BT_ERR_CUDA, "cudaMemsetAsync(status) failed");
  const int Emax = c->d.max_energies;
  for (long long e0 = 0; e0 < n_energies; e0 += Emax) {
    const int Ec = (int)std::min<long long>(Emax, n_energies - e0);
    // stage this chunk's energies (the previous chunk's copy may still be in flight)
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return set_err(c, BT_ERR_CUDA, "stream error");
    std::memcpy(c->h_E, energies_host + e0, sizeof(double) * Ec);
    if (cudaMemcpyAsync(c->Edev, c->h_E, sizeof(double) * Ec, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return set_err(c, BT_ERR_CUDA, "energy upload failed");
    fold_pending(c);  // the stream is idle here
    const bt_bt* in[5] = {H, S, sigR, sigL, sigG};
    bt_bt staged[5];
    long long ein = e0;
    if (c->d.graph) {
      BT_TRY(stage_inputs(c, in, staged, e0, Ec));
      ein = 0;
    }
    bt_status s;
    auto direct = [&]() {
      // a bounded wait of a sliced product that expires marks every energy of the chunk
      if (cudaMemsetAsync(c->tflag, 0, sizeof(int), c->st) != cudaSuccess) return BT_ERR_CUDA;
      const bt_status r = c->d.system == BT_SYS_G
                              ? solve_chunk_g(c, in[0], in[1], in[2], in[3], in[4], e0, ein, Ec, outR, outL, outG,
                                              status_device + e0)
                              : solve_chunk_w(c, in[0], in[2], in[3], in[4], e0, ein, Ec, outR, outL, outG,
                                              status_device + e0);
      if (r != BT_OK) return r;
      return bt::flag_status(c->st, Ec, c->tflag, status_device + e0);
    };
    if (c->d.graph)
      s = run_chunk_graph(c, in[0], in[1], in[2], in[3], in[4], e0, Ec, outR, outL, outG, status_device + e0, direct);
    else
      s = direct();
    if (s != BT_OK) {
      if (c->err.empty()) c->err = "a kernel launch failed";
      return s;
    }
  }
  c->stats.solves += 1;
  c->stats.energies += n_energies;
  c->stats.flops_model = c->flops;
  return BT_OK;
}

// ======================================================================================
// Host-buffer entry point: stages inputs chunk by chunk, runs the device path, copies back.
// ======================================================================================
namespace {

long long diag_out_extent(const bt_bt_out* o, int nb, int bs) {
  if (o->layout == BT_LAYOUT_DIAGVEC) return (long long)nb * bs;
  if (o->layout == BT_LAYOUT_PACKED_UPPER) return (long long)nb * bs * (bs + 1) / 2;
  return (long long)nb * bs * bs;
}

struct StagedOperand {
  bt_bt dev{};
  const bt_bt* host = nullptr;
  long long dext = 0, oext = 0;  // per-energy element extents (or whole operand when shared)
  zd *d = nullptr, *u = nullptr, *l = nullptr;
};

}  // namespace

extern "C" bt_status bt_selinv_solve_host(bt_ctx* c, const bt_bt* H, const bt_bt* S, const bt_bt* sigR,
                                          const bt_bt* sigL, const bt_bt* sigG, const double* energies_host,
                                          int n_energies, const bt_bt_out* outR, const bt_bt_out* outL,
                                          const bt_bt_out* outG, int* status_host) {
  if (!c) return BT_ERR_INVALID_ARG;
  c->err.clear();
  BT_TRY(check_solve_args(c, H, S, sigR, sigL, sigG, energies_host, n_energies, outR, outL, outG, status_host));
  if (n_energies == 0) return BT_OK;
  const int N = c->d.nb, bs = c->d.bs, Emax = c->d.max_energies;
  const long long B2 = (long long)bs * bs, N1B2 = (long long)(N > 1 ? N - 1 : 0) * B2;
  const bt_bt* ins[5] = {H, S, sigR, sigL, sigG};
  StagedOperand so[5];
  const bt_bt_out* outs[3] = {outR, outL, outG};
  // Output staging is double-buffered when there is more than one chunk: the copies of chunk k
  // back to the host run on a second stream while chunk k + 1 computes.
  const int n_chunks = (int)((n_energies + Emax - 1) / Emax);
  const int nbuf = n_chunks > 1 ? 2 : 1;
  // bytes: shared operands whole, per-energy operands for one chunk, outputs for nbuf chunks
  size_t need = 0;
  auto elems_d = [&](const bt_bt* b) { return diag_extent(*b, N, bs); };
  for (int k = 0; k < 5; ++k) {
    if (!ins[k]) continue;
    so[k].host = ins[k];
    so[k].dext = elems_d(ins[k]);
    so[k].oext = N1B2;
    const long long mult = ins[k]->per_energy ? Emax : 1;
    if (ins[k]->diag) need += al(sizeof(zd) * so[k].dext * mult);
    if (ins[k]->upper) need += al(sizeof(zd) * so[k].oext * mult);
    if (ins[k]->lower) need += al(sizeof(zd) * so[k].oext * mult);
  }
  for (int q = 0; q < nbuf; ++q) {
    for (int k = 0; k < 3; ++k) {
      if (!outs[k]) continue;
      if (outs[k]->diag) need += al(sizeof(zd) * diag_out_extent(outs[k], N, bs) * Emax);
      if (outs[k]->upper) need += al(sizeof(zd) * N1B2 * Emax);
      if (outs[k]->lower) need += al(sizeof(zd) * N1B2 * Emax);
    }
    need += al(sizeof(int) * Emax);
  }
  if (c->stage_bytes < need) {
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    if (cudaMalloc(&c->stage, need) != cudaSuccess) { cudaGetLastError(); return set_err(c, BT_ERR_OOM, "staging allocation failed"); }
    c->stage_bytes = need;
  }
  if (nbuf > 1 && !c->copy_st) {
    if (cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, BT_ERR_CUDA, "copy stream set-up failed");
    }
  }
  Carver cv(c->stage);
  for (int k = 0; k < 5; ++k) {
    if (!ins[k]) continue;
    const long long mult = ins[k]->per_energy ? Emax : 1;
    so[k].dev = *ins[k];
    if (ins[k]->diag) { so[k].d = cv.take<zd>(so[k].dext * mult); so[k].dev.diag = so[k].d; }
    if (ins[k]->upper) { so[k].u = cv.take<zd>(so[k].oext * mult); so[k].dev.upper = so[k].u; }
    if (ins[k]->lower) { so[k].l = cv.take<zd>(so[k].oext * mult); so[k].dev.lower = so[k].l; }
  }
  bt_bt_out dout[2][3] = {};
  int* dstatus[2] = {nullptr, nullptr};
  for (int q = 0; q < nbuf; ++q) {
    for (int k = 0; k < 3; ++k) {
      if (!outs[k]) continue;
      dout[q][k].layout = outs[k]->layout;
      if (outs[k]->diag) dout[q][k].diag = cv.take<zd>(diag_out_extent(outs[k], N, bs) * Emax);
      if (outs[k]->upper) dout[q][k].upper = cv.take<zd>(N1B2 * Emax);
      if (outs[k]->lower) dout[q][k].lower = cv.take<zd>(N1B2 * Emax);
    }
    dstatus[q] = cv.take<int>(Emax);
  }
  cudaStream_t st = c->st;
  cudaStream_t cs = nbuf > 1 ? c->copy_st : st;  // stream of the copies back to the host
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  auto d2h = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
  };
  // shared operands once
  for (int k = 0; k < 5; ++k) {
    if (!ins[k] || ins[k]->per_energy) continue;
    if (so[k].d && !h2d(so[k].d, ins[k]->diag, sizeof(zd) * so[k].dext)) return set_err(c, BT_ERR_CUDA, "H2D failed");
    if (so[k].u && !h2d(so[k].u, ins[k]->upper, sizeof(zd) * so[k].oext)) return set_err(c, BT_ERR_CUDA, "H2D failed");
    if (so[k].l && !h2d(so[k].l, ins[k]->lower, sizeof(zd) * so[k].oext)) return set_err(c, BT_ERR_CUDA, "H2D failed");
  }
  int chunk = 0;
  for (long long e0 = 0; e0 < n_energies; e0 += Emax, ++chunk) {
    const int Ec = (int)std::min<long long>(Emax, n_energies - e0);
    const int q = chunk % nbuf;
    // the copies out of this output set (two chunks ago) must be done before it is overwritten
    if (nbuf > 1 && chunk >= 2 && cudaStreamWaitEvent(st, c->ev_done[q], 0) != cudaSuccess)
      return set_err(c, BT_ERR_CUDA, "stream wait failed");
    for (int k = 0; k < 5; ++k) {
      if (!ins[k] || !ins[k]->per_energy) continue;
      const zd* hd = static_cast<const zd*>(ins[k]->diag);
      const zd* hu = static_cast<const zd*>(ins[k]->upper);
      const zd* hl = static_cast<const zd*>(ins[k]->lower);
      if (so[k].d && !h2d(so[k].d, hd + so[k].dext * e0, sizeof(zd) * so[k].dext * Ec)) return set_err(c, BT_ERR_CUDA, "H2D failed");
      if (so[k].u && !h2d(so[k].u, hu + so[k].oext * e0, sizeof(zd) * so[k].oext * Ec)) return set_err(c, BT_ERR_CUDA, "H2D failed");
      if (so[k].l && !h2d(so[k].l, hl + so[k].oext * e0, sizeof(zd) * so[k].oext * Ec)) return set_err(c, BT_ERR_CUDA, "H2D failed");
    }
    bt_status s = bt_selinv_solve(c, H ? &so[0].dev : nullptr, S ? &so[1].dev : nullptr, sigR ? &so[2].dev : nullptr,
                                  sigL ? &so[3].dev : nullptr, sigG ? &so[4].dev : nullptr, energies_host + e0, Ec,
                                  outR ? &dout[q][0] : nullptr, outL ? &dout[q][1] : nullptr,
                                  outG ? &dout[q][2] : nullptr, dstatus[q]);
    if (s != BT_OK) return s;
    if (nbuf > 1) {
      if (cudaEventRecord(c->ev_ready, st) != cudaSuccess || cudaStreamWaitEvent(cs, c->ev_ready, 0) != cudaSuccess)
        return set_err(c, BT_ERR_CUDA, "event record failed");
    }
    for (int k = 0; k < 3; ++k) {
      if (!outs[k]) continue;
      const long long dx = diag_out_extent(outs[k], N, bs);
      if (outs[k]->diag && !d2h(static_cast<zd*>(outs[k]->diag) + dx * e0, dout[q][k].diag, sizeof(zd) * dx * Ec)) return set_err(c, BT_ERR_CUDA, "D2H failed");
      if (outs[k]->upper && !d2h(static_cast<zd*>(outs[k]->upper) + N1B2 * e0, dout[q][k].upper, sizeof(zd) * N1B2 * Ec)) return set_err(c, BT_ERR_CUDA, "D2H failed");
      if (outs[k]->lower && !d2h(static_cast<zd*>(outs[k]->lower) + N1B2 * e0, dout[q][k].lower, sizeof(zd) * N1B2 * Ec)) return set_err(c, BT_ERR_CUDA, "D2H failed");
    }
    if (!d2h(status_host + e0, dstatus[q], sizeof(int) * Ec)) return set_err(c, BT_ERR_CUDA, "D2H failed");
    if (nbuf > 1 && cudaEventRecord(c->ev_done[q], cs) != cudaSuccess) return set_err(c, BT_ERR_CUDA, "event record failed");
  }
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess)
    return set_err(c, BT_ERR_CUDA, "stream error");
  return BT_OK;
}
