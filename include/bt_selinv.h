/*
 * bt_selinv.h -- C ABI of the GB300 (sm_103a) block-tridiagonal selected-inversion library.
 *
 * The library computes, for a batch of energies, the selected blocks of the solution of the
 * quadratic system of Sec. 3, Eq. 1 of "QuaTrEx: ... NEGF+scGW" (arXiv 2508.19138):
 *
 *     (M - B^R) X^<> (M - B^R)^H = B^<>,      X^R = (M - B^R)^{-1} = M~^{-1},
 *
 * with the quantities of Table 2:
 *   electrons (BT_SYS_G):          M = E S - H,  B^R = Sigma^R,   B^<> = Sigma^<>
 *   screened Coulomb (BT_SYS_W):   M = I,        B^R = V P^R,     B^<> = V P^<> V^H
 * plus the open-boundary blocks B_OBC of Sec. 4.2 (Eq. 4, Sancho-Rubio decimation; lesser /
 * greater by fluctuation-dissipation).  The solver is the recursive Green's function method
 * of Sec. 4.3.2 (forward pass Eq. 9-10, backward pass Eq. 11-12), with the symmetrisation of
 * Sec. 5.2.  Outputs are the diagonal and first off-diagonal blocks.
 *
 * Conventions shared by every entry point:
 *   - complex numbers are complex128: two doubles (re, im), the layout of cuDoubleComplex,
 *     std::complex<double> and torch.complex128;
 *   - a block is bs x bs, row-major; block arrays are [nb][bs][bs] (diagonal blocks) and
 *     [nb-1][bs][bs] (upper blocks (i,i+1) or lower blocks (i+1,i)), with a leading
 *     [n_energies] dimension for per-energy data;
 *   - unless an entry point says otherwise all data pointers are DEVICE pointers owned by the
 *     caller; the library owns only its workspace (allocated in bt_selinv_create);
 *   - calls are asynchronous on the stream given at creation; the return code reports
 *     argument and launch errors, numerical failures are reported per energy in a device
 *     status array (bt_status codes);
 *   - no C++ exception crosses this boundary; a context is bound to one stream and is not
 *     thread-safe.
 */
#ifndef BT_SELINV_H
#define BT_SELINV_H

#include <stddef.h>

#if defined(__GNUC__)
#define BT_API __attribute__((visibility("default")))
#else
#define BT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BT_OK = 0,
  BT_ERR_INVALID_ARG = 1,   /* a size, pointer or flag is out of range                      */
  BT_ERR_OOM = 2,           /* cudaMalloc of the workspace failed                            */
  BT_ERR_BUDGET = 3,        /* the workspace would exceed hbm_budget_bytes                   */
  BT_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed                   */
  BT_ERR_SINGULAR = 5,      /* per energy: a zero pivot in a block inversion                 */
  BT_ERR_NOT_CONVERGED = 6, /* per energy: decimation reached decim_maxit                    */
  BT_ERR_NONFINITE = 7,     /* per energy: NaN / Inf reached a pivot of a block inversion or */
                            /* the decimation's convergence test (non-finite H, S, Sigma^R,  */
                            /* P^R or V); non-finite lesser/greater inputs are not scanned:  */
                            /* they reach the lesser/greater outputs with status BT_OK       */
  BT_ERR_TIMEOUT = 8,       /* a bounded device wait expired                                 */
  BT_ERR_UNSUPPORTED = 9,   /* valid request this build does not implement                   */
  BT_ERR_CANCELLED = 10     /* serving: the request was cancelled (server destroyed)         */
} bt_status;

typedef enum { BT_SYS_G = 0, BT_SYS_W = 1 } bt_system;           /* Table 2 columns      */
typedef enum { BT_FP64 = 0, BT_SPLIT = 1 } bt_precision;         /* see bt_selinv_desc   */
typedef enum { BT_LAYOUT_BLOCKS = 0, BT_LAYOUT_DIAGVEC = 1, BT_LAYOUT_PACKED_UPPER = 2 } bt_layout;
typedef enum { BT_SYM_GENERAL = 0, BT_SYM_HERMITIAN = 1, BT_SYM_ANTIHERMITIAN = 2 } bt_symmetry;

/* A block-tridiagonal input operand.
 *   diag   BT_LAYOUT_BLOCKS : [nb][bs][bs] diagonal blocks
 *          BT_LAYOUT_DIAGVEC: [nb][bs] the diagonal entries only (a diagonal matrix; upper and
 *                             lower must be NULL)
 *          BT_LAYOUT_PACKED_UPPER (Sigma^< / Sigma^> of the G system, P^< / P^> of the W system,
 *                             symmetry BT_SYM_ANTIHERMITIAN; Sec. 5.2): [nb][bs (bs + 1) / 2]
 *                             the upper triangle of each anti-Hermitian diagonal block, row by
 *                             row, entry (r, c >= r) at r bs - r (r - 1) / 2 + (c - r); upper
 *                             blocks in full
 *   upper  [nb-1][bs][bs] blocks (i,i+1); NULL means all off-diagonal blocks are zero
 *   lower  [nb-1][bs][bs] blocks (i+1,i); read only when symmetry == BT_SYM_GENERAL, else
 *          block (i+1,i) is upper[i]^H (HERMITIAN) or -upper[i]^H (ANTIHERMITIAN)
 *   per_energy  0: one operand shared by every energy; 1: each pointer addresses
 *          [n_energies][...] with the per-energy extent given above
 * Pointers are device pointers (host pointers for bt_selinv_solve_host).  diag may be NULL
 * only for optional operands (then the whole operand is zero). */
typedef struct {
  const void* diag;
  const void* upper;
  const void* lower;
  int layout;
  int symmetry;
  int per_energy;
} bt_bt;

/* An output operand: [n_energies][nb][bs][bs] diagonal blocks, [n_energies][nb-1][bs][bs]
 * upper (i,i+1) and lower (i+1,i) blocks.  A NULL pointer means "do not write".
 * layout BT_LAYOUT_DIAGVEC writes only the diagonal entries of the diagonal blocks,
 * [n_energies][nb][bs] (densities / local DOS), and requires upper = lower = NULL.
 * layout BT_LAYOUT_PACKED_UPPER (lesser / greater outputs with symmetrize = 1 only; Sec. 5.2:
 * anti-Hermitian quantities stored by their upper triangle) writes each diagonal block
 * X_ii = -X_ii^H as its upper triangle, row by row: [n_energies][nb][bs (bs + 1) / 2], entry
 * (r, c >= r) at r bs - r (r - 1) / 2 + (c - r), the lower triangle being -conj of it; upper
 * (i,i+1) blocks are written in full as with BT_LAYOUT_BLOCKS; lower must be NULL. */
typedef struct {
  void* diag;
  void* upper;
  void* lower;
  int layout;
} bt_bt_out;

typedef struct {
  int nb;              /* number of diagonal blocks N_B >= 1                                  */
  int bs;              /* block size N_BS >= 1                                                */
  int max_energies;    /* energies processed per chunk; sizes the workspace                   */
  int system;          /* bt_system                                                            */
  int precision;       /* BT_FP64: every product in FP64.  BT_SPLIT: the off-diagonal block
                          products of the sweeps as sliced (Ozaki) products on the bf16 tensor
                          cores with exact fp32 accumulation; inversions, decimation and
                          symmetrisation stay FP64                                              */
  int split_slices;    /* BT_SPLIT: slices per operand (0 = default 6, range 2..8)            */
  int symmetrize;      /* 1: lesser/greater diagonal blocks returned as (X - X^H)/2 (Sec. 5.2) */
  int obc;             /* 1: contacts on both ends (nb >= 2), each lead repeating the device's
                          edge cell.  G: Sancho-Rubio surface functions and fluctuation-
                          dissipation (Sec. 4.2, Eq. 4).  W: the lead cells repeat the edge
                          cell of V and P and its coupling inward; retarded boundary by
                          decimation (Eq. 4), lesser / greater boundary by the Stein equation
                          w = q + a w a^H (Eq. 7; solved by doubling), plus the edge cells'
                          products with the first lead cell                                   */
  double eta;          /* G: z = E + i eta                                                     */
  double kT;           /* contact temperature (energy units of H)                              */
  double mu_left;      /* contact Fermi levels                                                 */
  double mu_right;
  double decim_tol;    /* decimation stops when max|a|,max|b| <= decim_tol * max|n| (<=0: 1e-14) */
  int decim_maxit;     /* decimation iteration cap (<= 0: 100)                                 */
  size_t hbm_budget_bytes; /* 0 = unlimited; otherwise the workspace must fit                  */
  /* Contact memoization (Sec. 5.3): the surface functions of every solved energy are kept in
   * the workspace (memo_capacity energies, oldest evicted first).  A later solve of the same
   * energy starts the fixed-point iteration x <- (m - n x n')^{-1} (Eq. 5) from the kept value
   * and runs at most memo_nfpi iterations; leads that do not converge within them (judged from
   * the update ratio) fall back to decimation.  0 = off.                                        */
  int obc_memo;
  int memo_nfpi;           /* <= 0: 20                                                          */
  int memo_capacity;       /* energies kept; <= 0: 4 * max_energies                             */
  int split_scope;         /* BT_SPLIT only.  0: sliced products in the sweeps (the default
                              split); 1: also the products inside the block inversions (the
                              rank-kb updates), the decimation and the memoized fixed point,
                              those with one slice more (split_slices + 1, at most 8)         */
  /* Graph mode (the batching pattern: one launch per chunk).  1: the first solve of a chunk
   * with a given set of operand pointers captures all of its launches into a CUDA graph, with
   * the decimation loop as a device-side conditional while node (the iteration stops when the
   * device count of unconverged leads reaches zero or at decim_maxit), and later solves with the
   * same pointers replay it as one graph launch (the 8 most recent chunks are kept).  Needs a
   * non-default stream; exclusive with obc_memo.  The decimation statistics of a replay are
   * read back asynchronously and folded in at the next solve or bt_selinv_get_stats (which then
   * synchronises the stream).  0: direct launches.                                              */
  int graph;
  /* Newton step on the decimated surface functions (Sec. 4.2, Eq. 4).  FP64 decimation loses
   * accuracy where a lead mode decays slowly (energies near a band edge at small eta; up to
   * ~1e-8 relative after 25 iterations).  Leads whose decimation took more than this many
   * iterations get one Newton step on x^{-1} (a Stein equation solved by doubling), which brings
   * the surface function back to FP64 accuracy.  0: 14; negative: never.                        */
  int decim_newton_after;
  /* Kernel shape overrides (the autotuner's knobs; 0 = the built-in rule).  gemm_tile: output
   * tile of the FP64 products, 16 or 32 (rule: 32 unless that leaves SMs idle).  inv_panel:
   * panel width of the blocked inversions, 4, 8, 16 or 32, used only when narrower than the
   * built-in width (16 with FP64 updates, 32 with sliced ones).                                 */
  int gemm_tile;
  int inv_panel;
} bt_selinv_desc;

typedef struct bt_ctx bt_ctx;

typedef struct {
  long long solves;            /* bt_selinv_solve calls completed (host count)                */
  long long energies;          /* energies processed                                          */
  long long decim_iterations;  /* sum over chunks of the decimation iterations executed       */
  double flops_model;          /* minimal-model flops of the last solve (8 b^3 per block
                                  product or inversion, actual decimation iterations)         */
  size_t workspace_bytes;
  long long kernel_launches;   /* kernels this context launched (all solves)                  */
  long long lead_iterations;   /* decimation iterations summed over leads (all solves)        */
  long long fpi_iterations;    /* memoized fixed-point iterations summed over leads           */
  long long memo_hits;         /* energies whose contacts started from a kept surface function*/
  long long newton_leads;      /* leads that took the Newton step after decimation            */
  long long newton_iterations; /* doubling iterations of those steps, summed over leads       */
} bt_stats;

/* Sizes of the workspace bt_selinv_create would allocate for `desc`. */
BT_API bt_status bt_selinv_workspace_bytes(const bt_selinv_desc* desc, size_t* bytes);

/* Validate `desc`, allocate the workspace on the current device, bind `cuda_stream`
 * (a cudaStream_t; NULL = default stream).  On success *out owns the workspace. */
BT_API bt_status bt_selinv_create(const bt_selinv_desc* desc, void* cuda_stream, bt_ctx** out);

/* Selected inversion for n_energies energies (processed in chunks of max_energies): the
 * selected blocks of X^R, X^<, X^> of Sec. 3, Eq. 1 with the quantities of Table 2, by the RGF
 * passes of Sec. 4.3.2 (Eq. 9-12) and, with desc->obc, the contacts of Sec. 4.2 (Eq. 4).
 *   H       G: Hamiltonian H (BLOCKS, Hermitian or general, shared or per energy)
 *           W: bare Coulomb V (BLOCKS, Hermitian, shared)
 *   S       G: overlap (NULL = identity); W: must be NULL
 *   sigR    G: retarded scattering self-energy Sigma^R (NULL = 0; BLOCKS or DIAGVEC)
 *           W: retarded polarisation P^R (BLOCKS, per energy)
 *   sigL/G  G: Sigma^< / Sigma^> (NULL = 0); W: P^< / P^> (BLOCKS, per energy, anti-Hermitian)
 *   energies_host  [n_energies] energies E (host memory; read before the call returns)
 *   outR    G: X^R = G^R blocks (diag, upper, lower); W: W^R = X^R V blocks
 *   outL/G  G: G^< / G^> (diag, upper; lower = -upper^H is not written); W: W^< / W^>
 *   status_device  [n_energies] ints, BT_OK or the first numerical failure of that energy
 * Returns BT_OK when every launch was issued. */
BT_API bt_status bt_selinv_solve(bt_ctx* ctx, const bt_bt* H, const bt_bt* S, const bt_bt* sigR,
                          const bt_bt* sigL, const bt_bt* sigG, const double* energies_host,
                          int n_energies, const bt_bt_out* outR, const bt_bt_out* outL,
                          const bt_bt_out* outG, int* status_device);

/* Same as bt_selinv_solve, but every data pointer (inputs, outputs, status) is HOST memory.
 * Inputs are copied to the device chunk by chunk, outputs copied back; the call returns
 * after the last copy completed (synchronous).  Pinned host memory gives full copy speed.
 * With more than one chunk the device staging of the outputs is double-buffered and the copies
 * of chunk k back to the host run on a second stream while chunk k + 1 computes. */
BT_API bt_status bt_selinv_solve_host(bt_ctx* ctx, const bt_bt* H, const bt_bt* S, const bt_bt* sigR,
                               const bt_bt* sigL, const bt_bt* sigG, const double* energies_host,
                               int n_energies, const bt_bt_out* outR, const bt_bt_out* outL,
                               const bt_bt_out* outG, int* status_host);

/* Counters of ctx (host struct *out).  In graph mode it first synchronises ctx's stream to
 * fold in the device-side iteration counts.  BT_ERR_INVALID_ARG for NULL arguments. */
BT_API bt_status bt_selinv_get_stats(const bt_ctx* ctx, bt_stats* out);
/* Waits for ctx's work, frees its workspace and graphs; NULL is a no-op. */
BT_API bt_status bt_selinv_destroy(bt_ctx* ctx);
/* Text of the last error recorded on ctx (or of the last failed create when ctx is NULL). */
BT_API const char* bt_selinv_last_error(const bt_ctx* ctx);

/* ---------------------------------------------------------------------------------------
 * Serving: solves of different device sizes arriving over time (G system).  The paper has no
 * counterpart (its energies are distributed over ranks, Sec. 4.4); each unit of work is the
 * solve of bt_selinv_solve (Sec. 3, Eq. 1; Sec. 4.3.2).
 *   - a request is split into work units of max_energies_per_chunk energies each;
 *   - bt_server_create allocates ONE device arena of hbm_budget_bytes; each unit borrows its
 *     workspace (bt_selinv_workspace_bytes for one chunk) from it while it runs;
 *   - a free worker starts the next unit chosen round robin over the requests with units left
 *     (every admitted request progresses chunk by chunk); a unit that does not fit in the free
 *     memory now is passed by smaller ones, at most max_skips times (<= 0: 2 max_active) for the
 *     oldest waiting request;
 *   - max_active worker threads, each with its own stream, run units concurrently (continuous
 *     batching: new requests start while earlier ones are still on the GPU);
 *   - a unit whose solve reports BT_ERR_TIMEOUT (a bounded device wait expired) is started
 *     again, up to max_retries times; requests not started when the server is destroyed end
 *     with BT_ERR_CANCELLED;
 *   - a request's inputs / outputs are the caller's device buffers and must stay valid until
 *     the request is done; results equal those of bt_selinv_solve with the same chunking.
 * ------------------------------------------------------------------------------------- */
typedef struct bt_server bt_server;

typedef struct {
  size_t hbm_budget_bytes;    /* arena size (device memory reserved at create)             */
  int max_active;             /* concurrent requests, 1..64                                */
  int max_energies_per_chunk; /* energies per batched launch of one request                */
  int precision;              /* bt_precision                                              */
  int split_slices;           /* BT_SPLIT slices (0 = default)                             */
  int device;                 /* CUDA device ordinal                                       */
  int split_scope;            /* BT_SPLIT: as bt_selinv_desc.split_scope (0 or 1)          */
  int max_retries;            /* restarts of a unit that timed out (>= 0)                  */
  int max_skips;              /* passes of the oldest waiting request (<= 0: 2 max_active) */
  int graph;                  /* 1: each unit runs as one captured graph (its decimation and
                                 Newton loops on the device, no host round trip per loop
                                 iteration); 0: direct launches.  A unit's graph is captured
                                 for one launch, so its capture cost is not amortised: direct
                                 launches serve the mixed request stream faster (measured)    */
} bt_server_desc;

typedef struct {
  int nb, bs, n_energies;
  bt_bt H;                    /* shared across energies (device)                           */
  bt_bt S, sigR, sigL, sigG;  /* optional: diag == NULL means absent                       */
  const double* energies_host;/* [n_energies], copied by bt_server_submit                  */
  double eta, kT, mu_left, mu_right;
  int obc;                    /* Sancho-Rubio contacts from the edge blocks (nb >= 2)      */
  bt_bt_out outR, outL, outG; /* device outputs (NULL pointers = not written)              */
  int* status_device;         /* [n_energies]                                              */
} bt_request;

typedef struct {
  long long submitted, completed, failed, rejected, energies_done, queued;
  int active, peak_active;
  double p50_latency_s, p99_latency_s, mean_latency_s; /* submit -> completion, completed  */
  double busy_seconds;        /* time with at least one work unit running (idle gaps       */
                              /* between arrivals excluded)                                */
  double energies_per_s;      /* energies_done / busy_seconds                              */
  size_t peak_bytes;          /* largest arena occupancy                                   */
  long long units_done;       /* work units (energy chunks) completed                      */
  long long retries;          /* units started again after a device timeout                */
} bt_server_stats;

BT_API bt_status bt_server_create(const bt_server_desc* desc, bt_server** out);
/* Queue a request; returns a ticket.  BT_ERR_BUDGET if its workspace can never fit. */
BT_API bt_status bt_server_submit(bt_server* srv, const bt_request* req, long long* ticket);
/* state: 0 queued, 1 running, 2 done, 3 failed or cancelled (the return code is then the
 * failure, BT_ERR_CANCELLED for a cancelled request). */
BT_API bt_status bt_server_poll(bt_server* srv, long long ticket, int* state);
/* Block until the request is done or failed, or timeout_s passed (BT_ERR_TIMEOUT). */
BT_API bt_status bt_server_wait(bt_server* srv, long long ticket, double timeout_s, int* state);
BT_API bt_status bt_server_get_stats(bt_server* srv, bt_server_stats* out);
/* Cancels requests with units not yet started (BT_ERR_CANCELLED), waits for running units,
 * frees the arena. */
BT_API bt_status bt_server_destroy(bt_server* srv);

/* ---------------------------------------------------------------------------------------
 * Building blocks, exported for callers that assemble their own sweeps (and for tests).
 * ------------------------------------------------------------------------------------- */

enum { BT_OP_N = 0, BT_OP_C = 1 };  /* op(X) = X or X^H (conjugate transpose) */

/* C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b] for b < batch, complex128, FP64 arithmetic
 * (the dense products of Eq. 9-12).  op(A) is m x k, op(B) is k x n, C is m x n, all row-major
 * with leading dimensions lda/ldb/ldc (elements); strideX is the element distance between
 * batch entries (0 = the same matrix for every batch entry).  beta = 0 does not read C.
 * C must not alias A or B. */
BT_API bt_status bt_zgemm_batched(int m, int n, int k, double alpha_re, double alpha_im,
                           const void* A, int lda, long long strideA, int opA,
                           const void* B, int ldb, long long strideB, int opB,
                           double beta_re, double beta_im, void* C, int ldc, long long strideC,
                           int batch, void* stream);

/* Same product with the sliced split-precision scheme used by BT_SPLIT: each operand is
 * scaled per row (A) / per column (B) by a power of two and cut into `slices` 7-bit integer
 * slices held exactly in bf16; slice products run on the tcgen05 tensor cores with fp32
 * accumulation that is exact (K segments of at most 480 complex terms; the slice pairs of one
 * weight class share an accumulator while its sum stays an integer below 2^24), and are summed
 * exactly in a 64-bit fixed point per output, converted to FP64 once.
 * Any m, n, k >= 1: ragged edges are zero padded.
 * `workspace` must hold bt_split_zgemm_workspace_bytes(m, n, k, slices, batch) bytes. */
BT_API bt_status bt_split_zgemm_workspace_bytes(int m, int n, int k, int slices, int batch, size_t* bytes);
BT_API bt_status bt_split_zgemm_batched(int m, int n, int k, double alpha_re, double alpha_im,
                                 const void* A, int lda, long long strideA, int opA,
                                 const void* B, int ldb, long long strideB, int opB,
                                 double beta_re, double beta_im, void* C, int ldc, long long strideC,
                                 int batch, int slices, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* In-place inverse of `batch` n x n complex128 matrices (A + b*strideA), Gauss-Jordan
 * elimination with partial (row) pivoting -- the block LU of the forward pass (Eq. 9) carried
 * to the full inverse; pivots chosen by max |re| + |im|, first index on ties.
 * info_device[b] = 0, or BT_ERR_SINGULAR / BT_ERR_NONFINITE (matrix b is then undefined).
 * `workspace` must hold bt_zinv_workspace_bytes(n, batch) bytes (may be 0 for small n). */
BT_API bt_status bt_zinv_workspace_bytes(int n, int batch, size_t* bytes);
BT_API bt_status bt_zinv_batched(int n, void* A, long long strideA, int batch, int* info_device,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free bt_zinv_batched (the paper has no counterpart: this is a service for callers
 * that cannot allocate device memory when they invert, e.g. code running inside its own pool
 * allocator or with all free memory already handed to an arena).  Same inputs, outputs and
 * numerics as bt_zinv_batched, but the scratch is a fixed array of
 * BT_ZINV_NOALLOC_SCRATCH_BYTES bytes inside the library (present on every GPU that loads the
 * library until the process exits); the call itself never allocates.
 *   - needs bt_zinv_workspace_bytes(n, batch) <= BT_ZINV_NOALLOC_SCRATCH_BYTES, else returns
 *     BT_ERR_BUDGET and launches nothing (n <= 96 needs no scratch at all);
 *   - the first call on a device, with that device current, looks up the array's device
 *     address; under CUDA's default lazy module loading that lookup also loads the library's
 *     device code for the array and so reserves its memory on that device (an allocation made
 *     by the CUDA driver, which can fail when the device is full).  Make that first call before
 *     the caller's pool or arena takes the device's free memory, and before any stream
 *     capture; later calls on that device allocate nothing;
 *   - every call shares the array: calls that overlap on the GPU (other streams or threads)
 *     race; calls on one stream are ordered.  The array keeps the last call's contents and
 *     needs no clearing (every word is written before it is read). */
#define BT_ZINV_NOALLOC_SCRATCH_BYTES (16u << 20)
BT_API bt_status bt_zinv_batched_noalloc(int n, void* A, long long strideA, int batch, int* info_device,
                                         void* stream);

/* Surface Green's function of semi-infinite leads, x = (m - n x n')^{-1} (Eq. 4), by
 * Sancho-Rubio decimation for `batch` independent leads (m, n, n' each [batch][bs][bs]); leads
 * that needed more than 14 iterations then get one Newton step on x^{-1} (see
 * bt_selinv_desc.decim_newton_after), which restores FP64 accuracy near band edges.
 * Writes x [batch][bs][bs] and the boundary block sigma = n x n' [batch][bs][bs];
 * iters_device[b] = iterations used, info_device[b] = 0 / BT_ERR_NOT_CONVERGED / _SINGULAR /
 * _NONFINITE (x and sigma of lead b are then undefined).
 * `workspace` must hold bt_decimate_workspace_bytes(bs, batch) bytes. */
BT_API bt_status bt_decimate_workspace_bytes(int bs, int batch, size_t* bytes);
BT_API bt_status bt_decimate_batched(int bs, int batch, const void* m, const void* n, const void* n_prime,
                              double tol, int maxit, void* x, void* sigma, int* iters_device,
                              int* info_device, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Element-wise energy convolution (Sec. 4.4, Eq. 3): the scattering self-energy / polarization of
 * an (i, j) entry is an energy integral of products of two particle descriptors, each entry
 * independent of the others.  On a uniform grid it is, for every element series e < n_elem,
 *     C[m - m0][e] = s * sum_k A[m - k][e] * B'[k][e],      m0 <= m < m0 + n_out,
 * with A[i][e] = 0 outside 0 <= i < na and B'[k][e] = B[k][e] (or B[nb - 1 - k][e] with
 * BT_CONV_REVERSE_B, a cross-correlation; conjugated with BT_CONV_CONJ_B) zero outside
 * 0 <= k < nb; the full result has na + nb - 1 entries (m0 + n_out must not exceed that).  The
 * factor s = scale_re + i scale_im carries the proportionality constant and the energy step.
 * Layout: energy-major complex128, element e of energy k at A + k lda + e (lda >= n_elem; the
 * outputs of bt_selinv_solve are element series with lda = nb bs^2, or nb bs (bs + 1) / 2 for
 * packed upper triangles).  Device pointers; C must not alias A or B.  Computed by FFTs of
 * length L = the power of two >= na + nb - 1 in FP64 (L <= 4096, else BT_ERR_UNSUPPORTED);
 * asynchronous on `stream`; allocates nothing.
 * ------------------------------------------------------------------------------------- */
enum { BT_CONV_REVERSE_B = 1, BT_CONV_CONJ_B = 2 };
BT_API bt_status bt_energy_convolve(int n_elem, int na, int nb, int m0, int n_out, const void* A, long long lda,
                                    const void* B, long long ldb, void* C, long long ldc, double scale_re,
                                    double scale_im, int flags, void* stream);

/* ---------------------------------------------------------------------------------------
 * Test hook (no counterpart in the paper).  Every wait of the tensor-core GEMM's pipeline on a
 * shared-memory barrier is bounded (2 s); when one expires, the CTA records BT_ERR_TIMEOUT, stops
 * issuing work, waits (bounded) for the copies and products it already issued, frees its tensor
 * memory and exits, and every energy of the chunk gets BT_ERR_TIMEOUT in the solve's status.
 * With ns > 0, the MMA warp of the next `launches` launches of that GEMM (every later launch when
 * launches < 0) first waits up to ns nanoseconds on a barrier that nothing completes, so that
 * this path runs on demand; ns = 0 turns the hook off.  Process-wide, read when a launch is
 * issued (a captured graph keeps the value it was captured with).
 * ------------------------------------------------------------------------------------- */
BT_API void bt_debug_split_stall(unsigned long long ns, long long launches);

/* Measurement aid (no counterpart in the paper): the FP64 multiply-add rate of this GPU on
 * registers only, which = 0 for DFMA (fma.rn.f64), 1 for the FP64 tensor instruction
 * (mma.sync m8n8k4 f64); one launch of iters iterations after a warm-up launch, timed with CUDA
 * events on `stream`.  Writes TFLOP/s (2 flops per multiply-add) and the launch time in ms. */
BT_API bt_status bt_debug_fp64_rate(int which, int iters, double* tflops, double* ms, void* stream);

/* Measurement aid (no counterpart in the paper): forces the cluster size of the Gauss-Jordan
 * panel kernel of the blocked inverse (n >= 192) to cl = 2, 4 or 8 CTAs per matrix; any other
 * value restores the default (the largest cluster for which the whole batch is resident at
 * once, by the occupancy the device reports).  Process-wide, read when a launch is issued (a
 * captured graph keeps the size it was captured with).  Results do not depend on it. */
BT_API void bt_debug_panel_cluster(int cl);

/* Measurement aid (no counterpart in the paper): enable = 1 zeroes a set of device counters that
 * every later launch of the tensor-core GEMM of bt_split_zgemm_batched (and of the BT_SPLIT
 * solves) adds to; enable = 0 stops counting, synchronizes the device and copies up to
 * n_counters of them to host memory `counters`:
 *   [0] SM cycles the MMA-issuing thread waited for a pipeline stage's TMA data,
 *   [1] ... waited for an accumulator the epilogue had not drained yet,
 *   [2] ... spent in its whole loop, [3] cycles the TMA-issuing thread waited for a free stage,
 *   [4] cycles epilogue warp 0 spent draining accumulators, [5] ... writing C, [6] tiles,
 * each summed over all CTAs.  Off by default; a launch reads the setting when issued. */
BT_API bt_status bt_debug_split_profile(int enable, unsigned long long* counters, int n_counters);

/* Measurement aid (no counterpart in the paper): the preferred L1 / shared-memory split of the
 * current device for kernels without a carveout of their own, config = 0 no preference,
 * 1 prefer shared memory, 2 prefer L1, 3 equal (cudaDeviceSetCacheConfig: state of the calling
 * process's CUDA context, nothing that outlasts it). */
BT_API bt_status bt_debug_cache_config(int config);

/* Measurement aid (no counterpart in the paper): the tensor-core GEMM's CTA arrangement for later
 * launches, mode 1 = one CTA per 128-row tile, 2 = CTA pairs (tcgen05 cta_group::2: a pair of
 * CTAs on two SMs computes two 128-row tiles that share their At tile, each CTA holding half of
 * it) wherever the shape has two or more 128-row tiles and the device holds most SMs as pairs,
 * 3 = CTA pairs whose pipeline stages hold two 64-deep K blocks (half the waits and commits per
 * MMA, three stages), 0 = the default (mode 3 when the 2n rows of C^T are an even number of
 * 128-row tiles, else mode 1).  Results are bitwise the same either way (exact fixed-point accumulation).
 * Process-wide, read when a launch is issued. */
BT_API void bt_debug_split_pair(int mode);

/* Measurement aid (no counterpart in the paper): how the tensor-core GEMM groups the slice-pair
 * products of one K segment into TMEM accumulators for later launches.  mode 0 (default): the
 * pairs of one weight class s + t share an accumulator while its fp32 sum stays an exact integer
 * (below 2^24), classes two by two in dual jobs, a lane of several pairs drained by an exact
 * float -> int conversion; mode 1: one pair per accumulator (several only in short segments, below
 * 2^22).  Both sum the same exact products into the same fixed point; they round the classes of
 * weight below 2^-F (F = the fixed point's fraction bits) at different points, so results agree
 * to that resolution, not bitwise.  Process-wide, read when a launch is issued. */
BT_API void bt_debug_split_sched(int mode);

/* Host-only query (no GPU work): the accumulation schedule of the tensor-core GEMM for `slices`
 * slices per operand and k_blocks 64-deep K blocks (K' = 64 k_blocks real terms), mode as in
 * bt_debug_split_sched.  Writes up to max_jobs rows of 8 ints to `jobs` (dual, first item, end
 * item, first K block, end K block, lane 0 converted exactly, lane 1 converted exactly, 0), up to
 * max_items rows of 3 ints to `items` (slice s of op(A) for lane 0, slice s2 for lane 1, slice t
 * of op(B); 1-based), and the fixed point's fraction bits F to *fix_bits (any pointer may be
 * NULL).  Returns the number of jobs, or -1 for unsupported arguments (slices outside 2..8,
 * k_blocks outside 1..255, or a schedule beyond the kernel's job or item capacity). */
BT_API int bt_debug_split_schedule(int slices, int k_blocks, int mode, int* jobs, int max_jobs, int* items,
                                   int max_items, int* fix_bits);

/* Measurement aid (no counterpart in the paper): the busy fraction of the tensor pipe when one
 * thread per SM issues tcgen05.mma (M = 128, N = 224, K = 16; four per 64-deep K block and a
 * commit, the GEMM's pattern) on operands already in shared memory, while busy_warps (0..16)
 * other warps of the CTA run multiply-add chains and, with wait != 0, an already-completed
 * mbarrier is waited on before each K block.  One launch on all SMs, timed with the SM clock. */
BT_API bt_status bt_debug_mma_issue_rate(int busy_warps, int wait, double* frac, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BT_SELINV_H */
