/*
 * tdc.h -- C ABI of the GB300 structured divide-and-conquer tridiagonal
 * eigensolver (Liao, Li, Lu, Roman, "A parallel structured divide-and-conquer
 * algorithm for symmetric tridiagonal eigenvalue problems", IEEE TPDS 2020).
 *
 * Problem (Section 2, Eq. (t)): T is a real symmetric tridiagonal n x n matrix
 * with diagonal d[0..n) and off-diagonal e[0..n-1) (T(i,i+1) = T(i+1,i) = e[i]).
 * The solver returns T = Q diag(lam) Q^T with lam ascending and Q orthogonal,
 * by Cuppen's divide and conquer (Algorithm 1 / Algorithm 3): leaf eigensolves,
 * then a level-by-level merge that deflates (Section 3.2), solves the secular
 * equation (Eq. (secular)), recomputes zhat, and updates the eigenvectors as
 * Q * U with the Cauchy-like U of Eq. (Q_Cauchy) generated from (d, lambda,
 * zhat) inside the GEMM (Section 3.1's generator observation) -- densely, with
 * off-diagonal tiles compressed (Section 2.1, SRRSC), or as split-precision
 * BF16 slice products.
 *
 * Conventions for every entry point:
 *   - all array pointers are DEVICE pointers unless the name ends in _host;
 *     the caller owns every buffer, including the workspace; the library
 *     allocates no device memory on these paths;
 *   - matrices are column-major FP64 with a leading dimension argument;
 *   - work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without synchronising.  The eigensolvers
 *     also use a second, high-priority stream of the calling host thread
 *     (created on first use and kept) for each level's products, forked from
 *     and joined back into `stream` with events: the call stays ordered on
 *     `stream` and can be captured in a CUDA graph like single-stream work.
 *     That stream and the thread's event pool are created by the first call
 *     from each host thread on each device, so make that call before capturing
 *     from the thread;
 *   - the return value is a status: TDC_OK (0); -i when argument i (1-based)
 *     is invalid, checked on the host before anything is enqueued; or one of
 *     the TDC_E* codes below.  Device-side failures (secular non-convergence,
 *     a bounded wait that expired) and warnings are recorded in the status
 *     slot of the call's stream, which tdc_sync_status() returns;
 *   - inputs d and e are never modified.
 */
#ifndef TDC_H
#define TDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tdc_stream_t; /* identical to cudaStream_t */

/* status codes */
#define TDC_OK 0
#define TDC_ENOWS (-101)       /* workspace pointer NULL or smaller than tdc_*workspace_size */
#define TDC_ENONFINITE (-102)  /* non-finite value produced (device status) */
#define TDC_ENOCONV (-103)     /* secular or leaf iteration hit its cap (device status) */
#define TDC_ETIMEOUT (-104)    /* a bounded device-side wait expired (device status) */
#define TDC_ECUDA (-105)       /* a CUDA runtime call failed */
#define TDC_EUNSUPPORTED (-106) /* option combination not supported */
#define TDC_ETOOLARGE (-107)   /* problem needs more than the fixed scratch of tdc_eig_noalloc */
/* warning (device status, positive): the results were written, but a level sum of the split
 * product reached 2^23, half of the range its FP32 accumulators hold exactly, so the
 * eigenvectors may miss the FP64 accuracy bound (use a smaller split_chunk_k or
 * TDC_MERGE_DENSE).  Errors take precedence over it. */
#define TDC_WPRECISION 1

/* merge modes: how the eigenvector update Q * U is computed */
#define TDC_MERGE_AUTO 0        /* library choice: merges with K >= structured_min_K take the structured path on
                                   the split GEMM (TDC_MERGE_STRUCTURED_SPLIT), merges with K >= split_min_K
                                   the split path, smaller ones FP64 */
#define TDC_MERGE_DENSE 1       /* FP64 GEMM, U generated from its generators in the producer */
#define TDC_MERGE_STRUCTURED 2  /* near-diagonal tiles dense, off-diagonal tiles SRRSC-compressed */
#define TDC_MERGE_SPLIT 3       /* BF16 slice products on tcgen05 tensor cores, FP32/FP64 accumulation, for
                                   merges with K >= split_min_K (FP64 below), every merge unstructured */
#define TDC_MERGE_STRUCTURED_SPLIT 4 /* the structured update (near-diagonal tiles dense, off-diagonal tiles
                                        SRRSC-compressed) with all of its products on the split tensor-core
                                        path, for merges with K >= max(structured_min_K, split_min_K); a merge
                                        half whose far tiles pass the rank cap (64) or need more low-rank
                                        columns than the path's buffer takes the split path whole; smaller
                                        merges as TDC_MERGE_SPLIT.  This is AUTO's choice. */
/* Accuracy of the split path (SPLIT and AUTO): the digit products of one level are
 * summed in FP32 accumulators, exact only while each level's sum stays below 2^24.
 * The default schedule drains them into 64-bit integer sums every split_chunk_k = 256
 * terms, which keeps every level sum far below that limit: the residual and
 * orthogonality ratios ||TQ - Q Lam||_1 / (n ||T|| eps) and ||Q^T Q - I||_1 / (n eps)
 * stay below 2 on random spectra, tridiag(1,2,1), d ~ U(0,1) with e = 1, and on the
 * smooth-eigenvector families (Clement/Kac, Hermite, spherical-harmonic) up to n = 30000.
 * Summing over a tile's whole reduction instead (split_chunk_k = 0) is about 10 %
 * faster at n = 16384 but not exact on smooth-eigenvector matrices from n = 8192 on
 * (orthogonality ratios of 1e3 to 1e5).  Every drain checks its level sums; one that
 * reached 2^23 raises the warning TDC_WPRECISION and is counted in
 * tdc_stats.split_level_max. */

typedef struct {
  int32_t leaf;             /* leaf size L in 2..64: the tree depth is the smallest t with ceil(n/2^t) <= L */
  int32_t merge_mode;       /* TDC_MERGE_* */
  int32_t structured_min_K; /* STRUCTURED: merges with K >= this use the structured path, smaller ones FP64 */
  int32_t lr_tile;          /* tile size m of the structured path (multiple of 64) */
  double lr_tol;            /* SRRSC stopping tolerance, relative to the tile's largest entry */
  int32_t split_slices;     /* base-256 BF16 digits per operand on the split path (3..7) */
  int32_t split_min_K;      /* SPLIT/AUTO: merges with K >= this use the split path, smaller ones FP64 */
  int32_t max_iter;         /* secular iteration cap per root (>= 1) */
  int32_t sign_normalise;   /* 1: make the largest-magnitude entry of every column positive */
  int32_t collect_stats;    /* 1: record per-level statistics for tdc_get_stats (adds a sync) */
  int64_t spin_budget;      /* bounded-wait iteration cap for persistent kernels */
  int32_t split_chunk_k;    /* SPLIT/AUTO: a positive multiple of 16 (default 256) drains the FP32 level
                               sums into 64-bit running sums every split_chunk_k terms, which bounds
                               them for any order; 0 sums each level over a tile's whole reduction
                               (faster, not exact on smooth eigenvectors) */
} tdc_opts;

#define TDC_MAX_LEVELS 32

typedef struct {
  int32_t levels;                        /* merge levels of the last call */
  int64_t n_merges[TDC_MAX_LEVELS];      /* index 0 = top level */
  int64_t sum_n[TDC_MAX_LEVELS];
  int64_t sum_K[TDC_MAX_LEVELS];         /* non-deflated sizes */
  int64_t max_K[TDC_MAX_LEVELS];
  int64_t n_rot[TDC_MAX_LEVELS];         /* type-2 (rotation) deflations */
  int64_t n_type1[TDC_MAX_LEVELS];       /* type-1 (small z) deflations */
  int64_t secular_iter_max;
  double secular_iter_mean;
  /* CUDA-event times on the call's stream: 0 leaf, 1 prepare+rotate, 2 secular,
   * 3 zhat+norms+order, 4 FP64 GEMM, 5 split digit images, 6 split tensor-core GEMM,
   * 7 deflated copies, 8 output, 9 total */
  float phase_ms[12];
  double gemm_flops[TDC_MAX_LEVELS];     /* algorithmic flops of the Q*U products (2 per multiply-add) */
  double split_flops;                    /* part of gemm_flops computed on the split path */
  double split_bytes;                    /* algorithmic HBM bytes of the split products: digit images
                                            read once (2 B per slice per entry of each operand) and
                                            the FP64 result written once */
  double struct_flops;                   /* flops executed by the structured path (dense near-diagonal
                                            tiles + the two thin products of the low-rank tiles) */
  int64_t launches;                      /* kernel launches of the call */
  int64_t secular_handoffs;              /* roots of small merges whose thread-per-root solve was not
                                            certified in one pass and went to a warp-per-root solve */
  float split_level_max;                 /* largest |level sum| / 2^24 that a hand-off of the split
                                            product's FP32 accumulators held (levels 0-4); the
                                            product is exact while it stays below 1 */
  int64_t lr_tiles;                      /* structured path: off-diagonal tiles compressed by SRRSC */
  int64_t lr_rank_sum;                   /* sum of their ranks (mean rank = lr_rank_sum / (lr_tiles -
                                            lr_dense_fallbacks)) */
  int64_t lr_dense_fallbacks;            /* tiles whose rank exceeded the cap and stayed dense */
  int64_t lr_rank_max;                   /* largest rank kept in low-rank form */
  int64_t lr_parts_structured;           /* TDC_MERGE_STRUCTURED_SPLIT: merge parts (one per half of a
                                            merge) the structured products took */
  int64_t lr_parts_split;                /* ... parts left to the plain split product: a far tile past
                                            the rank cap, or more low-rank columns than its buffer */
} tdc_stats;

/* Fill *o with the defaults (leaf 16, AUTO, structured_min_K 4096, lr_tile 256,
 * lr_tol 1e-15, split_slices 7, split_min_K 128, max_iter 64, sign_normalise 1,
 * collect_stats 0, spin_budget 2^24, split_chunk_k 256). */
void tdc_default_opts(tdc_opts* o);

/* Workspace bytes tdc_eig needs for order n (o may be NULL = defaults).
 * Returns TDC_OK, -1 if n < 0, -2 if the options are invalid. */
int tdc_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes);

/* Eigen-decomposition of one tridiagonal (Algorithm 1 / 3).
 *   n       order (n = 0: nothing is done; n = 1: lam = d, Q = 1)
 *   d[n]    diagonal, e[n-1] off-diagonal (device, FP64, not modified)
 *   lam[n]  eigenvalues, ascending (device, written)
 *   Q       n x n column-major, leading dimension ldq >= max(1, n) (device, written);
 *           T = Q diag(lam) Q^T
 *   ws      device workspace of at least tdc_workspace_size(n) bytes, 256-byte aligned
 *   o       options (NULL = defaults)
 * Errors: -1 n < 0; -2/-3 NULL d/e when n > 0 (e may be NULL when n = 1);
 * -4/-5 NULL lam/Q; -6 ldq < max(1,n); TDC_ENOWS; -9 invalid options; TDC_ECUDA.
 * A non-finite entry of d or e is read as zero (in every problem of a batch alike) and
 * the stream's status records TDC_ENONFINITE: lam and Q are then the finite
 * eigendecomposition of the input with those entries zeroed.  A problem whose largest
 * finite |d|, |e| lies outside [2^-400, 2^400] is solved scaled by the power of two that
 * puts it in [1, 2) (exact), its eigenvalues scaled back (they overflow only where the
 * exact ones exceed the FP64 range); other problems are solved as given. */
int tdc_eig(int64_t n, const double* d, const double* e, double* lam, double* Q, int64_t ldq, void* ws,
            size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream);

/* Workspace for a batch (n_host[batch] on the host). */
int tdc_eig_batched_workspace_size(int32_t batch, const int64_t* n_host, const tdc_opts* o, size_t* bytes);

/* Many independent tridiagonals in one call: problem b has order n_host[b], its
 * diagonal at d + off_de_host[b] and off-diagonal at e + off_de_host[b]
 * (n_b - 1 entries), eigenvalues written to lam + off_de_host[b], eigenvectors to
 * Q + off_q_host[b] with leading dimension n_b.  All merges of one tree level of
 * every problem run in the same launches; the host plan is passed to the device
 * by value inside kernel parameters, so the whole call can be captured in a CUDA
 * graph and replayed (the captured graph reuses the same pointers and sizes).
 * Errors: -1 batch < 0, -2 NULL n_host, -3/-4 NULL offsets, -5..-8 NULL arrays,
 * TDC_ENOWS, -11 invalid options, -1000-b when problem b has n_b < 0. */
int tdc_eig_batched(int32_t batch, const int64_t* n_host, const int64_t* off_de_host, const int64_t* off_q_host,
                    const double* d, const double* e, double* lam, double* Q, void* ws, size_t ws_bytes,
                    const tdc_opts* o, tdc_stream_t stream);

/* tdc_eig for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment convenience.  Some callers cannot call
 * cudaMalloc -- code in a process whose device memory is already fully reserved
 * by another allocator, plugins that must not touch the allocator, and
 * latency-critical paths where an allocation may block or fail -- so they cannot
 * provide tdc_eig's workspace.  This entry point takes the same arguments as
 * tdc_eig minus the workspace and uses instead a fixed 24 MiB array in the
 * library's own device memory (a file-scope __device__ array that every GPU which
 * loads the library holds until the process exits).  That covers orders up to
 * about n = 1730 with the FP64 merge (whatever tdc_workspace_size(n, o) fits in
 * 24 MiB); with merge_mode AUTO the FP64 merge is used whenever the split path's
 * digit images would not fit, and larger n returns TDC_ETOOLARGE before
 * anything is enqueued.  The first call on each
 * device looks the array's device address up (cudaGetSymbolAddress, with that
 * device current), and the first call from each host thread on each device creates
 * that thread's second stream and event pool, so make those first calls before
 * any stream capture.  All
 * calls share the one array and it keeps the last call's contents (nothing in it
 * has to start at zero): calls that overlap on the GPU race on it and must be
 * ordered by the caller.  Allocates nothing; collect_stats is ignored.
 * Errors: as tdc_eig (-1 n < 0, -2..-6 arguments, -7 invalid options),
 * TDC_ETOOLARGE, TDC_ECUDA. */
int tdc_eig_noalloc(int64_t n, const double* d, const double* e, double* lam, double* Q, int64_t ldq,
                    const tdc_opts* o, tdc_stream_t stream);

/* Adjoint of the eigen-decomposition (reverse mode): given lam[n], Q (n x n, ldq)
 * from tdc_eig and the cotangents lam_bar[n] and Q_bar (n x n, ldq; either may be
 * NULL = zero), writes the cotangents of the tridiagonal entries
 *   M = diag(lam_bar) + F o skew(Q^T Q_bar),  F_ij = 1/(lam_j - lam_i) (i != j), F_ii = 0,
 *   d_bar[i] = (Q M Q^T)_{ii},  e_bar[i] = 2 (Q M Q^T)_{i,i+1}.
 * Requires distinct eigenvalues.  ws of tdc_backward_workspace_size(n) bytes. */
int tdc_backward_workspace_size(int64_t n, size_t* bytes);
int tdc_eig_backward(int64_t n, const double* lam, const double* Q, int64_t ldq, const double* lam_bar,
                     const double* Q_bar, double* d_bar, double* e_bar, void* ws, size_t ws_bytes,
                     tdc_stream_t stream);

/* Batched adjoint over `batch` problems of the same order n stored back to back
 * (lam: batch*n, Q and Q_bar: batch*n*n with ld n, d_bar: batch*n, e_bar: batch*(n-1)). */
int tdc_backward_batched_workspace_size(int32_t batch, int64_t n, size_t* bytes);
int tdc_eig_backward_batched(int32_t batch, int64_t n, const double* lam, const double* Q,
                             const double* lam_bar, const double* Q_bar, double* d_bar, double* e_bar,
                             void* ws, size_t ws_bytes, tdc_stream_t stream);

/* Rank-one eigenproblem D + rho z z^T (one merge's secular stage on its own):
 * D[K] strictly ascending, z[K] nonzero, rho > 0.  Writes org[K] (int32: index of
 * the pole the root is measured from, j or j+1), tau[K] (lambda_j = D[org_j] + tau_j),
 * zhat[K] (Loewner recomputation) and s[K] (column normalisers of Eq. (Q_Cauchy)).
 * ws: device scratch of tdc_rank_one_workspace_size(K) bytes (the FP32 copies of the
 * poles for the roots' pre-iteration, about 20 K bytes); smaller or NULL: TDC_ENOWS. */
int tdc_rank_one_workspace_size(int64_t K, size_t* bytes);
int tdc_rank_one(int64_t K, const double* D, const double* z, double rho, int32_t* org, double* tau,
                 double* zhat, double* s, int32_t max_iter, void* ws, size_t ws_bytes, tdc_stream_t stream);

/* Structured product C = A * Qhat with Qhat the K x K Cauchy-like matrix
 * Qhat_ij = zhat_i s_j / ((D_i - D_org_j) - tau_j) given by its generators
 * (Eq. (Q_Cauchy) with Eq. (d-lambda)); A is m x K (lda), C is m x K (ldc).
 * mode: TDC_MERGE_DENSE (FP64); TDC_MERGE_STRUCTURED (Section 2.1: Qhat cut into
 * o->lr_tile square tiles, the tiles on and next to the diagonal multiplied densely
 * in FP64, every other tile replaced by its SRRSC skeleton Qhat(I,T) [I Z] at
 * tolerance o->lr_tol and applied as two thin FP64 products, Z generated from its
 * generators; tiles whose rank would exceed 64 stay dense); or TDC_MERGE_SPLIT
 * (base-256 BF16 digit products on the tensor cores; requires |A_ij| <= 1, which
 * holds for the orthogonal factors the merge multiplies, and uses
 * o->split_slices digits).
 * ws of tdc_cauchy_gemm_workspace_size(m, K, mode, o) bytes. */
int tdc_cauchy_gemm_workspace_size(int64_t m, int64_t K, int32_t mode, const tdc_opts* o, size_t* bytes);
int tdc_cauchy_gemm(int64_t m, int64_t K, const double* A, int64_t lda, const double* D, const int32_t* org,
                    const double* tau, const double* zhat, const double* s, double* C, int64_t ldc, int32_t mode,
                    const tdc_opts* o, void* ws, size_t ws_bytes, tdc_stream_t stream);

/* General Cauchy-like product (Section 4, Example 1): C = A * B for the n x n matrix
 *   B_ij = u_i v_j / (d_i - w_j)
 * given by its generators (device FP64): row nodes d[n] and column nodes w[n], both
 * ascending, with d_i != w_j, and vectors u[n], v[n].  A is m x n (lda), C is m x n
 * (ldc).  B is brought to the form of a merge's Qhat (each column node as the nearest
 * row node plus an offset), so every mode of tdc_cauchy_gemm applies: TDC_MERGE_DENSE
 * (FP64), TDC_MERGE_STRUCTURED (SRRSC low-rank far tiles, FP64), TDC_MERGE_SPLIT (BF16
 * digit products on the tensor cores) and TDC_MERGE_STRUCTURED_SPLIT (the structured
 * products on the split path).  The structured modes assume the row and column nodes
 * interlace (tiles far apart in index are far apart in value), as in Example 1.  For
 * the split modes A and the columns of B are scaled by powers of two (exactly) so that
 * every operand entry is at most 1, and the product is scaled back.
 * ws of tdc_cauchy_like_gemm_workspace_size(m, n, mode, o) bytes.
 * Errors: -1 m, -2 n, -3 A, -4 lda, -5..-8 d, w, u, v, -9 C, -10 ldc, -11 mode,
 * -12 options, TDC_ENOWS, TDC_ECUDA. */
int tdc_cauchy_like_gemm_workspace_size(int64_t m, int64_t n, int32_t mode, const tdc_opts* o, size_t* bytes);
int tdc_cauchy_like_gemm(int64_t m, int64_t n, const double* A, int64_t lda, const double* d, const double* w,
                         const double* u, const double* v, double* C, int64_t ldc, int32_t mode, const tdc_opts* o,
                         void* ws, size_t ws_bytes, tdc_stream_t stream);

/* Rank profile of a Cauchy-like operand (the ranks of Table 2): B of
 * tdc_cauchy_like_gemm cut into o->lr_tile square tiles (T = ceil(n / lr_tile) per
 * dimension); ranks[I * T + J] (device int32, T x T) receives the SRRSC rank at
 * tolerance o->lr_tol of every tile off the diagonal (I != J), -1 when it exceeds the
 * rank cap (64), and 0 on the diagonal.  ws of tdc_cauchy_like_ranks_workspace_size
 * bytes. */
int tdc_cauchy_like_ranks_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes);
int tdc_cauchy_like_ranks(int64_t n, const double* d, const double* w, const double* u, const double* v,
                          const tdc_opts* o, int32_t* ranks, void* ws, size_t ws_bytes, tdc_stream_t stream);

/* Dense symmetric eigenproblems (Section 4, Example 3: each matrix is first reduced to
 * tridiagonal form, then the tridiagonal solver runs on T).
 *
 * tdc_sytrd: Householder reduction A = Q T Q^T of the n x n symmetric A (device FP64,
 * column-major, n <= lda <= 2^27; only the lower triangle is read).  Reflector k = 0 .. n-3 is
 * H_k = I - tau[k] v_k v_k^T with v_k(0:k+1) = 0, v_k(k+1) = 1, mapping column k below the
 * diagonal to a multiple of e_1 (LAPACK's xLARFG convention: beta = -sign(alpha) ||x||);
 * Q = H_0 H_1 ... H_{n-3}.  Outputs: d[n], e[n-1] (T's diagonal and off-diagonal),
 * tau[n-1] (tau[n-2] = 0), and A overwritten: A(k+2:n, k) holds v_k(k+2:n), A(k+1, k) = e[k],
 * A(k, k) = d[k]; the strict upper triangle is scratch.  Computed in FP64 with the
 * trailing rank-2nb updates as split-precision tensor-core products (base-256 BF16
 * digits, exact level sums): backward error of the order of FP64 rounding times ||A||.
 * ws of tdc_sytrd_workspace_size(n) bytes.  Errors: -1 n, -2 A, -3 lda, -4 d, -5 e,
 * -6 tau, -9 options (spin_budget and split_chunk_k are used), TDC_ENOWS, TDC_ECUDA;
 * device status TDC_ETIMEOUT if a grid barrier of the panel kernel gave up. */
int tdc_sytrd_workspace_size(int64_t n, size_t* bytes);
int tdc_sytrd(int64_t n, double* A, int64_t lda, double* d, double* e, double* tau, void* ws, size_t ws_bytes,
              const tdc_opts* o, tdc_stream_t stream);

/* tdc_ormtr: X <- Q X for the Q of tdc_sytrd (A and tau as tdc_sytrd left them), X n x ncols
 * (ldx >= n, device FP64), in place.  Blocks of 128 reflectors in compact WY form, applied
 * from the last block back as split-precision products (X's columns enter scaled by powers
 * of two from their norms, which the orthogonal updates keep).  ws of
 * tdc_ormtr_workspace_size(n, ncols) bytes.  Errors: -1 n, -2 ncols, -3 A, -4 lda, -5 tau,
 * -6 X, -7 ldx, -10 options, TDC_ENOWS, TDC_ECUDA. */
int tdc_ormtr_workspace_size(int64_t n, int64_t ncols, size_t* bytes);
int tdc_ormtr(int64_t n, int64_t ncols, const double* A, int64_t lda, const double* tau, double* X, int64_t ldx,
              void* ws, size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream);

/* tdc_syevd: A = Z diag(lam) Z^T for the dense symmetric A (lower triangle read, A
 * destroyed): tdc_sytrd, tdc_eig on (d, e) with the options o, tdc_ormtr on the
 * eigenvectors.  lam[n] ascending, Z n x n (ldz >= n).  One status for the whole call.
 * A whose largest finite |entry| lies outside [2^-400, 2^400] is scaled in place by the
 * power of two that puts it in [1, 2) before the reduction (exact), and lam scaled back.
 * ws of tdc_syevd_workspace_size(n, o) bytes.  Errors: -1 n, -2 A, -3 lda, -4 lam, -5 Z,
 * -6 ldz, -9 options, TDC_ENOWS, TDC_ECUDA, or those of the steps. */
int tdc_syevd_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes);
int tdc_syevd(int64_t n, double* A, int64_t lda, double* lam, double* Z, int64_t ldz, void* ws, size_t ws_bytes,
              const tdc_opts* o, tdc_stream_t stream);

/* Products with a structured operand given by generators (the further structured
 * matrices of Sections 1, 3.1 and 5, given by O(n) parameters): C = A * B, A m x n (lda),
 * C m x n (ldc), the n x n B generated from t (device FP64):
 *   TDC_TOEPLITZ     B(k, j) = t[k - j + n - 1], t[2n-1] (t[n-1+i] on the i-th
 *                    subdiagonal, t[n-1-i] on the i-th superdiagonal)
 *   TDC_HANKEL       B(k, j) = t[k + j], t[2n-1]
 *   TDC_VANDERMONDE  B(k, j) = t[k]^j, the n nodes t[n] (powers by repeated squaring;
 *                    max|t|^(n-1) must stay below 2^1000)
 * B never exists in memory: the FP64 tiles (TDC_MERGE_DENSE) and the split product's digit
 * images (TDC_MERGE_SPLIT, o->split_slices digits; A and each column of B scaled by powers
 * of two so that every operand entry is at most 1, the product scaled back) generate it.
 * ws of tdc_structured_gemm_workspace_size(m, n, mode, o) bytes.  Errors: -1 m, -2 n, -3 A,
 * -4 lda, -5 kind, -6 t, -7 C, -8 ldc, -9 mode, -10 options, TDC_ENOWS, TDC_ECUDA. */
#define TDC_TOEPLITZ 1
#define TDC_HANKEL 2
#define TDC_VANDERMONDE 3
int tdc_structured_gemm_workspace_size(int64_t m, int64_t n, int32_t mode, const tdc_opts* o, size_t* bytes);
int tdc_structured_gemm(int64_t m, int64_t n, const double* A, int64_t lda, int32_t kind, const double* t, double* C,
                        int64_t ldc, int32_t mode, const tdc_opts* o, void* ws, size_t ws_bytes,
                        tdc_stream_t stream);

/* tdc_dft_gemm: C = A F with F the DFT matrix of order n, F(k, j) = exp(-2 pi i k j / n), for
 * a real A (m x n, lda): Cre = A Re(F), Cim = A Im(F) (m x n each, ldc), the two real
 * operands cos(2 pi m / n) and -sin(2 pi m / n) generated from n-entry tables at
 * m = (k j) mod n.  Modes and workspace as tdc_structured_gemm (ws of
 * tdc_dft_gemm_workspace_size bytes).  Errors: -1 m, -2 n, -3 A, -4 lda, -5 Cre, -6 Cim,
 * -7 ldc, -8 mode, -9 options, TDC_ENOWS, TDC_ECUDA. */
int tdc_dft_gemm_workspace_size(int64_t m, int64_t n, int32_t mode, const tdc_opts* o, size_t* bytes);
int tdc_dft_gemm(int64_t m, int64_t n, const double* A, int64_t lda, double* Cre, double* Cim, int64_t ldc,
                 int32_t mode, const tdc_opts* o, void* ws, size_t ws_bytes, tdc_stream_t stream);

/* tdc_sbevd: A = Q diag(lam) Q^T for the n x n symmetric band matrix of bandwidth b
 * (0 <= b < n, b <= 64) in LAPACK's lower band storage: AB(i - j, j) = A(i, j) for
 * j <= i <= min(n - 1, j + b), AB column-major with ldab >= b + 1 (device FP64, not
 * modified).  Divide and conquer for band matrices (Section 5's band case): a node splits
 * at its middle; the b x b coupling block, row k being B_k, is written as
 * sum_k (x_k; y_k)(x_k; y_k)^T with x_k = s_k e, y_k = B_k / s_k, s_k = sqrt(||B_k||), and
 * subtracted from the two halves' corners; leaves of at most max(128, 8b) rows are solved
 * densely, as one batch (a block per leaf reduces it to tridiagonal form and
 * back-transforms, tdc_eig_batched solves the tridiagonals); a merge takes the b terms in turn as rank-one
 * modifications D + z z^T with z = Q^T (x_k; y_k): sort, deflation (Section 3.2's two
 * tests), the secular equation, the Cauchy-like update of the non-deflated columns (split
 * tensor-core product from K = 128 on).  A band whose largest finite |entry| lies
 * outside [2^-400, 2^400] is solved scaled by the power of two that puts it in [1, 2)
 * (exact; AB itself is not modified) and lam scaled back.  lam[n] ascending, Q n x n
 * (ldq >= n).  The call
 * reads each rank-one step's deflation count back to the host, so it returns when the
 * solve is done.  ws of tdc_sbevd_workspace_size(n, b, o) bytes.  Errors: -1 n, -2 b,
 * -3 AB, -4 ldab, -5 lam, -6 Q, -7 ldq, -10 options, TDC_ENOWS, TDC_ECUDA, or those of
 * the steps. */
int tdc_sbevd_workspace_size(int64_t n, int64_t b, const tdc_opts* o, size_t* bytes);
int tdc_sbevd(int64_t n, int64_t b, const double* AB, int64_t ldab, double* lam, double* Q, int64_t ldq, void* ws,
              size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream);

/* tdc_bdsdc: SVD B = U diag(sigma) VT of the n x n upper bidiagonal B (diagonal d[n],
 * superdiagonal e[n-1], device FP64, not modified) through the divide and conquer (the
 * paper's introduction points to it for the bidiagonal SVD): tdc_eig on the Golub-Kahan
 * tridiagonal of order 2n (zero diagonal, off-diagonal d_1, e_1, d_2, ..., e_{n-1}, d_n),
 * whose eigenvalues are +-sigma_i and whose eigenvector of +sigma_i is
 * (v_1, u_1, ..., v_n, u_n) / sqrt(2).  sigma[n] descending; U (ldu >= n) holds the left
 * singular vectors as columns, VT (ldvt >= n) the right ones as rows.  Singular values and
 * the residuals B V - U Sigma, B^T U - V Sigma are accurate to FP64 rounding times ||B||;
 * the singular vectors of sigma_i hold to about eps ||B|| / sigma_i (the pair +-sigma_i of
 * the Golub-Kahan matrix is 2 sigma_i apart), so orthogonality degrades by ||B|| / sigma_min
 * for ill-conditioned B, and an exactly singular B is not supported.  ws of
 * tdc_bdsdc_workspace_size(n, o) bytes (the order-2n eigensolve and its 4 n^2 matrix).
 * Errors: -1 n, -2 d, -3 e, -4 sigma, -5 U, -6 ldu, -7 VT, -8 ldvt, -11 options, TDC_ENOWS,
 * TDC_ECUDA, or those of tdc_eig. */
int tdc_bdsdc_workspace_size(int64_t n, const tdc_opts* o, size_t* bytes);
int tdc_bdsdc(int64_t n, const double* d, const double* e, double* sigma, double* U, int64_t ldu, double* VT,
              int64_t ldvt, void* ws, size_t ws_bytes, const tdc_opts* o, tdc_stream_t stream);

/* Synchronise `stream` and return the device status of the last call enqueued on it
 * (TDC_OK, TDC_ENOCONV, TDC_ETIMEOUT, TDC_ENONFINITE, TDC_EUNSUPPORTED, or the warning
 * TDC_WPRECISION), then clear it.  Each stream that calls the library gets its own
 * status slot (two words in a fixed device array of the library, assigned on the
 * stream's first call; beyond 1024 streams per device the later ones share the last
 * slot).  A call clears its stream's slot when it is enqueued, so calls on different
 * streams never see or clear each other's status, and the status outlives the call's
 * workspace.  A stream that no call was enqueued on (for example one a captured
 * graph is replayed on) reports the slot of the last call made on the device. */
int tdc_sync_status(tdc_stream_t stream);

/* Copy the statistics of the last call made with collect_stats = 1. */
int tdc_get_stats(tdc_stats* out);

/* Static text for a status code. */
const char* tdc_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* TDC_H */
