/*
 * cpinv -- Moore-Penrose inverse by full-rank Cholesky factorisation, on one
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Method (P. Courrieu, "Fast Computation of Moore-Penrose Inverse Matrices"):
 *   Sec. 1       G+ is the unique n x m matrix satisfying the four Penrose
 *                conditions; W = G+ F solves min |G W - F|^2 with minimum norm.
 *   Sec. 2 Eq.(1) G'G = L L', L (n x r) of full column rank r.
 *   Theorem 1    G+ = L (L'L)^-1 (L'L)^-1 L' G'.
 *   Appendix     A = G'G (A = G G' and a transposed result when m < n);
 *                tol = rel_tol * min{A_jj : A_jj > 0}; full-rank Cholesky in
 *                natural column order keeping column k iff its updated pivot
 *                is > tol; M = inv(L'L); G+ = L M M L' G'.
 *
 * Conventions for every entry point below:
 *   - Matrices are dense, ROW-MAJOR, FP64, with an explicit leading dimension
 *     (elements between the starts of two consecutive rows), ld >= #columns.
 *   - Every matrix pointer is a DEVICE pointer (cudaMalloc'd or equivalent)
 *     on the current CUDA device.  The caller owns all buffers; the library
 *     never frees or keeps them past the call.
 *   - `workspace` is a device buffer of at least the size returned by the
 *     matching *_workspace_size function, aligned to 256 bytes; the call
 *     uses it as scratch and keeps nothing in it.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued on it.  If `rank_out` is non-NULL the call synchronizes that
 *     stream, writes the numerical rank r to *rank_out and returns the status
 *     the kernels recorded (non-finite input, failed inverse); if it is NULL
 *     the call returns after enqueueing, and only argument errors are
 *     reported.
 *   - Return value: a CPINV_* status.  On error the outputs are unspecified
 *     and *rank_out (if given) is -1.
 *   - m = 0 or n = 0 gives an empty result and r = 0.  A G with no positive
 *     diagonal entry in its Gram matrix (e.g. G = 0) gives G+ = 0 and r = 0,
 *     like the Appendix listing (min over an empty set makes every test false).
 *   - The library keeps per-device state for the life of the process (its
 *     streams, events, captured CUDA graphs and constant tables), all in the
 *     device's primary context: do not reset the device (cudaDeviceReset)
 *     between calls.
 */
#ifndef CPINV_H
#define CPINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CPINV_OK                  0
#define CPINV_ERR_INVALID_ARG     1  /* NULL pointer, negative size, ld too small, bad option */
#define CPINV_ERR_NONFINITE_INPUT 2  /* G holds a NaN or an Inf */
#define CPINV_ERR_WORKSPACE       3  /* workspace NULL, misaligned or too small */
#define CPINV_ERR_CUDA            4  /* a CUDA runtime call failed */
#define CPINV_ERR_NUMERICAL       5  /* L'L was not positive definite in FP64 */
#define CPINV_ERR_UNSUPPORTED     6  /* mode or size not supported by this build */
#define CPINV_ERR_TIMEOUT         7  /* a bounded device-side wait expired (kernels exited early) */

/* Arithmetic of the dense contractions (Gram, L'L, inverse, chain).
 * The pivot decisions, square roots and the small diagonal-block solves are
 * FP64 in every mode. */
#define CPINV_MODE_FP64         0  /* FP64 fused multiply-add everywhere */
#define CPINV_MODE_EXACT_SLICE  1  /* tcgen05 BF16 tensor cores on integer slices of the
                                      FP64 operands with exact FP32/INT32 sums
                                      (Ozaki scheme), FP64-accurate products */
#define CPINV_MODE_SPLIT_BF16X3 2  /* tcgen05 BF16 tensor cores, hi/lo split, three
                                      products accumulated in FP32 (reduced accuracy) */

typedef struct cpinv_opts {
  int32_t mode;      /* CPINV_MODE_* (default CPINV_MODE_FP64) */
  int32_t slices;    /* reserved for the exact-slice mode, ignored: that mode
                        picks its moduli count itself from the inner dimension
                        and the operands' integer width (62 bits for the Gram
                        matrix, 60 for the factorisation, 53 for the other
                        products); any value is accepted */
  int32_t panel;     /* Cholesky panel width: 1, 2, 4, 8, 16 or 32; 0 = default (32) */
  int32_t reserved;  /* must be 0 */
  double rel_tol;    /* pivot threshold factor; default 1e-9 (Appendix) */
} cpinv_opts;

/* Fills *o with the defaults (FP64 mode, rel_tol = 1e-9). */
void cpinv_default_opts(cpinv_opts* o);

/* Human-readable name of a status code (static string). */
const char* cpinv_status_string(int status);

/* Library version, as major*10000 + minor*100 + patch. */
int cpinv_version(void);

/* ---------------------------------------------------------------------------
 * Moore-Penrose inverse (Theorem 1, Appendix `geninv`).
 *   G   : m x n, row-major, leading dimension ldg >= n.
 *   Gp  : n x m output G+, row-major, leading dimension ldgp >= m.
 * For m < n the Appendix's transposed branch is taken (A = G G', m x m).
 * ------------------------------------------------------------------------- */
size_t cpinv_pinv_workspace_size(int64_t m, int64_t n, const cpinv_opts* o);
int cpinv_pinv(const double* G, int64_t m, int64_t n, int64_t ldg,
               double* Gp, int64_t ldgp,
               void* workspace, size_t workspace_bytes,
               const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * Minimum-norm least squares W = G+ F (Sec. 1; the printed "W = G+ W" is
 * read as W = G+ F).  G+ is never formed: W = L (M (M (L' (G'F)))).
 *   F : m x k, row-major, ldf >= k.     W : n x k output, ldw >= k.
 * ------------------------------------------------------------------------- */
size_t cpinv_lstsq_workspace_size(int64_t m, int64_t n, int64_t k, const cpinv_opts* o);
int cpinv_lstsq(const double* G, int64_t m, int64_t n, int64_t ldg,
                const double* F, int64_t k, int64_t ldf,
                double* W, int64_t ldw,
                void* workspace, size_t workspace_bytes,
                const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * Least squares from accumulated normal equations (incremental learning,
 * Sec. 4: the network is trained as data arrive).  The method (Appendix,
 * Theorem 1) needs G only through A = G'G and B = G'F:
 *   W = L (L'L)^-1 (L'L)^-1 L' B,   L the full-rank Cholesky factor of A,
 * so blocks of rows G_i, F_i can be folded in one at a time.
 *
 * cpinv_gram_update: A += G'G (lower triangle written; the upper one is not
 *   read by the solver) and, if F != NULL, B += G'F, in the arithmetic of
 *   `mode` (exact-slice: each increment correctly rounded, then added in
 *   FP64).  G: m x n, F: m x k, A: n x n (lda >= n), B: n x k (ldb >= k);
 *   device pointers; workspace cpinv_gram_update_workspace_size(m, n, k,
 *   mode) bytes, 256-byte aligned.  Enqueues only.
 * cpinv_lstsq_gram: W (n x k) from A (lower triangle) and B, with the
 *   Appendix tolerance taken over A's diagonal; rank_out as for cpinv_lstsq.
 *   Equals cpinv_lstsq(G, F) when A and B were accumulated from all rows of
 *   G and F (up to the roundings of the accumulation).
 * ------------------------------------------------------------------------- */
size_t cpinv_gram_update_workspace_size(int64_t m, int64_t n, int64_t k, int32_t mode);
int cpinv_gram_update(const double* G, int64_t m, int64_t n, int64_t ldg,
                      const double* F, int64_t k, int64_t ldf,
                      double* A, int64_t lda, double* B, int64_t ldb,
                      int32_t mode, void* workspace, size_t workspace_bytes, void* stream);
size_t cpinv_lstsq_gram_workspace_size(int64_t n, int64_t k, const cpinv_opts* o);
int cpinv_lstsq_gram(const double* A, int64_t n, int64_t lda, const double* B, int64_t k,
                     int64_t ldb, double* W, int64_t ldw,
                     void* workspace, size_t workspace_bytes,
                     const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * Gaussian radial-basis design matrices (Sec. 1 and Sec. 4: an RBF network's
 * output weights are W = G+ F for the design matrix G of its hidden layer):
 *   G_ij = exp(-|x_i - c_j|^2 / (2 w^2)),
 * the squared distance summed over the d coordinates in order (FP64, fused
 * multiply-adds), the exponential in FP64.
 *   X : m x d data (row-major, ldx >= d), C : n x d centres (ldc >= d),
 *   width w > 0 and finite, 0 <= d <= CPINV_RBF_MAX_D (else
 *   CPINV_ERR_UNSUPPORTED).  Device pointers.
 * cpinv_rbf_design: G (m x n, ldg >= n) written to device memory.  Enqueues
 *   only (non-finite X or C give non-finite G).
 * cpinv_rbf_normal_equations: the normal equations of W = G+ F without G
 *   in memory: A = G'G (n x n, lower triangle written, lda >= n) and, if F !=
 *   NULL, B = G'F (n x k, ldb >= k; F m x k, ldf >= k), in the exact-slice
 *   arithmetic (each chunk of at most 4096 rows of X summed exactly and
 *   rounded once, chunks added in FP64 -- as cpinv_gram_update in that mode).
 *   Each tile of G is generated in FP64 and cut into the tensor-core residue
 *   planes directly.  Solve with cpinv_lstsq_gram.  Workspace:
 *   cpinv_rbf_normal_equations_workspace_size(m, n, d, k) bytes, 256-byte
 *   aligned.  `check` != 0 synchronizes the stream and reports
 *   CPINV_ERR_NONFINITE_INPUT (NaN/Inf in X or C) and CPINV_ERR_NUMERICAL
 *   (the per-centre scale bound did not cover an entry; not expected);
 *   with check = 0 the call only enqueues.
 * ------------------------------------------------------------------------- */
#define CPINV_RBF_MAX_D 32
int cpinv_rbf_design(const double* X, int64_t m, int64_t d, int64_t ldx,
                     const double* C, int64_t n, int64_t ldc, double width,
                     double* G, int64_t ldg, void* stream);
size_t cpinv_rbf_normal_equations_workspace_size(int64_t m, int64_t n, int64_t d, int64_t k);
int cpinv_rbf_normal_equations(const double* X, int64_t m, int64_t d, int64_t ldx,
                               const double* C, int64_t n, int64_t ldc, double width,
                               const double* F, int64_t k, int64_t ldf,
                               double* A, int64_t lda, double* B, int64_t ldb,
                               void* workspace, size_t workspace_bytes, int32_t check,
                               void* stream);

/* ---------------------------------------------------------------------------
 * Failure path of the device-side waits, exercised without a fault: one
 * thread runs the bounded wait of the factorisation kernels on a counter that
 * nothing advances (workspace: >= 128 bytes of device memory, overwritten),
 * so the wait gives up after about a second and records the timeout.
 * Returns CPINV_ERR_TIMEOUT when the wait expired as designed (the expected
 * result; the context stays usable), CPINV_OK if it did not, CPINV_ERR_CUDA
 * or CPINV_ERR_INVALID_ARG otherwise.  Synchronises the stream.
 * ------------------------------------------------------------------------- */
int cpinv_selftest_wait_timeout(void* workspace, size_t workspace_bytes, void* stream);

/* The same for the batched path's queue-fed factorisation: one task whose
 * input no task produces (workspace: >= 64 KiB of device memory, 256-byte
 * aligned, overwritten).  Its bounded wait gives up after about a second,
 * records the timeout and raises the launch's abort flag.  Returns
 * CPINV_ERR_TIMEOUT when that happened (expected), CPINV_OK if not. */
int cpinv_selftest_queue_timeout(void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Adjoint of the least-squares weights (reverse mode): given the cotangent
 * Wbar = dL/dW (n x k) of a scalar L of W = G+ F, returns
 *   dG = dL/dG (m x n)  and, if dF != NULL, dF = dL/dF (m x k),
 * the derivative of the function the Appendix computes with the kept-pivot
 * set S held fixed (the rank decision is piecewise constant).  Steps: the
 * chain of Theorem 1 reversed, the inverse of L'L, the full-rank Cholesky
 * (kept rows: Cholesky adjoint; rejected rows: triangular solve, on the
 * factor's structural pattern), and the Gram matrix A = G'G.  On inputs of
 * exact rank whose rejected columns all follow the kept ones this equals
 * the Golub-Pereyra derivative of G+.  The forward factors are recomputed
 * (no state is kept between calls); W (if non-NULL) receives G+ F.
 * Requires m >= n (else CPINV_ERR_UNSUPPORTED).  Arithmetic per opts->mode
 * as for cpinv_lstsq.
 *   dW : n x k, ld lddw >= k.  dG : m x n, ld lddg >= n.
 *   dF : m x k, ld lddf >= k, or NULL.  W : n x k, ld ldw >= k, or NULL.
 * ------------------------------------------------------------------------- */
size_t cpinv_lstsq_backward_workspace_size(int64_t m, int64_t n, int64_t k,
                                           const cpinv_opts* o);
int cpinv_lstsq_backward(const double* G, int64_t m, int64_t n, int64_t ldg,
                         const double* F, int64_t k, int64_t ldf,
                         const double* dW, int64_t lddw,
                         double* dG, int64_t lddg, double* dF, int64_t lddf,
                         double* W, int64_t ldw,
                         void* workspace, size_t workspace_bytes,
                         const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * The same adjoint without recomputing the forward pass (training loops:
 * the forward W = G+ F and the reverse pass share the factors).
 * cpinv_lstsq_forward: W = G+ F as cpinv_lstsq, and leaves the forward
 *   factors -- L, M = (L'L)^-1, the kept-pivot mask and index, the rank --
 *   in `state`, a caller-owned device buffer of cpinv_lstsq_state_size(m,
 *   n, k, o) bytes (256-byte aligned).  Requires m >= n and m, n, k >= 1
 *   (else CPINV_ERR_UNSUPPORTED).
 * cpinv_lstsq_backward_from_state: dG (and dF if non-NULL) for the
 *   cotangent dW, as cpinv_lstsq_backward, reading the factors from
 *   `state` instead of factoring again.  G, F, the sizes, the options and
 *   the state must be those of the forward call, and the state must not
 *   have been touched since (the call reads and overwrites its scratch part,
 *   so one forward serves one reverse pass).
 * ------------------------------------------------------------------------- */
size_t cpinv_lstsq_state_size(int64_t m, int64_t n, int64_t k, const cpinv_opts* o);
int cpinv_lstsq_forward(const double* G, int64_t m, int64_t n, int64_t ldg,
                        const double* F, int64_t k, int64_t ldf,
                        double* W, int64_t ldw, void* state, size_t state_bytes,
                        const cpinv_opts* o, int64_t* rank_out, void* stream);
int cpinv_lstsq_backward_from_state(const double* G, int64_t m, int64_t n, int64_t ldg,
                                    const double* F, int64_t k, int64_t ldf,
                                    const double* dW, int64_t lddw,
                                    double* dG, int64_t lddg, double* dF, int64_t lddf,
                                    void* state, size_t state_bytes,
                                    const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * Batched least squares/* ---------------------------------------------------------------------------
 * Batched least squares: W_p = G_p+ F_p for P independent problems of
 * uneven size (Theorem 1 and the Appendix applied to each problem on its
 * own, with its own tolerance and rank), all enqueued on `stream` as one
 * batch.  Problems are grouped by n (rounded up to 128); every stage is one
 * launch per group.  Arithmetic: CPINV_MODE_FP64, or CPINV_MODE_EXACT_SLICE,
 * in which the Gram matrices G_p'G_p, the products L_p'L_p and the inverses
 * (L_p'L_p)^-1 = W_p'W_p of a group are one block-diagonal tensor-core
 * residue product each (every entry the exact sum rounded once; requires
 * m <= 4096) and the rest is FP64.
 *   probs : HOST array of P descriptors; G, F, W in each are DEVICE pointers
 *           (row-major, as for cpinv_lstsq).  Requires 1 <= n <= m,
 *           n <= CPINV_BATCHED_MAX_N, 1 <= k <= CPINV_BATCHED_MAX_K,
 *           m <= CPINV_BATCHED_MAX_M (else CPINV_ERR_UNSUPPORTED).
 *   o     : mode CPINV_MODE_FP64 or CPINV_MODE_EXACT_SLICE (else
 *           CPINV_ERR_UNSUPPORTED); panel 0 (chosen by timing the candidates
 *           on the first call of each group shape), 16 or 32; in the
 *           exact-slice mode the residue products' tile width (128 or 256
 *           columns) is tuned the same way.  Set CPINV_TUNE_FILE to a path to
 *           keep the choices as JSON lines.  rel_tol as for cpinv_lstsq.
 *   ranks_out, status_out : HOST arrays of P entries, or NULL.  If either
 *           is non-NULL the call synchronizes `stream` and writes each
 *           problem's rank r_p (-1 on failure) and CPINV_* status; the
 *           return value is then the first non-OK problem status (or OK).
 *           With both NULL the call returns after enqueueing.
 *   workspace : cpinv_lstsq_batched_workspace_size(P, probs, o) bytes (0 on
 *           invalid arguments), 256-byte aligned, on the current device.
 * A second call with identical arguments (same pointers, sizes, workspace
 * and options) replays the whole batch as one CUDA graph.  The workspace and
 * the descriptors' buffers must stay valid until the stream reaches the end
 * of the batch.
 * ------------------------------------------------------------------------- */
#define CPINV_BATCHED_MAX_N 512
#define CPINV_BATCHED_MAX_K 256
#define CPINV_BATCHED_MAX_M 1048576

typedef struct cpinv_problem {
  int64_t m, n, k;   /* G is m x n, F is m x k, W is n x k */
  const double* G;
  int64_t ldg;
  const double* F;
  int64_t ldf;
  double* W;
  int64_t ldw;
} cpinv_problem;

size_t cpinv_lstsq_batched_workspace_size(int32_t P, const cpinv_problem* probs,
                                          const cpinv_opts* o);
int cpinv_lstsq_batched(int32_t P, const cpinv_problem* probs, int64_t* ranks_out,
                        int32_t* status_out, void* workspace, size_t workspace_bytes,
                        const cpinv_opts* o, void* stream);

/* ---------------------------------------------------------------------------
 * Numerical rank and kept-pivot mask (Appendix: tol rule and full-rank
 * Cholesky).  accepted_out (device, may be NULL) receives one byte per
 * column of the factored Gram matrix -- min(m, n) bytes: columns of G when
 * m >= n, rows of G when m < n -- 1 if that pivot was kept, else 0.
 * ------------------------------------------------------------------------- */
size_t cpinv_rank_workspace_size(int64_t m, int64_t n, const cpinv_opts* o);
int cpinv_rank(const double* G, int64_t m, int64_t n, int64_t ldg,
               uint8_t* accepted_out,
               void* workspace, size_t workspace_bytes,
               const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * The dense contraction of the library on its own:
 *   C = alpha op(A) op(B) + beta C,   op(X) = X or X' (transX != 0),
 * op(A) M x K, op(B) K x N, C M x N, all row-major FP64 device matrices;
 * C must not overlap A or B.
 * This is the product the pipeline uses for G'G, L'L, the inverse and the
 * chain (Theorem 1); exposed for callers who want the same arithmetic.
 *   mode CPINV_MODE_FP64: FP64 fused multiply-adds.
 *   mode CPINV_MODE_EXACT_SLICE: each row of op(A) and column of op(B) is
 *     scaled by a power of two and rounded to a signed integer of `bits`
 *     bits (1..62, 0 = 53); the integer products are computed exactly by
 *     residue arithmetic on the BF16 tensor cores and each entry of the result
 *     is rounded once to FP64 (when K > 4096, per 4096-wide chunk of K).
 * Workspace: cpinv_matmul_workspace_size(M, N, K, mode, bits, symmetric)
 * bytes, 256-byte aligned (`symmetric` != 0 if B == A and op(B) = op(A)').
 * `check` != 0 synchronizes the stream and reports device-side errors
 * (non-finite input, timeout).
 * ------------------------------------------------------------------------- */
size_t cpinv_matmul_workspace_size(int64_t M, int64_t N, int64_t K, int32_t mode,
                                   int32_t bits, int32_t symmetric);
int cpinv_matmul(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, double* C, int64_t ldc, int32_t mode, int32_t bits,
                 void* workspace, size_t workspace_bytes, int32_t check, void* stream);

/* ---------------------------------------------------------------------------
 * Allocation-free pseudoinverse of small matrices.  The paper has no
 * counterpart to this entry point; it serves callers that cannot allocate
 * device memory at all -- for instance a real-time loop where cudaMalloc or
 * cudaFree would block the host or synchronize the device, or a plugin inside
 * a host application that owns all GPU memory and offers no allocator.
 *
 * Same computation, arguments and results as cpinv_pinv, minus the workspace:
 * the scratch is a fixed array of CPINV_STATIC_SCRATCH_BYTES (1 MiB) compiled
 * into the library as device memory, which every GPU that loads the library
 * keeps until the process exits.  No cudaMalloc, cudaFree or other allocating
 * routine is called.
 *   Limit: min(m, n) <= CPINV_STATIC_MAX_ORDER (128) and a workspace that fits
 *          in the array (cpinv_pinv_workspace_size(m, n, o) <= 1 MiB); larger
 *          requests return CPINV_ERR_UNSUPPORTED before any GPU work.  In
 *          practice that means CPINV_MODE_FP64: it fits for every order up
 *          to 128 and every panel width.  CPINV_MODE_EXACT_SLICE never fits
 *          (the residue buffers of its tensor-core Gram product alone exceed
 *          1 MiB, even for a 40 x 20 input) and CPINV_MODE_SPLIT_BF16X3 fits
 *          only for orders of about 32 and below; both are refused with
 *          CPINV_ERR_UNSUPPORTED when they do not fit.
 *   Set-up: the first call on each device looks up the array's device address
 *          (cudaGetSymbolAddress) with that device current and keeps it for
 *          later calls on that device; make that first call before any stream
 *          capture begins.  The address belongs to the device's context: do
 *          not reset the device (cudaDeviceReset) between calls in one
 *          process, or later calls would launch kernels on a stale address.
 *   Sharing: all calls on a device use the same array, which keeps whatever
 *          the last call left in it (each call clears the state it needs).
 *          Calls that overlap on the GPU -- on different streams, or from
 *          several host threads -- race on the array and give wrong results;
 *          order them on one stream or serialize them.
 * ------------------------------------------------------------------------- */
#define CPINV_STATIC_SCRATCH_BYTES (1u << 20)
#define CPINV_STATIC_MAX_ORDER 128
int cpinv_pinv_static(const double* G, int64_t m, int64_t n, int64_t ldg,
                      double* Gp, int64_t ldgp,
                      const cpinv_opts* o, int64_t* rank_out, void* stream);

/* ---------------------------------------------------------------------------
 * Tracing.  When enabled, every kernel the library launches is bracketed by
 * two CUDA events recorded on the stream it is launched on; reading the
 * profile synchronizes the device and returns, per kernel class, the number
 * of launches, the summed event-to-event device time and the algorithmic
 * floating-point operations of those launches (a symmetric product that
 * computes one triangle counts n(n+1)K, a full one 2MNK).  Off by default;
 * the records are process-global and not thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct cpinv_profile_entry {
  char name[32];     /* kernel class: "gemm_fp64", "gemm_slice", "diag_factor", "aux", ... */
  int64_t launches;
  double ms;         /* summed device time of those launches */
  double flops;      /* algorithmic flops (0 for non-contractions) */
} cpinv_profile_entry;

/* Enables (on != 0) or disables tracing and clears the records.  Returns the
 * previous state. */
int cpinv_profile_enable(int on);
/* Writes up to max_entries classes to out, returns how many classes there
 * are (may exceed max_entries), and clears the records.  Returns -1 on a CUDA
 * error. */
int cpinv_profile_read(cpinv_profile_entry* out, int max_entries);
/* The same records as a timeline, without clearing them: for each traced
 * launch in launch order, its kernel class and the device times (ms) of its
 * two events relative to the first record's start.  Writes up to
 * max_entries, returns the number of records (or -1 on a CUDA error).  Call
 * it before cpinv_profile_read. */
typedef struct cpinv_timeline_entry {
  char name[32];     /* kernel class, as in cpinv_profile_entry */
  double start_ms;
  double end_ms;
} cpinv_timeline_entry;
int cpinv_profile_timeline(cpinv_timeline_entry* out, int max_entries);
/* Number of kernels the library has launched in this process. */
int64_t cpinv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* CPINV_H */
