/*
 * rrf.h -- C ABI of the GB300 (sm_103a) randomized rank-revealing factorization library.
 *
 * Computes A = U T V^T (Sec. 1.1, Eq. (1)) for a real m x n matrix A with m >= n, where U (m x m) and
 * V (n x n) are orthogonal and T (m x n) is upper trapezoidal, by one of the paper's two methods:
 *   rrf_randutv  -- blocked randUTV_basic (Algorithm 3; Sec. 4.1);
 *   rrf_powerurv -- powerURV (Algorithm 1; Sec. 3.2).
 * For m < n both factor A^T instead and transpose the result (Sec. 1.3 footnote): with A^T = U' T' V'^T
 * they return U = V' (m x m), T = T'^T (m x n, LOWER trapezoidal: zero above the diagonal; for randUTV
 * with diagonal b x b blocks) and V = U' (n x n), so A = U T V^T still holds.  The workspace query covers
 * A^T and T'; the status word stays at the start of the workspace.
 *
 * Common conventions (every entry point):
 *  - Matrices are column-major FP64 with an explicit leading dimension (ld >= rows).  Unless an entry
 *    point says "host", every matrix pointer is a DEVICE pointer owned by the caller.
 *  - A is read-only.  U, T and V are written completely (every entry of the m x m, m x n and n x n
 *    blocks).  The output buffers must not alias A or each other, with one exception: rrf_randutv
 *    (device and host forms) accepts T == A with ldt == lda and then factors in place (A is
 *    overwritten by T); so does rrf_powerurv for m < n, which consumes A into A^T first.  For m >= n
 *    rrf_powerurv rejects T == A (it reads A after writing T).
 *  - The Gaussian matrices the methods draw (randn in Algorithms 1 and 3) come from the
 *    counter-based Philox-4x32-10 stream (Salmon et al., SC'11) with key = (seed lo32, seed hi32).
 *    Block t of a draw uses counter (t lo32, t hi32, step, tag) and yields column-major elements
 *    2t and 2t+1 by the Box-Muller transform u1 = ((x0:x1 >> 11) + 1) 2^-53, u2 = (x2:x3 >> 11) 2^-53,
 *    z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).  randUTV step i (1-based) draws
 *    (m - b(i-1)) x b with tag 1; powerURV draws n x n with step 0, tag 2.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  Device-side
 *    entry points only enqueue work and return; results are valid once the stream reaches them.
 *  - `workspace` is caller-owned device memory of at least the size the matching *_workspace query
 *    returns, 256-byte aligned.  The library never allocates in the device entry points.  One
 *    workspace must not be used by two calls that overlap on the GPU.
 *  - Host threads: calls may come from several threads at once, each with its own workspace.  Kernel
 *    attributes (shared-memory sizes) are set once per process, on the device current at first use:
 *    one process drives one GPU.
 *  - Errors: argument errors are detected on the host and returned immediately (nothing is
 *    enqueued); rrf_last_arg_error() then names the offending argument (1-based position, LAPACK
 *    style).  Device-side conditions (Jacobi sweep cap, barrier timeout, non-finite input) are
 *    recorded in a status word at the start of the workspace, which every device entry point
 *    clears when it starts: rrf_workspace_status() reads the outcome of the last call.
 */
#ifndef RRF_H
#define RRF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RRF_API __attribute__((visibility("default")))
#else
#define RRF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RRF_OK = 0,
  RRF_INVALID_ARG = 1,      /* an argument is out of range; see rrf_last_arg_error()            */
  RRF_CUDA_ERROR = 2,       /* a CUDA runtime call failed                                        */
  RRF_NOT_CONVERGED = 3,    /* a b x b Jacobi SVD reached its 40-sweep cap (result still written) */
  RRF_TIMEOUT = 4,          /* a bounded device-side wait (grid or cluster barrier) gave up       */
  RRF_NUMERICAL = 5,        /* non-finite value met                                              */
  RRF_UNSUPPORTED = 6,      /* option this entry point does not handle (e.g. oversampling in powerURV) */
  RRF_WORKSPACE_TOO_SMALL = 7
} rrf_status;

/* Precision of the sketch products Y = T22^T G and the power iterations (Algorithm 3). */
enum { RRF_SKETCH_FP64 = 0, RRF_SKETCH_BF16 = 1 };

/* How the power-iteration count q of each randUTV step is chosen. */
enum { RRF_Q_FIXED = 0, RRF_Q_LEARNED = 1 };

/* How the FP64 products run.  RRF_GEMM_AUTO (default): products of at least 2e7 flops whose short side is
 * >= 64, long side >= 128 and inner size >= 32 use the FP64 emulation on the BF16 tensor cores
 * (rrf_gemm_emulated, exact digit products, error relative to row / column maxima), the rest the DFMA
 * kernel.  RRF_GEMM_NATIVE: the DFMA kernel for every product (the plain FP64 method).
 * RRF_GEMM_EMULATED: the emulation for every eligible shape, whatever its size. */
enum { RRF_GEMM_AUTO = 0, RRF_GEMM_NATIVE = 1, RRF_GEMM_EMULATED = 2 };

/* Options; a NULL opts pointer means all defaults (FP64 sketch, no re-orthonormalization, fixed q). */
typedef struct rrf_opts {
  int sketch_prec;   /* RRF_SKETCH_FP64 (default) or RRF_SKETCH_BF16: the sketch GEMMs take BF16 operands
                        with FP32 accumulation on the tensor cores; everything else stays FP64.       */
  int reorth;        /* 1: orthonormalize the sample between applications of T22 and T22^T (Sec. 2.5
                        (ii)); forced on for the BF16 sketch.  0 follows Algorithm 3 literally.       */
  const int* q_per_block; /* optional HOST array of length ceil(n/b): power-iteration count of each
                        step, overriding q; NULL uses q everywhere.                                  */
  int q_policy;      /* RRF_Q_FIXED (default) or RRF_Q_LEARNED: each step first forms the q = 0 sketch,
                        computes 16 features from it (see rrf_mlp_forward), runs the MLP whose FP16
                        parameters mlp_params points to (DEVICE) and uses its argmax as that step's q;
                        with mlp_params == NULL the fallback is the q argument.  The learned policy
                        synchronizes the stream once per step (the host launches the chosen count). */
  const void* mlp_params;
  int* q_used_out;   /* optional HOST array [steps]: the q each step used                              */
  float* features_out; /* optional HOST array [steps x 16]: the features of each step (learned policy) */
  int gemm_mode;     /* RRF_GEMM_AUTO (default), RRF_GEMM_NATIVE or RRF_GEMM_EMULATED */
  int oversample;    /* p >= 0.  p > 0 runs randUTV_boosted (Algorithm 2, Secs. 4.2-4.3) instead of
                        randUTV_basic: b + p sample columns, V_i from the leading b left singular vectors
                        of the sample, and the other p carried into the next step (see rrf_randutv).
                        1 <= b + p <= 256; p > 0 requires the FP64 sketch, reorth = 0 and fixed q
                        (q_per_block allowed).  0 (default) is randUTV_basic.                       */
  double frob_tol;   /* > 0: early termination by the Frobenius recurrence of Sec. 4.1 (see rrf_randutv); 0 off */
  double* frob_out;  /* optional HOST array [ceil(n/b) + 1]: e_0 = ||A||_F, e_1, ..., e_steps (recurrence)   */
  int* steps_out;    /* optional HOST int: the number of steps performed                                 */
  int resume_steps;  /* s0 > 0: U, T, V already hold a factorization stopped after s0 steps (e.g. by
                        frob_tol); continue from step s0 + 1 (see rrf_randutv).  0: start from A.      */
  int reserved[1];   /* must be zero */
} rrf_opts;

/* ------------------------------------------------------------------------------------------------
 * randUTV_basic (Algorithm 3).  For step i = 1 .. min(ceil(m/b), ceil(n/b)) with I2/J2 the current
 * b rows/columns: sketch Y = (T22^T T22)^q T22^T G, V_i from HQR_full(Y), T(:, J2 u J3) <- T V_i,
 * V <- V V_i, U_i and R from HQR_full(T(I2 u I3, J2)), U <- U U_i, T(I2 u I3, J3) <- U_i^T T,
 * T(I3, J2) = 0, then the SVD of R(1:b, 1:b) makes T(I2, J2) diagonal (descending, >= 0).  The last
 * step takes the SVD of the remaining block (via HQR then SVD when it is tall, Sec. 4.2).
 *   m, n      : rows, columns, >= 1 (m < n: through A^T, see the top of this file).
 *   A, lda    : input (device), lda >= m.
 *   b         : block size, 1 <= b <= 256.
 *   q         : power-iteration count, 0 <= q <= 16.
 *   U, ldu    : output m x m orthogonal, ldu >= m.
 *   T, ldt    : output m x n upper trapezoidal with diagonal b x b blocks, ldt >= m.
 *   V, ldv    : output n x n orthogonal, ldv >= n.
 *   seed      : key of the Gaussian stream.
 * Returns RRF_OK once all work is enqueued.
 *
 * With opts->oversample = p > 0 the sample of each step is that of randUTV_boosted (Algorithm 2), with
 * k = b + min(p, c - b) columns.  Step 1: G = randn(r, k) (step 1, tag 1; its first b columns are
 * randUTV_basic's G), Y = (T22^T T22)^q T22^T G.  Later steps recycle the previous step's p extra
 * directions W_next (c x p, expressed in the current trailing columns): G = randn(r, b) (tag 1),
 * Y1 = (T22^T T22)^(q-1) T22^T G, X = T22 Y1, Z = orth(T22 W_next), X <- X - Z (Z^T X), Q = orth(X),
 * Y = T22^T [Q, Z].  Then W_Y = the left singular vectors of Y (Householder QR of Y, Jacobi SVD of its
 * k x k R, both FP64), V_i = HQR_full(W_Y(:, 1:b)) and W_next = rows b.. of V_i^T W_Y(:, b+1:k).  The
 * rest of the step (and the last step) is that of randUTV_basic.
 *
 * Early termination (Sec. 4.1; any sampling option).  With opts->frob_tol > 0 or opts->frob_out set, the
 * library evaluates e_0 = ||A||_F and, after each step i, e_i^2 = max(e_{i-1}^2 - ||T(I2, J2 u J3)||_F^2, 0)
 * on the device (e_i = ||T(ib:, ib:)||_F up to rounding of order eps ||A||_F^2 / e_i; once e_i^2 falls
 * below 2^-30 e_0^2, where that rounding would dominate, ||T(ib:, ib:)||_F is summed directly instead, so
 * tolerances down to ~1e-13 ||A||_F stay meaningful; the last step gives e = 0).  With frob_tol > 0 the call stops after the first step i >= 0 with e_i <= frob_tol (absolute):
 * A = U T V^T still holds with U, V orthogonal, T's first ib columns are upper trapezoidal with diagonal
 * b x b blocks and T(ib:, ib:) is the unreduced trailing block (i = 0: T = A, U = I, V = I).  Checking the
 * tolerance synchronizes the stream once per step, so such a call cannot be captured in a CUDA graph.
 * frob_out receives e_0 .. e_done (written before return: with frob_tol = 0 the call synchronizes once
 * at the end to fill it); steps_out (any mode) receives the number of steps done.
 *
 * Resume (checkpoint at a block boundary: the state after step s0 is (U, T, V, s0), Sec. 4.1).  With
 * opts->resume_steps = s0 > 0 the call does not read A: it takes U, T, V as a factorization of A after s0
 * steps (as left by a call that stopped there) and runs steps s0 + 1, ...; step i still draws the Gaussian
 * of step i, so stopping and resuming gives the same U, T, V bit for bit as one uninterrupted call.  With
 * the Frobenius options, e_s0 is computed directly from T(s0 b:, s0 b:) and frob_out[0 .. s0 - 1] are NaN.
 * Requires m >= n, the randUTV_basic sample (oversample = 0) and fixed q.
 * ---------------------------------------------------------------------------------------------- */
RRF_API size_t rrf_randutv_workspace(int64_t m, int64_t n, int64_t b, const rrf_opts* opts);
RRF_API rrf_status rrf_randutv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                       double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                       uint64_t seed, void* workspace, size_t ws_bytes, const rrf_opts* opts,
                       void* stream);

/* ------------------------------------------------------------------------------------------------
 * powerURV (Algorithm 1): V = randn(n, n); q times { Yh = A V; Vh = HQR_thin(Yh); Y = A^T Vh;
 * V = HQR_thin(Y) }; Ah = A V; [U, R] = HQR_full(Ah).  For q = 0, V is the Q factor of
 * HQR_full(G) (RURV, Sec. 3.1).  R is returned in T (entries below the diagonal exactly 0).
 * b is the panel width of the blocked Householder QRs (1 <= b <= 256).  Other arguments as above.
 * ---------------------------------------------------------------------------------------------- */
RRF_API size_t rrf_powerurv_workspace(int64_t m, int64_t n, int64_t b, const rrf_opts* opts);
RRF_API rrf_status rrf_powerurv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                        double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                        uint64_t seed, void* workspace, size_t ws_bytes, const rrf_opts* opts,
                        void* stream);

/* ------------------------------------------------------------------------------------------------
 * Host-buffer forms (the paper's setting, Sec. 1.3 remark: input and outputs in CPU memory).  Same
 * arguments, but A, U, T, V are HOST pointers (pageable or pinned; leading dimensions as above).
 * The call allocates device buffers and a workspace with cudaMallocAsync on `stream`, copies A in,
 * factors, copies U, T, V out, frees, and returns after the stream has finished (synchronous).  The
 * device status word is folded into the return value.
 * ---------------------------------------------------------------------------------------------- */
RRF_API rrf_status rrf_randutv_host(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                            double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                            uint64_t seed, const rrf_opts* opts, void* stream);
RRF_API rrf_status rrf_powerurv_host(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                             double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                             uint64_t seed, const rrf_opts* opts, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Batched FP32 powerURV (Algorithm 1) for many matrices of uneven shape (m_i >= n_i, m_i <= 2^20).
 * rrf_batch_plan_create fixes count, shapes (HOST arrays m, n), panel width b (1..64) and q; the
 * workspace size follows from the plan.  rrf_powerurv_batched_f32 takes HOST arrays of DEVICE pointers
 * (A_i read-only; U_i m x m, T_i m x n with R, V_i n x n written) and leading dimensions.  Its first call
 * (and any call whose pointers, workspace, seed or stream differ from the previous one) uploads the
 * descriptor table, autotunes the GEMM tile shape on the batch's own problems (first time only),
 * captures the whole batched method as a CUDA graph and launches it; other calls replay the graph.
 * Matrix i draws its Gaussian with key seed + i (step 0, tag 2): what rrf_powerurv draws for it with
 * that seed.  Same Householder convention as the FP64 path, FP32 arithmetic throughout.
 * rrf_batch_plan_tiles(plan, 0 | 1): index of the tile shape chosen for large | skinny GEMM phases. */
typedef struct rrf_batch_plan rrf_batch_plan;
RRF_API rrf_status rrf_batch_plan_create(rrf_batch_plan** plan, int count, const int64_t* m, const int64_t* n,
                                         int64_t b, int q);
RRF_API size_t rrf_batch_plan_workspace(const rrf_batch_plan* plan);
RRF_API int rrf_batch_plan_tiles(const rrf_batch_plan* plan, int which);
RRF_API rrf_status rrf_batch_plan_destroy(rrf_batch_plan* plan);
RRF_API rrf_status rrf_powerurv_batched_f32(rrf_batch_plan* plan, const float* const* A, const int64_t* lda,
                                            float* const* U, const int64_t* ldu, float* const* T,
                                            const int64_t* ldt, float* const* V, const int64_t* ldv,
                                            uint64_t seed, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Building blocks, exported for kernel-level testing.  All pointers are device pointers; all calls
 * enqueue on `stream`.
 * ---------------------------------------------------------------------------------------------- */

/* G = randn(rows, cols) from the stream described above (Sec. 2.1 "standard Gaussian matrix"). */
RRF_API rrf_status rrf_randn(int64_t rows, int64_t cols, double* G, int64_t ldg, uint64_t seed, uint32_t step,
                     uint32_t tag, void* stream);

/* FP64 GEMM C = alpha op(A) op(B) + beta C (the products of Algorithms 1 and 3), transa/transb 'N'
 * or 'T'.  beta == 0 does not read C.  Needs rrf_gemm_workspace(m, n, k) bytes of scratch for its
 * split-K partial sums (0 allowed when that query returns 0). */
RRF_API size_t rrf_gemm_workspace(int64_t m, int64_t n, int64_t k);
RRF_API rrf_status rrf_gemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                    int64_t ldc, void* workspace, size_t ws_bytes, void* stream);

/* FP64 GEMM emulated on the BF16 tensor cores (error-free splitting, Ozaki et al. 2012): same arguments and
 * result convention as rrf_gemm.  Each row of op(A) and column of op(B) is scaled by a power of two and split
 * into 7 signed 8-bit digits (exact in BF16; remainder below 2^-55 of the row / column maximum); the digit
 * products of each 32-wide K chunk accumulate exactly in FP32 on tcgen05 and then exactly in an int64 per
 * output; only digit products below 2^-56 of the scale are dropped.  Error relative to the row and column
 * maxima: |error_ij| <~ 2^-53 |C_ij| + 2^-51.4 K max_k|a_ik| max_k|b_kj| (worst case; random digits give
 * about 2^-55 sqrt(K) max|a_i.| max|b_.j|), so entries far below their row / column scale lose relative
 * accuracy that the native FP64 GEMM keeps.  Needs max(m, n) >= 128, min(m, n) >= 64, k >= 32, and
 * rrf_gemm_emulated_workspace(m, n, k) bytes of workspace. */
RRF_API size_t rrf_gemm_emulated_workspace(int64_t m, int64_t n, int64_t k);
RRF_API rrf_status rrf_gemm_emulated(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                     double* C, int64_t ldc, void* workspace, size_t ws_bytes, void* stream);

/* BF16 x BF16 GEMM with FP32 accumulation on the tensor cores (the products of the BF16 sketch,
 * Sec. 2.5: the range finder only needs a subspace): D = alpha A B^T, where A (m x k) and B (n x k) are
 * stored as rows of k contiguous BF16 values (raw 16-bit patterns), leading dimensions lda, ldb in
 * elements (multiples of 8, bases 16-byte aligned); D is FP64 column-major, ldd >= m; 1 <= n <= 256.
 * Needs rrf_gemm_bf16_workspace(m, n, k) bytes (split-K partial sums, summed in split order). */
RRF_API size_t rrf_gemm_bf16_workspace(int64_t m, int64_t n, int64_t k);
RRF_API rrf_status rrf_gemm_bf16(int64_t m, int64_t n, int64_t k, double alpha, const uint16_t* A, int64_t lda,
                                 const uint16_t* B, int64_t ldb, double* D, int64_t ldd, void* workspace,
                                 size_t ws_bytes, void* stream);

/* Householder QR of an r x w panel (Sec. 2.4, HQR), 1 <= w <= 256, r >= w.  P is overwritten with R
 * (upper triangle) and the Householder vectors (below the diagonal, unit leading entry implicit).
 * Also writes tau (w), the explicit vectors Y (r x w, unit diagonal, zeros above, ldy >= r) and the
 * compact-WY factor Tf (w x w upper triangular, H_0 ... H_{w-1} = I - Y Tf Y^T).  Reflector rule:
 * beta = -sign(alpha) ||x|| with sign(0) = +1, tau = (beta - alpha)/beta, and tau = 0 when the
 * entries below the diagonal are all zero. */
RRF_API size_t rrf_panel_qr_workspace(int64_t r, int64_t w);
RRF_API rrf_status rrf_panel_qr(int64_t r, int64_t w, double* P, int64_t ldp, double* tau, double* Y,
                        int64_t ldy, double* Tf, int64_t ldtf, void* workspace, size_t ws_bytes,
                        void* stream);

/* One-sided Jacobi SVD of an r x c block with r == c <= 256 (the b x b core SVD of Algorithm 3):
 * M = Us diag(s) Vs^T, s descending and >= 0, each pair (u_k, v_k) signed so that v_k's
 * largest-magnitude entry is positive.  Columns with s_k = 0 get u_k by Gram-Schmidt completion.
 * The rotation rule and stopping test are those of Hestenes' method with tolerance c * 2^-53;
 * the column pairs follow a round-robin (tournament) ordering.  Status (converged or not) goes to
 * the workspace status word.  For 32 <= c <= 256 with rrf_jacobi_svd_workspace(c) bytes, FP32 sweeps
 * first give a starting V (made orthogonal in FP64 by two Newton-Schulz steps) and the FP64 sweeps run
 * on M V from there; the FP64 sweeps also stop after a sweep whose rotations all had
 * |gamma| <= 2^-30 sqrt(alpha beta) and tangent |t| <= 2^-24 (which keeps every normalized inner
 * product of the result below about 2 c 2^-53, clusters included).  A workspace of just the header size runs the FP64 sweeps from
 * V = I. */
RRF_API size_t rrf_jacobi_svd_workspace(int64_t c);
RRF_API rrf_status rrf_jacobi_svd(int64_t c, const double* M, int64_t ldm, double* Us, int64_t ldu, double* s,
                          double* Vs, int64_t ldv, void* workspace, size_t ws_bytes, void* stream);

/* Rank-k approximation from a (partial) randUTV factorization (Sec. 4.1): Ak = U(:, 1:k) (T(1:k, :) V^T),
 * i.e. U1 (T11 V1^T + T12 V2^T), whose error ||A - Ak|| equals ||T(k+1:m, k+1:n)|| in the 2- and Frobenius
 * norms.  U is m x m (its first k columns are read), T m x n, V n x n, Ak m x n (ldak >= m, written
 * completely; must not alias the inputs); 0 <= k <= min(m, n) (k = 0 gives Ak = 0).  Both products run on
 * the FP64 DFMA GEMM.  Workspace: rrf_low_rank_workspace(m, n, k) bytes (the k x n product T(1:k, :) V^T
 * and split-K partial sums), 256-byte aligned. */
RRF_API size_t rrf_low_rank_workspace(int64_t m, int64_t n, int64_t k);
RRF_API rrf_status rrf_low_rank(int64_t m, int64_t n, int64_t k, const double* U, int64_t ldu, const double* T,
                                int64_t ldt, const double* V, int64_t ldv, double* Ak, int64_t ldak, void* workspace,
                                size_t ws_bytes, void* stream);

/* Householder panel QR that allocates nothing and takes no workspace.  The paper has no counterpart:
 * this serves callers that cannot give the library device memory for scratch -- code running under
 * a memory manager that owns the whole device, or loops that must not allocate once running.
 * Arguments r, w, P, ldp, tau, Y, ldy are those of rrf_panel_qr (same results; no compact-WY
 * factor).  `status`: optional DEVICE pointer to one int that receives the device status
 * (0 = ok, RRF_TIMEOUT if a grid-barrier wait gave up).
 * Scratch: a fixed 2 MiB array in device global memory, held by every GPU that loads the library
 * until the process exits; w <= 256 with up to 152 cooperating CTAs fits (larger needs return
 * RRF_UNSUPPORTED).  All calls share the array, so calls that overlap on the GPU (different
 * streams, or threads) race and must be serialized by the caller.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) and sets the panel kernel's shared-memory
 * attribute on that device; make that first call before any stream capture.  Unlike the other entry
 * points (one GPU per process), this one may be called on any device of the process, with that device
 * current.  Nothing is allocated: no cudaMalloc/cudaFree, no allocating library routine. */
RRF_API rrf_status rrf_panel_qr_noalloc(int64_t r, int64_t w, double* P, int64_t ldp, double* tau, double* Y,
                                        int64_t ldy, int* status, void* stream);

/* ------------------------------------------------------------------------------------------------
 * The learned power-iteration policy (not in the paper: chooses q per randUTV step).  An MLP
 * 16 -> 64 (ReLU) -> 64 (ReLU) -> 4 logits over q = 0..3, FP16 parameters packed as
 * [W1 (64 x 16 row-major), b1, W2 (64 x 64), b2, W3 (4 x 64), b3] (rrf_mlp_param_count() values),
 * FP16 activations, FP32 accumulation.  All pointers are DEVICE pointers; X is N x 16 row-major FP32,
 * logits N x 4, labels N ints in 0..3.
 * rrf_mlp_grad: mean softmax-cross-entropy loss (optional *loss) and its gradient (FP32, packed like the
 *   parameters) over the N samples; workspace rrf_mlp_train_workspace(N) bytes.
 * rrf_mlp_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master copy and moments
 *   m, v (all packed like the parameters), refreshing the FP16 parameters; step counts from 1. */
RRF_API int rrf_mlp_param_count(void);
RRF_API size_t rrf_mlp_train_workspace(int N);
RRF_API rrf_status rrf_mlp_forward(const void* params, const float* X, int N, float* logits, void* stream);
RRF_API rrf_status rrf_mlp_grad(const void* params, const float* X, const int* labels, int N, float* grad,
                                float* loss, void* workspace, size_t ws_bytes, void* stream);
RRF_API rrf_status rrf_mlp_adam(float* master, float* m, float* v, const float* grad, void* params, int step,
                                float lr, void* stream);

/* Reads the device status word of a workspace used by any call above (synchronizes `stream`).
 * Returns RRF_OK or the first device-side condition the last call recorded. */
RRF_API rrf_status rrf_workspace_status(void* workspace, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Diagnostics (not part of the method).
 * rrf_launch_count: number of GPU kernels this library has launched in this process so far.
 * rrf_gemm_profile_begin: from now on, bracket every FP64 GEMM launch (including its split-K
 *   reduction) with CUDA events on its stream, up to max_launches launches; returns 0 on success.
 * rrf_gemm_profile_end: stop, wait for the recorded events and return the summed DFMA GEMM device
 *   time (ms), the algorithmic flops of those launches (sum of 2 M N K over their problems) and the
 *   number of launches timed.  Returns 0 on success.
 * rrf_gemm_profile_emulated (after rrf_gemm_profile_end): the same for the tensor-core kernel of the
 *   emulated GEMM (its digit splitting and split-K reduction launches are not included): device time,
 *   FP64-equivalent flops 2 M N K, tensor flops 28 x 2 M N K' (K' = K rounded up to 32) and launches.
 * rrf_gemm_profile_emulated_bytes (after rrf_gemm_profile_end): the algorithmic DRAM bytes of those same
 *   launches: 14 (M + N) K' for the digit slices of op(A) and op(B), read once, plus 8 M N for C written
 *   once (twice when beta != 0: C is read too; splits x 8 M N of partial sums when K is split).
 * rrf_gemm_profile_panel (after rrf_gemm_profile_end): the same for the Householder panel kernel of every
 *   panel factorization (its compact-WY factor not included): device time, flops 2 r w^2 - 2 w^3 / 3,
 *   algorithmic bytes 24 r w (the panel read and written back, the reflectors written) and launches.
 * rrf_gemm_profile_bf16 (after rrf_gemm_profile_end): the same for the tensor-core kernel of the BF16
 *   sketch GEMM (its split-K reduction not included): device time, flops 2 M N K, algorithmic bytes
 *   2 (M + N) K (BF16 operands read once) + 4 M N (one FP32 result per output) and launches.
 * ---------------------------------------------------------------------------------------------- */
RRF_API int64_t rrf_launch_count(void);
RRF_API int rrf_gemm_profile_begin(int max_launches);
RRF_API int rrf_gemm_profile_end(double* ms, double* flops, int64_t* launches);
RRF_API int rrf_gemm_profile_emulated(double* ms, double* flops, double* tensor_flops, int64_t* launches);
RRF_API int rrf_gemm_profile_bf16(double* ms, double* flops, double* bytes, int64_t* launches);
RRF_API int rrf_gemm_profile_emulated_bytes(double* bytes);
RRF_API int rrf_gemm_profile_panel(double* ms, double* flops, double* bytes, int64_t* launches);

/* ------------------------------------------------------------------------------------------------
 * Failure injection for tests (not part of the method; no counterpart in the paper).  Drives the
 * bounded-wait and sweep-cap paths on purpose, without faulting or hanging the GPU:
 *   RRF_INJECT_NONE          -- normal operation (default).
 *   RRF_INJECT_PANEL_STALL   -- the Householder panel kernel's grid barrier waits for one CTA more
 *                               than it launched, so no barrier completes; every CTA gives up after
 *                               `value` clock cycles (>= 1), records RRF_TIMEOUT and returns.
 *   RRF_INJECT_GEMM_STALL    -- in the emulated FP64 GEMM's tensor-core kernel the MMA warp first
 *                               waits `value` cycles on a barrier nothing arrives on, then aborts: no
 *                               MMA is issued, the other warps give up after their normal limit (~2 s),
 *                               the tile copies already in flight are waited for, TMEM is released, and
 *                               RRF_TIMEOUT is recorded.
 *   RRF_INJECT_JACOBI_CAP    -- the FP64 Jacobi sweeps are capped at `value` (>= 1) instead of 40, so a
 *                               matrix that needs more sweeps records RRF_NOT_CONVERGED.
 * The setting is process-wide and applies to every call made while it is active; results of those
 * calls are not meaningful.  Returns RRF_INVALID_ARG for an unknown kind or value < 1. */
enum { RRF_INJECT_NONE = 0, RRF_INJECT_PANEL_STALL = 1, RRF_INJECT_GEMM_STALL = 2, RRF_INJECT_JACOBI_CAP = 3 };
RRF_API rrf_status rrf_test_inject(int kind, long long value);

/* Human-readable name of a status code (static storage). */
RRF_API const char* rrf_status_string(rrf_status s);

/* 1-based position of the first invalid argument of the last call on this thread, 0 if none. */
RRF_API int rrf_last_arg_error(void);

/* Library version string (static storage). */
RRF_API const char* rrf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RRF_H */
