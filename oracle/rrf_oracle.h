/*
 * rrf_oracle.h -- FP64 CPU oracle for the randomized rank-revealing factorizations of
 * "Efficient algorithms for computing rank-revealing factorizations on a GPU"
 * (randUTV_basic, Algorithm 3 / appendix "randUTV algorithm adapted from ...", powerURV, Algorithm 1, and
 * randUTV_boosted, Algorithm 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the CUDA path is checked
 * against.  Only the test suite, the package's smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Conventions: every matrix is column-major FP64 with an explicit leading dimension; indices are
 * 0-based here, while the paper uses 1-based Matlab notation.  Status codes: 0 = ok,
 * 1 = invalid argument, 3 = Jacobi sweep cap reached (not converged).
 */
#ifndef RRF_ORACLE_H
#define RRF_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Philox-4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Gaussian matrix G = randn(rows, cols) of Sec. 2.1 ("standard Gaussian matrix"), drawn from the
 * counter-based stream: key = (seed lo32, seed hi32); block t -> counter (t lo32, t hi32, step, tag);
 * block t gives the column-major elements 2t and 2t+1 by the Box-Muller transform. */
void orc_randn(int64_t rows, int64_t cols, double* G, int64_t ldg, uint64_t seed, uint32_t step,
               uint32_t tag);

/* Plain GEMM C = alpha*op(A)*op(B) + beta*C, op = 'N' or 'T'. (Sec. 2.4's "gemm"; a library-style step.) */
void orc_gemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc);

/* Householder QR (HQR, Sec. 2.4) in place: R in the upper triangle, Householder vectors below the
 * diagonal (unit leading entry implicit), tau[j] with H_j = I - tau_j v_j v_j^T. */
void orc_hqr(int64_t m, int64_t n, double* A, int64_t lda, double* tau);

/* Compact-WY factor (Sec. 2.4): upper triangular Tf (k x k) with H_0 H_1 ... H_{k-1} = I - Y Tf Y^T. */
void orc_larft(int64_t m, int64_t k, const double* Y, int64_t ldy, const double* tau, double* Tf,
               int64_t ldtf);

/* Apply Q = H_0 H_1 ... H_{k-1} (reflectors stored as by orc_hqr) one reflector at a time:
 * side 'L': C <- op(Q) C  (C is m x n, reflectors have length m)
 * side 'R': C <- C op(Q)  (C is m x n, reflectors have length n)            trans = 'N' or 'T'. */
void orc_apply_q(char side, char trans, int64_t m, int64_t n, int64_t k, const double* Y, int64_t ldy,
                 const double* tau, double* C, int64_t ldc);

/* Explicit Q(:, 0:ncols) of HQR (HQR_full when ncols = m, HQR_thin when ncols = k). */
void orc_form_q(int64_t m, int64_t ncols, int64_t k, const double* Y, int64_t ldy, const double* tau,
                double* Q, int64_t ldq);

/* One-sided (Hestenes) Jacobi SVD of an r x c block M (r >= c), cyclic-by-rows ordering:
 * M = Us * diag(s) * Vs^T with Us r x c orthonormal, s descending, Vs c x c orthogonal, and each
 * column pair (u_k, v_k) signed so that v_k's largest-magnitude entry is positive.
 * Returns 0, or 3 when 40 sweeps did not converge.  *sweeps_out (optional) receives the sweep count. */
int orc_jacobi_svd(int64_t r, int64_t c, const double* M, int64_t ldm, double* Us, int64_t ldu,
                   double* s, double* Vs, int64_t ldv, int* sweeps_out);

/* randUTV_basic (Algorithm 3).  U (m x m), T (m x n), V (n x n) outputs; requires m >= n >= 1, b >= 1,
 * q >= 0.  max_steps > 0 stops after that many steps (a partial factorization, Sec. 4.1); 0 runs all.
 * The Gaussian of step i (1-based) is orc_randn(m - b(i-1), b, ..., seed, step = i, tag = 1). */
int orc_randutv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, uint64_t seed,
                double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, int max_steps);

/* randUTV_basic with the power iteration re-orthonormalized (Sec. 2.5 (ii); Sec. 4.3): in step i,
 * Y = T22^T G, then q times { Y <- thin Q of HQR(Y); Z = T22 Y; Z <- thin Q of HQR(Z); Y = T22^T Z }.
 * Everything else, and the Gaussian stream, as orc_randutv.  In exact arithmetic step 1 samples the
 * same subspace as orc_randutv; in floating point it keeps directions that the plain iteration loses
 * below about eps^(1/(2q+1)) of the block's largest singular value. */
int orc_randutv_reorth(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, uint64_t seed,
                       double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, int max_steps);

/* randUTV_boosted (Algorithm 2) with oversampling p and recycled samples; p = 0 samples the subspace of
 * randUTV_basic (q >= 1).  Same outputs and conventions as orc_randutv. */
int orc_randutv_boosted(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, int64_t p,
                        uint64_t seed, double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                        int max_steps);
/* powerURV (Algorithm 1).  U (m x m), R (m x n, upper trapezoidal), V (n x n).  The Gaussian is
 * orc_randn(n, n, ..., seed, step = 0, tag = 2).  For q = 0, V is the Q factor of HQR_full(G) (RURV). */
int orc_powerurv(int64_t m, int64_t n, const double* A, int64_t lda, int q, uint64_t seed, double* U,
                 int64_t ldu, double* R, int64_t ldr, double* V, int64_t ldv);

/* Number of OpenMP threads the oracle uses. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
