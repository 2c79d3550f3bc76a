/*
 * rrf_oracle.c -- FP64 CPU oracle for randUTV_basic (Algorithm 3) and powerURV (Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct reference the CUDA path is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code with the CUDA path: reflectors are applied one at a time (the definition of
 * Q = H_0 H_1 ... H_{k-1}, Sec. 2.4), never in compact-WY blocks; the small SVD is a textbook
 * one-sided Jacobi with cyclic-by-rows ordering; GEMMs are triple loops.  OpenMP only distributes
 * independent columns (or rows) over threads, which does not change any result bit.
 *
 * Parity status of each function (what pins it) is listed in the test suite's oracle tests.
 */
#include "rrf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 * One round: two 32x32->64 multiplies of counter words 0 and 2 by the round multipliers, the high
 * halves xored with the other two counter words and the round key; the key is bumped by the Weyl
 * constants between rounds.  Ten rounds.
 * ------------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t p0 = (uint64_t)mul0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)mul1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* randn(rows, cols) (Sec. 2.1).  Block t of the stream feeds column-major elements 2t and 2t+1:
 * u1 = (((x0:x1) >> 11) + 1) * 2^-53 in (0,1], u2 = ((x2:x3) >> 11) * 2^-53 in [0,1),
 * rho = sqrt(-2 ln u1), element 2t = rho cos(2 pi u2), element 2t+1 = rho sin(2 pi u2)
 * (Box & Muller 1958). */
void orc_randn(int64_t rows, int64_t cols, double* G, int64_t ldg, uint64_t seed, uint32_t step,
               uint32_t tag) {
  const int64_t total = rows * cols;
  const int64_t nblocks = (total + 1) / 2;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < nblocks; ++t) {
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)((uint64_t)t >> 32), step, tag};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint64_t a = ((uint64_t)x[0] << 32) | x[1];
    uint64_t c = ((uint64_t)x[2] << 32) | x[3];
    double u1 = (double)((a >> 11) + 1) * 0x1p-53;
    double u2 = (double)(c >> 11) * 0x1p-53;
    double rho = sqrt(-2.0 * log(u1));
    double ang = two_pi * u2;
    double z[2] = {rho * cos(ang), rho * sin(ang)};
    for (int e = 0; e < 2; ++e) {
      int64_t lin = 2 * t + e;
      if (lin < total) {
        int64_t i = lin % rows, j = lin / rows;
        G[IDX(i, j, ldg)] = z[e];
      }
    }
  }
}

/* ---------------------------------------------------------------------------------------------
 * Plain GEMM: C(i,j) = alpha * sum_l op(A)(i,l) op(B)(l,j) + beta * C(i,j), summed in l order.
 * ------------------------------------------------------------------------------------------- */
void orc_gemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  const int tA = (ta == 'T' || ta == 't');
  const int tB = (tb == 'T' || tb == 't');
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double* acc = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    for (int64_t l = 0; l < k; ++l) {
      const double bl = tB ? B[IDX(j, l, ldb)] : B[IDX(l, j, ldb)];
      if (tA) {
        for (int64_t i = 0; i < m; ++i) acc[i] += A[IDX(l, i, lda)] * bl;
      } else {
        const double* a = A + IDX(0, l, lda);
        for (int64_t i = 0; i < m; ++i) acc[i] += a[i] * bl;
      }
    }
    for (int64_t i = 0; i < m; ++i) {
      double c0 = (beta == 0.0) ? 0.0 : beta * C[IDX(i, j, ldc)];
      C[IDX(i, j, ldc)] = alpha * acc[i] + c0;
    }
    free(acc);
  }
}

/* ---------------------------------------------------------------------------------------------
 * Householder QR (HQR, Sec. 2.4).  Column j: x = A(j:m, j), alpha = x(0), sigma^2 = ||x(1:)||^2.
 * If sigma^2 == 0 the reflector is the identity (tau = 0).  Otherwise
 *   beta = -sign(alpha) ||x|| with sign(0) = +1,  v = (x - beta e1) / (alpha - beta),  tau = (beta - alpha)/beta,
 * so (I - tau v v^T) x = beta e1.  This is the paper's H = I - 2 y y^T with y = v / ||v||.
 * The reflector is then applied to the remaining columns.
 * ------------------------------------------------------------------------------------------- */
void orc_hqr(int64_t m, int64_t n, double* A, int64_t lda, double* tau) {
  const int64_t kmax = m < n ? m : n;
  for (int64_t j = 0; j < kmax; ++j) {
    double* x = A + IDX(j, j, lda);
    const int64_t len = m - j;
    double alpha = x[0];
    double sig2 = 0.0;
    for (int64_t i = 1; i < len; ++i) sig2 += x[i] * x[i];
    if (sig2 == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    double nrm = sqrt(alpha * alpha + sig2);
    double beta = (alpha >= 0.0) ? -nrm : nrm;
    double t = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int64_t i = 1; i < len; ++i) x[i] *= scal;
    x[0] = beta;
    tau[j] = t;
#pragma omp parallel for schedule(static)
    for (int64_t c = j + 1; c < n; ++c) {
      double* a = A + IDX(j, c, lda);
      double w = a[0];
      for (int64_t i = 1; i < len; ++i) w += x[i] * a[i];
      w *= t;
      a[0] -= w;
      for (int64_t i = 1; i < len; ++i) a[i] -= w * x[i];
    }
  }
}

/* Element l of reflector v_j stored below the diagonal of column j (l >= j). */
static inline double refl(const double* Y, int64_t ldy, int64_t j, int64_t l) {
  return (l == j) ? 1.0 : Y[IDX(l, j, ldy)];
}

/* Compact-WY (Sec. 2.4, Schreiber & Van Loan): forward recurrence
 *   Tf(j,j) = tau_j,   Tf(0:j, j) = -tau_j * Tf(0:j, 0:j) * (Y(:, 0:j)^T v_j). */
void orc_larft(int64_t m, int64_t k, const double* Y, int64_t ldy, const double* tau, double* Tf,
               int64_t ldtf) {
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i < k; ++i) Tf[IDX(i, j, ldtf)] = 0.0;
  double* w = (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
  for (int64_t j = 0; j < k; ++j) {
    for (int64_t p = 0; p < j; ++p) {
      double s = 0.0;
      for (int64_t l = j; l < m; ++l) s += refl(Y, ldy, p, l) * refl(Y, ldy, j, l);
      w[p] = s;
    }
    for (int64_t p = 0; p < j; ++p) {
      double s = 0.0;
      for (int64_t l = p; l < j; ++l) s += Tf[IDX(p, l, ldtf)] * w[l];
      Tf[IDX(p, j, ldtf)] = -tau[j] * s;
    }
    Tf[IDX(j, j, ldtf)] = tau[j];
  }
  free(w);
}

/* Apply one reflector sequence to independent columns ('L') or rows ('R') of C. */
void orc_apply_q(char side, char trans, int64_t m, int64_t n, int64_t k, const double* Y, int64_t ldy,
                 const double* tau, double* C, int64_t ldc) {
  const int left = (side == 'L' || side == 'l');
  const int tr = (trans == 'T' || trans == 't');
  /* Left: Q C applies H_{k-1} first; Q^T C applies H_0 first.
   * Right: C Q applies H_0 first; C Q^T applies H_{k-1} first. */
  const int forward = left ? tr : !tr;
  if (left) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      double* x = C + IDX(0, c, ldc);
      for (int64_t s = 0; s < k; ++s) {
        int64_t j = forward ? s : (k - 1 - s);
        if (tau[j] == 0.0) continue;
        double w = x[j];
        for (int64_t l = j + 1; l < m; ++l) w += Y[IDX(l, j, ldy)] * x[l];
        w *= tau[j];
        x[j] -= w;
        for (int64_t l = j + 1; l < m; ++l) x[l] -= w * Y[IDX(l, j, ldy)];
      }
    }
  } else {
    const int64_t RB = 32; /* rows handled together; each row sees the same operation sequence */
    const int64_t nrb = (m + RB - 1) / RB;
#pragma omp parallel for schedule(static)
    for (int64_t rb = 0; rb < nrb; ++rb) {
      int64_t r0 = rb * RB, r1 = r0 + RB < m ? r0 + RB : m;
      double w[32];
      for (int64_t s = 0; s < k; ++s) {
        int64_t j = forward ? s : (k - 1 - s);
        if (tau[j] == 0.0) continue;
        for (int64_t i = r0; i < r1; ++i) w[i - r0] = C[IDX(i, j, ldc)];
        for (int64_t l = j + 1; l < n; ++l) {
          const double y = Y[IDX(l, j, ldy)];
          const double* cl = C + IDX(0, l, ldc);
          for (int64_t i = r0; i < r1; ++i) w[i - r0] += cl[i] * y;
        }
        for (int64_t i = r0; i < r1; ++i) w[i - r0] *= tau[j];
        for (int64_t i = r0; i < r1; ++i) C[IDX(i, j, ldc)] -= w[i - r0];
        for (int64_t l = j + 1; l < n; ++l) {
          const double y = Y[IDX(l, j, ldy)];
          double* cl = C + IDX(0, l, ldc);
          for (int64_t i = r0; i < r1; ++i) cl[i] -= w[i - r0] * y;
        }
      }
    }
  }
}

void orc_form_q(int64_t m, int64_t ncols, int64_t k, const double* Y, int64_t ldy, const double* tau,
                double* Q, int64_t ldq) {
  for (int64_t j = 0; j < ncols; ++j)
    for (int64_t i = 0; i < m; ++i) Q[IDX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
  orc_apply_q('L', 'N', m, ncols, k, Y, ldy, tau, Q, ldq);
}

/* ---------------------------------------------------------------------------------------------
 * One-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992) of an r x c block, r >= c.
 * For each column pair (p, q) in cyclic-by-rows order: alpha = ||m_p||^2, beta = ||m_q||^2,
 * gamma = m_p . m_q; skip when |gamma| <= tol sqrt(alpha beta) (tol = r 2^-53); otherwise the
 * rotation that diagonalises [[alpha, gamma], [gamma, beta]]:
 *   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
 *   cs = 1 / sqrt(1 + t^2), sn = cs t,   (m_p, m_q) <- (cs m_p - sn m_q, sn m_p + cs m_q),
 * and the same on the columns of V.  Stop after a sweep without rotations (cap: 40 sweeps).
 * Then sigma_k = ||m_k||, u_k = m_k / sigma_k, sorted descending (ties keep index order), each pair
 * signed so the largest-magnitude entry of v_k (first on ties) is positive; columns with
 * sigma_k = 0 get u_k by Gram-Schmidt against the canonical basis.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  double s;
  int64_t idx;
} orc_sv;

static int orc_sv_cmp(const void* a, const void* b) {
  const orc_sv* x = (const orc_sv*)a;
  const orc_sv* y = (const orc_sv*)b;
  if (x->s > y->s) return -1;
  if (x->s < y->s) return 1;
  return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

int orc_jacobi_svd(int64_t r, int64_t c, const double* M, int64_t ldm, double* Us, int64_t ldu,
                   double* s, double* Vs, int64_t ldv, int* sweeps_out) {
  if (r < c || c < 0) return 1;
  double* W = (double*)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1) * (size_t)(c > 0 ? c : 1));
  double* V = (double*)malloc(sizeof(double) * (size_t)(c > 0 ? c : 1) * (size_t)(c > 0 ? c : 1));
  for (int64_t j = 0; j < c; ++j) {
    for (int64_t i = 0; i < r; ++i) W[IDX(i, j, r)] = M[IDX(i, j, ldm)];
    for (int64_t i = 0; i < c; ++i) V[IDX(i, j, c)] = (i == j) ? 1.0 : 0.0;
  }
  const double tol = (double)r * 0x1p-53;
  int sweeps = 0, status = 3;
  while (sweeps < 40) {
    ++sweeps;
    int64_t rotations = 0;
    for (int64_t p = 0; p + 1 < c; ++p) {
      for (int64_t q = p + 1; q < c; ++q) {
        double* mp = W + IDX(0, p, r);
        double* mq = W + IDX(0, q, r);
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t i = 0; i < r; ++i) {
          alpha += mp[i] * mp[i];
          beta += mq[i] * mq[i];
          gamma += mp[i] * mq[i];
        }
        if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        ++rotations;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t);
        double sn = cs * t;
        for (int64_t i = 0; i < r; ++i) {
          double a = mp[i], b = mq[i];
          mp[i] = cs * a - sn * b;
          mq[i] = sn * a + cs * b;
        }
        double* vp = V + IDX(0, p, c);
        double* vq = V + IDX(0, q, c);
        for (int64_t i = 0; i < c; ++i) {
          double a = vp[i], b = vq[i];
          vp[i] = cs * a - sn * b;
          vq[i] = sn * a + cs * b;
        }
      }
    }
    if (rotations == 0) {
      status = 0;
      break;
    }
  }
  if (sweeps_out) *sweeps_out = sweeps;
  orc_sv* order = (orc_sv*)malloc(sizeof(orc_sv) * (size_t)(c > 0 ? c : 1));
  for (int64_t j = 0; j < c; ++j) {
    double ss = 0.0;
    for (int64_t i = 0; i < r; ++i) ss += W[IDX(i, j, r)] * W[IDX(i, j, r)];
    order[j].s = sqrt(ss);
    order[j].idx = j;
  }
  qsort(order, (size_t)c, sizeof(orc_sv), orc_sv_cmp);
  for (int64_t k = 0; k < c; ++k) {
    const int64_t src = order[k].idx;
    const double sig = order[k].s;
    s[k] = sig;
    for (int64_t i = 0; i < c; ++i) Vs[IDX(i, k, ldv)] = V[IDX(i, src, c)];
    for (int64_t i = 0; i < r; ++i) Us[IDX(i, k, ldu)] = (sig > 0.0) ? W[IDX(i, src, r)] / sig : 0.0;
    int64_t imax = 0;
    double vmax = -1.0;
    for (int64_t i = 0; i < c; ++i) {
      double a = fabs(Vs[IDX(i, k, ldv)]);
      if (a > vmax) {
        vmax = a;
        imax = i;
      }
    }
    if (Vs[IDX(imax, k, ldv)] < 0.0) {
      for (int64_t i = 0; i < c; ++i) Vs[IDX(i, k, ldv)] = -Vs[IDX(i, k, ldv)];
      for (int64_t i = 0; i < r; ++i) Us[IDX(i, k, ldu)] = -Us[IDX(i, k, ldu)];
    }
  }
  /* Gram-Schmidt completion (two passes) for exactly-zero singular values. */
  double* w = (double*)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
  for (int64_t k = 0; k < c; ++k) {
    if (s[k] > 0.0) continue;
    for (int64_t e = 0; e < r; ++e) {
      for (int64_t i = 0; i < r; ++i) w[i] = (i == e) ? 1.0 : 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int64_t j = 0; j < c; ++j) {
          if (j == k || (j > k && s[j] == 0.0)) continue;
          double d = 0.0;
          for (int64_t i = 0; i < r; ++i) d += Us[IDX(i, j, ldu)] * w[i];
          for (int64_t i = 0; i < r; ++i) w[i] -= d * Us[IDX(i, j, ldu)];
        }
      }
      double nn = 0.0;
      for (int64_t i = 0; i < r; ++i) nn += w[i] * w[i];
      nn = sqrt(nn);
      if (nn > 0.5) {
        for (int64_t i = 0; i < r; ++i) Us[IDX(i, k, ldu)] = w[i] / nn;
        break;
      }
    }
  }
  free(w);
  free(order);
  free(W);
  free(V);
  return status;
}

/* ---------------------------------------------------------------------------------------------
 * randUTV_basic (Algorithm 3).  0-based: step i (1-based) has offset o = b(i-1),
 * I2 = o:min(bi,m), I3 = bi:m, J2 = o:min(bi,n), J3 = bi:n.
 * ------------------------------------------------------------------------------------------- */
static void copy_block(int64_t r, int64_t c, const double* S, int64_t lds, double* D, int64_t ldd) {
  for (int64_t j = 0; j < c; ++j)
    for (int64_t i = 0; i < r; ++i) D[IDX(i, j, ldd)] = S[IDX(i, j, lds)];
}

/* C(0:rows, 0:k) <- C(0:rows, 0:k) * S  with S k x k (via a temporary, plain GEMM). */
static void right_mul_small(int64_t rows, int64_t k, double* C, int64_t ldc, const double* S, int64_t lds) {
  if (rows <= 0 || k <= 0) return;
  double* tmp = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)k);
  orc_gemm('N', 'N', rows, k, k, 1.0, C, ldc, S, lds, 0.0, tmp, rows);
  copy_block(rows, k, tmp, rows, C, ldc);
  free(tmp);
}

/* C(0:k, 0:cols) <- S^T * C(0:k, 0:cols). */
static void left_mul_small_t(int64_t k, int64_t cols, double* C, int64_t ldc, const double* S, int64_t lds) {
  if (cols <= 0 || k <= 0) return;
  double* tmp = (double*)malloc(sizeof(double) * (size_t)k * (size_t)cols);
  orc_gemm('T', 'N', k, cols, k, 1.0, S, lds, C, ldc, 0.0, tmp, k);
  copy_block(k, cols, tmp, k, C, ldc);
  free(tmp);
}

static void thin_q(int64_t rows, int64_t k, const double* X, int64_t ldx, double* Q, int64_t ldq);

/* randUTV_basic; reorth != 0 orthonormalizes the sample before every application of T22 and of T22^T
 * (the power iteration with re-orthonormalization of Sec. 2.5 (ii), recommended again in Sec. 4.3). */
static int randutv_impl(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, uint64_t seed,
                        double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, int max_steps,
                        int reorth) {
  if (m < n || n < 1 || b < 1 || q < 0 || lda < m || ldu < m || ldt < m || ldv < n) return 1;
  int status = 0;
  /* T = A; U = I_m; V = I_n. */
  copy_block(m, n, A, lda, T, ldt);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) U[IDX(i, j, ldu)] = (i == j) ? 1.0 : 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) V[IDX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;

  const int64_t steps_m = (m + b - 1) / b, steps_n = (n + b - 1) / b;
  const int64_t s = steps_m < steps_n ? steps_m : steps_n;
  double* G = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n * (size_t)b);
  double* Z = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
  double* tauv = (double*)malloc(sizeof(double) * (size_t)b);
  double* tauu = (double*)malloc(sizeof(double) * (size_t)b);
  double* Rs = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double* Usm = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double* Vsm = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double* sig = (double*)malloc(sizeof(double) * (size_t)b);
  double* Qo = reorth ? (double*)malloc(sizeof(double) * (size_t)m * (size_t)b) : NULL;

  for (int64_t i = 1; i <= s; ++i) {
    if (max_steps > 0 && i > max_steps) break;
    const int64_t o = b * (i - 1);
    const int64_t r = m - o, c = n - o;
    double* T22 = T + IDX(o, o, ldt);
    if (b * i < m && b * i < n) {
      /* G = randn(m - b(i-1), b); Y = T22^T G; Y = T22^T (T22 Y) q times.  With reorth the input of
       * each application is replaced by an orthonormal basis of its columns (thin Q of its HQR). */
      orc_randn(r, b, G, r, seed, (uint32_t)i, 1u);
      orc_gemm('T', 'N', c, b, r, 1.0, T22, ldt, G, r, 0.0, Y, c);
      for (int j = 0; j < q; ++j) {
        if (reorth) {
          thin_q(c, b, Y, c, Qo, c);
          copy_block(c, b, Qo, c, Y, c);
        }
        orc_gemm('N', 'N', r, b, c, 1.0, T22, ldt, Y, c, 0.0, Z, r);
        if (reorth) {
          thin_q(r, b, Z, r, Qo, r);
          copy_block(r, b, Qo, r, Z, r);
        }
        orc_gemm('T', 'N', c, b, r, 1.0, T22, ldt, Z, r, 0.0, Y, c);
      }
      /* [V_i, ~] = HQR_full(Y); T(:, J2 u J3) <- T(:, J2 u J3) V_i; V(:, J2 u J3) <- V(:, J2 u J3) V_i. */
      orc_hqr(c, b, Y, c, tauv);
      orc_apply_q('R', 'N', m, c, b, Y, c, tauv, T + IDX(0, o, ldt), ldt);
      orc_apply_q('R', 'N', n, c, b, Y, c, tauv, V + IDX(0, o, ldv), ldv);
      /* [U_i, R] = HQR_full(T(I2 u I3, J2)); U(:, I2 u I3) <- U(:, I2 u I3) U_i;
       * T(I2 u I3, J3) <- U_i^T T(I2 u I3, J3); T(I3, J2) = 0. */
      copy_block(r, b, T22, ldt, P, r);
      orc_hqr(r, b, P, r, tauu);
      orc_apply_q('R', 'N', m, r, b, P, r, tauu, U + IDX(0, o, ldu), ldu);
      orc_apply_q('L', 'T', r, c - b, b, P, r, tauu, T + IDX(o, o + b, ldt), ldt);
      for (int64_t jj = 0; jj < b; ++jj)
        for (int64_t ii = 0; ii < b; ++ii) Rs[IDX(ii, jj, b)] = (ii <= jj) ? P[IDX(ii, jj, r)] : 0.0;
      for (int64_t jj = 0; jj < b; ++jj)
        for (int64_t ii = b; ii < r; ++ii) T[IDX(o + ii, o + jj, ldt)] = 0.0;
      /* [U_small, D_small, V_small] = svd(R(1:b, 1:b)) and the small updates. */
      int st = orc_jacobi_svd(b, b, Rs, b, Usm, b, sig, Vsm, b, NULL);
      if (st != 0) status = st;
      right_mul_small(m, b, U + IDX(0, o, ldu), ldu, Usm, b);
      right_mul_small(n, b, V + IDX(0, o, ldv), ldv, Vsm, b);
      for (int64_t jj = 0; jj < b; ++jj)
        for (int64_t ii = 0; ii < b; ++ii) T[IDX(o + ii, o + jj, ldt)] = (ii == jj) ? sig[ii] : 0.0;
      left_mul_small_t(b, c - b, T + IDX(o, o + b, ldt), ldt, Usm, b);
      right_mul_small(o, b, T + IDX(0, o, ldt), ldt, Vsm, b);
    } else {
      /* Final block: SVD of T(I2 u I3, J2 u J3) (r x c, r >= c).  A tall block goes through
       * HQR_full first and the SVD of its square R (Sec. 4.2, tall-thin SVD remark). */
      double* Uf = (double*)malloc(sizeof(double) * (size_t)r * (size_t)c);
      double* Vf = (double*)malloc(sizeof(double) * (size_t)c * (size_t)c);
      double* sf = (double*)malloc(sizeof(double) * (size_t)c);
      int st;
      if (r > c) {
        double* Pf = (double*)malloc(sizeof(double) * (size_t)r * (size_t)c);
        double* tf = (double*)malloc(sizeof(double) * (size_t)c);
        double* Rf = (double*)malloc(sizeof(double) * (size_t)c * (size_t)c);
        copy_block(r, c, T22, ldt, Pf, r);
        orc_hqr(r, c, Pf, r, tf);
        for (int64_t jj = 0; jj < c; ++jj)
          for (int64_t ii = 0; ii < c; ++ii) Rf[IDX(ii, jj, c)] = (ii <= jj) ? Pf[IDX(ii, jj, r)] : 0.0;
        st = orc_jacobi_svd(c, c, Rf, c, Uf, c, sf, Vf, c, NULL);
        orc_apply_q('R', 'N', m, r, c, Pf, r, tf, U + IDX(0, o, ldu), ldu);
        right_mul_small(m, c, U + IDX(0, o, ldu), ldu, Uf, c);
        free(Pf);
        free(tf);
        free(Rf);
      } else {
        st = orc_jacobi_svd(r, c, T22, ldt, Uf, r, sf, Vf, c, NULL);
        right_mul_small(m, c, U + IDX(0, o, ldu), ldu, Uf, r);
      }
      if (st != 0) status = st;
      right_mul_small(n, c, V + IDX(0, o, ldv), ldv, Vf, c);
      for (int64_t jj = 0; jj < c; ++jj)
        for (int64_t ii = 0; ii < r; ++ii) T[IDX(o + ii, o + jj, ldt)] = (ii == jj) ? sf[ii] : 0.0;
      right_mul_small(o, c, T + IDX(0, o, ldt), ldt, Vf, c);
      free(Uf);
      free(Vf);
      free(sf);
    }
  }
  free(G); free(Y); free(Z); free(P); free(tauv); free(tauu);
  free(Rs); free(Usm); free(Vsm); free(sig); free(Qo);
  return status;
}

int orc_randutv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, uint64_t seed,
                double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, int max_steps) {
  return randutv_impl(m, n, A, lda, b, q, seed, U, ldu, T, ldt, V, ldv, max_steps, 0);
}

int orc_randutv_reorth(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, uint64_t seed,
                       double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, int max_steps) {
  return randutv_impl(m, n, A, lda, b, q, seed, U, ldu, T, ldt, V, ldv, max_steps, 1);
}

/* ---------------------------------------------------------------------------------------------
 * randUTV_boosted (Algorithm 2): randUTV with p oversampled columns whose extra samples are carried
 * from one step to the next.  Step 1 samples Y = (T^T T)^q T^T G with G of b + p columns; later steps
 * draw b fresh columns, apply (T22^T T22)^(q-1) T22^T, take X = T22 Y1, remove from X its component
 * along the recycled directions, orthonormalize, and apply T22^T once more to both blocks.  The left
 * singular vectors W_Y of the c x (b+p) sample (tall-thin SVD: HQR, then the SVD of the square R)
 * give V_i = HQR_full(W_Y(:, 1:b)), and W_next = V_i(:, b+1:c)^T W_Y(:, b+1:b+p) carries the rest.
 * Reading: W_next lives in the column (right-singular) space of the next T22, while X lives in its row
 * space; the printed lines use W_next where a row-space block is needed, which agrees in shape only
 * for m = n.  Here the recycled block enters the row space as Z = orth(T22 W_next), so the last
 * application of T22^T scales fresh and recycled samples alike: X <- X - Z Z^T X, Q = orth(X),
 * Y = T22^T [Q, Z].  With p = 0 the sampled subspace is that of randUTV_basic for the same q >= 1.
 * ------------------------------------------------------------------------------------------- */
/* Orthonormal basis (thin Q, rows x k) of the columns of X (rows x k, k <= rows), via HQR. */
static void thin_q(int64_t rows, int64_t k, const double* X, int64_t ldx, double* Q, int64_t ldq) {
  if (k <= 0) return;
  double* P = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)k);
  double* tau = (double*)malloc(sizeof(double) * (size_t)k);
  copy_block(rows, k, X, ldx, P, rows);
  orc_hqr(rows, k, P, rows, tau);
  orc_form_q(rows, k, k, P, rows, tau, Q, ldq);
  free(P);
  free(tau);
}

int orc_randutv_boosted(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, int64_t p,
                        uint64_t seed, double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                        int max_steps) {
  if (m < n || n < 1 || b < 1 || q < 0 || p < 0 || lda < m || ldu < m || ldt < m || ldv < n) return 1;
  int status = 0;
  copy_block(m, n, A, lda, T, ldt);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) U[IDX(i, j, ldu)] = (i == j) ? 1.0 : 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) V[IDX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;

  const int64_t steps_m = (m + b - 1) / b, steps_n = (n + b - 1) / b;
  const int64_t s = steps_m < steps_n ? steps_m : steps_n;
  const int64_t bp = b + p;
  double* G = (double*)malloc(sizeof(double) * (size_t)m * (size_t)bp);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n * (size_t)bp);
  double* Z = (double*)malloc(sizeof(double) * (size_t)m * (size_t)bp);
  double* X = (double*)malloc(sizeof(double) * (size_t)m * (size_t)bp);
  double* Qx = (double*)malloc(sizeof(double) * (size_t)m * (size_t)bp);
  double* Wn = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(p > 0 ? p : 1));
  double* Wy = (double*)malloc(sizeof(double) * (size_t)n * (size_t)bp);
  double* Py = (double*)malloc(sizeof(double) * (size_t)n * (size_t)bp);
  double* ty = (double*)malloc(sizeof(double) * (size_t)bp);
  double* Ry = (double*)malloc(sizeof(double) * (size_t)bp * (size_t)bp);
  double* Uy = (double*)malloc(sizeof(double) * (size_t)bp * (size_t)bp);
  double* Vy = (double*)malloc(sizeof(double) * (size_t)bp * (size_t)bp);
  double* sy = (double*)malloc(sizeof(double) * (size_t)bp);
  double* tauv = (double*)malloc(sizeof(double) * (size_t)b);
  double* tauu = (double*)malloc(sizeof(double) * (size_t)b);
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
  double* Rs = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double* Usm = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double* Vsm = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double* sig = (double*)malloc(sizeof(double) * (size_t)b);
  int have_next = 0;

  for (int64_t i = 1; i <= s; ++i) {
    if (max_steps > 0 && i > max_steps) break;
    const int64_t o = b * (i - 1);
    const int64_t r = m - o, c = n - o;
    double* T22 = T + IDX(o, o, ldt);
    if (b * i < m && b * i < n) {
      /* the sample has k columns: b + p, or fewer when the trailing block is narrower */
      const int64_t pk = (bp <= c) ? p : (c - b);
      const int64_t k = b + pk;
      if (i == 1 || !have_next || pk == 0) {
        /* G = randn(r, k); Y = T22^T G; Y = T22^T (T22 Y) q times (at step 1; later steps without a
         * recycled block fall back to this form with k = b). */
        const int64_t kk = (i == 1) ? k : b;
        orc_randn(r, kk, G, r, seed, (uint32_t)i, 1u);
        orc_gemm('T', 'N', c, kk, r, 1.0, T22, ldt, G, r, 0.0, Y, c);
        for (int j = 0; j < q; ++j) {
          orc_gemm('N', 'N', r, kk, c, 1.0, T22, ldt, Y, c, 0.0, Z, r);
          orc_gemm('T', 'N', c, kk, r, 1.0, T22, ldt, Z, r, 0.0, Y, c);
        }
        if (kk < k) { /* no recycled block available: sample the extra columns fresh as well */
          orc_randn(r, k, G, r, seed, (uint32_t)i, 3u);
          orc_gemm('T', 'N', c, k - kk, r, 1.0, T22, ldt, G + IDX(0, kk, r), r, 0.0, Y + IDX(0, kk, c), c);
          for (int j = 0; j < q; ++j) {
            orc_gemm('N', 'N', r, k - kk, c, 1.0, T22, ldt, Y + IDX(0, kk, c), c, 0.0, Z, r);
            orc_gemm('T', 'N', c, k - kk, r, 1.0, T22, ldt, Z, r, 0.0, Y + IDX(0, kk, c), c);
          }
        }
      } else {
        /* G = randn(r, b); Y1 = T22^T G; Y1 = T22^T (T22 Y1) q - 1 times; X = T22 Y1. */
        orc_randn(r, b, G, r, seed, (uint32_t)i, 1u);
        orc_gemm('T', 'N', c, b, r, 1.0, T22, ldt, G, r, 0.0, Y, c);
        for (int j = 0; j + 1 < q; ++j) {
          orc_gemm('N', 'N', r, b, c, 1.0, T22, ldt, Y, c, 0.0, Z, r);
          orc_gemm('T', 'N', c, b, r, 1.0, T22, ldt, Z, r, 0.0, Y, c);
        }
        orc_gemm('N', 'N', r, b, c, 1.0, T22, ldt, Y, c, 0.0, X, r);
        /* Z = orth(T22 W_next) (r x pk); X <- X - Z (Z^T X); Q = orth(X); Y = T22^T [Q, Z]. */
        orc_gemm('N', 'N', r, pk, c, 1.0, T22, ldt, Wn, c, 0.0, Qx, r);
        thin_q(r, pk, Qx, r, Z, r);
        double* ZtX = (double*)malloc(sizeof(double) * (size_t)pk * (size_t)b);
        orc_gemm('T', 'N', pk, b, r, 1.0, Z, r, X, r, 0.0, ZtX, pk);
        orc_gemm('N', 'N', r, b, pk, -1.0, Z, r, ZtX, pk, 1.0, X, r);
        free(ZtX);
        thin_q(r, b, X, r, Qx, r);
        copy_block(r, pk, Z, r, Qx + IDX(0, b, r), r);
        orc_gemm('T', 'N', c, k, r, 1.0, T22, ldt, Qx, r, 0.0, Y, c);
      }
      /* W_Y = left singular vectors of Y (c x k): HQR_full(Y) = Q_Y [R; 0], svd(R) = U_R D V_R^T,
       * W_Y(:, 1:k) = Q_Y(:, 1:k) U_R. */
      copy_block(c, k, Y, c, Py, c);
      orc_hqr(c, k, Py, c, ty);
      for (int64_t jj = 0; jj < k; ++jj)
        for (int64_t ii = 0; ii < k; ++ii) Ry[IDX(ii, jj, k)] = (ii <= jj) ? Py[IDX(ii, jj, c)] : 0.0;
      int st = orc_jacobi_svd(k, k, Ry, k, Uy, k, sy, Vy, k, NULL);
      if (st != 0) status = st;
      for (int64_t jj = 0; jj < k; ++jj)
        for (int64_t ii = 0; ii < c; ++ii) Wy[IDX(ii, jj, c)] = (ii < k) ? Uy[IDX(ii, jj, k)] : 0.0;
      orc_apply_q('L', 'N', c, k, k, Py, c, ty, Wy, c);
      /* [V_i, ~] = HQR_full(W_Y(:, 1:b)); T(:, J2 u J3) V_i; V(:, J2 u J3) V_i. */
      double* Yv = (double*)malloc(sizeof(double) * (size_t)c * (size_t)b);
      copy_block(c, b, Wy, c, Yv, c);
      orc_hqr(c, b, Yv, c, tauv);
      orc_apply_q('R', 'N', m, c, b, Yv, c, tauv, T + IDX(0, o, ldt), ldt);
      orc_apply_q('R', 'N', n, c, b, Yv, c, tauv, V + IDX(0, o, ldv), ldv);
      /* W_next = V_i(:, b+1:c)^T W_Y(:, b+1:b+pk): rows b..c-1 of V_i^T W_Y(:, b:k). */
      have_next = 0;
      if (pk > 0) {
        orc_apply_q('L', 'T', c, pk, b, Yv, c, tauv, Wy + IDX(0, b, c), c);
        for (int64_t jj = 0; jj < pk; ++jj)
          for (int64_t ii = 0; ii < c - b; ++ii) Wn[IDX(ii, jj, c - b)] = Wy[IDX(b + ii, b + jj, c)];
        have_next = 1;
      }
      free(Yv);
      /* The rest of the step is that of randUTV_basic. */
      copy_block(r, b, T22, ldt, P, r);
      orc_hqr(r, b, P, r, tauu);
      orc_apply_q('R', 'N', m, r, b, P, r, tauu, U + IDX(0, o, ldu), ldu);
      orc_apply_q('L', 'T', r, c - b, b, P, r, tauu, T + IDX(o, o + b, ldt), ldt);
      for (int64_t jj = 0; jj < b; ++jj)
        for (int64_t ii = 0; ii < b; ++ii) Rs[IDX(ii, jj, b)] = (ii <= jj) ? P[IDX(ii, jj, r)] : 0.0;
      for (int64_t jj = 0; jj < b; ++jj)
        for (int64_t ii = b; ii < r; ++ii) T[IDX(o + ii, o + jj, ldt)] = 0.0;
      st = orc_jacobi_svd(b, b, Rs, b, Usm, b, sig, Vsm, b, NULL);
      if (st != 0) status = st;
      right_mul_small(m, b, U + IDX(0, o, ldu), ldu, Usm, b);
      right_mul_small(n, b, V + IDX(0, o, ldv), ldv, Vsm, b);
      for (int64_t jj = 0; jj < b; ++jj)
        for (int64_t ii = 0; ii < b; ++ii) T[IDX(o + ii, o + jj, ldt)] = (ii == jj) ? sig[ii] : 0.0;
      left_mul_small_t(b, c - b, T + IDX(o, o + b, ldt), ldt, Usm, b);
      right_mul_small(o, b, T + IDX(0, o, ldt), ldt, Vsm, b);
    } else {
      /* Final block, as in randUTV_basic. */
      double* Uf = (double*)malloc(sizeof(double) * (size_t)r * (size_t)c);
      double* Vf = (double*)malloc(sizeof(double) * (size_t)c * (size_t)c);
      double* sf = (double*)malloc(sizeof(double) * (size_t)c);
      int st;
      if (r > c) {
        double* Pf = (double*)malloc(sizeof(double) * (size_t)r * (size_t)c);
        double* tf = (double*)malloc(sizeof(double) * (size_t)c);
        double* Rf = (double*)malloc(sizeof(double) * (size_t)c * (size_t)c);
        copy_block(r, c, T22, ldt, Pf, r);
        orc_hqr(r, c, Pf, r, tf);
        for (int64_t jj = 0; jj < c; ++jj)
          for (int64_t ii = 0; ii < c; ++ii) Rf[IDX(ii, jj, c)] = (ii <= jj) ? Pf[IDX(ii, jj, r)] : 0.0;
        st = orc_jacobi_svd(c, c, Rf, c, Uf, c, sf, Vf, c, NULL);
        orc_apply_q('R', 'N', m, r, c, Pf, r, tf, U + IDX(0, o, ldu), ldu);
        right_mul_small(m, c, U + IDX(0, o, ldu), ldu, Uf, c);
        free(Pf);
        free(tf);
        free(Rf);
      } else {
        st = orc_jacobi_svd(r, c, T22, ldt, Uf, r, sf, Vf, c, NULL);
        right_mul_small(m, c, U + IDX(0, o, ldu), ldu, Uf, r);
      }
      if (st != 0) status = st;
      right_mul_small(n, c, V + IDX(0, o, ldv), ldv, Vf, c);
      for (int64_t jj = 0; jj < c; ++jj)
        for (int64_t ii = 0; ii < r; ++ii) T[IDX(o + ii, o + jj, ldt)] = (ii == jj) ? sf[ii] : 0.0;
      right_mul_small(o, c, T + IDX(0, o, ldt), ldt, Vf, c);
      free(Uf);
      free(Vf);
      free(sf);
    }
  }
  free(G); free(Y); free(Z); free(X); free(Qx); free(Wn); free(Wy); free(Py); free(ty); free(Ry);
  free(Uy); free(Vy); free(sy); free(tauv); free(tauu); free(P); free(Rs); free(Usm); free(Vsm); free(sig);
  return status;
}

/* ---------------------------------------------------------------------------------------------
 * powerURV (Algorithm 1): V = randn(n, n); q times { Yh = A V; Vh = HQR_thin(Yh); Y = A^T Vh;
 * V = HQR_thin(Y) }; Ah = A V; [U, R] = HQR_full(Ah).  For q = 0, V = Q of HQR_full(G) (RURV, Sec. 3.1).
 * ------------------------------------------------------------------------------------------- */
int orc_powerurv(int64_t m, int64_t n, const double* A, int64_t lda, int q, uint64_t seed, double* U,
                 int64_t ldu, double* R, int64_t ldr, double* V, int64_t ldv) {
  if (m < n || n < 1 || q < 0 || lda < m || ldu < m || ldr < m || ldv < n) return 1;
  double* W = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  double* tau = (double*)malloc(sizeof(double) * (size_t)n);
  orc_randn(n, n, V, ldv, seed, 0u, 2u);
  if (q == 0) {
    copy_block(n, n, V, ldv, W, n);
    orc_hqr(n, n, W, n, tau);
    orc_form_q(n, n, n, W, n, tau, V, ldv);
  }
  for (int it = 0; it < q; ++it) {
    orc_gemm('N', 'N', m, n, n, 1.0, A, lda, V, ldv, 0.0, W, m);     /* Yh = A V        */
    orc_hqr(m, n, W, m, tau);                                         /* Vh = HQR_thin(Yh) */
    orc_form_q(m, n, n, W, m, tau, R, ldr);                           /* (R holds Vh)    */
    orc_gemm('T', 'N', n, n, m, 1.0, A, lda, R, ldr, 0.0, W, n);      /* Y = A^T Vh      */
    orc_hqr(n, n, W, n, tau);                                         /* V = HQR_thin(Y) */
    orc_form_q(n, n, n, W, n, tau, V, ldv);
  }
  orc_gemm('N', 'N', m, n, n, 1.0, A, lda, V, ldv, 0.0, R, ldr);      /* Ah = A V        */
  orc_hqr(m, n, R, ldr, tau);                                         /* [U, R] = HQR_full(Ah) */
  orc_form_q(m, m, n, R, ldr, tau, U, ldu);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = j + 1; i < m; ++i) R[IDX(i, j, ldr)] = 0.0;
  free(W);
  free(tau);
  return 0;
}
