// powerurv.cu -- host driver of powerURV (Algorithm 1) on one GPU.
//
//   V = randn(n, n)
//   q times: Yh = A V; Vh = HQR_thin(Yh); Y = A^T Vh; V = HQR_thin(Y)
//   Ah = A V; [U, R] = HQR_full(Ah)
// (q = 0: V = Q of HQR_full(G), i.e. RURV, Sec. 3.1.)  Householder QRs are blocked: panels of width
// b go through the cooperative panel kernel, the trailing matrix is updated with the compact-WY form
// (I - Y Tf^T Y^T) C, and explicit Q factors are formed by applying the stored panels to the identity
// in reverse order.  All products run through the FP64 GEMM.
#include <algorithm>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

struct PWs {
  WsHeader* hdr = nullptr;
  double *W = nullptr, *Ys = nullptr, *tau = nullptr, *Tall = nullptr, *Wa = nullptr, *Wb = nullptr;
  double* panel = nullptr;
  size_t panel_bytes = 0;
  double* gemm = nullptr;
  size_t gemm_bytes = 0;
  GemmEngine eng;
};

size_t layout(int64_t m, int64_t n, int64_t b, int gemm_mode, Arena& ar, PWs& w) {
  const int64_t mx = std::max(m, n);
  const int64_t nblk = (n + b - 1) / b;
  w.hdr = reinterpret_cast<WsHeader*>(ar.take<char>(kHeaderBytes));
  w.W = ar.take<double>(m * n);
  w.Ys = ar.take<double>(m * n);
  w.tau = ar.take<double>(n);
  w.Tall = ar.take<double>(nblk * b * b);
  w.Wa = ar.take<double>(b * mx);
  w.Wb = ar.take<double>(b * mx);
  w.panel_bytes = panel_scratch_bytes(mx, b);
  w.panel = reinterpret_cast<double*>(ar.take<char>(w.panel_bytes));
  w.gemm_bytes = (size_t)16 * mx * b * sizeof(double);
  w.gemm = reinterpret_cast<double*>(ar.take<char>(w.gemm_bytes));
  w.eng.scratch = w.gemm;
  w.eng.scratch_bytes = w.gemm_bytes;
  w.eng.status = w.hdr ? &w.hdr->status : nullptr;
  w.eng.emulate = gemm_mode != RRF_GEMM_NATIVE;
  w.eng.force = gemm_mode == RRF_GEMM_EMULATED;
  if (w.eng.emulate) {
    w.eng.oz_bytes = ozaki_bound(m, n, b);
    w.eng.oz = ar.take<char>(w.eng.oz_bytes);
  }
  return ar.off;
}

GemmDesc gd(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, int ta, const double* B,
            int64_t ldb, int tb, double* C, int64_t ldc, double alpha = 1.0, double beta = 0.0) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.ta = ta;
  g.B = B; g.ldb = ldb; g.tb = tb;
  g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta;
  return g;
}

// Blocked Householder QR of the rows x cols matrix X (in place, R above the diagonal).  Panel j's
// explicit reflectors go to Ys(j0:, j0:j0+w) and its compact-WY factor to Tall[j].
cudaError_t blocked_hqr(int64_t rows, int64_t cols, double* X, int64_t ldx, int64_t b, const PWs& w,
                        cudaStream_t s) {
  for (int64_t j0 = 0; j0 < cols; j0 += b) {
    const int64_t wd = std::min(b, cols - j0);
    const int64_t rr = rows - j0;
    double* Yj = w.Ys + j0 + j0 * rows;
    double* Tj = w.Tall + (j0 / b) * b * b;
    cudaError_t e = panel_qr(rr, wd, X + j0 + j0 * ldx, ldx, w.tau + j0, Yj, rows, Tj, b, nullptr, 0,
                             w.panel, w.panel_bytes, w.hdr, s, &w.eng);
    if (e != cudaSuccess) return e;
    const int64_t nc = cols - j0 - wd;
    if (nc <= 0) continue;
    double* C = X + j0 + (j0 + wd) * ldx;
    GemmDesc g1 = gd(wd, nc, rr, Yj, rows, 1, C, ldx, 0, w.Wa, b);
    if ((e = gemm_run(w.eng, &g1, 1, s)) != cudaSuccess) return e;
    GemmDesc g2 = gd(wd, nc, wd, Tj, b, 1, w.Wa, b, 0, w.Wb, b);
    if ((e = gemm_run(w.eng, &g2, 1, s)) != cudaSuccess) return e;
    GemmDesc g3 = gd(rr, nc, wd, Yj, rows, 0, w.Wb, b, 0, C, ldx, -1.0, 1.0);
    if ((e = gemm_run(w.eng, &g3, 1, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Q(:, 0:ncols) of the factorization stored by blocked_hqr (k factored columns).
cudaError_t form_q(int64_t rows, int64_t ncols, int64_t k, int64_t b, double* Q, int64_t ldq, const PWs& w,
                   cudaStream_t s) {
  cudaError_t e = fill_identity(rows, ncols, Q, ldq, s);
  if (e != cudaSuccess) return e;
  const int64_t nblk = (k + b - 1) / b;
  for (int64_t jb = nblk - 1; jb >= 0; --jb) {
    const int64_t j0 = jb * b;
    const int64_t wd = std::min(b, k - j0);
    const int64_t rr = rows - j0;
    const int64_t nc = ncols - j0;
    if (nc <= 0) continue;
    const double* Yj = w.Ys + j0 + j0 * rows;
    const double* Tj = w.Tall + jb * b * b;
    double* C = Q + j0 + j0 * ldq;
    GemmDesc g1 = gd(wd, nc, rr, Yj, rows, 1, C, ldq, 0, w.Wa, b);
    if ((e = gemm_run(w.eng, &g1, 1, s)) != cudaSuccess) return e;
    GemmDesc g2 = gd(wd, nc, wd, Tj, b, 0, w.Wa, b, 0, w.Wb, b);
    if ((e = gemm_run(w.eng, &g2, 1, s)) != cudaSuccess) return e;
    GemmDesc g3 = gd(rr, nc, wd, Yj, rows, 0, w.Wb, b, 0, C, ldq, -1.0, 1.0);
    if ((e = gemm_run(w.eng, &g3, 1, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace rrf

using namespace rrf;

extern "C" size_t rrf_powerurv_workspace(int64_t m, int64_t n, int64_t b, const rrf_opts* opts) {
  if (m < 1 || n < 1 || b < 1) return 0;
  if (m < n) return wide_workspace(rrf_powerurv_workspace, m, n, b, opts);
  Arena ar;
  PWs w;
  return layout(m, n, b, opts ? opts->gemm_mode : RRF_GEMM_AUTO, ar, w);
}

extern "C" rrf_status rrf_powerurv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                                   double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                                   uint64_t seed, void* workspace, size_t ws_bytes, const rrf_opts* opts,
                                   void* stream_) {
  clear_arg_error();
  if (m < 1) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (n < 1) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (m < n)  // wide: factor A^T and transpose the result
    return factor_wide(rrf_powerurv_workspace, rrf_powerurv, m, n, A, lda, b, q, U, ldu, T, ldt, V, ldv, seed,
                       workspace, ws_bytes, opts, stream_);
  if (A == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (lda < m) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (b < 1 || b > 256) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (q < 0 || q > 16) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (U == nullptr) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (ldu < m) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (T == nullptr) { set_arg_error(9); return RRF_INVALID_ARG; }
  if (ldt < m) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (V == nullptr) { set_arg_error(11); return RRF_INVALID_ARG; }
  if (ldv < n) { set_arg_error(12); return RRF_INVALID_ARG; }
  if (T == A) { set_arg_error(9); return RRF_INVALID_ARG; }  // A is read after T is written
  if (opts != nullptr && (opts->sketch_prec != RRF_SKETCH_FP64 || opts->q_per_block != nullptr ||
                          opts->q_policy != RRF_Q_FIXED || opts->gemm_mode < RRF_GEMM_AUTO ||
                          opts->gemm_mode > RRF_GEMM_EMULATED || opts->oversample != 0 ||
                          opts->frob_tol != 0.0 || opts->frob_out != nullptr || opts->steps_out != nullptr ||
                          opts->resume_steps != 0)) {
    set_arg_error(16);
    return RRF_UNSUPPORTED;
  }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(14);
    return RRF_INVALID_ARG;
  }
  if (ws_bytes < rrf_powerurv_workspace(m, n, b, opts)) {
    set_arg_error(15);
    return RRF_WORKSPACE_TOO_SMALL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  Arena ar;
  ar.base = reinterpret_cast<char*>(workspace);
  ar.cap = ws_bytes;
  PWs w;
  layout(m, n, b, opts ? opts->gemm_mode : RRF_GEMM_AUTO, ar, w);
  if (ar.overflow) return RRF_WORKSPACE_TOO_SMALL;

  RRF_CUDA_TRY(cudaMemsetAsync(w.hdr, 0, kHeaderBytes, s));
  RRF_CUDA_TRY(check_finite(m, n, A, lda, &w.hdr->status, s));
  // V = randn(n, n).
  RRF_CUDA_TRY(randn_f64(n, n, V, ldv, seed, 0u, 2u, s));
  if (q == 0) {
    RRF_CUDA_TRY(copy_matrix(n, n, V, ldv, w.W, n, s));
    RRF_CUDA_TRY(blocked_hqr(n, n, w.W, n, b, w, s));
    RRF_CUDA_TRY(form_q(n, n, n, b, V, ldv, w, s));
  }
  for (int it = 0; it < q; ++it) {
    GemmDesc g1 = gd(m, n, n, A, lda, 0, V, ldv, 0, w.W, m);           // Yh = A V
    RRF_CUDA_TRY(gemm_run(w.eng, &g1, 1, s));
    RRF_CUDA_TRY(blocked_hqr(m, n, w.W, m, b, w, s));                  // Vh = HQR_thin(Yh) -> T
    RRF_CUDA_TRY(form_q(m, n, n, b, T, ldt, w, s));
    GemmDesc g2 = gd(n, n, m, A, lda, 1, T, ldt, 0, w.W, n);           // Y = A^T Vh
    RRF_CUDA_TRY(gemm_run(w.eng, &g2, 1, s));
    RRF_CUDA_TRY(blocked_hqr(n, n, w.W, n, b, w, s));                  // V = HQR_thin(Y)
    RRF_CUDA_TRY(form_q(n, n, n, b, V, ldv, w, s));
  }
  GemmDesc g3 = gd(m, n, n, A, lda, 0, V, ldv, 0, T, ldt);             // Ah = A V
  RRF_CUDA_TRY(gemm_run(w.eng, &g3, 1, s));
  RRF_CUDA_TRY(blocked_hqr(m, n, T, ldt, b, w, s));                    // [U, R] = HQR_full(Ah)
  RRF_CUDA_TRY(form_q(m, m, n, b, U, ldu, w, s));
  RRF_CUDA_TRY(zero_lower(m, n, T, ldt, s));
  return RRF_OK;
}
