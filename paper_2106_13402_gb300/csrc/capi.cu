// capi.cu -- the remaining C-ABI entry points: building blocks exported for testing, status helpers,
// and the host-buffer forms of the two factorizations.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "rrf_internal.cuh"

namespace rrf {

namespace {
thread_local int g_arg_error = 0;
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_inject_kind{0};
std::atomic<long long> g_inject_value{0};
}
Inject inject_state() {
  Inject x;
  x.kind = g_inject_kind.load(std::memory_order_relaxed);
  x.value = g_inject_value.load(std::memory_order_relaxed);
  return x;
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_arg_error(int pos) { g_arg_error = pos; }
void clear_arg_error() { g_arg_error = 0; }

const DevInfo& dev_info() {
  static DevInfo info[64];
  static bool have[64] = {};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    cudaDeviceGetAttribute(&info[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&info[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&info[dev].cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&info[dev].cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (info[dev].sms <= 0) info[dev].sms = 1;
    have[dev] = true;
  }
  return info[dev];
}

}  // namespace rrf

using namespace rrf;

extern "C" const char* rrf_status_string(rrf_status s) {
  switch (s) {
    case RRF_OK: return "RRF_OK";
    case RRF_INVALID_ARG: return "RRF_INVALID_ARG";
    case RRF_CUDA_ERROR: return "RRF_CUDA_ERROR";
    case RRF_NOT_CONVERGED: return "RRF_NOT_CONVERGED";
    case RRF_TIMEOUT: return "RRF_TIMEOUT";
    case RRF_NUMERICAL: return "RRF_NUMERICAL";
    case RRF_UNSUPPORTED: return "RRF_UNSUPPORTED";
    case RRF_WORKSPACE_TOO_SMALL: return "RRF_WORKSPACE_TOO_SMALL";
  }
  return "RRF_UNKNOWN";
}

extern "C" int rrf_last_arg_error(void) { return g_arg_error; }

extern "C" rrf_status rrf_test_inject(int kind, long long value) {
  clear_arg_error();
  if (kind < RRF_INJECT_NONE || kind > RRF_INJECT_JACOBI_CAP) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (kind != RRF_INJECT_NONE && value < 1) { set_arg_error(2); return RRF_INVALID_ARG; }
  g_inject_value.store(kind == RRF_INJECT_NONE ? 0 : value);
  g_inject_kind.store(kind);
  return RRF_OK;
}

extern "C" int64_t rrf_launch_count(void) { return g_launches.load(); }

extern "C" const char* rrf_version(void) { return "rrf-gb300 0.1 (sm_103a)"; }

extern "C" rrf_status rrf_workspace_status(void* workspace, void* stream) {
  if (workspace == nullptr) return RRF_INVALID_ARG;
  int st = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RRF_CUDA_TRY(cudaMemcpyAsync(&st, workspace, sizeof(int), cudaMemcpyDeviceToHost, s));
  RRF_CUDA_TRY(cudaStreamSynchronize(s));
  return static_cast<rrf_status>(st);
}

extern "C" rrf_status rrf_randn(int64_t rows, int64_t cols, double* G, int64_t ldg, uint64_t seed, uint32_t step,
                                uint32_t tag, void* stream) {
  clear_arg_error();
  if (rows < 0) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (cols < 0) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (G == nullptr && rows * cols > 0) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (ldg < std::max<int64_t>(rows, 1)) { set_arg_error(4); return RRF_INVALID_ARG; }
  RRF_CUDA_TRY(randn_f64(rows, cols, G, ldg, seed, step, tag, reinterpret_cast<cudaStream_t>(stream)));
  return RRF_OK;
}

extern "C" size_t rrf_gemm_workspace(int64_t m, int64_t n, int64_t k) {
  GemmDesc g;
  g.M = m; g.N = n; g.K = k;
  return gemm_scratch_bytes(&g, 1);
}

extern "C" rrf_status rrf_gemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                               int64_t ldc, void* workspace, size_t ws_bytes, void* stream) {
  clear_arg_error();
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') { set_arg_error(1); return RRF_INVALID_ARG; }
  if (!tb && transb != 'N' && transb != 'n') { set_arg_error(2); return RRF_INVALID_ARG; }
  if (m < 0) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (n < 0) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (k < 0) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (lda < std::max<int64_t>(1, ta ? k : m)) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (ldb < std::max<int64_t>(1, tb ? n : k)) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (ldc < std::max<int64_t>(1, m)) { set_arg_error(13); return RRF_INVALID_ARG; }
  GemmDesc g;
  g.M = m; g.N = n; g.K = k;
  g.A = A; g.lda = lda; g.ta = ta;
  g.B = B; g.ldb = ldb; g.tb = tb;
  g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta;
  RRF_CUDA_TRY(gemm_f64(&g, 1, reinterpret_cast<double*>(workspace), workspace ? ws_bytes : 0,
                        reinterpret_cast<cudaStream_t>(stream)));
  return RRF_OK;
}

// ---- rank-k approximation of a (partial) randUTV factorization (Sec. 4.1) ------------------------------
namespace {
void low_rank_descs(int64_t m, int64_t n, int64_t k, const double* U, int64_t ldu, const double* T, int64_t ldt,
                    const double* V, int64_t ldv, double* X, double* Ak, int64_t ldak, GemmDesc* g) {
  g[0].M = k; g[0].N = n; g[0].K = n;  // X = T(0:k, :) V^T
  g[0].A = T; g[0].lda = ldt; g[0].ta = 0;
  g[0].B = V; g[0].ldb = ldv; g[0].tb = 1;
  g[0].C = X; g[0].ldc = std::max<int64_t>(k, 1);
  g[1].M = m; g[1].N = n; g[1].K = k;  // Ak = U(:, 0:k) X
  g[1].A = U; g[1].lda = ldu; g[1].ta = 0;
  g[1].B = X; g[1].ldb = std::max<int64_t>(k, 1); g[1].tb = 0;
  g[1].C = Ak; g[1].ldc = ldak;
}
}  // namespace

extern "C" size_t rrf_low_rank_workspace(int64_t m, int64_t n, int64_t k) {
  if (m < 1 || n < 1 || k < 0) return 0;
  GemmDesc g[2];
  low_rank_descs(m, n, k, nullptr, m, nullptr, m, nullptr, n, nullptr, nullptr, m, g);
  return align_up(sizeof(double) * (size_t)std::max<int64_t>(k, 1) * (size_t)n, 256) +
         std::max(gemm_scratch_bytes(&g[0], 1), gemm_scratch_bytes(&g[1], 1));
}

extern "C" rrf_status rrf_low_rank(int64_t m, int64_t n, int64_t k, const double* U, int64_t ldu, const double* T,
                                   int64_t ldt, const double* V, int64_t ldv, double* Ak, int64_t ldak,
                                   void* workspace, size_t ws_bytes, void* stream) {
  clear_arg_error();
  if (m < 1) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (n < 1) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (k < 0 || k > std::min(m, n)) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (U == nullptr) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (ldu < m) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (T == nullptr) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (ldt < m) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (V == nullptr) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (ldv < n) { set_arg_error(9); return RRF_INVALID_ARG; }
  if (Ak == nullptr) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (ldak < m) { set_arg_error(11); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(12);
    return RRF_INVALID_ARG;
  }
  if (ws_bytes < rrf_low_rank_workspace(m, n, k)) { set_arg_error(13); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (k == 0) {
    RRF_CUDA_TRY(zero_matrix(m, n, Ak, ldak, s));
    return RRF_OK;
  }
  double* X = reinterpret_cast<double*>(workspace);
  const size_t xb = align_up(sizeof(double) * (size_t)k * (size_t)n, 256);
  double* scratch = reinterpret_cast<double*>(reinterpret_cast<char*>(workspace) + xb);
  GemmDesc g[2];
  low_rank_descs(m, n, k, U, ldu, T, ldt, V, ldv, X, Ak, ldak, g);
  RRF_CUDA_TRY(gemm_f64(&g[0], 1, scratch, ws_bytes - xb, s));
  RRF_CUDA_TRY(gemm_f64(&g[1], 1, scratch, ws_bytes - xb, s));
  return RRF_OK;
}

extern "C" size_t rrf_gemm_bf16_workspace(int64_t m, int64_t n, int64_t k) {
  if (m < 1 || n < 1) return kHeaderBytes;
  return kHeaderBytes + tc_part_bytes(m, n, k);
}

extern "C" rrf_status rrf_gemm_bf16(int64_t m, int64_t n, int64_t k, double alpha, const uint16_t* A, int64_t lda,
                                    const uint16_t* B, int64_t ldb, double* D, int64_t ldd, void* workspace,
                                    size_t ws_bytes, void* stream) {
  clear_arg_error();
  if (m < 1) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (n < 1 || n > 256) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (k < 0) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (A == nullptr || (reinterpret_cast<uintptr_t>(A) & 15) != 0) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (lda < std::max<int64_t>(k, 1) || (lda % 8) != 0) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (B == nullptr || (reinterpret_cast<uintptr_t>(B) & 15) != 0) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (ldb < std::max<int64_t>(k, 1) || (ldb % 8) != 0) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (D == nullptr) { set_arg_error(9); return RRF_INVALID_ARG; }
  if (ldd < m) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(11);
    return RRF_INVALID_ARG;
  }
  if (ws_bytes < rrf_gemm_bf16_workspace(m, n, k)) { set_arg_error(12); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(workspace);
  RRF_CUDA_TRY(cudaMemsetAsync(hdr, 0, kHeaderBytes, s));
  RRF_CUDA_TRY(gemm_bf16_tn(m, n, k, reinterpret_cast<const __nv_bfloat16*>(A), lda,
                            reinterpret_cast<const __nv_bfloat16*>(B), ldb, alpha, D, ldd,
                            reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + kHeaderBytes),
                            ws_bytes - kHeaderBytes, &hdr->status, s));
  return RRF_OK;
}

extern "C" size_t rrf_panel_qr_workspace(int64_t r, int64_t w) {
  return kHeaderBytes + align_up(panel_scratch_bytes(r, w), 256);
}

extern "C" rrf_status rrf_panel_qr(int64_t r, int64_t w, double* P, int64_t ldp, double* tau, double* Y,
                                   int64_t ldy, double* Tf, int64_t ldtf, void* workspace, size_t ws_bytes,
                                   void* stream) {
  clear_arg_error();
  if (r < 1) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (w < 1 || w > 256 || w > r) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (P == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (ldp < r) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (tau == nullptr) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (Y == nullptr) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (ldy < r) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (Tf != nullptr && ldtf < w) { set_arg_error(9); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(10);
    return RRF_INVALID_ARG;
  }
  if (ws_bytes < rrf_panel_qr_workspace(r, w)) { set_arg_error(11); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(workspace);
  RRF_CUDA_TRY(cudaMemsetAsync(hdr, 0, kHeaderBytes, s));
  RRF_CUDA_TRY(panel_qr(r, w, P, ldp, tau, Y, ldy, Tf, ldtf, nullptr, 0,
                        reinterpret_cast<double*>(reinterpret_cast<char*>(workspace) + kHeaderBytes),
                        ws_bytes - kHeaderBytes, hdr, s));
  return RRF_OK;
}

extern "C" size_t rrf_jacobi_svd_workspace(int64_t c) {
  return kHeaderBytes + (c >= 1 && c <= 256 ? jacobi_scratch_bytes(c) : 0);
}

extern "C" rrf_status rrf_jacobi_svd(int64_t c, const double* M, int64_t ldm, double* Us, int64_t ldu, double* s,
                                     double* Vs, int64_t ldv, void* workspace, size_t ws_bytes, void* stream) {
  clear_arg_error();
  if (c < 1 || c > 256) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (M == nullptr) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (ldm < c) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (Us == nullptr) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (ldu < c) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (s == nullptr) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (Vs == nullptr) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (ldv < c) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(9);
    return RRF_INVALID_ARG;
  }
  if (ws_bytes < kHeaderBytes) { set_arg_error(10); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(workspace);
  RRF_CUDA_TRY(cudaMemsetAsync(hdr, 0, kHeaderBytes, st));
  RRF_CUDA_TRY(jacobi_svd(c, M, ldm, Us, ldu, s, Vs, ldv, hdr, st,
                          reinterpret_cast<double*>(reinterpret_cast<char*>(workspace) + kHeaderBytes),
                          ws_bytes - kHeaderBytes));
  return RRF_OK;
}

// ---- m < n: factor A^T and transpose the result (Sec. 1.3 footnote) ---------------------------------------
namespace rrf {

size_t wide_workspace(WsFn wsfn, int64_t m, int64_t n, int64_t b, const rrf_opts* opts) {
  const size_t inner = wsfn(n, m, b, opts);
  if (inner == 0) return 0;
  return align_up(inner, 256) + 2 * align_up(sizeof(double) * (size_t)m * (size_t)n, 256);
}

rrf_status factor_wide(WsFn wsfn, RunFn run, int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                       double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, uint64_t seed,
                       void* workspace, size_t ws_bytes, const rrf_opts* opts, void* stream_) {
  clear_arg_error();
  if (A == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (lda < m) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (b < 1 || b > 256) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (U == nullptr) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (ldu < m) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (T == nullptr) { set_arg_error(9); return RRF_INVALID_ARG; }
  if (ldt < m) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (V == nullptr) { set_arg_error(11); return RRF_INVALID_ARG; }
  if (ldv < n) { set_arg_error(12); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(14);
    return RRF_INVALID_ARG;
  }
  if (opts != nullptr && opts->resume_steps != 0) { set_arg_error(16); return RRF_UNSUPPORTED; }  // state is A^T's
  const size_t inner = wsfn(n, m, b, opts);
  double* At = reinterpret_cast<double*>(reinterpret_cast<char*>(workspace) + align_up(inner, 256));
  double* Tt = reinterpret_cast<double*>(reinterpret_cast<char*>(At) +
                                         align_up(sizeof(double) * (size_t)m * (size_t)n, 256));
  // The tall call checks q and the options on the buffers it will get; with no workspace it stops before
  // enqueuing anything (nothing is dereferenced).
  const rrf_status v = run(n, m, At, n, b, q, V, ldv, Tt, n, U, ldu, seed, workspace, 0, opts, stream_);
  if (v != RRF_WORKSPACE_TOO_SMALL && v != RRF_OK) return v;
  clear_arg_error();
  if (ws_bytes < wide_workspace(wsfn, m, n, b, opts)) { set_arg_error(15); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  RRF_CUDA_TRY(transpose_matrix(m, n, A, lda, At, n, s));
  // A^T (n x m, tall) = U' T' V'^T: U' (n x n) lands in V, V' (m x m) in U.
  const rrf_status r = run(n, m, At, n, b, q, V, ldv, Tt, n, U, ldu, seed, workspace, inner, opts, stream_);
  if (r != RRF_OK) return r;
  RRF_CUDA_TRY(transpose_matrix(n, m, Tt, n, T, ldt, s));
  return RRF_OK;
}

}  // namespace rrf

// ---- host-buffer forms -----------------------------------------------------------------------------
namespace {

rrf_status run_host(WsFn wsfn, RunFn run, int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                    double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, uint64_t seed,
                    const rrf_opts* opts, void* stream_) {
  clear_arg_error();
  if (m < 1 || n < 1) { set_arg_error(m < 1 ? 1 : 2); return RRF_INVALID_ARG; }
  if (A == nullptr || lda < m) { set_arg_error(A == nullptr ? 3 : 4); return RRF_INVALID_ARG; }
  if (U == nullptr || ldu < m) { set_arg_error(U == nullptr ? 7 : 8); return RRF_INVALID_ARG; }
  if (T == nullptr || ldt < m) { set_arg_error(T == nullptr ? 9 : 10); return RRF_INVALID_ARG; }
  if (V == nullptr || ldv < n) { set_arg_error(V == nullptr ? 11 : 12); return RRF_INVALID_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  const size_t ws = wsfn(m, n, b, opts);
  double *dA = nullptr, *dU = nullptr, *dT = nullptr, *dV = nullptr;
  void* dW = nullptr;
  rrf_status st = RRF_OK;
  auto fail = [&](rrf_status x) { if (st == RRF_OK) st = x; };
  if (cudaMallocAsync((void**)&dA, sizeof(double) * m * n, s) != cudaSuccess ||
      cudaMallocAsync((void**)&dU, sizeof(double) * m * m, s) != cudaSuccess ||
      cudaMallocAsync((void**)&dT, sizeof(double) * m * n, s) != cudaSuccess ||
      cudaMallocAsync((void**)&dV, sizeof(double) * n * n, s) != cudaSuccess ||
      cudaMallocAsync(&dW, ws + 256, s) != cudaSuccess) {
    fail(RRF_CUDA_ERROR);
  }
  if (st == RRF_OK) {
    if (cudaMemcpy2DAsync(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                          cudaMemcpyHostToDevice, s) != cudaSuccess)
      fail(RRF_CUDA_ERROR);
  }
  void* wsa = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(dW) + 255) & ~uintptr_t(255));
  if (st == RRF_OK) {
    rrf_status r = run(m, n, dA, m, b, q, dU, m, dT, m, dV, n, seed, wsa, ws, opts, s);
    if (r != RRF_OK) fail(r);
  }
  if (st == RRF_OK) {
    if (cudaMemcpy2DAsync(U, sizeof(double) * ldu, dU, sizeof(double) * m, sizeof(double) * m, m,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpy2DAsync(T, sizeof(double) * ldt, dT, sizeof(double) * m, sizeof(double) * m, n,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpy2DAsync(V, sizeof(double) * ldv, dV, sizeof(double) * n, sizeof(double) * n, n,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess)
      fail(RRF_CUDA_ERROR);
  }
  int dev_status = 0;
  if (st == RRF_OK && cudaMemcpyAsync(&dev_status, wsa, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    fail(RRF_CUDA_ERROR);
  if (dA) cudaFreeAsync(dA, s);
  if (dU) cudaFreeAsync(dU, s);
  if (dT) cudaFreeAsync(dT, s);
  if (dV) cudaFreeAsync(dV, s);
  if (dW) cudaFreeAsync(dW, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) fail(RRF_CUDA_ERROR);
  if (st == RRF_OK && dev_status != 0) st = static_cast<rrf_status>(dev_status);
  return st;
}

}  // namespace

extern "C" rrf_status rrf_randutv_host(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                                       double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                                       uint64_t seed, const rrf_opts* opts, void* stream) {
  return run_host(rrf_randutv_workspace, rrf_randutv, m, n, A, lda, b, q, U, ldu, T, ldt, V, ldv, seed, opts,
                  stream);
}

extern "C" rrf_status rrf_powerurv_host(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                                        double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                                        uint64_t seed, const rrf_opts* opts, void* stream) {
  return run_host(rrf_powerurv_workspace, rrf_powerurv, m, n, A, lda, b, q, U, ldu, T, ldt, V, ldv, seed, opts,
                  stream);
}
