// rrf_internal.cuh -- shared declarations of the CUDA path (device kernels live in their own .cu files).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include "../../include/rrf.h"

namespace rrf {

// ---- workspace header (first 256 bytes of every workspace) -------------------------------------
// word 0: device status (first error wins).  Words 16..: grid-barrier counters (zeroed per call).
constexpr size_t kHeaderBytes = 256;
struct WsHeader {
  int status;
  int pad0[15];
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int pad1[14];
  int flags[32];  // per-call scratch flags (e.g. "a zero singular value was met")
};
static_assert(sizeof(WsHeader) <= kHeaderBytes, "header too large");

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-owned device workspace (host-side bookkeeping only).
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  size_t cap = 0;
  bool overflow = false;
  template <class T>
  T* take(size_t count) {
    size_t bytes = align_up(count * sizeof(T), 256);
    if (base == nullptr) {  // size query
      off += bytes;
      return nullptr;
    }
    if (off + bytes > cap) {
      overflow = true;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// ---- per-device properties -----------------------------------------------------------------------
struct DevInfo {
  int sms = 0;
  int smem_optin = 0;
  int cc_major = 0, cc_minor = 0;
};
const DevInfo& dev_info();

// ---- launch accounting (every kernel launch of the library calls this once) -------------------------
void count_launch();
// adjust the counter by n (negative for captured-but-not-launched kernels, positive per graph replay)
void add_launches(int64_t n);

// ---- failure injection for tests (rrf_test_inject): kind RRF_INJECT_*, and its value ------------------
struct Inject {
  int kind = 0;
  long long value = 0;
};
Inject inject_state();

// ---- thread-local argument-error slot ------------------------------------------------------------
void set_arg_error(int pos);
void clear_arg_error();

// ---- FP64 GEMM (gemm_f64.cu) ---------------------------------------------------------------------
struct GemmDesc {
  int64_t M = 0, N = 0, K = 0;
  const double* A = nullptr;
  int64_t lda = 0;
  int ta = 0;  // 1: op(A) = A^T
  const double* B = nullptr;
  int64_t ldb = 0;
  int tb = 0;
  double* C = nullptr;
  int64_t ldc = 0;
  double alpha = 1.0, beta = 0.0;
};
// Bytes of split-K scratch the planner may use for one batch of problems.
size_t gemm_scratch_bytes(const GemmDesc* d, int count);
// Enqueue up to 4 independent GEMMs as one launch (plus a reduction launch when split-K is used).
cudaError_t gemm_f64(const GemmDesc* d, int count, double* scratch, size_t scratch_bytes,
                     cudaStream_t stream);

// While GEMM profiling is on: record a start event on `stream` and return the end event to record after
// the launch (null when profiling is off or its event pool is used up).  kind 0 = DFMA GEMM, 1 = emulated,
// 2 = BF16 sketch GEMM (its third argument then carries algorithmic bytes).
// `bytes`: the launch's algorithmic DRAM bytes (recorded for the emulated GEMM's tensor-core kernel).
cudaEvent_t profile_launch_begin(int kind, double flops, double tensor_flops, cudaStream_t stream, double bytes = 0.0);

// ---- FP64 GEMM emulated on the BF16 tensor cores (gemm_ozaki.cu) -------------------------------------
bool ozaki_eligible(const GemmDesc& d, bool force);
size_t ozaki_scratch_bytes(int64_t M, int64_t N, int64_t K);
// d.M is the long side (>= 256); set out_transposed to write C^T (element (i, j) at C[j + i ldc]).
cudaError_t gemm_ozaki(const GemmDesc& d, bool out_transposed, char* scratch, size_t scratch_bytes, int* status,
                       cudaStream_t s, int max_ctas = 0);

// Where the drivers send FP64 GEMMs: the DFMA kernel, or the emulation for the large ones.
struct GemmEngine {
  double* scratch = nullptr;  // DFMA split-K scratch
  size_t scratch_bytes = 0;
  char* oz = nullptr;         // emulation scratch (slices, exponents, split partials)
  size_t oz_bytes = 0;
  int* status = nullptr;
  bool emulate = false;
  bool force = false;  // emulate every eligible shape, not only large products
  int max_ctas = 0;    // > 0: persistent and cooperative kernels use at most this many CTAs (SMs left free
                       // for work on another stream)
};
// Bytes of emulation scratch that cover every GEMM of a factorization of an m x n matrix with panel b.
size_t ozaki_bound(int64_t m, int64_t n, int64_t b);
cudaError_t gemm_run(const GemmEngine& eng, const GemmDesc* d, int count, cudaStream_t s);

// ---- Gaussian generator (philox.cu) --------------------------------------------------------------
cudaError_t randn_f64(int64_t rows, int64_t cols, double* G, int64_t ldg, uint64_t seed,
                      uint32_t step, uint32_t tag, cudaStream_t stream);

// ---- Householder panel (panel_qr.cu) ---------------------------------------------------------------
size_t panel_scratch_bytes(int64_t r, int64_t w);
// P (r x w, ld) overwritten with R / reflectors; writes tau, explicit Y (r x w), (if Tf != null)
// the compact-WY factor and (if Rout != null) a w x w copy of R with zeros below the diagonal.
// hdr: workspace header (barrier words + status).
// eng (optional): GEMM router for the Gram matrix Y^T Y (else the DFMA kernel with `scratch`).
struct GemmEngine;
cudaError_t panel_qr(int64_t r, int64_t w, double* P, int64_t ldp, double* tau, double* Y,
                     int64_t ldy, double* Tf, int64_t ldtf, double* Rout, int64_t ldr, double* scratch,
                     size_t scratch_bytes, WsHeader* hdr, cudaStream_t stream, const GemmEngine* eng = nullptr);

// ---- Jacobi SVD (jacobi.cu) -----------------------------------------------------------------------
// One-sided Jacobi SVD of a c x c block (c <= 256) on one thread-block cluster.  With scratch of at least
// jacobi_scratch_bytes(c) (> 0 for 32 <= c <= 256) an FP32 pre-pass supplies the starting V.
size_t jacobi_scratch_bytes(int64_t c);
cudaError_t jacobi_svd(int64_t c, const double* M, int64_t ldm, double* Us, int64_t ldu, double* s,
                       double* Vs, int64_t ldv, WsHeader* hdr, cudaStream_t stream, double* scratch = nullptr,
                       size_t scratch_bytes = 0);

// ---- BF16 tensor-core GEMM (gemm_bf16_tc.cu) ------------------------------------------------------
// D (FP64, M x N, ldd) = alpha * A (M x K) B (N x K)^T, BF16 operands with K contiguous (ld multiple of 8,
// 16-byte aligned), FP32 accumulation on tcgen05; N <= 256.  part: FP32 split-K scratch.
int tc_plan_splits(int64_t M, int64_t N, int64_t K);
size_t tc_part_bytes(int64_t M, int64_t N, int64_t K);
cudaError_t gemm_bf16_tn(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                         const __nv_bfloat16* B, int64_t ldb, double alpha, double* D, int64_t ldd, float* part,
                         size_t part_bytes, int* status, cudaStream_t s);
// FP64 column-major rows x cols -> BF16 with the same layout (ldd) or transposed (D[j + i ldd] = S(i, j)).
cudaError_t to_bf16(int64_t rows, int64_t cols, const double* S, int64_t lds, __nv_bfloat16* D, int64_t ldd,
                    cudaStream_t s);
cudaError_t to_bf16_t(int64_t rows, int64_t cols, const double* S, int64_t lds, __nv_bfloat16* D, int64_t ldd,
                      cudaStream_t s);

// ---- learned q policy (mlp.cu) ------------------------------------------------------------------------
// features of one step from the panel-factored q = 0 sketch (R on and above the diagonal of Rfac, ld ldr)
// and the previous step's singular values Dprev (b of them; null at step 1)
cudaError_t policy_features(const double* Rfac, int64_t ldr, int b, const double* Dprev, int step, int steps,
                            int64_t n, int64_t c, float* feat, cudaStream_t s);
cudaError_t policy_decide(const void* params, const float* feat, int* q_dev, cudaStream_t s);

// ---- small kernels (aux.cu) ------------------------------------------------------------------------
cudaError_t fill_identity(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t s);
cudaError_t copy_matrix(int64_t rows, int64_t cols, const double* S, int64_t lds, double* D,
                        int64_t ldd, cudaStream_t s);
cudaError_t zero_matrix(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t s);
// X(0:rows, 0:cols) = [diag(d); 0] (d has min(rows, cols) entries)
cudaError_t set_diag_block(int64_t rows, int64_t cols, const double* d, double* X, int64_t ld,
                           cudaStream_t s);
// D (cols x rows, ldd) = S^T (S rows x cols, lds)
cudaError_t transpose_matrix(int64_t rows, int64_t cols, const double* S, int64_t lds, double* D, int64_t ldd,
                             cudaStream_t s);
// zero the strictly lower triangle of an rows x cols block
cudaError_t zero_lower(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t s);
// Frobenius recurrence (Sec. 4.1): e2[idx] = ||X||_F^2 (first) or max(e2[idx - 1] - ||X||_F^2, 0); part holds
// frob_scratch_bytes() of partial sums.  A recurrence step also sets *gate when e2[idx] fell below 2^-30
// e2[base], where the recurrence is no longer accurate; frob_refresh then replaces e2[idx] by the directly
// summed ||X||_F^2 of the trailing block X (and does nothing while *gate == 0).
size_t frob_scratch_bytes();
cudaError_t frob_step(int64_t rows, int64_t cols, const double* X, int64_t ld, double* part, double* e2, int64_t idx,
                      bool first, int64_t base, int* gate, cudaStream_t s);
cudaError_t frob_refresh(int64_t rows, int64_t cols, const double* X, int64_t ld, double* part, double* e2,
                         int64_t idx, int* gate, cudaStream_t s);
// *dst = *src if *dst is still 0 (the first recorded device condition wins)
cudaError_t merge_status(int* dst, const int* src, cudaStream_t s);
// status |= NUMERICAL if any entry of the block is not finite
cudaError_t check_finite(int64_t rows, int64_t cols, const double* X, int64_t ld, int* status,
                         cudaStream_t s);

// ---- m < n through the transpose (capi.cu) ------------------------------------------------------------
typedef size_t (*WsFn)(int64_t, int64_t, int64_t, const rrf_opts*);
typedef rrf_status (*RunFn)(int64_t, int64_t, const double*, int64_t, int64_t, int, double*, int64_t, double*,
                            int64_t, double*, int64_t, uint64_t, void*, size_t, const rrf_opts*, void*);
// Workspace of a wide (m < n) call: the tall call's workspace first (its status word stays at the start),
// then A^T (n x m) and the tall call's T (n x m).
size_t wide_workspace(WsFn wsfn, int64_t m, int64_t n, int64_t b, const rrf_opts* opts);
// A (m x n, m < n) = U T V^T from the tall factorization A^T = U' T' V'^T: U = V', T = T'^T, V = U'.
rrf_status factor_wide(WsFn wsfn, RunFn run, int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                       double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, uint64_t seed,
                       void* workspace, size_t ws_bytes, const rrf_opts* opts, void* stream);

}  // namespace rrf

#define RRF_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return RRF_CUDA_ERROR;  \
  } while (0)
