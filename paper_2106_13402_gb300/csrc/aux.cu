// aux.cu -- small memory-bound kernels of the drivers (initialisation of U = I, V = I, T = A; block
// copies for the in-place small products; writing D_small and the zero blocks of Algorithm 3; the
// Frobenius norms of the early-termination rule).
#include <algorithm>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

enum Op { kIdentity = 0, kCopy = 1, kZero = 2, kDiag = 3, kZeroLower = 4, kTranspose = 5 };

__global__ void block_kernel(int op, int64_t rows, int64_t cols, const double* __restrict__ S, int64_t lds,
                             double* __restrict__ D, int64_t ldd, const double* __restrict__ d) {
  const int64_t total = rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % rows, j = idx / rows;
    double* dst = D + i + j * ldd;
    switch (op) {
      case kIdentity: *dst = (i == j) ? 1.0 : 0.0; break;
      case kCopy: *dst = S[i + j * lds]; break;
      case kZero: *dst = 0.0; break;
      case kDiag: *dst = (i == j) ? d[i] : 0.0; break;
      case kZeroLower: if (i > j) *dst = 0.0; break;
      case kTranspose: D[j + i * ldd] = S[i + j * lds]; break;  // D is cols x rows
    }
  }
}

cudaError_t launch(int op, int64_t rows, int64_t cols, const double* S, int64_t lds, double* D, int64_t ldd,
                   const double* d, cudaStream_t s) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t grid = std::min<int64_t>((total + threads - 1) / threads, (int64_t)dev_info().sms * 16);
  block_kernel<<<(unsigned)grid, threads, 0, s>>>(op, rows, cols, S, lds, D, ldd, d);
  count_launch();
  return cudaGetLastError();
}

__global__ void finite_kernel(int64_t rows, int64_t cols, const double* __restrict__ X, int64_t ld, int* status) {
  const int64_t total = rows * cols;
  bool bad = false;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = X[(idx % rows) + (idx / rows) * ld];
    bad |= !isfinite(v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, RRF_NUMERICAL);
}

// Frobenius norms of the early-termination rule (Sec. 4.1): per-block partial sums of squares in a fixed
// grid-stride order, then one block sums the partials in a fixed tree, so the result is repeatable.
constexpr int kSumsqThreads = 256;
constexpr int kSumsqMaxBlocks = 1024;
// The recurrence subtracts sums of squares of size up to e_0^2, so its absolute error is a few hundred
// units of 2^-53 e_0^2 (rounding of the sums and of the subtraction, and the departure of the computed
// transformations from orthogonality).  Once e_i^2 < 2^-30 e_0^2 that error would exceed ~2^-15 of the
// value, so from there the norm of the trailing block is summed directly.
constexpr double kFrobFloor = 0x1p-30;

// gate == null: always run; else only when *gate != 0 (the partial sums are then zero)
__global__ void sumsq_kernel(int64_t rows, int64_t cols, const double* __restrict__ X, int64_t ld,
                             double* __restrict__ part, const int* gate) {
  __shared__ double sh[kSumsqThreads];
  if (gate != nullptr && *(volatile const int*)gate == 0) return;
  const int64_t total = rows * cols;
  double acc = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = X[(idx % rows) + (idx / rows) * ld];
    acc = fma(v, v, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kSumsqThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// mode 0: e2[idx] = the sum of the nblk partials.  mode 1: e2[idx] = max(e2[idx - 1] - sum, 0), and
// *gate = (e2[idx] < kFrobFloor e2[base]).  mode 2: e2[idx] = sum when *gate != 0.
__global__ void frob_update_kernel(const double* __restrict__ part, int nblk, double* e2, int64_t idx, int mode,
                                   int64_t base, int* gate) {
  __shared__ double sh[kSumsqMaxBlocks];
  if (mode == 2 && *(volatile const int*)gate == 0) return;
  double acc = 0.0;
  for (int t = threadIdx.x; t < nblk; t += blockDim.x) acc += part[t];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kSumsqMaxBlocks / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (mode == 1) {
      const double v = fmax(e2[idx - 1] - sh[0], 0.0);
      e2[idx] = v;
      *gate = (v < kFrobFloor * e2[base]) ? 1 : 0;
    } else {
      e2[idx] = sh[0];
    }
  }
}

int64_t sumsq_grid(int64_t rows, int64_t cols) {
  const int64_t total = std::max<int64_t>(rows, 0) * std::max<int64_t>(cols, 0);
  return std::max<int64_t>(1, std::min<int64_t>((total + 4 * kSumsqThreads - 1) / (4 * kSumsqThreads),
                                                kSumsqMaxBlocks));
}

cudaError_t frob_launch(int64_t rows, int64_t cols, const double* X, int64_t ld, double* part, double* e2,
                        int64_t idx, int mode, int64_t base, int* gate, cudaStream_t s) {
  const int64_t total = std::max<int64_t>(rows, 0) * std::max<int64_t>(cols, 0);
  const int64_t grid = sumsq_grid(rows, cols);
  sumsq_kernel<<<(unsigned)grid, kSumsqThreads, 0, s>>>(total > 0 ? rows : 1, total > 0 ? cols : 0, X, ld, part,
                                                        mode == 2 ? gate : nullptr);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  frob_update_kernel<<<1, kSumsqMaxBlocks, 0, s>>>(part, (int)grid, e2, idx, mode, base, gate);
  count_launch();
  return cudaGetLastError();
}

__global__ void merge_status_kernel(int* dst, const int* src) {
  const int v = *(volatile const int*)src;
  if (v != 0) atomicCAS(dst, 0, v);
}

}  // namespace

cudaError_t merge_status(int* dst, const int* src, cudaStream_t s) {
  merge_status_kernel<<<1, 1, 0, s>>>(dst, src);
  count_launch();
  return cudaGetLastError();
}

size_t frob_scratch_bytes() { return kSumsqMaxBlocks * sizeof(double); }

cudaError_t frob_step(int64_t rows, int64_t cols, const double* X, int64_t ld, double* part, double* e2, int64_t idx,
                      bool first, int64_t base, int* gate, cudaStream_t s) {
  return frob_launch(rows, cols, X, ld, part, e2, idx, first ? 0 : 1, base, gate, s);
}

cudaError_t frob_refresh(int64_t rows, int64_t cols, const double* X, int64_t ld, double* part, double* e2,
                         int64_t idx, int* gate, cudaStream_t s) {
  return frob_launch(rows, cols, X, ld, part, e2, idx, 2, 0, gate, s);
}

cudaError_t fill_identity(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t s) {
  return launch(kIdentity, rows, cols, nullptr, 0, X, ld, nullptr, s);
}
cudaError_t copy_matrix(int64_t rows, int64_t cols, const double* S, int64_t lds, double* D, int64_t ldd,
                        cudaStream_t s) {
  return launch(kCopy, rows, cols, S, lds, D, ldd, nullptr, s);
}
cudaError_t zero_matrix(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t s) {
  return launch(kZero, rows, cols, nullptr, 0, X, ld, nullptr, s);
}
cudaError_t set_diag_block(int64_t rows, int64_t cols, const double* d, double* X, int64_t ld, cudaStream_t s) {
  return launch(kDiag, rows, cols, nullptr, 0, X, ld, d, s);
}
cudaError_t transpose_matrix(int64_t rows, int64_t cols, const double* S, int64_t lds, double* D, int64_t ldd,
                             cudaStream_t s) {
  return launch(kTranspose, rows, cols, S, lds, D, ldd, nullptr, s);
}
cudaError_t zero_lower(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t s) {
  return launch(kZeroLower, rows, cols, nullptr, 0, X, ld, nullptr, s);
}
cudaError_t check_finite(int64_t rows, int64_t cols, const double* X, int64_t ld, int* status, cudaStream_t s) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t grid = std::min<int64_t>((total + threads - 1) / threads, (int64_t)dev_info().sms * 8);
  finite_kernel<<<(unsigned)grid, threads, 0, s>>>(rows, cols, X, ld, status);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rrf
