// gemm_bf16_tc.cu -- BF16 x BF16 -> FP32 tensor-core GEMM on sm_103a (tcgen05 + TMA + TMEM), used by the
// BF16 form of the randUTV sketch (Y = T22^T G and the power iterations, Algorithm 3; the range finder
// only needs a subspace, Sec. 2.5).
//
//   D (M x N, FP32) = A (M x K) * B (N x K)^T, both operands K-contiguous ("K-major").
//
// One CTA computes a 128 x BN tile of D for one K range (split-K partials are summed later in split
// order, so results are deterministic).  Four warps: warp 0 lane 0 issues TMA loads of 128 x 64 (A)
// and BN x 64 (B) BF16 boxes with 128-byte swizzle into a 4-stage shared-memory ring; warp 1 lane 0
// issues tcgen05.mma (M = 128, N = BN, K = 16) into a TMEM accumulator and releases each stage with
// tcgen05.commit; after the last commit all four warps read their 32 TMEM lanes with tcgen05.ld and
// write FP32 partials.  Every mbarrier wait is bounded; on timeout the CTA records RRF_TIMEOUT, waits
// (bounded) for its loads in flight, frees its TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

constexpr int kStages = 4;
constexpr int BM = 128;
constexpr int BKE = 64;                       // K elements per stage (128 bytes of BF16)
constexpr int kThreads = 128;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s

struct TcParams {
  int64_t M, N, K;
  int64_t kchunk;   // K per split (multiple of BKE)
  float* part;      // [splits][N][M]
  int* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  const uint64_t addr = (smem_u32(p) >> 4) & 0x3FFF;
  return addr | (uint64_t(0) << 16) | (uint64_t(1024 >> 4) << 32) | (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const __grid_constant__ TcParams p) {
  constexpr uint32_t kBytesA = BM * BKE * 2;
  constexpr uint32_t kBytesB = BN * BKE * 2;
  constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sa = smem;                              // [kStages][kBytesA]
  unsigned char* sb = smem + kStages * kBytesA;          // [kStages][kBytesB]
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  const int split = blockIdx.z;
  const int64_t kb0 = (int64_t)split * p.kchunk;
  const int64_t kb1 = min(p.K, kb0 + p.kchunk);
  const int nkb = kb1 > kb0 ? (int)((kb1 - kb0 + BKE - 1) / BKE) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  int issued = 0;  // TMA stages issued by the producer (for the bounded drain on abort)
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (i >= kStages) {
        if (!mbar_wait(&empty_bar[s], ((i / kStages) - 1) & 1)) {
          set_status(p.status, RRF_TIMEOUT);
          atomicExch(&abort_flag, 1);
          break;
        }
      }
      if (*(volatile int*)&abort_flag) break;
      mbar_expect_tx(&full_bar[s], kBytesA + kBytesB);
      const int kx = (int)(kb0 + (int64_t)i * BKE);
      tma_load_2d(sa + s * kBytesA, &map_a, &full_bar[s], kx, (int)m0);
      tma_load_2d(sb + s * kBytesB, &map_b, &full_bar[s], kx, (int)n0);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    // instruction descriptor: D f32, A bf16, B bf16, both K-major, N = BN, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(&full_bar[s], (i / kStages) & 1)) {
        set_status(p.status, RRF_TIMEOUT);
        atomicExch(&abort_flag, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = smem_desc_sw128(sa + s * kBytesA);
      const uint64_t db = smem_desc_sw128(sb + s * kBytesB);
#pragma unroll
      for (int kk = 0; kk < BKE / 16; ++kk)
        mma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);
    }
    // Always commit: done_bar then fires once every MMA issued so far has finished (immediately if
    // none was), so the TMEM is never freed under an MMA in flight.
    (void)ok;
    if (nkb > 0) mma_commit(&done_bar);
  }
  __syncwarp();
  // Epilogue: every warp owns 32 TMEM lanes (= 32 rows of the tile).  The decision to read TMEM must be
  // uniform across the CTA (tcgen05.ld is a warp-collective), hence the vote.
  int failed = 0;
  if (nkb > 0 && !mbar_wait(&done_bar, 0)) {
    set_status(p.status, RRF_TIMEOUT);
    failed = 1;
  }
  const int any_fail = __syncthreads_or(failed);
  const bool have = (nkb > 0) && !any_fail && (*(volatile int*)&abort_flag == 0);
  if (any_fail && threadIdx.x == 0) abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int64_t row = m0 + warp * 32 + lane;
  float* out = p.part + (int64_t)split * p.N * p.M;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float v[16];
    if (have) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
    if (row < p.M) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int64_t col = n0 + c0 + i;
        if (col < p.N) out[row + col * p.M] = v[i];
      }
    }
  }
  __syncthreads();
  // On abort, drain the loads still in flight (the last kStages issued; bounded waits) before the
  // CTA's shared memory goes away.
  if (abort_flag && warp == 0 && lane == 0) {
    for (int i = (issued > kStages ? issued - kStages : 0); i < issued; ++i)
      mbar_wait(&full_bar[i % kStages], (i / kStages) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// D(FP64, ldd) = alpha * sum_s part[s] (split order).
__global__ void tc_reduce_kernel(int64_t M, int64_t N, int splits, const float* __restrict__ part, double alpha,
                                 double* __restrict__ D, int64_t ldd) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += (double)part[sp * total + idx];
    D[(idx % M) + (idx / M) * ldd] = alpha * s;
  }
}

// FP64 column-major (rows x cols, lds) -> BF16 with K = rows contiguous (dst row j = column j), ldd.
__global__ void to_bf16_kernel(int64_t rows, int64_t cols, const double* __restrict__ S, int64_t lds,
                               __nv_bfloat16* __restrict__ D, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % rows, j = idx / rows;
    D[i + j * ldd] = __double2bfloat16(S[i + j * lds]);
  }
}

// FP64 column-major (rows x cols, lds) -> BF16 transposed: D[j + i * ldd] = S(i, j) (tiled through shared memory).
__global__ void to_bf16_t_kernel(int64_t rows, int64_t cols, const double* __restrict__ S, int64_t lds,
                                 __nv_bfloat16* __restrict__ D, int64_t ldd) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int64_t i = i0 + tx, j = j0 + k;
    tile[k][tx] = (i < rows && j < cols) ? __bfloat162float(__double2bfloat16(S[i + j * lds])) : 0.f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t j = j0 + tx, i = i0 + k;
    if (i < rows && j < cols) D[j + i * ldd] = __float2bfloat16(tile[tx][k]);
  }
}

// ---- host side ---------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// rows x K BF16 matrix, row r at base + r * ld (elements); box = box_rows x 64.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((ld * 2) & 15) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BKE, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN>
size_t tc_smem_bytes() {
  return (size_t)kStages * (BM * BKE * 2 + BN * BKE * 2) + 1024;
}

template <int BN>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& p, int splits, cudaStream_t s) {
  static std::atomic<bool> attr{false};  // set once per process (one GPU each)
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((unsigned)((p.M + BM - 1) / BM), (unsigned)((p.N + BN - 1) / BN), (unsigned)splits);
  tc_gemm_kernel<BN><<<grid, kThreads, tc_smem_bytes<BN>(), s>>>(ma, mb, p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int tc_plan_splits(int64_t M, int64_t N, int64_t K) {
  const int sms = dev_info().sms;
  const int bn = N > 128 ? 256 : (N > 64 ? 128 : 64);
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + bn - 1) / bn);
  const int64_t kblocks = (K + BKE - 1) / BKE;
  int s = 1;
  while (tiles * s < sms && s * 2 <= 16 && kblocks / (s * 2) >= 4) s *= 2;
  return s;
}

size_t tc_part_bytes(int64_t M, int64_t N, int64_t K) {
  return align_up((size_t)tc_plan_splits(M, N, K) * M * N * sizeof(float), 256);
}

// D (FP64, M x N, ldd) = alpha * A (M x K) * B (N x K)^T with BF16 operands (K-contiguous rows, lda/ldb in
// elements, multiples of 8, 16-byte aligned bases) and FP32 accumulation.
cudaError_t gemm_bf16_tn(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                         const __nv_bfloat16* B, int64_t ldb, double alpha, double* D, int64_t ldd, float* part,
                         size_t part_bytes, int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (N > 256) return cudaErrorInvalidValue;
  const int bn = N > 128 ? 256 : (N > 64 ? 128 : 64);
  int splits = tc_plan_splits(M, N, K);
  if ((size_t)splits * M * N * sizeof(float) > part_bytes) return cudaErrorInvalidValue;
  const int64_t kblocks = (K + BKE - 1) / BKE;
  int64_t kchunk = ((kblocks + splits - 1) / splits) * BKE;
  if (kchunk <= 0) kchunk = BKE;
  splits = (int)std::max<int64_t>(1, (K + kchunk - 1) / kchunk);
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, BM) || !make_map(&mb, B, N, K, ldb, bn)) return cudaErrorInvalidValue;
  TcParams p;
  p.M = M; p.N = N; p.K = K;
  p.kchunk = kchunk;
  p.part = part;
  p.status = status;
  cudaError_t e;
  // profiler: 2MNK BF16 flops; algorithmic bytes = the BF16 operands read once + one FP32 result each
  cudaEvent_t ev_end = profile_launch_begin(2, 2.0 * M * N * K, 2.0 * (double)(M + N) * K + 4.0 * M * N, s);
  if (bn == 64) e = launch_tc<64>(ma, mb, p, splits, s);
  else if (bn == 128) e = launch_tc<128>(ma, mb, p, splits, s);
  else e = launch_tc<256>(ma, mb, p, splits, s);
  if (ev_end != nullptr) cudaEventRecord(ev_end, s);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((M * N + threads - 1) / threads, (int64_t)dev_info().sms * 16);
  tc_reduce_kernel<<<(unsigned)blocks, threads, 0, s>>>(M, N, splits, part, alpha, D, ldd);
  count_launch();
  return cudaGetLastError();
}

cudaError_t to_bf16(int64_t rows, int64_t cols, const double* S, int64_t lds, __nv_bfloat16* D, int64_t ldd,
                    cudaStream_t s) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, (int64_t)dev_info().sms * 16);
  to_bf16_kernel<<<(unsigned)blocks, threads, 0, s>>>(rows, cols, S, lds, D, ldd);
  count_launch();
  return cudaGetLastError();
}

cudaError_t to_bf16_t(int64_t rows, int64_t cols, const double* S, int64_t lds, __nv_bfloat16* D, int64_t ldd,
                      cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  to_bf16_t_kernel<<<grid, dim3(32, 8), 0, s>>>(rows, cols, S, lds, D, ldd);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rrf
