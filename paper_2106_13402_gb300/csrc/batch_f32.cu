// batch_f32.cu -- many powerURV factorizations (Algorithm 1) of uneven shapes in FP32, as one CUDA graph.
//
// A plan fixes the shapes; its first run uploads a per-matrix descriptor table, autotunes the GEMM tile
// shape on the batch's own problems, and captures the whole method -- randn, the q power steps, every
// Householder panel, compact-WY trailing update and explicit-Q step of every matrix -- as a CUDA graph
// of batched kernels; later runs with the same buffers replay the graph (one launch).  Each batched
// kernel covers all matrices that are active in that phase: GEMM phases are persistent kernels that
// walk a global tile list (per-matrix tile counts prefix-summed in shared memory, binary search per
// tile); a panel phase gives each matrix one CTA (m <= 2048 here, so no grid barrier is needed).
//
// Householder convention and Gaussian stream are those of the FP64 path; matrix i draws its Gaussian
// with key seed + i (step 0, tag 2), i.e. exactly what rrf_powerurv would draw for it with that seed.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

constexpr int kMaxBatch = 4096;

struct BMat {
  int m, n;
  int64_t lda, ldu, ldt, ldv;
  const float* A;
  float* U;
  float* T;
  float* V;
  float* W;     // max(m,n) x n work (ld m or n)
  float* Ys;    // m x n explicit reflectors (ld = rows of the factored matrix)
  float* Tall;  // npanels x nb x nb compact-WY factors
  float* Wa;    // nb x max(m, n)
  float* Wb;    // nb x max(m, n)
  float* tau;   // n
};

// Which matrix a QR / explicit-Q phase works on.
enum Target : int { kTgtWmn = 0, kTgtWnn = 1, kTgtTmn = 2, kTgtQT = 3, kTgtQV = 4, kTgtQU = 5 };

__host__ __device__ inline void target_of(const BMat& b, int tgt, float*& X, int64_t& ldx, int& rows, int& cols) {
  switch (tgt) {
    case kTgtWmn: X = b.W; ldx = b.m; rows = b.m; cols = b.n; break;
    case kTgtWnn: X = b.W; ldx = b.n; rows = b.n; cols = b.n; break;
    case kTgtTmn: X = b.T; ldx = b.ldt; rows = b.m; cols = b.n; break;
    case kTgtQT: X = b.T; ldx = b.ldt; rows = b.m; cols = b.n; break;   // thin Q (m x n) of an m x n QR
    case kTgtQV: X = b.V; ldx = b.ldv; rows = b.n; cols = b.n; break;   // Q (n x n) of an n x n QR
    default: X = b.U; ldx = b.ldu; rows = b.m; cols = b.m; break;       // full U (m x m) of an m x n QR
  }
}

// ---- GEMM phases ------------------------------------------------------------------------------------
enum GemmKind : int {
  kAV_W = 0,    // W (m x n) = A V
  kAtT_W = 1,   // W (n x n) = A^T T           (T holds the thin Q of A V)
  kAV_T = 2,    // T (m x n) = A V
  kTrail1 = 3,  // Wa = Y_p^T X(j0:, j0+w:)
  kTrail2 = 4,  // Wb = Tf_p^T Wa
  kTrail3 = 5,  // X(j0:, j0+w:) -= Y_p Wb
  kFormQ1 = 6,  // Wa = Y_p^T Q(j0:, j0:)
  kFormQ2 = 7,  // Wb = Tf_p Wa
  kFormQ3 = 8,  // Q(j0:, j0:) -= Y_p Wb
};

struct GemmPhase {
  int kind;
  int p;        // panel index (trailing / explicit-Q phases)
  int nb;       // panel width
  int qr_tgt;   // matrix the panels were computed on (decides the rows of Y_p)
  int out_tgt;  // matrix updated (trailing: == qr_tgt; explicit Q: the Q target)
};

struct Prob {
  int M, N, K;
  const float* A;
  int64_t lda;
  int ta;
  const float* B;
  int64_t ldb;
  int tb;
  float* C;
  int64_t ldc;
  float alpha, beta;
};

__host__ __device__ inline Prob problem_of(const BMat& b, const GemmPhase& ph) {
  Prob P;
  P.M = P.N = P.K = 0;
  P.alpha = 1.f;
  P.beta = 0.f;
  P.ta = P.tb = 0;
  P.A = P.B = nullptr;
  P.C = nullptr;
  P.lda = P.ldb = P.ldc = 1;
  switch (ph.kind) {
    case kAV_W: P.M = b.m; P.N = b.n; P.K = b.n; P.A = b.A; P.lda = b.lda; P.B = b.V; P.ldb = b.ldv; P.C = b.W; P.ldc = b.m; return P;
    case kAV_T: P.M = b.m; P.N = b.n; P.K = b.n; P.A = b.A; P.lda = b.lda; P.B = b.V; P.ldb = b.ldv; P.C = b.T; P.ldc = b.ldt; return P;
    case kAtT_W: P.M = b.n; P.N = b.n; P.K = b.m; P.A = b.A; P.lda = b.lda; P.ta = 1; P.B = b.T; P.ldb = b.ldt; P.C = b.W; P.ldc = b.n; return P;
    default: break;
  }
  float* Xq; int64_t ldq; int qrows, qcols;
  target_of(b, ph.qr_tgt, Xq, ldq, qrows, qcols);
  const int j0 = ph.p * ph.nb;
  if (j0 >= qcols) return P;
  const int wd = min(ph.nb, qcols - j0);
  const int rr = qrows - j0;
  const float* Yp = b.Ys + j0 + (int64_t)j0 * qrows;
  const float* Tp = b.Tall + (int64_t)ph.p * ph.nb * ph.nb;
  float* X; int64_t ldx; int xrows, xcols;
  target_of(b, ph.out_tgt, X, ldx, xrows, xcols);
  const bool formq = ph.kind >= kFormQ1;
  const int c0 = formq ? j0 : j0 + wd;          // first column of the block the reflectors act on
  const int nc = xcols - c0;
  if (nc <= 0) return P;
  float* Cb = X + j0 + (int64_t)c0 * ldx;       // rows j0.., columns c0..
  switch (ph.kind) {
    case kTrail1: case kFormQ1:
      P.M = wd; P.N = nc; P.K = rr; P.A = Yp; P.lda = qrows; P.ta = 1; P.B = Cb; P.ldb = ldx; P.C = b.Wa; P.ldc = ph.nb;
      break;
    case kTrail2: case kFormQ2:
      P.M = wd; P.N = nc; P.K = wd; P.A = Tp; P.lda = ph.nb; P.ta = (ph.kind == kTrail2); P.B = b.Wa; P.ldb = ph.nb;
      P.C = b.Wb; P.ldc = ph.nb;
      break;
    default:  // kTrail3, kFormQ3
      P.M = rr; P.N = nc; P.K = wd; P.A = Yp; P.lda = qrows; P.B = b.Wb; P.ldb = ph.nb; P.C = Cb; P.ldc = ldx;
      P.alpha = -1.f; P.beta = 1.f;
      break;
  }
  return P;
}

// Persistent batched FP32 GEMM: BM x BN tiles, TM x TN register tile per thread, BK = 16.
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    batch_gemm_kernel(const BMat* __restrict__ mats, int count, GemmPhase ph) {
  constexpr int NTH = (BM / TM) * (BN / TN);
  constexpr int BK = 16;
  constexpr int TX = BM / TM;  // threads along M
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  __shared__ int prefix[kMaxBatch + 1];
  const int tid = threadIdx.x;
  // per-matrix tile counts, then an exclusive prefix sum (single warp scan over chunks)
  for (int i = tid; i < count; i += NTH) {
    const Prob P = problem_of(mats[i], ph);
    prefix[i + 1] = (P.M > 0 && P.N > 0) ? ((P.M + BM - 1) / BM) * ((P.N + BN - 1) / BN) : 0;
  }
  if (tid == 0) prefix[0] = 0;
  __syncthreads();
  if (tid == 0)
    for (int i = 1; i <= count; ++i) prefix[i] += prefix[i - 1];
  __syncthreads();
  const int total = prefix[count];
  const int tx = tid % TX, ty = tid / TX;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int lo = 0, hi = count;  // largest i with prefix[i] <= tile
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    const Prob P = problem_of(mats[lo], ph);
    const int local = tile - prefix[lo];
    const int tiles_m = (P.M + BM - 1) / BM;
    const int m0 = (local % tiles_m) * BM, n0 = (local / tiles_m) * BN;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < P.K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += NTH) {
        int m, k;
        if (!P.ta) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
        const int gm = m0 + m, gk = k0 + k;
        float v = 0.f;
        if (gm < P.M && gk < P.K) v = P.ta ? P.A[gk + (int64_t)gm * P.lda] : P.A[gm + (int64_t)gk * P.lda];
        As[k][m] = v;
      }
      for (int e = tid; e < BN * BK; e += NTH) {
        int n, k;
        if (!P.tb) { k = e % BK; n = e / BK; } else { n = e % BN; k = e / BN; }
        const int gn = n0 + n, gk = k0 + k;
        float v = 0.f;
        if (gn < P.N && gk < P.K) v = P.tb ? P.B[gn + (int64_t)gk * P.ldb] : P.B[gk + (int64_t)gn * P.ldb];
        Bs[k][n] = v;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        float a[TM], bb[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[k][tx + TX * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bb[j] = Bs[k][ty + (NTH / TX) * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + ty + (NTH / TX) * j;
      if (gn >= P.N) continue;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int gm = m0 + tx + TX * i;
        if (gm >= P.M) continue;
        float* c = P.C + gm + (int64_t)gn * P.ldc;
        float v = P.alpha * acc[i][j];
        if (P.beta != 0.f) v = fmaf(P.beta, *c, v);
        *c = v;
      }
    }
  }
}

// ---- panel phase: one CTA per matrix --------------------------------------------------------------------
constexpr int kPanelThreads = 512;
constexpr int kMaxNb = 64;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ float block_sum_f(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_f(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kPanelThreads / 32; ++i) t += red[i];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(kPanelThreads) batch_panel_kernel(const BMat* __restrict__ mats, int tgt, int p,
                                                                    int nb) {
  __shared__ float red[33];
  __shared__ float z[kMaxNb];
  __shared__ float S[kMaxNb][kMaxNb + 1];
  __shared__ float Tf[kMaxNb][kMaxNb + 1];
  const BMat b = mats[blockIdx.x];
  float* X; int64_t ldx; int rows, cols;
  target_of(b, tgt, X, ldx, rows, cols);
  const int j0 = p * nb;
  if (j0 >= cols) return;
  const int wd = min(nb, cols - j0), rr = rows - j0;
  float* P = X + j0 + (int64_t)j0 * ldx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kPanelThreads / 32;
  for (int j = 0; j < wd; ++j) {
    float* x = P + (int64_t)j * ldx;
    float s2 = 0.f;
    for (int l = j + 1 + tid; l < rr; l += kPanelThreads) s2 = fmaf(x[l], x[l], s2);
    const float sig2 = block_sum_f(s2, red);
    const float alpha = x[j];
    float tau = 0.f, beta = alpha, scal = 0.f;
    if (sig2 != 0.f) {
      const float nrm = sqrtf(alpha * alpha + sig2);
      beta = (alpha >= 0.f) ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scal = 1.f / (alpha - beta);
    }
    __syncthreads();
    if (tau != 0.f)
      for (int l = j + 1 + tid; l < rr; l += kPanelThreads) x[l] *= scal;
    if (tid == 0) {
      x[j] = beta;
      b.tau[j0 + j] = tau;
    }
    __syncthreads();
    if (tau != 0.f) {
      // z_k = v^T P(j:, k) for k > j (one warp per column), then P(:, k) -= tau z_k v.
      for (int k = j + 1 + warp; k < wd; k += NW) {
        const float* pk = P + (int64_t)k * ldx;
        float acc = (lane == 0) ? pk[j] : 0.f;
        for (int l = j + 1 + lane; l < rr; l += 32) acc = fmaf(x[l], pk[l], acc);
        acc = warp_sum_f(acc);
        if (lane == 0) z[k] = tau * acc;
      }
      __syncthreads();
      for (int k = j + 1 + warp; k < wd; k += NW) {
        float* pk = P + (int64_t)k * ldx;
        const float zz = z[k];
        if (lane == 0) pk[j] -= zz;
        for (int l = j + 1 + lane; l < rr; l += 32) pk[l] = fmaf(-zz, x[l], pk[l]);
      }
    }
    __syncthreads();
  }
  // Explicit reflectors into Ys(j0:, j0:j0+wd) (ld rows) and the compact-WY factor from S = Y^T Y.
  float* Yp = b.Ys + j0 + (int64_t)j0 * rows;
  for (int k = warp; k < wd; k += NW) {
    const float* pk = P + (int64_t)k * ldx;
    float* yk = Yp + (int64_t)k * rows;
    for (int l = lane; l < rr; l += 32) yk[l] = (l < k) ? 0.f : (l == k ? 1.f : pk[l]);
  }
  __syncthreads();
  for (int e = warp; e < wd * wd; e += NW) {
    const int a = e % wd, c = e / wd;
    if (a > c) continue;
    const float* ya = Yp + (int64_t)a * rows;
    const float* yc = Yp + (int64_t)c * rows;
    float acc = 0.f;
    for (int l = c + lane; l < rr; l += 32) acc = fmaf(ya[l], yc[l], acc);
    acc = warp_sum_f(acc);
    if (lane == 0) S[a][c] = acc;
  }
  __syncthreads();
  for (int j = 0; j < wd; ++j) {
    const float tj = b.tau[j0 + j];
    if (tid < wd) {
      float v = 0.f;
      if (tid < j) {
        float acc = 0.f;
        for (int l = tid; l < j; ++l) acc = fmaf(Tf[tid][l], S[l][j], acc);
        v = -tj * acc;
      } else if (tid == j) {
        v = tj;
      }
      Tf[tid][j] = v;
    }
    __syncthreads();
  }
  float* Tp = b.Tall + (int64_t)p * nb * nb;
  for (int e = tid; e < wd * wd; e += kPanelThreads) Tp[(e % wd) + (int64_t)(e / wd) * nb] = Tf[e % wd][e / wd];
}

// ---- elementwise batched phases -------------------------------------------------------------------------
enum ElemKind : int { kRandnV = 0, kCopyVtoW = 1, kIdentity = 2, kZeroLowerT = 3 };

__device__ __forceinline__ void philox_b(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__global__ void batch_elem_kernel(const BMat* __restrict__ mats, int kind, int tgt, uint64_t seed) {
  const BMat b = mats[blockIdx.y];
  if (kind == kRandnV) {
    const int64_t total = (int64_t)b.n * b.n;
    const int64_t nblk = (total + 1) / 2;
    const uint64_t key = seed + blockIdx.y;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nblk; t += (int64_t)gridDim.x * blockDim.x) {
      uint32_t x[4];
      philox_b((uint32_t)t, (uint32_t)((uint64_t)t >> 32), 0u, 2u, (uint32_t)key, (uint32_t)(key >> 32), x);
      const uint64_t a = ((uint64_t)x[0] << 32) | x[1];
      const uint64_t c = ((uint64_t)x[2] << 32) | x[3];
      const double u1 = (double)((a >> 11) + 1) * 0x1p-53;
      const double u2 = (double)(c >> 11) * 0x1p-53;
      const double rho = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincos(6.283185307179586476925286766559 * u2, &sn, &cs);
      const int64_t l0 = 2 * t, l1 = l0 + 1;
      b.V[(l0 % b.n) + (l0 / b.n) * b.ldv] = (float)(rho * cs);
      if (l1 < total) b.V[(l1 % b.n) + (l1 / b.n) * b.ldv] = (float)(rho * sn);
    }
    return;
  }
  float* X; int64_t ldx; int rows, cols;
  target_of(b, tgt, X, ldx, rows, cols);
  if (kind == kCopyVtoW) { X = b.W; ldx = b.n; rows = b.n; cols = b.n; }
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    float* d = X + i + j * ldx;
    if (kind == kCopyVtoW) *d = b.V[i + j * b.ldv];
    else if (kind == kIdentity) *d = (i == j) ? 1.f : 0.f;
    else if (i > j) *d = 0.f;
  }
}

}  // namespace
}  // namespace rrf

// ---- plan ----------------------------------------------------------------------------------------------
struct rrf_batch_plan {
  int count = 0;
  std::vector<int> m, n;
  int nb = 64;
  int q = 1;
  int max_m = 0, max_n = 0;
  size_t table_bytes = 0, per_off_bytes = 0, ws_bytes = 0;
  std::vector<size_t> offsets;  // per-matrix workspace offsets (after the table)
  int tile_big = -1, tile_skinny = -1;  // autotuned GEMM configurations (index into the candidate list)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<rrf::BMat> host_table;
  void* pinned = nullptr;  // pinned copy of the table (source of the upload)
  void* graph_ws = nullptr;
  uint64_t graph_seed = 0;
  cudaStream_t graph_stream = nullptr;
  int64_t graph_kernels = 0;  // kernel nodes in the captured graph
};

namespace rrf {
namespace {

struct Cand {
  const char* name;
  void (*launch)(const BMat*, int, GemmPhase, int, cudaStream_t);
};

template <int BM, int BN, int TM, int TN>
void launch_gemm(const BMat* mats, int count, GemmPhase ph, int grid, cudaStream_t s) {
  batch_gemm_kernel<BM, BN, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(mats, count, ph);
  count_launch();
}

const Cand kCands[] = {
    {"64x64/4x4", launch_gemm<64, 64, 4, 4>},
    {"128x64/8x4", launch_gemm<128, 64, 8, 4>},
    {"128x128/8x8", launch_gemm<128, 128, 8, 8>},
    {"32x64/2x4", launch_gemm<32, 64, 2, 4>},
};
constexpr int kNumCands = sizeof(kCands) / sizeof(kCands[0]);

void gemm_phase(const rrf_batch_plan* pl, const BMat* mats, GemmPhase ph, cudaStream_t s) {
  const bool skinny = (ph.kind == kTrail1 || ph.kind == kFormQ1 || ph.kind == kTrail2 || ph.kind == kFormQ2);
  const int c = skinny ? (pl->tile_skinny >= 0 ? pl->tile_skinny : 0) : (pl->tile_big >= 0 ? pl->tile_big : 0);
  kCands[c].launch(mats, pl->count, ph, dev_info().sms * 4, s);
}

void elem_phase(const rrf_batch_plan* pl, const BMat* mats, int kind, int tgt, uint64_t seed, cudaStream_t s) {
  dim3 grid(8, (unsigned)pl->count);
  batch_elem_kernel<<<grid, 256, 0, s>>>(mats, kind, tgt, seed);
  count_launch();
}

void qr_phase(const rrf_batch_plan* pl, const BMat* mats, int tgt, int cols_max, cudaStream_t s) {
  const int np = (cols_max + pl->nb - 1) / pl->nb;
  for (int p = 0; p < np; ++p) {
    batch_panel_kernel<<<pl->count, kPanelThreads, 0, s>>>(mats, tgt, p, pl->nb);
    count_launch();
    for (int k = kTrail1; k <= kTrail3; ++k) gemm_phase(pl, mats, GemmPhase{k, p, pl->nb, tgt, tgt}, s);
  }
}

void formq_phase(const rrf_batch_plan* pl, const BMat* mats, int qr_tgt, int q_tgt, int cols_max, cudaStream_t s) {
  elem_phase(pl, mats, kIdentity, q_tgt, 0, s);
  const int np = (cols_max + pl->nb - 1) / pl->nb;
  for (int p = np - 1; p >= 0; --p)
    for (int k = kFormQ1; k <= kFormQ3; ++k) gemm_phase(pl, mats, GemmPhase{k, p, pl->nb, qr_tgt, q_tgt}, s);
}

// The whole method for every matrix (Algorithm 1), batched.
void enqueue_all(const rrf_batch_plan* pl, const BMat* mats, uint64_t seed, cudaStream_t s) {
  elem_phase(pl, mats, kRandnV, 0, seed, s);
  if (pl->q == 0) {
    elem_phase(pl, mats, kCopyVtoW, 0, 0, s);
    qr_phase(pl, mats, kTgtWnn, pl->max_n, s);
    formq_phase(pl, mats, kTgtWnn, kTgtQV, pl->max_n, s);
  }
  for (int it = 0; it < pl->q; ++it) {
    gemm_phase(pl, mats, GemmPhase{kAV_W, 0, pl->nb, 0, 0}, s);
    qr_phase(pl, mats, kTgtWmn, pl->max_n, s);
    formq_phase(pl, mats, kTgtWmn, kTgtQT, pl->max_n, s);
    gemm_phase(pl, mats, GemmPhase{kAtT_W, 0, pl->nb, 0, 0}, s);
    qr_phase(pl, mats, kTgtWnn, pl->max_n, s);
    formq_phase(pl, mats, kTgtWnn, kTgtQV, pl->max_n, s);
  }
  gemm_phase(pl, mats, GemmPhase{kAV_T, 0, pl->nb, 0, 0}, s);
  qr_phase(pl, mats, kTgtTmn, pl->max_n, s);
  formq_phase(pl, mats, kTgtTmn, kTgtQU, pl->max_n, s);
  elem_phase(pl, mats, kZeroLowerT, kTgtTmn, 0, s);
}

// Autotune: time each candidate on the batch's first GEMM phase (big) and on the first trailing
// reduction (skinny), using the real buffers; the phases are re-run for real afterwards.
cudaError_t autotune(rrf_batch_plan* pl, const BMat* mats, cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_big = 1e30f, best_sk = 1e30f;
  for (int c = 0; c < kNumCands; ++c) {
    for (int pass = 0; pass < 2; ++pass) {
      const GemmPhase ph = pass == 0 ? GemmPhase{kAV_W, 0, pl->nb, 0, 0} : GemmPhase{kTrail1, 0, pl->nb, kTgtWmn, kTgtWmn};
      kCands[c].launch(mats, pl->count, ph, dev_info().sms * 4, s);  // warm-up
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) kCands[c].launch(mats, pl->count, ph, dev_info().sms * 4, s);
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return e;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (pass == 0 && ms < best_big) { best_big = ms; pl->tile_big = c; }
      if (pass == 1 && ms < best_sk) { best_sk = ms; pl->tile_skinny = c; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace rrf

using namespace rrf;

extern "C" rrf_status rrf_batch_plan_create(rrf_batch_plan** out, int count, const int64_t* m, const int64_t* n,
                                            int64_t b, int q) {
  clear_arg_error();
  if (out == nullptr) { set_arg_error(1); return RRF_INVALID_ARG; }
  *out = nullptr;
  if (count < 1 || count > kMaxBatch) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (m == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (n == nullptr) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (b < 1 || b > kMaxNb) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (q < 0 || q > 16) { set_arg_error(6); return RRF_INVALID_ARG; }
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || m[i] < 1 || m[i] > (1 << 20)) { set_arg_error(3); return RRF_INVALID_ARG; }
    if (m[i] < n[i]) { set_arg_error(3); return RRF_UNSUPPORTED; }
  }
  rrf_batch_plan* pl = new rrf_batch_plan();
  pl->count = count;
  pl->nb = (int)b;
  pl->q = q;
  pl->m.assign(m, m + count);
  pl->n.assign(n, n + count);
  pl->max_m = *std::max_element(pl->m.begin(), pl->m.end());
  pl->max_n = *std::max_element(pl->n.begin(), pl->n.end());
  pl->table_bytes = align_up(sizeof(BMat) * count, 256);
  size_t off = kHeaderBytes + pl->table_bytes;
  pl->offsets.resize(count);
  for (int i = 0; i < count; ++i) {
    const size_t mi = pl->m[i], ni = pl->n[i], mx = std::max(mi, ni);
    const size_t np = (ni + b - 1) / b;
    pl->offsets[i] = off;
    off += align_up(sizeof(float) * mi * ni, 256);           // W
    off += align_up(sizeof(float) * mi * ni, 256);           // Ys
    off += align_up(sizeof(float) * np * b * b, 256);        // Tall
    off += 2 * align_up(sizeof(float) * b * mx, 256);        // Wa, Wb
    off += align_up(sizeof(float) * ni, 256);                // tau
  }
  pl->ws_bytes = off;
  pl->host_table.resize(count);
  if (cudaMallocHost(&pl->pinned, sizeof(BMat) * count) != cudaSuccess) {
    delete pl;
    return RRF_CUDA_ERROR;
  }
  *out = pl;
  return RRF_OK;
}

extern "C" size_t rrf_batch_plan_workspace(const rrf_batch_plan* pl) { return pl ? pl->ws_bytes : 0; }

extern "C" int rrf_batch_plan_tiles(const rrf_batch_plan* pl, int which) {
  if (pl == nullptr) return -1;
  return which == 0 ? pl->tile_big : pl->tile_skinny;
}

extern "C" rrf_status rrf_batch_plan_destroy(rrf_batch_plan* pl) {
  if (pl == nullptr) return RRF_OK;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->pinned) cudaFreeHost(pl->pinned);
  delete pl;
  return RRF_OK;
}

extern "C" rrf_status rrf_powerurv_batched_f32(rrf_batch_plan* pl, const float* const* A, const int64_t* lda,
                                               float* const* U, const int64_t* ldu, float* const* T,
                                               const int64_t* ldt, float* const* V, const int64_t* ldv,
                                               uint64_t seed, void* workspace, size_t ws_bytes, void* stream) {
  clear_arg_error();
  if (pl == nullptr) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (A == nullptr || lda == nullptr || U == nullptr || ldu == nullptr || T == nullptr || ldt == nullptr ||
      V == nullptr || ldv == nullptr) {
    set_arg_error(2);
    return RRF_INVALID_ARG;
  }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) { set_arg_error(11); return RRF_INVALID_ARG; }
  if (ws_bytes < pl->ws_bytes) { set_arg_error(12); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* base = reinterpret_cast<char*>(workspace);
  bool changed = pl->exec == nullptr || pl->graph_ws != workspace || pl->graph_seed != seed || pl->graph_stream != s;
  for (int i = 0; i < pl->count; ++i) {
    const int64_t mi = pl->m[i], ni = pl->n[i], mx = std::max(mi, ni);
    if (A[i] == nullptr || lda[i] < mi || U[i] == nullptr || ldu[i] < mi || T[i] == nullptr || ldt[i] < mi ||
        V[i] == nullptr || ldv[i] < ni) {
      set_arg_error(2);
      return RRF_INVALID_ARG;
    }
    BMat bm;
    bm.m = (int)mi;
    bm.n = (int)ni;
    bm.lda = lda[i]; bm.ldu = ldu[i]; bm.ldt = ldt[i]; bm.ldv = ldv[i];
    bm.A = A[i]; bm.U = U[i]; bm.T = T[i]; bm.V = V[i];
    size_t off = pl->offsets[i];
    const size_t np = (ni + pl->nb - 1) / pl->nb;
    bm.W = reinterpret_cast<float*>(base + off); off += align_up(sizeof(float) * mi * ni, 256);
    bm.Ys = reinterpret_cast<float*>(base + off); off += align_up(sizeof(float) * mi * ni, 256);
    bm.Tall = reinterpret_cast<float*>(base + off); off += align_up(sizeof(float) * np * pl->nb * pl->nb, 256);
    bm.Wa = reinterpret_cast<float*>(base + off); off += align_up(sizeof(float) * pl->nb * mx, 256);
    bm.Wb = reinterpret_cast<float*>(base + off); off += align_up(sizeof(float) * pl->nb * mx, 256);
    bm.tau = reinterpret_cast<float*>(base + off);
    if (std::memcmp(&bm, &pl->host_table[i], sizeof(BMat)) != 0) changed = true;
    pl->host_table[i] = bm;
  }
  const BMat* dmats = reinterpret_cast<const BMat*>(base + kHeaderBytes);
  if (changed) {
    std::memcpy(pl->pinned, pl->host_table.data(), sizeof(BMat) * pl->count);
    RRF_CUDA_TRY(cudaMemsetAsync(base, 0, kHeaderBytes, s));
    RRF_CUDA_TRY(cudaMemcpyAsync(const_cast<BMat*>(dmats), pl->pinned, sizeof(BMat) * pl->count,
                                 cudaMemcpyHostToDevice, s));
    if (pl->tile_big < 0) RRF_CUDA_TRY(autotune(pl, dmats, s));
    if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
    if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
    cudaStream_t cap;
    RRF_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    RRF_CUDA_TRY(cudaStreamSynchronize(s));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int64_t before = rrf_launch_count();
      enqueue_all(pl, dmats, seed, cap);
      pl->graph_kernels = rrf_launch_count() - before;
      add_launches(-pl->graph_kernels);  // captured, not launched
      e = cudaStreamEndCapture(cap, &pl->graph);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return RRF_CUDA_ERROR;
    RRF_CUDA_TRY(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
    pl->graph_ws = workspace;
    pl->graph_seed = seed;
    pl->graph_stream = s;
  }
  RRF_CUDA_TRY(cudaGraphLaunch(pl->exec, s));
  add_launches(pl->graph_kernels);
  return RRF_OK;
}
