// gemm_f64.cu -- FP64 GEMM for the sketch products and compact-WY updates of Algorithms 1 and 3.
//
// On GB300 the FP64 rate is ~2 DFMA/clk/SM (measured 1.19 TFLOP/s with DFMA, 1.04 with the legacy
// m8n8k4 f64 mma.sync), and tcgen05 has no f64 kind, so FP64 GEMMs run on the DFMA pipe.  A 64 x 64
// output tile with a 4 x 4 register micro-tile per thread reads 8 operands from shared memory per
// 16 DFMAs, far below what the shared-memory and L2 paths sustain; the DFMA pipe is the bound, so
// the design goal is keeping every SM's pipe busy: up to four independent problems share one launch
// and thin outputs are split along K (deterministic two-pass reduction) until the units fill the
// SMs evenly.
#include <algorithm>
#include <mutex>
#include <vector>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int kMaxProb = 4;

struct Prob {
  GemmDesc d;
  int tiles_m, tiles_n, splits;
  int64_t kchunk;
  double* part;        // [splits][N][M] partial sums when splits > 1
  int64_t unit_begin;  // first CTA of this problem in the launch
  int64_t elem_begin;  // first element index of this problem in the reduction launch
};
struct Batch {
  Prob p[kMaxProb];
  int count;
  int64_t total_units;
  int64_t total_elems;  // sum of M*N over split problems
};

__global__ void __launch_bounds__(NT) gemm_f64_kernel(const __grid_constant__ Batch batch) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  int pi = 0;
  for (int i = 1; i < batch.count; ++i)
    if ((int64_t)blockIdx.x >= batch.p[i].unit_begin) pi = i;
  const Prob& P = batch.p[pi];
  const GemmDesc& d = P.d;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t unit = (int64_t)blockIdx.x - P.unit_begin;
  const int64_t tiles = (int64_t)P.tiles_m * P.tiles_n;
  const int split = (int)(unit / tiles);
  const int64_t t = unit % tiles;
  const int64_t m0 = (t % P.tiles_m) * BM, n0 = (t / P.tiles_m) * BN;
  const int64_t kb = (int64_t)split * P.kchunk;
  const int64_t ke = min(d.K, kb + P.kchunk);
  const int64_t M = d.M, N = d.N;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    if (!d.ta) {  // element (m, k) at A[m + k lda]: consecutive threads walk m
      const int m = tid & 63;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = (tid >> 6) + 4 * e;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < M && gk < ke) ? d.A[gm + gk * d.lda] : 0.0;
      }
    } else {  // element (m, k) at A[k + m lda]: consecutive threads walk k
      const int k = tid & 15;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = (tid >> 4) + 16 * e;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < M && gk < ke) ? d.A[gk + gm * d.lda] : 0.0;
      }
    }
    if (!d.tb) {  // element (k, n) at B[k + n ldb]
      const int k = tid & 15;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int n = (tid >> 4) + 16 * e;
        const int64_t gn = n0 + n, gk = k0 + k;
        Bs[k][n] = (gn < N && gk < ke) ? d.B[gk + gn * d.ldb] : 0.0;
      }
    } else {  // element (k, n) at B[n + k ldb]
      const int n = tid & 63;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = (tid >> 6) + 4 * e;
        const int64_t gn = n0 + n, gk = k0 + k;
        Bs[k][n] = (gn < N && gk < ke) ? d.B[gn + gk * d.ldb] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t gn = n0 + ty + 16 * j;
    if (gn >= N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t gm = m0 + tx + 16 * i;
      if (gm >= M) continue;
      if (P.splits == 1) {
        double v = d.alpha * acc[i][j];
        if (d.beta != 0.0) v = fma(d.beta, d.C[gm + gn * d.ldc], v);
        d.C[gm + gn * d.ldc] = v;
      } else {
        P.part[((int64_t)split * N + gn) * M + gm] = acc[i][j];
      }
    }
  }
}

// Sums the split-K partials in split order: C = alpha * sum_s part[s] + beta * C.
__global__ void gemm_reduce_kernel(const __grid_constant__ Batch batch) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < batch.total_elems;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int pi = -1;
    for (int i = 0; i < batch.count; ++i)
      if (batch.p[i].splits > 1 && idx >= batch.p[i].elem_begin) pi = i;
    const Prob& P = batch.p[pi];
    const int64_t local = idx - P.elem_begin;
    const int64_t M = P.d.M, N = P.d.N;
    const int64_t gm = local % M, gn = local / M;
    double s = 0.0;
    for (int sp = 0; sp < P.splits; ++sp) s += P.part[((int64_t)sp * N + gn) * M + gm];
    double v = P.d.alpha * s;
    if (P.d.beta != 0.0) v = fma(P.d.beta, P.d.C[gm + gn * P.d.ldc], v);
    P.d.C[gm + gn * P.d.ldc] = v;
  }
}

int plan_splits(const GemmDesc& d, int sms) {
  const int64_t tiles = ((d.M + BM - 1) / BM) * ((d.N + BN - 1) / BN);
  if (tiles >= 4LL * sms || d.K < 64) return 1;
  const int max_s = (int)std::min<int64_t>(32, d.K / 32);
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= max_s; ++s) {
    const int64_t units = tiles * s;
    const int64_t waves = (units + sms - 1) / sms;
    const double eff = (double)units / (double)(waves * sms);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = s;
    }
    if (eff >= 0.94) break;
  }
  return best;
}

// Optional instrumentation: CUDA events around each launch (diagnostics API of rrf.h).
// Event pairs around GEMM launches while profiling is on; kind 0 = DFMA GEMM (kernel + split-K reduce),
// kind 1 = the emulated GEMM's tensor-core kernel, kind 2 = the BF16 sketch GEMM's tensor-core kernel,
// kind 3 = the Householder panel kernel.
constexpr int kKinds = 4;
struct GemmProfile {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  std::vector<double> flops, tflops, bytes;
  size_t used = 0;
  double ms_k[kKinds] = {}, flops_k[kKinds] = {}, tflops_k[kKinds] = {}, bytes_k[kKinds] = {};
  int64_t launches_k[kKinds] = {};
};
GemmProfile& prof() {
  static GemmProfile p;
  return p;
}

}  // namespace

cudaEvent_t profile_launch_begin(int kind, double flops, double tensor_flops, cudaStream_t stream, double bytes) {
  GemmProfile& pf = prof();
  if (!pf.on) return nullptr;
  std::lock_guard<std::mutex> lock(pf.mu);
  if (!pf.on || pf.used + 2 > pf.ev.size()) return nullptr;
  cudaEventRecord(pf.ev[pf.used], stream);
  const size_t r = pf.used / 2;
  pf.kind[r] = kind;
  pf.flops[r] = flops;
  pf.tflops[r] = tensor_flops;
  pf.bytes[r] = bytes;
  cudaEvent_t end = pf.ev[pf.used + 1];
  pf.used += 2;
  return end;
}

size_t gemm_scratch_bytes(const GemmDesc* d, int count) {
  const int sms = dev_info().sms;
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const int s = plan_splits(d[i], sms);
    if (s > 1) total += align_up((size_t)s * d[i].M * d[i].N * sizeof(double), 256);
  }
  return total;
}

cudaError_t gemm_f64(const GemmDesc* d, int count, double* scratch, size_t scratch_bytes,
                     cudaStream_t stream) {
  if (count <= 0 || count > kMaxProb) return cudaErrorInvalidValue;
  const int sms = dev_info().sms;
  Batch batch{};
  batch.count = 0;
  int64_t units = 0, elems = 0;
  size_t used = 0;
  for (int i = 0; i < count; ++i) {
    if (d[i].M <= 0 || d[i].N <= 0) continue;
    Prob& P = batch.p[batch.count];
    P.d = d[i];
    P.tiles_m = (int)((d[i].M + BM - 1) / BM);
    P.tiles_n = (int)((d[i].N + BN - 1) / BN);
    int s = d[i].K > 0 ? plan_splits(d[i], sms) : 1;
    // Clamp to the scratch that is left.
    while (s > 1) {
      size_t need = align_up((size_t)s * d[i].M * d[i].N * sizeof(double), 256);
      if (scratch != nullptr && used + need <= scratch_bytes) break;
      --s;
    }
    int64_t kchunk = d[i].K;
    if (s > 1) {
      kchunk = ((d[i].K + s - 1) / s + BK - 1) / BK * BK;
      s = (int)((d[i].K + kchunk - 1) / kchunk);
    }
    P.splits = s;
    P.kchunk = std::max<int64_t>(kchunk, 1);
    P.part = nullptr;
    if (s > 1) {
      P.part = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) + used);
      used += align_up((size_t)s * d[i].M * d[i].N * sizeof(double), 256);
      P.elem_begin = elems;
      elems += d[i].M * d[i].N;
    }
    P.unit_begin = units;
    units += (int64_t)P.tiles_m * P.tiles_n * s;
    ++batch.count;
  }
  if (batch.count == 0) return cudaSuccess;
  batch.total_units = units;
  batch.total_elems = elems;
  double fl = 0.0;
  for (int i = 0; i < batch.count; ++i) fl += 2.0 * batch.p[i].d.M * batch.p[i].d.N * batch.p[i].d.K;
  cudaEvent_t ev_end = profile_launch_begin(0, fl, 0.0, stream);
  gemm_f64_kernel<<<(unsigned)units, NT, 0, stream>>>(batch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (elems > 0) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((elems + threads - 1) / threads, (int64_t)sms * 16);
    gemm_reduce_kernel<<<(unsigned)blocks, threads, 0, stream>>>(batch);
    count_launch();
    e = cudaGetLastError();
  }
  if (ev_end != nullptr) cudaEventRecord(ev_end, stream);
  return e;
}

}  // namespace rrf

extern "C" int rrf_gemm_profile_begin(int max_launches) {
  rrf::GemmProfile& pf = rrf::prof();
  std::lock_guard<std::mutex> lock(pf.mu);
  const size_t want = (size_t)2 * (max_launches > 0 ? max_launches : 0);
  while (pf.ev.size() < want) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return 1;
    pf.ev.push_back(e);
  }
  pf.kind.assign(pf.ev.size() / 2, 0);
  pf.flops.assign(pf.ev.size() / 2, 0.0);
  pf.tflops.assign(pf.ev.size() / 2, 0.0);
  pf.bytes.assign(pf.ev.size() / 2, 0.0);
  pf.used = 0;
  for (int k = 0; k < rrf::kKinds; ++k) {
    pf.ms_k[k] = pf.flops_k[k] = pf.tflops_k[k] = pf.bytes_k[k] = 0.0;
    pf.launches_k[k] = 0;
  }
  pf.on = true;
  return 0;
}

extern "C" int rrf_gemm_profile_end(double* ms, double* flops, int64_t* launches) {
  rrf::GemmProfile& pf = rrf::prof();
  std::lock_guard<std::mutex> lock(pf.mu);
  if (pf.on) {
    pf.on = false;
    for (size_t i = 0; i + 1 < pf.used; i += 2) {
      if (cudaEventSynchronize(pf.ev[i + 1]) != cudaSuccess) return 1;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pf.ev[i], pf.ev[i + 1]) != cudaSuccess) return 1;
      const int k = pf.kind[i / 2];
      if (k < 0 || k >= rrf::kKinds) continue;
      pf.ms_k[k] += t;
      pf.flops_k[k] += pf.flops[i / 2];
      pf.tflops_k[k] += pf.tflops[i / 2];
      pf.bytes_k[k] += pf.bytes[i / 2];
      pf.launches_k[k] += 1;
    }
  }
  if (ms) *ms = pf.ms_k[0];
  if (flops) *flops = pf.flops_k[0];
  if (launches) *launches = pf.launches_k[0];
  return 0;
}

extern "C" int rrf_gemm_profile_bf16(double* ms, double* flops, double* bytes, int64_t* launches) {
  rrf::GemmProfile& pf = rrf::prof();
  std::lock_guard<std::mutex> lock(pf.mu);
  if (pf.on) return 1;
  if (ms) *ms = pf.ms_k[2];
  if (flops) *flops = pf.flops_k[2];
  if (bytes) *bytes = pf.tflops_k[2];
  if (launches) *launches = pf.launches_k[2];
  return 0;
}

extern "C" int rrf_gemm_profile_emulated(double* ms, double* flops, double* tensor_flops, int64_t* launches) {
  rrf::GemmProfile& pf = rrf::prof();
  std::lock_guard<std::mutex> lock(pf.mu);
  if (pf.on) return 1;
  if (ms) *ms = pf.ms_k[1];
  if (flops) *flops = pf.flops_k[1];
  if (tensor_flops) *tensor_flops = pf.tflops_k[1];
  if (launches) *launches = pf.launches_k[1];
  return 0;
}

extern "C" int rrf_gemm_profile_emulated_bytes(double* bytes) {
  rrf::GemmProfile& pf = rrf::prof();
  std::lock_guard<std::mutex> lock(pf.mu);
  if (pf.on) return 1;
  if (bytes) *bytes = pf.bytes_k[1];
  return 0;
}

extern "C" int rrf_gemm_profile_panel(double* ms, double* flops, double* bytes, int64_t* launches) {
  rrf::GemmProfile& pf = rrf::prof();
  std::lock_guard<std::mutex> lock(pf.mu);
  if (pf.on) return 1;
  if (ms) *ms = pf.ms_k[3];
  if (flops) *flops = pf.flops_k[3];
  if (bytes) *bytes = pf.bytes_k[3];
  if (launches) *launches = pf.launches_k[3];
  return 0;
}
