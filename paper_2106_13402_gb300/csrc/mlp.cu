// mlp.cu -- the learned power-iteration policy: a 16 -> 64 -> 64 -> 4 MLP (ReLU, softmax over
// q = 0..3) with FP16 parameters and activations and FP32 accumulation; forward, backward and Adam
// kernels for training on the GPU, and the features each randUTV step feeds it.
//
// Parameters are packed as [W1 (64 x 16, row-major out x in), b1 (64), W2 (64 x 64), b2 (64),
// W3 (4 x 64), b3 (4)] = 5508 values.  Training keeps an FP32 master copy plus Adam moments.
//
// Features of step i (from the q = 0 sketch Y0 = T22^T G and the R factor of its Householder QR, whose
// diagonal magnitudes |R(j, j)| approximate the energy of T22 beyond its first j sampled directions, and
// from the singular values D of the previous step's b x b core, the exact spectrum just before the block):
//   f0..f7 = log10(|R(k_j, k_j)| / |R(0, 0)|), k_j = (j + 1) b / 8 - 1       (decay inside the block)
//   f8 = (i - 1) / steps                                                      (where in the factorization)
//   f9 = f10 = 0: reserved.  Features that scale with n or c (such as log2 n) would put every size the
//   network was not trained on outside its input range; size enters through f8 and the ratios below.
//   f11 = log10(|R(b-1, b-1)| / |R(b/2, b/2)|)                              (decay at the block edge)
//   f12 = mean_k log10(|R(k, k)| / |R(0, 0)|)
//   f13 = log10(|R(0, 0)| / D(b-1))         (energy of T22 against the last singular value before it)
//   f14 = log10(D(b-1) / D(0))              (decay rate over the previous block)
//   f15 = log10(|R(b-1, b-1)| / D(b-1))     (energy beyond the block against that singular value)
// f13..f15 are 0 at step 1 (no previous block); every feature is clamped to [-30, 30].
// The policy takes the smallest q whose cumulative softmax probability reaches kQConfidence, so an
// uncertain network errs towards more power iterations.
#include <algorithm>

#include "rrf_internal.cuh"

namespace rrf {

constexpr int kIn = 16, kH = 64, kOut = 4;
constexpr float kQConfidence = 0.8f;  // cumulative probability the chosen q must reach
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kOut * kH, kNumParams = kOffB3 + kOut;

namespace {

__device__ __forceinline__ float h2f(__half x) { return __half2float(x); }

// Forward of one sample with parameters in shared memory; returns logits, optionally the activations.
__device__ void mlp_forward_one(const __half* P, const float* x, float* z, __half* h1o, __half* h2o) {
  __half h1[kH], h2[kH];
#pragma unroll 4
  for (int o = 0; o < kH; ++o) {
    float acc = h2f(P[kOffB1 + o]);
#pragma unroll
    for (int i = 0; i < kIn; ++i) acc = fmaf(h2f(P[kOffW1 + o * kIn + i]), x[i], acc);
    h1[o] = __float2half(fmaxf(acc, 0.f));
  }
#pragma unroll 4
  for (int o = 0; o < kH; ++o) {
    float acc = h2f(P[kOffB2 + o]);
    for (int i = 0; i < kH; ++i) acc = fmaf(h2f(P[kOffW2 + o * kH + i]), h2f(h1[i]), acc);
    h2[o] = __float2half(fmaxf(acc, 0.f));
  }
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    float acc = h2f(P[kOffB3 + o]);
    for (int i = 0; i < kH; ++i) acc = fmaf(h2f(P[kOffW3 + o * kH + i]), h2f(h2[i]), acc);
    z[o] = acc;
  }
  if (h1o)
    for (int o = 0; o < kH; ++o) h1o[o] = h1[o];
  if (h2o)
    for (int o = 0; o < kH; ++o) h2o[o] = h2[o];
}

__global__ void mlp_forward_kernel(const __half* __restrict__ params, const float* __restrict__ X, int N,
                                   float* __restrict__ logits) {
  __shared__ __half P[kNumParams];
  for (int i = threadIdx.x; i < kNumParams; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    float x[kIn], z[kOut];
    for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)s * kIn + i];
    mlp_forward_one(P, x, z, nullptr, nullptr);
    for (int o = 0; o < kOut; ++o) logits[(int64_t)s * kOut + o] = z[o];
  }
}

// Per-sample pass of training: forward, softmax cross-entropy, and the backpropagated signals
// dz (N x 4), dh2 (N x 64), dh1 (N x 64) plus the activations h1, h2 (FP16) for the weight gradients.
__global__ void mlp_sample_grad_kernel(const __half* __restrict__ params, const float* __restrict__ X,
                                       const int* __restrict__ labels, int N, __half* __restrict__ H1,
                                       __half* __restrict__ H2, float* __restrict__ DZ, float* __restrict__ DH1,
                                       float* __restrict__ DH2, float* __restrict__ loss_per) {
  __shared__ __half P[kNumParams];
  for (int i = threadIdx.x; i < kNumParams; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    float x[kIn], z[kOut];
    __half h1[kH], h2[kH];
    for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)s * kIn + i];
    mlp_forward_one(P, x, z, h1, h2);
    float mx = z[0];
    for (int o = 1; o < kOut; ++o) mx = fmaxf(mx, z[o]);
    float e[kOut], se = 0.f;
    for (int o = 0; o < kOut; ++o) {
      e[o] = expf(z[o] - mx);
      se += e[o];
    }
    const int y = labels[s];
    float dz[kOut];
    for (int o = 0; o < kOut; ++o) dz[o] = e[o] / se - (o == y ? 1.f : 0.f);
    loss_per[s] = -(z[y] - mx - logf(se));
    float dh2[kH];
    for (int i = 0; i < kH; ++i) {
      float acc = 0.f;
      for (int o = 0; o < kOut; ++o) acc = fmaf(h2f(P[kOffW3 + o * kH + i]), dz[o], acc);
      dh2[i] = (h2f(h2[i]) > 0.f) ? acc : 0.f;
    }
    for (int i = 0; i < kH; ++i) {
      float acc = 0.f;
      for (int o = 0; o < kH; ++o) acc = fmaf(h2f(P[kOffW2 + o * kH + i]), dh2[o], acc);
      DH1[(int64_t)s * kH + i] = (h2f(h1[i]) > 0.f) ? acc : 0.f;
    }
    for (int i = 0; i < kH; ++i) {
      H1[(int64_t)s * kH + i] = h1[i];
      H2[(int64_t)s * kH + i] = h2[i];
      DH2[(int64_t)s * kH + i] = dh2[i];
    }
    for (int o = 0; o < kOut; ++o) DZ[(int64_t)s * kOut + o] = dz[o];
  }
}

// Weight gradients (mean over the N samples), one block per parameter row, samples summed in order
// by a fixed block reduction (deterministic).
__global__ void mlp_weight_grad_kernel(const float* __restrict__ X, const __half* __restrict__ H1,
                                       const __half* __restrict__ H2, const float* __restrict__ DZ,
                                       const float* __restrict__ DH1, const float* __restrict__ DH2, int N,
                                       float* __restrict__ grad) {
  // rows: 64 of W1 (+b1), 64 of W2 (+b2), 4 of W3 (+b3)
  const int row = blockIdx.x;
  int layer, o, nin;
  if (row < kH) { layer = 0; o = row; nin = kIn; }
  else if (row < 2 * kH) { layer = 1; o = row - kH; nin = kH; }
  else { layer = 2; o = row - 2 * kH; nin = kH; }
  __shared__ float red[256];
  const float inv = 1.f / (float)N;
  for (int i = 0; i <= nin; ++i) {  // i == nin: bias
    float acc = 0.f;
    for (int s = threadIdx.x; s < N; s += blockDim.x) {
      float d, a;
      if (layer == 0) { d = DH1[(int64_t)s * kH + o]; a = (i < nin) ? X[(int64_t)s * kIn + i] : 1.f; }
      else if (layer == 1) { d = DH2[(int64_t)s * kH + o]; a = (i < nin) ? __half2float(H1[(int64_t)s * kH + i]) : 1.f; }
      else { d = DZ[(int64_t)s * kOut + o]; a = (i < nin) ? __half2float(H2[(int64_t)s * kH + i]) : 1.f; }
      acc = fmaf(d, a, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      int idx;
      if (layer == 0) idx = (i < nin) ? kOffW1 + o * kIn + i : kOffB1 + o;
      else if (layer == 1) idx = (i < nin) ? kOffW2 + o * kH + i : kOffB2 + o;
      else idx = (i < nin) ? kOffW3 + o * kH + i : kOffB3 + o;
      grad[idx] = red[0] * inv;
    }
    __syncthreads();
  }
}

__global__ void mean_kernel(const float* __restrict__ v, int N, float* __restrict__ out) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int s = threadIdx.x; s < N; s += blockDim.x) acc += v[s];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (float)N;
}

// Adam (Kingma & Ba 2015) on the FP32 master copy; the FP16 parameters are refreshed from it.
__global__ void adam_kernel(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, __half* __restrict__ params, int step, float lr,
                            float beta1, float beta2, float eps) {
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNumParams; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    master[i] = w;
    params[i] = __float2half(w);
  }
}

// Features of one randUTV step (see the file comment) from the panel-factored q = 0 sketch.
__global__ void features_kernel(const double* __restrict__ Rdiag_src, int64_t ldr, int b,
                                const double* __restrict__ Dprev, int step, int steps, int64_t n, int64_t c,
                                float* __restrict__ f) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  auto d = [&](int k) { return fabs(Rdiag_src[k + (int64_t)k * ldr]) + 1e-300; };
  auto lg = [](double x) { return (float)fmin(30.0, fmax(-30.0, log10(x))); };
  const double d0 = d(0);
  for (int j = 0; j < 8; ++j) {
    int k = (j + 1) * b / 8 - 1;
    if (k < 0) k = 0;
    f[j] = lg(d(k) / d0);
  }
  f[8] = (float)(step - 1) / (float)steps;
  f[9] = 0.f;
  f[10] = 0.f;
  f[11] = lg(d(b - 1) / d(b / 2));
  double mean = 0.0;
  for (int k = 0; k < b; ++k) mean += log10(d(k) / d0);
  f[12] = (float)fmin(30.0, fmax(-30.0, mean / b));
  if (Dprev != nullptr) {
    const double dl = fabs(Dprev[b - 1]) + 1e-300, df = fabs(Dprev[0]) + 1e-300;
    f[13] = lg(d0 / dl);
    f[14] = lg(dl / df);
    f[15] = lg(d(b - 1) / dl);
  } else {
    f[13] = f[14] = f[15] = 0.f;
  }
}

// Policy inference for one feature vector: argmax of the logits -> q (device int).
__global__ void policy_kernel(const __half* __restrict__ params, const float* __restrict__ f, int* q_out,
                              float* logits_out) {
  __shared__ __half P[kNumParams];
  for (int i = threadIdx.x; i < kNumParams; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    float x[kIn], z[kOut];
    for (int i = 0; i < kIn; ++i) x[i] = f[i];
    mlp_forward_one(P, x, z, nullptr, nullptr);
    float zmax = z[0];
    for (int o = 1; o < kOut; ++o) zmax = fmaxf(zmax, z[o]);
    float e[kOut], tot = 0.f;
    for (int o = 0; o < kOut; ++o) tot += (e[o] = expf(z[o] - zmax));
    int pick = kOut - 1;
    float cum = 0.f;
    for (int o = 0; o < kOut; ++o) {
      cum += e[o];
      if (cum >= kQConfidence * tot) { pick = o; break; }
    }
    *q_out = pick;
    if (logits_out)
      for (int o = 0; o < kOut; ++o) logits_out[o] = z[o];
  }
}

}  // namespace

// ---- internal entry points used by the randUTV driver --------------------------------------------------
cudaError_t policy_features(const double* Rfac, int64_t ldr, int b, const double* Dprev, int step, int steps,
                            int64_t n, int64_t c, float* feat, cudaStream_t s) {
  features_kernel<<<1, 32, 0, s>>>(Rfac, ldr, b, Dprev, step, steps, n, c, feat);
  count_launch();
  return cudaGetLastError();
}

cudaError_t policy_decide(const void* params, const float* feat, int* q_dev, cudaStream_t s) {
  policy_kernel<<<1, 128, 0, s>>>(reinterpret_cast<const __half*>(params), feat, q_dev, nullptr);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rrf

using namespace rrf;

extern "C" int rrf_mlp_param_count(void) { return kNumParams; }

extern "C" size_t rrf_mlp_train_workspace(int N) {
  if (N < 1) return 0;
  size_t b = 0;
  b += align_up(sizeof(__half) * (size_t)N * kH, 256) * 2;  // H1, H2
  b += align_up(sizeof(float) * (size_t)N * kOut, 256);     // DZ
  b += align_up(sizeof(float) * (size_t)N * kH, 256) * 2;   // DH1, DH2
  b += align_up(sizeof(float) * (size_t)N, 256);            // loss per sample
  return b;
}

extern "C" rrf_status rrf_mlp_forward(const void* params, const float* X, int N, float* logits, void* stream) {
  clear_arg_error();
  if (params == nullptr) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (X == nullptr && N > 0) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (N < 0) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (logits == nullptr && N > 0) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (N == 0) return RRF_OK;
  const int blocks = std::min((N + 127) / 128, dev_info().sms * 4);
  mlp_forward_kernel<<<blocks, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const __half*>(params), X, N, logits);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RRF_OK : RRF_CUDA_ERROR;
}

extern "C" rrf_status rrf_mlp_grad(const void* params, const float* X, const int* labels, int N, float* grad,
                                   float* loss, void* workspace, size_t ws_bytes, void* stream) {
  clear_arg_error();
  if (params == nullptr) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (X == nullptr) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (labels == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (N < 1) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (grad == nullptr) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (ws_bytes < rrf_mlp_train_workspace(N)) { set_arg_error(8); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* base = reinterpret_cast<char*>(workspace);
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base + off; off += align_up(bytes, 256); return p; };
  __half* H1 = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)N * kH));
  __half* H2 = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)N * kH));
  float* DZ = reinterpret_cast<float*>(take(sizeof(float) * (size_t)N * kOut));
  float* DH1 = reinterpret_cast<float*>(take(sizeof(float) * (size_t)N * kH));
  float* DH2 = reinterpret_cast<float*>(take(sizeof(float) * (size_t)N * kH));
  float* LP = reinterpret_cast<float*>(take(sizeof(float) * (size_t)N));
  const int blocks = std::min((N + 127) / 128, dev_info().sms * 4);
  mlp_sample_grad_kernel<<<blocks, 128, 0, s>>>(reinterpret_cast<const __half*>(params), X, labels, N, H1, H2, DZ,
                                                DH1, DH2, LP);
  count_launch();
  mlp_weight_grad_kernel<<<2 * kH + kOut, 256, 0, s>>>(X, H1, H2, DZ, DH1, DH2, N, grad);
  count_launch();
  if (loss != nullptr) {
    mean_kernel<<<1, 256, 0, s>>>(LP, N, loss);
    count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? RRF_OK : RRF_CUDA_ERROR;
}

extern "C" rrf_status rrf_mlp_adam(float* master, float* m, float* v, const float* grad, void* params, int step,
                                   float lr, void* stream) {
  clear_arg_error();
  if (master == nullptr || m == nullptr || v == nullptr || grad == nullptr || params == nullptr) {
    set_arg_error(1);
    return RRF_INVALID_ARG;
  }
  if (step < 1) { set_arg_error(6); return RRF_INVALID_ARG; }
  adam_kernel<<<(kNumParams + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      master, m, v, grad, reinterpret_cast<__half*>(params), step, lr, 0.9f, 0.999f, 1e-8f);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RRF_OK : RRF_CUDA_ERROR;
}
