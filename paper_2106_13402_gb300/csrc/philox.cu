// philox.cu -- the Gaussian matrices of Algorithms 1 and 3 (randn), drawn on the device.
//
// Counter-based Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64-bit
// multiplies (round multipliers 0xD2511F53, 0xCD9E8D57) with the key bumped by the Weyl constants
// 0x9E3779B9, 0xBB67AE85 between rounds.  Block t of a draw uses counter (t lo, t hi, step, tag) under
// key (seed lo, seed hi) and feeds column-major elements 2t and 2t+1 through Box-Muller.  Because the
// stream is indexed by t, every thread computes its own block with no shared state.
#include <algorithm>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

__device__ __forceinline__ void philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             uint32_t k0, uint32_t k1, uint32_t out[4]) {
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
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

__global__ void randn_kernel(double* __restrict__ G, int64_t rows, int64_t ldg, int64_t total,
                             uint32_t k0, uint32_t k1, uint32_t step, uint32_t tag) {
  const int64_t nblocks = (total + 1) / 2;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nblocks;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x[4];
    philox_block((uint32_t)t, (uint32_t)((uint64_t)t >> 32), step, tag, k0, k1, x);
    const uint64_t a = ((uint64_t)x[0] << 32) | x[1];
    const uint64_t c = ((uint64_t)x[2] << 32) | x[3];
    const double u1 = (double)((a >> 11) + 1) * 0x1p-53;
    const double u2 = (double)(c >> 11) * 0x1p-53;
    const double rho = sqrt(-2.0 * log(u1));
    const double ang = two_pi * u2;
    double sn, cs;
    sincos(ang, &sn, &cs);
    const int64_t lin0 = 2 * t;
    G[(lin0 % rows) + (lin0 / rows) * ldg] = rho * cs;
    const int64_t lin1 = lin0 + 1;
    if (lin1 < total) G[(lin1 % rows) + (lin1 / rows) * ldg] = rho * sn;
  }
}

}  // namespace

cudaError_t randn_f64(int64_t rows, int64_t cols, double* G, int64_t ldg, uint64_t seed, uint32_t step,
                      uint32_t tag, cudaStream_t stream) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int64_t nblocks = (total + 1) / 2;
  const int threads = 256;
  const int64_t grid = std::min<int64_t>((nblocks + threads - 1) / threads, (int64_t)dev_info().sms * 32);
  randn_kernel<<<(unsigned)grid, threads, 0, stream>>>(G, rows, ldg, total, (uint32_t)seed,
                                                        (uint32_t)(seed >> 32), step, tag);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rrf
