// noalloc.cu -- rrf_panel_qr_noalloc: the Householder panel QR without any caller-provided workspace.
//
// Some callers cannot hand this library device memory for scratch: code that runs under a memory
// manager which owns the whole device (where a raw cudaMalloc would fail or fragment its pool),
// and latency-critical loops that must not allocate once they are running.  For them this entry
// point keeps the panel kernel's scratch -- the status word and grid-barrier counters, the per-CTA
// partial sums and the owner's copy of the current row -- in one fixed array in device global
// memory that every GPU loading the library holds until the process exits.
#include <mutex>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

// 2 MiB: header (256 B) + partial sums 2 x nb x w doubles + row copies 2 x w doubles + the w x w
// region the panel layout reserves for a Gram matrix; for w <= 256 and nb <= 152 CTAs (one per SM on
// GB300) that is at most 1,151,232 bytes.
constexpr size_t kNoAllocBytes = size_t(2) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array for the current device, looked up once per device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in, never a device address.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rrf

using namespace rrf;

extern "C" rrf_status rrf_panel_qr_noalloc(int64_t r, int64_t w, double* P, int64_t ldp, double* tau, double* Y,
                                           int64_t ldy, int* status, void* stream) {
  clear_arg_error();
  if (r < 1) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (w < 1 || w > 256 || w > r) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (P == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (ldp < r) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (tau == nullptr) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (Y == nullptr) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (ldy < r) { set_arg_error(7); return RRF_INVALID_ARG; }
  // The kernel's scratch for this shape.  No compact-WY factor is formed, so the split-K scratch of
  // its Gram-matrix GEMM is not needed.
  GemmDesc gram;
  gram.M = w; gram.N = w; gram.K = r;
  const size_t need = kHeaderBytes + panel_scratch_bytes(r, w) - gemm_scratch_bytes(&gram, 1);
  if (need > kNoAllocBytes) { set_arg_error(1); return RRF_UNSUPPORTED; }
  void* base = nullptr;
  RRF_CUDA_TRY(scratch_address(&base));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
  // The array keeps the previous call's contents: the status word and barrier counters must start at 0.
  RRF_CUDA_TRY(cudaMemsetAsync(hdr, 0, kHeaderBytes, s));
  RRF_CUDA_TRY(panel_qr(r, w, P, ldp, tau, Y, ldy, nullptr, 0, nullptr, 0,
                        reinterpret_cast<double*>(reinterpret_cast<char*>(base) + kHeaderBytes),
                        kNoAllocBytes - kHeaderBytes, hdr, s));
  if (status != nullptr)
    RRF_CUDA_TRY(cudaMemcpyAsync(status, &hdr->status, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return RRF_OK;
}
