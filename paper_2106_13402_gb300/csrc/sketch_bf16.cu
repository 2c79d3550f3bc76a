// sketch_bf16.cu -- BF16 tensor-core sketch (placeholder until the tcgen05 kernel lands).
#include "rrf_internal.cuh"

namespace rrf {

size_t sketch_bf16_scratch_bytes(int64_t, int64_t, int64_t) { return 256; }

cudaError_t sketch_bf16(int64_t, int64_t, int64_t, const double*, int64_t, const double*, int, double*, double*,
                        double*, char*, size_t, double*, size_t, double*, size_t, WsHeader*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace rrf
