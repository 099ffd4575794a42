// Chunk products on the tcgen05 tensor cores (placeholder until the kernel lands).
#include "hmm_internal.cuh"

namespace hmm {

bool chunk_tc_supported(int K, int precision) {
    (void)K;
    (void)precision;
    return false;
}

cudaError_t launch_chunk_tc(int, int, int, int, int, const ConstLayout &, const float *,
                            const ChunkDesc *, const float2 *, float *, int32_t *, unsigned *,
                            cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace hmm
