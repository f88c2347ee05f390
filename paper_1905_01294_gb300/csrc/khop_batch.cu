// Bit-sliced 64-lane batched k-hop count (placeholder until the kernel lands).
#include "khop_internal.cuh"

namespace khop {

int batch_launch(khop_graph *, const uint32_t *, const uint32_t *, uint64_t, uint64_t *,
                 cudaStream_t) {
    return KHOP_EINVAL;
}

}  // namespace khop
