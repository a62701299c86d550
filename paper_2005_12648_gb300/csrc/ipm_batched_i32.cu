// Batched segmented merge kernels for int32_t keys (one translation unit per key type so
// the variants compile in parallel).
#include "ipm_batched.cuh"

namespace ipm {

ipm_status batched_launch_i32(void *buf, uint32_t *vals, uint64_t buf_len,
                               batched::QueueArea qa, uint32_t nseg, uint32_t variant,
                               uint32_t ctas_per_sm, uint32_t one_launch,
                               const ipm_segment *segs, uint32_t by_size, StatusBlock *sb,
                               cudaStream_t stream) {
    return batched::batched_dispatch<int32_t>(buf, vals, buf_len, qa, nseg, variant, ctas_per_sm,
                                          one_launch, segs, by_size, sb, stream);
}

}  // namespace ipm
