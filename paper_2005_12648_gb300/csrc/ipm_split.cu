// Split step: early-exit test (Alg. 2/3) and exact stable merge-path splits (Sec. 3.1).
//
// For a diagonal d (an output count), the stable split i is the number of A elements
// among the first d keys of the stable merge; A[m] is among them exactly when
// A[m] <= B[d-1-m].  That predicate is true for m < i and false for m >= i, so one
// warp brackets i with 32 evenly spaced probes per step: the ballot of the probes is
// a prefix of ones, its popcount locates the bracket, and the range shrinks ~33x per
// step (log_33 of the run length dependent steps instead of log_2).
#include "ipm_internal.h"

namespace ipm {

namespace {

template <typename K>
__global__ void early_exit_kernel(const K *buf, uint64_t la, uint64_t lb, StatusBlock *sb) {
    if (threadIdx.x == 0) {
        unsigned int done = (la == 0 || lb == 0) ? 1u : 0u;
        if (!done) done = key_le(buf[la - 1], buf[la]) ? 1u : 0u;
        sb->status = 0u;
        sb->done = done;
        sb->exchange_bytes = 0ull;
        for (int q = 0; q < 60; ++q) sb->counters[q] = 0u;
    }
}

template <typename K>
__global__ void __launch_bounds__(256) split_kernel(const K *__restrict__ A, uint64_t la,
                                                    const K *__restrict__ B, uint64_t lb,
                                                    uint64_t P, uint64_t *__restrict__ out,
                                                    const StatusBlock *sb) {
    if (sb != nullptr && *((volatile const unsigned int *)&sb->done)) return;
    const uint64_t k = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (k > P) return;  // whole warp exits together
    const uint64_t n = la + lb;
    const uint64_t d = (k * n) / P;
    uint64_t lo = d > lb ? d - lb : 0;
    uint64_t hi = d < la ? d : la;
    while (hi - lo > 32) {
        const uint64_t R = hi - lo;
        const uint64_t m = lo + (R * (lane + 1)) / 33;  // strictly increasing, in [lo,hi)
        const bool p = key_le(__ldg(A + m), __ldg(B + (d - 1 - m)));
        const unsigned bal = __ballot_sync(0xffffffffu, p);
        const int c = __popc(bal);
        const uint64_t m_lo = __shfl_sync(0xffffffffu, m, c > 0 ? c - 1 : 0);
        const uint64_t m_hi = __shfl_sync(0xffffffffu, m, c < 32 ? c : 31);
        const uint64_t nlo = c > 0 ? m_lo + 1 : lo;
        const uint64_t nhi = c < 32 ? m_hi : hi;
        lo = nlo;
        hi = nhi;
    }
    const uint64_t R = hi - lo;
    bool p = false;
    if (lane < R) {
        const uint64_t m = lo + lane;
        p = key_le(__ldg(A + m), __ldg(B + (d - 1 - m)));
    }
    const int c = __popc(__ballot_sync(0xffffffffu, p));
    if (lane == 0) out[k] = lo + uint64_t(c);
}

template <typename K>
ipm_status splits_t(const void *buf, uint64_t la, uint64_t lb, uint64_t P, uint64_t *split,
                    const StatusBlock *sb, cudaStream_t stream) {
    const K *A = static_cast<const K *>(buf);
    const uint64_t warps = P + 1;
    const uint64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > 0x7fffffffull) return IPM_ERR_INVALID_ARG;
    split_kernel<K><<<unsigned(blocks), 256, 0, stream>>>(A, la, A + la, lb, P, split, sb);
    return last_launch_status();
}

}  // namespace

ipm_status launch_early_exit(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                             StatusBlock *sb, cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        early_exit_kernel<int32_t><<<1, 32, 0, stream>>>((const int32_t *)buf, la, lb, sb);
        break;
    case IPM_UINT32:
        early_exit_kernel<uint32_t><<<1, 32, 0, stream>>>((const uint32_t *)buf, la, lb, sb);
        break;
    case IPM_UINT64:
        early_exit_kernel<uint64_t><<<1, 32, 0, stream>>>((const uint64_t *)buf, la, lb, sb);
        break;
    case IPM_FLOAT32:
        early_exit_kernel<float><<<1, 32, 0, stream>>>((const float *)buf, la, lb, sb);
        break;
    default:
        return IPM_ERR_UNSUPPORTED_DTYPE;
    }
    return last_launch_status();
}

ipm_status launch_splits(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                         uint64_t P, uint64_t *split, const StatusBlock *sb,
                         cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        return splits_t<int32_t>(buf, la, lb, P, split, sb, stream);
    case IPM_UINT32:
        return splits_t<uint32_t>(buf, la, lb, P, split, sb, stream);
    case IPM_UINT64:
        return splits_t<uint64_t>(buf, la, lb, P, split, sb, stream);
    case IPM_FLOAT32:
        return splits_t<float>(buf, la, lb, P, split, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
