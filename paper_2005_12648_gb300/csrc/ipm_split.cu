// Split step: early-exit test (Alg. 2/3) and the exact stable merge-path splits
// (Sec. 3.1) of every diagonal d_k = floor(k*n/P), one warp per diagonal
// (warp_split, ipm_split.cuh).
#include "ipm_internal.h"
#include "ipm_split.cuh"

namespace ipm {

namespace {

template <typename K>
__global__ void early_exit_kernel(const K *buf, uint64_t la, uint64_t lb, StatusBlock *sb,
                                  unsigned long long wait_limit_ns) {
    if (threadIdx.x == 0) {
        unsigned int done = (la == 0 || lb == 0) ? 1u : 0u;
        if (!done) done = key_le(buf[la - 1], buf[la]) ? 1u : 0u;
        sb->status = 0u;
        sb->done = done;
        sb->exchange_bytes = 0ull;
        sb->merge_bytes = 0ull;
        sb->wait_limit_ns = wait_limit_ns;
        for (int q = 0; q < kNumCounters; ++q) sb->counters[q] = 0u;
    }
}

// The diagonals k = 0, S, 2S, ..., P (S = stride, a divisor of P): one warp each, over
// the diagonal's whole range.
template <typename K>
__global__ void __launch_bounds__(256) split_kernel(const K *__restrict__ A, uint64_t la,
                                                    const K *__restrict__ B, uint64_t lb,
                                                    uint64_t P, uint64_t stride,
                                                    uint64_t *__restrict__ out,
                                                    const StatusBlock *sb) {
    if (call_finished(sb)) return;
    const uint64_t k = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * stride;
    const unsigned lane = threadIdx.x & 31u;
    if (k > P) return;  // whole warp exits together
    const uint64_t n = la + lb;
    const uint64_t d = (k * n) / P;
    const uint64_t i = warp_split<true>(A, la, B, lb, d);
    if (lane == 0) out[k] = i;
}

// The other diagonals, once those of split_kernel with this stride are known: both
// i_k and j_k = d_k - i_k grow with k, so between the coarse neighbours k0 < k < k1
//   max(i_k0, d_k - j_k1) <= i_k <= min(i_k1, d_k - j_k0),
// a bracket of at most d_k1 - d_k0 positions instead of the diagonal's whole range.
template <typename K>
__global__ void __launch_bounds__(256) split_fine_kernel(const K *__restrict__ A, uint64_t la,
                                                         const K *__restrict__ B, uint64_t lb,
                                                         uint64_t P, uint64_t stride,
                                                         uint64_t *__restrict__ out,
                                                         const StatusBlock *sb) {
    if (call_finished(sb)) return;
    const uint64_t k = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (k > P || k % stride == 0) return;  // whole warp exits together
    const uint64_t n = la + lb;
    const uint64_t k0 = k / stride * stride, k1 = k0 + stride;  // k1 <= P: stride | P
    const uint64_t d = (k * n) / P, d0 = (k0 * n) / P, d1 = (k1 * n) / P;
    const uint64_t i0 = out[k0], i1 = out[k1];
    const uint64_t j0 = d0 - i0, j1 = d1 - i1;
    uint64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    if (i0 > lo) lo = i0;
    if (d > j1 && d - j1 > lo) lo = d - j1;
    if (i1 < hi) hi = i1;
    if (d - j0 < hi) hi = d - j0;  // j0 <= j_k <= d
    const uint64_t i = warp_split_bracket<true>(A, B, d, lo, hi);
    if (lane == 0) out[k] = i;
}

// Coarse diagonals first when there are many: the fine ones then search ~32x narrower
// brackets (about two rounds of 33 probes fewer each).
constexpr uint64_t kSplitStride = 32;
constexpr uint64_t kTwoPassPairs = 2048;

bool two_pass(uint64_t P) { return P >= kTwoPassPairs && P % kSplitStride == 0; }

template <typename K>
ipm_status splits_t(const void *buf, uint64_t la, uint64_t lb, uint64_t P, uint64_t *split,
                    const StatusBlock *sb, cudaStream_t stream) {
    const K *A = static_cast<const K *>(buf);
    const bool two = two_pass(P);
    const uint64_t stride = two ? kSplitStride : 1;
    const uint64_t warps = P / stride + 1;
    const uint64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > 0x7fffffffull || (P + 1) * 32 / 256 + 1 > 0x7fffffffull)
        return IPM_ERR_INVALID_ARG;
    split_kernel<K><<<unsigned(blocks), 256, 0, stream>>>(A, la, A + la, lb, P, stride, split,
                                                          sb);
    if (!two) return last_launch_status();
    IPM_TRY(last_launch_status());
    const uint64_t fblocks = ((P + 1) * 32 + 255) / 256;
    split_fine_kernel<K><<<unsigned(fblocks), 256, 0, stream>>>(A, la, A + la, lb, P, stride,
                                                                split, sb);
    return last_launch_status();
}

}  // namespace

ipm_status launch_early_exit(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                             StatusBlock *sb, unsigned long long wait_limit_ns,
                             cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        early_exit_kernel<int32_t><<<1, 32, 0, stream>>>((const int32_t *)buf, la, lb, sb,
                                                         wait_limit_ns);
        break;
    case IPM_UINT32:
        early_exit_kernel<uint32_t><<<1, 32, 0, stream>>>((const uint32_t *)buf, la, lb, sb,
                                                         wait_limit_ns);
        break;
    case IPM_UINT64:
        early_exit_kernel<uint64_t><<<1, 32, 0, stream>>>((const uint64_t *)buf, la, lb, sb,
                                                         wait_limit_ns);
        break;
    case IPM_INT64:
        early_exit_kernel<int64_t><<<1, 32, 0, stream>>>((const int64_t *)buf, la, lb, sb,
                                                         wait_limit_ns);
        break;
    case IPM_FLOAT32:
        early_exit_kernel<float><<<1, 32, 0, stream>>>((const float *)buf, la, lb, sb,
                                                         wait_limit_ns);
        break;
    default:
        return IPM_ERR_UNSUPPORTED_DTYPE;
    }
    return last_launch_status();
}

uint32_t split_launches(uint64_t P) { return two_pass(P) ? 2u : 1u; }

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
    case IPM_INT64:
        return splits_t<int64_t>(buf, la, lb, P, split, sb, stream);
    case IPM_FLOAT32:
        return splits_t<float>(buf, la, lb, P, split, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
