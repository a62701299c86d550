// Merge step: every pair (A_k, B_k) of the arranged buffer is merged stably in place by
// one CTA (the per-thread std::inplace_merge of Alg. 2/3, here per CTA).
//
// Pair k occupies [d_k, d_{k+1}) as A[i_k, i_{k+1}) | B[j_k, j_{k+1}); the shared-memory
// merge of one pair is merge_pair_smem (ipm_tile_merge.cuh).  The kernel is persistent
// (one CTA per SM, grid-stride over pairs); a pair never straddles two CTAs, so the
// in-place write-back touches only the CTA's own range.
#include "ipm_internal.h"
#include "ipm_tile_merge.cuh"

namespace ipm {

namespace {

template <typename K, bool KV, int THREADS, int E>
__global__ void __launch_bounds__(THREADS, 1)
    tile_merge_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, uint64_t la,
                      uint64_t lb, const uint64_t *__restrict__ split, uint32_t G,
                      StatusBlock *sb) {
    using Shape = TileShape<K, KV, THREADS, E>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    __shared__ int abort_flag;
    K *skeys = reinterpret_cast<K *>(smem_raw + 128);
    uint32_t *svals = reinterpret_cast<uint32_t *>(smem_raw + 128 + Shape::kKeyBytes);
    if (sb != nullptr && *((volatile unsigned int *)&sb->done)) return;

    const uint32_t tid = threadIdx.x;
    const uint64_t n = la + lb;
    const uint64_t P = 1ull << G;
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        abort_flag = 0;
    }
    __syncthreads();
    uint32_t parity = 0;

    for (uint64_t k = blockIdx.x; k < P; k += gridDim.x) {
        const uint64_t d0 = (k * n) >> G, d1 = ((k + 1) * n) >> G;
        const uint32_t c = uint32_t(d1 - d0);
        const uint32_t a = uint32_t(split[k + 1] - split[k]);
        if (c == 0) continue;
        if (split[k + 1] < split[k] || a > c) {  // inconsistent split table
            if (tid == 0 && sb != nullptr) set_status(sb, IPM_ERR_DEVICE);
            continue;
        }
        if (merge_pair_smem<K, KV, THREADS, E>(buf + d0, KV ? vals + d0 : nullptr, a, c, skeys,
                                               svals, mbar, parity, abort_flag,
                                               sb) == kPairAbort)
            break;
    }
    if (tid == 0) bulk_wait_all0();
}

template <typename K, bool KV, int THREADS, int E>
ipm_status tile_merge_t(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                        const uint64_t *split, uint32_t G, StatusBlock *sb,
                        cudaStream_t stream) {
    using Shape = TileShape<K, KV, THREADS, E>;
    static bool configured = false;
    auto kern = tile_merge_kernel<K, KV, THREADS, E>;
    if (!configured) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Shape::kSmem)) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        configured = true;
    }
    const uint64_t P = 1ull << G;
    const uint64_t grid = P < uint64_t(num_sms()) ? P : uint64_t(num_sms());
    kern<<<unsigned(grid), THREADS, Shape::kSmem, stream>>>((K *)buf, vals, la, lb, split, G,
                                                            sb);
    return last_launch_status();
}

// Tile shapes: 4-byte keys 1024 x 33, 8-byte keys and key-value 512 x 33.
template <typename K, bool KV>
struct TileOf;
template <>
struct TileOf<int32_t, false> { static constexpr int T = 1024, E = 33; };
template <>
struct TileOf<uint32_t, false> { static constexpr int T = 1024, E = 33; };
template <>
struct TileOf<float, false> { static constexpr int T = 1024, E = 33; };
template <>
struct TileOf<uint64_t, false> { static constexpr int T = 512, E = 33; };
template <>
struct TileOf<int32_t, true> { static constexpr int T = 512, E = 33; };
template <>
struct TileOf<uint32_t, true> { static constexpr int T = 512, E = 33; };
template <>
struct TileOf<float, true> { static constexpr int T = 512, E = 33; };
template <>
struct TileOf<uint64_t, true> { static constexpr int T = 512, E = 33; };
template <>
struct TileOf<int64_t, false> { static constexpr int T = 512, E = 33; };
template <>
struct TileOf<int64_t, true> { static constexpr int T = 512, E = 33; };

template <typename K>
ipm_status tile_merge_dispatch(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                               const uint64_t *split, uint32_t G, StatusBlock *sb,
                               cudaStream_t stream) {
    if (vals)
        return tile_merge_t<K, true, TileOf<K, true>::T, TileOf<K, true>::E>(
            buf, vals, la, lb, split, G, sb, stream);
    return tile_merge_t<K, false, TileOf<K, false>::T, TileOf<K, false>::E>(
        buf, nullptr, la, lb, split, G, sb, stream);
}

}  // namespace

uint64_t tile_capacity(ipm_dtype key, bool with_values) {
    switch (key) {
    case IPM_INT32:
    case IPM_UINT32:
    case IPM_FLOAT32:
        return with_values ? uint64_t(TileOf<int32_t, true>::T) * TileOf<int32_t, true>::E
                           : uint64_t(TileOf<int32_t, false>::T) * TileOf<int32_t, false>::E;
    case IPM_UINT64:
    case IPM_INT64:
        return with_values ? uint64_t(TileOf<uint64_t, true>::T) * TileOf<uint64_t, true>::E
                           : uint64_t(TileOf<uint64_t, false>::T) * TileOf<uint64_t, false>::E;
    }
    return 0;
}

ipm_status launch_tile_merge(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                             ipm_dtype key, const uint64_t *split, uint32_t G,
                             StatusBlock *sb, cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        return tile_merge_dispatch<int32_t>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_UINT32:
        return tile_merge_dispatch<uint32_t>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_UINT64:
        return tile_merge_dispatch<uint64_t>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_INT64:
        return tile_merge_dispatch<int64_t>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_FLOAT32:
        return tile_merge_dispatch<float>(buf, vals, la, lb, split, G, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
