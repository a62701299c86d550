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

template <typename K, bool KV, int THREADS, int E, typename V>
__global__ void __launch_bounds__(THREADS, 1)
    tile_merge_kernel(K *__restrict__ buf, V *__restrict__ vals, uint64_t la,
                      uint64_t lb, const uint64_t *__restrict__ split, uint32_t G,
                      StatusBlock *sb) {
    using Shape = TileShape<K, KV, THREADS, E, V>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    __shared__ int abort_flag;
    K *skeys = reinterpret_cast<K *>(smem_raw + 128);
    V *svals = reinterpret_cast<V *>(smem_raw + 128 + Shape::kKeyBytes);
    if (call_finished(sb)) return;

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
        if (merge_pair_smem<K, KV, THREADS, E, V>(buf + d0, KV ? vals + d0 : nullptr, a, c, skeys,
                                               svals, mbar, parity, abort_flag,
                                               sb) == kPairAbort)
            break;
    }
    if (tid == 0) bulk_wait_all0();
}

template <typename K, bool KV, int THREADS, int E, typename V>
ipm_status tile_merge_t(void *buf, void *vals, uint64_t la, uint64_t lb,
                        const uint64_t *split, uint32_t G, StatusBlock *sb,
                        cudaStream_t stream) {
    using Shape = TileShape<K, KV, THREADS, E, V>;
    static std::atomic<bool> configured{false};  // a racing first call repeats the set-up
    auto kern = tile_merge_kernel<K, KV, THREADS, E, V>;
    if (!configured.load(std::memory_order_relaxed)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Shape::kSmem)) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        configured.store(true, std::memory_order_relaxed);
    }
    const uint64_t P = 1ull << G;
    const uint64_t grid = P < uint64_t(num_sms()) ? P : uint64_t(num_sms());
    kern<<<unsigned(grid), THREADS, Shape::kSmem, stream>>>((K *)buf, (V *)vals, la, lb, split,
                                                            G, sb);
    return last_launch_status();
}

// Tile shapes: 4-byte keys alone 1024 x 33; up to 12 bytes per element (8-byte keys,
// 4-byte keys with a payload, 8-byte keys with a 4-byte payload) 512 x 33; 16 bytes
// (8-byte keys with an 8-byte payload) 256 x 33.
template <typename K, bool KV, typename V>
struct TileOf {
    static constexpr int kElem = int(sizeof(K)) + (KV ? int(sizeof(V)) : 0);
    static constexpr int T = kElem == 4 ? 1024 : (kElem <= 12 ? 512 : 256), E = 33;
};

template <typename K, typename V>
ipm_status tile_merge_kv(void *buf, void *vals, uint64_t la, uint64_t lb,
                         const uint64_t *split, uint32_t G, StatusBlock *sb,
                         cudaStream_t stream) {
    return tile_merge_t<K, true, TileOf<K, true, V>::T, TileOf<K, true, V>::E, V>(
        buf, vals, la, lb, split, G, sb, stream);
}

template <typename K>
ipm_status tile_merge_dispatch(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                               const uint64_t *split, uint32_t G, StatusBlock *sb,
                               cudaStream_t stream) {
    if (vb == 8) return tile_merge_kv<K, uint64_t>(buf, vals, la, lb, split, G, sb, stream);
    if (vb != 0) return tile_merge_kv<K, uint32_t>(buf, vals, la, lb, split, G, sb, stream);
    return tile_merge_t<K, false, TileOf<K, false, uint32_t>::T, TileOf<K, false, uint32_t>::E,
                        uint32_t>(buf, nullptr, la, lb, split, G, sb, stream);
}

}  // namespace

template <typename K>
static uint64_t tile_of(uint32_t vb) {
    if (vb == 8) return uint64_t(TileOf<K, true, uint64_t>::T) * TileOf<K, true, uint64_t>::E;
    if (vb != 0) return uint64_t(TileOf<K, true, uint32_t>::T) * TileOf<K, true, uint32_t>::E;
    return uint64_t(TileOf<K, false, uint32_t>::T) * TileOf<K, false, uint32_t>::E;
}

uint64_t tile_capacity(ipm_dtype key, uint32_t vb) {
    const int kb = dtype_bytes(key);
    return kb == 4 ? tile_of<int32_t>(vb) : (kb == 8 ? tile_of<uint64_t>(vb) : 0);
}

ipm_status launch_tile_merge(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                             ipm_dtype key, const uint64_t *split, uint32_t G,
                             StatusBlock *sb, cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        return tile_merge_dispatch<int32_t>(buf, vals, vb, la, lb, split, G, sb, stream);
    case IPM_UINT32:
        return tile_merge_dispatch<uint32_t>(buf, vals, vb, la, lb, split, G, sb, stream);
    case IPM_UINT64:
        return tile_merge_dispatch<uint64_t>(buf, vals, vb, la, lb, split, G, sb, stream);
    case IPM_FLOAT32:
        return tile_merge_dispatch<float>(buf, vals, vb, la, lb, split, G, sb, stream);
    case IPM_INT64:
        return tile_merge_dispatch<int64_t>(buf, vals, vb, la, lb, split, G, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
