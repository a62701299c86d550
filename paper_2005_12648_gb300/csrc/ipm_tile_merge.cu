// Merge step: every pair (A_k, B_k) of the arranged buffer is merged stably in place by
// one CTA (the per-thread std::inplace_merge of Alg. 2/3, here per CTA).
//
// Pair k occupies [d_k, d_{k+1}) as A[i_k, i_{k+1}) | B[j_k, j_{k+1}).  The CTA
//   1. stages the pair in shared memory: the 16-byte-aligned body with one TMA bulk
//      copy (cp.async.bulk, completion on an mbarrier), the unaligned head and tail
//      (< 16 bytes each) with plain loads;
//   2. gives each thread E consecutive outputs: a binary search on its diagonal of
//      the pair's merge path (stable predicate A[m] <= B[d-1-m]), then E sequential
//      merge steps into registers;
//   3. writes the registers back over the staged pair (E odd keeps the blocked
//      writes conflict-free across banks) and stores the body with one TMA bulk store,
//      head and tail with plain stores.
// The kernel is persistent (one CTA per SM, grid-stride over pairs); a pair never
// straddles two CTAs, so the in-place write-back touches only the CTA's own range.
#include "ipm_internal.h"
#include "ipm_tma.cuh"

namespace ipm {

namespace {

template <typename K, bool KV, int THREADS, int E>
struct TileShape {
    static constexpr int kTile = THREADS * E;
    static constexpr int kKeyPad = 16 / int(sizeof(K));
    static constexpr size_t kKeyBytes = ((size_t(kTile + kKeyPad) * sizeof(K)) + 15) / 16 * 16;
    static constexpr size_t kValBytes = KV ? ((size_t(kTile + 4) * 4 + 15) / 16 * 16) : 0;
    static constexpr size_t kSmem = 128 + kKeyBytes + kValBytes;
};

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
        const uint32_t b = c - a;
        K *g = buf + d0;
        uint32_t *gv = KV ? vals + d0 : nullptr;
        const Geo<int(sizeof(K))> gk(g, c);
        const Geo<4> gvv(KV ? (const void *)gv : (const void *)g, KV ? c : 0u);
        K *tk = skeys + gk.off;          // staged keys: tk[0, c)
        uint32_t *tv = svals + gvv.off;  // staged values: tv[0, c)

        // ---- 1. stage
        if (tid == 0) {
            const uint32_t kb = gk.body * uint32_t(sizeof(K));
            const uint32_t vb = KV ? gvv.body * 4u : 0u;
            mbar_arrive_expect_tx(mbar, kb + vb);
            if (kb) bulk_load(tk + gk.head, g + gk.head, kb, mbar);
            if (KV && vb) bulk_load(tv + gvv.head, gv + gvv.head, vb, mbar);
        }
        for (uint32_t j = tid; j < gk.head; j += THREADS) tk[j] = g[j];
        for (uint32_t j = gk.tail_start + tid; j < c; j += THREADS) tk[j] = g[j];
        if (KV) {
            for (uint32_t j = tid; j < gvv.head; j += THREADS) tv[j] = gv[j];
            for (uint32_t j = gvv.tail_start + tid; j < c; j += THREADS) tv[j] = gv[j];
        }
        if (!mbar_wait_bounded(mbar, parity)) atomicOr(&abort_flag, 1);
        parity ^= 1u;
        __syncthreads();
        if (abort_flag) {
            if (tid == 0 && sb != nullptr) set_status(sb, IPM_ERR_TIMEOUT);
            break;
        }

        // ---- 2. merge path split of this thread's diagonal, then E merge steps
        const K *sA = tk;
        const K *sB = tk + a;
        const uint32_t dt = tid * uint32_t(E);
        K ok[E];
        uint32_t oi[KV ? E : 1];
        if (dt < c) {
            uint32_t lo = dt > b ? dt - b : 0u;
            uint32_t hi = dt < a ? dt : a;
            while (lo < hi) {
                const uint32_t m = (lo + hi) >> 1;
                if (key_le(sA[m], sB[dt - 1 - m]))
                    lo = m + 1;
                else
                    hi = m;
            }
            uint32_t ia = lo, ib = dt - lo;
            K va = ia < a ? sA[ia] : K(0);
            K vb = ib < b ? sB[ib] : K(0);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const bool takeA = (ib >= b) || (ia < a && key_le(va, vb));
                if (KV)
                    oi[KV ? e : 0] = takeA ? ia : a + ib;
                else
                    ok[e] = takeA ? va : vb;
                if (takeA) {
                    ++ia;
                    if (ia < a) va = sA[ia];
                } else {
                    ++ib;
                    if (ib < b) vb = sB[ib];
                }
            }
        }
        uint32_t ov[KV ? E : 1];
        if (KV && dt < c) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint32_t src = (dt + e < c) ? oi[KV ? e : 0] : 0u;
                ok[e] = tk[src];
                ov[KV ? e : 0] = tv[src];
            }
        }
        __syncthreads();

        // ---- 3. write back in place, then store
        if (dt < c) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (dt + e < c) {
                    tk[dt + e] = ok[e];
                    if (KV) tv[dt + e] = ov[KV ? e : 0];
                }
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const uint32_t kb = gk.body * uint32_t(sizeof(K));
            const uint32_t vb = KV ? gvv.body * 4u : 0u;
            if (kb) bulk_store(g + gk.head, tk + gk.head, kb);
            if (KV && vb) bulk_store(gv + gvv.head, tv + gvv.head, vb);
            bulk_commit();
        }
        for (uint32_t j = tid; j < gk.head; j += THREADS) g[j] = tk[j];
        for (uint32_t j = gk.tail_start + tid; j < c; j += THREADS) g[j] = tk[j];
        if (KV) {
            for (uint32_t j = tid; j < gvv.head; j += THREADS) gv[j] = tv[j];
            for (uint32_t j = gvv.tail_start + tid; j < c; j += THREADS) gv[j] = tv[j];
        }
        if (tid == 0) bulk_wait_read0();
        fence_proxy_async_smem();
        __syncthreads();
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
    case IPM_FLOAT32:
        return tile_merge_dispatch<float>(buf, vals, la, lb, split, G, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
