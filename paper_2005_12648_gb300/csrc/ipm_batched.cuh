// Batched segmented merge: every segment {offset, len_a, len_b} of a table is an
// independent in-place merge of two sorted runs (Sec. 1).  Each segment is handled by
// ONE CTA, so segments need no inter-CTA coordination; CTAs take segments from an
// atomic work queue.  Three launches, all capturable in one CUDA graph:
//   prep    (one CTA) resets the status block, writes the queue of descriptors --
//           largest segment first (4 buckets per octave) so the long segments start
//           early and the short ones fill the tail -- and lists the segments longer
//           than one merge tile;
//   levels  (persistent) for each listed segment: the early exit of Alg. 2/3, the exact
//           stable splits of its P = 2^G diagonals d_k = floor(k*n/P) (Sec. 3.1), its
//           sRecPar exchange levels (Alg. 3) executed by the CTA with the
//           linear-shifting phases of the plain path (x_phase: one-pass SINGLE / SWAP /
//           PAIR / SHIFT, LS steps when neither block fits the on-chip stash,
//           Sec. 3.4/3.5) chunk by chunk through shared memory; the split table goes to
//           the workspace;
//   merge   (persistent) for each segment in queue order: its pairs merged through
//           shared memory (merge_pair_smem); a segment that fits one tile is one pair
//           and takes its early-exit test on the staged copy.
// Keeping the exchange code out of the merge kernel keeps the merge loop free of
// register spills.
//
// The same work also runs as ONE persistent launch (batched_fused_kernel, the "one
// launch" form of the options): after a memset node clears the status block and the
// queue counters, CTAs take tickets in order -- the first tickets build the size
// histogram of the table chunk by chunk, the next ones scatter the descriptors into
// size order (each waits, bounded, for every histogram chunk), and every later ticket is
// one segment, done whole by its CTA (early exit, splits, exchange levels, pair merges).
// Every wait is on an earlier ticket, held by a running CTA, so none can deadlock.
#pragma once

#include "ipm_exchange.cuh"
#include "ipm_internal.h"
#include "ipm_split.cuh"
#include "ipm_tile_merge.cuh"

namespace ipm {
namespace batched {

// Status-block counters used by the batched launches.
constexpr uint32_t kMergeTicket = 0;   // merge kernel work queue
constexpr uint32_t kLevelsTicket = 1;  // levels kernel work queue
constexpr uint32_t kMultiCount = 2;    // segments longer than one tile (prep)
constexpr uint32_t kPoolTop = 3;       // split-pool entries allocated (levels)

constexpr uint32_t kMaxPairs = 512;    // pairs per segment (split table in shared memory)
constexpr uint32_t kInOrder = 0xffffffffu;  // soff: segment already in order
constexpr uint32_t kSkipped = 0xfffffffeu;  // soff: split pool exhausted, left untouched

// Segment classes.
enum : uint32_t { kSegInvalid = 0, kSegTrivial = 1, kSegSingle = 2, kSegMulti = 3 };

// invalid: leaves [0, buf_len) or is longer than max_seg; trivial: a run is empty;
// single: fits one merge tile; multi: needs splits and exchange levels.
__device__ __forceinline__ uint32_t seg_class(const ipm_segment &sg, uint64_t buf_len,
                                              uint64_t tile, uint64_t max_seg) {
    const bool inside = sg.len_a <= buf_len && sg.len_b <= buf_len - sg.len_a &&
                        sg.offset <= buf_len - sg.len_a - sg.len_b;
    if (!inside) return kSegInvalid;
    const uint64_t n = sg.len_a + sg.len_b;
    if (n > max_seg) return kSegInvalid;
    if (sg.len_a == 0 || sg.len_b == 0) return kSegTrivial;
    return n <= tile ? kSegSingle : kSegMulti;
}

// Least G with every pair of the n elements on P = 2^G diagonals fitting the tile.
__device__ __forceinline__ uint32_t seg_levels(uint64_t n, uint64_t tile) {
    uint32_t G = 0;
    while (((n + (1ull << G) - 1) >> G) > tile) ++G;
    return G;
}

// Workspace areas of a batched call (after the 256-byte status block).
struct QueueArea {
    ipm_segment *queue;  // [nseg] descriptors in processing order
    uint32_t *multi;     // [nseg] queue positions of the multi-tile segments
    uint32_t *soff;      // [nseg] per queue position: split-table offset in the pool
    uint64_t *pool;      // [cap] split tables
    uint64_t pool_cap;
    uint32_t *hist;      // [kOrderBuckets] one-launch form: segments per length bucket
    uint32_t *cursor;    // [kOrderBuckets] one-launch form: queue slots taken per bucket
};

constexpr uint32_t kOrderBuckets = 256;  // 4 per octave of the segment length

// Bucket of a segment of n >= 1 elements: 4 * floor(log2 n) + the next two bits.
__device__ __forceinline__ uint32_t size_bucket(uint64_t n) {
    const uint32_t lg = 63u - uint32_t(__clzll(n));
    const uint32_t frac = lg >= 2 ? uint32_t(n >> (lg - 2)) & 3u : uint32_t(n << (2 - lg)) & 3u;
    return (lg << 2) | frac;
}

// Asynchronous global -> shared copies (cp.async), for the queue entry of the next
// segment while the current one is processed.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---------------------------------------------------------------------------------
// CTA-wide copies between global memory and shared memory.  A staged range keeps the
// 16-byte phase of its global source: element j lives at region[phase + j].  Global
// loads bypass L1 (ld.global.cg): the data is rewritten by this CTA between levels.
// ---------------------------------------------------------------------------------
template <typename T, int THREADS>
__device__ __forceinline__ uint32_t stage_in(T *region, const T *src, uint32_t len) {
    constexpr uint32_t W = sizeof(T);
    const uint32_t tid = threadIdx.x;
    const uint32_t mis = uint32_t(reinterpret_cast<uintptr_t>(src) & 15u);
    const uint32_t phase = mis / W;
    uint32_t head = ((16u - mis) & 15u) / W;
    head = head < len ? head : len;
    const uint32_t nv = (len - head) * W / 16u;
    const uint32_t tail = head + nv * (16u / W);
    T *dst = region + phase;
    if (tid < head) dst[tid] = __ldcg(src + tid);
    if (tid >= head && tid < head + (len - tail)) dst[tail + (tid - head)] = __ldcg(src + tail + (tid - head));
    const uint4 *vs = reinterpret_cast<const uint4 *>(src + head);
    uint4 *vd = reinterpret_cast<uint4 *>(dst + head);
    uint32_t v = tid;
    for (; v + 3u * THREADS < nv; v += 4u * THREADS) {
        const uint4 x0 = __ldcg(vs + v);
        const uint4 x1 = __ldcg(vs + v + THREADS);
        const uint4 x2 = __ldcg(vs + v + 2u * THREADS);
        const uint4 x3 = __ldcg(vs + v + 3u * THREADS);
        vd[v] = x0;
        vd[v + THREADS] = x1;
        vd[v + 2u * THREADS] = x2;
        vd[v + 3u * THREADS] = x3;
    }
    for (; v < nv; v += THREADS) vd[v] = __ldcg(vs + v);
    return phase;
}

// Four consecutive 32-bit words of shared memory starting `ow` words (0..3) into the
// 16-byte-aligned vector q: two aligned vector reads and a word shift.
__device__ __forceinline__ uint4 lds_words(const uint4 *q, uint32_t ow) {
    const uint4 x = q[0];
    if (ow == 0) return x;
    const uint4 y = q[1];
    if (ow == 1) return make_uint4(x.y, x.z, x.w, y.x);
    if (ow == 2) return make_uint4(x.z, x.w, y.x, y.y);
    return make_uint4(x.w, y.x, y.y, y.z);
}

// dst[j] = s[j] for j < len; s is a shared-memory pointer at element granularity.
template <typename T, int THREADS>
__device__ __forceinline__ void stage_out(T *dst, const T *s, uint32_t len) {
    constexpr uint32_t W = sizeof(T);
    const uint32_t tid = threadIdx.x;
    const uint32_t mis = uint32_t(reinterpret_cast<uintptr_t>(dst) & 15u);
    uint32_t head = ((16u - mis) & 15u) / W;
    head = head < len ? head : len;
    const uint32_t nv = (len - head) * W / 16u;
    const uint32_t tail = head + nv * (16u / W);
    if (tid < head) dst[tid] = s[tid];
    if (tid >= head && tid < head + (len - tail)) dst[tail + (tid - head)] = s[tail + (tid - head)];
    // source words of the body: s + head, as 16-byte vector index + word offset
    const uint32_t saddr = uint32_t(reinterpret_cast<uintptr_t>(s + head));
    const uint32_t ow = (saddr & 15u) >> 2;
    const uint4 *q0 = reinterpret_cast<const uint4 *>(s + head) - 0;
    const uint4 *qa = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(q0) -
                                                      (saddr & 15u));
    uint4 *vd = reinterpret_cast<uint4 *>(dst + head);
    uint32_t v = tid;
    for (; v + 3u * THREADS < nv; v += 4u * THREADS) {
        const uint4 x0 = lds_words(qa + v, ow);
        const uint4 x1 = lds_words(qa + v + THREADS, ow);
        const uint4 x2 = lds_words(qa + v + 2u * THREADS, ow);
        const uint4 x3 = lds_words(qa + v + 3u * THREADS, ow);
        __stcg(vd + v, x0);
        __stcg(vd + v + THREADS, x1);
        __stcg(vd + v + 2u * THREADS, x2);
        __stcg(vd + v + 3u * THREADS, x3);
    }
    for (; v < nv; v += THREADS) __stcg(vd + v, lds_words(qa + v, ow));
}

// ---------------------------------------------------------------------------------
// Levels kernel: the exchange arena of one CTA, split into four regions.
// ---------------------------------------------------------------------------------
template <typename K, bool KV>
struct Arena {
    static constexpr uint32_t kElem = uint32_t(sizeof(K)) + (KV ? 4u : 0u);
    static constexpr uint32_t kSize = (65536u / kElem) / 16u * 16u;  // ~64 KiB per CTA
    static constexpr uint32_t kQ = kSize / 4u;                       // region, elements
    static constexpr uint32_t kPad = 4;                              // >= 16 B / element
    static constexpr uint32_t kQuarterCap = kQ - kPad;               // one region
    static constexpr uint32_t kHalfCap = 2u * kQ - kPad;             // two adjacent regions
    static constexpr uint32_t kSingleCap = kSize - kPad;             // the whole arena
    static constexpr size_t kKeyBytes = size_t(kSize + kPad) * sizeof(K);
    static constexpr size_t kValBytes = KV ? size_t(kSize + kPad) * 4u : 0u;
    static constexpr size_t kSmem = kKeyBytes + kValBytes;
    __host__ __device__ static XParams params() {
        // stash of one CTA = two regions; PAIR chunks use one region per block
        return XParams{kQuarterCap, kHalfCap, kHalfCap, 1u, kSingleCap};
    }
};

template <typename K, bool KV, int THREADS>
struct SegmentCtx {
    using S = Arena<K, KV>;
    K *g;           // segment base (keys)
    uint32_t *gv;   // segment base (payload)
    K *ak;          // key arena
    uint32_t *av;   // payload arena

    // stage [p, p+len) of the segment into region r; returns the key/payload phases
    __device__ __forceinline__ void load(uint32_t r, uint64_t p, uint32_t len, uint32_t &pk,
                                         uint32_t &pv) const {
        pk = stage_in<K, THREADS>(ak + r * S::kQ, g + p, len);
        if (KV) pv = stage_in<uint32_t, THREADS>(av + r * S::kQ, gv + p, len);
    }
    // write `len` staged elements of region r starting at staged index j0 to [q, q+len)
    __device__ __forceinline__ void store(uint64_t q, uint32_t r, uint32_t pk, uint32_t pv,
                                          uint32_t j0, uint32_t len) const {
        stage_out<K, THREADS>(g + q, ak + r * S::kQ + pk + j0, len);
        if (KV) stage_out<uint32_t, THREADS>(gv + q, av + r * S::kQ + pv + j0, len);
    }
};

// Physical start of the primed range [x0, x0+len) of exchange (s, m): mirrored
// coordinates map p -> m-1-p, which keeps a contiguous range contiguous.
__device__ __forceinline__ uint64_t primed(uint64_t s, uint64_t m, uint32_t mirror, uint64_t x0,
                                           uint64_t len) {
    return mirror ? s + m - x0 - len : s + x0;
}

// Exchange [X (a) | Y (b)] at segment offset s into [Y | X], CTA-wide.
template <typename K, bool KV, int THREADS>
__device__ __forceinline__ void cta_exchange(const SegmentCtx<K, KV, THREADS> &cx, uint64_t s,
                                             uint64_t a, uint64_t b) {
    using S = Arena<K, KV>;
    const XParams prm = S::params();
    XPhase ph;
    uint32_t pk0 = 0, pv0 = 0, pk1 = 0, pv1 = 0;
    while (x_phase(prm, s, a, b, ph)) {
        const uint64_t m = ph.a + ph.b;
        const uint64_t mn = ph.a < ph.b ? ph.a : ph.b;
        if (ph.kind == XK_SINGLE) {
            // the whole exchange on chip, written rotated
            cx.load(0, ph.s, uint32_t(m), pk0, pv0);
            __syncthreads();
            cx.store(ph.s, 0, pk0, pv0, uint32_t(ph.a), uint32_t(ph.b));
            cx.store(ph.s + ph.b, 0, pk0, pv0, 0u, uint32_t(ph.a));
            __syncthreads();
        } else if (ph.kind == XK_SWAP) {
            // [s, s+mn) <-> [s+m-mn, s+m): the final swap when a == b, else one LS step
            const uint64_t q = ph.s + m - mn;
            for (uint64_t c0 = 0; c0 < mn; c0 += S::kHalfCap) {
                const uint32_t L = uint32_t(mn - c0 < S::kHalfCap ? mn - c0 : S::kHalfCap);
                cx.load(0, ph.s + c0, L, pk0, pv0);
                cx.load(2, q + c0, L, pk1, pv1);
                __syncthreads();
                cx.store(ph.s + c0, 2, pk1, pv1, 0u, L);
                cx.store(q + c0, 0, pk0, pv0, 0u, L);
                __syncthreads();
            }
        } else if (ph.kind == XK_SHIFT) {
            // primed [S (mn) | big (mx)] -> [big | S]: stash S, move big down by mn in
            // ascending primed chunks (each chunk overwrites only elements already read)
            const uint64_t mx = m - mn;
            const uint32_t mir = ph.mirror;
            cx.load(0, primed(ph.s, m, mir, 0, mn), uint32_t(mn), pk0, pv0);
            for (uint64_t t0 = 0; t0 < mx; t0 += S::kHalfCap) {
                const uint32_t L = uint32_t(mx - t0 < S::kHalfCap ? mx - t0 : S::kHalfCap);
                cx.load(2, primed(ph.s, m, mir, mn + t0, L), L, pk1, pv1);
                __syncthreads();
                cx.store(primed(ph.s, m, mir, t0, L), 2, pk1, pv1, 0u, L);
                __syncthreads();
            }
            cx.store(primed(ph.s, m, mir, mx, mn), 0, pk0, pv0, 0u, uint32_t(mn));
            __syncthreads();
        } else {  // XK_PAIR
            // primed [X' (mn+e) | Y' (mn)] -> [Y' | X']: stash X'[mn, mn+e); chunk t
            // moves Y'[t] -> t and X'[t] -> mn+t; the stash lands at [2mn, 2mn+e)
            const uint64_t e = ph.delta;
            const uint32_t mir = ph.mirror;
            cx.load(0, primed(ph.s, m, mir, mn, e), uint32_t(e), pk0, pv0);
            uint32_t pk2 = 0, pv2 = 0;
            for (uint64_t t0 = 0; t0 < mn; t0 += S::kQuarterCap) {
                const uint32_t L =
                    uint32_t(mn - t0 < S::kQuarterCap ? mn - t0 : S::kQuarterCap);
                cx.load(2, primed(ph.s, m, mir, t0, L), L, pk1, pv1);
                cx.load(3, primed(ph.s, m, mir, mn + e + t0, L), L, pk2, pv2);
                __syncthreads();
                cx.store(primed(ph.s, m, mir, t0, L), 3, pk2, pv2, 0u, L);
                cx.store(primed(ph.s, m, mir, mn + t0, L), 2, pk1, pv1, 0u, L);
                __syncthreads();
            }
            cx.store(primed(ph.s, m, mir, 2 * mn, e), 0, pk0, pv0, 0u, uint32_t(e));
            __syncthreads();
        }
        if (ph.final_phase) break;
        x_after_step(ph, s, a, b);
    }
}

constexpr int kLevelsThreads = 256;

// For every multi-tile segment: a0, a1 (splits), a2 (exchange levels); the split table
// is written to the pool and its offset to soff.
template <typename K, bool KV>
__global__ void __launch_bounds__(kLevelsThreads)
    batched_levels_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, QueueArea qa,
                          uint64_t tile, StatusBlock *sb) {
    using S = Arena<K, KV>;
    constexpr int THREADS = kLevelsThreads;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t ssplit[kMaxPairs + 1];
    __shared__ uint32_t s_t, s_off;
    constexpr uint32_t kElem = S::kElem;
    const uint32_t tid = threadIdx.x;
    SegmentCtx<K, KV, THREADS> cx;
    cx.ak = reinterpret_cast<K *>(smem_raw);
    cx.av = reinterpret_cast<uint32_t *>(smem_raw + S::kKeyBytes);
    const uint32_t count = *((volatile const uint32_t *)&sb->counters[kMultiCount]);

    for (;;) {
        if (tid == 0) s_t = atomicAdd(&sb->counters[kLevelsTicket], 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= count) break;
        const uint32_t q = qa.multi[t];
        const ipm_segment sg = qa.queue[q];
        const uint64_t la = sg.len_a, n = sg.len_a + sg.len_b;
        cx.g = buf + sg.offset;
        cx.gv = KV ? vals + sg.offset : nullptr;
        // a0: already in order -> nothing moves, every pair is trivial or in order
        if (key_le(cx.g[la - 1], cx.g[la])) {
            if (tid == 0) qa.soff[q] = kInOrder;
            __syncthreads();  // s_t is rewritten on the next round
            continue;
        }
        const uint32_t G = seg_levels(n, tile);
        const uint32_t P = 1u << G;
        if (tid == 0) {
            const uint32_t off = atomicAdd(&sb->counters[kPoolTop], P + 1u);
            const bool fits = uint64_t(off) + P + 1u <= qa.pool_cap;
            if (!fits) set_status(sb, IPM_ERR_INVALID_ARG);  // overlapping segments
            s_off = fits ? off : kSkipped;
        }
        // a1: splits of the P = 2^G diagonals
        for (uint32_t k = tid >> 5; k <= P; k += THREADS / 32) {
            const uint64_t d = (uint64_t(k) * n) >> G;
            const uint64_t i = warp_split<false>(cx.g, la, cx.g + la, n - la, d);
            if ((tid & 31u) == 0) ssplit[k] = i;
        }
        __syncthreads();
        const uint32_t off = s_off;
        if (off == kSkipped) {
            if (tid == 0) qa.soff[q] = kSkipped;
            continue;
        }
        // a2: the sRecPar levels
        uint64_t xbytes = 0;
        for (uint32_t l = 0; l < G; ++l) {
            for (uint32_t r = 0; r < (1u << l); ++r) {
                const uint32_t k_lo = r << (G - l);
                const uint32_t k_mid = k_lo + (1u << (G - l - 1));
                const uint32_t k_hi = k_lo + (1u << (G - l));
                const uint64_t d_lo = (uint64_t(k_lo) * n) >> G;
                const uint64_t d_mid = (uint64_t(k_mid) * n) >> G;
                const uint64_t i_lo = ssplit[k_lo], i_mid = ssplit[k_mid], i_hi = ssplit[k_hi];
                const uint64_t s = d_lo + (i_mid - i_lo);
                const uint64_t a = i_hi - i_mid;
                const uint64_t b = (d_mid - i_mid) - (d_lo - i_lo);
                if (tid == 0) {
                    uint64_t it = 0, by = 0;
                    x_count(S::params(), s, a, b, kElem, it, by);
                    xbytes += by;
                }
                cta_exchange<K, KV, THREADS>(cx, s, a, b);
            }
        }
        for (uint32_t k = tid; k <= P; k += THREADS) qa.pool[off + k] = ssplit[k];
        if (tid == 0) {
            qa.soff[q] = off;
            if (xbytes) atomicAdd(&sb->exchange_bytes, xbytes);
        }
        __syncthreads();  // ssplit and s_t are rewritten on the next round
    }
}

// ---------------------------------------------------------------------------------
// Merge kernel: the pairs of every segment, one CTA per segment.
// ---------------------------------------------------------------------------------

// Per-segment state, kept in shared memory so that the inlined pair merge does not
// have to hold it in registers.
template <typename K>
struct SegState {
    K *g;
    uint32_t *gv;
    uint64_t n;
    uint32_t G;     // pairs P = 2^G
    uint32_t mode;  // 0 = nothing to do, 1 = merge the pairs, 2 = stop
};

template <typename K, bool KV, int THREADS, int E, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    batched_merge_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, uint64_t buf_len,
                         QueueArea qa, uint32_t nseg, uint64_t max_seg, StatusBlock *sb) {
    using Tile = TileShape<K, KV, THREADS, E>;
    constexpr uint64_t kTile = uint64_t(Tile::kTile);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    K *skeys = reinterpret_cast<K *>(smem_raw + 128);
    uint32_t *svals = reinterpret_cast<uint32_t *>(smem_raw + 128 + Tile::kKeyBytes);
    __shared__ uint64_t ssplit[kMaxPairs + 1];
    __shared__ SegState<K> st;
    __shared__ __align__(16) ipm_segment s_desc[2];  // current / next queue entry
    __shared__ uint32_t s_soff[2];
    __shared__ uint32_t s_valid[2];
    __shared__ int abort_flag;
    constexpr uint32_t kElem = uint32_t(sizeof(K)) + (KV ? 4u : 0u);
    volatile SegState<K> &vst = st;

    const uint32_t tid = threadIdx.x;
    // Thread 0 runs the queue one segment ahead: while segment i is processed, the
    // queue entry of segment i+1 is in flight (cp.async) and the ticket of segment i+2
    // is claimed, so no queue latency sits between two segments.
    uint32_t ahead = 0;  // thread 0: ticket of the segment after the next one
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        abort_flag = 0;
        const uint32_t t0 = atomicAdd(&sb->counters[kMergeTicket], 1u);
        s_valid[0] = t0 < nseg ? 1u : 0u;
        if (t0 < nseg) {
            s_desc[0] = qa.queue[t0];
            s_soff[0] = qa.soff[t0];
        }
        ahead = t0 < nseg ? atomicAdd(&sb->counters[kMergeTicket], 1u) : nseg;
    }
    uint32_t parity = 0;
    uint32_t cur = 0;

    for (;; cur ^= 1u) {
        if (tid == 0) cp_async_wait_all();
        __syncthreads();  // previous segment finished; queue entry `cur` has landed
        if (tid == 0) {
            uint32_t mode = 0;
            if (!s_valid[cur] || abort_flag) {
                mode = 2;
            } else {
                const ipm_segment sg = s_desc[cur];
                const uint32_t soff = s_soff[cur];
                // prefetch the next queue entry, claim the one after it
                const uint32_t nx = cur ^ 1u;
                s_valid[nx] = ahead < nseg ? 1u : 0u;
                if (ahead < nseg) {
                    const char *src = reinterpret_cast<const char *>(qa.queue + ahead);
                    char *dst = reinterpret_cast<char *>(&s_desc[nx]);
                    cp_async8(dst, src);
                    cp_async8(dst + 8, src + 8);
                    cp_async8(dst + 16, src + 16);
                    cp_async4(&s_soff[nx], qa.soff + ahead);
                    cp_async_commit();
                    ahead = atomicAdd(&sb->counters[kMergeTicket], 1u);
                }
                const uint32_t cls = seg_class(sg, buf_len, kTile, max_seg);
                bool multi_ok = cls == kSegMulti && soff != kInOrder && soff != kSkipped;
                if (multi_ok) {  // the split table must lie inside the pool
                    const uint32_t P = 1u << seg_levels(sg.len_a + sg.len_b, kTile);
                    if (uint64_t(soff) + P + 1u > qa.pool_cap) {
                        set_status(sb, IPM_ERR_DEVICE);
                        multi_ok = false;
                    }
                }
                if (cls == kSegSingle || multi_ok) {
                    const uint64_t n = sg.len_a + sg.len_b;
                    st.g = buf + sg.offset;
                    st.gv = KV ? vals + sg.offset : nullptr;
                    st.n = n;
                    st.G = cls == kSegSingle ? 0u : seg_levels(n, kTile);
                    ssplit[0] = 0;
                    ssplit[1] = sg.len_a;  // the one pair when G = 0
                    st.mode = cls == kSegSingle ? 1u : 3u;  // 3: splits from the pool
                    mode = 1;
                }
            }
            if (mode != 1) st.mode = mode;
        }
        __syncthreads();
        uint32_t mode = vst.mode;
        if (mode == 2) break;
        if (mode == 0) continue;
        if (mode == 3) {  // split table of a multi-tile segment, written by the levels kernel
            const uint32_t P = 1u << vst.G;
            const uint64_t *src = qa.pool + s_soff[cur];
            for (uint32_t k = tid; k <= P; k += THREADS) ssplit[k] = src[k];
            __syncthreads();
        }

        // a3: the pairs (one pair when G = 0)
        uint64_t moved = 0;  // thread 0: algorithmic bytes of the pair merges
        for (uint32_t k = 0; k < (1u << vst.G); ++k) {
            const uint64_t n = vst.n;
            const uint32_t Gk = vst.G;
            const uint64_t d0 = (uint64_t(k) * n) >> Gk, d1 = (uint64_t(k + 1) * n) >> Gk;
            const uint32_t c = uint32_t(d1 - d0);
            if (c == 0) continue;
            if (ssplit[k + 1] < ssplit[k] || ssplit[k + 1] - ssplit[k] > c) {  // inconsistent
                if (tid == 0) set_status(sb, IPM_ERR_DEVICE);
                continue;
            }
            const uint32_t a = uint32_t(ssplit[k + 1] - ssplit[k]);
            K *g = vst.g + d0;
            uint32_t *gv = KV ? vst.gv + d0 : nullptr;
            const int r = merge_pair_smem<K, KV, THREADS, E>(g, gv, a, c, skeys, svals, mbar,
                                                             parity, abort_flag, sb);
            if (r == kPairAbort) break;  // abort_flag is set: the next claim stops the CTA
            moved += r == kPairMerged ? 2ull * c * kElem : r == kPairInOrder ? 1ull * c * kElem : 0;
        }
        if (tid == 0 && moved) atomicAdd(&sb->merge_bytes, moved);
    }
    if (tid == 0) {
        cp_async_wait_all();
        bulk_wait_all0();
    }
}

// ---------------------------------------------------------------------------------
// One-launch form: the queue preparation, the levels and the pair merges in one
// persistent kernel (see the top of this file).
// ---------------------------------------------------------------------------------
constexpr uint32_t kFusedTicket = 4;    // status-block counters of the one-launch form
constexpr uint32_t kHistDone = 5;       // histogram tickets finished
constexpr uint32_t kScatterDone = 6;    // scatter tickets finished
constexpr uint32_t kFusedChunk = 4096;  // descriptors per preparation ticket
constexpr uint32_t kNoTicket = 0xffffffffu;

__device__ __forceinline__ uint32_t ld_acquire_gpu_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *ctr >= target; false after the call's wait limit.
__device__ __forceinline__ bool wait_at_least(const uint32_t *ctr, uint32_t target,
                                              unsigned long long lim) {
    DepTimer tm(lim);
    while (ld_acquire_gpu_u32(ctr) < target)
        if (tm.expired()) return false;
    return true;
}

template <typename K, bool KV, int THREADS, int E>
constexpr size_t fused_smem() {
    constexpr size_t merge = TileShape<K, KV, THREADS, E>::kSmem;
    constexpr size_t levels = 128 + Arena<K, KV>::kSmem;
    return merge > levels ? merge : levels;
}

template <typename K, bool KV, int THREADS, int E, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    batched_fused_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, uint64_t buf_len,
                         const ipm_segment *__restrict__ segs, uint32_t nseg, uint32_t by_size,
                         QueueArea qa, uint64_t max_seg, StatusBlock *sb) {
    using Tile = TileShape<K, KV, THREADS, E>;
    using S = Arena<K, KV>;
    constexpr uint64_t kTile = uint64_t(Tile::kTile);
    constexpr uint32_t kElem = uint32_t(sizeof(K)) + (KV ? 4u : 0u);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    // the pair merges stage through [128, 128 + tile); the exchange levels use the same
    // bytes as their arena (never at the same time)
    K *skeys = reinterpret_cast<K *>(smem_raw + 128);
    uint32_t *svals = reinterpret_cast<uint32_t *>(smem_raw + 128 + Tile::kKeyBytes);
    __shared__ uint64_t ssplit[kMaxPairs + 1];
    __shared__ uint32_t s_cnt[kOrderBuckets], s_base[kOrderBuckets];
    __shared__ uint32_t s_t;
    __shared__ int abort_flag, s_ready;
    __shared__ ipm_segment s_sg;
    const uint32_t tid = threadIdx.x;
    const unsigned long long lim = wait_limit(sb);
    const uint32_t C = by_size ? (nseg + kFusedChunk - 1) / kFusedChunk : 0u;
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        abort_flag = 0;
        s_ready = by_size ? 0 : 1;
    }
    uint32_t parity = 0;
    uint64_t moved = 0, xbytes = 0;  // thread 0: algorithmic bytes of merges / exchanges

    for (;;) {
        __syncthreads();  // the previous ticket's shared state is no longer read
        if (tid == 0)
            s_t = abort_flag ? kNoTicket : atomicAdd(&sb->counters[kFusedTicket], 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t == kNoTicket) break;
        if (t < 2 * C) {
            // ---- preparation: histogram tickets (t < C), then scatter tickets
            const uint32_t chunk = t < C ? t : t - C;
            const uint32_t i0 = chunk * kFusedChunk;
            const uint32_t i1 = nseg - i0 < kFusedChunk ? nseg : i0 + kFusedChunk;
            for (uint32_t q = tid; q < kOrderBuckets; q += THREADS) s_cnt[q] = 0u;
            if (t >= C && tid == 0 && !wait_at_least(&sb->counters[kHistDone], C, lim)) {
                set_status(sb, IPM_ERR_TIMEOUT);
                abort_flag = 1;
            }
            __syncthreads();
            if (abort_flag) continue;
            for (uint32_t i = i0 + tid; i < i1; i += THREADS) {
                const uint64_t n = segs[i].len_a + segs[i].len_b;
                atomicAdd(&s_cnt[n ? size_bucket(n) : 0u], 1u);
            }
            __syncthreads();
            if (t < C) {
                for (uint32_t q = tid; q < kOrderBuckets; q += THREADS)
                    if (s_cnt[q]) atomicAdd(&qa.hist[q], s_cnt[q]);
                __threadfence();
                __syncthreads();
                if (tid == 0) atomicAdd(&sb->counters[kHistDone], 1u);
                continue;
            }
            // bucket starts: exclusive scan of the totals from the largest bucket down
            if (tid < 32) {
                uint32_t carry = 0;
                for (int base = int(kOrderBuckets) - 32; base >= 0; base -= 32) {
                    const uint32_t q = uint32_t(base) + 31u - tid;  // descending in the chunk
                    const uint32_t v = __ldcg(&qa.hist[q]);
                    uint32_t x = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                        if (int(tid) >= o) x += y;
                    }
                    s_base[q] = carry + x - v;
                    carry += __shfl_sync(0xffffffffu, x, 31);
                }
            }
            __syncthreads();
            // this chunk's slots in every bucket
            for (uint32_t q = tid; q < kOrderBuckets; q += THREADS)
                if (s_cnt[q]) s_base[q] += atomicAdd(&qa.cursor[q], s_cnt[q]);
            __syncthreads();
            for (uint32_t i = i0 + tid; i < i1; i += THREADS) {
                const ipm_segment sg = segs[i];
                const uint64_t n = sg.len_a + sg.len_b;
                qa.queue[atomicAdd(&s_base[n ? size_bucket(n) : 0u], 1u)] = sg;
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(&sb->counters[kScatterDone], 1u);
            continue;
        }

        // ---- one segment, in queue order
        const uint32_t q = t - 2 * C;
        if (q >= nseg) break;
        if (tid == 0) {
            if (!s_ready) {
                if (wait_at_least(&sb->counters[kScatterDone], C, lim)) {
                    s_ready = 1;
                } else {
                    set_status(sb, IPM_ERR_TIMEOUT);
                    abort_flag = 1;
                }
            }
            if (!abort_flag) {
                ipm_segment sg;
                if (by_size) {  // written by other CTAs of this launch: read through L2
                    sg.offset = __ldcg(reinterpret_cast<const unsigned long long *>(&qa.queue[q].offset));
                    sg.len_a = __ldcg(reinterpret_cast<const unsigned long long *>(&qa.queue[q].len_a));
                    sg.len_b = __ldcg(reinterpret_cast<const unsigned long long *>(&qa.queue[q].len_b));
                } else {
                    sg = segs[q];
                }
                s_sg = sg;
            }
        }
        __syncthreads();
        if (abort_flag) continue;
        const ipm_segment sg = s_sg;
        const uint32_t cls = seg_class(sg, buf_len, kTile, max_seg);
        if (cls == kSegInvalid) {
            if (tid == 0) set_status(sb, IPM_ERR_INVALID_ARG);  // left untouched
            continue;
        }
        if (cls == kSegTrivial) continue;
        K *g = buf + sg.offset;
        uint32_t *gv = KV ? vals + sg.offset : nullptr;
        const uint64_t la = sg.len_a, n = sg.len_a + sg.len_b;
        if (cls == kSegSingle) {
            const int r = merge_pair_smem<K, KV, THREADS, E>(g, gv, uint32_t(la), uint32_t(n),
                                                             skeys, svals, mbar, parity,
                                                             abort_flag, sb);
            if (tid == 0)
                moved += r == kPairMerged ? 2ull * n * kElem : r == kPairInOrder ? n * kElem : 0;
            continue;
        }
        // a multi-tile segment: a0 (already in order: nothing moves), a1, a2, a3
        if (key_le(g[la - 1], g[la])) continue;
        const uint32_t G = seg_levels(n, kTile);
        const uint32_t P = 1u << G;
        SegmentCtx<K, KV, THREADS> cx;
        cx.ak = reinterpret_cast<K *>(smem_raw + 128);
        cx.av = reinterpret_cast<uint32_t *>(smem_raw + 128 + S::kKeyBytes);
        cx.g = g;
        cx.gv = gv;
        for (uint32_t k = tid >> 5; k <= P; k += THREADS / 32) {
            const uint64_t d = (uint64_t(k) * n) >> G;
            const uint64_t i = warp_split<false>(g, la, g + la, n - la, d);
            if ((tid & 31u) == 0) ssplit[k] = i;
        }
        __syncthreads();
        for (uint32_t l = 0; l < G; ++l) {
            for (uint32_t r = 0; r < (1u << l); ++r) {
                const uint32_t k_lo = r << (G - l);
                const uint32_t k_mid = k_lo + (1u << (G - l - 1));
                const uint32_t k_hi = k_lo + (1u << (G - l));
                const uint64_t d_lo = (uint64_t(k_lo) * n) >> G;
                const uint64_t d_mid = (uint64_t(k_mid) * n) >> G;
                const uint64_t i_lo = ssplit[k_lo], i_mid = ssplit[k_mid], i_hi = ssplit[k_hi];
                const uint64_t xs = d_lo + (i_mid - i_lo);
                const uint64_t xa = i_hi - i_mid;
                const uint64_t xb = (d_mid - i_mid) - (d_lo - i_lo);
                if (tid == 0) {
                    uint64_t it = 0, by = 0;
                    x_count(S::params(), xs, xa, xb, kElem, it, by);
                    xbytes += by;
                }
                cta_exchange<K, KV, THREADS>(cx, xs, xa, xb);
            }
        }
        // the exchanges' global writes precede the bulk copies that read them back, and
        // their shared-memory accesses precede the bulk copies into the same bytes
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        fence_proxy_async_smem();
        __syncthreads();
        for (uint32_t k = 0; k < P; ++k) {
            const uint64_t d0 = (uint64_t(k) * n) >> G, d1 = (uint64_t(k + 1) * n) >> G;
            const uint32_t c = uint32_t(d1 - d0);
            if (c == 0) continue;
            if (ssplit[k + 1] < ssplit[k] || ssplit[k + 1] - ssplit[k] > c) {  // inconsistent
                if (tid == 0) set_status(sb, IPM_ERR_DEVICE);
                continue;
            }
            const uint32_t a = uint32_t(ssplit[k + 1] - ssplit[k]);
            const int r = merge_pair_smem<K, KV, THREADS, E>(g + d0, KV ? gv + d0 : nullptr, a, c,
                                                             skeys, svals, mbar, parity,
                                                             abort_flag, sb);
            if (r == kPairAbort) break;  // abort_flag is set: the next claim stops the CTA
            if (tid == 0)
                moved += r == kPairMerged ? 2ull * c * kElem : r == kPairInOrder ? 1ull * c * kElem : 0;
        }
    }
    if (tid == 0) {
        if (moved) atomicAdd(&sb->merge_bytes, moved);
        if (xbytes) atomicAdd(&sb->exchange_bytes, xbytes);
        bulk_wait_all0();
    }
}

// Merge tile variants: 0 wide = the plain path's tile (one CTA per SM), 1 narrow = half
// of it (two CTAs per SM), 2 quarter = a quarter (four CTAs per SM): the smaller the
// tile, the more CTAs overlap one another's staging latency, and the more exchange
// levels a long segment needs.
template <typename K, bool KV, int VARIANT>
struct BatchTile;
template <typename K, bool KV>
struct BatchTile<K, KV, 0> {
    static constexpr bool kSmall = sizeof(K) == 4 && !KV;
    static constexpr int T = kSmall ? 1024 : 512, E = 33, MINB = 1;
};
template <typename K, bool KV>
struct BatchTile<K, KV, 1> {
    static constexpr bool kSmall = sizeof(K) == 4 && !KV;
    static constexpr int T = kSmall ? 512 : 256, E = 33, MINB = 2;
};
template <typename K, bool KV>
struct BatchTile<K, KV, 2> {
    static constexpr bool kSmall = sizeof(K) == 4 && !KV;
    static constexpr int T = kSmall ? 256 : 128, E = 33, MINB = 4;
};

template <typename K, bool KV, int VARIANT>
constexpr uint64_t tile_of() {
    return uint64_t(BatchTile<K, KV, VARIANT>::T) * BatchTile<K, KV, VARIANT>::E;
}

// Resident CTAs per SM of a kernel, queried once per (kernel, device).
template <typename F>
ipm_status occupancy_of(F kern, int threads, size_t smem, std::atomic<int> &cache,
                        int &occ) {
    occ = cache.load(std::memory_order_relaxed);  // set once; a racing first call repeats it
    if (occ == 0) {
        IPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(smem)));
        IPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        if (occ < 1) return IPM_ERR_CUDA;
        cache.store(occ, std::memory_order_relaxed);
    }
    return IPM_OK;
}

template <typename K, bool KV, int VARIANT>
ipm_status batched_launch_t(void *buf, uint32_t *vals, uint64_t buf_len, QueueArea qa,
                            uint32_t nseg, uint32_t ctas_per_sm, uint32_t one_launch,
                            const ipm_segment *segs, uint32_t by_size, StatusBlock *sb,
                            cudaStream_t stream) {
    using BT = BatchTile<K, KV, VARIANT>;
    using Tile = TileShape<K, KV, BT::T, BT::E>;
    using S = Arena<K, KV>;
    constexpr uint64_t kTile = tile_of<K, KV, VARIANT>();
    if (nseg == 0) return IPM_OK;
    if (one_launch) {
        auto fk = batched_fused_kernel<K, KV, BT::T, BT::E, BT::MINB>;
        constexpr size_t smem = fused_smem<K, KV, BT::T, BT::E>();
        static std::atomic<int> occ_fused_cache{0};
        int occ = 0;
        IPM_TRY(occupancy_of(fk, BT::T, smem, occ_fused_cache, occ));
        uint32_t per_sm = uint32_t(occ);
        if (ctas_per_sm != 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
        const uint64_t tickets =
            uint64_t(nseg) + 2ull * (by_size ? (nseg + kFusedChunk - 1) / kFusedChunk : 0u);
        uint64_t grid = uint64_t(per_sm) * uint64_t(num_sms());
        if (grid > tickets) grid = tickets;
        fk<<<unsigned(grid), BT::T, smem, stream>>>((K *)buf, vals, buf_len, segs, nseg, by_size,
                                                    qa, uint64_t(kMaxPairs) * kTile, sb);
        return last_launch_status();
    }
    // levels: one CTA per multi-tile segment (the prep kernel lists them)
    auto lk = batched_levels_kernel<K, KV>;
    static std::atomic<int> occ_levels_cache{0};
    int occ_levels = 0;
    IPM_TRY(occupancy_of(lk, kLevelsThreads, S::kSmem, occ_levels_cache, occ_levels));
    uint64_t lgrid = uint64_t(occ_levels) * uint64_t(num_sms());
    if (lgrid > nseg) lgrid = nseg;
    lk<<<unsigned(lgrid), kLevelsThreads, S::kSmem, stream>>>((K *)buf, vals, qa, kTile, sb);
    IPM_TRY(last_launch_status());
    // merge: every segment
    auto mk = batched_merge_kernel<K, KV, BT::T, BT::E, BT::MINB>;
    static std::atomic<int> occ_merge_cache{0};
    int occ_merge = 0;
    IPM_TRY(occupancy_of(mk, BT::T, Tile::kSmem, occ_merge_cache, occ_merge));
    uint32_t per_sm = uint32_t(occ_merge);
    if (ctas_per_sm != 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    uint64_t grid = uint64_t(per_sm) * uint64_t(num_sms());
    if (grid > nseg) grid = nseg;
    mk<<<unsigned(grid), BT::T, Tile::kSmem, stream>>>((K *)buf, vals, buf_len, qa, nseg,
                                                      uint64_t(kMaxPairs) * kTile, sb);
    return last_launch_status();
}

template <typename K>
ipm_status batched_dispatch(void *buf, uint32_t *vals, uint64_t buf_len, QueueArea qa,
                            uint32_t nseg, uint32_t variant, uint32_t ctas_per_sm,
                            uint32_t one_launch, const ipm_segment *segs, uint32_t by_size,
                            StatusBlock *sb, cudaStream_t stream) {
    if (vals != nullptr) {
        if (variant == 2)
            return batched_launch_t<K, true, 2>(buf, vals, buf_len, qa, nseg, ctas_per_sm,
                                                one_launch, segs, by_size, sb, stream);
        if (variant == 1)
            return batched_launch_t<K, true, 1>(buf, vals, buf_len, qa, nseg, ctas_per_sm,
                                                one_launch, segs, by_size, sb, stream);
        return batched_launch_t<K, true, 0>(buf, vals, buf_len, qa, nseg, ctas_per_sm,
                                            one_launch, segs, by_size, sb, stream);
    }
    if (variant == 2)
        return batched_launch_t<K, false, 2>(buf, nullptr, buf_len, qa, nseg, ctas_per_sm,
                                             one_launch, segs, by_size, sb, stream);
    if (variant == 1)
        return batched_launch_t<K, false, 1>(buf, nullptr, buf_len, qa, nseg, ctas_per_sm,
                                             one_launch, segs, by_size, sb, stream);
    return batched_launch_t<K, false, 0>(buf, nullptr, buf_len, qa, nseg, ctas_per_sm,
                                         one_launch, segs, by_size, sb, stream);
}

// Merge tile (elements) of a variant.
template <typename K, bool KV>
uint64_t tile_t(uint32_t variant) {
    return variant == 2 ? tile_of<K, KV, 2>() : variant == 1 ? tile_of<K, KV, 1>()
                                                              : tile_of<K, KV, 0>();
}

}  // namespace batched
}  // namespace ipm
