// The last log2(C) levels of the division stage (Alg. 3) fused with the pair merge,
// one thread-block cluster of C CTAs per group of C consecutive pairs (half-size
// tiles, two CTAs per SM).
//
// After the levels above it, the C pairs k0 .. k0+C-1 of a group occupy one contiguous
// region [d_k0, d_{k0+C}) holding A[i_k0, i_{k0+C}) followed by B[j_k0, j_{k0+C}):
// exactly the inputs of those pairs, and exactly the span their outputs fill.  So the
// group needs no exchange: CTA r of the cluster stages pair k0+r's two slices (its A
// part and its B part, wherever the group's layout puts them) in its shared memory,
// the cluster barrier guarantees that every CTA of the group has read its inputs, and
// then each CTA merges its pair on chip and stores it to [d_k, d_{k+1}).  The region is
// read once and written once, and log2(C) exchange levels over the whole buffer
// disappear.  Pairs with an empty run are moved too (their data still changes place).
#include "ipm_group_common.cuh"
#include "ipm_internal.h"
#include "ipm_tile_merge.cuh"
#include "ipm_tmem.cuh"

namespace ipm {

namespace {

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t nclusters_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives and waits (release / acquire).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}

template <typename K, bool KV, int THREADS, int E, int C>
__global__ void __launch_bounds__(THREADS, 2)
    cluster_merge_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, uint64_t la,
                         uint64_t lb, const uint64_t *__restrict__ split, uint32_t G,
                         StatusBlock *sb) {
    using Shape = ClusterShape<K, KV, THREADS, E>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    K *R = reinterpret_cast<K *>(smem_raw + 128);
    uint32_t *RV = reinterpret_cast<uint32_t *>(smem_raw + 128 + Shape::kKeyBytes);
    __shared__ int abort_flag;
    __shared__ PairGeo<K> pg;
    volatile PairGeo<K> &vg = pg;
    constexpr uint32_t VK = 16u / uint32_t(sizeof(K));  // keys per 16 bytes
    constexpr uint32_t VV = 4u;                          // payloads per 16 bytes

    // every CTA of a cluster runs the same number of iterations (cluster barriers)
    const bool done = sb != nullptr && *((volatile unsigned int *)&sb->done);
    const uint32_t tid = threadIdx.x;
    const uint64_t P = 1ull << G;
    const uint64_t groups = done ? 0 : P / C;
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        abort_flag = 0;
    }
    uint32_t parity = 0;

    for (uint64_t t = cluster_id_x(); t < groups; t += nclusters_x()) {
        if (tid == 0) {
            const uint64_t n = la + lb;
            const uint64_t k0 = t * C, k1 = k0 + C, k = k0 + cluster_ctarank();
            const uint64_t dlo = (k0 * n) >> G, dhi = (k1 * n) >> G;
            const uint64_t ilo = split[k0], ihi = split[k1];
            const uint64_t d0 = (k * n) >> G, d1 = ((k + 1) * n) >> G;
            const uint64_t i0 = split[k], i1 = split[k + 1];
            // the group's layout: A[ilo, ihi) at dlo, then B[jlo, jhi); a consistent split
            // table keeps both slices of pair k inside it
            const bool ok = ilo <= i0 && i0 <= i1 && i1 <= ihi && ihi <= dhi && ilo <= dlo &&
                            i0 <= d0 && i1 - i0 <= d1 - d0 && d0 - i0 >= dlo - ilo &&
                            d1 - i1 <= dhi - ihi && d1 - d0 <= uint64_t(Shape::kTile);
            if (!ok && sb != nullptr) set_status(sb, IPM_ERR_DEVICE);
            const uint32_t c = ok ? uint32_t(d1 - d0) : 0u;
            const uint32_t a = ok ? uint32_t(i1 - i0) : 0u;
            const uint64_t posA = dlo + (i0 - ilo);
            const uint64_t posB = dlo + (ihi - ilo) + ((d0 - i0) - (dlo - ilo));
            K *gA = buf + posA, *gB = buf + posB, *gO = buf + d0;
            // staged offsets with the 16-byte phases of their global ranges
            const uint32_t oo = phase_of(gO);
            const uint32_t offA = oo + ((phase_of(gA) + VK - oo) % VK);
            const uint32_t offB = offA + a + ((phase_of(gB) + VK - (offA + a) % VK) % VK);
            pg.gA = gA;
            pg.gB = gB;
            pg.gO = gO;
            pg.a = a;
            pg.b = c - a;
            pg.offA = offA;
            pg.offB = offB;
            pg.oo = oo;
            if (KV) {
                uint32_t *vA = vals + posA, *vB = vals + posB, *vO = vals + d0;
                const uint32_t ooV = phase_of(vO);
                const uint32_t offAV = ooV + ((phase_of(vA) + VV - ooV) % VV);
                pg.vA = vA;
                pg.vB = vB;
                pg.vO = vO;
                pg.ooV = ooV;
                pg.offAV = offAV;
                pg.offBV = offAV + a + ((phase_of(vB) + VV - (offAV + a) % VV) % VV);
            }
        }
        __syncthreads();
        const uint32_t a = vg.a, b = vg.b;

        // ---- stage both slices
        if (a + b > 0) {
            if (tid == 0) {
                uint32_t tx = body_bytes(pg.gA, a) + body_bytes(pg.gB, b);
                if (KV) tx += body_bytes(pg.vA, a) + body_bytes(pg.vB, b);
                mbar_arrive_expect_tx(mbar, tx);
            }
            stage_range<K, THREADS>(R + vg.offA, vg.gA, a, mbar);
            stage_range<K, THREADS>(R + vg.offB, vg.gB, b, mbar);
            if (KV) {
                stage_range<uint32_t, THREADS>(RV + vg.offAV, vg.vA, a, mbar);
                stage_range<uint32_t, THREADS>(RV + vg.offBV, vg.vB, b, mbar);
            }
            if (!mbar_wait_bounded(mbar, parity)) atomicOr(&abort_flag, 1);
            parity ^= 1u;
        }
        __syncthreads();
        // ---- every CTA of the group has its inputs on chip: the region may be written
        cluster_sync_all();
        if (abort_flag) {
            if (tid == 0 && sb != nullptr) set_status(sb, IPM_ERR_TIMEOUT);
            continue;  // keep taking part in the cluster barriers, write nothing
        }
        if (a + b == 0) continue;

        // ---- merge on chip into the output's phase (a move when a run is empty); A at
        // R + offA and B at R + offB (payloads: RV + offAV, RV + offBV)
        merge_two<K, KV, THREADS, E, true>(R + vg.offA, RV + vg.offAV, a, vg.offB - vg.offA,
                                           vg.offBV - vg.offAV, b, R + vg.oo, RV + vg.ooV);
        fence_proxy_async_smem();
        __syncthreads();

        // ---- store
        const uint32_t c = vg.a + vg.b;
        store_range<K, THREADS>(vg.gO, R + vg.oo, c);
        if (KV) store_range<uint32_t, THREADS>(vg.vO, RV + vg.ooV, c);
        if (tid == 0) {
            bulk_commit();
            bulk_wait_read0();
        }
        fence_proxy_async_smem();
        __syncthreads();
    }
    if (tid == 0) bulk_wait_all0();
}

// ---------------------------------------------------------------------------------
// The same fusion with a group barrier in global memory instead of a cluster: groups
// of 2^F consecutive pairs (any F with 2^F <= the resident CTAs), members taken from a
// ticket.  Tickets are claimed in order, so only the newest group can be partially
// claimed; every older group is complete, its members finish, and the CTAs they free
// claim the remaining tickets: with at least 2^F resident CTAs no group waits forever.
// A member counts itself in once its slices are on chip, merges them on chip (the
// merge writes only shared memory), then waits (bounded) until the whole group has
// counted in before it stores.  The next ticket is claimed once the current pair has
// passed its barrier, while the pair's bulk store drains.
// ---------------------------------------------------------------------------------
// Claim the next pair (thread 0): its ticket and, when it is a pair, its geometry
// within its group's region.  Returns the ticket.
template <typename K, bool KV, uint32_t TILE, typename V>
__device__ __forceinline__ uint32_t group_claim(PairGeo<K, V> &pg, K *buf, V *vals,
                                                uint64_t la, uint64_t lb,
                                                const uint64_t *__restrict__ split,
                                                uint32_t G, uint32_t F, StatusBlock *sb) {
    const uint32_t t = atomicAdd(&sb->counters[kGroupTicket], 1u);
    if (uint64_t(t) < (1ull << G))
        pair_geometry<K, KV, TILE, V>(pg, buf, vals, la, lb, split, G, F, t, sb);
    return t;
}

template <typename K, bool KV, int THREADS, int E, typename V>
__global__ void __launch_bounds__(THREADS, 2)
    group_merge_kernel(K *__restrict__ buf, V *__restrict__ vals, uint64_t la,
                       uint64_t lb, const uint64_t *__restrict__ split, uint32_t G, uint32_t F,
                       uint32_t *__restrict__ gctr, StatusBlock *sb) {
    using Shape = ClusterShape<K, KV, THREADS, E, V>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    K *R = reinterpret_cast<K *>(smem_raw + 128);
    V *RV = reinterpret_cast<V *>(smem_raw + 128 + Shape::kKeyBytes);
    __shared__ int abort_flag;
    __shared__ uint32_t s_t[2];
    __shared__ PairGeo<K, V> pgs[2];  // the current pair and the next one
    if (sb == nullptr || call_finished(sb)) return;
    const uint32_t tid = threadIdx.x;
    const uint64_t P = 1ull << G;
    const uint32_t gsize = 1u << F;
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        abort_flag = 0;
        s_t[0] = group_claim<K, KV, Shape::kTile, V>(pgs[0], buf, vals, la, lb, split, G, F, sb);
    }
    __syncthreads();
    uint32_t parity = 0, cur = 0;

    for (;;) {
        const uint32_t t = s_t[cur];
        if (t >= P) break;
        volatile PairGeo<K, V> &vg = pgs[cur];
        const uint32_t a = vg.a, b = vg.b;

        // ---- stage both slices
        if (a + b > 0) {
            if (tid == 0) {
                uint32_t tx = body_bytes(pgs[cur].gA, a) + body_bytes(pgs[cur].gB, b);
                if (KV) tx += body_bytes(pgs[cur].vA, a) + body_bytes(pgs[cur].vB, b);
                mbar_arrive_expect_tx(mbar, tx);
            }
            stage_range<K, THREADS>(R + vg.offA, vg.gA, a, mbar);
            stage_range<K, THREADS>(R + vg.offB, vg.gB, b, mbar);
            if (KV) {
                stage_range<V, THREADS>(RV + vg.offAV, vg.vA, a, mbar);
                stage_range<V, THREADS>(RV + vg.offBV, vg.vB, b, mbar);
            }
            if (!mbar_wait_bounded(mbar, parity)) atomicOr(&abort_flag, 1);
            parity ^= 1u;
        }
        __syncthreads();  // every thread's head / tail loads have landed too
        uint32_t *ctr = gctr + (t >> F);
        // ---- count in: this pair's slices are on chip (a timed-out stage counts in
        // too, so that the other members are not held up before they see the error)
        if (tid == 0) atomicAdd(ctr, 1u);

        // ---- merge on chip into the output's phase (a move when a run is empty); only
        // shared memory is written, so this needs no barrier
        if (a + b > 0 && !abort_flag)
            merge_two<K, KV, THREADS, E, true, V>(R + vg.offA, RV + vg.offAV, a,
                                               vg.offB - vg.offA, vg.offBV - vg.offAV, b,
                                               R + vg.oo, RV + vg.ooV);
        fence_proxy_async_smem();

        // ---- group barrier: the group's region may be written once every member has
        // its slices on chip
        if (tid == 0 && !abort_flag) {
            DepTimer tm(wait_limit(sb));
            while (ld_acquire_u32(ctr) < gsize)
                if (tm.expired()) {
                    abort_flag = 1;
                    break;
                }
        }
        __syncthreads();
        if (abort_flag) {
            if (tid == 0) set_status(sb, IPM_ERR_TIMEOUT);
            break;
        }

        // ---- store, and claim the next pair while the bulk store reads shared memory
        if (a + b > 0) {
            store_range<K, THREADS>(vg.gO, R + vg.oo, a + b);
            if (KV) store_range<V, THREADS>(vg.vO, RV + vg.ooV, a + b);
        }
        if (tid == 0) {
            bulk_commit();
            s_t[cur ^ 1u] =
                group_claim<K, KV, Shape::kTile, V>(pgs[cur ^ 1u], buf, vals, la, lb, split, G, F, sb);
            bulk_wait_read0();
        }
        fence_proxy_async_smem();
        __syncthreads();
        cur ^= 1u;
    }
    if (tid == 0) bulk_wait_all0();
}

// ---------------------------------------------------------------------------------
// Two pairs per CTA (keys, with or without payload): the first pair is merged on chip
// and its output parked in tensor memory (TMEM, 256 columns of the SM's 512 per CTA),
// then the second is staged and merged in shared memory, so a CTA holds two merged
// pairs and a group of 2^F pairs needs 2^(F-1) resident CTAs: one more level is fused
// than with one pair per CTA.  After the barrier below the second pair is stored from shared memory and the first brought back from TMEM (each thread
// its own lane and columns) and stored the same way.  Tickets cover pairs 2t and 2t+1
// (one group: groups are aligned to 2^F >= 2 pairs); the ticket-order argument of the
// one-pair kernel holds with 2^(F-1) claims per group.  The barrier is per pair: a pair,
// once staged, counts its slices in at the pairs whose outputs overwrite them
// (count_in_slice), and a pair stores once its own count covers its output, that is
// once the few members that read its destination have their data on chip, not the
// whole group.  Exactly two CTAs fit an SM (each CTA takes at least kGroup2Smem of
// shared memory), so the two allocations never wait.
// ---------------------------------------------------------------------------------
constexpr uint32_t kGroup2Cols = 256;
// more than a third of the SM's 228 KB (no third CTA fits), less than half with each
// CTA's static and reserved bytes (two fit the carveout)
constexpr size_t kGroup2Smem = 78u << 10;

// The dynamic shared memory of a two-pairs CTA: its staging buffer, at least kGroup2Smem.
template <typename K, bool KV, typename V>
constexpr size_t group2_smem() {
    constexpr size_t need =
        ClusterShape<K, KV, ClusterTileOf<K, KV, V>::T, ClusterTileOf<K, KV, V>::E, V>::kSmem;
    return need > kGroup2Smem ? need : kGroup2Smem;
}

template <typename K, bool KV, typename V, int THREADS, int E>
__global__ void __launch_bounds__(THREADS, 2)
    group2_merge_kernel(K *__restrict__ buf, V *__restrict__ vals, uint64_t la, uint64_t lb,
                        const uint64_t *__restrict__ split, uint32_t G, uint32_t F,
                        uint32_t *__restrict__ gctr, StatusBlock *sb) {
    // a thread parks its E keys (and E payloads) as W 32-bit words in W consecutive
    // columns of its lane; the warps sharing a lane quarter take column blocks of CS (W
    // rounded up to 64, so every 32-column access starts at a multiple of 32)
    constexpr int WK = E * int(sizeof(K)) / 4, WV = KV ? E * int(sizeof(V)) / 4 : 0;
    constexpr int W = WK + WV;
    constexpr uint32_t CS = uint32_t((W + 63) / 64 * 64);
    static_assert(E % 2 == 1 && THREADS % 128 == 0 && sizeof(K) % 4 == 0 && sizeof(V) % 4 == 0,
                  "shape");
    static_assert((THREADS / 128) * CS <= kGroup2Cols, "a thread's outputs fit its columns");
    using Shape = ClusterShape<K, KV, THREADS, E, V>;
    static_assert(Shape::kSmem <= group2_smem<K, KV, V>(), "launched with the staging buffer");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    K *R = reinterpret_cast<K *>(smem_raw + 128);
    V *RV = reinterpret_cast<V *>(smem_raw + 128 + Shape::kKeyBytes);
    __shared__ int abort_flag;
    __shared__ uint32_t s_t[2], s_taddr;
    __shared__ PairGeo<K, V> pgs[2][2];  // [current / next claim][first / second pair]
    if (sb == nullptr || call_finished(sb)) return;
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    const uint64_t claims = (1ull << G) >> 1;
    if (warp == 0) {
        tmem_alloc<kGroup2Cols>(&s_taddr);
        tmem_relinquish();
    }
    auto claim = [&](uint32_t q) {  // thread 0
        const uint32_t t = atomicAdd(&sb->counters[kGroupTicket], 1u);
        s_t[q] = t;
        if (uint64_t(t) < claims) {
            pair_geometry<K, KV, Shape::kTile, V>(pgs[q][0], buf, vals, la, lb, split, G, F,
                                                  2ull * t, sb);
            pair_geometry<K, KV, Shape::kTile, V>(pgs[q][1], buf, vals, la, lb, split, G, F,
                                                  2ull * t + 1, sb);
        }
    };
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        abort_flag = 0;
        claim(0);
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    // this thread's TMEM cells: its warp's lane quarter, columns CS (warp / 4) + 0..W-1
    // (recomputed from shared memory where used, so it is not live across the merge)
    auto tcol = [&]() {
        return tmem_warp_addr(*((volatile uint32_t *)&s_taddr), (warp >> 2) * CS);
    };
    uint32_t parity = 0, cur = 0;

    // stage one pair's two slices (bodies by bulk copy, heads / tails by plain loads)
    auto stage = [&](volatile PairGeo<K, V> &vg) {
        const uint32_t a = vg.a, b = vg.b;
        if (a + b == 0) return;
        if (tid == 0) {
            uint32_t tx = body_bytes(const_cast<K *>(vg.gA), a) +
                          body_bytes(const_cast<K *>(vg.gB), b);
            if (KV)
                tx += body_bytes(const_cast<V *>(vg.vA), a) + body_bytes(const_cast<V *>(vg.vB), b);
            mbar_arrive_expect_tx(mbar, tx);
        }
        stage_range<K, THREADS>(R + vg.offA, vg.gA, a, mbar);
        stage_range<K, THREADS>(R + vg.offB, vg.gB, b, mbar);
        if (KV) {
            stage_range<V, THREADS>(RV + vg.offAV, vg.vA, a, mbar);
            stage_range<V, THREADS>(RV + vg.offBV, vg.vB, b, mbar);
        }
        if (!mbar_wait_bounded(mbar, parity)) atomicOr(&abort_flag, 1);
        parity ^= 1u;
    };
    // store one pair's merged keys (and payloads) from the staging buffer
    auto store = [&](volatile PairGeo<K, V> &vg) {
        const uint32_t c = vg.a + vg.b;
        if (c == 0) return;
        store_range<K, THREADS>(const_cast<K *>(vg.gO), R + vg.oo, c);
        if (KV) store_range<V, THREADS>(const_cast<V *>(vg.vO), RV + vg.ooV, c);
    };

    for (;;) {
        if (uint64_t(*((volatile uint32_t *)&s_t[cur])) >= claims) break;
        volatile PairGeo<K, V> &g0 = pgs[cur][0];
        volatile PairGeo<K, V> &g1 = pgs[cur][1];

        // ---- first pair: stage, merge into registers, park in TMEM
        stage(g0);
        __syncthreads();  // every thread's head / tail loads have landed too
        if (tid == 0 && !abort_flag) {  // its slices are on chip
            count_in_slice(gctr, la + lb, G, uint64_t(g0.gA - buf), g0.a);
            count_in_slice(gctr, la + lb, G, uint64_t(g0.gB - buf), g0.b);
        }
        {
            K ok[E] = {};  // outputs past the pair's end are parked but never read back
            V ov[KV ? E : 1] = {};
            uint32_t oi[KV ? E : 1];
            const uint32_t a0 = g0.a, c0 = g0.a + g0.b;
            const K *sk = R + g0.offA;
            if (!abort_flag) {
                merge_path_regs<K, KV, THREADS, E, true>(sk, a0, g0.offB - g0.offA, g0.b, ok,
                                                         oi);
                const uint32_t dt = tid * uint32_t(E);
                if (KV && dt < c0) {  // the merge gave staged indices: gather both
                    const V *sv = RV + g0.offAV;
                    const uint32_t bo = g0.offB - g0.offA, bov = g0.offBV - g0.offAV;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const uint32_t q = (dt + e < c0) ? oi[KV ? e : 0] : 0u;
                        ok[e] = sk[q];
                        ov[KV ? e : 0] = sv[q < a0 ? q : bov + (q - bo)];
                    }
                }
            }
            uint32_t w[W];
            memcpy(w, ok, sizeof(ok));
            if (KV) memcpy(w + WK, ov, size_t(WV) * 4);
            const uint32_t ta = tcol();
#pragma unroll
            for (int c = 0; c + 32 <= W; c += 32)
                tmem_st32(ta + uint32_t(c), *reinterpret_cast<const uint32_t(*)[32]>(w + c));
#pragma unroll
            for (int c = W / 32 * 32; c < W; ++c) tmem_st1(ta + uint32_t(c), w[c]);
            tmem_wait_st();
        }
        __syncthreads();  // the staging buffer is read: free for the second pair

        // ---- second pair: stage, count in, merge on chip into the output's phase
        stage(g1);
        __syncthreads();
        if (tid == 0 && !abort_flag) {
            count_in_slice(gctr, la + lb, G, uint64_t(g1.gA - buf), g1.a);
            count_in_slice(gctr, la + lb, G, uint64_t(g1.gB - buf), g1.b);
        }
        if (!abort_flag && g1.a + g1.b > 0)
            merge_two<K, KV, THREADS, E, true, V>(R + g1.offA, RV + g1.offAV, g1.a,
                                                  g1.offB - g1.offA, g1.offBV - g1.offAV, g1.b,
                                                  R + g1.oo, RV + g1.ooV);
        fence_proxy_async_smem();

        // ---- barrier: each pair's output range may be written once every element it
        // overwrites is on chip (its count reaches its length)
        if (tid == 0 && !abort_flag) {
            const uint64_t p0 = 2ull * *((volatile uint32_t *)&s_t[cur]);
            const uint32_t c0 = g0.a + g0.b, c1 = g1.a + g1.b;
            DepTimer tm(wait_limit(sb));
            while (ld_acquire_u32(gctr + p0) < c0 || ld_acquire_u32(gctr + p0 + 1) < c1)
                if (tm.expired() || *((volatile unsigned *)&sb->status) != 0) {
                    abort_flag = 1;
                    break;
                }
        }
        __syncthreads();
        if (abort_flag) {
            if (tid == 0) set_status(sb, IPM_ERR_TIMEOUT);
            break;
        }

        // ---- store the second pair, then bring the first back from TMEM and store it
        store(g1);
        if (tid == 0) {
            bulk_commit();
            bulk_wait_read0();
        }
        fence_proxy_async_smem();
        __syncthreads();  // the staging buffer is free again
        {
            uint32_t w[W];
            const uint32_t ta = tcol();
#pragma unroll
            for (int c = 0; c + 32 <= W; c += 32)
                tmem_ld32(ta + uint32_t(c), *reinterpret_cast<uint32_t(*)[32]>(w + c));
#pragma unroll
            for (int c = W / 32 * 32; c < W; ++c) w[c] = tmem_ld1(ta + uint32_t(c));
            tmem_wait_ld();
            const uint32_t c0 = g0.a + g0.b;
            const uint32_t dt = tid * uint32_t(E);
            K ok[E];
            memcpy(ok, w, sizeof(ok));
            K *out = R + g0.oo;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (dt + e < c0) out[dt + e] = ok[e];
            if (KV) {
                V ov[KV ? E : 1];
                memcpy(ov, w + WK, size_t(WV) * 4);
                V *vout = RV + g0.ooV;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (dt + e < c0) vout[dt + e] = ov[KV ? e : 0];
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        store(g0);
        if (tid == 0) {
            bulk_commit();
            claim(cur ^ 1u);  // the next claim, while the bulk store reads shared memory
            bulk_wait_read0();
        }
        fence_proxy_async_smem();
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        cur ^= 1u;
    }
    if (tid == 0) bulk_wait_all0();
    // every TMEM access of the CTA has completed (the waits above): free the columns
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc<kGroup2Cols>(s_taddr);
}

template <typename K, bool KV, int THREADS, int E, typename V>
int group_grid() {
    // computed by the first call (static initialisation: other threads wait for it)
    static const int cached = []() -> int {
        using Shape = ClusterShape<K, KV, THREADS, E, V>;
        auto kern = group_merge_kernel<K, KV, THREADS, E, V>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Shape::kSmem)) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS,
                                                          Shape::kSmem) != cudaSuccess) {
            (void)cudaGetLastError();
            per_sm = 0;
        }
        return per_sm > 0 ? per_sm * num_sms() : 0;
    }();
    return cached;
}

template <typename K, bool KV, int THREADS, int E, typename V>
ipm_status group_merge_t(void *buf, void *vals, uint64_t la, uint64_t lb,
                         const uint64_t *split, uint32_t G, uint32_t F, uint32_t *gctr,
                         StatusBlock *sb, cudaStream_t stream) {
    using Shape = ClusterShape<K, KV, THREADS, E, V>;
    const int grid = group_grid<K, KV, THREADS, E, V>();
    if (grid < (1 << F)) return IPM_ERR_CUDA;
    const uint64_t P = 1ull << G;
    const unsigned g = unsigned(P < uint64_t(grid) ? P : uint64_t(grid));
    group_merge_kernel<K, KV, THREADS, E, V><<<g, THREADS, Shape::kSmem, stream>>>(
        (K *)buf, (V *)vals, la, lb, split, G, F, gctr, sb);
    return last_launch_status();
}

// Resident CTAs of the two-pairs kernel (0 unless exactly two fit an SM: each CTA
// holds half of the SM's TMEM), computed once from its registers, shared memory and
// threads against the SM's limits.  (The occupancy query answers one CTA per SM for any
// kernel that allocates TMEM, whatever it allocates; two such CTAs do run side by side.)
template <typename K, bool KV, typename V>
int group2_grid() {
    // computed by the first call (static initialisation: other threads wait for it)
    static const int cached = []() -> int {
        constexpr int T = ClusterTileOf<K, KV, V>::T;
        auto kern = group2_merge_kernel<K, KV, V, T, 33>;
        int dev = 0, regs_sm = 0, smem_sm = 0, threads_sm = 0, reserved = 0;
        cudaFuncAttributes fa;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(group2_smem<K, KV, V>())) != cudaSuccess ||
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 int(cudaSharedmemCarveoutMaxShared)) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        const long regs_cta = long(fa.numRegs) * T;
        const long smem_cta =
            long(group2_smem<K, KV, V>()) + long(fa.sharedSizeBytes) + long(reserved);
        long per_sm = threads_sm / T;
        if (regs_cta > 0 && regs_sm / regs_cta < per_sm) per_sm = regs_sm / regs_cta;
        if (smem_sm / smem_cta < per_sm) per_sm = smem_sm / smem_cta;
        return per_sm == 2 ? 2 * num_sms() : 0;
    }();
    return cached;
}

template <typename K, bool KV, typename V>
ipm_status group2_merge_t(void *buf, void *vals, uint64_t la, uint64_t lb,
                          const uint64_t *split, uint32_t G, uint32_t F, uint32_t *gctr,
                          StatusBlock *sb, cudaStream_t stream) {
    const int grid = group2_grid<K, KV, V>();
    if (F < 1 || grid < (1 << (F - 1))) return IPM_ERR_CUDA;
    const uint64_t claims = (1ull << G) >> 1;
    const unsigned g = unsigned(claims < uint64_t(grid) ? claims : uint64_t(grid));
    constexpr int T = ClusterTileOf<K, KV, V>::T;
    static_assert(ClusterTileOf<K, KV, V>::E == 33, "the instantiated shape");
    group2_merge_kernel<K, KV, V, T, 33><<<g, T, group2_smem<K, KV, V>(), stream>>>(
        (K *)buf, (V *)vals, la, lb, split, G, F, gctr, sb);
    return last_launch_status();
}

template <typename K>
int group2_grid_vb(uint32_t vb) {
    return vb == 8   ? group2_grid<K, true, uint64_t>()
           : vb != 0 ? group2_grid<K, true, uint32_t>()
                     : group2_grid<K, false, uint32_t>();
}

template <typename K>
ipm_status group2_dispatch(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                           const uint64_t *split, uint32_t G, uint32_t F, uint32_t *gctr,
                           StatusBlock *sb, cudaStream_t stream) {
    if (vb == 8)
        return group2_merge_t<K, true, uint64_t>(buf, vals, la, lb, split, G, F, gctr, sb,
                                                 stream);
    if (vb != 0)
        return group2_merge_t<K, true, uint32_t>(buf, vals, la, lb, split, G, F, gctr, sb,
                                                 stream);
    return group2_merge_t<K, false, uint32_t>(buf, nullptr, la, lb, split, G, F, gctr, sb,
                                              stream);
}

// Resident clusters of the kernel on the current device (0 when clusters of C CTAs
// cannot be scheduled), queried once per instantiation.
template <typename K, bool KV, int THREADS, int E, int C>
int cluster_capacity() {
    // computed by the first call (static initialisation: other threads wait for it)
    static const int cached = []() -> int {
        using Shape = ClusterShape<K, KV, THREADS, E>;
        auto kern = cluster_merge_kernel<K, KV, THREADS, E, C>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Shape::kSmem)) != cudaSuccess ||
            (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                           1) != cudaSuccess)) {
            (void)cudaGetLastError();
            return 0;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C * 64, 1, 1);
        cfg.blockDim = dim3(THREADS, 1, 1);
        cfg.dynamicSmemBytes = Shape::kSmem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int mc = 0;
        if (cudaOccupancyMaxActiveClusters(&mc, kern, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            mc = 0;
        }
        return mc > 0 ? mc : 0;
    }();
    return cached;
}

template <typename K, bool KV, int THREADS, int E, int C>
ipm_status cluster_merge_t(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                           const uint64_t *split, uint32_t G, StatusBlock *sb,
                           cudaStream_t stream) {
    using Shape = ClusterShape<K, KV, THREADS, E>;
    auto kern = cluster_merge_kernel<K, KV, THREADS, E, C>;
    const int max_clusters = cluster_capacity<K, KV, THREADS, E, C>();
    if (max_clusters < 1) return IPM_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = Shape::kSmem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const uint64_t groups = (1ull << G) / C;
    uint64_t nc = groups < uint64_t(max_clusters) ? groups : uint64_t(max_clusters);
    if (nc == 0) nc = 1;
    cfg.gridDim = dim3(unsigned(nc * C), 1, 1);
    IPM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, (K *)buf, vals, la, lb, split, G, sb));
    return IPM_OK;
}

// Half the plain merge's tile (two CTAs per SM, so one CTA's merge overlaps the
// other's staging): 4-byte keys 512 x 33, 8-byte keys and key-value 256 x 33.  The
// caller splits one level deeper so that every pair fits.

template <typename K, int C>
ipm_status cluster_dispatch(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                            const uint64_t *split, uint32_t G, StatusBlock *sb,
                            cudaStream_t stream) {
    if (vals != nullptr)
        return cluster_merge_t<K, true, ClusterTileOf<K, true>::T, ClusterTileOf<K, true>::E,
                               C>(buf, vals, la, lb, split, G, sb, stream);
    return cluster_merge_t<K, false, ClusterTileOf<K, false>::T, ClusterTileOf<K, false>::E,
                           C>(buf, nullptr, la, lb, split, G, sb, stream);
}

template <typename K, int C>
int capacity_kv(bool kv) {
    return kv ? cluster_capacity<K, true, ClusterTileOf<K, true>::T, ClusterTileOf<K, true>::E,
                                 C>()
              : cluster_capacity<K, false, ClusterTileOf<K, false>::T,
                                 ClusterTileOf<K, false>::E, C>();
}

template <int C>
int capacity_by_key(ipm_dtype key, bool kv) {
    switch (key) {
    case IPM_INT32:
        return capacity_kv<int32_t, C>(kv);
    case IPM_UINT32:
        return capacity_kv<uint32_t, C>(kv);
    case IPM_UINT64:
    case IPM_INT64:
        return capacity_kv<uint64_t, C>(kv);
    case IPM_FLOAT32:
        return capacity_kv<float, C>(kv);
    }
    return 0;
}

template <int C>
ipm_status cluster_by_key(void *buf, uint32_t *vals, uint64_t la, uint64_t lb, ipm_dtype key,
                          const uint64_t *split, uint32_t G, StatusBlock *sb,
                          cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        return cluster_dispatch<int32_t, C>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_UINT32:
        return cluster_dispatch<uint32_t, C>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_UINT64:
        return cluster_dispatch<uint64_t, C>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_INT64:
        return cluster_dispatch<int64_t, C>(buf, vals, la, lb, split, G, sb, stream);
    case IPM_FLOAT32:
        return cluster_dispatch<float, C>(buf, vals, la, lb, split, G, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

template <typename K, bool KV, typename V>
ipm_status group_shape_t(void *buf, void *vals, uint64_t la, uint64_t lb,
                         const uint64_t *split, uint32_t G, uint32_t F, uint32_t *gctr,
                         StatusBlock *sb, cudaStream_t stream) {
    return group_merge_t<K, KV, ClusterTileOf<K, KV, V>::T, ClusterTileOf<K, KV, V>::E, V>(
        buf, vals, la, lb, split, G, F, gctr, sb, stream);
}

template <typename K>
ipm_status group_dispatch(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                          const uint64_t *split, uint32_t G, uint32_t F, uint32_t *gctr,
                          StatusBlock *sb, cudaStream_t stream) {
    if (vb == 8)
        return group_shape_t<K, true, uint64_t>(buf, vals, la, lb, split, G, F, gctr, sb,
                                                stream);
    if (vb != 0)
        return group_shape_t<K, true, uint32_t>(buf, vals, la, lb, split, G, F, gctr, sb,
                                                stream);
    return group_shape_t<K, false, uint32_t>(buf, nullptr, la, lb, split, G, F, gctr, sb,
                                             stream);
}

template <typename K>
int group_grid_kv(uint32_t vb) {
    if (vb == 8)
        return group_grid<K, true, ClusterTileOf<K, true, uint64_t>::T,
                          ClusterTileOf<K, true, uint64_t>::E, uint64_t>();
    if (vb != 0)
        return group_grid<K, true, ClusterTileOf<K, true>::T, ClusterTileOf<K, true>::E,
                          uint32_t>();
    return group_grid<K, false, ClusterTileOf<K, false>::T, ClusterTileOf<K, false>::E,
                      uint32_t>();
}

}  // namespace

uint32_t usable_group_levels(ipm_dtype key, uint32_t vb, uint32_t wanted) {
    int grid = 0;
    switch (key) {
    case IPM_INT32: grid = group_grid_kv<int32_t>(vb); break;
    case IPM_UINT32: grid = group_grid_kv<uint32_t>(vb); break;
    case IPM_UINT64: grid = group_grid_kv<uint64_t>(vb); break;
    case IPM_INT64: grid = group_grid_kv<int64_t>(vb); break;
    case IPM_FLOAT32: grid = group_grid_kv<float>(vb); break;
    }
    uint32_t f = wanted;
    while (f > 0 && (1 << f) > grid) --f;  // a whole group must fit the resident CTAs
    return f;
}

ipm_status launch_group_merge(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                              ipm_dtype key, const uint64_t *split, uint32_t G, uint32_t F,
                              uint32_t *gctr, StatusBlock *sb, cudaStream_t stream) {
    IPM_CUDA_TRY(cudaMemsetAsync(gctr, 0, sizeof(uint32_t) * size_t((1ull << G) >> F), stream));
    switch (key) {
    case IPM_INT32:
        return group_dispatch<int32_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_UINT32:
        return group_dispatch<uint32_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_UINT64:
        return group_dispatch<uint64_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_INT64:
        return group_dispatch<int64_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_FLOAT32:
        return group_dispatch<float>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

uint32_t usable_group2_levels(ipm_dtype key, uint32_t vb, uint32_t wanted) {
    int grid = 0;
    switch (key) {
    case IPM_INT32: grid = group2_grid_vb<int32_t>(vb); break;
    case IPM_UINT32: grid = group2_grid_vb<uint32_t>(vb); break;
    case IPM_FLOAT32: grid = group2_grid_vb<float>(vb); break;
    case IPM_UINT64: grid = group2_grid_vb<uint64_t>(vb); break;
    case IPM_INT64: grid = group2_grid_vb<int64_t>(vb); break;
    }
    if (grid == 0 || wanted == 0) return 0;
    uint32_t f = wanted;
    while (f > 1 && (1 << (f - 1)) > grid) --f;  // a group's claims must fit the residents
    return f;
}

ipm_status launch_group2_merge(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                               ipm_dtype key, const uint64_t *split, uint32_t G, uint32_t F,
                               uint32_t *gctr, StatusBlock *sb, cudaStream_t stream) {
    // one count per pair (the per-pair barrier)
    IPM_CUDA_TRY(cudaMemsetAsync(gctr, 0, sizeof(uint32_t) * size_t(1ull << G), stream));
    switch (key) {
    case IPM_INT32:
        return group2_dispatch<int32_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_UINT32:
        return group2_dispatch<uint32_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_FLOAT32:
        return group2_dispatch<float>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_UINT64:
        return group2_dispatch<uint64_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    case IPM_INT64:
        return group2_dispatch<int64_t>(buf, vals, vb, la, lb, split, G, F, gctr, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

uint32_t usable_fused_levels(ipm_dtype key, bool with_values, uint32_t wanted) {
    for (uint32_t f = wanted; f > 0; --f) {
        int cap = 0;
        switch (f) {
        case 1: cap = capacity_by_key<2>(key, with_values); break;
        case 2: cap = capacity_by_key<4>(key, with_values); break;
        case 3: cap = capacity_by_key<8>(key, with_values); break;
        case 4: cap = capacity_by_key<16>(key, with_values); break;
        default: cap = 0;
        }
        if (cap > 0) return f;
    }
    return 0;
}

ipm_status launch_cluster_merge(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                                ipm_dtype key, const uint64_t *split, uint32_t G,
                                uint32_t log2_cluster, StatusBlock *sb, cudaStream_t stream) {
    switch (log2_cluster) {
    case 1:
        return cluster_by_key<2>(buf, vals, la, lb, key, split, G, sb, stream);
    case 2:
        return cluster_by_key<4>(buf, vals, la, lb, key, split, G, sb, stream);
    case 3:
        return cluster_by_key<8>(buf, vals, la, lb, key, split, G, sb, stream);
    case 4:
        return cluster_by_key<16>(buf, vals, la, lb, key, split, G, sb, stream);
    }
    return IPM_ERR_INVALID_ARG;
}

}  // namespace ipm

namespace ipm {

uint64_t cluster_tile_capacity(ipm_dtype key, uint32_t vb) {
    const uint32_t elem = uint32_t(dtype_bytes(key)) + vb;
    return uint64_t(elem == 4 ? 512 : (elem <= 12 ? 256 : 128)) * 33u;
}

}  // namespace ipm
