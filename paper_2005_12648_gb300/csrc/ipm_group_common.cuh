// Pieces of the fused bottom-level kernels (ipm_cluster_merge.cu): the half-size pair
// tile, the staging of unaligned ranges through shared memory, and the geometry of a
// pair inside its group's region.
#pragma once

#include "ipm_internal.h"
#include "ipm_tile_merge.cuh"

namespace ipm {

template <typename K, bool KV, int THREADS, int E, typename V = uint32_t>
struct ClusterShape {
    static constexpr int kTile = THREADS * E;
    static constexpr int kSlack = 16;  // phase offsets of the three ranges
    static constexpr size_t kKeyBytes = (size_t(kTile + kSlack) * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t kValBytes =
        KV ? (size_t(kTile + kSlack) * sizeof(V) + 15) / 16 * 16 : 0;
    static constexpr size_t kSmem = 128 + kKeyBytes + kValBytes;
};

// Half the plain merge's tile: 4-byte keys alone 512 x 33; up to 12 bytes per element
// 256 x 33; 16 bytes (8-byte keys with an 8-byte payload) 128 x 33.
template <typename K, bool KV, typename V = uint32_t>
struct ClusterTileOf {
    static constexpr int kElem = int(sizeof(K)) + (KV ? int(sizeof(V)) : 0);
    static constexpr int T = kElem == 4 ? 512 : (kElem <= 12 ? 256 : 128), E = 33;
};

// Element phase of an address within its 16-byte line.
template <typename T>
__device__ __forceinline__ uint32_t phase_of(const T *p) {
    return uint32_t(reinterpret_cast<uintptr_t>(p) & 15u) / uint32_t(sizeof(T));
}

// Issue the staging of src[0, len) into dst[0, len) (dst has src's 16-byte phase): the
// body with one bulk copy counted on mbar, head and tail with plain loads.  Returns
// the body bytes.
template <typename T, int THREADS>
__device__ __forceinline__ uint32_t stage_range(T *dst, const T *src, uint32_t len,
                                                uint64_t *mbar) {
    const Geo<int(sizeof(T))> gg(src, len);
    const uint32_t tid = threadIdx.x;
    const uint32_t bytes = gg.body * uint32_t(sizeof(T));
    if (tid == 0 && bytes) bulk_load(dst + gg.head, src + gg.head, bytes, mbar);
    for (uint32_t j = tid; j < gg.head; j += THREADS) dst[j] = src[j];
    for (uint32_t j = gg.tail_start + tid; j < len; j += THREADS) dst[j] = src[j];
    return bytes;
}

template <typename T>
__device__ __forceinline__ uint32_t body_bytes(const T *src, uint32_t len) {
    const Geo<int(sizeof(T))> gg(src, len);
    return gg.body * uint32_t(sizeof(T));
}

// Store src[0, len) (src has dst's phase) to dst: body by one bulk store, head and tail
// with plain stores.
template <typename T, int THREADS>
__device__ __forceinline__ void store_range(T *dst, const T *src, uint32_t len) {
    const Geo<int(sizeof(T))> gg(dst, len);
    const uint32_t tid = threadIdx.x;
    const uint32_t bytes = gg.body * uint32_t(sizeof(T));
    if (tid == 0 && bytes) bulk_store(dst + gg.head, src + gg.head, bytes);
    for (uint32_t j = tid; j < gg.head; j += THREADS) dst[j] = src[j];
    for (uint32_t j = gg.tail_start + tid; j < len; j += THREADS) dst[j] = src[j];
}

// Geometry of one CTA's pair in the current group, computed by thread 0 into shared
// memory (so the merge does not have to keep it in registers).
template <typename K, typename V = uint32_t>
struct PairGeo {
    K *gA, *gB, *gO;              // the A slice, the B slice, the output range
    V *vA, *vB, *vO;              // payload ranges (key-value)
    uint32_t a, b;                // run lengths
    uint32_t offA, offB, oo;      // staged offsets (keys)
    uint32_t offAV, offBV, ooV;   // staged offsets (payloads)
};

constexpr uint32_t kGroupTicket = 40;  // status block counter of the group kernel

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 of a CTA that has a slice [s, s + len) of the buffer on chip: count it in at
// the pairs whose output ranges [d_k, d_k+1) (d_k = floor(k n / 2^G)) it overlaps, one
// count per element.  Within a group the members' slices tile the group's region
// exactly, so pair k's counter reaches d_k+1 - d_k once every element its output
// overwrites is on chip.  (k n and (x + 1) 2^G stay below 2^64: a plan has n < 2^38.)
__device__ __forceinline__ void count_in_slice(uint32_t *cnt, uint64_t n, uint32_t G,
                                               uint64_t s, uint64_t len) {
    const uint64_t e = s + len;
    for (uint64_t x = s; x < e;) {
        const uint64_t k = (((x + 1) << G) - 1) / n;  // the last k with d_k <= x
        const uint64_t dk1 = ((k + 1) * n) >> G;       // > x
        const uint64_t y = dk1 < e ? dk1 : e;
        atomicAdd(cnt + k, uint32_t(y - x));
        x = y;
    }
}

// The geometry of pair k within its group of 2^F pairs (the group's region holds A's
// slices of the group, then B's): where its two slices are, where its output goes, and
// their phases in the staging buffer.
template <typename K, bool KV, uint32_t TILE, typename V>
__device__ __forceinline__ void pair_geometry(PairGeo<K, V> &pg, K *buf, V *vals, uint64_t la,
                                              uint64_t lb, const uint64_t *__restrict__ split,
                                              uint32_t G, uint32_t F, uint64_t k,
                                              StatusBlock *sb) {
    constexpr uint32_t VK = 16u / uint32_t(sizeof(K));
    constexpr uint32_t VV = 16u / uint32_t(sizeof(V));
    const uint64_t n = la + lb;
    const uint64_t k0 = (k >> F) << F, k1 = k0 + (1ull << F);
    const uint64_t dlo = (k0 * n) >> G, dhi = (k1 * n) >> G;
    const uint64_t ilo = split[k0], ihi = split[k1];
    const uint64_t d0 = (k * n) >> G, d1 = ((k + 1) * n) >> G;
    const uint64_t i0 = split[k], i1 = split[k + 1];
    const bool ok = ilo <= i0 && i0 <= i1 && i1 <= ihi && ihi <= dhi && ilo <= dlo &&
                    i0 <= d0 && i1 - i0 <= d1 - d0 && d0 - i0 >= dlo - ilo &&
                    d1 - i1 <= dhi - ihi && d1 - d0 <= uint64_t(TILE);
    if (!ok) set_status(sb, IPM_ERR_DEVICE);
    const uint32_t c = ok ? uint32_t(d1 - d0) : 0u;
    const uint32_t a = ok ? uint32_t(i1 - i0) : 0u;
    // the group's layout: A[ilo, ihi) at dlo, then B
    const uint64_t posA = dlo + (i0 - ilo);
    const uint64_t posB = dlo + (ihi - ilo) + ((d0 - i0) - (dlo - ilo));
    K *gA = buf + posA, *gB = buf + posB, *gO = buf + d0;
    const uint32_t oo = phase_of(gO);
    const uint32_t offA = oo + ((phase_of(gA) + VK - oo) % VK);
    pg.gA = gA;
    pg.gB = gB;
    pg.gO = gO;
    pg.a = a;
    pg.b = c - a;
    pg.offA = offA;
    pg.offB = offA + a + ((phase_of(gB) + VK - (offA + a) % VK) % VK);
    pg.oo = oo;
    if (KV) {
        V *vA = vals + posA, *vB = vals + posB, *vO = vals + d0;
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

}  // namespace ipm
