// Division stage (Alg. 3): level-by-level exchange of the two middle blocks.
//
// With P = 2^G pairs and the split table i_k on d_k = floor(k*n/P), the level-l pair r
// (final pairs [r*2^{G-l}, (r+1)*2^{G-l})) holds A[i_lo, i_hi) | B[j_lo, j_hi) at d_lo
// when level l starts.  Its mid diagonal splits it into A_lo A_hi | B_lo B_hi and the
// middle X = A_hi = A[i_mid, i_hi), Y = B_lo = B[j_lo, j_mid) at s = d_lo + i_mid - i_lo
// is exchanged [X|Y] -> [Y|X] (Sec. 3.4), giving A_lo B_lo | A_hi B_hi.
//
// The exchange is executed as two batched reversal passes, rev(rev(X) rev(Y)) = Y X:
// pass 1 reverses X and Y of every rotation of the level, pass 2 reverses each whole
// middle.  Each pass is a set of independent element-pair swaps (front i <-> back
// len-1-i of a segment), so it needs no ordering between CTAs; loads are coalesced on
// both ends (consecutive threads take consecutive pairs).
#include "ipm_internal.h"

namespace ipm {

namespace {

constexpr uint32_t kPlanThreads = 1024;

__device__ __forceinline__ uint32_t rev_units(uint64_t len) {
    return uint32_t(((len >> 1) + kRevUnit - 1) / kRevUnit);
}

// Block-wide exclusive scan of one uint32 per thread (kPlanThreads threads).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[32];
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= unsigned(o)) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= unsigned(o)) w += y;
        }
        warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    const uint32_t warp_excl = wid ? warp_sums[wid - 1] : 0u;
    *total = warp_sums[31];
    __syncthreads();
    return warp_excl + x - v;
}

struct Rot {
    uint64_t s, a, b;
};

__device__ __forceinline__ Rot level_rotation(const uint64_t *split, uint64_t n, uint32_t G,
                                              uint32_t l, uint64_t r) {
    const uint64_t k_lo = r << (G - l);
    const uint64_t k_mid = k_lo + (1ull << (G - l - 1));
    const uint64_t k_hi = k_lo + (1ull << (G - l));
    const uint64_t d_lo = (k_lo * n) >> G, d_mid = (k_mid * n) >> G;
    const uint64_t i_lo = split[k_lo], i_mid = split[k_mid], i_hi = split[k_hi];
    Rot q;
    q.s = d_lo + (i_mid - i_lo);
    q.a = i_hi - i_mid;
    q.b = (d_mid - i_mid) - (d_lo - i_lo);
    return q;
}

// One block per level: the rotations of level l, their reversal segments and the
// exclusive unit prefixes of both passes.
__global__ void __launch_bounds__(kPlanThreads)
    plan_levels_kernel(const uint64_t *__restrict__ split, uint64_t n, uint32_t G,
                       PlanArea pa, const StatusBlock *sb) {
    if (sb != nullptr && *((volatile const unsigned int *)&sb->done)) return;
    const uint32_t l = blockIdx.x;
    const uint64_t R = 1ull << l;
    Seg *seg1 = pa.seg1 + 2ull * (R - 1);
    uint32_t *pf1 = pa.pf1 + 2ull * (R - 1) + l;
    Seg *seg2 = pa.seg2 + (R - 1);
    uint32_t *pf2 = pa.pf2 + (R - 1) + l;
    const uint64_t per = (R + kPlanThreads - 1) / kPlanThreads;
    const uint64_t r0 = per * threadIdx.x;
    const uint64_t r1 = r0 + per < R ? r0 + per : R;
    uint32_t u1 = 0, u2 = 0;
    for (uint64_t r = r0; r < r1; ++r) {
        Rot q = level_rotation(split, n, G, l, r);
        u1 += rev_units(q.a) + rev_units(q.b);
        u2 += rev_units(q.a + q.b);
    }
    uint32_t tot1, tot2;
    uint32_t e1 = block_exclusive_scan(u1, &tot1);
    uint32_t e2 = block_exclusive_scan(u2, &tot2);
    for (uint64_t r = r0; r < r1; ++r) {
        Rot q = level_rotation(split, n, G, l, r);
        seg1[2 * r] = Seg{q.s, q.a};
        seg1[2 * r + 1] = Seg{q.s + q.a, q.b};
        seg2[r] = Seg{q.s, q.a + q.b};
        pf1[2 * r] = e1;
        e1 += rev_units(q.a);
        pf1[2 * r + 1] = e1;
        e1 += rev_units(q.b);
        pf2[r] = e2;
        e2 += rev_units(q.a + q.b);
    }
    if (threadIdx.x == 0) {
        pf1[2 * R] = tot1;
        pf2[R] = tot2;
    }
}

__global__ void plan_single_kernel(uint64_t lx, uint64_t ly, PlanArea pa) {
    if (threadIdx.x == 0) {
        pa.seg1[0] = Seg{0, lx};
        pa.seg1[1] = Seg{lx, ly};
        pa.pf1[0] = 0;
        pa.pf1[1] = rev_units(lx);
        pa.pf1[2] = rev_units(lx) + rev_units(ly);
        pa.seg2[0] = Seg{0, lx + ly};
        pa.pf2[0] = 0;
        pa.pf2[1] = rev_units(lx + ly);
    }
}

// Reverse every segment of a list in place.  Block b owns the contiguous unit range
// [b*T/grid, (b+1)*T/grid) of the T units, so it locates its first segment once and
// then walks forward.
template <typename E, bool KV>
__global__ void __launch_bounds__(kRevThreads)
    reverse_segments_kernel(E *__restrict__ buf, uint32_t *__restrict__ vals,
                            const Seg *__restrict__ segs, const uint32_t *__restrict__ pf,
                            uint32_t nseg, uint64_t n_total, StatusBlock *sb) {
    if (sb != nullptr && *((volatile const unsigned int *)&sb->done)) return;
    const uint32_t total = pf[nseg];
    const uint32_t u0 = uint32_t((uint64_t(total) * blockIdx.x) / gridDim.x);
    const uint32_t u1 = uint32_t((uint64_t(total) * (blockIdx.x + 1)) / gridDim.x);
    if (u0 >= u1) return;
    // largest s with pf[s] <= u0 (pf is non-decreasing, pf[0] = 0, pf[nseg] = total > u0)
    uint32_t lo = 0, hi = nseg;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (pf[mid] <= u0)
            lo = mid;
        else
            hi = mid;
    }
    uint32_t s = lo;
    uint32_t s_end = pf[s + 1];
    Seg sg = segs[s];
    for (uint32_t u = u0; u < u1; ++u) {
        while (u >= s_end) {
            if (s + 1 >= nseg) {  // non-monotone prefix: inconsistent plan
                if (threadIdx.x == 0 && sb != nullptr) set_status(sb, IPM_ERR_DEVICE);
                return;
            }
            ++s;
            s_end = pf[s + 1];
            sg = segs[s];
        }
        // a segment outside the buffer means an inconsistent split table: record it
        // and touch nothing
        if (sg.start > n_total || sg.len > n_total - sg.start) {
            if (threadIdx.x == 0 && sb != nullptr) set_status(sb, IPM_ERR_DEVICE);
            continue;
        }
        const uint64_t half = sg.len >> 1;
        const uint64_t base = uint64_t(u - pf[s]) * kRevUnit;
        E fr[kRevItems], bk[kRevItems];
        uint32_t fv[kRevItems], bv[kRevItems];
#pragma unroll
        for (uint32_t it = 0; it < kRevItems; ++it) {
            const uint64_t p = base + it * kRevThreads + threadIdx.x;
            if (p < half) {
                fr[it] = buf[sg.start + p];
                bk[it] = buf[sg.start + sg.len - 1 - p];
                if (KV) {
                    fv[it] = vals[sg.start + p];
                    bv[it] = vals[sg.start + sg.len - 1 - p];
                }
            }
        }
#pragma unroll
        for (uint32_t it = 0; it < kRevItems; ++it) {
            const uint64_t p = base + it * kRevThreads + threadIdx.x;
            if (p < half) {
                buf[sg.start + p] = bk[it];
                buf[sg.start + sg.len - 1 - p] = fr[it];
                if (KV) {
                    vals[sg.start + p] = bv[it];
                    vals[sg.start + sg.len - 1 - p] = fv[it];
                }
            }
        }
    }
}

template <typename E>
ipm_status reverse_pass(void *buf, uint32_t *vals, const Seg *segs, const uint32_t *pf,
                        uint32_t nseg, uint64_t n, StatusBlock *sb, cudaStream_t stream) {
    const int grid = num_sms() * 8;
    if (vals)
        reverse_segments_kernel<E, true>
            <<<grid, kRevThreads, 0, stream>>>((E *)buf, vals, segs, pf, nseg, n, sb);
    else
        reverse_segments_kernel<E, false>
            <<<grid, kRevThreads, 0, stream>>>((E *)buf, nullptr, segs, pf, nseg, n, sb);
    return last_launch_status();
}

}  // namespace

size_t plan_area_bytes(uint32_t G) {
    if (G == 0) G = 1;  // room for a single exchange
    const uint64_t P = 1ull << G;
    size_t b = 0;
    b += align_up(sizeof(Seg) * 2 * (P - 1) + sizeof(Seg) * 2, 256);
    b += align_up(sizeof(uint32_t) * (2 * (P - 1) + G + 2), 256);
    b += align_up(sizeof(Seg) * (P - 1) + sizeof(Seg), 256);
    b += align_up(sizeof(uint32_t) * ((P - 1) + G + 2), 256);
    return b;
}

PlanArea plan_area_at(void *base, uint32_t G) {
    if (G == 0) G = 1;
    const uint64_t P = 1ull << G;
    char *p = static_cast<char *>(base);
    PlanArea pa;
    pa.seg1 = reinterpret_cast<Seg *>(p);
    p += align_up(sizeof(Seg) * 2 * (P - 1) + sizeof(Seg) * 2, 256);
    pa.pf1 = reinterpret_cast<uint32_t *>(p);
    p += align_up(sizeof(uint32_t) * (2 * (P - 1) + G + 2), 256);
    pa.seg2 = reinterpret_cast<Seg *>(p);
    p += align_up(sizeof(Seg) * (P - 1) + sizeof(Seg), 256);
    pa.pf2 = reinterpret_cast<uint32_t *>(p);
    return pa;
}

ipm_status launch_plan_levels(const uint64_t *split, uint64_t n, uint32_t G, PlanArea pa,
                              const StatusBlock *sb, cudaStream_t stream) {
    if (G == 0) return IPM_OK;
    plan_levels_kernel<<<G, kPlanThreads, 0, stream>>>(split, n, G, pa, sb);
    return last_launch_status();
}

ipm_status launch_plan_single(uint64_t lx, uint64_t ly, PlanArea pa, cudaStream_t stream) {
    plan_single_kernel<<<1, 32, 0, stream>>>(lx, ly, pa);
    return last_launch_status();
}

ipm_status launch_level_exchange(void *buf, uint32_t *vals, int elem_bytes, uint64_t n,
                                 uint32_t l, PlanArea pa, StatusBlock *sb,
                                 cudaStream_t stream) {
    const uint64_t R = 1ull << l;
    const Seg *s1 = pa.seg1 + seg1_base(l);
    const uint32_t *p1 = pa.pf1 + pf1_base(l);
    const Seg *s2 = pa.seg2 + seg2_base(l);
    const uint32_t *p2 = pa.pf2 + pf2_base(l);
    if (elem_bytes == 4) {
        IPM_TRY(reverse_pass<uint32_t>(buf, vals, s1, p1, uint32_t(2 * R), n, sb, stream));
        IPM_TRY(reverse_pass<uint32_t>(buf, vals, s2, p2, uint32_t(R), n, sb, stream));
    } else if (elem_bytes == 8) {
        IPM_TRY(reverse_pass<uint64_t>(buf, vals, s1, p1, uint32_t(2 * R), n, sb, stream));
        IPM_TRY(reverse_pass<uint64_t>(buf, vals, s2, p2, uint32_t(R), n, sb, stream));
    } else {
        return IPM_ERR_UNSUPPORTED_DTYPE;
    }
    return IPM_OK;
}

}  // namespace ipm
