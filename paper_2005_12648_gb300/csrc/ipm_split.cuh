// Exact stable merge-path split of one diagonal by one warp (Sec. 3.1).
//
// For a diagonal d (an output count), the stable split i is the number of A elements
// among the first d keys of the stable merge; A[m] is among them exactly when
// A[m] <= B[d-1-m].  That predicate is true for m < i and false for m >= i, so one
// warp brackets i with 32 evenly spaced probes per step: the ballot of the probes is
// a prefix of ones, its popcount locates the bracket, and the range shrinks ~33x per
// step (log_33 of the run length dependent steps instead of log_2).
#pragma once

#include "ipm_common.cuh"

namespace ipm {

// Read-only-path load (the runs are not written while the splits are computed) or a
// plain coherent load (NC = false: the same launch later rewrites the buffer).
template <bool NC, typename K>
__device__ __forceinline__ K split_load(const K *p) {
    if (NC) return __ldg(p);
    return *p;
}

// The split i on diagonal d, 0 <= d <= la + lb; every lane of the (full) warp calls it
// with the same arguments and receives the same i.  lo/hi may narrow the search when a
// bracket is already known (lo <= i <= hi); pass the trivial bracket otherwise.  With
// COUNT, *rounds and *probes receive the dependent probe rounds and the predicate
// evaluations the search made.
template <bool NC, bool COUNT = false, typename K>
__device__ __forceinline__ uint64_t warp_split_bracket(const K *A, const K *B, uint64_t d,
                                                       uint64_t lo, uint64_t hi,
                                                       uint32_t *rounds = nullptr,
                                                       uint32_t *probes = nullptr) {
    const unsigned lane = threadIdx.x & 31u;
    uint32_t nr = 0, np = 0;
    while (hi - lo > 32) {
        const uint64_t R = hi - lo;
        const uint64_t m = lo + (R * (lane + 1)) / 33;  // strictly increasing, in [lo,hi)
        const bool p = key_le(split_load<NC>(A + m), split_load<NC>(B + (d - 1 - m)));
        const unsigned bal = __ballot_sync(0xffffffffu, p);
        const int c = __popc(bal);
        const uint64_t m_lo = __shfl_sync(0xffffffffu, m, c > 0 ? c - 1 : 0);
        const uint64_t m_hi = __shfl_sync(0xffffffffu, m, c < 32 ? c : 31);
        const uint64_t nlo = c > 0 ? m_lo + 1 : lo;
        const uint64_t nhi = c < 32 ? m_hi : hi;
        lo = nlo;
        hi = nhi;
        if (COUNT) {
            ++nr;
            np += 32;
        }
    }
    const uint64_t R = hi - lo;
    bool p = false;
    if (lane < R) {
        const uint64_t m = lo + lane;
        p = key_le(split_load<NC>(A + m), split_load<NC>(B + (d - 1 - m)));
    }
    const int c = __popc(__ballot_sync(0xffffffffu, p));
    if (COUNT) {
        nr += R > 0 ? 1u : 0u;
        np += uint32_t(R);
        *rounds = nr;
        *probes = np;
    }
    return lo + uint64_t(c);
}

template <bool NC, typename K>
__device__ __forceinline__ uint64_t warp_split(const K *A, uint64_t la, const K *B,
                                               uint64_t lb, uint64_t d) {
    return warp_split_bracket<NC>(A, B, d, d > lb ? d - lb : 0, d < la ? d : la);
}

}  // namespace ipm
