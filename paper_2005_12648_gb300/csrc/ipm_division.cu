// The division of Alg. 3 (sRecPar, Sec. 3.3) without data movement: the pair
// boundaries its recursion reaches, for the balance comparison of Sec. 4 between
// FindMedian (Alg. 1, Sec. 3.1) and the optimal split.
//
// Level l has 2^l regions; region m spans boundaries k0 = m P / 2^l and k1 = k0 + P / 2^l
// and holds A[ia[k0], ia[k1]) and B[jb[k0], jb[k1]).  Its pivot (pA, pB) goes to the
// boundary halfway between.  One launch per level, one thread per region.
#include "ipm_internal.h"

namespace ipm {
namespace {

// FindMedian, Alg. 1, in this reading of the listing: the two corner cases first (all of
// A before B: (|A|, 0); all of A after B: (0, |B|)); then each iteration takes the two
// midpoints, returns them when the keys are equal, and otherwise moves the bound the
// listing moves (the side whose midpoint key is smaller is cut from below when the part
// before the midpoints holds fewer elements than the part after them, the other side is
// cut from above otherwise); when a search interval empties, the midpoints of the final
// intervals are the pivot.
template <typename K>
__device__ void findmedian_pivot(const K *a, uint64_t la, const K *b, uint64_t lb,
                                 uint64_t &pa, uint64_t &pb) {
    if (key_le(a[la - 1], b[0])) {
        pa = la;
        pb = 0;
        return;
    }
    if (!key_le(a[0], b[lb - 1])) {
        pa = 0;
        pb = lb;
        return;
    }
    uint64_t lo_a = 0, hi_a = la, lo_b = 0, hi_b = lb;
    while (lo_a < hi_a && lo_b < hi_b) {
        const uint64_t ma = lo_a + (hi_a - lo_a) / 2;
        const uint64_t mb = lo_b + (hi_b - lo_b) / 2;
        const K x = a[ma], y = b[mb];
        if (x == y) {
            pa = ma;
            pb = mb;
            return;
        }
        const bool before_smaller = ma + mb < (la - ma) + (lb - mb);
        if (x < y) {
            if (before_smaller)
                lo_a = ma + 1;
            else
                hi_b = mb;
        } else {
            if (before_smaller)
                lo_b = mb + 1;
            else
                hi_a = ma;
        }
    }
    pa = lo_a + (hi_a - lo_a) / 2;
    pb = lo_b + (hi_b - lo_b) / 2;
}

// The exact stable split on diagonal d: the number of A elements among the first d
// outputs of the stable merge (the smallest i with A[i] after B[d-1-i]).
template <typename K>
__device__ uint64_t half_split(const K *a, uint64_t la, const K *b, uint64_t lb, uint64_t d) {
    uint64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    while (lo < hi) {
        const uint64_t i = lo + (hi - lo) / 2;
        if (key_le(a[i], b[d - 1 - i]))
            lo = i + 1;
        else
            hi = i;
    }
    return lo;
}

__global__ void division_init_kernel(uint64_t *ia, uint64_t *jb, uint64_t P, uint64_t la,
                                     uint64_t lb) {
    ia[0] = 0;
    jb[0] = 0;
    ia[P] = la;
    jb[P] = lb;
}

template <typename K>
__global__ void division_level_kernel(const K *__restrict__ A, const K *__restrict__ B,
                                      uint64_t *ia, uint64_t *jb, uint64_t P, uint32_t l,
                                      uint32_t kind) {
    const uint64_t m = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= (1ull << l)) return;
    const uint64_t step = P >> l, k0 = m * step, k1 = k0 + step, mid = k0 + step / 2;
    const uint64_t a0 = ia[k0], b0 = jb[k0];
    const uint64_t ra = ia[k1] - a0, rb = jb[k1] - b0;
    uint64_t pa, pb;
    if (ra == 0 || rb == 0) {  // one-sided: left whole (Alg. 3 does not divide it)
        pa = ra;
        pb = rb;
    } else if (kind == IPM_SPLIT_EXACT) {
        const uint64_t d = (ra + rb) / 2;
        pa = half_split(A + a0, ra, B + b0, rb, d);
        pb = d - pa;
    } else {
        findmedian_pivot(A + a0, ra, B + b0, rb, pa, pb);
    }
    ia[mid] = a0 + pa;
    jb[mid] = b0 + pb;
}

template <typename K>
ipm_status division_t(const void *buf, uint64_t la, uint64_t lb, uint32_t depth,
                      uint32_t kind, uint64_t *ia, uint64_t *jb, cudaStream_t stream) {
    const K *A = static_cast<const K *>(buf);
    const uint64_t P = 1ull << depth;
    division_init_kernel<<<1, 1, 0, stream>>>(ia, jb, P, la, lb);
    IPM_TRY(last_launch_status());
    for (uint32_t l = 0; l < depth; ++l) {
        const uint64_t regions = 1ull << l;
        const unsigned threads = regions < 256 ? unsigned(regions) : 256u;
        const unsigned blocks = unsigned((regions + threads - 1) / threads);
        division_level_kernel<K><<<blocks, threads, 0, stream>>>(A, A + la, ia, jb, P, l, kind);
        IPM_TRY(last_launch_status());
    }
    return IPM_OK;
}

}  // namespace

ipm_status launch_division(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                           uint32_t depth, uint32_t kind, uint64_t *ia, uint64_t *jb,
                           cudaStream_t stream) {
    switch (key) {
    case IPM_INT32: return division_t<int32_t>(buf, la, lb, depth, kind, ia, jb, stream);
    case IPM_UINT32: return division_t<uint32_t>(buf, la, lb, depth, kind, ia, jb, stream);
    case IPM_UINT64: return division_t<uint64_t>(buf, la, lb, depth, kind, ia, jb, stream);
    case IPM_INT64: return division_t<int64_t>(buf, la, lb, depth, kind, ia, jb, stream);
    case IPM_FLOAT32: return division_t<float>(buf, la, lb, depth, kind, ia, jb, stream);
    default: return IPM_ERR_UNSUPPORTED_DTYPE;
    }
}

}  // namespace ipm
