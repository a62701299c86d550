// Division stage by one permutation (sOptMov, Alg. 2, Sec. 3.2).
//
// Once every pivot is known (the split table i_0..i_P on the diagonals
// d_k = floor(k n / 2^G)), the arranged layout A_0 B_0 A_1 B_1 ... is one fixed
// permutation of A|B, and sOptMov reaches it by moving each element once along the
// permutation's cycles.  The paper marks a moved element inside its value (which needs
// spare value range); here a bitmap of covered positions (n bits in the workspace)
// replaces the marker, so every key type keeps its full range.
//
// Position q of the arranged layout receives the element at src(q): with pair k the one
// where d_k <= q < d_{k+1}, off = q - d_k and a_k = i_{k+1} - i_k, src(q) = i_k + off when
// off < a_k (A's part), else la + (d_k - i_k) + (off - a_k) (B's part).
//
// Rounds.  Round r takes as starts the uncovered positions of the 32-position blocks
// b = r, r + S, r + 2S, ... (S = 31) and saves their elements; a warp's lanes start on
// the 32 positions of one block, and since the permutation moves runs of consecutive
// positions together, neighbouring lanes keep stepping through neighbouring positions
// and their accesses share sectors.  From each start a thread walks the cycle
// backwards: it fills q with the element at src(q), which it fills next, until src(q)
// is a start, whose saved element fills q.  The starts cut every cycle that holds one
// into disjoint segments (from a start back to the next), so no two threads touch the
// same position and the round completes exactly those cycles: a cycle is covered as a
// whole or not at all, and both ends of every step of an uncovered cycle are uncovered.
// Fixed points (the leading A and trailing B elements that stay put) are covered first.
// Once the uncovered positions fit the save area, a last round gathers the element of
// each out of place and scatters it.  Every block residue r < S serves once at most, so
// at most S + 1 rounds run; the host reads the uncovered count back between rounds.
#include "ipm_internal.h"

namespace ipm {

namespace {

constexpr uint64_t kPermStride = 31;
constexpr int kPermThreads = 256;

struct PermMap {
    const uint64_t *split;  // i_0 .. i_P
    uint64_t la, n;
    uint32_t G;
    double scale;  // 2^G / n

    // The pair k with d_k <= q < d_{k+1}: an estimate in double precision, then the
    // exact integer tests (d_k = floor(k n / 2^G), k n < 2^63) move it to the answer.
    __device__ __forceinline__ uint64_t pair_of(uint64_t q) const {
        const uint64_t P = 1ull << G;
        uint64_t k = uint64_t(double(q) * scale);
        if (k > P - 1) k = P - 1;
        while (k > 0 && ((k * n) >> G) > q) --k;
        while (k + 1 < P && (((k + 1) * n) >> G) <= q) ++k;
        return k;
    }

    // The position of A|B whose element belongs at q of the arranged layout.
    __device__ __forceinline__ uint64_t src(uint64_t q) const {
        const uint64_t k = pair_of(q);  // d_k <= q < d_{k+1}
        const uint64_t dk = (k * n) >> G;
        const uint64_t ik = split[k], ak = split[k + 1] - ik;
        const uint64_t off = q - dk;
        return off < ak ? ik + off : la + (dk - ik) + (off - ak);
    }
};

__device__ __forceinline__ bool is_covered(const uint32_t *bm, uint64_t q) {
    return (bm[q >> 5] >> (q & 31u)) & 1u;
}

__device__ __forceinline__ void cover(uint32_t *bm, uint64_t q) {
    atomicOr(bm + (q >> 5), 1u << (q & 31u));
}

__device__ __forceinline__ bool failed(const StatusBlock *sb) {
    return *((const volatile unsigned int *)&sb->status) != 0u;
}

// Round r's candidates: the positions of the blocks b = r, r + S, ... (32 per block;
// those of the last block past n are skipped).  Candidate c is lane c % 32 of the
// (c / 32)-th such block.
__host__ __device__ __forceinline__ uint64_t candidates(uint64_t n, uint64_t r) {
    const uint64_t blocks = (n + 31) / 32;
    return r < blocks ? (blocks - r + kPermStride - 1) / kPermStride * 32 : 0;
}

__device__ __forceinline__ uint64_t candidate_pos(uint64_t c, uint64_t r) {
    return ((c >> 5) * kPermStride + r) * 32 + (c & 31u);
}

// Whether position s is a round-r candidate, and its candidate index.
__device__ __forceinline__ bool candidate_of(uint64_t s, uint64_t r, uint64_t *c) {
    const uint64_t b = s >> 5;
    if (b % kPermStride != r) return false;
    *c = (b / kPermStride) * 32 + (s & 31u);
    return true;
}

// Set the bits of positions [lo, hi).
__device__ void cover_range(uint32_t *bm, uint64_t lo, uint64_t hi) {
    while (lo < hi) {
        const uint64_t w = lo >> 5, wend = (w + 1) << 5;
        const uint64_t e = hi < wend ? hi : wend;
        const uint32_t nb = uint32_t(e - lo);
        atomicOr(bm + w, (nb == 32 ? 0xffffffffu : ((1u << nb) - 1u)) << (lo & 31u));
        lo = e;
    }
}

// The table is a permutation's: i_0 = 0, i_P = la, and every pair's A and B parts are
// non-negative and inside A and B.  Anything else is reported before an element moves.
// The fixed points are covered here: pair k's A part when no B element comes before it
// (i_k = d_k), its B part when A is used up (i_{k+1} = la).
__global__ void perm_init_kernel(PermMap m, uint32_t *bm, StatusBlock *sb) {
    const uint64_t P = 1ull << m.G;
    for (uint64_t k = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < P;
         k += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t d0 = (k * m.n) >> m.G, d1 = ((k + 1) * m.n) >> m.G;
        const uint64_t i0 = m.split[k], i1 = m.split[k + 1];
        bool ok = i0 <= i1 && i1 - i0 <= d1 - d0 && i0 <= d0 && i1 <= m.la &&
                  d1 - i1 <= m.n - m.la;
        if (k == 0) ok = ok && i0 == 0;
        if (k + 1 == P) ok = ok && i1 == m.la;
        if (!ok) {
            set_status(sb, IPM_ERR_INVALID_ARG);
            continue;
        }
        if (i0 == d0) cover_range(bm, d0, d0 + (i1 - i0));
        if (i1 == m.la) cover_range(bm, d0 + (i1 - i0), d1);
    }
}

// Uncovered positions below n (the tail bits of the last word do not count).
__global__ void perm_count_kernel(const uint32_t *__restrict__ bm, uint64_t n,
                                  unsigned long long *out) {
    const uint64_t words = (n + 31) / 32;
    unsigned long long cnt = 0;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t x = ~bm[w];
        if (w + 1 == words && (n & 31u)) x &= (1u << (n & 31u)) - 1u;
        cnt += __popc(x);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31u) == 0 && cnt) atomicAdd(out, cnt);
}

// Round r, first half: save the elements of the uncovered candidates.
template <typename K, typename V>
__global__ void perm_start_kernel(const K *__restrict__ buf, const V *__restrict__ vals,
                                  const uint32_t *__restrict__ bm, uint64_t n, uint64_t r,
                                  K *__restrict__ sk, V *__restrict__ sv, StatusBlock *sb) {
    if (failed(sb)) return;
    const uint64_t C = candidates(n, r);
    for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C;
         c += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t p = candidate_pos(c, r);
        if (p >= n || is_covered(bm, p)) continue;
        sk[c] = buf[p];
        if (vals != nullptr) sv[c] = vals[p];
    }
}

// Round r, second half: each start's thread walks its segment backwards.  Only the
// thread of start p covers p, so p's bit still reads as at the round's start; every
// src(q) of a walk lies on the start's (uncovered) cycle, so a candidate residue there
// means a start whose element was saved.
template <typename K, typename V>
__global__ void perm_walk_kernel(K *__restrict__ buf, V *__restrict__ vals, uint32_t *bm,
                                 PermMap m, uint64_t r,
                                 const K *__restrict__ sk, const V *__restrict__ sv,
                                 StatusBlock *sb) {
    if (failed(sb)) return;
    const uint64_t C = candidates(m.n, r);
    for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C;
         c += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t p = candidate_pos(c, r);
        if (p >= m.n || is_covered(bm, p)) continue;
        uint64_t q = p;
        for (uint64_t step = 0;; ++step) {
            if (step >= m.n) {  // longer than any cycle: not a permutation
                set_status(sb, IPM_ERR_DEVICE);
                break;
            }
            const uint64_t s = m.src(q);
            cover(bm, q);
            uint64_t cs;
            if (candidate_of(s, r, &cs)) {
                buf[q] = sk[cs];
                if (vals != nullptr) vals[q] = sv[cs];
                break;
            }
            buf[q] = buf[s];
            if (vals != nullptr) vals[q] = vals[s];
            q = s;
        }
    }
}

// Last round, first half: every uncovered q takes a slot and keeps (q, element at
// src(q)); nothing is written to the buffer yet.
template <typename K, typename V>
__global__ void perm_gather_kernel(const K *__restrict__ buf, const V *__restrict__ vals,
                                   const uint32_t *__restrict__ bm, PermMap m,
                                   unsigned long long *slots, uint64_t cap,
                                   uint64_t *__restrict__ fpos, K *__restrict__ fk,
                                   V *__restrict__ fv, StatusBlock *sb) {
    if (failed(sb)) return;
    const uint64_t words = (m.n + 31) / 32;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t x = ~bm[w];
        if (w + 1 == words && (m.n & 31u)) x &= (1u << (m.n & 31u)) - 1u;
        if (x == 0) continue;
        const uint64_t base = atomicAdd(slots, (unsigned long long)__popc(x));
        if (base + __popc(x) > cap) {
            set_status(sb, IPM_ERR_DEVICE);
            continue;
        }
        uint64_t slot = base;
        while (x) {
            const uint64_t q = w * 32 + uint64_t(__ffs(x) - 1);
            x &= x - 1u;
            const uint64_t s = m.src(q);
            fpos[slot] = q;
            fk[slot] = buf[s];
            if (vals != nullptr) fv[slot] = vals[s];
            ++slot;
        }
    }
}

// Last round, second half: scatter the gathered elements.
template <typename K, typename V>
__global__ void perm_scatter_kernel(K *__restrict__ buf, V *__restrict__ vals,
                                    const uint64_t *__restrict__ fpos,
                                    const K *__restrict__ fk, const V *__restrict__ fv,
                                    uint64_t count, StatusBlock *sb) {
    if (failed(sb)) return;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += uint64_t(gridDim.x) * blockDim.x) {
        buf[fpos[i]] = fk[i];
        if (vals != nullptr) vals[fpos[i]] = fv[i];
    }
}

unsigned grid_for(uint64_t items) {
    const uint64_t g = (items + kPermThreads - 1) / kPermThreads;
    const uint64_t cap = uint64_t(num_sms()) * 64;
    return unsigned(g == 0 ? 1 : (g < cap ? g : cap));
}

struct PermLayout {
    size_t ctr_off, bm_off, sk_off, sv_off, fpos_off, total;
    uint64_t cap;  // saved / gathered elements per round
};

}  // namespace

static PermLayout perm_layout(uint64_t n, uint32_t kb, uint32_t vb) {
    PermLayout L;
    L.cap = candidates(n, 0);
    L.ctr_off = kStatusBytes;
    L.bm_off = L.ctr_off + 256;
    L.sk_off = L.bm_off + align_up(size_t((n + 31) / 32) * 4, 256);
    L.sv_off = L.sk_off + align_up(size_t(L.cap) * kb, 256);
    L.fpos_off = L.sv_off + align_up(size_t(L.cap) * vb, 256);
    L.total = L.fpos_off + align_up(size_t(L.cap) * 8, 256);
    return L;
}

size_t permute_workspace_bytes(uint64_t n, uint32_t kb, uint32_t vb) {
    return perm_layout(n, kb, vb).total;
}

template <typename K, typename V>
static ipm_status permute_t(void *buf_, void *vals_, uint64_t la, uint64_t lb,
                            const uint64_t *split, uint32_t G, char *w, cudaStream_t st) {
    K *buf = static_cast<K *>(buf_);
    V *vals = static_cast<V *>(vals_);
    const uint64_t n = la + lb;
    const PermLayout L = perm_layout(n, uint32_t(sizeof(K)), vals ? uint32_t(sizeof(V)) : 0u);
    StatusBlock *sb = reinterpret_cast<StatusBlock *>(w);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(w + L.ctr_off);
    uint32_t *bm = reinterpret_cast<uint32_t *>(w + L.bm_off);
    K *sk = reinterpret_cast<K *>(w + L.sk_off);
    V *sv = reinterpret_cast<V *>(w + L.sv_off);
    uint64_t *fpos = reinterpret_cast<uint64_t *>(w + L.fpos_off);
    const PermMap m{split, la, n, G, double(1ull << G) / double(n)};
    const uint64_t words = (n + 31) / 32;

    IPM_CUDA_TRY(cudaMemsetAsync(w, 0, L.bm_off + size_t(words) * 4, st));
    perm_init_kernel<<<grid_for(uint64_t(1) << G), kPermThreads, 0, st>>>(m, bm, sb);
    IPM_TRY(last_launch_status());
    for (uint64_t r = 0;; ++r) {
        IPM_CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), st));
        perm_count_kernel<<<grid_for(words), kPermThreads, 0, st>>>(bm, n, ctr);
        IPM_TRY(last_launch_status());
        unsigned long long uncovered = 0;
        unsigned int status = 0;
        IPM_CUDA_TRY(cudaMemcpyAsync(&uncovered, ctr, sizeof(uncovered),
                                     cudaMemcpyDeviceToHost, st));
        IPM_CUDA_TRY(cudaMemcpyAsync(&status, &sb->status, sizeof(status),
                                     cudaMemcpyDeviceToHost, st));
        IPM_CUDA_TRY(cudaStreamSynchronize(st));
        if (status != 0) return ipm_status(status);
        if (uncovered == 0) return IPM_OK;
        if (uncovered <= L.cap) {  // the rest out of place
            perm_gather_kernel<K, V><<<grid_for(words), kPermThreads, 0, st>>>(
                buf, vals, bm, m, ctr + 1, L.cap, fpos, sk, sv, sb);
            IPM_TRY(last_launch_status());
            perm_scatter_kernel<K, V><<<grid_for(uncovered), kPermThreads, 0, st>>>(
                buf, vals, fpos, sk, sv, uint64_t(uncovered), sb);
            IPM_TRY(last_launch_status());
            IPM_CUDA_TRY(cudaMemcpyAsync(&status, &sb->status, sizeof(status),
                                         cudaMemcpyDeviceToHost, st));
            IPM_CUDA_TRY(cudaStreamSynchronize(st));
            return ipm_status(status);
        }
        if (r >= kPermStride) return IPM_ERR_DEVICE;  // every residue served: unreachable
        const unsigned g = grid_for(candidates(n, r));
        perm_start_kernel<K, V><<<g, kPermThreads, 0, st>>>(buf, vals, bm, n, r, sk, sv, sb);
        IPM_TRY(last_launch_status());
        perm_walk_kernel<K, V><<<g, kPermThreads, 0, st>>>(buf, vals, bm, m, r, sk, sv, sb);
        IPM_TRY(last_launch_status());
    }
}

ipm_status launch_permute(void *buf, void *vals, uint32_t kb, uint32_t vb, uint64_t la,
                          uint64_t lb, const uint64_t *split, uint32_t G, void *ws,
                          cudaStream_t st) {
    char *w = static_cast<char *>(ws);
    if (kb == 4) {
        if (vb == 8) return permute_t<uint32_t, uint64_t>(buf, vals, la, lb, split, G, w, st);
        return permute_t<uint32_t, uint32_t>(buf, vb ? vals : nullptr, la, lb, split, G, w, st);
    }
    if (vb == 8) return permute_t<uint64_t, uint64_t>(buf, vals, la, lb, split, G, w, st);
    return permute_t<uint64_t, uint32_t>(buf, vb ? vals : nullptr, la, lb, split, G, w, st);
}

}  // namespace ipm
