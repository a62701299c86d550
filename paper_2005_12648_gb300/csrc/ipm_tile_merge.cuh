// Shared-memory merge of one pair (A_k, B_k) in place: the per-thread
// std::inplace_merge of Alg. 2/3, done here by one CTA.  Used by the per-pair merge
// kernel of the plain path and by the batched kernel.
//
// The pair [A (a) | B (c - a)] starting at g is
//   1. staged in shared memory: the 16-byte-aligned body with one TMA bulk copy
//      (cp.async.bulk, completion on an mbarrier), the unaligned head and tail
//      (< 16 bytes each) with plain loads;
//   2. merged (merge_staged): each thread owns E consecutive outputs, finds its diagonal
//      of the pair's merge path by binary search, takes E sequential merge steps into
//      registers and writes them back over the staged copy;
//   3. stored: the body with one TMA bulk store, head and tail with plain stores.
#pragma once

#include "ipm_common.cuh"
#include "ipm_tma.cuh"

namespace ipm {

// V: the payload type (4- or 8-byte; moved, never compared).
template <typename K, bool KV, int THREADS, int E, typename V = uint32_t>
struct TileShape {
    static constexpr int kTile = THREADS * E;
    static constexpr int kKeyPad = 16 / int(sizeof(K));
    static constexpr int kValPad = 16 / int(sizeof(V));
    static constexpr size_t kKeyBytes = ((size_t(kTile + kKeyPad) * sizeof(K)) + 15) / 16 * 16;
    static constexpr size_t kValBytes =
        KV ? ((size_t(kTile + kValPad) * sizeof(V) + 15) / 16 * 16) : 0;
    static constexpr size_t kSmem = 128 + kKeyBytes + kValBytes;
};

enum : int { kPairAbort = 0, kPairMerged = 1, kPairInOrder = 2, kPairTrivial = 3 };

// Merge of two staged runs A = sk[0, a) and B = sk[bo, bo + b) (payloads sv[0, a) and
// sv[bov, bov + b) when KV; bo, bov >= a) by the whole CTA with EC outputs per thread (EC odd,
// THREADS * EC >= a + b; a, b >= 1 unless MAY_BE_EMPTY, which makes an empty run a move
// of the other): each thread finds its diagonal of the merge path by binary search
// (stable predicate A[m] <= B[d-1-m]), takes EC branch-free merge steps into registers,
// and, after a barrier, writes them to dk[0, a + b) (dv for payloads), which may overlap
// the sources (EC odd keeps the blocked writes conflict-free across banks).  Both runs
// are addressed from one base so the merge loop keeps a single pointer.
// The merge-path part of merge_two for one thread: its EC outputs starting at output
// position tid * EC, into registers: the keys (ok) and, for KV, the staged index of
// each output (oi: A's at < a, B's at >= bo).  Threads past the end leave them unset.
template <typename K, bool KV, int THREADS, int EC, bool MAY_BE_EMPTY = false>
__device__ __forceinline__ void merge_path_regs(const K *sk, uint32_t a, uint32_t bo, uint32_t b,
                                                K (&ok)[EC], uint32_t (&oi)[KV ? EC : 1]) {
    const uint32_t c = a + b;
    const uint32_t dt = threadIdx.x * uint32_t(EC);
    if (dt < c) {
        uint32_t lo = dt > b ? dt - b : 0u;
        uint32_t hi = dt < a ? dt : a;
        while (lo < hi) {
            const uint32_t m = (lo + hi) >> 1;
            if (key_le(sk[m], sk[bo + dt - 1 - m]))
                lo = m + 1;
            else
                hi = m;
        }
        // Branch-free steps.  Each run keeps its current key and the two after it in
        // registers (indices clamped to the run); the taken side shifts its window and
        // loads the key three ahead, which is needed two steps later at the earliest, so
        // the shared-memory latency stays off the compare chain.  An exhausted (or empty)
        // side is never taken again, so its stale keys do not matter; an empty run reads
        // (and ignores) the first word of its staging area.
        // ia: A's position; jb: B's position in sk (B ends at eb = bo + b)
        uint32_t ia = lo, jb = bo + (dt - lo);
        const uint32_t eb = bo + b;
        const uint32_t la1 = MAY_BE_EMPTY && a == 0 ? 0u : a - 1;
        const uint32_t lb1 = MAY_BE_EMPTY && b == 0 ? bo : eb - 1;
        K va0 = sk[ia < la1 ? ia : la1], va1 = sk[ia + 1 < la1 ? ia + 1 : la1];
        K va2 = sk[ia + 2 < la1 ? ia + 2 : la1];
        K vb0 = sk[jb < lb1 ? jb : lb1], vb1 = sk[jb + 1 < lb1 ? jb + 1 : lb1];
        K vb2 = sk[jb + 2 < lb1 ? jb + 2 : lb1];
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const bool takeA = (jb >= eb) || (ia < a && key_le(va0, vb0));
            if (KV)
                oi[KV ? e : 0] = takeA ? ia : jb;  // an index of sk (A: < a, B: >= bo)
            else
                ok[e] = takeA ? va0 : vb0;
            const uint32_t src = takeA ? (ia + 3 < la1 ? ia + 3 : la1)
                                       : (jb + 3 < lb1 ? jb + 3 : lb1);
            const K nv = sk[src];
            ia += takeA ? 1u : 0u;
            jb += takeA ? 0u : 1u;
            va0 = takeA ? va1 : va0;
            va1 = takeA ? va2 : va1;
            va2 = takeA ? nv : va2;
            vb0 = takeA ? vb0 : vb1;
            vb1 = takeA ? vb1 : vb2;
            vb2 = takeA ? vb2 : nv;
        }
    }
}

template <typename K, bool KV, int THREADS, int EC, bool MAY_BE_EMPTY = false,
          typename V = uint32_t>
__device__ __forceinline__ void merge_two(const K *sk, const V *sv, uint32_t a,
                                          uint32_t bo, uint32_t bov, uint32_t b, K *dk,
                                          V *dv) {
    const uint32_t c = a + b;
    const uint32_t dt = threadIdx.x * uint32_t(EC);
    K ok[EC];
    uint32_t oi[KV ? EC : 1];
    merge_path_regs<K, KV, THREADS, EC, MAY_BE_EMPTY>(sk, a, bo, b, ok, oi);
    V ov[KV ? EC : 1];
    if (KV && dt < c) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const uint32_t q = (dt + e < c) ? oi[KV ? e : 0] : 0u;
            ok[e] = sk[q];
            ov[KV ? e : 0] = sv[q < a ? q : bov + (q - bo)];
        }
    }
    __syncthreads();
    if (dt < c) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            if (dt + e < c) {
                dk[dt + e] = ok[e];
                if (KV) dv[dt + e] = ov[KV ? e : 0];
            }
        }
    }
}

// Step 2 of merge_pair_smem: the staged pair tk[0, c) = [A (a) | B (c - a)] merged onto
// itself (a, c - a >= 1) by the whole CTA with EC outputs per thread, the same
// algorithm as merge_two for the contiguous layout (A and B as two pointers).
template <typename K, bool KV, int THREADS, int EC, typename V = uint32_t>
__device__ __forceinline__ void merge_staged(K *tk, V *tv, uint32_t a, uint32_t c) {
    const uint32_t tid = threadIdx.x;
    const uint32_t b = c - a;
    const K *sA = tk;
    const K *sB = tk + a;
    const uint32_t dt = tid * uint32_t(EC);
    K ok[EC];
    uint32_t oi[KV ? EC : 1];
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
        const uint32_t la1 = a - 1, lb1 = b - 1;
        K va0 = sA[ia < la1 ? ia : la1], va1 = sA[ia + 1 < la1 ? ia + 1 : la1];
        K va2 = sA[ia + 2 < la1 ? ia + 2 : la1];
        K vb0 = sB[ib < lb1 ? ib : lb1], vb1 = sB[ib + 1 < lb1 ? ib + 1 : lb1];
        K vb2 = sB[ib + 2 < lb1 ? ib + 2 : lb1];
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const bool takeA = (ib >= b) || (ia < a && key_le(va0, vb0));
            if (KV)
                oi[KV ? e : 0] = takeA ? ia : a + ib;
            else
                ok[e] = takeA ? va0 : vb0;
            const uint32_t src = takeA ? (ia + 3 < la1 ? ia + 3 : la1)
                                       : a + (ib + 3 < lb1 ? ib + 3 : lb1);
            const K nv = tk[src];
            ia += takeA ? 1u : 0u;
            ib += takeA ? 0u : 1u;
            va0 = takeA ? va1 : va0;
            va1 = takeA ? va2 : va1;
            va2 = takeA ? nv : va2;
            vb0 = takeA ? vb0 : vb1;
            vb1 = takeA ? vb1 : vb2;
            vb2 = takeA ? vb2 : nv;
        }
    }
    V ov[KV ? EC : 1];
    if (KV && dt < c) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const uint32_t src = (dt + e < c) ? oi[KV ? e : 0] : 0u;
            ok[e] = tk[src];
            ov[KV ? e : 0] = tv[src];
        }
    }
    __syncthreads();
    if (dt < c) {
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            if (dt + e < c) {
                tk[dt + e] = ok[e];
                if (KV) tv[dt + e] = ov[KV ? e : 0];
            }
        }
    }
}

// Merges the pair at g (payload at gv when KV) through skeys/svals.  All THREADS
// threads of the CTA call it together.  c <= THREADS * E, a <= c.  Returns
//   kPairTrivial  one run is empty: nothing to move, nothing read;
//   kPairInOrder  A[last] <= B[0] on the staged copy (the early exit of Alg. 2/3):
//                 read, nothing written;
//   kPairMerged   merged and written back;
//   kPairAbort    the staging copy did not complete within the wait limit (status set
//                 to IPM_ERR_TIMEOUT); the pair is left untouched.
// On return the shared buffers are free again (the bulk store has finished reading
// them).
template <typename K, bool KV, int THREADS, int E, typename V = uint32_t>
__device__ __forceinline__ int merge_pair_smem(K *g, V *gv, uint32_t a, uint32_t c,
                                               K *skeys, V *svals, uint64_t *mbar,
                                               uint32_t &parity, int &abort_flag,
                                               StatusBlock *sb) {
    const uint32_t tid = threadIdx.x;
    const uint32_t b = c - a;
    if (a == 0 || b == 0) return kPairTrivial;
    const Geo<int(sizeof(K))> gk(g, c);
    const Geo<int(sizeof(V))> gvv(KV ? (const void *)gv : (const void *)g, KV ? c : 0u);
    K *tk = skeys + gk.off;   // staged keys: tk[0, c)
    V *tv = svals + gvv.off;  // staged values: tv[0, c)

    // ---- 1. stage
    if (tid == 0) {
        const uint32_t kb = gk.body * uint32_t(sizeof(K));
        const uint32_t vb = KV ? gvv.body * uint32_t(sizeof(V)) : 0u;
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
        return kPairAbort;
    }
    if (key_le(tk[a - 1], tk[a])) {  // already in order: nothing to write
        __syncthreads();             // every thread has read tk before it is reused
        return kPairInOrder;
    }

    // ---- 2. merge in shared memory
    merge_staged<K, KV, THREADS, E, V>(tk, tv, a, c);

    // ---- 3. store the merged copy
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
        const uint32_t kb = gk.body * uint32_t(sizeof(K));
        const uint32_t vb = KV ? gvv.body * uint32_t(sizeof(V)) : 0u;
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
    return kPairMerged;
}

}  // namespace ipm
