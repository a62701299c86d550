// Batched segmented merge: the queue-preparation kernel, the workspace layout and the
// dispatch to the per-key-type kernels (ipm_batched.cuh, ipm_batched_<key>.cu).
#include "ipm_batched.cuh"

namespace ipm {

ipm_status batched_launch_i32(void *, uint32_t *, uint64_t, batched::QueueArea, uint32_t,
                              uint32_t, uint32_t, uint32_t, const ipm_segment *, uint32_t,
                              StatusBlock *, cudaStream_t);
ipm_status batched_launch_u32(void *, uint32_t *, uint64_t, batched::QueueArea, uint32_t,
                              uint32_t, uint32_t, uint32_t, const ipm_segment *, uint32_t,
                              StatusBlock *, cudaStream_t);
ipm_status batched_launch_u64(void *, uint32_t *, uint64_t, batched::QueueArea, uint32_t,
                              uint32_t, uint32_t, uint32_t, const ipm_segment *, uint32_t,
                              StatusBlock *, cudaStream_t);
ipm_status batched_launch_f32(void *, uint32_t *, uint64_t, batched::QueueArea, uint32_t,
                              uint32_t, uint32_t, uint32_t, const ipm_segment *, uint32_t,
                              StatusBlock *, cudaStream_t);
ipm_status batched_launch_i64(void *, uint32_t *, uint64_t, batched::QueueArea, uint32_t,
                              uint32_t, uint32_t, uint32_t, const ipm_segment *, uint32_t,
                              StatusBlock *, cudaStream_t);

namespace {

using namespace batched;

constexpr uint32_t kPrepThreads = 1024;

constexpr uint32_t kPrepBatch = 8;  // descriptors in flight per thread
constexpr uint32_t kPrepWarps = kPrepThreads / 32;

// Appends `q` to list[*ctr] for the active lanes: one atomic per warp.
__device__ __forceinline__ void warp_append(uint32_t *ctr, uint32_t *list, uint32_t q,
                                            bool active) {
    const uint32_t act = __ballot_sync(0xffffffffu, active);
    if (act == 0) return;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t leader = __ffs(act) - 1u;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(ctr, uint32_t(__popc(act)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (active) list[base + uint32_t(__popc(act & ((1u << lane) - 1u)))] = q;
}

// One CTA: resets the status block, writes the queue of descriptors (largest segment
// first when by_size, else table order) and lists the multi-tile segments in queue
// order; segments that leave the buffer or exceed the per-segment limit set
// IPM_ERR_INVALID_ARG.  The size order is a counting sort over 256 length buckets
// with one private histogram per warp (no contention between warps); every pass
// loads kPrepBatch descriptors per thread before using any of them.
__global__ void __launch_bounds__(kPrepThreads)
    batched_prep_kernel(const ipm_segment *__restrict__ segs, uint32_t nseg, uint32_t by_size,
                        uint64_t buf_len, uint64_t tile, uint64_t max_seg, QueueArea qa,
                        StatusBlock *sb) {
    __shared__ uint32_t hist[kPrepWarps][kOrderBuckets];  // per warp: count, then cursor
    __shared__ uint32_t total[kOrderBuckets];
    __shared__ uint32_t nmulti;
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        sb->status = 0u;
        sb->done = 0u;
        sb->exchange_bytes = 0ull;
        sb->merge_bytes = 0ull;
        sb->wait_limit_ns = 0ull;  // the batched kernels do not wait on other CTAs
        for (int q = 0; q < kNumCounters; ++q) sb->counters[q] = 0u;
        nmulti = 0;
    }
    constexpr uint32_t kStride = kPrepThreads * kPrepBatch;
    if (by_size) {
        for (uint32_t q = tid; q < kPrepWarps * kOrderBuckets; q += kPrepThreads)
            (&hist[0][0])[q] = 0u;
        __syncthreads();
        for (uint32_t t0 = 0; t0 < nseg; t0 += kStride) {
            uint64_t n[kPrepBatch];
#pragma unroll
            for (uint32_t j = 0; j < kPrepBatch; ++j) {
                const uint32_t t = t0 + j * kPrepThreads + tid;
                n[j] = t < nseg ? segs[t].len_a + segs[t].len_b : 0;
            }
#pragma unroll
            for (uint32_t j = 0; j < kPrepBatch; ++j)
                if (t0 + j * kPrepThreads + tid < nseg)
                    atomicAdd(&hist[warp][n[j] ? size_bucket(n[j]) : 0u], 1u);
        }
        __syncthreads();
        // bucket totals, then their exclusive scan from the largest bucket down
        for (uint32_t q = tid; q < kOrderBuckets; q += kPrepThreads) {
            uint32_t sum = 0;
            for (uint32_t w = 0; w < kPrepWarps; ++w) sum += hist[w][q];
            total[q] = sum;
        }
        __syncthreads();
        if (tid < 32) {
            uint32_t carry = 0;
            for (int base = int(kOrderBuckets) - 32; base >= 0; base -= 32) {
                const uint32_t q = uint32_t(base) + 31u - tid;  // descending in the chunk
                const uint32_t v = total[q];
                uint32_t x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (int(tid) >= o) x += y;
                }
                total[q] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        __syncthreads();
        // per-warp cursors: bucket start + the counts of the lower warps
        for (uint32_t q = tid; q < kOrderBuckets; q += kPrepThreads) {
            uint32_t run = total[q];
            for (uint32_t w = 0; w < kPrepWarps; ++w) {
                const uint32_t c = hist[w][q];
                hist[w][q] = run;
                run += c;
            }
        }
        __syncthreads();
    }
    // scatter into queue order (by_size) or copy (table order, listing the multi-tile
    // segments on the way)
    for (uint32_t t0 = 0; t0 < nseg; t0 += kStride) {
        ipm_segment sg[kPrepBatch];
#pragma unroll
        for (uint32_t j = 0; j < kPrepBatch; ++j) {
            const uint32_t t = t0 + j * kPrepThreads + tid;
            if (t < nseg) sg[j] = segs[t];
        }
#pragma unroll
        for (uint32_t j = 0; j < kPrepBatch; ++j) {
            const uint32_t t = t0 + j * kPrepThreads + tid;
            uint32_t cls = kSegTrivial;
            if (t < nseg) {
                const uint64_t n = sg[j].len_a + sg[j].len_b;
                const uint32_t q =
                    by_size ? atomicAdd(&hist[warp][n ? size_bucket(n) : 0u], 1u) : t;
                qa.queue[q] = sg[j];
                cls = seg_class(sg[j], buf_len, tile, max_seg);
                if (cls == kSegInvalid) set_status(sb, IPM_ERR_INVALID_ARG);  // untouched
            }
            if (!by_size) warp_append(&nmulti, qa.multi, t, cls == kSegMulti);
        }
    }
    if (by_size) {
        // list the multi-tile segments in queue order (largest first): they lead the
        // queue, so it is read back only until a bucket entirely below the tile shows
        __syncthreads();  // the queue is written (global writes of this CTA)
        __shared__ uint32_t done;
        if (tid == 0) done = 0;
        __syncthreads();
        const uint32_t first_multi_bucket = size_bucket(tile + 1);
        for (uint32_t t0 = 0; t0 < nseg && !done; t0 += kStride) {
            ipm_segment sg[kPrepBatch];
#pragma unroll
            for (uint32_t j = 0; j < kPrepBatch; ++j) {
                const uint32_t q = t0 + j * kPrepThreads + tid;
                if (q < nseg) sg[j] = qa.queue[q];
            }
            uint32_t below = 0;
#pragma unroll
            for (uint32_t j = 0; j < kPrepBatch; ++j) {
                const uint32_t q = t0 + j * kPrepThreads + tid;
                uint32_t cls = kSegTrivial;
                if (q < nseg) {
                    cls = seg_class(sg[j], buf_len, tile, max_seg);
                    const uint64_t n = sg[j].len_a + sg[j].len_b;
                    below |= (n == 0 || size_bucket(n) < first_multi_bucket) ? 1u : 0u;
                }
                warp_append(&nmulti, qa.multi, q, cls == kSegMulti);
            }
            // the queue is in descending bucket order: every segment after one whose
            // bucket lies below the first multi-tile bucket fits one tile
            if (__syncthreads_or(below) && tid == 0) done = 1;
            __syncthreads();
        }
    }
    __syncthreads();
    if (tid == 0) sb->counters[kMultiCount] = nmulti;
}

constexpr uint32_t kPrepChunk = 2048;  // descriptors per chunk of the many-CTA preparation

// Chunk c's length-bucket counts into s_cnt (the block; s_cnt zeroed here).
__device__ __forceinline__ void chunk_counts(const ipm_segment *__restrict__ segs,
                                             uint32_t nseg, uint32_t c, uint32_t *s_cnt) {
    const uint32_t tid = threadIdx.x;
    for (uint32_t q = tid; q < kOrderBuckets; q += kPrepThreads) s_cnt[q] = 0u;
    __syncthreads();
    const uint32_t i0 = c * kPrepChunk;
    const uint32_t i1 = nseg - i0 < kPrepChunk ? nseg : i0 + kPrepChunk;
    for (uint32_t i = i0 + tid; i < i1; i += kPrepThreads) {
        const uint64_t n = segs[i].len_a + segs[i].len_b;
        atomicAdd(&s_cnt[n ? size_bucket(n) : 0u], 1u);
    }
    __syncthreads();
}

// The size-ordered preparation by many CTAs (the grid is at most one CTA per SM, so all
// are resident and the waits on each other end).  The launcher has zeroed the status
// block, its counters and the global bucket counts and cursors.  Each CTA takes chunks
// blockIdx.x, blockIdx.x + gridDim.x, ... of kPrepChunk descriptors: it adds a chunk's
// bucket counts to the global ones; once every chunk is counted, it takes the chunk's
// slots in every bucket (bucket starts from the global counts, largest bucket first)
// and scatters the chunk's descriptors there, checking each segment.  CTA 0 then waits
// for every chunk to be scattered and lists the multi-tile segments, which lead the
// queue, as the one-CTA preparation does.  Waits are bounded (IPM_ERR_TIMEOUT).
__global__ void __launch_bounds__(kPrepThreads)
    batched_prep_multi_kernel(const ipm_segment *__restrict__ segs, uint32_t nseg,
                              uint64_t buf_len, uint64_t tile, uint64_t max_seg, QueueArea qa,
                              StatusBlock *sb) {
    __shared__ uint32_t s_cnt[kOrderBuckets], s_base[kOrderBuckets], s_slot[kOrderBuckets];
    __shared__ int s_ok;
    __shared__ uint32_t nmulti;
    const uint32_t tid = threadIdx.x;
    const uint32_t C = (nseg + kPrepChunk - 1) / kPrepChunk;
    const unsigned long long lim = wait_limit(sb);
    for (uint32_t c = blockIdx.x; c < C; c += gridDim.x) {
        chunk_counts(segs, nseg, c, s_cnt);
        for (uint32_t q = tid; q < kOrderBuckets; q += kPrepThreads)
            if (s_cnt[q]) atomicAdd(&qa.hist[q], s_cnt[q]);
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(&sb->counters[kHistDone], 1u);
    }
    if (tid == 0) s_ok = wait_at_least(&sb->counters[kHistDone], C, lim);
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) set_status(sb, IPM_ERR_TIMEOUT);
        return;
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
    for (uint32_t c = blockIdx.x; c < C; c += gridDim.x) {
        chunk_counts(segs, nseg, c, s_cnt);
        // this chunk's slots in every bucket
        for (uint32_t q = tid; q < kOrderBuckets; q += kPrepThreads)
            s_slot[q] = s_cnt[q] ? s_base[q] + atomicAdd(&qa.cursor[q], s_cnt[q]) : 0u;
        __syncthreads();
        const uint32_t i0 = c * kPrepChunk;
        const uint32_t i1 = nseg - i0 < kPrepChunk ? nseg : i0 + kPrepChunk;
        for (uint32_t i = i0 + tid; i < i1; i += kPrepThreads) {
            const ipm_segment sg = segs[i];
            const uint64_t n = sg.len_a + sg.len_b;
            qa.queue[atomicAdd(&s_slot[n ? size_bucket(n) : 0u], 1u)] = sg;
            if (seg_class(sg, buf_len, tile, max_seg) == kSegInvalid)
                set_status(sb, IPM_ERR_INVALID_ARG);  // left untouched
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(&sb->counters[kScatterDone], 1u);
    }
    if (blockIdx.x != 0) return;
    if (tid == 0) {
        s_ok = wait_at_least(&sb->counters[kScatterDone], C, lim);
        nmulti = 0;
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) set_status(sb, IPM_ERR_TIMEOUT);
        return;
    }
    // the multi-tile segments lead the queue (descending buckets): read it back, through
    // L2 (other CTAs wrote it), until a bucket entirely below the tile shows
    __shared__ uint32_t done;
    if (tid == 0) done = 0;
    __syncthreads();
    const uint32_t first_multi_bucket = size_bucket(tile + 1);
    constexpr uint32_t kStride = kPrepThreads * kPrepBatch;
    for (uint32_t t0 = 0; t0 < nseg && !done; t0 += kStride) {
        ipm_segment sg[kPrepBatch];
#pragma unroll
        for (uint32_t j = 0; j < kPrepBatch; ++j) {
            const uint32_t q = t0 + j * kPrepThreads + tid;
            if (q < nseg) {
                const unsigned long long *e =
                    reinterpret_cast<const unsigned long long *>(&qa.queue[q]);
                sg[j].offset = __ldcg(e);
                sg[j].len_a = __ldcg(e + 1);
                sg[j].len_b = __ldcg(e + 2);
            }
        }
        uint32_t below = 0;
#pragma unroll
        for (uint32_t j = 0; j < kPrepBatch; ++j) {
            const uint32_t q = t0 + j * kPrepThreads + tid;
            uint32_t cls = kSegTrivial;
            if (q < nseg) {
                cls = seg_class(sg[j], buf_len, tile, max_seg);
                const uint64_t n = sg[j].len_a + sg[j].len_b;
                below |= (n == 0 || size_bucket(n) < first_multi_bucket) ? 1u : 0u;
            }
            warp_append(&nmulti, qa.multi, q, cls == kSegMulti);
        }
        if (__syncthreads_or(below) && tid == 0) done = 1;
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) sb->counters[kMultiCount] = nmulti;
}

}  // namespace

uint64_t batched_tile(ipm_dtype key, bool with_values, uint32_t variant) {
    switch (key) {
    case IPM_INT32:
    case IPM_UINT32:
    case IPM_FLOAT32:
        return with_values ? tile_t<int32_t, true>(variant) : tile_t<int32_t, false>(variant);
    case IPM_UINT64:
    case IPM_INT64:
        return with_values ? tile_t<uint64_t, true>(variant)
                           : tile_t<uint64_t, false>(variant);
    }
    return 0;
}

uint64_t batched_max_segment(ipm_dtype key, bool with_values, uint32_t variant) {
    return uint64_t(kMaxPairs) * batched_tile(key, with_values, variant);
}

// Workspace layout: status block | bucket counts and cursors (one-launch form) | queue |
// multi | soff | split pool.  The pool holds every multi-tile segment's P + 1 splits;
// P < 2 n / tile, so for segments that do not overlap 2 (buf_len / tile + 1) + nseg
// entries suffice.
BatchedLayout batched_layout(uint64_t buf_len, uint32_t nseg, uint64_t tile) {
    BatchedLayout L;
    L.hist_off = kStatusBytes;
    L.queue_off = L.hist_off + 2 * sizeof(uint32_t) * kOrderBuckets;
    L.multi_off = L.queue_off + align_up(sizeof(ipm_segment) * size_t(nseg), 256);
    L.soff_off = L.multi_off + align_up(sizeof(uint32_t) * size_t(nseg), 256);
    L.pool_off = L.soff_off + align_up(sizeof(uint32_t) * size_t(nseg), 256);
    L.pool_cap = 2 * (buf_len / tile + 1) + uint64_t(nseg);
    L.total = L.pool_off + align_up(sizeof(uint64_t) * size_t(L.pool_cap), 256);
    return L;
}

ipm_status launch_batched(void *buf, uint32_t *vals, uint64_t buf_len, ipm_dtype key,
                          const ipm_segment *segs, uint32_t nseg, void *ws,
                          const BatchedLayout &L, uint32_t by_size, uint32_t variant,
                          uint32_t ctas_per_sm, uint32_t one_launch, cudaStream_t stream) {
    char *w = static_cast<char *>(ws);
    StatusBlock *sb = reinterpret_cast<StatusBlock *>(w);
    QueueArea qa;
    qa.queue = reinterpret_cast<ipm_segment *>(w + L.queue_off);
    qa.multi = reinterpret_cast<uint32_t *>(w + L.multi_off);
    qa.soff = reinterpret_cast<uint32_t *>(w + L.soff_off);
    qa.pool = reinterpret_cast<uint64_t *>(w + L.pool_off);
    qa.pool_cap = L.pool_cap;
    qa.hist = reinterpret_cast<uint32_t *>(w + L.hist_off);
    qa.cursor = qa.hist + kOrderBuckets;
    const uint64_t tile = batched_tile(key, vals != nullptr, variant);
    if (one_launch) {
        // the status block, its counters and the bucket counts start at zero; every other
        // area is written before it is read
        IPM_CUDA_TRY(cudaMemsetAsync(w, 0, L.queue_off, stream));
    } else if (by_size && nseg > 0) {
        // the size order prepared by up to one CTA per SM (the same zeroed start)
        IPM_CUDA_TRY(cudaMemsetAsync(w, 0, L.queue_off, stream));
        const uint32_t chunks = (nseg + kPrepChunk - 1) / kPrepChunk;
        const uint32_t sms = uint32_t(num_sms());
        batched_prep_multi_kernel<<<chunks < sms ? chunks : sms, kPrepThreads, 0, stream>>>(
            segs, nseg, buf_len, tile, batched_max_segment(key, vals != nullptr, variant), qa,
            sb);
        IPM_TRY(last_launch_status());
    } else {
        batched_prep_kernel<<<1, kPrepThreads, 0, stream>>>(
            segs, nseg, by_size, buf_len, tile,
            batched_max_segment(key, vals != nullptr, variant), qa, sb);
        IPM_TRY(last_launch_status());
    }
    switch (key) {
    case IPM_INT32:
        return batched_launch_i32(buf, vals, buf_len, qa, nseg, variant, ctas_per_sm,
                                  one_launch, segs, by_size, sb, stream);
    case IPM_UINT32:
        return batched_launch_u32(buf, vals, buf_len, qa, nseg, variant, ctas_per_sm,
                                  one_launch, segs, by_size, sb, stream);
    case IPM_UINT64:
        return batched_launch_u64(buf, vals, buf_len, qa, nseg, variant, ctas_per_sm,
                                  one_launch, segs, by_size, sb, stream);
    case IPM_FLOAT32:
        return batched_launch_f32(buf, vals, buf_len, qa, nseg, variant, ctas_per_sm,
                                  one_launch, segs, by_size, sb, stream);
    case IPM_INT64:
        return batched_launch_i64(buf, vals, buf_len, qa, nseg, variant, ctas_per_sm,
                                  one_launch, segs, by_size, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
