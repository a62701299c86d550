// Division stage (Alg. 3): level-by-level exchange of the two middle blocks, one pass.
// (All data loads use ld.global.cg: data written by other SMs during the launch must
// come from L2, and every element is read once per level, so L1 gains nothing.)
//
// With P = 2^G pairs and the split table i_k on d_k = floor(k*n/P), the level-l pair r
// (final pairs [r*2^{G-l}, (r+1)*2^{G-l})) holds A[i_lo, i_hi) | B[j_lo, j_hi) at d_lo
// when level l starts.  Its mid diagonal splits it into A_lo A_hi | B_lo B_hi and the
// middle [X|Y] = [A_hi | B_lo] at s = d_lo + i_mid - i_lo becomes [Y|X] (Sec. 3.4),
// giving A_lo B_lo | A_hi B_hi.  Every exchange of a level is independent.
//
// Each exchange is cut into items (ipm_exchange.cuh).  One persistent kernel per
// level hands the items of all the level's exchanges to CTAs in a fixed order through
// an atomic ticket.  The closed-form PAIR / SHIFT phases move data in place with one
// read and one write per element, so a tile may write only after the tiles (and stash
// holders) whose inputs lie under its outputs have read them: every item publishes
// "my reads are done" in a flag, and waits only on items with smaller tickets (a
// holder, which writes its stash last, also waits on the later tiles of its own
// exchange; at most max_holders such CTAs exist per exchange, fewer than the
// resident CTAs, so the tiles always find a CTA).  Consecutive phases of one exchange
// (LS steps) are ordered by a per-exchange completion counter.  Every wait is bounded
// in time; on expiry the kernel records IPM_ERR_TIMEOUT and all CTAs leave.
#include "ipm_exchange.cuh"
#include "ipm_internal.h"

namespace ipm {

namespace {

constexpr uint32_t kPlanThreads = 1024;

struct RotPlan {
    uint64_t s, a, b;
};

__device__ uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t *total) {
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
        warp_sums[lane] = w;
    }
    __syncthreads();
    const uint32_t warp_excl = wid ? warp_sums[wid - 1] : 0u;
    *total = warp_sums[31];
    __syncthreads();
    return warp_excl + x - v;
}

__device__ __forceinline__ RotPlan level_rotation(const uint64_t *split, uint64_t n,
                                                  uint32_t G, uint32_t l, uint64_t r) {
    const uint64_t k_lo = r << (G - l);
    const uint64_t k_mid = k_lo + (1ull << (G - l - 1));
    const uint64_t k_hi = k_lo + (1ull << (G - l));
    const uint64_t d_lo = (k_lo * n) >> G, d_mid = (k_mid * n) >> G;
    const uint64_t i_lo = split[k_lo], i_mid = split[k_mid], i_hi = split[k_hi];
    RotPlan q;
    q.s = d_lo + (i_mid - i_lo);
    q.a = i_hi - i_mid;
    q.b = (d_mid - i_mid) - (d_lo - i_lo);
    return q;
}

// One block per level: the exchanges of level l, their item prefix and (added into
// the status block) their algorithmic bytes.
__global__ void __launch_bounds__(kPlanThreads)
    xplan_levels_kernel(const uint64_t *__restrict__ split, uint64_t n, uint32_t G,
                        XPlanArea pa, XParams prm, uint32_t elem, StatusBlock *sb) {
    if (sb != nullptr && *((volatile const unsigned int *)&sb->done)) return;
    const uint32_t l = blockIdx.x;
    const uint64_t R = 1ull << l;
    RotPlan *plans = reinterpret_cast<RotPlan *>(pa.plans) + (R - 1);
    uint32_t *pf = pa.item_pf + (R - 1) + l;
    const uint64_t per = (R + kPlanThreads - 1) / kPlanThreads;
    const uint64_t r0 = per * threadIdx.x;
    const uint64_t r1 = r0 + per < R ? r0 + per : R;
    uint32_t items = 0;
    unsigned long long bytes = 0;
    for (uint64_t r = r0; r < r1; ++r) {
        RotPlan q = level_rotation(split, n, G, l, r);
        uint64_t it = 0, by = 0;
        x_count(prm, q.s, q.a, q.b, elem, it, by);
        items += uint32_t(it);
        bytes += by;
    }
    uint32_t total;
    uint32_t e = block_exclusive_scan_u32(items, &total);
    for (uint64_t r = r0; r < r1; ++r) {
        RotPlan q = level_rotation(split, n, G, l, r);
        uint64_t it = 0, by = 0;
        x_count(prm, q.s, q.a, q.b, elem, it, by);
        plans[r] = q;
        pf[r] = e;
        e += uint32_t(it);
    }
    if (threadIdx.x == 0) pf[R] = total;
    if (sb != nullptr && bytes) atomicAdd(&sb->exchange_bytes, bytes);
}

__global__ void xplan_single_kernel(uint64_t lx, uint64_t ly, XPlanArea pa, XParams prm) {
    if (threadIdx.x == 0) {
        RotPlan q{0, lx, ly};
        uint64_t it = 0, by = 0;
        x_count(prm, 0, lx, ly, 4, it, by);
        reinterpret_cast<RotPlan *>(pa.plans)[0] = q;
        pa.item_pf[0] = 0;
        pa.item_pf[1] = uint32_t(it);
    }
}

// ------------------------------------------------------------------ executor

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// "Reads done" flags.  A flag is stored after every thread of the CTA has consumed
// the registers its loads filled (so the loads have returned) and a __syncthreads;
// the reads are then over, and a relaxed store suffices: it does not wait for the
// CTA's earlier stores to drain, as a release would.  Waiters read flags relaxed too:
// the writes they guard are issued only after the flag value has been seen (a
// control dependency through a barrier).
__device__ __forceinline__ void st_flag(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_flag(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until flags[lo..hi] all reach tag.  False on timeout.
__device__ bool wait_flags(const uint32_t *flags, uint32_t lo, uint32_t hi, uint32_t tag) {
    unsigned long long t0 = 0;
    for (uint32_t q = lo; q <= hi; ++q) {
        uint32_t it = 0;
        while (ld_flag(flags + q) < tag) {
            if ((++it & 63u) == 0) {
                const unsigned long long now = globaltimer_ns();
                if (t0 == 0)
                    t0 = now;
                else if (now - t0 > kWaitLimitNs)
                    return false;
            }
        }
    }
    return true;
}

// Thread 0: wait until *ctr >= target.  False on timeout.
__device__ bool wait_count(const uint32_t *ctr, uint32_t target) {
    unsigned long long t0 = 0;
    uint32_t it = 0;
    while (ld_acquire(ctr) < target) {
        if ((++it & 63u) == 0) {
            const unsigned long long now = globaltimer_ns();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > kWaitLimitNs)
                return false;
        }
    }
    return true;
}

template <typename K, bool KV, int THREADS, int PP>
struct XCfg {
    static constexpr uint32_t kPairTile = uint32_t(THREADS) * PP;
    static constexpr uint32_t kShiftTile = 2u * kPairTile;
    static constexpr uint32_t kSmemBudget = 110u * 1024u;  // two CTAs per SM
    static constexpr uint32_t kCap = kSmemBudget / (sizeof(K) + (KV ? 4u : 0u));
    static constexpr uint32_t kMaxHolders = 8;
    static constexpr size_t kSmem = size_t(kCap) * sizeof(K) + (KV ? size_t(kCap) * 4 : 0);
    __host__ __device__ static XParams params() {
        return XParams{kPairTile, kShiftTile, kCap, kMaxHolders};
    }
};

constexpr int kCopyBatch = 8;

// All threads: stash[u - u0] = base[phys(off + u)] for u in [u0, u1), where
// phys(p) = mirror ? m-1-p : p; loads issued in batches.  u1 - u0 <= stash capacity.
template <typename K, bool KV, int THREADS>
__device__ __noinline__ void copy_in(K *stk, uint32_t *stv, const K *base,
                                     const uint32_t *vbase, uint32_t mirror, uint64_t m,
                                     uint64_t off, uint64_t u0, uint64_t u1) {
    const uint32_t cnt = uint32_t(u1 - u0);
    const uint64_t first = off + u0;
    for (uint32_t c = 0; c < cnt; c += uint32_t(THREADS) * kCopyBatch) {
        K kk[kCopyBatch];
        uint32_t vv[kCopyBatch];
#pragma unroll
        for (int k = 0; k < kCopyBatch; ++k) {
            const uint32_t u = c + uint32_t(k) * THREADS + threadIdx.x;
            if (u < cnt) {
                const uint64_t p = mirror ? m - 1 - (first + u) : first + u;
                kk[k] = __ldcg(base + p);
                if (KV) vv[k] = __ldcg(vbase + p);
            }
        }
#pragma unroll
        for (int k = 0; k < kCopyBatch; ++k) {
            const uint32_t u = c + uint32_t(k) * THREADS + threadIdx.x;
            if (u < cnt) {
                stk[u] = kk[k];
                if (KV) stv[u] = vv[k];
            }
        }
    }
}

// All threads: base[phys(off + u)] = stash[u - u0] for u in [u0, u1).
template <typename K, bool KV, int THREADS>
__device__ __noinline__ void copy_out(const K *stk, const uint32_t *stv, K *base,
                                      uint32_t *vbase, uint32_t mirror, uint64_t m,
                                      uint64_t off, uint64_t u0, uint64_t u1) {
    const uint32_t cnt = uint32_t(u1 - u0);
    const uint64_t first = off + u0;
    for (uint32_t u = threadIdx.x; u < cnt; u += THREADS) {
        const uint64_t p = mirror ? m - 1 - (first + u) : first + u;
        base[p] = stk[u];
        if (KV) vbase[p] = stv[u];
    }
}

// Thread 0: one non-blocking pass over flags[lo..hi]; true if all reached tag.
__device__ __forceinline__ bool flags_ready(const uint32_t *flags, uint32_t lo, uint32_t hi,
                                            uint32_t tag) {
    for (uint32_t q = lo; q <= hi; ++q)
        if (ld_flag(flags + q) < tag) return false;
    return true;
}

__device__ __forceinline__ uint32_t key_bits_lo(int32_t x) { return uint32_t(x); }
__device__ __forceinline__ uint32_t key_bits_lo(uint32_t x) { return x; }
__device__ __forceinline__ uint32_t key_bits_lo(float x) { return __float_as_uint(x); }
__device__ __forceinline__ uint32_t key_bits_lo(uint64_t x) {
    return uint32_t(x) ^ uint32_t(x >> 32);
}

// The flags a tile's writes depend on, as up to two index ranges (lo > hi: empty).
struct Deps {
    uint32_t lo0, hi0, lo1, hi1;
};

struct Shared {
    uint32_t next;
    int abort;
    uint32_t magic;  // runtime value the load fold is compared with
    uint32_t sink;   // written when the comparison happens to hold; never read
};

// Move of one tile: `cnt` element pairs (PAIR, SWAP) or single elements (SHIFT).
// Element k of this thread: source s0/s1, destination d0/d1 (physical offsets).
template <typename K, bool KV, int THREADS, int PP>
__device__ __noinline__ void tile_move(K *base, uint32_t *vbase, uint32_t kind,
                                          uint32_t mirror, uint64_t m, uint64_t t0,
                                          uint64_t t1, uint64_t rd1, uint64_t wr1,
                                          const uint32_t *flags, uint32_t my_flag,
                                          uint32_t tag, const Deps &dp, Shared &sh,
                                          StatusBlock *sb) {
    // PAIR : reads p(t), p(rd1+t); writes p(t) <- second, p(wr1+t) <- first
    // SWAP : reads t, rd1+t;        writes t <- second, rd1+t <- first  (mirror = 0)
    // SHIFT: reads p(rd1+t) for 2*PP elements per thread; writes p(t)
    const uint32_t tid = threadIdx.x;
    auto phys = [&](uint64_t x) -> uint64_t { return mirror ? m - 1 - x : x; };
    constexpr int NE = 2 * PP;  // registers per thread
    // zero-initialised: the fold below must read only defined values, or the compiler
    // could drop it (and with it the wait for the loads)
    K r[NE];
    uint32_t rv[KV ? NE : 1];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        r[k] = K(0);
        if (KV) rv[KV ? k : 0] = 0u;
    }
    if (kind == XK_SHIFT) {
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const uint64_t t = t0 + uint64_t(k) * THREADS + tid;
            if (t < t1) {
                const uint64_t p = phys(rd1 + t);
                r[k] = __ldcg(base + p);
                if (KV) rv[KV ? k : 0] = __ldcg(vbase + p);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const uint64_t t = t0 + uint64_t(k) * THREADS + tid;
            if (t < t1) {
                const uint64_t p0 = phys(t), p1 = phys(rd1 + t);
                r[2 * k] = __ldcg(base + p0);
                r[2 * k + 1] = __ldcg(base + p1);
                if (KV) {
                    rv[KV ? 2 * k : 0] = __ldcg(vbase + p0);
                    rv[KV ? 2 * k + 1 : 0] = __ldcg(vbase + p1);
                }
            }
        }
    }
    // while the loads are in flight, thread 0 checks whether the dependencies are met
    bool ready = true;
    if (tid == 0) {
        if (dp.lo0 <= dp.hi0) ready = flags_ready(flags, dp.lo0, dp.hi0, tag);
        if (ready && dp.lo1 <= dp.hi1) ready = flags_ready(flags, dp.lo1, dp.hi1, tag);
    }
    // A warp can reach a barrier with its loads still in flight: only reading the
    // destination registers waits for them.  Every loaded value is folded into one
    // word that is the operand of the barrier itself (a barrier reduction must have
    // its operand), so each warp's loads have returned before it arrives and the
    // "reads done" flag below is true.  (An operand of an empty asm would not do:
    // the assembler drops computations that no instruction consumes.)
    uint32_t fold = 0;
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        fold ^= key_bits_lo(r[k]);
        if (KV) fold ^= rv[KV ? k : 0];
    }
    if (__syncthreads_or(fold == sh.magic)) sh.sink = fold;  // rarely taken, harmless
    if (tid == 0) {
        if (flags != nullptr) st_flag(const_cast<uint32_t *>(flags) + my_flag, tag);
        if (!ready) {
            bool ok = true;
            if (dp.lo0 <= dp.hi0) ok = wait_flags(flags, dp.lo0, dp.hi0, tag);
            if (ok && dp.lo1 <= dp.hi1) ok = wait_flags(flags, dp.lo1, dp.hi1, tag);
            if (!ok) {
                set_status(sb, IPM_ERR_TIMEOUT);
                sh.abort = 1;
            }
        }
    }
    if (!(dp.lo0 > dp.hi0 && dp.lo1 > dp.hi1)) {
        __syncthreads();  // dependencies met (or abort) before any write
        if (sh.abort) return;
    }
    if (kind == XK_SHIFT) {
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const uint64_t t = t0 + uint64_t(k) * THREADS + tid;
            if (t < t1) {
                const uint64_t p = phys(t);
                base[p] = r[k];
                if (KV) vbase[p] = rv[KV ? k : 0];
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const uint64_t t = t0 + uint64_t(k) * THREADS + tid;
            if (t < t1) {
                const uint64_t p0 = phys(t), p1 = phys(wr1 + t);
                base[p0] = r[2 * k + 1];
                base[p1] = r[2 * k];
                if (KV) {
                    vbase[p0] = rv[KV ? 2 * k + 1 : 0];
                    vbase[p1] = rv[KV ? 2 * k : 0];
                }
            }
        }
    }
}

template <typename K, bool KV, int THREADS, int PP>
__global__ void __launch_bounds__(THREADS, 2)
    exchange_level_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, uint64_t n,
                          const RotPlan *__restrict__ plans, const uint32_t *__restrict__ pf,
                          uint32_t nrot, uint32_t *__restrict__ flags,
                          uint32_t *__restrict__ join, uint32_t tag, uint32_t ctr_index,
                          StatusBlock *sb) {
    using C = XCfg<K, KV, THREADS, PP>;
    extern __shared__ __align__(16) unsigned char xsmem[];
    K *stk = reinterpret_cast<K *>(xsmem);
    uint32_t *stv = reinterpret_cast<uint32_t *>(xsmem + size_t(C::kCap) * sizeof(K));
    __shared__ Shared sh;
    if (sb != nullptr && *((volatile unsigned int *)&sb->done)) return;
    const XParams prm = C::params();
    const uint32_t tid = threadIdx.x;
    const uint32_t total = pf[nrot];
    uint32_t *ctr = &sb->counters[ctr_index];
    if (tid == 0) {
        sh.next = atomicAdd(ctr, 1u);
        sh.abort = 0;
        sh.magic = tag * 0x9e3779b9u + blockIdx.x;
        sh.sink = 0;
    }
    __syncthreads();
    uint32_t rot = 0;  // search hint: a CTA's tickets only grow
    for (;;) {
        const uint32_t ticket = sh.next;
        const int aborted = sh.abort;
        __syncthreads();  // everyone has read the ticket before thread 0 replaces it
        if (ticket >= total || aborted) break;
        // ---- decode: the exchange r holding the ticket is the last one with
        // pf[r] <= ticket.  Tickets of a CTA only grow, so the block probes the THREADS
        // exchanges after the previous one in one coalesced round; a binary search
        // covers longer jumps.
        if (pf[rot + 1] <= ticket) {
            const uint32_t cand = rot + 1 + tid;
            const bool le = cand <= nrot && pf[cand] <= ticket;
            const int cnt = __syncthreads_count(le);  // pf non-decreasing: a prefix
            if (cnt < THREADS) {
                rot = rot + uint32_t(cnt);
            } else {
                uint32_t lo = rot + THREADS, hi = nrot;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (pf[mid] <= ticket)
                        lo = mid;
                    else
                        hi = mid;
                }
                rot = lo;
            }
        }
        const uint32_t r = rot;
        const uint32_t j = ticket - pf[r];
        const RotPlan q = plans[r];
        XPhase ph;
        uint64_t s = q.s, a = q.a, b = q.b;
        uint32_t before = 0;
        bool found = false;
        while (x_phase(prm, s, a, b, ph)) {
            if (j < before + ph.items()) {
                found = true;
                break;
            }
            before += ph.items();
            if (ph.final_phase) break;
            x_after_step(ph, s, a, b);
        }
        const uint64_t m = ph.a + ph.b;
        if (!found || ph.s > n || m > n - ph.s) {  // inconsistent plan or split table
            if (tid == 0) set_status(sb, IPM_ERR_DEVICE);
            break;
        }
        const uint32_t jj = j - before;
        const bool holder = (ph.kind == XK_PAIR || ph.kind == XK_SHIFT) && jj < ph.holders;
        uint32_t nxt = 0;
        if (tid == 0 && !holder) nxt = atomicAdd(ctr, 1u);  // result used at the end
        if (before > 0) {  // an earlier LS step of this exchange must be complete
            if (tid == 0 && !wait_count(join + r, before)) {
                set_status(sb, IPM_ERR_TIMEOUT);
                sh.abort = 1;
            }
            __syncthreads();
            if (sh.abort) break;
        }
        const uint32_t fb = pf[r] + before;  // flag of item 0 of this phase
        K *base = buf + ph.s;
        uint32_t *vbase = KV ? vals + ph.s : nullptr;
        const Deps none{1, 0, 1, 0};

        if (ph.kind == XK_SINGLE) {
            copy_in<K, KV, THREADS>(stk, stv, base, vbase, 0u, m, 0, 0, m);
            __syncthreads();
            const uint32_t mm = uint32_t(m), aa = uint32_t(ph.a);
            for (uint32_t t = tid; t < mm; t += THREADS) {
                uint32_t src = t + aa;
                if (src >= mm) src -= mm;
                base[t] = stk[src];
                if (KV) vbase[t] = stv[src];
            }
        } else if (ph.kind == XK_SWAP) {
            const uint64_t mn = ph.a < ph.b ? ph.a : ph.b;
            const uint64_t off2 = ph.a >= ph.b ? ph.a : ph.b;
            const uint64_t t0 = uint64_t(jj) * C::kPairTile;
            const uint64_t t1 = t0 + C::kPairTile < mn ? t0 + C::kPairTile : mn;
            tile_move<K, KV, THREADS, PP>(base, vbase, XK_SWAP, 0u, m, t0, t1, off2, off2,
                                          nullptr, 0, tag, none, sh, sb);
        } else if (holder) {
            // PAIR: stash = X'[Bp, Ap) -> X'2 lands at 2Bp; readers of the landing
            //       slots: tiles covering offsets [Bp-e+u).
            // SHIFT: stash = X'[0, sz) lands at rest; readers: tiles covering
            //       offsets [rest-sz+u).
            const bool pair = ph.kind == XK_PAIR;
            const uint64_t Bp = ph.a < ph.b ? ph.a : ph.b;
            const uint64_t dlt = ph.delta;
            const uint64_t h0 = uint64_t(jj) * prm.cap;
            const uint64_t h1 = h0 + prm.cap < dlt ? h0 + prm.cap : dlt;
            const uint64_t src_off = pair ? Bp : 0;
            const uint64_t dst_off = pair ? 2 * Bp : m - dlt;
            const uint64_t rd_off = pair ? Bp - dlt : m - 2 * dlt;
            const uint32_t tile = pair ? C::kPairTile : C::kShiftTile;
            copy_in<K, KV, THREADS>(stk, stv, base, vbase, ph.mirror, m, src_off, h0, h1);
            __syncthreads();
            if (tid == 0) {
                st_flag(flags + fb + jj, tag);
                const uint32_t qlo = uint32_t((rd_off + h0) / tile);
                const uint32_t qhi = uint32_t((rd_off + h1 - 1) / tile);
                if (!wait_flags(flags + fb + ph.holders, qlo, qhi, tag)) {
                    set_status(sb, IPM_ERR_TIMEOUT);
                    sh.abort = 1;
                }
            }
            __syncthreads();
            if (sh.abort) break;
            copy_out<K, KV, THREADS>(stk, stv, base, vbase, ph.mirror, m, dst_off, h0, h1);
        } else {
            const bool pair = ph.kind == XK_PAIR;
            const uint32_t qt = jj - ph.holders;
            const uint64_t dlt = ph.delta;
            const uint64_t Bp = ph.a < ph.b ? ph.a : ph.b;
            const uint64_t tile = pair ? C::kPairTile : C::kShiftTile;
            const uint64_t work = pair ? Bp : m - dlt;  // pairs (PAIR) or elements (SHIFT)
            const uint64_t t0 = uint64_t(qt) * tile;
            const uint64_t t1 = t0 + tile < work ? t0 + tile : work;
            // Writes that land in the stash region wait for its holders; writes over
            // the second block at offset t - dlt wait for the tiles that read it.
            Deps dp{1, 0, 1, 0};
            if (t0 < dlt) {
                dp.lo0 = fb + uint32_t(t0 / prm.cap);
                dp.hi0 = fb + uint32_t(((t1 < dlt ? t1 : dlt) - 1) / prm.cap);
            }
            if (t1 > dlt) {
                const uint32_t qlo = uint32_t(((t0 > dlt ? t0 : dlt) - dlt) / tile);
                const uint32_t qhi = uint32_t((t1 - 1 - dlt) / tile);
                if (qlo < qt) {
                    dp.lo1 = fb + ph.holders + qlo;
                    dp.hi1 = fb + ph.holders + (qhi < qt ? qhi : qt - 1);
                }
            }
            if (pair)
                tile_move<K, KV, THREADS, PP>(base, vbase, XK_PAIR, ph.mirror, m, t0, t1,
                                              m - Bp, Bp, flags, fb + jj, tag, dp, sh, sb);
            else
                tile_move<K, KV, THREADS, PP>(base, vbase, XK_SHIFT, ph.mirror, m, t0, t1,
                                              dlt, 0, flags, fb + jj, tag, dp, sh, sb);
            if (sh.abort) break;
        }
        // ---- item complete.  Only an LS step is waited for (by the next phase of its
        // exchange): every thread makes its own writes visible device-wide before the
        // barrier after which the step is counted.
        if (!ph.final_phase) __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (!ph.final_phase) atomicAdd(join + r, 1u);
            if (holder) nxt = atomicAdd(ctr, 1u);
            sh.next = nxt;
        }
        __syncthreads();
    }
}

template <typename K, bool KV>
struct XShape;
template <>
struct XShape<int32_t, false> { static constexpr int T = 256, PP = 16; };
template <>
struct XShape<uint32_t, false> { static constexpr int T = 256, PP = 16; };
template <>
struct XShape<float, false> { static constexpr int T = 256, PP = 16; };
template <>
struct XShape<uint64_t, false> { static constexpr int T = 256, PP = 8; };
template <>
struct XShape<int32_t, true> { static constexpr int T = 256, PP = 8; };
template <>
struct XShape<uint32_t, true> { static constexpr int T = 256, PP = 8; };
template <>
struct XShape<float, true> { static constexpr int T = 256, PP = 8; };
template <>
struct XShape<uint64_t, true> { static constexpr int T = 256, PP = 4; };

template <typename E, bool KV>
using XCfgOf = XCfg<E, KV, XShape<E, KV>::T, XShape<E, KV>::PP>;

template <typename E, bool KV>
ipm_status exchange_level_t(void *buf, uint32_t *vals, uint64_t n, uint32_t l,
                            XPlanArea pa, StatusBlock *sb, cudaStream_t stream) {
    using C = XCfgOf<E, KV>;
    auto kern = exchange_level_kernel<E, KV, XShape<E, KV>::T, XShape<E, KV>::PP>;
    static int grid = 0;
    if (grid == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(C::kSmem)) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, XShape<E, KV>::T,
                                                          C::kSmem) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        if (per_sm < 1) per_sm = 1;
        grid = per_sm * num_sms();
    }
    const uint64_t R = 1ull << l;
    const RotPlan *plans = reinterpret_cast<const RotPlan *>(pa.plans) + (R - 1);
    const uint32_t *pf = pa.item_pf + (R - 1) + l;
    kern<<<grid, XShape<E, KV>::T, C::kSmem, stream>>>(
        (E *)buf, vals, n, plans, pf, uint32_t(R), pa.flags, pa.join + (R - 1), l + 1,
        kTicketCounter0 + l, sb);
    return last_launch_status();
}

}  // namespace

XParams exchange_params(ipm_dtype key, bool with_values) {
    switch (key) {
    case IPM_INT32:
    case IPM_UINT32:
    case IPM_FLOAT32:
        return with_values ? XCfgOf<int32_t, true>::params() : XCfgOf<int32_t, false>::params();
    case IPM_UINT64:
        return with_values ? XCfgOf<uint64_t, true>::params()
                           : XCfgOf<uint64_t, false>::params();
    }
    return XParams{1, 2, 1, 1};
}

size_t xplan_area_bytes(uint32_t G, uint64_t n, ipm_dtype key, bool with_values) {
    if (G == 0) G = 1;
    const uint64_t P = 1ull << G;
    const XParams prm = exchange_params(key, with_values);
    size_t b = 0;
    b += align_up(sizeof(RotPlan) * P, 256);                  // plans of all levels
    b += align_up(sizeof(uint32_t) * (P + G + 1), 256);       // item prefixes
    b += align_up(sizeof(uint32_t) * P, 256);                 // per-exchange completion
    b += align_up(sizeof(uint32_t) * max_level_items(G, n, prm), 256);  // read flags
    return b;
}

uint64_t max_level_items(uint32_t G, uint64_t n, const XParams &prm) {
    // per exchange: tiles of its LS steps and of its final phase (<= 2 m / pair_tile + 2
    // per phase), at most n / (cap * max_holders) LS steps in all, max_holders + 1 more
    const uint64_t R = 1ull << (G ? G - 1 : 0);
    return 2 * n / prm.pair_tile + n / (uint64_t(prm.cap) * prm.max_holders) +
           R * (prm.max_holders + 6) + 16;
}

XPlanArea xplan_area_at(void *base, uint32_t G, uint64_t n, ipm_dtype key, bool with_values) {
    if (G == 0) G = 1;
    const uint64_t P = 1ull << G;
    const XParams prm = exchange_params(key, with_values);
    char *p = static_cast<char *>(base);
    XPlanArea pa;
    pa.plans = p;
    p += align_up(sizeof(RotPlan) * P, 256);
    pa.item_pf = reinterpret_cast<uint32_t *>(p);
    p += align_up(sizeof(uint32_t) * (P + G + 1), 256);
    pa.join = reinterpret_cast<uint32_t *>(p);
    p += align_up(sizeof(uint32_t) * P, 256);
    pa.flags = reinterpret_cast<uint32_t *>(p);
    pa.nflags = max_level_items(G, n, prm);
    pa.zero_bytes = size_t(reinterpret_cast<char *>(pa.flags) - reinterpret_cast<char *>(pa.join)) +
                    sizeof(uint32_t) * pa.nflags;
    return pa;
}

ipm_status launch_xplan_levels(const uint64_t *split, uint64_t n, uint32_t G, XPlanArea pa,
                               ipm_dtype key, bool with_values, StatusBlock *sb,
                               cudaStream_t stream) {
    if (G == 0) return IPM_OK;
    // completion counters and read flags start at zero on every call
    IPM_CUDA_TRY(cudaMemsetAsync(pa.join, 0, pa.zero_bytes, stream));
    const uint32_t elem = uint32_t(dtype_bytes(key)) + (with_values ? 4u : 0u);
    xplan_levels_kernel<<<G, kPlanThreads, 0, stream>>>(split, n, G, pa,
                                                        exchange_params(key, with_values),
                                                        elem, sb);
    return last_launch_status();
}

ipm_status launch_xplan_single(uint64_t lx, uint64_t ly, XPlanArea pa, ipm_dtype key,
                               cudaStream_t stream) {
    IPM_CUDA_TRY(cudaMemsetAsync(pa.join, 0, pa.zero_bytes, stream));
    xplan_single_kernel<<<1, 32, 0, stream>>>(lx, ly, pa, exchange_params(key, false));
    return last_launch_status();
}

ipm_status launch_exchange_level(void *buf, uint32_t *vals, ipm_dtype key, uint64_t n,
                                 uint32_t l, XPlanArea pa, StatusBlock *sb,
                                 cudaStream_t stream) {
    const bool kv = vals != nullptr;
    switch (key) {
    case IPM_INT32:
    case IPM_UINT32:
    case IPM_FLOAT32:
        return kv ? exchange_level_t<int32_t, true>(buf, vals, n, l, pa, sb, stream)
                  : exchange_level_t<int32_t, false>(buf, vals, n, l, pa, sb, stream);
    case IPM_UINT64:
        return kv ? exchange_level_t<uint64_t, true>(buf, vals, n, l, pa, sb, stream)
                  : exchange_level_t<uint64_t, false>(buf, vals, n, l, pa, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

}  // namespace ipm
