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
// resident CTAs, so the tiles always find a CTA).  The upper levels have few
// exchanges, so they get more holders (level_holders): a bigger on-chip stash turns an
// exchange of a large and a mid-sized block into one SHIFT pass instead of a long
// chain of LS steps.  Consecutive phases of one exchange
// (LS steps) are ordered by a per-exchange completion counter.  Every wait is bounded
// in time; on expiry the kernel records IPM_ERR_TIMEOUT and all CTAs leave.
//
// Ticket order within a level is phase-major: section k holds phase k of every exchange
// (exchange by exchange), and the last section holds every exchange's remaining phases
// (exchange-major).  An exchange whose blocks leave long chains of LS steps (heavy key
// repeats) thus has step k of every exchange in flight together instead of one step of
// one exchange at a time; an exchange that is done in one phase (the common case) lies
// in section 0 as before.  Every wait is still on earlier tickets: a phase waits for the
// earlier phases of its exchange (earlier sections, or earlier in the last one) and for
// items of its own phase.
#include "ipm_exchange.cuh"
#include "ipm_internal.h"
#include "ipm_tma.cuh"

namespace ipm {

namespace {

constexpr uint32_t kPlanThreads = 1024;

// Stash holders per exchange at level l: about half the resident CTAs shared by the
// level's 2^l exchanges (hcap = half the resident CTAs, from the host), at least the
// base 8 and at most 64.  The plan and the level kernels use the same value.
constexpr uint32_t kMinHolders = 8, kMaxHoldersCap = 64;
__host__ __device__ inline uint32_t level_holders(uint32_t l, uint32_t hcap) {
    const uint32_t h = l < 31 ? hcap >> l : 0u;
    return h < kMinHolders ? kMinHolders : (h > kMaxHoldersCap ? kMaxHoldersCap : h);
}

struct RotPlan {
    uint64_t s, a, b;
};

// Items of each section of one exchange (phase k in section k < kSections - 1, every
// later phase in the last section) and its algorithmic bytes.
__host__ __device__ inline void x_sections(const XParams &P, uint64_t s, uint64_t a, uint64_t b,
                                           uint32_t elem, uint32_t (&c)[kSections],
                                           uint64_t &bytes) {
    for (uint32_t k = 0; k < kSections; ++k) c[k] = 0;
    bytes = 0;
    XPhase ph;
    uint32_t p = 0;
    while (x_phase(P, s, a, b, ph)) {
        const uint32_t k = p < kSections - 1 ? p : kSections - 1;
        for (uint32_t q = 0; q < kSections; ++q)
            if (q == k) c[q] += ph.items();
        const uint64_t mn = ph.a < ph.b ? ph.a : ph.b;
        bytes += (ph.kind == XK_SWAP ? 4 * mn : 2 * (ph.a + ph.b)) * elem;
        if (ph.final_phase) break;
        x_after_step(ph, s, a, b);
        ++p;
    }
}

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

// One block per level: the exchanges of level l, the item prefix of every section over
// the exchanges, the section starts and (added into the status block) the algorithmic
// bytes.
__global__ void __launch_bounds__(kPlanThreads)
    xplan_levels_kernel(const uint64_t *__restrict__ split, uint64_t n, uint32_t G,
                        XPlanArea pa, XParams prm, uint32_t hcap, uint32_t elem,
                        StatusBlock *sb) {
    __shared__ uint32_t s_tot[kSections];
    if (call_finished(sb)) return;
    const uint32_t l = blockIdx.x;
    prm.max_holders = level_holders(l, hcap);
    const uint64_t R = 1ull << l;
    RotPlan *plans = reinterpret_cast<RotPlan *>(pa.plans) + (R - 1);
    uint32_t *pk = pa.item_pf + level_prefix_offset(l);
    uint32_t *sec = pa.sec_start + level_section_offset(l);
    const uint64_t per = (R + kPlanThreads - 1) / kPlanThreads;
    const uint64_t r0 = per * threadIdx.x;
    const uint64_t r1 = r0 + per < R ? r0 + per : R;
    uint32_t items[kSections] = {};
    unsigned long long bytes = 0;
    for (uint64_t r = r0; r < r1; ++r) {
        RotPlan q = level_rotation(split, n, G, l, r);
        uint32_t c[kSections];
        uint64_t by = 0;
        x_sections(prm, q.s, q.a, q.b, elem, c, by);
#pragma unroll
        for (uint32_t k = 0; k < kSections; ++k) items[k] += c[k];
        bytes += by;
    }
    uint32_t e[kSections];
#pragma unroll
    for (uint32_t k = 0; k < kSections; ++k) {
        uint32_t tot;
        e[k] = block_exclusive_scan_u32(items[k], &tot);
        if (threadIdx.x == 0) s_tot[k] = tot;
    }
    for (uint64_t r = r0; r < r1; ++r) {
        RotPlan q = level_rotation(split, n, G, l, r);
        uint32_t c[kSections];
        uint64_t by = 0;
        x_sections(prm, q.s, q.a, q.b, elem, c, by);
        plans[r] = q;
#pragma unroll
        for (uint32_t k = 0; k < kSections; ++k) {
            pk[k * (R + 1) + r] = e[k];
            e[k] += c[k];
        }
    }
    if (threadIdx.x == 0) {
        uint32_t start = 0;
        for (uint32_t k = 0; k < kSections; ++k) {
            pk[k * (R + 1) + R] = s_tot[k];
            sec[k] = start;
            start += s_tot[k];
        }
        sec[kSections] = start;
    }
    if (sb != nullptr && bytes) atomicAdd(&sb->exchange_bytes, bytes);
}

__global__ void xplan_single_kernel(uint64_t lx, uint64_t ly, XPlanArea pa, XParams prm,
                                    uint32_t hcap) {
    prm.max_holders = level_holders(0, hcap);
    if (threadIdx.x == 0) {
        RotPlan q{0, lx, ly};
        uint32_t c[kSections];
        uint64_t by = 0;
        x_sections(prm, 0, lx, ly, 4, c, by);
        reinterpret_cast<RotPlan *>(pa.plans)[0] = q;
        uint32_t start = 0;
        for (uint32_t k = 0; k < kSections; ++k) {
            pa.item_pf[2 * k] = 0;
            pa.item_pf[2 * k + 1] = c[k];
            pa.sec_start[k] = start;
            start += c[k];
        }
        pa.sec_start[kSections] = start;
    }
}

// ------------------------------------------------------------------ executor

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
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

// Thread 0: wait until *ctr >= target.  False after `lim` ns.
__device__ bool wait_count(const uint32_t *ctr, uint32_t target, unsigned long long lim) {
    DepTimer tm(lim);
    while (ld_acquire(ctr) < target)
        if (tm.expired()) return false;
    return true;
}

// ---- TMA-staged executor: one persistent 512-thread CTA per SM, two shared-memory
// stages.  A stage holds two "slots"; an item moves at most two contiguous blocks
// (physical ranges: a mirrored primed range is still contiguous and keeps its order),
// each staged in one slot (a SHIFT tile, stash chunk or SINGLE exchange spans both).

// V: the payload type (4- or 8-byte; moved like the keys).
template <typename K, bool KV, typename V = uint32_t>
struct XCfg {
    static constexpr int kThreads = 512;
    static constexpr uint32_t kStageBytes = 112u * 1024u;
    static constexpr uint32_t kElemBytes = uint32_t(sizeof(K)) + (KV ? uint32_t(sizeof(V)) : 0u);
    static constexpr uint32_t kKPad = 16u / uint32_t(sizeof(K));  // phase slack, keys
    static constexpr uint32_t kVPad = 16u / uint32_t(sizeof(V));  // phase slack, values
    // elements per slot, a multiple of 32
    static constexpr uint32_t kSlot =
        ((kStageBytes / (2u * kElemBytes)) - (kKPad > kVPad ? kKPad : kVPad) - 16u) / 32u * 32u;
    static constexpr uint32_t kSlotK = kSlot + kKPad;  // key slot stride (elements)
    static constexpr uint32_t kSlotV = kSlot + kVPad;  // value slot stride (elements)
    static constexpr size_t kStageKBytes = (size_t(2) * kSlotK * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t kStageVBytes =
        KV ? (size_t(2) * kSlotV * sizeof(V) + 15) / 16 * 16 : 0;
    static constexpr size_t kStageSize = kStageKBytes + kStageVBytes;
    static constexpr size_t kSmem = 2 * kStageSize + 64;  // two stages + two mbarriers
    // pair tile = one slot per block; shift tile, stash chunk and SINGLE exchange = two
    // slots (they start at slot 0 with their own phase offset < kKPad)
    // a SINGLE exchange is staged across both stages (keys, then values)
    static constexpr uint32_t kSingleCap =
        uint32_t((2 * kStageSize - 64) / kElemBytes) / 32u * 32u;
    __host__ __device__ static XParams params() {
        return XParams{kSlot, 2 * kSlot, 2 * kSlot, 8u, kSingleCap};  // holders: per level
    }
};

// The flags a store depends on, as up to two index ranges (lo > hi: empty).
struct Deps {
    uint32_t lo0, hi0, lo1, hi1;
};

struct Move {
    uint64_t src, dst, len;  // absolute element offsets in the buffer
};

// A decoded item.
struct Item {
    uint32_t r, before, nmoves;
    bool holder, final_phase, single, flag;
    uint32_t ticket;
    Move mv[2];
    uint64_t single_m, single_a;  // SINGLE: exchange size and rotation
    Deps dp;
};

struct Shared {
    uint32_t ticket[2];
    int abort;
};

// Thread 0: wait until flags[lo..hi] all reach tag (empty range: true).  While
// waiting, publish the prefetched item's flag (`my_flag`) as soon as its staging
// mbarrier completes.  False on timeout.
__device__ bool wait_flag_range_poll(const uint32_t *flags, uint32_t lo, uint32_t hi,
                                     uint32_t tag, bool nxt_loaded, bool nxt_flag,
                                     uint64_t *nbar, uint32_t nparity, uint32_t *my_flag,
                                     bool &published, unsigned long long lim) {
    DepTimer tm(lim);
    for (uint32_t q = lo; q <= hi && lo <= hi; ++q) {
        while (ld_flag(flags + q) < tag) {
            if (nxt_loaded && nxt_flag && !published && mbar_try_wait(nbar, nparity)) {
                st_flag(my_flag, tag);
                published = true;
            }
            if (tm.expired()) return false;
        }
    }
    return true;
}

// Item j - before of phase ph of exchange r (ticket t; fb = the flag index of the
// phase's item 0): its moves and the flags its stores depend on.
__device__ __forceinline__ void decode_phase_item(const XParams &prm, const XPhase &ph,
                                                  uint32_t t, uint32_t r, uint32_t j,
                                                  uint32_t before, uint32_t fb, Item &it) {
    const uint64_t m = ph.a + ph.b;
    const uint32_t jj = j - before;
    it.ticket = t;
    it.r = r;
    it.before = before;
    it.final_phase = ph.final_phase;
    it.single = ph.kind == XK_SINGLE;
    it.holder = (ph.kind == XK_PAIR || ph.kind == XK_SHIFT) && jj < ph.holders;
    it.flag = ph.kind == XK_PAIR || ph.kind == XK_SHIFT;
    it.dp = Deps{1, 0, 1, 0};
    it.single_m = 0;
    it.single_a = 0;
    const uint64_t base = ph.s;
    const uint32_t mirror = ph.mirror;
    // physical start of the primed range [x0, x0 + len)
    auto pr = [base, mirror, m](uint64_t x0, uint64_t len) -> uint64_t {
        return base + (mirror ? m - x0 - len : x0);
    };
    if (ph.kind == XK_SINGLE) {
        it.nmoves = 1;
        it.mv[0] = Move{base, base, m};
        it.single_m = m;
        it.single_a = ph.a;
    } else if (ph.kind == XK_SWAP) {
        const uint64_t mn = ph.a < ph.b ? ph.a : ph.b;
        const uint64_t off2 = ph.a >= ph.b ? ph.a : ph.b;
        const uint64_t t0 = uint64_t(jj) * prm.pair_tile;
        const uint64_t L = (t0 + prm.pair_tile < mn ? t0 + prm.pair_tile : mn) - t0;
        it.nmoves = 2;
        it.mv[0] = Move{base + t0, base + off2 + t0, L};
        it.mv[1] = Move{base + off2 + t0, base + t0, L};
    } else if (it.holder) {
        // PAIR: stash X'[Bp, Ap) lands at 2Bp; its landing slots hold Y'[Bp-e+u), read
        //       by the tiles covering those offsets.
        // SHIFT: stash X'[0, sz) lands at m-sz; the slots hold Y'[m-2sz+u).
        const bool pair = ph.kind == XK_PAIR;
        const uint64_t Bp = ph.a < ph.b ? ph.a : ph.b;
        const uint64_t dlt = ph.delta;
        const uint64_t h0 = uint64_t(jj) * prm.cap;
        const uint64_t h1 = h0 + prm.cap < dlt ? h0 + prm.cap : dlt;
        const uint64_t src_off = pair ? Bp : 0;
        const uint64_t dst_off = pair ? 2 * Bp : m - dlt;
        const uint64_t rd_off = pair ? Bp - dlt : m - 2 * dlt;
        const uint64_t tile = pair ? prm.pair_tile : prm.shift_tile;
        it.nmoves = 1;
        it.mv[0] = Move{pr(src_off + h0, h1 - h0), pr(dst_off + h0, h1 - h0), h1 - h0};
        it.dp.lo0 = fb + ph.holders + uint32_t((rd_off + h0) / tile);
        it.dp.hi0 = fb + ph.holders + uint32_t((rd_off + h1 - 1) / tile);
    } else {
        const bool pair = ph.kind == XK_PAIR;
        const uint32_t qt = jj - ph.holders;
        const uint64_t dlt = ph.delta;
        const uint64_t Bp = ph.a < ph.b ? ph.a : ph.b;
        const uint64_t tile = pair ? prm.pair_tile : prm.shift_tile;
        const uint64_t work = pair ? Bp : m - dlt;  // pairs (PAIR) or elements (SHIFT)
        const uint64_t t0 = uint64_t(qt) * tile;
        const uint64_t t1 = t0 + tile < work ? t0 + tile : work;
        const uint64_t L = t1 - t0;
        if (pair) {
            it.nmoves = 2;
            it.mv[0] = Move{pr(t0, L), pr(Bp + t0, L), L};      // X'[t] -> Bp + t
            it.mv[1] = Move{pr(m - Bp + t0, L), pr(t0, L), L};  // Y'[t] -> t
        } else {
            it.nmoves = 1;
            it.mv[0] = Move{pr(dlt + t0, L), pr(t0, L), L};     // Y'[t] -> t
        }
        // writes into the stash region wait for its holders; writes over the second
        // block at offset t - dlt wait for the tiles that read it
        if (t0 < dlt) {
            it.dp.lo0 = fb + uint32_t(t0 / prm.cap);
            it.dp.hi0 = fb + uint32_t(((t1 < dlt ? t1 : dlt) - 1) / prm.cap);
        }
        if (t1 > dlt) {
            const uint32_t qlo = uint32_t(((t0 > dlt ? t0 : dlt) - dlt) / tile);
            const uint32_t qhi = uint32_t((t1 - 1 - dlt) / tile);
            if (qlo < qt) {
                it.dp.lo1 = fb + ph.holders + qlo;
                it.dp.hi1 = fb + ph.holders + (qhi < qt ? qhi : qt - 1);
            }
        }
    }
}

// Item j (counted within section k) of exchange r: replay the exchange's phases to the
// one holding it (phase k when k < kSections - 1; in the last section, its phases from
// there on back to back).  t is the ticket; the phase's items have consecutive tickets,
// so its item 0 (the base of its flag indices) is t minus the item's index in the phase.
__device__ __forceinline__ bool decode_in_exchange(const XParams &prm, uint32_t t, uint32_t r,
                                                   uint32_t j, uint32_t k, const RotPlan &q,
                                                   uint64_t n, Item &it) {
    XPhase ph;
    uint64_t s = q.s, a = q.a, b = q.b;
    uint32_t before = 0, p = 0;
    bool found = false;
    while (x_phase(prm, s, a, b, ph)) {
        const uint32_t ps = p < kSections - 1 ? p : kSections - 1;
        if (ps == k) {
            if (j < ph.items()) {
                found = true;
                break;
            }
            if (k < kSections - 1) break;  // the section holds this one phase only
            j -= ph.items();
        }
        before += ph.items();
        if (ph.final_phase) break;
        x_after_step(ph, s, a, b);
        ++p;
    }
    const uint64_t m = ph.a + ph.b;
    if (!found || ph.s > n || m > n - ph.s) return false;
    decode_phase_item(prm, ph, t, r, before + j, before, t - j, it);
    return true;
}

// The section of ticket t (the last k with sec[k] <= t), from the previous one: a CTA's
// tickets only grow.  A new section restarts the exchange hint.
__device__ __forceinline__ uint32_t ticket_section(const uint32_t *sec, uint32_t t,
                                                   uint32_t &sec_hint, uint32_t &rot_hint) {
    uint32_t k = sec_hint;
    while (k + 1 < kSections && sec[k + 1] <= t) ++k;
    if (k != sec_hint) {
        sec_hint = k;
        rot_hint = 0;
    }
    return k;
}

// Decode ticket t of a level plan into an item.  Every thread computes the same item.
// pk: the level's per-section exchange prefixes (kSections x (nrot + 1)); sec: its
// section starts.
__device__ __forceinline__ bool decode_item(const XParams &prm, uint32_t t, uint32_t &rot_hint,
                                            uint32_t &sec_hint, const uint32_t *pk,
                                            const uint32_t *sec, const RotPlan *plans,
                                            uint32_t nrot, uint64_t n, Item &it) {
    const uint32_t k = ticket_section(sec, t, sec_hint, rot_hint);
    const uint32_t ts = t - sec[k];
    const uint32_t *pf = pk + size_t(k) * (nrot + 1);
    // the exchange holding ts is the last one with pf[r] <= ts.  A CTA's tickets only
    // grow: the block probes the 512 exchanges after the previous one in one coalesced
    // round (pf is non-decreasing, so the hits form a prefix); longer jumps bisect.
    if (pf[rot_hint + 1] <= ts) {
        const uint32_t cand = rot_hint + 1 + threadIdx.x;
        const int cnt = __syncthreads_count(cand <= nrot && pf[cand] <= ts);
        if (cnt < int(blockDim.x)) {
            rot_hint += uint32_t(cnt);
        } else {
            uint32_t lo = rot_hint + blockDim.x, hi = nrot;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (pf[mid] <= ts)
                    lo = mid;
                else
                    hi = mid;
            }
            rot_hint = lo;
        }
    }
    const uint32_t r = rot_hint;
    return decode_in_exchange(prm, t, r, ts - pf[r], k, plans[r], n, it);
}

// Shared-memory layout of a stage: two key slots, then two value slots.  A SINGLE
// exchange instead spans both stages from the base: keys, then values.
template <typename K, bool KV>
__device__ __forceinline__ K *stage_keys(const Item &it, unsigned char *stage,
                                         unsigned char *base) {
    return reinterpret_cast<K *>(it.single ? base : stage);
}
template <typename K, bool KV, typename V = uint32_t>
__device__ __forceinline__ V *stage_vals(const Item &it, unsigned char *stage,
                                         unsigned char *base) {
    using C = XCfg<K, KV, V>;
    return reinterpret_cast<V *>(
        it.single ? base + (size_t(C::kSingleCap + C::kKPad) * sizeof(K) + 15) / 16 * 16
                  : stage + C::kStageKBytes);
}

// Unaligned head/tail elements of a staged item, loaded into registers by threads
// 0..31 (keys) and 32..63 (values) and written to shared memory only later
// (flush_pending), so their load latency does not stall the CTA.  A thread holds at most
// one element per stage.
template <typename K>
struct Pending {
    K key;
    uint32_t val;
    uint32_t slot;  // element index from the shared-memory base, or ~0u if none
};

// Stage the item's source blocks: TMA bulk copies for the 16-byte-aligned bodies
// (thread 0 arms the mbarrier with their byte count and issues them); the heads and
// tails (under 16 bytes per end) go to `pd` and reach shared memory in flush_pending.
template <typename K, bool KV>
__device__ __forceinline__ void stage_load(const Item &it, const K *buf, const uint32_t *vals,
                                           unsigned char *stage, unsigned char *base,
                                           uint64_t *bar, Pending<K> &pd) {
    using C = XCfg<K, KV>;
    K *sk = stage_keys<K, KV>(it, stage, base);
    uint32_t *sv = stage_vals<K, KV>(it, stage, base);
    const uint32_t tid = threadIdx.x;
    pd.slot = ~0u;
    if (tid == 0) {
        uint32_t tx = 0;
        for (uint32_t i = 0; i < it.nmoves; ++i) {
            const Geo<int(sizeof(K))> gk(buf + it.mv[i].src, uint32_t(it.mv[i].len));
            tx += gk.body * uint32_t(sizeof(K));
            if (KV) {
                const Geo<4> gv(vals + it.mv[i].src, uint32_t(it.mv[i].len));
                tx += gv.body * 4u;
            }
        }
        mbar_arrive_expect_tx(bar, tx);
    }
    const uint32_t kofs = uint32_t((reinterpret_cast<unsigned char *>(sk) - base) / sizeof(K));
    const uint32_t vofs = uint32_t((reinterpret_cast<unsigned char *>(sv) - base) / 4);
    for (uint32_t i = 0; i < it.nmoves; ++i) {
        const Move &mv = it.mv[i];
        const uint32_t len = uint32_t(mv.len);
        const K *g = buf + mv.src;
        const Geo<int(sizeof(K))> gk(g, len);
        if (tid == 0 && gk.body)
            bulk_load(sk + i * C::kSlotK + gk.off + gk.head, g + gk.head,
                      gk.body * uint32_t(sizeof(K)), bar);
        // move i: lanes 8i .. 8i+7 of warp 0; lane e < 4 takes head element e, lane
        // e >= 4 tail element e-4 (at most 3 of each for 4-byte keys, 1 for 8-byte)
        if (tid >= 8 * i && tid < 8 * i + 8) {
            const uint32_t e = tid - 8 * i;
            const uint32_t ntail = len - gk.tail_start;
            uint32_t j = ~0u;
            if (e < 4 && e < gk.head)
                j = e;
            else if (e >= 4 && e - 4 < ntail)
                j = gk.tail_start + (e - 4);
            if (j != ~0u) {
                pd.key = __ldcg(g + j);
                pd.slot = kofs + i * C::kSlotK + gk.off + j;
            }
        }
        if (KV) {
            const uint32_t *gv = vals + mv.src;
            const Geo<4> gvv(gv, len);
            if (tid == 0 && gvv.body)
                bulk_load(sv + i * C::kSlotV + gvv.off + gvv.head, gv + gvv.head, gvv.body * 4u,
                          bar);
            if (tid >= 32 + 8 * i && tid < 40 + 8 * i) {
                const uint32_t e = tid - 32 - 8 * i;
                const uint32_t ntail = len - gvv.tail_start;
                uint32_t j = ~0u;
                if (e < 4 && e < gvv.head)
                    j = e;
                else if (e >= 4 && e - 4 < ntail)
                    j = gvv.tail_start + (e - 4);
                if (j != ~0u) {
                    pd.val = __ldcg(gv + j);
                    pd.slot = vofs + i * C::kSlotV + gvv.off + j;
                }
            }
        }
    }
}

// Write a pending head/tail element to shared memory (keys from threads 0..31, values
// from threads 32..63).  The caller's next barrier makes it visible to the CTA.
template <typename K>
__device__ __forceinline__ void flush_pending(Pending<K> &pd, unsigned char *base) {
    if (pd.slot != ~0u) {
        if (threadIdx.x < 32)
            reinterpret_cast<K *>(base)[pd.slot] = pd.key;
        else
            reinterpret_cast<uint32_t *>(base)[pd.slot] = pd.val;
        pd.slot = ~0u;
    }
}

// dst[0, len) = src[0, len) (src in shared memory): 8 independent shared loads per
// thread ahead of their 8 coalesced global stores, so the loop is not latency-bound.
template <typename T, int THREADS>
__device__ __forceinline__ void copy_out_unrolled(const T *src, T *dst, uint32_t len) {
    constexpr uint32_t U = 8;
    const uint32_t tid = threadIdx.x;
    uint32_t j0 = 0;
    for (; j0 + U * THREADS <= len; j0 += U * THREADS) {
        T v[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) v[u] = src[j0 + u * THREADS + tid];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) dst[j0 + u * THREADS + tid] = v[u];
    }
    for (uint32_t j = j0 + tid; j < len; j += THREADS) dst[j] = src[j];
}

// Write the staged blocks to their destinations (coalesced stores from shared memory).
template <typename K, bool KV>
__device__ __forceinline__ void stage_store(const Item &it, K *buf, uint32_t *vals,
                                            unsigned char *stage, unsigned char *base) {
    using C = XCfg<K, KV>;
    const K *sk = stage_keys<K, KV>(it, stage, base);
    const uint32_t *sv = stage_vals<K, KV>(it, stage, base);
    const uint32_t tid = threadIdx.x;
    if (it.single) {  // the whole exchange [X|Y] is staged; write it rotated by |X|
        const Move &mv = it.mv[0];
        const Geo<int(sizeof(K))> gk(buf + mv.src, uint32_t(mv.len));
        const uint32_t m = uint32_t(it.single_m), a = uint32_t(it.single_a);
        const K *k0 = sk + gk.off;
        K *dst = buf + mv.dst;
        for (uint32_t t = tid; t < m; t += C::kThreads) {
            uint32_t src = t + a;
            if (src >= m) src -= m;
            dst[t] = k0[src];
        }
        if (KV) {
            const Geo<4> gv(vals + mv.src, uint32_t(mv.len));
            const uint32_t *v0 = sv + gv.off;
            uint32_t *vd = vals + mv.dst;
            for (uint32_t t = tid; t < m; t += C::kThreads) {
                uint32_t src = t + a;
                if (src >= m) src -= m;
                vd[t] = v0[src];
            }
        }
        return;
    }
    for (uint32_t i = 0; i < it.nmoves; ++i) {
        const Move &mv = it.mv[i];
        const uint32_t len = uint32_t(mv.len);
        const Geo<int(sizeof(K))> gk(buf + mv.src, len);
        copy_out_unrolled<K, C::kThreads>(sk + i * C::kSlotK + gk.off, buf + mv.dst, len);
        if (KV) {
            const Geo<4> gv(vals + mv.src, len);
            copy_out_unrolled<uint32_t, C::kThreads>(sv + i * C::kSlotV + gv.off, vals + mv.dst,
                                                     len);
        }
    }
}

// One level: items in ticket order.  Per item: stage its blocks (TMA), publish "reads
// done" once the data has landed, wait for the flags its stores depend on, store.  The
// next item's blocks are staged into the other stage while the current one completes,
// unless the current item is a stash holder (it waits on later tickets, which must
// stay available to other CTAs) or the next item must first wait for an LS step.
template <typename K, bool KV>
__global__ void __launch_bounds__(512, 1)
    exchange_level_kernel(K *__restrict__ buf, uint32_t *__restrict__ vals, uint64_t n,
                          const RotPlan *__restrict__ plans, const uint32_t *__restrict__ pk,
                          const uint32_t *__restrict__ sec, uint32_t nrot,
                          uint32_t *__restrict__ flags,
                          uint32_t *__restrict__ join, uint32_t tag, uint32_t ctr_index,
                          uint32_t holders, StatusBlock *sb) {
    using C = XCfg<K, KV>;
    extern __shared__ __align__(128) unsigned char xsmem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(xsmem + 2 * C::kStageSize);
    __shared__ Shared sh;
    if (call_finished(sb)) return;
    const unsigned long long lim = wait_limit(sb);
    XParams prm = C::params();
    prm.max_holders = holders;
    const uint32_t tid = threadIdx.x;
    const uint32_t total = sec[kSections];
    uint32_t *ctr = &sb->counters[ctr_index];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        sh.ticket[0] = atomicAdd(ctr, 1u);
        sh.abort = 0;
    }
    __syncthreads();
    uint32_t parity0 = 0, parity1 = 0;
    uint32_t rot = 0, sech = 0;
    int cs = 0;  // stage of the current item
    Item cur;
    bool cur_loaded = false;
    uint32_t cur_t = sh.ticket[0];
    if (cur_t < total && !decode_item(prm, cur_t, rot, sech, pk, sec, plans, nrot, n, cur)) {
        if (tid == 0) set_status(sb, IPM_ERR_DEVICE);
        return;
    }
    uint32_t it_no = 0;
    bool cur_flag_done = false;  // thread 0: the current item's flag is published
    Pending<K> pd_cur, pd_nxt;   // head/tail elements staged by this thread
    pd_cur.slot = ~0u;
    pd_nxt.slot = ~0u;
    while (cur_t < total) {
        bool nxt_flag_done = false;
        unsigned char *st_cur = xsmem + (cs ? C::kStageSize : 0);
        unsigned char *st_nxt = xsmem + (cs ? 0 : C::kStageSize);
        // ---- the current item's earlier LS steps must be complete before it loads
        if (!cur_loaded) {
            if (cur.before > 0) {
                if (tid == 0 && !wait_count(join + cur.r, cur.before, lim)) {
                    set_status(sb, IPM_ERR_TIMEOUT);
                    sh.abort = 1;
                }
                __syncthreads();
                if (sh.abort) break;
            }
            stage_load<K, KV>(cur, buf, vals, st_cur, xsmem, &bar[cs], pd_cur);
        }
        // ---- reserve and decode the next ticket (alternating slots: no extra barrier).
        // A stash holder reserves it only once it is done: it waits on later tickets of
        // its own exchange, and one of them must never be parked behind it.
        uint32_t nxt_t = total;
        Item nxt;
        bool nxt_loaded = false;
        if (!cur.holder) {
            if (tid == 0) sh.ticket[(it_no + 1) & 1] = atomicAdd(ctr, 1u);
            __syncthreads();
            nxt_t = sh.ticket[(it_no + 1) & 1];
            if (nxt_t < total && !decode_item(prm, nxt_t, rot, sech, pk, sec, plans, nrot, n, nxt)) {
                if (tid == 0) set_status(sb, IPM_ERR_DEVICE);
                break;
            }
            // a SINGLE exchange needs both stages: it neither prefetches nor is prefetched
            if (nxt_t < total && nxt.before == 0 && !nxt.single && !cur.single) {
                stage_load<K, KV>(nxt, buf, vals, st_nxt, xsmem, &bar[cs ^ 1], pd_nxt);
                nxt_loaded = true;
            }
        }
        // ---- current item: staged -> reads done -> dependencies -> stores
        if (tid == 0 && !mbar_wait_bounded(&bar[cs], cs ? parity1 : parity0)) {
            set_status(sb, IPM_ERR_TIMEOUT);
            sh.abort = 1;
        }
        if (cs)
            parity1 ^= 1u;
        else
            parity0 ^= 1u;
        flush_pending<K>(pd_cur, xsmem);
        flush_pending<K>(pd_nxt, xsmem);  // the next item's reads are over once it lands
        __syncthreads();  // bulk data landed; heads and tails are in shared memory
        if (sh.abort) break;
        if (tid == 0) {
            if (cur.flag && !cur_flag_done) st_flag(flags + cur.ticket, tag);
            // The prefetched item's "reads done" is published as soon as its data has
            // landed (its heads and tails were loaded before the barrier above), not
            // when it becomes current: the tiles after it in the chain wait for it.
            const uint32_t np = cs ? parity0 : parity1;
            bool ok = wait_flag_range_poll(flags, cur.dp.lo0, cur.dp.hi0, tag, nxt_loaded,
                                           nxt.flag, &bar[cs ^ 1], np, flags + nxt_t,
                                           nxt_flag_done, lim);
            if (ok)
                ok = wait_flag_range_poll(flags, cur.dp.lo1, cur.dp.hi1, tag, nxt_loaded,
                                          nxt.flag, &bar[cs ^ 1], np, flags + nxt_t,
                                          nxt_flag_done, lim);
            if (!ok) {
                set_status(sb, IPM_ERR_TIMEOUT);
                sh.abort = 1;
            }
        }
        __syncthreads();
        if (sh.abort) break;
        stage_store<K, KV>(cur, buf, vals, st_cur, xsmem);
        if (tid == 0 && nxt_loaded && nxt.flag && !nxt_flag_done &&
            mbar_try_wait(&bar[cs ^ 1], cs ? parity0 : parity1)) {
            st_flag(flags + nxt_t, tag);
            nxt_flag_done = true;
        }
        if (!cur.final_phase) __threadfence();  // an LS step: writes visible device-wide
        fence_proxy_async_smem();  // our reads of the stage precede the next bulk copy into it
        __syncthreads();           // stage free again
        if (tid == 0 && !cur.final_phase) atomicAdd(join + cur.r, 1u);
        if (cur.holder) {  // now reserve the next ticket
            if (tid == 0) sh.ticket[(it_no + 1) & 1] = atomicAdd(ctr, 1u);
            __syncthreads();
            nxt_t = sh.ticket[(it_no + 1) & 1];
            if (nxt_t < total && !decode_item(prm, nxt_t, rot, sech, pk, sec, plans, nrot, n, nxt)) {
                if (tid == 0) set_status(sb, IPM_ERR_DEVICE);
                break;
            }
        }
        cur = nxt;
        cur_t = nxt_t;
        cur_loaded = nxt_loaded;
        cur_flag_done = nxt_flag_done;
        pd_cur = pd_nxt;
        pd_nxt.slot = ~0u;
        cs ^= 1;
        ++it_no;
    }
}

// ---------------------------------------------------------------------------------
// Warp-specialized executor: warp 0 is the producer (claims tickets, decodes items,
// waits for an item's earlier LS steps, stages its blocks into a free stage, publishes
// "reads done" as soon as the data has landed), warps 1..15 are the consumers (publish
// "reads done" if the producer has not, wait for the flags their stores depend on,
// store, release the stage).  Two stages; the producer stages the next item while the
// consumers store the current one, and claims the ticket after it as soon as it has
// staged one, so ticket claims and decoding stay off the consumers' path.  Deadlock
// freedom: a claimed item waits only for a stage of its own CTA (and, after LS steps,
// for those steps); the stages hold earlier items, which wait only on earlier tickets;
// a stash holder, the one item that waits on later tickets (of its own exchange), is
// drained before the next claim; and a SINGLE exchange (both stages) waits for both
// stages to drain.  So by induction on the ticket order every claimed item is staged,
// every "reads done" is published and every wait ends.
// ---------------------------------------------------------------------------------

constexpr uint32_t kWsConsumers = 480;  // threads 32..511

// Warp version of decode_item: the exchange holding ticket t by a 32-wide probe of the
// next exchanges, then a 33-way bracket search for longer jumps.
// sec_lane: lane q holds the level's section start q (q <= kSections), kept in registers
// so that finding the section costs one ballot.
__device__ __forceinline__ bool decode_item_warp(const XParams &prm, uint32_t t,
                                                 uint32_t &rot_hint, uint32_t &sec_hint,
                                                 const uint32_t *pk, uint32_t sec_lane,
                                                 const RotPlan *plans, uint32_t nrot,
                                                 uint64_t n, Item &it) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t k =
        uint32_t(__popc(__ballot_sync(0xffffffffu, lane < kSections && sec_lane <= t))) - 1u;
    if (k != sec_hint) {
        sec_hint = k;
        rot_hint = 0;
    }
    const uint32_t ts = t - __shfl_sync(0xffffffffu, sec_lane, k);
    const uint32_t *pf = pk + size_t(k) * (nrot + 1);
    if (pf[rot_hint + 1] <= ts) {
        uint32_t lo = rot_hint + 1;  // pf[lo] <= ts; pf[nrot] = section total > ts
        const uint32_t cand = lo + lane;
        const bool p = cand <= nrot && pf[cand] <= ts;
        const int c = __popc(__ballot_sync(0xffffffffu, p));
        if (c < 32) {
            rot_hint = lo + uint32_t(c) - 1;
        } else {
            lo += 31;
            uint32_t hi = nrot;
            while (hi - lo > 1) {
                const uint32_t R = hi - lo;
                const uint32_t m = lo + uint32_t((uint64_t(R) * (lane + 1)) / 33);
                const bool q = pf[m] <= ts;
                const int cc = __popc(__ballot_sync(0xffffffffu, q));
                const uint32_t m_lo = __shfl_sync(0xffffffffu, m, cc > 0 ? cc - 1 : 0);
                const uint32_t m_hi = __shfl_sync(0xffffffffu, m, cc < 32 ? cc : 31);
                if (cc > 0) lo = m_lo;
                if (cc < 32) hi = m_hi;
            }
            rot_hint = lo;
        }
    }
    const uint32_t r = rot_hint;
    return decode_in_exchange(prm, t, r, ts - pf[r], k, plans[r], n, it);
}

// Producer warp: stage the item's source blocks, then arrive on the stage's "full"
// barrier.  Each range is loaded whole by one bulk copy of the 16-byte lines it
// occupies (its first line from the start, its last line to the end): the copy keeps
// the range's phase in shared memory (element j at offset off + j, as the stores
// expect) and never leaves the lines that hold the range's own elements, so it stays
// within the buffer's pages; the few neighbouring elements it also copies are never
// stored.  No element is loaded with a plain load, so the producer never waits for
// global memory here.
template <typename T>
__device__ __forceinline__ uint32_t line_span_bytes(const T *g, uint32_t len) {
    if (len == 0) return 0;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(g) & ~uintptr_t(15);
    const uintptr_t hi = (reinterpret_cast<uintptr_t>(g + len) + 15) & ~uintptr_t(15);
    return uint32_t(hi - lo);
}

template <typename T>
__device__ __forceinline__ void load_line_span(T *slot, const T *g, uint32_t len,
                                               uint64_t *full) {
    const uint32_t bytes = line_span_bytes(g, len);
    if (bytes)
        bulk_load(slot, reinterpret_cast<const T *>(reinterpret_cast<uintptr_t>(g) &
                                                    ~uintptr_t(15)),
                  bytes, full);
}

template <typename K, bool KV, typename V>
__device__ __forceinline__ void stage_load_ws(const Item &it, const K *buf, const V *vals,
                                              unsigned char *stage, unsigned char *base,
                                              uint64_t *full) {
    using C = XCfg<K, KV, V>;
    K *sk = stage_keys<K, KV>(it, stage, base);
    V *sv = stage_vals<K, KV, V>(it, stage, base);
    if ((threadIdx.x & 31u) != 0) return;
    uint32_t tx = 0;
    for (uint32_t i = 0; i < it.nmoves; ++i) {
        const uint32_t len = uint32_t(it.mv[i].len);
        tx += line_span_bytes(buf + it.mv[i].src, len);
        if (KV) tx += line_span_bytes(vals + it.mv[i].src, len);
    }
    mbar_expect_tx(full, tx);
    for (uint32_t i = 0; i < it.nmoves; ++i) {
        const uint32_t len = uint32_t(it.mv[i].len);
        load_line_span(sk + i * C::kSlotK, buf + it.mv[i].src, len, full);
        if (KV) load_line_span(sv + i * C::kSlotV, vals + it.mv[i].src, len, full);
    }
    mbar_arrive(full);
}

// dst[0, len) = src[0, len) by the consumer threads (ctid < kWsConsumers).
template <typename T>
__device__ __forceinline__ void copy_out_ws(const T *src, T *dst, uint32_t len, uint32_t ctid) {
    constexpr uint32_t U = 8, NT = kWsConsumers;
    uint32_t j0 = 0;
    for (; j0 + U * NT <= len; j0 += U * NT) {
        T v[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) v[u] = src[j0 + u * NT + ctid];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) dst[j0 + u * NT + ctid] = v[u];
    }
    for (uint32_t j = j0 + ctid; j < len; j += NT) dst[j] = src[j];
}

template <typename K, bool KV, typename V>
__device__ __forceinline__ void stage_store_ws(const Item &it, K *buf, V *vals,
                                               unsigned char *stage, unsigned char *base,
                                               uint32_t ctid) {
    using C = XCfg<K, KV, V>;
    const K *sk = stage_keys<K, KV>(it, stage, base);
    const V *sv = stage_vals<K, KV, V>(it, stage, base);
    if (it.single) {  // the whole exchange [X|Y] is staged; write it rotated by |X|
        const Move &mv = it.mv[0];
        const Geo<int(sizeof(K))> gk(buf + mv.src, uint32_t(mv.len));
        const uint32_t m = uint32_t(it.single_m), a = uint32_t(it.single_a);
        const K *k0 = sk + gk.off;
        K *dst = buf + mv.dst;
        for (uint32_t t = ctid; t < m; t += kWsConsumers) {
            uint32_t src = t + a;
            if (src >= m) src -= m;
            dst[t] = k0[src];
        }
        if (KV) {
            const Geo<int(sizeof(V))> gv(vals + mv.src, uint32_t(mv.len));
            const V *v0 = sv + gv.off;
            V *vd = vals + mv.dst;
            for (uint32_t t = ctid; t < m; t += kWsConsumers) {
                uint32_t src = t + a;
                if (src >= m) src -= m;
                vd[t] = v0[src];
            }
        }
        return;
    }
    for (uint32_t i = 0; i < it.nmoves; ++i) {
        const Move &mv = it.mv[i];
        const uint32_t len = uint32_t(mv.len);
        const Geo<int(sizeof(K))> gk(buf + mv.src, len);
        copy_out_ws<K>(sk + i * C::kSlotK + gk.off, buf + mv.dst, len, ctid);
        if (KV) {
            const Geo<int(sizeof(V))> gv(vals + mv.src, len);
            copy_out_ws<V>(sv + i * C::kSlotV + gv.off, vals + mv.dst, len, ctid);
        }
    }
}

__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kWsConsumers) : "memory");
}

struct WsShared {
    Item item[2];
    uint32_t end[2];  // the producer's end marker for the stage
    int abort;        // set by any role on an error
    // the consumers' decisions, written by the lead before the barrier they follow;
    // one variable per barrier, so a slow consumer never sees the next one's value
    int stop_wait, stop_deps;
};

// Lead consumer: wait until flags[lo..hi] all reach tag (empty range: true).  While
// waiting, publish the next stage's item flag as soon as that stage's data has landed
// (its descriptor is read only after the barrier shows the producer's arrival).
// False on timeout.
__device__ bool ws_wait_deps(const uint32_t *flags, uint32_t lo, uint32_t hi, uint32_t tag,
                             uint64_t *nbar, uint32_t nparity, const WsShared *sh,
                             uint32_t ns, uint32_t *wflags, bool &next_pub,
                             unsigned long long lim) {
    auto poll_next = [&]() {
        if (!next_pub && mbar_try_wait(nbar, nparity)) {
            const volatile WsShared *v = sh;
            if (!v->end[ns] && v->item[ns].flag) st_flag(wflags + v->item[ns].ticket, tag);
            next_pub = true;
        }
    };
    poll_next();
    DepTimer tm(lim);
    for (uint32_t q = lo; q <= hi && lo <= hi; ++q) {
        while (ld_flag(flags + q) < tag) {
            poll_next();
            if (tm.expired()) return false;
        }
    }
    return true;
}

template <typename K, bool KV, typename V>
__global__ void __launch_bounds__(512, 1)
    exchange_level_ws_kernel(K *__restrict__ buf, V *__restrict__ vals, uint64_t n,
                             const RotPlan *__restrict__ plans, const uint32_t *__restrict__ pk,
                             const uint32_t *__restrict__ sec, uint32_t nrot,
                             uint32_t *__restrict__ flags,
                             uint32_t *__restrict__ join, uint32_t tag, uint32_t ctr_index,
                             uint32_t holders, StatusBlock *sb) {
    using C = XCfg<K, KV, V>;
    extern __shared__ __align__(128) unsigned char xsmem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(xsmem + 2 * C::kStageSize);
    uint64_t *empty = full + 2;
    __shared__ WsShared sh;
    if (call_finished(sb)) return;
    const unsigned long long lim = wait_limit(sb);
    const uint32_t tid = threadIdx.x;
    const uint32_t total = sec[kSections];
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
        mbar_fence_init();
        sh.abort = 0;
        sh.end[0] = sh.end[1] = 0;
    }
    __syncthreads();

    if (tid < 32) {
        // ------------------------------------------------------------- producer warp
        XParams prm = C::params();
        prm.max_holders = holders;
        const uint32_t lane = tid;
        uint32_t *ctr = &sb->counters[ctr_index];
        uint32_t issued[2] = {0, 0}, drained[2] = {0, 0};
        uint32_t arrivals[2] = {0, 0};  // phases of full[q] the producer has started
        uint32_t rot = 0, sech = 0;
        const uint32_t sec_lane = lane <= kSections ? sec[lane] : ~0u;
        uint32_t st = 0;
        // "reads done" of the items staged last, published (lane 0) as soon as their
        // data has landed, while the producer waits for a stage: the flags never wait
        // for this CTA's consumers to reach the item
        bool pend_on[2] = {false, false};
        uint32_t pend_par[2] = {0, 0}, pend_ticket[2] = {0, 0};
        auto try_publish = [&]() {
            for (uint32_t q = 0; q < 2; ++q)
                if (pend_on[q] && mbar_try_wait(&full[q], pend_par[q])) {
                    st_flag(flags + pend_ticket[q], tag);
                    pend_on[q] = false;
                }
        };
        // wait until every item issued to stage q has been released by the consumers
        auto drain = [&](uint32_t q) -> bool {
            while (drained[q] < issued[q]) {
                bool ok = true;
                if (lane == 0) {
                    unsigned long long t0 = 0;
                    for (uint32_t i = 0;; ++i) {
                        if (mbar_try_wait(&empty[q], drained[q] & 1u)) break;
                        // the consumers left (an error): nothing will be released
                        if (*((volatile int *)&sh.abort)) {
                            ok = false;
                            break;
                        }
                        try_publish();
                        if ((i & 255u) == 0) {
                            const unsigned long long now = globaltimer_ns();
                            if (t0 == 0) {
                                t0 = now;
                            } else if (now - t0 > kWaitLimitNs) {
                                ok = false;
                                break;
                            }
                        }
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
                if (!ok) return false;
                ++drained[q];
            }
            return true;
        };
        // claim and decode the next ticket (the whole warp)
        auto claim = [&](Item &it, uint32_t &t) -> bool {
            t = 0;
            if (lane == 0) t = atomicAdd(ctr, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t < total && !decode_item_warp(prm, t, rot, sech, pk, sec_lane, plans, nrot, n, it)) {
                if (lane == 0) set_status(sb, IPM_ERR_DEVICE);
                return false;
            }
            return true;
        };
        auto fail_timeout = [&]() {
            if (lane == 0) {
                set_status(sb, IPM_ERR_TIMEOUT);
                sh.abort = 1;
            }
        };
        // The next ticket is claimed as soon as the current item is staged, so its
        // claim and decode overlap the wait for a free stage.  A claimed item waits for
        // nothing but a stage of this CTA (and, after LS steps, for those steps), and
        // the stages hold only earlier items that wait on earlier tickets; a stash
        // holder, the one item that waits on later tickets, is drained before the next
        // claim.  So every claimed ticket gets staged and every "reads done" gets
        // published.
        Item it;
        uint32_t t = 0;
        bool ok_claim = claim(it, t);
        for (;;) {
            if (!drain(st)) {
                fail_timeout();
                break;
            }
            if (t >= total || !ok_claim || *((volatile int *)&sh.abort)) {
                // end marker for the consumers in the next stage (free: drained above)
                if (lane == 0) {
                    sh.end[st] = 1;
                    mbar_arrive(&full[st]);
                }
                ++arrivals[st];
                break;
            }
            // a SINGLE exchange spans both stages; an item after LS steps of its
            // exchange waits until they are complete
            bool ok = !it.single || drain(st ^ 1u);
            if (ok && it.before > 0) {
                bool w = true;
                if (lane == 0) w = wait_count(join + it.r, it.before, lim);
                ok = __shfl_sync(0xffffffffu, w, 0) != 0;
            }
            if (!ok) {
                fail_timeout();
                break;
            }
            if (lane == 0) {
                sh.item[st] = it;
                sh.end[st] = 0;
            }
            __syncwarp();
            unsigned char *stage = xsmem + (st ? C::kStageSize : 0);
            stage_load_ws<K, KV, V>(it, buf, vals, stage, xsmem, &full[st]);
            if (lane == 0 && it.flag) {
                pend_on[st] = true;
                pend_par[st] = arrivals[st] & 1u;
                pend_ticket[st] = it.ticket;
            }
            ++arrivals[st];
            ++issued[st];
            if (it.single) ++issued[st ^ 1u];  // the consumers release both stages
            // a stash holder waits on later tickets of its own exchange: claim no ticket
            // that could be parked behind it
            if (it.holder && !drain(st)) {
                fail_timeout();
                break;
            }
            st ^= 1u;
            ok_claim = claim(it, t);
        }
        // leave only once every bulk copy this warp issued has landed (no copy may
        // write the CTA's shared memory after it exits)
        if (lane == 0)
            for (uint32_t q = 0; q < 2; ++q)
                if (arrivals[q] > 0) (void)mbar_wait_bounded(&full[q], (arrivals[q] - 1) & 1u);
        return;
    }

    // ----------------------------------------------------------------- consumers
    // Only the lead waits on the stage barrier and reads the shared error / end state;
    // its decisions are read by all consumers after a barrier, so they always leave the
    // loop together.
    const uint32_t ctid = tid - 32;
    const bool lead = ctid == 0;
    uint32_t fullph[2] = {0, 0};
    uint32_t st = 0;
    bool cur_pub = false;  // lead: the current item's flag was published early
    for (;;) {
        if (lead) {
            int stop = 0;
            // (the producer may leave on an error without marking the stage's end)
            if (!mbar_wait_or_abort(&full[st], fullph[st], &sh.abort)) {
                set_status(sb, IPM_ERR_TIMEOUT);
                sh.abort = 1;
                stop = 1;
            } else if (*((volatile uint32_t *)&sh.end[st]) || *((volatile int *)&sh.abort)) {
                stop = 1;
            }
            sh.stop_wait = stop;
        }
        consumers_sync();  // the stage's data and descriptor are visible to all consumers
        fullph[st] ^= 1u;
        if (sh.stop_wait) break;
        const Item it = sh.item[st];
        if (lead) {
            // reads done: the data is on chip
            if (it.flag && !cur_pub) st_flag(flags + it.ticket, tag);
            // wait for the flags this item's stores depend on, publishing the next
            // stage's flag as soon as its data lands
            const uint32_t ns = st ^ 1u;
            bool next_pub = false;
            bool w = ws_wait_deps(flags, it.dp.lo0, it.dp.hi0, tag, &full[ns], fullph[ns], &sh,
                                  ns, flags, next_pub, lim);
            if (w)
                w = ws_wait_deps(flags, it.dp.lo1, it.dp.hi1, tag, &full[ns], fullph[ns], &sh,
                                 ns, flags, next_pub, lim);
            cur_pub = next_pub;
            int stop = 0;
            if (!w) {
                set_status(sb, IPM_ERR_TIMEOUT);
                sh.abort = 1;
                stop = 1;
            }
            sh.stop_deps = stop;
        }
        consumers_sync();
        if (sh.stop_deps) break;
        unsigned char *stage = xsmem + (st ? C::kStageSize : 0);
        stage_store_ws<K, KV, V>(it, buf, vals, stage, xsmem, ctid);
        if (!it.final_phase) __threadfence();  // an LS step: writes visible device-wide
        fence_proxy_async_smem();  // our reads of the stage precede the next bulk copy into it
        consumers_sync();
        if (lead) {
            if (!it.final_phase) atomicAdd(join + it.r, 1u);
            mbar_arrive(&empty[st]);
            if (it.single) mbar_arrive(&empty[st ^ 1u]);
        }
        st ^= 1u;
    }
}

// Half the resident CTAs of the level kernels (one per SM at least), the base of the
// per-level holder count; the same on the plan side.
uint32_t holder_cap() { return uint32_t(num_sms()) / 2u; }

// WS: the warp-specialized executor; the single-role one moves 4-byte payloads only.
template <typename E, bool KV, bool WS, typename V = uint32_t>
ipm_status exchange_level_t(void *buf, void *vals, uint64_t n, uint32_t l,
                            XPlanArea pa, StatusBlock *sb, cudaStream_t stream) {
    static_assert(WS || sizeof(V) == 4, "the single-role executor moves 4-byte payloads");
    using C = XCfg<E, KV, V>;
    using Kern = void (*)(E *, V *, uint64_t, const RotPlan *, const uint32_t *,
                          const uint32_t *, uint32_t, uint32_t *, uint32_t *, uint32_t, uint32_t,
                          uint32_t, StatusBlock *);
    Kern kern;
    if constexpr (WS)
        kern = exchange_level_ws_kernel<E, KV, V>;
    else
        kern = exchange_level_kernel<E, KV>;
    static std::atomic<int> grid_cache{0};  // set once; a racing first call repeats it
    int grid = grid_cache.load(std::memory_order_relaxed);
    if (grid == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(C::kSmem)) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::kThreads,
                                                          C::kSmem) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        if (per_sm < 1) per_sm = 1;
        grid = per_sm * num_sms();
        grid_cache.store(grid, std::memory_order_relaxed);
    }
    const uint64_t R = 1ull << l;
    const RotPlan *plans = reinterpret_cast<const RotPlan *>(pa.plans) + (R - 1);
    const uint32_t *pk = pa.item_pf + level_prefix_offset(l);
    const uint32_t *sec = pa.sec_start + level_section_offset(l);
    kern<<<grid, C::kThreads, C::kSmem, stream>>>((E *)buf, (V *)vals, n, plans, pk, sec,
                                                  uint32_t(R),
                                                  pa.flags, pa.join + (R - 1), l + 1,
                                                  kTicketCounter0 + l,
                                                  level_holders(l, holder_cap()), sb);
    return last_launch_status();
}

}  // namespace

template <typename E>
XParams params_by_payload(uint32_t vb) {
    return vb == 8   ? XCfg<E, true, uint64_t>::params()
           : vb != 0 ? XCfg<E, true, uint32_t>::params()
                     : XCfg<E, false>::params();
}

XParams exchange_params(ipm_dtype key, uint32_t vb) {
    switch (key) {
    case IPM_INT32:
    case IPM_UINT32:
    case IPM_FLOAT32:
        return params_by_payload<int32_t>(vb);
    case IPM_UINT64:
    case IPM_INT64:  // moved, never compared
        return params_by_payload<uint64_t>(vb);
    }
    return XParams{1, 2, 1, 1, 1};
}

size_t xplan_area_bytes(uint32_t G, uint64_t n, ipm_dtype key, uint32_t vb) {
    if (G == 0) G = 1;
    const uint64_t P = 1ull << G;
    const XParams prm = exchange_params(key, vb);
    size_t b = 0;
    b += align_up(sizeof(RotPlan) * P, 256);                  // plans of all levels
    b += align_up(sizeof(uint32_t) * prefix_entries(G), 256);   // item prefixes
    b += align_up(sizeof(uint32_t) * section_entries(G), 256);  // section starts
    b += align_up(sizeof(uint32_t) * P, 256);                 // per-exchange completion
    b += align_up(sizeof(uint32_t) * max_level_items(G, n, prm), 256);  // read flags
    return b;
}

uint64_t max_level_items(uint32_t G, uint64_t n, const XParams &prm) {
    // per exchange: tiles of its LS steps and of its final phase (<= 2 m / pair_tile + 2
    // per phase), at most n / (cap * kMinHolders) LS steps in all, and its holders: a
    // level's R exchanges hold at most max(kMinHolders R, kMaxHoldersCap) of them
    (void)prm.max_holders;
    const uint64_t R = 1ull << (G ? G - 1 : 0);
    return 2 * n / prm.pair_tile + n / (uint64_t(prm.cap) * kMinHolders) +
           R * (kMinHolders + 6) + kMaxHoldersCap + 16;
}

XPlanArea xplan_area_at(void *base, uint32_t G, uint64_t n, ipm_dtype key, uint32_t vb) {
    if (G == 0) G = 1;
    const uint64_t P = 1ull << G;
    const XParams prm = exchange_params(key, vb);
    char *p = static_cast<char *>(base);
    XPlanArea pa;
    pa.plans = p;
    p += align_up(sizeof(RotPlan) * P, 256);
    pa.item_pf = reinterpret_cast<uint32_t *>(p);
    p += align_up(sizeof(uint32_t) * prefix_entries(G), 256);
    pa.sec_start = reinterpret_cast<uint32_t *>(p);
    p += align_up(sizeof(uint32_t) * section_entries(G), 256);
    pa.join = reinterpret_cast<uint32_t *>(p);
    p += align_up(sizeof(uint32_t) * P, 256);
    pa.flags = reinterpret_cast<uint32_t *>(p);
    pa.nflags = max_level_items(G, n, prm);
    pa.zero_bytes = size_t(reinterpret_cast<char *>(pa.flags) - reinterpret_cast<char *>(pa.join)) +
                    sizeof(uint32_t) * pa.nflags;
    return pa;
}

ipm_status launch_xplan_levels(const uint64_t *split, uint64_t n, uint32_t G,
                               uint32_t levels, XPlanArea pa, ipm_dtype key, uint32_t vb,
                               StatusBlock *sb, cudaStream_t stream) {
    if (G == 0 || levels == 0) return IPM_OK;
    if (levels > G) levels = G;
    // completion counters and read flags start at zero on every call
    IPM_CUDA_TRY(cudaMemsetAsync(pa.join, 0, pa.zero_bytes, stream));
    const uint32_t elem = uint32_t(dtype_bytes(key)) + vb;
    xplan_levels_kernel<<<levels, kPlanThreads, 0, stream>>>(split, n, G, pa,
                                                             exchange_params(key, vb),
                                                             holder_cap(), elem, sb);
    return last_launch_status();
}

ipm_status launch_xplan_single(uint64_t lx, uint64_t ly, XPlanArea pa, ipm_dtype key,
                               cudaStream_t stream) {
    IPM_CUDA_TRY(cudaMemsetAsync(pa.join, 0, pa.zero_bytes, stream));
    xplan_single_kernel<<<1, 32, 0, stream>>>(lx, ly, pa, exchange_params(key, 0u),
                                               holder_cap());
    return last_launch_status();
}

uint32_t g_exchange_engine = 1;

ipm_status launch_exchange_level(void *buf, void *vals, uint32_t vb, ipm_dtype key,
                                 uint64_t n, uint32_t l, XPlanArea pa, StatusBlock *sb,
                                 cudaStream_t stream) {
    // 8-byte payloads always go through the warp-specialized executor
    const bool ws = g_exchange_engine == 1 || vb == 8;
    const bool four = dtype_bytes(key) == 4;
    if (dtype_bytes(key) == 0) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (vb == 8)
        return four ? exchange_level_t<int32_t, true, true, uint64_t>(buf, vals, n, l, pa, sb,
                                                                      stream)
                    : exchange_level_t<uint64_t, true, true, uint64_t>(buf, vals, n, l, pa, sb,
                                                                       stream);
    const bool kv = vb != 0;
    if (four) {
        if (ws)
            return kv ? exchange_level_t<int32_t, true, true>(buf, vals, n, l, pa, sb, stream)
                      : exchange_level_t<int32_t, false, true>(buf, vals, n, l, pa, sb, stream);
        return kv ? exchange_level_t<int32_t, true, false>(buf, vals, n, l, pa, sb, stream)
                  : exchange_level_t<int32_t, false, false>(buf, vals, n, l, pa, sb, stream);
    }
    // 8-byte keys (uint64, int64): moved, never compared
    if (ws)
        return kv ? exchange_level_t<uint64_t, true, true>(buf, vals, n, l, pa, sb, stream)
                  : exchange_level_t<uint64_t, false, true>(buf, vals, n, l, pa, sb, stream);
    return kv ? exchange_level_t<uint64_t, true, false>(buf, vals, n, l, pa, sb, stream)
              : exchange_level_t<uint64_t, false, false>(buf, vals, n, l, pa, sb, stream);
}

}  // namespace ipm
