// Decomposition of one partition exchange [X|Y] -> [Y|X] (Sec. 3.4) into GPU work
// items, shared by the plan kernel (counting) and the exchange kernel (executing).
//
// The exchange follows linear shifting (LS): while both the size difference
// e = |a-b| and the smaller block exceed what the on-chip stash can hold, one LS step
// swaps the smaller block into its final place (a fully parallel block swap) and the
// same problem remains on the rest.  Once the rest is small enough, the remaining LS
// steps are executed in closed form in a single pass, reading and writing every
// element exactly once:
//   PAIR   (e small)    X'[t] -> B'+t and Y'[t] -> t for the B' = min(a,b) pairs; the
//                       e = |a-b| extra elements of the bigger block are held on chip
//                       (the "stash") and written last.  This is the first LS swap
//                       fused with the closed form of all the small-block steps after it.
//   SHIFT  (min small)  the smaller block is held on chip, the bigger block moves by its
//                       size, the stash lands at the other end (the closed form of a run
//                       of LS steps that all swap the same small block).
//   SWAP   (a == b)     one pairwise swap, no stash (Sec. 3.5: exactly L_A swaps).
//   SINGLE (a+b small)  one CTA loads the whole exchange on chip and writes it rotated.
// PAIR and SHIFT run in "primed" coordinates: mirrored (p -> m-1-p) when needed so the
// big block (PAIR) or the small block (SHIFT) comes first; a mirrored contiguous range
// is still a contiguous physical range, so every access stays coalesced.
#pragma once

#include <stdint.h>

namespace ipm {

enum : uint32_t { XK_NONE = 0, XK_SWAP = 1, XK_SINGLE = 2, XK_PAIR = 3, XK_SHIFT = 4 };

// Engine constants of one (key type, payload) instantiation.
struct XParams {
    uint32_t pair_tile;    // pairs per PAIR / SWAP tile
    uint32_t shift_tile;   // elements per SHIFT tile
    uint32_t cap;          // stash capacity of one CTA, in elements
    uint32_t max_holders;  // stash CTAs per exchange (must stay below the resident CTAs)
    uint32_t single_cap;   // largest exchange one CTA stages whole (SINGLE)
};

// One phase of an exchange.  (s, a, b): the exchange [X|Y] the phase works on.
struct XPhase {
    uint32_t kind;
    uint32_t mirror;
    uint64_t s, a, b;
    uint64_t delta;    // stash size (PAIR: |a-b|, SHIFT: min(a,b))
    uint32_t holders;  // stash items (PAIR, SHIFT)
    uint32_t tiles;    // tile items
    bool final_phase;
    __host__ __device__ uint32_t items() const {
        return kind == XK_SINGLE ? 1u : holders + tiles;
    }
};

__host__ __device__ inline uint64_t xdiv_up(uint64_t x, uint64_t y) { return (x + y - 1) / y; }

// The phase of exchange (s, a, b) in its current state.  Returns false when there is
// nothing left to do (a or b empty).
__host__ __device__ inline bool x_phase(const XParams &P, uint64_t s, uint64_t a, uint64_t b,
                                        XPhase &ph) {
    if (a == 0 || b == 0) return false;
    const uint64_t m = a + b;
    ph.s = s;
    ph.a = a;
    ph.b = b;
    ph.mirror = 0;
    ph.delta = 0;
    ph.holders = 0;
    ph.final_phase = true;
    const uint64_t mn = a < b ? a : b;
    const uint64_t e = a > b ? a - b : b - a;
    if (m <= P.single_cap) {
        ph.kind = XK_SINGLE;
        ph.tiles = 0;
        return true;
    }
    if (e == 0) {
        ph.kind = XK_SWAP;
        ph.tiles = uint32_t(xdiv_up(mn, P.pair_tile));
        return true;
    }
    const uint64_t budget = uint64_t(P.cap) * P.max_holders;
    if (e <= mn && e <= budget) {
        ph.kind = XK_PAIR;
        ph.mirror = a < b ? 1u : 0u;  // big block first
        ph.delta = e;
        ph.holders = uint32_t(xdiv_up(e, P.cap));
        ph.tiles = uint32_t(xdiv_up(mn, P.pair_tile));
        return true;
    }
    if (mn <= budget) {
        ph.kind = XK_SHIFT;
        ph.mirror = a > b ? 1u : 0u;  // small block first
        ph.delta = mn;
        ph.holders = uint32_t(xdiv_up(mn, P.cap));
        ph.tiles = uint32_t(xdiv_up(m - mn, P.shift_tile));
        return true;
    }
    // One LS step: swap the smaller block into its final place.
    ph.kind = XK_SWAP;
    ph.tiles = uint32_t(xdiv_up(mn, P.pair_tile));
    ph.final_phase = false;
    return true;
}

// State after a non-final LS step of phase ph.
__host__ __device__ inline void x_after_step(const XPhase &ph, uint64_t &s, uint64_t &a,
                                             uint64_t &b) {
    s = ph.s;
    a = ph.a;
    b = ph.b;
    if (a > b) {  // [Y | X_tail | X_head]: rotate [X_tail | X_head] at s+b
        s += b;
        a -= b;
    } else {  // [Y_tail | Y_head | X]: rotate [Y_tail | Y_head] at s
        b -= a;
    }
}

// Total items and algorithmic bytes (elem = bytes per element incl. payload) of one
// exchange.
__host__ __device__ inline void x_count(const XParams &P, uint64_t s, uint64_t a, uint64_t b,
                                        uint32_t elem, uint64_t &items, uint64_t &bytes) {
    items = 0;
    bytes = 0;
    XPhase ph;
    while (x_phase(P, s, a, b, ph)) {
        items += ph.items();
        const uint64_t mn = ph.a < ph.b ? ph.a : ph.b;
        bytes += (ph.kind == XK_SWAP ? 4 * mn : 2 * (ph.a + ph.b)) * elem;
        if (ph.final_phase) break;
        x_after_step(ph, s, a, b);
    }
}

}  // namespace ipm
