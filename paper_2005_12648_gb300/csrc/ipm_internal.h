// Internal launcher interface between the C ABI (ipm_api.cu) and the kernel files.
#pragma once

#include "ipm_common.cuh"

namespace ipm {

// One contiguous range of a reversal pass: elements [start, start + len).
struct Seg {
    uint64_t start;
    uint64_t len;
};

// Reversal work is cut into units of kRevUnit element pairs.
constexpr uint32_t kRevThreads = 256;
constexpr uint32_t kRevItems = 8;
constexpr uint64_t kRevUnit = uint64_t(kRevThreads) * kRevItems;

// Per-level exchange plans, all levels in one area of the workspace.  Level l
// (2^l rotations) owns
//   seg1[2(2^l-1) .. +2^{l+1})   pass 1: X_r and Y_r of rotation r
//   pf1 [2(2^l-1) + l .. +2^{l+1}+1)  unit prefix of pass 1
//   seg2[(2^l-1) .. +2^l)        pass 2: the whole middle X_r|Y_r
//   pf2 [(2^l-1) + l .. +2^l+1)  unit prefix of pass 2
struct PlanArea {
    Seg *seg1;
    uint32_t *pf1;
    Seg *seg2;
    uint32_t *pf2;
};

inline uint64_t seg1_base(uint32_t l) { return 2ull * ((1ull << l) - 1); }
inline uint64_t pf1_base(uint32_t l) { return 2ull * ((1ull << l) - 1) + l; }
inline uint64_t seg2_base(uint32_t l) { return (1ull << l) - 1; }
inline uint64_t pf2_base(uint32_t l) { return ((1ull << l) - 1) + l; }

// Bytes of a PlanArea for G levels (each array 256-byte aligned).
size_t plan_area_bytes(uint32_t G);
PlanArea plan_area_at(void *base, uint32_t G);

// Tile (pair) capacity of the shared-memory merge, in elements.
uint64_t tile_capacity(ipm_dtype key, bool with_values);

// ---- launchers (all asynchronous on `stream`; return IPM_ERR_CUDA on launch failure)

// Resets the status block and sets its early-exit flag when A is empty, B is empty
// or A[last] <= B[0].
ipm_status launch_early_exit(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                             StatusBlock *sb, cudaStream_t stream);

// Exact stable splits on d_k = floor(k*n/P), k = 0..P.  sb may be NULL.
ipm_status launch_splits(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                         uint64_t P, uint64_t *split, const StatusBlock *sb,
                         cudaStream_t stream);

// Plans of all G levels from a split table with P = 2^G.
ipm_status launch_plan_levels(const uint64_t *split, uint64_t n, uint32_t G,
                              PlanArea pa, const StatusBlock *sb, cudaStream_t stream);

// Plan of a single exchange [X|Y] at offset 0 (G = 1 layout, level 0).
ipm_status launch_plan_single(uint64_t lx, uint64_t ly, PlanArea pa, cudaStream_t stream);

// The two reversal passes of level l (the exchange of every middle pair).
ipm_status launch_level_exchange(void *buf, uint32_t *vals, int elem_bytes, uint64_t n,
                                 uint32_t l, PlanArea pa, StatusBlock *sb,
                                 cudaStream_t stream);

// Per-pair shared-memory merge of an arranged buffer.
ipm_status launch_tile_merge(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                             ipm_dtype key, const uint64_t *split, uint32_t G,
                             StatusBlock *sb, cudaStream_t stream);

}  // namespace ipm
