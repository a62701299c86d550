// Internal launcher interface between the C ABI (ipm_api.cu) and the kernel files.
#pragma once

#include "ipm_common.cuh"

namespace ipm {

// Sections of a level's ticket order (ipm_exchange.cu): section k < kSections - 1
// holds phase k of every exchange, the last one every later phase.
constexpr uint32_t kSections = 8;
// Level l's per-section exchange prefixes: kSections arrays of 2^l + 1 entries.
__host__ __device__ inline uint64_t level_prefix_offset(uint32_t l) {
    return uint64_t(kSections) * ((1ull << l) - 1 + l);
}
// Level l's section starts: kSections + 1 entries.
__host__ __device__ inline uint64_t level_section_offset(uint32_t l) {
    return uint64_t(l) * (kSections + 1);
}
inline uint64_t prefix_entries(uint32_t G) { return level_prefix_offset(G); }
inline uint64_t section_entries(uint32_t G) { return uint64_t(G) * (kSections + 1); }

// Exchange plans of all levels in one workspace area (see ipm_exchange.cu).
struct XPlanArea {
    void *plans;          // RotPlan per exchange, level l at offset 2^l - 1
    uint32_t *item_pf;    // per-section item prefixes, level l at level_prefix_offset(l)
    uint32_t *sec_start;  // section starts, level l at level_section_offset(l)
    uint32_t *join;     // per-exchange completed-item counters, level l at 2^l - 1
    uint32_t *flags;    // per-item "reads done" flags, shared by the levels
    uint64_t nflags;
    size_t zero_bytes;  // join .. end of flags, cleared on every call
};

struct XParams;
// vb: payload bytes per element (0: keys only, 4, 8); payloads are moved, never compared.
XParams exchange_params(ipm_dtype key, uint32_t vb);
uint64_t max_level_items(uint32_t G, uint64_t n, const XParams &prm);
size_t xplan_area_bytes(uint32_t G, uint64_t n, ipm_dtype key, uint32_t vb);
XPlanArea xplan_area_at(void *base, uint32_t G, uint64_t n, ipm_dtype key, uint32_t vb);

// Tile (pair) capacity of the shared-memory merge, in elements.
uint64_t tile_capacity(ipm_dtype key, uint32_t vb);

// ---- launchers (all asynchronous on `stream`; return IPM_ERR_CUDA on launch failure)

// Resets the status block, stores the call's limit for waits on other CTAs (0: the
// default) and sets the early-exit flag when A is empty, B is empty or A[last] <= B[0].
ipm_status launch_early_exit(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                             StatusBlock *sb, unsigned long long wait_limit_ns,
                             cudaStream_t stream);

// Exact stable splits on d_k = floor(k*n/P), k = 0..P.  sb may be NULL.  Many diagonals
// take two launches (split_launches): every 32nd diagonal first, then the others inside
// the brackets their coarse neighbours give.
uint32_t split_launches(uint64_t P);
// The same for the learned splits (launch_learned_splits).
uint32_t learned_split_launches(uint64_t P);
ipm_status launch_splits(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                         uint64_t P, uint64_t *split, const StatusBlock *sb,
                         cudaStream_t stream);

// Plans (and zeroed flags) of the first `levels` of the G levels of a split table with
// P = 2^G; only the planned levels add to the status block's exchange bytes.
ipm_status launch_xplan_levels(const uint64_t *split, uint64_t n, uint32_t G,
                               uint32_t levels, XPlanArea pa, ipm_dtype key, uint32_t vb,
                               StatusBlock *sb, cudaStream_t stream);

// Plan of a single exchange [X|Y] at offset 0 (level 0 of a G = 1 layout).
ipm_status launch_xplan_single(uint64_t lx, uint64_t ly, XPlanArea pa, ipm_dtype key,
                               cudaStream_t stream);

// Exchange executor of launch_exchange_level: 0 = every thread in every role,
// 1 = warp-specialized (a producer warp stages, 15 consumer warps store).
extern uint32_t g_exchange_engine;

// The exchanges of level l, one persistent launch.
ipm_status launch_exchange_level(void *buf, void *vals, uint32_t vb, ipm_dtype key,
                                 uint64_t n, uint32_t l, XPlanArea pa, StatusBlock *sb,
                                 cudaStream_t stream);

// The last log2_cluster levels fused with the pair merge (ipm_cluster_merge.cu): run
// after levels 0 .. G - log2_cluster - 1; clusters of 2^log2_cluster CTAs.
// (4-byte payloads only: vals is NULL or uint32_t *.)
ipm_status launch_cluster_merge(void *buf, uint32_t *vals, uint64_t la, uint64_t lb,
                                ipm_dtype key, const uint64_t *split, uint32_t G,
                                uint32_t log2_cluster, StatusBlock *sb, cudaStream_t stream);
// The largest F <= wanted whose clusters of 2^F CTAs the device can schedule (0: none).
uint32_t usable_fused_levels(ipm_dtype key, bool with_values, uint32_t wanted);
// Pair capacity of the fused kernels' tile (half the plain merge's tile).
uint64_t cluster_tile_capacity(ipm_dtype key, uint32_t vb);
// The same fusion with a group barrier in global memory: groups of 2^F pairs taken from
// a ticket (gctr: (2^G >> F) uint32 group counters in the workspace, zeroed here).
ipm_status launch_group_merge(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                              ipm_dtype key, const uint64_t *split, uint32_t G, uint32_t F,
                              uint32_t *gctr, StatusBlock *sb, cudaStream_t stream);
// The largest F <= wanted with at least 2^F resident CTAs of the group kernel.
uint32_t usable_group_levels(ipm_dtype key, uint32_t vb, uint32_t wanted);

// Two pairs per CTA, the first merged pair parked in TMEM (every key type, with or
// without payload), each pair written once the pairs reading its destination have
// counted their slices in (gctr: one count per pair, zeroed here): groups of 2^F pairs
// need 2^(F-1) resident CTAs.
ipm_status launch_group2_merge(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                               ipm_dtype key, const uint64_t *split, uint32_t G, uint32_t F,
                               uint32_t *gctr, StatusBlock *sb, cudaStream_t stream);
// The largest F <= wanted the two-pairs kernel can run (0: not for this key / payload).
uint32_t usable_group2_levels(ipm_dtype key, uint32_t vb, uint32_t wanted);

// Division of Alg. 3 to 2^depth pairs (ipm_division.cu): the pair boundaries only.
ipm_status launch_division(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                           uint32_t depth, uint32_t kind, uint64_t *ia, uint64_t *jb,
                           cudaStream_t stream);

// Circular-shifting exchange (ipm_cs_rotate.cu): g = gcd(lx, ly) cycles of L = n / g
// positions, cut into segments of S steps (W segments, each with a saved first value)
// unless every cycle fits one worker (whole).
struct CsPlan {
    uint64_t lx, n, g, L, S, W;
    bool whole;
};
// The division stage by one permutation (sOptMov): workspace bytes for n elements of kb
// key bytes and vb payload bytes, and the rounds themselves (host-synchronous).
size_t permute_workspace_bytes(uint64_t n, uint32_t kb, uint32_t vb);
ipm_status launch_permute(void *buf, void *vals, uint32_t kb, uint32_t vb, uint64_t la,
                          uint64_t lb, const uint64_t *split, uint32_t G, void *ws,
                          cudaStream_t st);

CsPlan cs_plan(uint64_t lx, uint64_t ly);
ipm_status launch_cs_rotate(void *ptr, uint32_t elem_bytes, const CsPlan &pl, void *save,
                            cudaStream_t stream);

// Per-pair shared-memory merge of an arranged buffer.
ipm_status launch_tile_merge(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                             ipm_dtype key, const uint64_t *split, uint32_t G,
                             StatusBlock *sb, cudaStream_t stream);

// Batched segmented merge (ipm_batched.cu): workspace layout, queue preparation and
// the levels + merge kernels.  variant 0 = wide, 1 = narrow, 2 = quarter merge tile.
struct BatchedLayout {
    size_t hist_off, queue_off, multi_off, soff_off, pool_off, total;
    uint64_t pool_cap;
};
uint64_t batched_tile(ipm_dtype key, bool with_values, uint32_t variant);
uint64_t batched_max_segment(ipm_dtype key, bool with_values, uint32_t variant);
BatchedLayout batched_layout(uint64_t buf_len, uint32_t nseg, uint64_t tile);
// one_launch: the one-launch form (a memset node, then one persistent kernel), else
// three launches (queue preparation, levels, merges).
ipm_status launch_batched(void *buf, uint32_t *vals, uint64_t buf_len, ipm_dtype key,
                          const ipm_segment *segs, uint32_t nseg, void *ws,
                          const BatchedLayout &L, uint32_t by_size, uint32_t variant,
                          uint32_t ctas_per_sm, uint32_t one_launch, cudaStream_t stream);

// Learned split proposer (ipm_learned.cu).
ipm_status launch_learned_splits(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                                 uint64_t P, const ipm_split_model *model, uint64_t *split,
                                 ipm_split_stats *stats, const StatusBlock *sb,
                                 cudaStream_t stream);
size_t split_model_train_ws_bytes(uint32_t nsamples);
ipm_status launch_split_model_train(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                                    const uint64_t *diags, uint32_t n,
                                    const ipm_split_train_options &opt,
                                    ipm_split_model *model, void *ws, cudaStream_t stream);
ipm_status launch_split_model_forward(const ipm_split_model *model, const float *x, uint32_t n,
                                      float *y, cudaStream_t stream);
ipm_status launch_split_model_loss_grad(const ipm_split_model *model, const float *x,
                                        const float *t, uint32_t n, float *grad,
                                        cudaStream_t stream);

}  // namespace ipm
