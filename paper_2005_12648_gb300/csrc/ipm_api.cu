// The extern "C" entry points of include/ipmerge.h: argument checks, workspace layout
// and the launch sequence of the hot path (split -> level exchanges -> pair merge).
#include <cstddef>
#include <vector>

#include "ipm_exchange.cuh"
#include "ipm_internal.h"

namespace ipm {

int num_sms() {
    static std::atomic<int> cached[64];  // zero-initialised; a racing first call repeats it
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < 64) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v <= 0) {
        (void)cudaGetLastError();
        v = 1;
    }
    if (dev >= 0 && dev < 64) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

ipm_status last_launch_status() {
    return cudaGetLastError() == cudaSuccess ? IPM_OK : IPM_ERR_CUDA;
}

namespace {

// ---- optional per-phase timing (ipm_timing_enable / ipm_timing_read), per host thread
struct TimingRec {
    int phase;
    uint32_t launches;
    cudaEvent_t a, b;
};
struct TimingState {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;
    std::vector<TimingRec> recs;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return e;
    }
};
thread_local TimingState g_timing;

// Records an event pair around one launch group when timing is enabled.
class PhaseScope {
  public:
    PhaseScope(int phase, uint32_t launches, cudaStream_t s) : s_(s) {
        if (!g_timing.enabled) return;
        rec_.phase = phase;
        rec_.launches = launches;
        rec_.a = g_timing.get();
        rec_.b = g_timing.get();
        if (rec_.a && rec_.b && cudaEventRecord(rec_.a, s_) == cudaSuccess) on_ = true;
    }
    ~PhaseScope() {
        if (!on_) return;
        if (cudaEventRecord(rec_.b, s_) == cudaSuccess)
            g_timing.recs.push_back(rec_);
        else
            (void)cudaGetLastError();
    }

  private:
    cudaStream_t s_;
    TimingRec rec_{};
    bool on_ = false;
};

constexpr uint32_t kMaxLog2Pairs = 22;

// Bottom levels of the division stage fused with the pair merge (ipm_set_fused_levels)
// and how the groups synchronise: 0 = thread-block clusters (F <= 4), 1 = group
// barriers in global memory (ipm_set_fused_engine).
uint32_t g_fused_levels = 10;  // as many as the engine can (8 or 9 on GB300)
// Limit of the merge calls' waits on other CTAs (ipm_set_wait_limit_ns; 0 = 2 s).
std::atomic<unsigned long long> g_wait_limit_ns{0};
uint32_t g_fused_engine = 2;  // TMEM two-pairs kernel where it applies, else 1

bool valid_key(ipm_dtype t) {
    return t == IPM_INT32 || t == IPM_UINT32 || t == IPM_UINT64 || t == IPM_FLOAT32 ||
           t == IPM_INT64;
}

// Smallest G with 2^G * tile >= n.
uint32_t auto_log2_pairs(uint64_t n, uint64_t tile) {
    uint32_t G = 0;
    while ((uint64_t(1) << G) * tile < n) ++G;
    return G;
}

// Checks shared by the merge entry points; resolves G.
// vb: payload bytes per element (0 keys only, 4 or 8).
ipm_status check_merge_args(uint64_t la, uint64_t lb, ipm_dtype key, uint32_t vb,
                            uint32_t log2_pairs, uint32_t *G_out) {
    if (!valid_key(key)) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (vb != 0 && vb != 4 && vb != 8) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (la > (uint64_t(1) << 40) || lb > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    const uint64_t n = la + lb;
    const uint64_t tile = tile_capacity(key, vb);
    const uint32_t G = log2_pairs ? log2_pairs : auto_log2_pairs(n, tile);
    if (G > kMaxLog2Pairs) return IPM_ERR_INVALID_ARG;
    // every pair must fit one tile: ceil(n / 2^G) <= tile
    if (((n + (uint64_t(1) << G) - 1) >> G) > tile) return IPM_ERR_INVALID_ARG;
    *G_out = G;
    return IPM_OK;
}

// Kernel variant of a batched options struct (NULL = defaults): 0 wide, 1 narrow,
// 2 quarter tile; and whether the one-launch form runs.
constexpr uint32_t kDefaultBatchedVariant = 1;
constexpr uint32_t kDefaultBatchedOneLaunch = 0;

ipm_status batched_variant(const ipm_batched_options *opt, uint32_t *variant,
                           uint32_t *one_launch = nullptr) {
    *variant = kDefaultBatchedVariant;
    if (one_launch) *one_launch = kDefaultBatchedOneLaunch;
    if (opt == nullptr) return IPM_OK;
    if (opt->tile > 3 || opt->order > 1 || opt->form > 2 || opt->ctas_per_sm > 64)
        return IPM_ERR_INVALID_ARG;
    *variant = opt->tile == 0 ? kDefaultBatchedVariant : opt->tile - 1;
    if (one_launch && opt->form != 0) *one_launch = opt->form == 2 ? 1u : 0u;
    return IPM_OK;
}

struct MergeLayout {
    size_t split_off, group_off, plan_off, total;
};

// status block | split table (P+1) | group counters (P) | exchange plans
MergeLayout merge_layout(uint32_t G, uint64_t n, ipm_dtype key, uint32_t vb) {
    MergeLayout L;
    const uint64_t P = uint64_t(1) << G;
    L.split_off = kStatusBytes;
    L.group_off = L.split_off + align_up(sizeof(uint64_t) * (P + 1), 256);
    L.plan_off = L.group_off + align_up(sizeof(uint32_t) * P, 256);
    L.total = L.plan_off + xplan_area_bytes(G, n, key, vb);
    return L;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// The with_values argument of the queries: 0 keys only, 1 or 4 a 4-byte payload, 8 an
// 8-byte payload; anything else is returned as 1 (rejected by check_merge_args).
uint32_t payload_bytes(int with_values) {
    if (with_values == 0) return 0;
    if (with_values == 1 || with_values == 4) return 4;
    return with_values == 8 ? 8u : 1u;
}

// The fused engine and level count a merge with 2^G plain pairs uses: the selected
// engine where it applies (the cluster kernels move 4-byte payloads, so 8-byte ones take
// the group barrier; the two-pairs TMEM kernel takes every key type and payload, the
// group barrier only where it cannot keep two CTAs on an SM), and the most levels it can
// fuse up to the setting.
struct FusedChoice {
    uint32_t engine, levels;
};
FusedChoice fused_choice(ipm_dtype key, uint32_t vb, uint32_t G) {
    const uint32_t Fwant = g_fused_levels < G + 1 ? g_fused_levels : G + 1;
    if (g_fused_engine == 0 && vb != 8)
        return {0u, usable_fused_levels(key, vb != 0, Fwant > 4 ? 4 : Fwant)};
    if (g_fused_engine == 2) {
        const uint32_t f2 = usable_group2_levels(key, vb, Fwant);
        if (f2 > 0) return {2u, f2};
    }
    return {1u, usable_group_levels(key, vb, Fwant)};
}

ipm_status merge_core(void *buf, void *vals, uint32_t vb, uint64_t la, uint64_t lb,
                      ipm_dtype key, uint32_t log2_pairs, void *ws, size_t ws_bytes,
                      cudaStream_t stream, const ipm_split_model *model = nullptr) {
    if (vals == nullptr) vb = 0;
    uint32_t G = 0;
    IPM_TRY(check_merge_args(la, lb, key, vb, log2_pairs, &G));
    if (la + lb == 0) return IPM_OK;
    if (buf == nullptr || ws == nullptr) return buf ? IPM_ERR_WORKSPACE : IPM_ERR_INVALID_ARG;
    if (!aligned(buf, size_t(dtype_bytes(key))) || (vb && !aligned(vals, vb)))
        return IPM_ERR_ALIGNMENT;
    if (!aligned(ws, 256)) return IPM_ERR_ALIGNMENT;
    const uint64_t n = la + lb;
    // The fused path (the last F levels done by groups of CTAs with half-size tiles:
    // thread-block clusters for F <= 4 when selected, else global-memory group
    // barriers) splits one level deeper: every pair then fits the half tile.
    const FusedChoice fc = fused_choice(key, vb, G);
    const bool use_clusters = fc.engine == 0, use_tmem = fc.engine == 2;
    const uint32_t F = fc.levels;
    const uint32_t Gs = F > 0 ? G + 1 : G;  // depth of the split table
    const MergeLayout L = merge_layout(Gs, n, key, vb);
    if (ws_bytes < L.total) return IPM_ERR_WORKSPACE;
    char *w = static_cast<char *>(ws);
    StatusBlock *sb = reinterpret_cast<StatusBlock *>(w);
    uint64_t *split = reinterpret_cast<uint64_t *>(w + L.split_off);
    const XPlanArea pa = xplan_area_at(w + L.plan_off, Gs, n, key, vb);
    const uint64_t P = uint64_t(1) << Gs;

    {
        PhaseScope ps(model ? 6 : 0,
                      1u + (model ? learned_split_launches(P) : split_launches(P)), stream);
        // a0: early exit (A empty, B empty, or A[last] <= B[0]) -> later steps are no-ops
        IPM_TRY(launch_early_exit(buf, la, lb, key, sb,
                                  g_wait_limit_ns.load(std::memory_order_relaxed), stream));
        // a1: exact stable splits on every diagonal (from the model's proposals when one
        // is given: the same splits)
        if (model != nullptr)
            IPM_TRY(launch_learned_splits(buf, la, lb, key, P, model, split, nullptr, sb,
                                          stream));
        else
            IPM_TRY(launch_splits(buf, la, lb, key, P, split, sb, stream));
    }
    // a2: division stage, one exchange level at a time; the last F levels are fused
    // with the pair merge (clusters of 2^F CTAs)
    if (Gs > F) {
        PhaseScope ps(1, 1, stream);
        IPM_TRY(launch_xplan_levels(split, n, Gs, Gs - F, pa, key, vb, sb, stream));
    }
    for (uint32_t l = 0; l + F < Gs; ++l) {
        PhaseScope ps(2, 1, stream);
        IPM_TRY(launch_exchange_level(buf, vals, vb, key, n, l, pa, sb, stream));
    }
    // a3: pair merge (fused with the last F levels when F > 0)
    PhaseScope ps(3, 1, stream);
    if (F > 0 && use_clusters)
        return launch_cluster_merge(buf, static_cast<uint32_t *>(vals), la, lb, key, split, Gs,
                                    F, sb, stream);
    if (F > 0 && use_tmem)
        return launch_group2_merge(buf, vals, vb, la, lb, key, split, Gs, F,
                                   reinterpret_cast<uint32_t *>(w + L.group_off), sb, stream);
    if (F > 0)
        return launch_group_merge(buf, vals, vb, la, lb, key, split, Gs, F,
                                  reinterpret_cast<uint32_t *>(w + L.group_off), sb, stream);
    return launch_tile_merge(buf, vals, vb, la, lb, key, split, G, sb, stream);
}

}  // namespace
}  // namespace ipm

using namespace ipm;

extern "C" {

const char *ipm_status_string(ipm_status s) {
    switch (s) {
    case IPM_OK:
        return "IPM_OK";
    case IPM_ERR_INVALID_ARG:
        return "IPM_ERR_INVALID_ARG";
    case IPM_ERR_UNSUPPORTED_DTYPE:
        return "IPM_ERR_UNSUPPORTED_DTYPE";
    case IPM_ERR_ALIGNMENT:
        return "IPM_ERR_ALIGNMENT";
    case IPM_ERR_WORKSPACE:
        return "IPM_ERR_WORKSPACE";
    case IPM_ERR_CUDA:
        return "IPM_ERR_CUDA";
    case IPM_ERR_TIMEOUT:
        return "IPM_ERR_TIMEOUT";
    case IPM_ERR_DEVICE:
        return "IPM_ERR_DEVICE";
    }
    return "IPM_ERR_UNKNOWN";
}

int ipm_version(void) { return 100; }

ipm_status ipm_merge_plan(uint64_t len_a, uint64_t len_b, ipm_dtype key_dtype,
                          int with_values, uint32_t *log2_pairs, uint64_t *tile_cap) {
    uint32_t G = 0;
    const uint32_t vb = payload_bytes(with_values);
    IPM_TRY(check_merge_args(len_a, len_b, key_dtype, vb, 0, &G));
    if (log2_pairs) *log2_pairs = G;
    if (tile_cap) *tile_cap = tile_capacity(key_dtype, vb);
    return IPM_OK;
}

ipm_status ipm_merge_workspace_bytes(uint64_t len_a, uint64_t len_b, ipm_dtype key_dtype,
                                     int with_values, uint32_t log2_pairs, size_t *bytes) {
    if (bytes == nullptr) return IPM_ERR_INVALID_ARG;
    uint32_t G = 0;
    const uint32_t vb = payload_bytes(with_values);
    IPM_TRY(check_merge_args(len_a, len_b, key_dtype, vb, log2_pairs, &G));
    // room for the fused path's split table one level deeper
    *bytes = merge_layout(G + 1, len_a + len_b, key_dtype, vb).total;
    return IPM_OK;
}

ipm_status ipm_merge_inplace(void *d_buf, uint64_t len_a, uint64_t len_b,
                             ipm_dtype key_dtype, uint32_t log2_pairs, void *d_ws,
                             size_t ws_bytes, ipm_stream_t stream) {
    return merge_core(d_buf, nullptr, 0, len_a, len_b, key_dtype, log2_pairs, d_ws, ws_bytes,
                      (cudaStream_t)stream);
}

ipm_status ipm_merge_inplace_kv(void *d_keys, void *d_vals, uint64_t len_a,
                                uint64_t len_b, ipm_dtype key_dtype, ipm_dtype val_dtype,
                                uint32_t log2_pairs, void *d_ws, size_t ws_bytes,
                                ipm_stream_t stream) {
    // payloads are moved, never compared: any 4- or 8-byte type
    if (!valid_key(val_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    const uint32_t vb = uint32_t(dtype_bytes(val_dtype));
    if (d_vals == nullptr && len_a + len_b > 0) return IPM_ERR_INVALID_ARG;
    if (len_a + len_b == 0) return valid_key(key_dtype) ? IPM_OK : IPM_ERR_UNSUPPORTED_DTYPE;
    return merge_core(d_keys, d_vals, vb, len_a, len_b, key_dtype, log2_pairs, d_ws, ws_bytes,
                      (cudaStream_t)stream);
}

ipm_status ipm_merge_splits(const void *d_buf, uint64_t len_a, uint64_t len_b,
                            ipm_dtype key_dtype, uint64_t num_pairs, uint64_t *d_split_a,
                            ipm_stream_t stream) {
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (num_pairs == 0 || d_split_a == nullptr) return IPM_ERR_INVALID_ARG;
    if (len_a > (uint64_t(1) << 40) || len_b > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    const uint64_t n = len_a + len_b;
    if (n > 0 && num_pairs > (~uint64_t(0)) / n) return IPM_ERR_INVALID_ARG;
    if (num_pairs > (uint64_t(1) << 30)) return IPM_ERR_INVALID_ARG;
    if (n > 0 && d_buf == nullptr) return IPM_ERR_INVALID_ARG;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || !aligned(d_split_a, 8))
        return IPM_ERR_ALIGNMENT;
    return launch_splits(d_buf, len_a, len_b, key_dtype, num_pairs, d_split_a, nullptr,
                         (cudaStream_t)stream);
}

ipm_status ipm_merge_rearrange(void *d_buf, void *d_vals, uint64_t len_a, uint64_t len_b,
                               ipm_dtype key_dtype, const uint64_t *d_split_a,
                               uint32_t log2_pairs, void *d_ws, size_t ws_bytes,
                               ipm_stream_t stream) {
    const bool kv = d_vals != nullptr;
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    // the exchange levels do not depend on the tile capacity: any P = 2^G works
    if (log2_pairs == 0 || log2_pairs > kMaxLog2Pairs) return IPM_ERR_INVALID_ARG;
    if (len_a > (uint64_t(1) << 40) || len_b > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    const uint32_t G = log2_pairs;
    if (d_buf == nullptr || d_split_a == nullptr) return IPM_ERR_INVALID_ARG;
    if (d_ws == nullptr) return IPM_ERR_WORKSPACE;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || (kv && !aligned(d_vals, 4)) ||
        !aligned(d_ws, 256))
        return IPM_ERR_ALIGNMENT;
    const uint64_t n = len_a + len_b;
    const uint32_t vb = kv ? 4u : 0u;  // uint32 payloads
    const MergeLayout L = merge_layout(G, n, key_dtype, vb);
    if (ws_bytes < L.total) return IPM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = static_cast<char *>(d_ws);
    StatusBlock *sb = reinterpret_cast<StatusBlock *>(w);
    IPM_CUDA_TRY(cudaMemsetAsync(sb, 0, kStatusBytes, st));
    const XPlanArea pa = xplan_area_at(w + L.plan_off, G, n, key_dtype, vb);
    IPM_TRY(launch_xplan_levels(d_split_a, n, G, G, pa, key_dtype, vb, sb, st));
    for (uint32_t l = 0; l < G; ++l)
        IPM_TRY(launch_exchange_level(d_buf, d_vals, vb, key_dtype, n, l, pa, sb, st));
    return IPM_OK;
}

ipm_status ipm_rearrange_permute_workspace_bytes(uint64_t len_a, uint64_t len_b,
                                                 ipm_dtype key_dtype, int with_values,
                                                 size_t *bytes) {
    if (bytes == nullptr) return IPM_ERR_INVALID_ARG;
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    const uint32_t vb = payload_bytes(with_values);
    if (vb != 0 && vb != 4 && vb != 8) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (len_a > (uint64_t(1) << 40) || len_b > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    *bytes = permute_workspace_bytes(len_a + len_b, uint32_t(dtype_bytes(key_dtype)), vb);
    return IPM_OK;
}

ipm_status ipm_rearrange_permute(void *d_buf, void *d_vals, uint64_t len_a, uint64_t len_b,
                                 ipm_dtype key_dtype, int with_values,
                                 const uint64_t *d_split_a, uint32_t log2_pairs, void *d_ws,
                                 size_t ws_bytes, ipm_stream_t stream) {
    size_t need = 0;
    IPM_TRY(ipm_rearrange_permute_workspace_bytes(len_a, len_b, key_dtype, with_values, &need));
    const uint32_t vb = payload_bytes(with_values);
    const uint32_t kb = uint32_t(dtype_bytes(key_dtype));
    const uint64_t n = len_a + len_b;
    if (log2_pairs > kMaxLog2Pairs || n > (~uint64_t(0) >> log2_pairs))
        return IPM_ERR_INVALID_ARG;
    if (d_buf == nullptr || d_split_a == nullptr || (vb != 0) != (d_vals != nullptr))
        return IPM_ERR_INVALID_ARG;
    if (d_ws == nullptr || ws_bytes < need) return IPM_ERR_WORKSPACE;
    if (!aligned(d_buf, kb) || (vb && !aligned(d_vals, vb)) || !aligned(d_split_a, 8) ||
        !aligned(d_ws, 256))
        return IPM_ERR_ALIGNMENT;
    if (n == 0) return IPM_OK;
    return launch_permute(d_buf, d_vals, kb, vb, len_a, len_b, d_split_a, log2_pairs, d_ws,
                          (cudaStream_t)stream);
}

ipm_status ipm_merge_pairs(void *d_buf, void *d_vals, uint64_t len_a, uint64_t len_b,
                           ipm_dtype key_dtype, const uint64_t *d_split_a,
                           uint32_t log2_pairs, ipm_stream_t stream) {
    const bool kv = d_vals != nullptr;
    uint32_t G = 0;
    const uint32_t vb = kv ? 4u : 0u;  // uint32 payloads
    IPM_TRY(check_merge_args(len_a, len_b, key_dtype, vb, log2_pairs, &G));
    if (G != log2_pairs) return IPM_ERR_INVALID_ARG;
    if (len_a + len_b == 0) return IPM_OK;
    if (d_buf == nullptr || d_split_a == nullptr) return IPM_ERR_INVALID_ARG;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || (kv && !aligned(d_vals, 4)))
        return IPM_ERR_ALIGNMENT;
    return launch_tile_merge(d_buf, d_vals, vb, len_a, len_b, key_dtype, d_split_a, G, nullptr,
                             (cudaStream_t)stream);
}

ipm_status ipm_rotate_workspace_bytes(uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                                      size_t *bytes) {
    if (bytes == nullptr) return IPM_ERR_INVALID_ARG;
    if (elem_bytes != 4 && elem_bytes != 8) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (len_x > (uint64_t(1) << 40) || len_y > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    const ipm_dtype t = elem_bytes == 4 ? IPM_UINT32 : IPM_UINT64;
    *bytes = kStatusBytes + xplan_area_bytes(1, 2 * (len_x + len_y), t, 0u);
    return IPM_OK;
}

ipm_status ipm_rotate(void *d_ptr, uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                      void *d_ws, size_t ws_bytes, ipm_stream_t stream) {
    size_t need = 0;
    IPM_TRY(ipm_rotate_workspace_bytes(len_x, len_y, elem_bytes, &need));
    if (len_x == 0 || len_y == 0) return IPM_OK;
    if (d_ptr == nullptr) return IPM_ERR_INVALID_ARG;
    if (d_ws == nullptr || ws_bytes < need) return IPM_ERR_WORKSPACE;
    if (!aligned(d_ptr, elem_bytes) || !aligned(d_ws, 256)) return IPM_ERR_ALIGNMENT;
    const ipm_dtype t = elem_bytes == 4 ? IPM_UINT32 : IPM_UINT64;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = static_cast<char *>(d_ws);
    StatusBlock *sb = reinterpret_cast<StatusBlock *>(w);
    IPM_CUDA_TRY(cudaMemsetAsync(sb, 0, kStatusBytes, st));
    // one exchange at offset 0: level 0 of a layout sized for 2(len_x + len_y) keys, so
    // the flag area covers every item of this exchange
    const XPlanArea pa = xplan_area_at(w + kStatusBytes, 1, 2 * (len_x + len_y), t, 0u);
    IPM_TRY(launch_xplan_single(len_x, len_y, pa, t, st));
    return launch_exchange_level(d_ptr, nullptr, 0u, t, len_x + len_y, 0, pa, sb, st);
}

ipm_status ipm_division_splits(const void *d_buf, uint64_t len_a, uint64_t len_b,
                               ipm_dtype key_dtype, uint32_t depth, uint32_t split_kind,
                               uint64_t *d_ia, uint64_t *d_jb, ipm_stream_t stream) {
    if (dtype_bytes(key_dtype) == 0) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (depth > 24 || split_kind > IPM_SPLIT_FINDMEDIAN) return IPM_ERR_INVALID_ARG;
    if (d_ia == nullptr || d_jb == nullptr) return IPM_ERR_INVALID_ARG;
    if (len_a + len_b > 0 && d_buf == nullptr) return IPM_ERR_INVALID_ARG;
    if (len_a > (uint64_t(1) << 40) || len_b > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || !aligned(d_ia, 8) || !aligned(d_jb, 8))
        return IPM_ERR_ALIGNMENT;
    return launch_division(d_buf, len_a, len_b, key_dtype, depth, split_kind, d_ia, d_jb,
                           (cudaStream_t)stream);
}

ipm_status ipm_rotate_cs_workspace_bytes(uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                                         size_t *bytes) {
    if (bytes == nullptr) return IPM_ERR_INVALID_ARG;
    if (elem_bytes != 4 && elem_bytes != 8) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (len_x > (uint64_t(1) << 40) || len_y > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    const CsPlan pl = cs_plan(len_x, len_y);
    *bytes = kStatusBytes + align_up(size_t(pl.W) * elem_bytes, 256);
    return IPM_OK;
}

ipm_status ipm_rotate_cs(void *d_ptr, uint64_t len_x, uint64_t len_y, uint32_t elem_bytes,
                         void *d_ws, size_t ws_bytes, ipm_stream_t stream) {
    size_t need = 0;
    IPM_TRY(ipm_rotate_cs_workspace_bytes(len_x, len_y, elem_bytes, &need));
    if (len_x == 0 || len_y == 0) return IPM_OK;
    if (d_ptr == nullptr) return IPM_ERR_INVALID_ARG;
    if (d_ws == nullptr || ws_bytes < need) return IPM_ERR_WORKSPACE;
    if (!aligned(d_ptr, elem_bytes) || !aligned(d_ws, 256)) return IPM_ERR_ALIGNMENT;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = static_cast<char *>(d_ws);
    IPM_CUDA_TRY(cudaMemsetAsync(w, 0, kStatusBytes, st));
    return launch_cs_rotate(d_ptr, elem_bytes, cs_plan(len_x, len_y), w + kStatusBytes, st);
}

ipm_status ipm_read_exchange_bytes(const void *d_ws, ipm_stream_t stream, uint64_t *out) {
    if (d_ws == nullptr || out == nullptr) return IPM_ERR_INVALID_ARG;
    unsigned long long v = 0;
    IPM_CUDA_TRY(cudaMemcpyAsync(&v, static_cast<const char *>(d_ws) +
                                         offsetof(StatusBlock, exchange_bytes),
                                 sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    IPM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *out = uint64_t(v);
    return IPM_OK;
}

ipm_status ipm_read_merge_bytes(const void *d_ws, ipm_stream_t stream, uint64_t *out) {
    if (d_ws == nullptr || out == nullptr) return IPM_ERR_INVALID_ARG;
    unsigned long long v = 0;
    IPM_CUDA_TRY(cudaMemcpyAsync(&v, static_cast<const char *>(d_ws) +
                                         offsetof(StatusBlock, merge_bytes),
                                 sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    IPM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *out = uint64_t(v);
    return IPM_OK;
}

ipm_status ipm_merge_batched_workspace_bytes(uint64_t buf_len, uint32_t nseg,
                                            ipm_dtype key_dtype, int with_values,
                                            const ipm_batched_options *opt, size_t *bytes) {
    uint32_t variant = 0;
    IPM_TRY(batched_variant(opt, &variant));
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (bytes == nullptr || buf_len > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    *bytes = batched_layout(buf_len, nseg, batched_tile(key_dtype, with_values != 0, variant))
                 .total;
    return IPM_OK;
}

ipm_status ipm_merge_batched_max_segment(ipm_dtype key_dtype, int with_values,
                                         const ipm_batched_options *opt, uint64_t *elems) {
    uint32_t variant = 0;
    IPM_TRY(batched_variant(opt, &variant));
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (elems == nullptr) return IPM_ERR_INVALID_ARG;
    *elems = batched_max_segment(key_dtype, with_values != 0, variant);
    return IPM_OK;
}

ipm_status ipm_merge_batched(void *d_buf, void *d_vals, uint64_t buf_len,
                             const ipm_segment *d_segs, uint32_t nseg, ipm_dtype key_dtype,
                             ipm_dtype val_dtype, const ipm_batched_options *opt,
                             void *d_ws, size_t ws_bytes, ipm_stream_t stream) {
    uint32_t variant = 0, one_launch = 0;
    IPM_TRY(batched_variant(opt, &variant, &one_launch));
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    const bool kv = d_vals != nullptr;
    if (kv && val_dtype != IPM_UINT32) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (buf_len > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    if (nseg > 0 && d_segs == nullptr) return IPM_ERR_INVALID_ARG;
    if (buf_len > 0 && d_buf == nullptr) return IPM_ERR_INVALID_ARG;
    if (d_ws == nullptr) return IPM_ERR_WORKSPACE;
    const BatchedLayout L =
        batched_layout(buf_len, nseg, batched_tile(key_dtype, kv, variant));
    if (ws_bytes < L.total) return IPM_ERR_WORKSPACE;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || (kv && !aligned(d_vals, 4)) ||
        !aligned(d_segs, 8) || !aligned(d_ws, 256))
        return IPM_ERR_ALIGNMENT;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t by_size = (opt == nullptr || opt->order == 0) ? 1u : 0u;
    const uint32_t per_sm = opt ? opt->ctas_per_sm : 0u;
    PhaseScope ps(4, nseg == 0 ? 0u : one_launch ? 1u : 3u, st);
    return launch_batched(d_buf, static_cast<uint32_t *>(d_vals), buf_len, key_dtype, d_segs,
                          nseg, d_ws, L, by_size, variant, per_sm, one_launch, st);
}

ipm_status ipm_split_model_train_workspace_bytes(uint32_t nsamples, size_t *bytes) {
    if (bytes == nullptr || nsamples == 0 || nsamples > (1u << 20)) return IPM_ERR_INVALID_ARG;
    *bytes = split_model_train_ws_bytes(nsamples);
    return IPM_OK;
}

ipm_status ipm_split_model_train(const void *d_buf, uint64_t len_a, uint64_t len_b,
                                 ipm_dtype key_dtype, const uint64_t *d_diags,
                                 uint32_t nsamples, const ipm_split_train_options *opt,
                                 ipm_split_model *d_model, void *d_ws, size_t ws_bytes,
                                 ipm_stream_t stream) {
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (opt == nullptr || d_model == nullptr || d_diags == nullptr || d_buf == nullptr)
        return IPM_ERR_INVALID_ARG;
    if (len_a == 0 || len_a > (uint64_t(1) << 40) || len_b > (uint64_t(1) << 40))
        return IPM_ERR_INVALID_ARG;
    if (nsamples == 0 || nsamples > (1u << 20) || opt->steps > 1000000u) return IPM_ERR_INVALID_ARG;
    if (!(opt->lr > 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) ||
        !(opt->beta2 >= 0.f && opt->beta2 < 1.f) || !(opt->eps > 0.f))
        return IPM_ERR_INVALID_ARG;
    if (d_ws == nullptr || ws_bytes < split_model_train_ws_bytes(nsamples))
        return IPM_ERR_WORKSPACE;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || !aligned(d_diags, 8) ||
        !aligned(d_model, 4) || !aligned(d_ws, 256))
        return IPM_ERR_ALIGNMENT;
    cudaStream_t st = (cudaStream_t)stream;
    PhaseScope ps(5, 3, st);
    return launch_split_model_train(d_buf, len_a, len_b, key_dtype, d_diags, nsamples, *opt,
                                    d_model, d_ws, st);
}

ipm_status ipm_split_model_forward(const ipm_split_model *d_model, const float *d_x,
                                   uint32_t n, float *d_y, ipm_stream_t stream) {
    if (n > 0 && (d_model == nullptr || d_x == nullptr || d_y == nullptr))
        return IPM_ERR_INVALID_ARG;
    if (!aligned(d_model, 4) || !aligned(d_x, 4) || !aligned(d_y, 4)) return IPM_ERR_ALIGNMENT;
    return launch_split_model_forward(d_model, d_x, n, d_y, (cudaStream_t)stream);
}

ipm_status ipm_split_model_loss_grad(const ipm_split_model *d_model, const float *d_x,
                                     const float *d_t, uint32_t n, float *d_grad,
                                     ipm_stream_t stream) {
    if (d_model == nullptr || d_x == nullptr || d_t == nullptr || d_grad == nullptr ||
        n == 0 || n > (1u << 20))
        return IPM_ERR_INVALID_ARG;
    if (!aligned(d_model, 4) || !aligned(d_x, 4) || !aligned(d_t, 4) || !aligned(d_grad, 4))
        return IPM_ERR_ALIGNMENT;
    return launch_split_model_loss_grad(d_model, d_x, d_t, n, d_grad, (cudaStream_t)stream);
}

ipm_status ipm_merge_splits_learned(const void *d_buf, uint64_t len_a, uint64_t len_b,
                                    ipm_dtype key_dtype, uint64_t num_pairs,
                                    const ipm_split_model *d_model, uint64_t *d_split_a,
                                    ipm_split_stats *d_stats, ipm_stream_t stream) {
    if (!valid_key(key_dtype)) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (num_pairs == 0 || d_split_a == nullptr) return IPM_ERR_INVALID_ARG;
    if (len_a > (uint64_t(1) << 40) || len_b > (uint64_t(1) << 40)) return IPM_ERR_INVALID_ARG;
    const uint64_t n = len_a + len_b;
    if (n > 0 && num_pairs > (~uint64_t(0)) / n) return IPM_ERR_INVALID_ARG;
    if (num_pairs > (uint64_t(1) << 30)) return IPM_ERR_INVALID_ARG;
    if (n > 0 && d_buf == nullptr) return IPM_ERR_INVALID_ARG;
    if (!aligned(d_buf, size_t(dtype_bytes(key_dtype))) || !aligned(d_split_a, 8) ||
        !aligned(d_model, 4) || !aligned(d_stats, 8))
        return IPM_ERR_ALIGNMENT;
    cudaStream_t st = (cudaStream_t)stream;
    PhaseScope ps(6, learned_split_launches(num_pairs), st);
    return launch_learned_splits(d_buf, len_a, len_b, key_dtype, num_pairs, d_model, d_split_a,
                                 d_stats, nullptr, st);
}

ipm_status ipm_merge_inplace_learned(void *d_buf, uint64_t len_a, uint64_t len_b,
                                     ipm_dtype key_dtype, uint32_t log2_pairs,
                                     const ipm_split_model *d_model, void *d_ws,
                                     size_t ws_bytes, ipm_stream_t stream) {
    if (d_model == nullptr) return IPM_ERR_INVALID_ARG;
    if (!aligned(d_model, 4)) return IPM_ERR_ALIGNMENT;
    return merge_core(d_buf, nullptr, 0, len_a, len_b, key_dtype, log2_pairs, d_ws, ws_bytes,
                      (cudaStream_t)stream, d_model);
}

ipm_status ipm_merge_fused_plan(uint64_t len_a, uint64_t len_b, ipm_dtype key_dtype,
                                int with_values, uint32_t *engine, uint32_t *levels) {
    uint32_t G = 0;
    const uint32_t vb = payload_bytes(with_values);
    IPM_TRY(check_merge_args(len_a, len_b, key_dtype, vb, 0, &G));
    const FusedChoice fc = fused_choice(key_dtype, vb, G);
    if (engine) *engine = fc.levels > 0 ? fc.engine : 0xFFFFFFFFu;
    if (levels) *levels = fc.levels;
    return IPM_OK;
}

ipm_status ipm_set_fused_engine(uint32_t engine) {
    if (engine > 2) return IPM_ERR_INVALID_ARG;
    g_fused_engine = engine;
    return IPM_OK;
}

ipm_status ipm_set_fused_levels(uint32_t levels) {
    if (levels > 10) return IPM_ERR_INVALID_ARG;
    g_fused_levels = levels;
    return IPM_OK;
}

ipm_status ipm_get_fused_levels(uint32_t *levels) {
    if (levels == nullptr) return IPM_ERR_INVALID_ARG;
    *levels = g_fused_levels;
    return IPM_OK;
}

ipm_status ipm_set_wait_limit_ns(uint64_t ns) {
    if (ns > kWaitLimitNs) return IPM_ERR_INVALID_ARG;
    g_wait_limit_ns.store(ns, std::memory_order_relaxed);
    return IPM_OK;
}

ipm_status ipm_get_wait_limit_ns(uint64_t *ns) {
    if (ns == nullptr) return IPM_ERR_INVALID_ARG;
    const unsigned long long v = g_wait_limit_ns.load(std::memory_order_relaxed);
    *ns = v ? v : kWaitLimitNs;
    return IPM_OK;
}

ipm_status ipm_set_exchange_engine(uint32_t engine) {
    if (engine > 1) return IPM_ERR_INVALID_ARG;
    g_exchange_engine = engine;
    return IPM_OK;
}

ipm_status ipm_timing_enable(int enable) {
    g_timing.enabled = enable != 0;
    return IPM_OK;
}

ipm_status ipm_timing_read(ipm_timing *out) {
    if (out == nullptr) return IPM_ERR_INVALID_ARG;
    ipm_status st = IPM_OK;
    for (const TimingRec &r : g_timing.recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            (void)cudaGetLastError();
            st = IPM_ERR_CUDA;
        } else {
            out->ms[r.phase] += double(ms);
            out->launches[r.phase] += r.launches;
        }
        g_timing.pool.push_back(r.a);
        g_timing.pool.push_back(r.b);
    }
    g_timing.recs.clear();
    return st;
}

ipm_status ipm_read_device_status(const void *d_ws, ipm_stream_t stream, ipm_status *out) {
    if (d_ws == nullptr || out == nullptr) return IPM_ERR_INVALID_ARG;
    unsigned int word = 0;
    IPM_CUDA_TRY(cudaMemcpyAsync(&word, d_ws, sizeof(word), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
    IPM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *out = static_cast<ipm_status>(word);
    return IPM_OK;
}

}  // extern "C"
