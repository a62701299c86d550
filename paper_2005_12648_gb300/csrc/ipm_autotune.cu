// Autotuner of the batched segmented merge (ipm_merge_batched_tune).  The paper has no
// counterpart: it tunes the launch of the batched form, whose every option set gives
// the same result.
//
// The tuner times each candidate option set (merge tile, which also fixes the pair
// count P of every segment longer than one tile; resident CTAs per SM; work-queue
// order) on a scratch copy of the caller's input, restored before every run, and
// returns the fastest.  The choice is cached in a small text file under a signature of
// the workload (key type, payload width and coarse size statistics of the segment
// table), so a later call with a similar table reads it instead of timing again.
//
// Cache file format: one line per signature, "ipmtune2 <signature hex> <tile>
// <ctas_per_sm> <order> <form> <ms>"; unknown or malformed lines are ignored, and a new
// choice is appended.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "ipm_internal.h"

namespace ipm {
namespace {

std::mutex g_tune_file_mutex;

uint32_t floor_log2(uint64_t x) { return x ? 63u - uint32_t(__builtin_clzll(x)) : 0u; }

// FNV-1a over 64-bit words.
uint64_t fnv1a(const uint64_t *w, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i)
        for (int b = 0; b < 8; ++b) {
            h ^= (w[i] >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    return h;
}

// Signature of a segment table: key type, payload width, and the floor(log2) of the
// segment count, of the total length, of the longest and of the median segment.
uint64_t tune_signature(const ipm_segment *segs, uint32_t nseg, ipm_dtype key, uint32_t vb) {
    std::vector<uint64_t> len(nseg);
    uint64_t total = 0, mx = 0;
    for (uint32_t i = 0; i < nseg; ++i) {
        len[i] = segs[i].len_a + segs[i].len_b;
        total += len[i];
        mx = std::max(mx, len[i]);
    }
    uint64_t med = 0;
    if (nseg) {
        std::nth_element(len.begin(), len.begin() + nseg / 2, len.end());
        med = len[nseg / 2];
    }
    const uint64_t w[7] = {0x69706d74756e6531ull, uint64_t(key), uint64_t(vb),
                           floor_log2(nseg),      floor_log2(total), floor_log2(mx),
                           floor_log2(med)};
    return fnv1a(w, 7);
}

bool cache_lookup(const char *path, uint64_t sig, ipm_batched_options *opt, float *ms) {
    std::lock_guard<std::mutex> lock(g_tune_file_mutex);
    FILE *f = std::fopen(path, "r");
    if (f == nullptr) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long s = 0;
        unsigned t = 0, c = 0, o = 0, fm = 0;
        float m = 0.f;
        if (std::sscanf(line, "ipmtune2 %llx %u %u %u %u %f", &s, &t, &c, &o, &fm, &m) != 6)
            continue;
        if (s != sig || t > 3 || c > 64 || o > 1 || fm > 2) continue;
        opt->tile = t;
        opt->ctas_per_sm = c;
        opt->order = o;
        opt->form = fm;
        *ms = m;
        found = true;  // the last matching line wins
    }
    std::fclose(f);
    return found;
}

void cache_append(const char *path, uint64_t sig, const ipm_batched_options &opt, float ms) {
    std::lock_guard<std::mutex> lock(g_tune_file_mutex);
    FILE *f = std::fopen(path, "a");
    if (f == nullptr) return;  // an unwritable cache only costs a later re-tune
    std::fprintf(f, "ipmtune2 %016llx %u %u %u %u %.6f\n", (unsigned long long)sig, opt.tile,
                 opt.ctas_per_sm, opt.order, opt.form, double(ms));
    std::fclose(f);
}

const char *cache_path_of(const char *arg) {
    if (arg != nullptr) return arg[0] ? arg : nullptr;
    const char *env = std::getenv("IPM_TUNE_CACHE");
    return (env != nullptr && env[0]) ? env : nullptr;
}

// The candidate option sets: both launch forms, every tile, each at its full occupancy
// and at fewer resident CTAs per SM, each with both queue orders.
std::vector<ipm_batched_options> candidates() {
    std::vector<ipm_batched_options> v;
    const uint32_t per_sm[3][2] = {{0, 0}, {0, 1}, {0, 2}};  // wide, narrow, quarter
    for (uint32_t fm = 1; fm <= 2; ++fm)
        for (uint32_t t = 1; t <= 3; ++t)
            for (uint32_t c = 0; c < 2; ++c) {
                if (c == 1 && per_sm[t - 1][1] == 0) continue;
                for (uint32_t o = 0; o <= 1; ++o) {
                    ipm_batched_options op{};
                    op.tile = t;
                    op.ctas_per_sm = per_sm[t - 1][c];
                    op.order = o;
                    op.form = fm;
                    v.push_back(op);
                }
            }
    return v;
}

// Median time (ms) of `reps` runs of one option set (opt NULL: the defaults) on the
// scratch copy, restored before every run; a negative value when a run failed.
float time_candidate(const void *buf, const void *vals, uint64_t buf_len, size_t kbytes,
                     const ipm_segment *segs, uint32_t nseg, ipm_dtype key, ipm_dtype val,
                     void *sbuf, void *svals, void *ws, size_t ws_bytes, uint32_t reps,
                     const ipm_batched_options *opt, cudaStream_t st, ipm_status *err) {
    const size_t bytes = size_t(buf_len) * kbytes;
    const size_t vbytes = vals ? size_t(buf_len) * 4u : 0u;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        (void)cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        *err = IPM_ERR_CUDA;
        return -1.f;
    }
    std::vector<float> t;
    for (uint32_t r = 0; r <= reps; ++r) {  // run 0 warms up
        if (cudaMemcpyAsync(sbuf, buf, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            (vbytes && cudaMemcpyAsync(svals, vals, vbytes, cudaMemcpyDeviceToDevice, st) !=
                           cudaSuccess) ||
            cudaEventRecord(e0, st) != cudaSuccess) {
            (void)cudaGetLastError();
            *err = IPM_ERR_CUDA;
            break;
        }
        const ipm_status s = ipm_merge_batched(sbuf, vals ? svals : nullptr, buf_len, segs, nseg,
                                               key, val, opt, ws, ws_bytes, (ipm_stream_t)st);
        if (s != IPM_OK) {
            *err = s;
            break;
        }
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            (void)cudaGetLastError();
            *err = IPM_ERR_CUDA;
            break;
        }
        ipm_status dev = IPM_OK;
        if (ipm_read_device_status(ws, (ipm_stream_t)st, &dev) != IPM_OK || dev != IPM_OK) {
            *err = dev != IPM_OK ? dev : IPM_ERR_CUDA;
            break;
        }
        if (r > 0) t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (t.size() != reps) return -1.f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace
}  // namespace ipm

using namespace ipm;

extern "C" {

ipm_status ipm_merge_batched_tune_workspace_bytes(uint64_t buf_len, uint32_t nseg,
                                                  ipm_dtype key_dtype, int with_values,
                                                  size_t *bytes) {
    if (bytes == nullptr) return IPM_ERR_INVALID_ARG;
    size_t most = 0;
    for (uint32_t t = 1; t <= 3; ++t) {
        ipm_batched_options op{};
        op.tile = t;
        size_t b = 0;
        IPM_TRY(ipm_merge_batched_workspace_bytes(buf_len, nseg, key_dtype, with_values, &op, &b));
        most = std::max(most, b);
    }
    *bytes = most;
    return IPM_OK;
}

ipm_status ipm_batched_tune_signature(const ipm_segment *h_segs, uint32_t nseg,
                                      ipm_dtype key_dtype, int with_values, uint64_t *out) {
    if (out == nullptr || (nseg > 0 && h_segs == nullptr)) return IPM_ERR_INVALID_ARG;
    if (dtype_bytes(key_dtype) == 0) return IPM_ERR_UNSUPPORTED_DTYPE;
    *out = tune_signature(h_segs, nseg, key_dtype, with_values ? 4u : 0u);
    return IPM_OK;
}

ipm_status ipm_merge_batched_tune(const void *d_buf, const void *d_vals, uint64_t buf_len,
                                  const ipm_segment *d_segs, const ipm_segment *h_segs,
                                  uint32_t nseg, ipm_dtype key_dtype, ipm_dtype val_dtype,
                                  void *d_scratch, void *d_scratch_vals, void *d_ws,
                                  size_t ws_bytes, uint32_t reps, const char *cache_path,
                                  ipm_batched_tune_result *out, ipm_stream_t stream) {
    if (out == nullptr || reps == 0 || reps > 100) return IPM_ERR_INVALID_ARG;
    const int kb = dtype_bytes(key_dtype);
    if (kb == 0) return IPM_ERR_UNSUPPORTED_DTYPE;
    const bool kv = d_vals != nullptr;
    if (kv && val_dtype != IPM_UINT32) return IPM_ERR_UNSUPPORTED_DTYPE;
    if (kv != (d_scratch_vals != nullptr)) return IPM_ERR_INVALID_ARG;
    if (nseg > 0 && d_segs == nullptr) return IPM_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    cudaStream_t st = (cudaStream_t)stream;

    // the segment table on the host (for the signature)
    std::vector<ipm_segment> hs;
    const ipm_segment *segs_host = h_segs;
    if (segs_host == nullptr && nseg > 0) {
        hs.resize(nseg);
        IPM_CUDA_TRY(cudaMemcpyAsync(hs.data(), d_segs, sizeof(ipm_segment) * nseg,
                                     cudaMemcpyDeviceToHost, st));
        IPM_CUDA_TRY(cudaStreamSynchronize(st));
        segs_host = hs.data();
    }
    out->signature = tune_signature(segs_host, nseg, key_dtype, kv ? 4u : 0u);
    const char *path = cache_path_of(cache_path);
    if (path != nullptr && cache_lookup(path, out->signature, &out->best, &out->best_ms)) {
        out->from_cache = 1;
        return IPM_OK;
    }

    if (buf_len > 0 && (d_buf == nullptr || d_scratch == nullptr)) return IPM_ERR_INVALID_ARG;
    size_t need = 0;
    IPM_TRY(ipm_merge_batched_tune_workspace_bytes(buf_len, nseg, key_dtype, kv ? 1 : 0, &need));
    if (d_ws == nullptr || ws_bytes < need) return IPM_ERR_WORKSPACE;

    ipm_status err = IPM_OK;
    out->default_ms = time_candidate(d_buf, d_vals, buf_len, size_t(kb), d_segs, nseg, key_dtype,
                                     val_dtype, d_scratch, d_scratch_vals, d_ws, ws_bytes, reps,
                                     nullptr, st, &err);
    // the defaults may refuse a segment longer than their tile allows (IPM_ERR_INVALID_ARG
    // on the device): default_ms stays negative and the search goes on
    if (out->default_ms < 0.f && err != IPM_ERR_INVALID_ARG)
        return err != IPM_OK ? err : IPM_ERR_CUDA;
    float best = -1.f;
    for (const ipm_batched_options &op : candidates()) {
        ipm_status e = IPM_OK;
        const float ms = time_candidate(d_buf, d_vals, buf_len, size_t(kb), d_segs, nseg,
                                        key_dtype, val_dtype, d_scratch, d_scratch_vals, d_ws,
                                        ws_bytes, reps, &op, st, &e);
        if (ms < 0.f) {
            // a segment beyond this tile's limit is refused by the device (every option set
            // gives the same result where it runs): the candidate is skipped
            if (e == IPM_ERR_INVALID_ARG) continue;
            return e != IPM_OK ? e : IPM_ERR_CUDA;
        }
        if (out->candidates < IPM_TUNE_MAX_CANDIDATES) {
            out->table[out->candidates].options = op;
            out->table[out->candidates].ms = ms;
        }
        ++out->candidates;
        if (best < 0.f || ms < best) {
            best = ms;
            out->best = op;
        }
    }
    if (best < 0.f) return IPM_ERR_INVALID_ARG;  // no option set handles this table
    out->best_ms = best;
    if (path != nullptr) cache_append(path, out->signature, out->best, best);
    return IPM_OK;
}

}  // extern "C"
