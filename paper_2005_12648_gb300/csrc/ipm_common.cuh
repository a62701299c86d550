// Shared device/host helpers of the ipmerge CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "ipmerge.h"

namespace ipm {

// ---------------------------------------------------------------------------------
// Key types.  Keys are compared with their own "<=" and otherwise only moved.
// ---------------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ bool key_le(K x, K y) { return x <= y; }

// ---------------------------------------------------------------------------------
// Workspace status block (first 256 bytes of every workspace).
//   status          device status (ipm_status), first error wins
//   done            early-exit flag: nonzero when the runs are already in order
//   exchange_bytes  algorithmic bytes of the exchange levels of the current call
//   merge_bytes     algorithmic bytes of the pair merges (batched calls only)
//   wait_limit_ns   limit of this call's waits on other CTAs (0: kWaitLimitNs)
//   counters        per-call ticket counters of the persistent kernels
// All of it is reset at the start of every call.
// ---------------------------------------------------------------------------------
constexpr int kNumCounters = 56;

struct StatusBlock {
    unsigned int status;
    unsigned int done;
    unsigned long long exchange_bytes;
    unsigned long long merge_bytes;
    unsigned long long wait_limit_ns;
    unsigned int counters[kNumCounters];
};

constexpr uint32_t kTicketCounter0 = 0;  // counters[l]: exchange tickets of level l
static_assert(sizeof(StatusBlock) == 256, "status block is 256 bytes");

constexpr size_t kStatusBytes = 256;

__device__ __forceinline__ void set_status(StatusBlock *sb, unsigned int code) {
    atomicCAS(&sb->status, 0u, code);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Upper bound for every device-side wait (mbarrier, flags): 2 s of wall time.  Waits
// on another CTA's progress (flags, joins, group barriers) use the call's own limit
// (wait_limit below), which defaults to this; waits for this CTA's own bulk copies
// always use this one, so a CTA never leaves with a copy into its shared memory in
// flight.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// The limit of this call's waits on other CTAs.
__device__ __forceinline__ unsigned long long wait_limit(const StatusBlock *sb) {
    if (sb == nullptr) return kWaitLimitNs;
    const unsigned long long v = *((volatile const unsigned long long *)&sb->wait_limit_ns);
    return v ? v : kWaitLimitNs;
}

// True when the call this kernel belongs to needs no more work: the runs were already
// in order (early exit) or an earlier kernel of the call recorded an error.
__device__ __forceinline__ bool call_finished(const StatusBlock *sb) {
    if (sb == nullptr) return false;
    const volatile StatusBlock *v = sb;
    return v->done != 0u || v->status != 0u;
}

// Clock of a wait on another CTA: call expired() after every poll that found the
// condition unmet.  The clock starts at the first failed poll and is read again every
// 8th one; expired() turns true once more than `lim` ns have passed.
struct DepTimer {
    unsigned long long t0, lim;
    uint32_t it;
    __device__ __forceinline__ explicit DepTimer(unsigned long long l) : t0(0), lim(l), it(0) {}
    __device__ __forceinline__ bool expired() {
        ++it;
        if (it == 1) {
            t0 = globaltimer_ns();
            return false;
        }
        return (it & 7u) == 0 && globaltimer_ns() - t0 > lim;
    }
};

// ---------------------------------------------------------------------------------
// Small host helpers.
// ---------------------------------------------------------------------------------
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int dtype_bytes(ipm_dtype t) {
    switch (t) {
    case IPM_INT32:
    case IPM_UINT32:
    case IPM_FLOAT32:
        return 4;
    case IPM_UINT64:
    case IPM_INT64:
        return 8;
    }
    return 0;
}

int num_sms();                 // cached multiprocessor count of the current device
ipm_status last_launch_status();  // IPM_ERR_CUDA if the last launch failed

}  // namespace ipm

#define IPM_TRY(expr)                          \
    do {                                       \
        ipm_status _s = (expr);                \
        if (_s != IPM_OK) return _s;           \
    } while (0)

#define IPM_CUDA_TRY(expr)                     \
    do {                                       \
        if ((expr) != cudaSuccess) {           \
            (void)cudaGetLastError();          \
            return IPM_ERR_CUDA;               \
        }                                      \
    } while (0)
