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
//   counters        per-call ticket counters of the persistent kernels
// All of it is reset at the start of every call.
// ---------------------------------------------------------------------------------
constexpr int kNumCounters = 58;

struct StatusBlock {
    unsigned int status;
    unsigned int done;
    unsigned long long exchange_bytes;
    unsigned long long merge_bytes;
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

// Upper bound for every device-side wait (mbarrier, flags): 2 s of wall time.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

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
